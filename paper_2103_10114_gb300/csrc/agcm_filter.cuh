// agcm_filter.cuh — the low-latitude filters the leap format keeps (Table
// "Conventional Filtering scheme"): per zonal row, by the row's latitude band,
//   band 1 (|lat| < 38 deg): removal of the two-grid-interval wave,
//          F_x -= (-1)^x (1/I) sum_x' (-1)^x' F_x'   (I even; FP64 sum);
//   band 2 (38..70 deg): 3-point operator F_x += r (F_{x-1} - 2 F_x + F_{x+1});
//   band 0 (poleward of 70 deg): nothing (the leap format replaces the filter).
// One block per row; the row is staged in shared memory, so the 3-point
// operator reads the unfiltered row and writes in place.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

template <class T>
__global__ void __launch_bounds__(256) k_filter(const int* __restrict__ band_of_row, T* F, int I,
                                                int rows_per_level, int nrows, T r) {
  extern __shared__ __align__(16) unsigned char fsm[];
  T* row = reinterpret_cast<T*>(fsm);
  __shared__ double red[256];
  const int q = blockIdx.x;
  if (q >= nrows) return;
  const int band = band_of_row[q % rows_per_level];
  if (band == 0 || (band == 1 && (I & 1))) return;  // uniform per block
  T* f = F + (size_t)q * I;
  for (int x = threadIdx.x; x < I; x += blockDim.x) row[x] = f[x];
  __syncthreads();
  if (band == 1) {
    double acc = 0.0;
    for (int x = threadIdx.x; x < I; x += blockDim.x) acc += (x & 1) ? -(double)row[x] : (double)row[x];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    const double a = red[0] / I;
    for (int x = threadIdx.x; x < I; x += blockDim.x) f[x] = (T)((double)row[x] - ((x & 1) ? -a : a));
  } else {
    for (int x = threadIdx.x; x < I; x += blockDim.x) {
      const T l = row[x == 0 ? I - 1 : x - 1], c = row[x], rr = row[x == I - 1 ? 0 : x + 1];
      f[x] = c + r * (l - T(2) * c + rr);
    }
  }
}

}  // namespace agcm
