// agcm_filter.cuh — the low-latitude filters the leap format keeps (Table
// "Conventional Filtering scheme"), per zonal row by the row's latitude band:
//   band 1 (|lat| < 38 deg): removal of the two-grid-interval wave,
//          F_x -= (-1)^x a,  a = (1/I) sum_x' (-1)^x' F_x'   (I even);
//   band 2 (38..70 deg): the 3-point operator F_x + r (F_{x-1} - 2 F_x + F_{x+1});
//   poleward of 70 deg nothing (the leap format replaces the filter there).
// The host lists only the rows the filter changes.  One launch covers all four
// fields: a warp takes one row at a time, stages it in its slice of shared
// memory with VW-wide loads, and writes it back in place.  The FP32 two-grid
// sum is an error-free (TwoSum, Knuth) accumulation per lane, combined across
// the warp in FP64, so no FP64 operation runs per element.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

template <class T>
struct FiltArgs {
  T *U, *V, *Ph, *pi;
  const int *filtU, *filtV;  // entries 4 j + band
  int nU, nV, I, J, K;
  int row_bytes;      // shared-memory slice per warp (16-byte multiple)
  long long items;    // (2K + 1) nU + K nV rows
  T r;
};

template <class T, int VW> struct VecT { using type = T; };
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 2> { using type = double2; };

template <class T> __device__ __forceinline__ T comp(const T& v, int) { return v; }
__device__ __forceinline__ float comp(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ double comp(const double2& v, int e) { return e == 0 ? v.x : v.y; }
template <class T> __device__ __forceinline__ void setc(T& v, int, T x) { v = x; }
__device__ __forceinline__ void setc(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void setc(double2& v, int e, double x) {
  if (e == 0) v.x = x; else v.y = x;
}

// s + c += x without rounding loss in s (TwoSum: c collects the exact error)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

template <class T, int VW>
__global__ void __launch_bounds__(256) k_filter(FiltArgs<T> a) {
  using V = typename VecT<T, VW>::type;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  V* sv = reinterpret_cast<V*>(fsm + (size_t)wib * a.row_bytes);
  const int I = a.I, nv = I / VW;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long it = (long long)blockIdx.x * (blockDim.x >> 5) + wib; it < a.items; it += nwarps) {
    // item -> (field, level, row); U and Phi levels first, then pi, then V
    long long q = it;
    T* base;
    int e;
    size_t row;
    const long long nUK = (long long)a.K * a.nU;
    if (q < 2 * nUK) {
      base = q < nUK ? a.U : a.Ph;
      q = q < nUK ? q : q - nUK;
      e = a.filtU[q % a.nU];
      row = (size_t)(q / a.nU) * a.J + (e >> 2);
    } else if ((q -= 2 * nUK) < a.nU) {
      base = a.pi;
      e = a.filtU[q];
      row = (size_t)(e >> 2);
    } else {
      q -= a.nU;
      base = a.V;
      e = a.filtV[q % a.nV];
      row = (size_t)(q / a.nV) * (a.J - 1) + (e >> 2);
    }
    V* f = reinterpret_cast<V*>(base + row * I);
#pragma unroll 4
    for (int v = lane; v < nv; v += 32) sv[v] = f[v];
    __syncwarp();
    if ((e & 3) == 1) {
      double tot;
      if constexpr (sizeof(T) == 4) {
        float s = 0.f, c = 0.f;
        for (int v = lane; v < nv; v += 32) {
          const V x = sv[v];
#pragma unroll
          for (int k = 0; k < VW; ++k) {
            const float y = comp(x, k);
            two_sum_acc(s, c, ((v * VW + k) & 1) ? -y : y);
          }
        }
        tot = (double)s + (double)c;
      } else {
        tot = 0.0;
        for (int v = lane; v < nv; v += 32) {
          const V x = sv[v];
#pragma unroll
          for (int k = 0; k < VW; ++k) tot += ((v * VW + k) & 1) ? -comp(x, k) : comp(x, k);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      const T am = (T)(tot / I);
      for (int v = lane; v < nv; v += 32) {
        V x = sv[v];
#pragma unroll
        for (int k = 0; k < VW; ++k) setc(x, k, ((v * VW + k) & 1) ? comp(x, k) + am : comp(x, k) - am);
        f[v] = x;
      }
    } else {
      const T r = a.r;
      for (int v = lane; v < nv; v += 32) {
        const V x = sv[v];
        const T l0 = comp(sv[v == 0 ? nv - 1 : v - 1], VW - 1);
        const T rn = comp(sv[v == nv - 1 ? 0 : v + 1], 0);
        V y = x;
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          const T l = k == 0 ? l0 : comp(x, k - 1);
          const T c = comp(x, k);
          const T rr = k == VW - 1 ? rn : comp(x, k + 1);
          setc(y, k, c + r * (l - T(2) * c + rr));
        }
        f[v] = y;
      }
    }
    __syncwarp();  // the slice is reloaded for the next row
  }
}

}  // namespace agcm
