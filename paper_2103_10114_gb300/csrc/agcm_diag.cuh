// agcm_diag.cuh — FP64 global sums (a11): mass, kinetic, available potential
// and available surface potential energy, max |U|, max |V|, non-finite count.
// Deterministic: fixed grid, fixed-order tree reductions, one final block.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

constexpr int kDiagPartials = 304;  // two blocks per SM on a 152-SM part
constexpr int kDiagThreads = 256;

__device__ __forceinline__ void diag_reduce_block(double v[7], double* part) {
  __shared__ double red[7][kDiagThreads];
  for (int q = 0; q < 7; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 7; ++q) {
        const double a = red[q][threadIdx.x], b = red[q][threadIdx.x + w];
        red[q][threadIdx.x] = (q == 4 || q == 5) ? fmax(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 7; ++q) part[q] = red[q][0];
}

template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_diag(Geom<double> g, const T* __restrict__ U,
                                                       const T* __restrict__ V, const T* __restrict__ Phi,
                                                       const T* __restrict__ pi, double* __restrict__ part) {
  const int I = g.I, J = g.J, K = g.K;
  const size_t n3 = (size_t)K * J * I, nv = (size_t)K * (J - 1) * I, n2 = (size_t)J * I;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};  // mass, ek, ep, eps, max|U|, max|V|, nonfinite
  for (size_t n = t0; n < n3; n += stride) {
    const int j = (int)((n / I) % J), k = (int)(n / ((size_t)I * J));
    const double u = (double)U[n], f = (double)Phi[n];
    const double w = 0.5 * g.dsd[k] * g.Ad[j];
    v[1] += w * u * u;
    v[2] += w * f * f;
    v[4] = fmax(v[4], fabs(u));
    v[6] += (isfinite(u) ? 0.0 : 1.0) + (isfinite(f) ? 0.0 : 1.0);
  }
  for (size_t n = t0; n < nv; n += stride) {
    const int j = (int)((n / I) % (J - 1)), k = (int)(n / ((size_t)I * (J - 1)));
    const double x = (double)V[n];
    v[1] += 0.5 * g.dsd[k] * g.Avd[j] * x * x;
    v[5] = fmax(v[5], fabs(x));
    v[6] += isfinite(x) ? 0.0 : 1.0;
  }
  for (size_t n = t0; n < n2; n += stride) {
    const int j = (int)(n / I);
    const double p = (double)pi[n];
    v[0] += g.Ad[j] * (g.pit[n] + p);
    v[3] += 0.5 * g.Ad[j] * g.rt0pit[n] * p * p;
    v[6] += isfinite(p) ? 0.0 : 1.0;
  }
  diag_reduce_block(v, part + 8 * blockIdx.x);
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double* __restrict__ part, int nb,
                                                             double* __restrict__ out) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    for (int q = 0; q < 7; ++q) v[q] = (q == 4 || q == 5) ? fmax(v[q], part[8 * b + q]) : v[q] + part[8 * b + q];
  diag_reduce_block(v, out);
}

}  // namespace agcm
