// agcm_common.cuh — device-side geometry and indexing shared by the kernels.
//
// Grid conventions (pole-free C grid): scalar/U rows j = 0..J-1 at colatitude
// (j+1/2) dth, V rows j = 0..J-2 at (j+1) dth, U index i at longitude
// (i+1/2) dlam.  Storage [k][j][i], longitude contiguous.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace agcm {

// Stride classes of the row-segment stage kernel: rows whose strides Mu_j,
// Mv_j, Mu_{j+1} all equal kRowClsM[c] (compile-time partner offsets), and
// a last class of rows with any strides.
constexpr int kRowCls = 5;
constexpr int kRowClsM[kRowCls] = {1, 3, 5, 7, 0};

// Per-grid tables on the device, in the arithmetic type T of the kernels.
// Built once per (grid, precision) by the host from the FP64 geometry.
template <class T>
struct Geom {
  int I, J, K;
  // scalar / U rows (J)
  const int* Mu;    // leap stride M_j (odd), Eq. 6 / Eq. 7
  const T* rdx;     // 1 / (a sin(theta_j) M_j dlam): leap zonal difference
  const T* rdy;     // 1 / (a sin(theta_j) dth): meridional divergence
  const T* zf;      // a dth / M_j: zonal face length over the leap stride
  const T* r2A;     // 1 / (2 A_j)
  const T* f0;      // 2 Omega cos(theta_j)
  const T* cota;    // cot(theta_j) / a
  // V rows (J-1)
  const int* Mv;    // leap stride of the V rows
  const T* sv;      // sin(theta^v_j)
  const T* yv;      // a dlam sin(theta^v_j): meridional face length
  const T* zfv;     // a dth / Mv_j
  const T* r2Av;    // 1 / (2 Av_j)
  const T* cn;      // A_j / (4 Av_j)   Coriolis weight of the northern U row
  const T* cs;      // A_{j+1} / (4 Av_j) Coriolis weight of the southern U row
  // levels
  const T* ds;      // dsigma_k (K)
  const T* r2ds;    // 1 / (2 dsigma_k) (K)
  // hydrostatic weights times the level coefficient beta_k = (1 - delta_p)
  // (1 + delta_c) b_k of Eq. 1 (b_k = sqrt(kappa R T~(sigma_k))):
  const T* hk;      // beta_k ln(sh_{k+1}/sh_k), the off-diagonal weight; hk[0] = 0 (K)
  const T* Hkk;     // beta_k ln(sh_{k+1}/sigma_k), the diagonal (K)
  const T* hk_rds;  // hk / dsigma_k (K)
  const T* rho;     // beta2 / beta_k: the delta kappa Phi/P part of the coefficient (K)
  const T* oms;     // 1 - sigma_hat_k (K): W_k = SD_k - (1 - sigma_hat_k) C
  // rows the low-latitude filter changes, entry 4 j + band (1 two-grid, 2 3-point)
  const int* filtU; // scalar / U rows
  const int* filtV; // V rows
  int nfU, nfV;
  const double* dsd;  // dsigma_k in FP64 (column integral of the divergence)
  const double* shd;  // half levels sigma_hat_h in FP64 (K+1)
  const double* Ad;   // A_j in FP64 (J)     (diagnostics)
  const double* Avd;  // Av_j in FP64 (J-1)  (diagnostics)
  // columns (J*I)
  const T* rt0pit;  // R T~_s / pi~
  const T* pit;     // pi~: standard surface pressure / p0 under phi_s
  int nl;           // 1: the delta kappa Phi/P term is on (beta2 != 0)
  int l1lo, l1hi;   // rows [l1lo, l1hi): interior rows whose strides Mu_j, Mv_j, Mu_{j+1} are all 1
  T rady;           // 1 / (a dth)
  T adl;            // a dlam
  // work items of the row-segment stage kernel (agcm_row.cuh), j << 8 | segment:
  // nk[c] items of the rows of stride class c, listed by class: strides all
  // kRowClsM[c] (1, 3, 5, 7), then (c = kRowCls - 1) the other rows; and the
  // nrowc rows left to the column kernel (agcm_fused.cuh)
  const int* rowk;
  const int* rowc;
  int nk[kRowCls], nrowc;
  int rowfill;      // 1: the row-segment items fill the GPU at least four times over
};

__device__ __forceinline__ int wrapi(int i, int I) {
  return i < 0 ? i + I : (i >= I ? i - I : i);
}

template <class T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

// sqrt in the kernel's type
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }

}  // namespace agcm
