// agcm_phases.cuh — phases A and B of the spatial operator T(x), the forward
// recompute that the adjoint needs.
//
//  phase A (colstate): m = pi~ + pi, P = sqrt(m) and its U/V-point values and
//                      reciprocals (2-D, one thread per column).
//  phase B (column):   leap divergence D_k (Eq. 6 on the staggered mass flux),
//                      the column sum C (FP64) that gives dpi/dt = -C, the
//                      sigma mass flux W_h = sh_h C - sum_{k<h} dsigma D
//                      (Alg. 1 / Alg. 2), the Omega~ term and the
//                      hydrostatic psi = phi' + R T~_s pi/pi~ (one thread per column,
//                      loops over k).
//  phase C:            advection (skew form, zonal partners at +-M),
//                      pressure gradient at the (x+N, x-N+1) pair, Coriolis
//                      pair and the stage update; the forward step computes
//                      it inside the fused kernel of agcm_fused.cuh (with the
//                      phase-B intermediates kept on chip), and its reverse is
//                      k_adj_update in agcm_adjoint.cuh.
// The adjoint kernels mirror this decomposition.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

template <class T>
struct ColState {  // phase-A outputs, J*I each (Pv/rPv: (J-1)*I)
  T *P, *rP, *Pu, *rPu, *Pv, *rPv;
};

template <class T>
__global__ void __launch_bounds__(256) k_colstate(Geom<T> g, const T* __restrict__ pi, ColState<T> cs) {
  const int I = g.I, J = g.J;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I, i = n - j * I;
  const T m = g.pit[n] + pi[n];
  const T P = sqrt_t(m);
  cs.P[n] = P;
  cs.rP[n] = T(1) / P;
  const int ip = wrapi(i + 1, I);
  const T mu = T(0.5) * (m + (g.pit[j * I + ip] + pi[j * I + ip]));
  const T Pu = sqrt_t(mu);
  cs.Pu[n] = Pu;
  cs.rPu[n] = T(1) / Pu;
  if (j < J - 1) {
    const T mv = T(0.5) * (m + (g.pit[n + I] + pi[n + I]));
    const T Pv = sqrt_t(mv);
    cs.Pv[n] = Pv;
    cs.rPv[n] = T(1) / Pv;
  }
}

// Leap-format divergence of the mass flux at scalar point (k, j, i).
template <class T>
__device__ __forceinline__ T divergence(const Geom<T>& g, const T* __restrict__ U, const T* __restrict__ V,
                                        const T* __restrict__ Pu, const T* __restrict__ Pv, int k, int j,
                                        int i) {
  const int I = g.I, J = g.J;
  const int M = g.Mu[j];
  const int ue = wrapi(i + (M - 1) / 2, I), uw = wrapi(i - (M + 1) / 2, I);
  const size_t r3 = ((size_t)k * J + j) * I;
  const size_t r2 = (size_t)j * I;
  T d = (ldg(Pu + r2 + ue) * ldg(U + r3 + ue) - ldg(Pu + r2 + uw) * ldg(U + r3 + uw)) * g.rdx[j];
  T mer = T(0);
  const size_t rv = ((size_t)k * (J - 1) + j) * I;
  if (j < J - 1) mer += g.sv[j] * ldg(Pv + r2 + i) * ldg(V + rv + i);
  if (j > 0) mer -= g.sv[j - 1] * ldg(Pv + r2 - I + i) * ldg(V + rv - I + i);
  // (sin(theta^v_j) F_j - sin(theta^v_{j-1}) F_{j-1}) / (a sin(theta_j) dth)
  return d + mer * g.rdy[j];
}

// Phase B outputs.  W: (K+1)*J*I half-level mass fluxes; X: the factor
// S_k = Hkk_k D_k + hkr_k Q_k of the Omega~ tendency -rP c_k S_k (Q_k the
// divergence integrated from the top; c_k = 1, or 1 + rho_k Phi_k / P with
// Eq. 1's delta kappa Phi/P term); psi: hydrostatic potential;
// pi_out = pi_base - c*dt*C (or -C when pi_base == nullptr and c*dt = 1).
template <class T>
__global__ void __launch_bounds__(128) k_column(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                                const T* __restrict__ Phi, const T* __restrict__ pi,
                                                ColState<T> cs, T* __restrict__ W, T* __restrict__ X,
                                                T* __restrict__ psi, const T* pi_base, T* pi_out,
                                                double cdt, double* __restrict__ Cout) {
  const int I = g.I, J = g.J, K = g.K;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I, i = n - j * I;
  const size_t plane = (size_t)J * I;
  // pass 1: column integral of the divergence (FP64 in every precision)
  double C = 0.0;
  for (int k = 0; k < K; ++k) C += g.dsd[k] * (double)divergence(g, U, V, cs.Pu, cs.Pv, k, j, i);
  if (Cout) Cout[n] = C;
  const double pb = pi_base ? (double)pi_base[n] : 0.0;
  pi_out[n] = (T)(pb - cdt * C);
  // pass 2: prefix sum from the top -> W at half levels and the Omega~ factor
  const T bP = cs.rP[n];  // the level coefficient sits in the H tables
  double Q = 0.0;
  W[n] = T(0);
  for (int k = 0; k < K; ++k) {
    const T D = divergence(g, U, V, cs.Pu, cs.Pv, k, j, i);
    if (k > 0) W[(size_t)k * plane + n] = (T)(g.shd[k] * C - Q);
    X[(size_t)k * plane + n] = g.Hkk[k] * D + g.hk_rds[k] * (T)Q;
    Q += g.dsd[k] * (double)D;
  }
  W[(size_t)K * plane + n] = T(0);
  // pass 3: suffix sum from the surface -> phi' + R T~_s pi / pi~, with
  // B = Phi/P, times 1 + rho_k Phi/P under the delta kappa Phi/P term
  const T ps = g.rt0pit[n] * pi[n];
  T S = T(0);
  for (int k = K - 1; k >= 0; --k) {
    T B = bP * Phi[(size_t)k * plane + n];
    if (g.nl) B *= T(1) + g.rho[k] * B;
    psi[(size_t)k * plane + n] = g.Hkk[k] * B + S + ps;
    S += g.hk[k] * B;
  }
}

}  // namespace agcm
