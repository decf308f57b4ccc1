// agcm_phases.cuh — the spatial operator T(x) as three phase kernels.
//
//  phase A (colstate): m = pi~ + pi, P = sqrt(m) and its U/V-point values and
//                      reciprocals (2-D, one thread per column).
//  phase B (column):   leap divergence D_k (Eq. 6 on the staggered mass flux),
//                      the column sum C (FP64) that gives dpi/dt = -C, the
//                      sigma mass flux W_h = sh_h C - sum_{k<h} dsigma D
//                      (Alg. 1 / Alg. 2), the Omega~ term and the
//                      hydrostatic psi = phi' + R T0 pi/pi~ (one thread per column,
//                      loops over k).
//  phase C (update):   advection (skew form, zonal partners at +-M),
//                      pressure gradient at the (x+N, x-N+1) pair, Coriolis
//                      pair, and the stage update out = base + c*dt*T
//                      (one thread per grid point).
// The adjoint kernels mirror this decomposition.  The production forward step
// uses the fused kernel of agcm_fused.cuh, which computes the same arithmetic
// with the phase-B intermediates kept on chip.
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

// Phase B outputs.  W: (K+1)*J*I half-level mass fluxes; X: Omega~ tendency;
// psi: hydrostatic potential; pi_out = pi_base - c*dt*C (or -C when
// pi_base == nullptr and c*dt = 1).
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
  // pass 2: prefix sum from the top -> W at half levels and the Omega~ term
  const T bP = cs.rP[n];  // the level coefficient sits in the H tables
  double Q = 0.0;
  W[n] = T(0);
  for (int k = 0; k < K; ++k) {
    const T D = divergence(g, U, V, cs.Pu, cs.Pv, k, j, i);
    if (k > 0) W[(size_t)k * plane + n] = (T)(g.shd[k] * C - Q);
    X[(size_t)k * plane + n] = -bP * (g.Hkk[k] * D + g.hk_rds[k] * (T)Q);
    Q += g.dsd[k] * (double)D;
  }
  W[(size_t)K * plane + n] = T(0);
  // pass 3: suffix sum from the surface -> phi' + R T~_s pi / pi~
  const T ps = g.rt0pit[n] * pi[n];
  T S = T(0);
  for (int k = K - 1; k >= 0; --k) {
    const T B = bP * Phi[(size_t)k * plane + n];
    psi[(size_t)k * plane + n] = g.Hkk[k] * B + S + ps;
    S += g.hk[k] * B;
  }
}

// Phase C: tendencies of U, V, Phi at (k, j, i) and the stage update.
template <class T>
__global__ void __launch_bounds__(256) k_update(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                                const T* __restrict__ Phi, ColState<T> cs,
                                                const T* __restrict__ W, const T* __restrict__ X,
                                                const T* __restrict__ psi, const T* Ub, const T* Vb,
                                                const T* Phib, T* Uo, T* Vo, T* Phio, T cdt) {
  // base and out may alias (the last stage updates x_n in place); each thread
  // reads base and writes out at its own point only.
  const int I = g.I, J = g.J, K = g.K;
  const size_t N = (size_t)K * J * I;
  const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int i = (int)(n % I);
  const size_t kj = n / I;
  const int j = (int)(kj % J), k = (int)(kj / J);
  const size_t plane = (size_t)J * I, vplane = (size_t)(J - 1) * I;
  const size_t r3 = ((size_t)k * J + j) * I;  // scalar/U row base
  const size_t r2 = (size_t)j * I;
  const size_t rv = ((size_t)k * (J - 1) + j) * I;  // V row base (valid for j < J-1)
  const T* Pu = cs.Pu;
  const T* rPu = cs.rPu;
  const T* Pv = cs.Pv;
  const T* rPv = cs.rPv;
  const T* rP = cs.rP;
  const bool hasS = j < J - 1, hasN = j > 0;
  const int M = g.Mu[j];
  const T zf = g.zf[j];

  auto Fl = [&](size_t row3, size_t row2, int u) { return ldg(Pu + row2 + u) * ldg(U + row3 + u); };
  auto Ft = [&](size_t rowv, size_t row2, int ii) { return ldg(Pv + row2 + ii) * ldg(V + rowv + ii); };

  // ---------------- Phi at scalar point (k, j, i) ----------------
  {
    const int ue = wrapi(i + (M - 1) / 2, I), uw = wrapi(i - (M + 1) / 2, I);
    const int ie = wrapi(i + M, I), iw = wrapi(i - M, I);
    T hor = zf * (Fl(r3, r2, ue) * ldg(Phi + r3 + ie) * ldg(rP + r2 + ie) -
                  Fl(r3, r2, uw) * ldg(Phi + r3 + iw) * ldg(rP + r2 + iw));
    if (hasS) hor += g.yv[j] * Ft(rv, r2, i) * ldg(Phi + r3 + I + i) * ldg(rP + r2 + I + i);
    if (hasN) hor -= g.yv[j - 1] * Ft(rv - I, r2 - I, i) * ldg(Phi + r3 - I + i) * ldg(rP + r2 - I + i);
    T ver = T(0);
    const T rPc = ldg(rP + r2 + i);
    if (k < K - 1) ver += ldg(W + (size_t)(k + 1) * plane + r2 + i) * ldg(Phi + r3 + plane + i) * rPc;
    if (k > 0) ver -= ldg(W + (size_t)k * plane + r2 + i) * ldg(Phi + r3 - plane + i) * rPc;
    const T L = (hor * g.r2A[j] + ver * g.r2ds[k]) * rPc;
    const T tend = -L + ldg(X + n);
    Phio[n] = (Phib ? Phib[n] : T(0)) + cdt * tend;
  }
  // ---------------- U at (k, j, u = i) ----------------
  {
    const int u = i;
    const int iE = u + (M + 1) / 2, iW = u - (M - 1) / 2;
    const T ZE = zf * T(0.5) * (Fl(r3, r2, wrapi(iE - 1, I)) + Fl(r3, r2, wrapi(iE, I)));
    const T ZW = zf * T(0.5) * (Fl(r3, r2, wrapi(iW - 1, I)) + Fl(r3, r2, wrapi(iW, I)));
    const int ue = wrapi(u + M, I), uw = wrapi(u - M, I);
    const int up = wrapi(u + 1, I);
    T hor = ZE * ldg(U + r3 + ue) * ldg(rPu + r2 + ue) - ZW * ldg(U + r3 + uw) * ldg(rPu + r2 + uw);
    if (hasS) {
      const T YS = T(0.5) * g.yv[j] * (Ft(rv, r2, u) + Ft(rv, r2, up));
      hor += YS * ldg(U + r3 + I + u) * ldg(rPu + r2 + I + u);
    }
    if (hasN) {
      const T YN = T(0.5) * g.yv[j - 1] * (Ft(rv - I, r2 - I, u) + Ft(rv - I, r2 - I, up));
      hor -= YN * ldg(U + r3 - I + u) * ldg(rPu + r2 - I + u);
    }
    const T rPc = ldg(rPu + r2 + u);
    T ver = T(0);
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      ver += T(0.5) * (ldg(W + wb + u) + ldg(W + wb + up)) * ldg(U + r3 + plane + u) * ldg(rPu + r2 + u);
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      ver -= T(0.5) * (ldg(W + wt + u) + ldg(W + wt + up)) * ldg(U + r3 - plane + u) * ldg(rPu + r2 + u);
    }
    const T L = (hor * g.r2A[j] + ver * g.r2ds[k]) * rPc;
    const T pgf = ldg(Pu + r2 + u) *
                  (ldg(psi + r3 + wrapi(u + (M + 1) / 2, I)) - ldg(psi + r3 + wrapi(u - (M - 1) / 2, I))) *
                  g.rdx[j];
    const T Uc = ldg(U + r3 + u);
    const T fs = g.f0[j] + Uc * rPc * g.cota[j];
    T vs = T(0);
    if (hasN) vs += ldg(V + rv - I + u) + ldg(V + rv - I + up);
    if (hasS) vs += ldg(V + rv + u) + ldg(V + rv + up);
    const T tend = -L - pgf - T(0.25) * fs * vs;
    Uo[n] = (Ub ? Ub[n] : T(0)) + cdt * tend;
  }
  // ---------------- V at (k, j, i), j < J-1 ----------------
  if (hasS) {
    const int Mv = g.Mv[j];
    const T zfv = g.zfv[j];
    const int uE = wrapi(i + (Mv - 1) / 2, I), uW = wrapi(i - (Mv + 1) / 2, I);
    const T ZE = zfv * T(0.5) * (Fl(r3, r2, uE) + Fl(r3 + I, r2 + I, uE));
    const T ZW = zfv * T(0.5) * (Fl(r3, r2, uW) + Fl(r3 + I, r2 + I, uW));
    const int ie = wrapi(i + Mv, I), iw = wrapi(i - Mv, I);
    T hor = ZE * ldg(V + rv + ie) * ldg(rPv + r2 + ie) - ZW * ldg(V + rv + iw) * ldg(rPv + r2 + iw);
    const T Fc = Ft(rv, r2, i);
    if (j + 1 < J - 1) {
      const T YS = T(0.5) * (g.yv[j] * Fc + g.yv[j + 1] * Ft(rv + I, r2 + I, i));
      hor += YS * ldg(V + rv + I + i) * ldg(rPv + r2 + I + i);
    }
    if (hasN) {
      const T YN = T(0.5) * (g.yv[j - 1] * Ft(rv - I, r2 - I, i) + g.yv[j] * Fc);
      hor -= YN * ldg(V + rv - I + i) * ldg(rPv + r2 - I + i);
    }
    const T rPc = ldg(rPv + r2 + i);
    T ver = T(0);
    const size_t vpl = vplane;
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      ver += T(0.5) * (ldg(W + wb + i) + ldg(W + wb + I + i)) * ldg(V + rv + vpl + i) * rPc;
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      ver -= T(0.5) * (ldg(W + wt + i) + ldg(W + wt + I + i)) * ldg(V + rv - vpl + i) * rPc;
    }
    const T L = (hor * g.r2Av[j] + ver * g.r2ds[k]) * rPc;
    const T pgf = ldg(Pv + r2 + i) * (ldg(psi + r3 + I + i) - ldg(psi + r3 + i)) * g.rady;
    const int im = wrapi(i - 1, I);
    auto fU = [&](size_t row3, size_t row2, int jj, int uu) {
      const T Uv = ldg(U + row3 + uu);
      return (g.f0[jj] + Uv * ldg(rPu + row2 + uu) * g.cota[jj]) * Uv;
    };
    const T cor = g.cn[j] * (fU(r3, r2, j, im) + fU(r3, r2, j, i)) +
                  g.cs[j] * (fU(r3 + I, r2 + I, j + 1, im) + fU(r3 + I, r2 + I, j + 1, i));
    const T tend = -L - pgf + cor;
    const size_t nv = rv + i;
    Vo[nv] = (Vb ? Vb[nv] : T(0)) + cdt * tend;
  }
}

}  // namespace agcm
