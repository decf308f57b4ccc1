// agcm_adjoint.cuh — hand-written adjoint (vector-Jacobian product) of the
// spatial operator T at a state x, in the phase decomposition of
// agcm_phases.cuh, run in reverse:
//
//   k_adj_update   reverse of phase C: every term c*a*b of the advection,
//                  pressure-gradient and Coriolis tendencies sends c*b*ybar to
//                  a and c*a*ybar to b.  Flux and G = F/P adjoints are scattered
//                  with atomics into 3-D accumulators; the adjoints of the
//                  level-independent factors P^u, 1/P, ... of a point's own
//                  tendency are stored per point (no atomics) and summed over k
//                  later.
//   k_adj_column   reverse of phase B (one thread per column): the column
//                  integral C, the sigma mass flux W (Alg. 1 / Alg. 2), the
//                  hydrostatic psi and the Omega~ term are linear in D and
//                  B = Phi / P (the level coefficient of Eq. 1 sits in the H
//                  tables), so their adjoints are the transposed prefix /
//                  suffix scans; D's adjoint is scattered to the fluxes.
// With Eq. 1's nonlinear delta kappa Phi/P term the level coefficient of
// psi and Omega~ becomes c_k = 1 + rho_k G (G = Phi/P, the level's beta_k in
// the tables): B_k = G c_k enters psi and -rP c_k S_k is the Omega~ tendency,
// so the reverse column pass carries dB/dG = 1 + 2 rho_k G and the
// derivatives of c_k.
//   k_adj_conv     F = P^u U, G = U / P^u, ... -> adjoints of U, V, Phi and the
//                  2-D adjoints of P, P^u, P^v, folded into the adjoint of the
//                  mass m = pi~ + pi.
//   k_adj_colstate m^u, m^v are stride-1 means of m; gathers the adjoint of pi.
//
// Output: out = (accumulate ? out : 0) + scale * J(x)^T ybar, and optionally
// sum += scale * J(x)^T ybar in the same pass (the stage accumulation).
#pragma once
#include "agcm_common.cuh"
#include "agcm_phases.cuh"

namespace agcm {

template <class T>
struct AdjBufs {
  // 3-D accumulators (atomic targets, zeroed before each product)
  T *aU, *aV, *aFl, *aFt, *aGu, *aGv, *aGs, *aW, *aPsi;
  // 3-D per-point stores (every element written)
  T *aPhi, *tRP, *tRPu, *tPu, *tRPv, *tPv;
  // 2-D per-column stores
  T *arPcol, *aPiD, *mub, *mvb, *mcb;
};

template <class T>
__device__ __forceinline__ void aadd(T* p, T v) {
  atomicAdd(p, v);
}

// Reverse of phase C at (k, j, i): U point (j, u = i), Phi point, V point.
template <class T>
__device__ __forceinline__ void adj_update_point(
    const Geom<T>& g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ Phi,
    const T* __restrict__ Pu, const T* __restrict__ rPu, const T* __restrict__ Pv, const T* __restrict__ rPv,
    const T* __restrict__ rP, const T* __restrict__ W, const T* __restrict__ psi, const T* __restrict__ yU,
    const T* __restrict__ yV, const T* __restrict__ yPhi, const AdjBufs<T>& a, const int k, const int j,
    const int i) {
  // every input is read-only here and every output is written with atomics
  // or plain stores to other arrays, so the reads are declared restrict and
  // the row tables read once, letting loads move ahead of the atomics
  const int I = g.I, J = g.J, K = g.K;
  const bool hasS_ = j < J - 1, hasN_ = j > 0, hasSS_ = j + 1 < J - 1;
  const T yvj = hasS_ ? g.yv[j] : T(0), yvjm = hasN_ ? g.yv[j - 1] : T(0), yvjp = hasSS_ ? g.yv[j + 1] : T(0);
  const T r2Aj = g.r2A[j], r2dsk = g.r2ds[k], rdxj = g.rdx[j], f0j = g.f0[j], cotaj = g.cota[j];
  const T zfvj = hasS_ ? g.zfv[j] : T(0), r2Avj = hasS_ ? g.r2Av[j] : T(0);
  const T cnj = hasS_ ? g.cn[j] : T(0), csj = hasS_ ? g.cs[j] : T(0);
  const T f0j1 = hasS_ ? g.f0[j + 1] : T(0), cotaj1 = hasS_ ? g.cota[j + 1] : T(0);
  const int Mvj = hasS_ ? g.Mv[j] : 1;
  const T rady = g.rady;
  const size_t n = ((size_t)k * J + j) * I + i;
  const size_t plane = (size_t)J * I, vplane = (size_t)(J - 1) * I;
  const size_t r3 = ((size_t)k * J + j) * I, r2 = (size_t)j * I, rv = ((size_t)k * (J - 1) + j) * I;
  const bool hasS = j < J - 1, hasN = j > 0;
  const int M = g.Mu[j];
  const T zf = g.zf[j];
  auto Fl = [&](size_t row3, size_t row2, int u) { return Pu[row2 + u] * U[row3 + u]; };
  auto Ft = [&](size_t rowv, size_t row2, int ii) { return Pv[row2 + ii] * V[rowv + ii]; };

  // ---------------- Phi point ----------------
  {
    const T yb = yPhi[n];
    const int fE = wrapi(i + (M - 1) / 2, I), fW = wrapi(i - (M + 1) / 2, I);
    const int ie = wrapi(i + M, I), iw = wrapi(i - M, I);
    const T ZE = zf * Fl(r3, r2, fE), ZW = zf * Fl(r3, r2, fW);
    const T Ge = Phi[r3 + ie] * rP[r2 + ie], Gw = Phi[r3 + iw] * rP[r2 + iw];
    T hor = ZE * Ge - ZW * Gw;
    T Gs_s = 0, Gs_n = 0, Ft_c = 0, Ft_n = 0;
    if (hasS) {
      Gs_s = Phi[r3 + I + i] * rP[r2 + I + i];
      Ft_c = Ft(rv, r2, i);
      hor += yvj * Ft_c * Gs_s;
    }
    if (hasN) {
      Gs_n = Phi[r3 - I + i] * rP[r2 - I + i];
      Ft_n = Ft(rv - I, r2 - I, i);
      hor -= yvjm * Ft_n * Gs_n;
    }
    const T rPc = rP[r2 + i];
    T ver = 0, Wb = 0, Wt = 0, Gb = 0, Gt = 0;
    if (k < K - 1) {
      Wb = W[(size_t)(k + 1) * plane + r2 + i];
      Gb = Phi[r3 + plane + i] * rPc;
      ver += Wb * Gb;
    }
    if (k > 0) {
      Wt = W[(size_t)k * plane + r2 + i];
      Gt = Phi[r3 - plane + i] * rPc;
      ver -= Wt * Gt;
    }
    // T = -(hor r2A + ver r2ds) rPc + X
    const T Lb = -yb;
    const T hb = Lb * r2Aj * rPc, vb = Lb * r2dsk * rPc;
    a.tRP[n] = Lb * (hor * r2Aj + ver * r2dsk);
    aadd(a.aFl + r3 + fE, zf * hb * Ge);
    aadd(a.aFl + r3 + fW, -zf * hb * Gw);
    aadd(a.aGs + r3 + ie, hb * ZE);
    aadd(a.aGs + r3 + iw, -hb * ZW);
    if (hasS) {
      aadd(a.aFt + rv + i, hb * yvj * Gs_s);
      aadd(a.aGs + r3 + I + i, hb * yvj * Ft_c);
    }
    if (hasN) {
      aadd(a.aFt + rv - I + i, -hb * yvjm * Gs_n);
      aadd(a.aGs + r3 - I + i, -hb * yvjm * Ft_n);
    }
    if (k < K - 1) {
      aadd(a.aW + (size_t)(k + 1) * plane + r2 + i, vb * Gb);
      aadd(a.aGs + r3 + plane + i, vb * Wb);
    }
    if (k > 0) {
      aadd(a.aW + (size_t)k * plane + r2 + i, -vb * Gt);
      aadd(a.aGs + r3 - plane + i, -vb * Wt);
    }
  }
  // ---------------- U point ----------------
  {
    const int u = i;
    const T yb = yU[n];
    const int fE = wrapi(u + (M - 1) / 2, I), fE1 = wrapi(u + (M + 1) / 2, I);
    const int fW = wrapi(u - (M + 1) / 2, I), fW1 = wrapi(u - (M - 1) / 2, I);
    const int ue = wrapi(u + M, I), uw = wrapi(u - M, I), up = wrapi(u + 1, I);
    const T ZE = zf * T(0.5) * (Fl(r3, r2, fE) + Fl(r3, r2, fE1));
    const T ZW = zf * T(0.5) * (Fl(r3, r2, fW) + Fl(r3, r2, fW1));
    const T Ge = U[r3 + ue] * rPu[r2 + ue], Gw = U[r3 + uw] * rPu[r2 + uw];
    T hor = ZE * Ge - ZW * Gw;
    T YS = 0, YN = 0, Gs_ = 0, Gn_ = 0;
    if (hasS) {
      YS = T(0.5) * yvj * (Ft(rv, r2, u) + Ft(rv, r2, up));
      Gs_ = U[r3 + I + u] * rPu[r2 + I + u];
      hor += YS * Gs_;
    }
    if (hasN) {
      YN = T(0.5) * yvjm * (Ft(rv - I, r2 - I, u) + Ft(rv - I, r2 - I, up));
      Gn_ = U[r3 - I + u] * rPu[r2 - I + u];
      hor -= YN * Gn_;
    }
    const T rPc = rPu[r2 + u];
    T ver = 0, WB = 0, WT = 0, Gb = 0, Gt = 0;
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      WB = T(0.5) * (W[wb + u] + W[wb + up]);
      Gb = U[r3 + plane + u] * rPc;
      ver += WB * Gb;
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      WT = T(0.5) * (W[wt + u] + W[wt + up]);
      Gt = U[r3 - plane + u] * rPc;
      ver -= WT * Gt;
    }
    const T dpsi = psi[r3 + fE1] - psi[r3 + fW1];
    const T Puc = Pu[r2 + u];
    const T Uc = U[r3 + u];
    const T Gc = Uc * rPc;
    const T fs = f0j + Gc * cotaj;
    T vs = 0;
    if (hasN) vs += V[rv - I + u] + V[rv - I + up];
    if (hasS) vs += V[rv + u] + V[rv + up];
    // T = -(hor r2A + ver r2ds) rPu - Pu dpsi rdx - 1/4 fs vs
    const T Lb = -yb;
    const T hb = Lb * r2Aj * rPc, vb = Lb * r2dsk * rPc;
    a.tRPu[n] = Lb * (hor * r2Aj + ver * r2dsk);
    a.tPu[n] = -yb * dpsi * rdxj;
    aadd(a.aPsi + r3 + fE1, -yb * Puc * rdxj);
    aadd(a.aPsi + r3 + fW1, yb * Puc * rdxj);
    const T fsb = -T(0.25) * yb * vs, vsb = -T(0.25) * yb * fs;
    aadd(a.aGu + r3 + u, fsb * cotaj);
    if (hasN) {
      aadd(a.aV + rv - I + u, vsb);
      aadd(a.aV + rv - I + up, vsb);
    }
    if (hasS) {
      aadd(a.aV + rv + u, vsb);
      aadd(a.aV + rv + up, vsb);
    }
    const T ZEb = hb * Ge, ZWb = -hb * Gw;
    aadd(a.aGu + r3 + ue, hb * ZE);
    aadd(a.aGu + r3 + uw, -hb * ZW);
    aadd(a.aFl + r3 + fE, T(0.5) * zf * ZEb);
    aadd(a.aFl + r3 + fE1, T(0.5) * zf * ZEb);
    aadd(a.aFl + r3 + fW, T(0.5) * zf * ZWb);
    aadd(a.aFl + r3 + fW1, T(0.5) * zf * ZWb);
    if (hasS) {
      const T YSb = hb * Gs_;
      aadd(a.aGu + r3 + I + u, hb * YS);
      aadd(a.aFt + rv + u, T(0.5) * yvj * YSb);
      aadd(a.aFt + rv + up, T(0.5) * yvj * YSb);
    }
    if (hasN) {
      const T YNb = -hb * Gn_;
      aadd(a.aGu + r3 - I + u, -hb * YN);
      aadd(a.aFt + rv - I + u, T(0.5) * yvjm * YNb);
      aadd(a.aFt + rv - I + up, T(0.5) * yvjm * YNb);
    }
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      aadd(a.aW + wb + u, T(0.5) * vb * Gb);
      aadd(a.aW + wb + up, T(0.5) * vb * Gb);
      aadd(a.aGu + r3 + plane + u, vb * WB);
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      aadd(a.aW + wt + u, -T(0.5) * vb * Gt);
      aadd(a.aW + wt + up, -T(0.5) * vb * Gt);
      aadd(a.aGu + r3 - plane + u, -vb * WT);
    }
  }
  // ---------------- V point (j < J-1) ----------------
  if (hasS) {
    const size_t nv = rv + i;
    const T yb = yV[nv];
    const int Mv = Mvj;
    const T zfv = zfvj;
    const int uE = wrapi(i + (Mv - 1) / 2, I), uW = wrapi(i - (Mv + 1) / 2, I);
    const int ie = wrapi(i + Mv, I), iw = wrapi(i - Mv, I);
    const T ZE = zfv * T(0.5) * (Fl(r3, r2, uE) + Fl(r3 + I, r2 + I, uE));
    const T ZW = zfv * T(0.5) * (Fl(r3, r2, uW) + Fl(r3 + I, r2 + I, uW));
    const T Ge = V[rv + ie] * rPv[r2 + ie], Gw = V[rv + iw] * rPv[r2 + iw];
    T hor = ZE * Ge - ZW * Gw;
    const T Fc = Ft(rv, r2, i);
    T YS = 0, YN = 0, Gs_ = 0, Gn_ = 0;
    const bool hasSS = j + 1 < J - 1;
    if (hasSS) {
      YS = T(0.5) * (yvj * Fc + yvjp * Ft(rv + I, r2 + I, i));
      Gs_ = V[rv + I + i] * rPv[r2 + I + i];
      hor += YS * Gs_;
    }
    if (hasN) {
      YN = T(0.5) * (yvjm * Ft(rv - I, r2 - I, i) + yvj * Fc);
      Gn_ = V[rv - I + i] * rPv[r2 - I + i];
      hor -= YN * Gn_;
    }
    const T rPc = rPv[r2 + i];
    T ver = 0, WB = 0, WT = 0, Gb = 0, Gt = 0;
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      WB = T(0.5) * (W[wb + i] + W[wb + I + i]);
      Gb = V[rv + vplane + i] * rPc;
      ver += WB * Gb;
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      WT = T(0.5) * (W[wt + i] + W[wt + I + i]);
      Gt = V[rv - vplane + i] * rPc;
      ver -= WT * Gt;
    }
    const T dpsi = psi[r3 + I + i] - psi[r3 + i];
    const T Pvc = Pv[r2 + i];
    // T = -(hor r2Av + ver r2ds) rPv - Pv dpsi rady + cor
    const T Lb = -yb;
    const T hb = Lb * r2Avj * rPc, vb = Lb * r2dsk * rPc;
    a.tRPv[nv] = Lb * (hor * r2Avj + ver * r2dsk);
    a.tPv[nv] = -yb * dpsi * rady;
    aadd(a.aPsi + r3 + I + i, -yb * Pvc * rady);
    aadd(a.aPsi + r3 + i, yb * Pvc * rady);
    // Coriolis: cor = cn (fU(j,im) + fU(j,i)) + cs (fU(j+1,im) + fU(j+1,i)),
    // fU = (f0 + G cota) U with G = U / P^u:  dU += c (f0 + G cota), dG += c U cota
    const int im = wrapi(i - 1, I);
    auto corb = [&](size_t row3, int jj, int uu, T c) {
      const T f0r = jj == j ? f0j : f0j1, cotar = jj == j ? cotaj : cotaj1;
      const T Uv = U[row3 + uu];
      const T Gv_ = Uv * rPu[(size_t)jj * I + uu];
      aadd(a.aU + row3 + uu, c * (f0r + Gv_ * cotar));
      aadd(a.aGu + row3 + uu, c * Uv * cotar);
    };
    corb(r3, j, im, yb * cnj);
    corb(r3, j, i, yb * cnj);
    corb(r3 + I, j + 1, im, yb * csj);
    corb(r3 + I, j + 1, i, yb * csj);
    // advection
    const T ZEb = hb * Ge, ZWb = -hb * Gw;
    aadd(a.aGv + rv + ie, hb * ZE);
    aadd(a.aGv + rv + iw, -hb * ZW);
    aadd(a.aFl + r3 + uE, T(0.5) * zfv * ZEb);
    aadd(a.aFl + r3 + I + uE, T(0.5) * zfv * ZEb);
    aadd(a.aFl + r3 + uW, T(0.5) * zfv * ZWb);
    aadd(a.aFl + r3 + I + uW, T(0.5) * zfv * ZWb);
    if (hasSS) {
      const T YSb = hb * Gs_;
      aadd(a.aGv + rv + I + i, hb * YS);
      aadd(a.aFt + rv + i, T(0.5) * yvj * YSb);
      aadd(a.aFt + rv + I + i, T(0.5) * yvjp * YSb);
    }
    if (hasN) {
      const T YNb = -hb * Gn_;
      aadd(a.aGv + rv - I + i, -hb * YN);
      aadd(a.aFt + rv - I + i, T(0.5) * yvjm * YNb);
      aadd(a.aFt + rv + i, T(0.5) * yvj * YNb);
    }
    if (k < K - 1) {
      const size_t wb = (size_t)(k + 1) * plane + r2;
      aadd(a.aW + wb + i, T(0.5) * vb * Gb);
      aadd(a.aW + wb + I + i, T(0.5) * vb * Gb);
      aadd(a.aGv + rv + vplane + i, vb * WB);
    }
    if (k > 0) {
      const size_t wt = (size_t)k * plane + r2;
      aadd(a.aW + wt + i, -T(0.5) * vb * Gt);
      aadd(a.aW + wt + I + i, -T(0.5) * vb * Gt);
      aadd(a.aGv + rv - vplane + i, -vb * WT);
    }
  }
}

// One thread per column of a kAdjTileX x kAdjTileY tile, levels in a loop (at
// most 102 registers: 5 blocks per SM):
// the 2-D factors of a column and the level above and below are re-read from
// L1 instead of from other SMs' working sets.
constexpr int kAdjTileX = 32, kAdjTileY = 4;
template <class T>
__global__ void __launch_bounds__(kAdjTileX* kAdjTileY, 5) k_adj_update(
    Geom<T> g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ Phi, ColState<T> cs,
    const T* __restrict__ W, const T* __restrict__ psi, const T* __restrict__ yU, const T* __restrict__ yV,
    const T* __restrict__ yPhi, AdjBufs<T> a) {
  const int i = blockIdx.x * kAdjTileX + (int)(threadIdx.x % kAdjTileX);
  const int j = blockIdx.y * kAdjTileY + (int)(threadIdx.x / kAdjTileX);
  if (i >= g.I || j >= g.J) return;
  for (int k = 0; k < g.K; ++k)
    adj_update_point<T>(g, U, V, Phi, cs.Pu, cs.rPu, cs.Pv, cs.rPv, cs.rP, W, psi, yU, yV, yPhi, a, k, j, i);
}

// Reverse of phase B, one thread per column.  Forward (per column):
//   D_k  = (Fl[fE] - Fl[fW]) rdx + (sv_j Ft_j - sv_{j-1} Ft_{j-1}) rdy
//   C    = sum_k ds_k D_k;  dpi/dt = -C
//   W_h  = sh_h C - sum_{k<h} ds_k D_k               (h = 1..K-1)
//   G_k  = rP Phi_k;  c_k = 1 (+ rho_k G_k with the delta kappa Phi/P term)
//   B_k  = G_k c_k;  psi_k = sum_k' H[k][k'] B_k' + R T~_s pi / pi~
//   S_k  = (1/ds_k) sum_k' H[k'][k] ds_k' D_k'  (stored as X),
//   Omega~ tendency -rP c_k S_k
//   (H carries the level coefficient beta of its source level)
template <class T>
__global__ void __launch_bounds__(128) k_adj_column(Geom<T> g, const T* __restrict__ Phi, ColState<T> cs,
                                                    const T* __restrict__ X, const T* __restrict__ yPhi,
                                                    const T* __restrict__ ypi, AdjBufs<T> a) {
  const int I = g.I, J = g.J, K = g.K;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I, i = n - j * I;
  const size_t plane = (size_t)J * I;
  const T rPc = ldg(cs.rP + n);
  const T bP = rPc;  // the level coefficient sits in the H tables
  // C-bar = -ypi + sum_h sh_h Wbar_h
  double Cb = -(double)ldg(ypi + n);
  for (int h = 1; h < K; ++h) Cb += ldg(g.shd + h) * (double)ldg(a.aW + (size_t)h * plane + n);
  // psi: Bbar_k = Hkk psibar_k + h_k sum_{k'<k} psibar_k' (prefix from the top);
  // Omega~: the tendency -rP c_k S_k gives rP-bar -= ybar c' S and, with the
  // delta kappa Phi/P term, G-bar -= ybar rP rho_k S
  const bool nl = g.nl != 0;
  T pre = 0, psum = 0, arp = 0;
  for (int k = 0; k < K; ++k) {
    const T pb = ldg(a.aPsi + (size_t)k * plane + n);
    const T Bb = ldg(g.Hkk + k) * pb + ldg(g.hk + k) * pre;
    pre += pb;
    psum += pb;
    const T ph = ldg(Phi + (size_t)k * plane + n);
    const T Sx = ldg(X + (size_t)k * plane + n), yx = ldg(yPhi + (size_t)k * plane + n);
    if (!nl) {
      a.aPhi[(size_t)k * plane + n] = Bb * bP;
      arp += Bb * ph - yx * Sx;
    } else {
      const T rho = ldg(g.rho + k), G = bP * ph;
      const T dB = T(1) + T(2) * rho * G;      // dB/dG
      const T Gb = Bb * dB - yx * rPc * rho * Sx;  // G-bar from psi and Omega~
      a.aPhi[(size_t)k * plane + n] = Gb * bP;
      arp += Gb * ph - yx * (T(1) + rho * G) * Sx;
    }
  }
  a.arPcol[n] = arp;
  a.aPiD[n] = psum * ldg(g.rt0pit + n);
  // Dbar_k = ds_k (Cb - sum_{h>k} Wbar_h) - bP ds_k (Hkk Xbar_k / ds_k + sum_{k'>k} h_k' Xbar_k' / ds_k')
  const int M = ldg(g.Mu + j);
  const int fE = wrapi(i + (M - 1) / 2, I), fW = wrapi(i - (M + 1) / 2, I);
  // the inputs are read through the read-only path so that the reads of a
  // level need not wait behind the previous level's atomics
  const T rdxj = ldg(g.rdx + j), rdyj = ldg(g.rdy + j);
  const T csS = j < J - 1 ? ldg(g.sv + j) * rdyj : T(0), csN = j > 0 ? ldg(g.sv + j - 1) * rdyj : T(0);
  double SW = 0.0;
  T SX = 0;
  for (int k = K - 1; k >= 0; --k) {
    // Omega~ carries c_k: its D-dependence is that of -rP c_k S_k
    T xb = ldg(yPhi + (size_t)k * plane + n);
    if (nl) xb *= T(1) + ldg(g.rho + k) * bP * ldg(Phi + (size_t)k * plane + n);
    const T ds = ldg(g.ds + k);
    const T Db = (T)(ldg(g.dsd + k) * (Cb - SW)) - bP * (ldg(g.Hkk + k) * xb + ds * SX);
    SX += ldg(g.hk_rds + k) * xb;
    if (k > 0) SW += (double)ldg(a.aW + (size_t)k * plane + n);
    const size_t r3 = (size_t)k * plane + (size_t)j * I;
    aadd(a.aFl + r3 + fE, Db * rdxj);
    aadd(a.aFl + r3 + fW, -Db * rdxj);
    const size_t rv = ((size_t)k * (J - 1) + j) * I;
    if (j < J - 1) aadd(a.aFt + rv + i, Db * csS);
    if (j > 0) aadd(a.aFt + rv - I + i, -Db * csN);
  }
}

// F = P U, G = U / P -> adjoints of U, V, Phi; 2-D adjoints -> adjoint of m.
template <class T>
__global__ void __launch_bounds__(128) k_adj_conv(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                                  const T* __restrict__ Phi, ColState<T> cs, AdjBufs<T> a,
                                                  T* oU, T* oV, T* oPhi, T scale, int accumulate, T* sU, T* sV,
                                                  T* sPhi) {
  // out = (accumulate ? out : 0) + scale * b; when sU is given, also sum += scale * b
  const int I = g.I, J = g.J, K = g.K;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I;
  const size_t plane = (size_t)J * I, vplane = (size_t)(J - 1) * I;
  const bool hasV = j < J - 1;
  const T Puc = cs.Pu[n], rPuc = cs.rPu[n], rPc = cs.rP[n];
  const T Pvc = hasV ? cs.Pv[n] : T(0), rPvc = hasV ? cs.rPv[n] : T(0);
  T aPu = 0, arPu = 0, aPv = 0, arPv = 0, arP = ldg(a.arPcol + n);
  for (int k = 0; k < K; ++k) {
    const size_t o = (size_t)k * plane + n;
    const T Uk = ldg(U + o), Pk = ldg(Phi + o);
    const T bu = ldg(a.aU + o) + ldg(a.aFl + o) * Puc + ldg(a.aGu + o) * rPuc;
    aPu += ldg(a.aFl + o) * Uk + ldg(a.tPu + o);
    arPu += ldg(a.aGu + o) * Uk + ldg(a.tRPu + o);
    const T bp = ldg(a.aPhi + o) + ldg(a.aGs + o) * rPc;
    arP += ldg(a.aGs + o) * Pk + ldg(a.tRP + o);
    oU[o] = (accumulate ? oU[o] : T(0)) + scale * bu;
    oPhi[o] = (accumulate ? oPhi[o] : T(0)) + scale * bp;
    if (sU) {
      sU[o] += scale * bu;
      sPhi[o] += scale * bp;
    }
    if (hasV) {
      const size_t ov = (size_t)k * vplane + n;
      const T Vk = ldg(V + ov);
      const T bv = ldg(a.aV + ov) + ldg(a.aFt + ov) * Pvc + ldg(a.aGv + ov) * rPvc;
      aPv += ldg(a.aFt + ov) * Vk + ldg(a.tPv + ov);
      arPv += ldg(a.aGv + ov) * Vk + ldg(a.tRPv + ov);
      oV[ov] = (accumulate ? oV[ov] : T(0)) + scale * bv;
      if (sU) sV[ov] += scale * bv;
    }
  }
  // P^u = sqrt(m^u): dP^u/dm^u = 1/(2 P^u), d(1/P^u)/dm^u = -1/(2 P^u^3)
  a.mub[n] = aPu * T(0.5) * rPuc - arPu * T(0.5) * rPuc * rPuc * rPuc;
  a.mvb[n] = hasV ? aPv * T(0.5) * rPvc - arPv * T(0.5) * rPvc * rPvc * rPvc : T(0);
  a.mcb[n] = -arP * T(0.5) * rPc * rPc * rPc;
}

// pi-bar = direct psi part + m-bar, with m^u_i = (m_i + m_{i+1})/2 and
// m^v_j = (m_j + m_{j+1})/2 transposed as gathers.
template <class T>
__global__ void __launch_bounds__(256) k_adj_colstate(Geom<T> g, AdjBufs<T> a, T* opi, T scale, int accumulate,
                                                      T* spi) {
  const int I = g.I, J = g.J;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I, i = n - j * I;
  T mb = a.mcb[n] + T(0.5) * (a.mub[n] + a.mub[j * I + wrapi(i - 1, I)]);
  if (j < J - 1) mb += T(0.5) * a.mvb[n];
  if (j > 0) mb += T(0.5) * a.mvb[n - I];
  const T v = a.aPiD[n] + mb;
  opi[n] = (accumulate ? opi[n] : T(0)) + scale * v;
  if (spi) spi[n] += scale * v;
}

}  // namespace agcm
