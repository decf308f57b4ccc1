// agcm_fused.cuh — the production stage kernel: one launch per stage.
//
// One thread owns the column (j, i): the scalar/Phi point (j, i), the U point
// (j, u = i) and, for j < J-1, the V point (j, i).  It streams the levels from
// the surface (k = K-1) to the top (k = 0) and keeps every column quantity in
// registers:
//   * SD  — suffix sum of dsigma*D (Alg. 1 / Alg. 2 turned upside down):
//           the sigma mass flux at the top face of level k is
//           W_k = SD_k - (1 - sh_k) C, with C the column integral;
//           it is carried for the own column, the column to the east (U cell
//           needs W at u and u+1) and the column to the south (V cell).
//   * dS  — suffix sums of the *differences* of the hydrostatic integrand
//           h_k' (b/P) Phi_k' between the two columns that enter each pressure
//           gradient (Eq. 6's pair for U, the j/j+1 pair for V), so psi is
//           never needed away from the thread's own stencil, however wide the
//           leap stride M_j is.
//   * the vertical advection of level k needs level k-1, which is read one
//     iteration later: each level's tendency is completed and written one
//     iteration late.
// The column integral C (dpi/dt = -C) comes from the FP64 vertical means
// Ubar = sum_k dsigma U_k and Vbar of the stage input — C = D(P^u Ubar, P^v Vbar)
// because P does not depend on k — and every stage accumulates Ubar/Vbar of
// its own output for the next stage.  One stage therefore reads x_s and x_n
// and writes x_{s+1}: the 6/9/9 words per grid point of the algorithmic model.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

// Launch shape of the stage kernel: one warp per block covering 32 columns of
// one row (the row index is then warp-uniform, so the row geometry and leap
// strides live in uniform registers), and a register cap from the number of
// resident blocks requested (measured on GB300 at 1440x720x30: 20 one-warp
// blocks per SM, i.e. <= 96 registers, is the fastest FP32 shape; FP64 is
// bound by the FP64 pipe and keeps more registers).
#ifndef AGCM_FUSED_BY
#define AGCM_FUSED_BY 1
#endif
#ifndef AGCM_FUSED_MINB
#define AGCM_FUSED_MINB 20
#endif
#ifndef AGCM_FUSED_MINB64
#define AGCM_FUSED_MINB64 8
#endif
constexpr int kFusedBX = 32, kFusedBY = AGCM_FUSED_BY;

// The work of one thread: the column (j, i) through all levels of one stage.
// MODE 0: out = T(xs) (validation); MODE 1: base = xs (first stage);
// MODE 2: base given (later stages; may alias out).
template <class T, int MODE>
__device__ __forceinline__ void fused_column(
    const Geom<T>& g, const int i, const int j, const T* __restrict__ U, const T* __restrict__ V,
    const T* __restrict__ Phi, const T* __restrict__ pi, const double* __restrict__ Ubar,
    const double* __restrict__ Vbar, const T* Ub, const T* Vb, const T* Phib, const T* pib, T* Uo, T* Vo, T* Phio,
    T* pio, double* __restrict__ Ubar_o, double* __restrict__ Vbar_o, const T cdt) {
  const int I = g.I, J = g.J, K = g.K;
  const bool hasS = j < J - 1;   // V row j exists, scalar row j+1 exists
  const bool hasN = j > 0;       // V row j-1 exists
  const bool hasSS = j + 1 < J - 1;  // V row j+1 exists
  const unsigned plane = (unsigned)J * I, vplane = (unsigned)(J - 1) * I;
  const int rj = j * I, rjm = hasN ? rj - I : rj, rjp = hasS ? rj + I : rj;

  // ---- level-independent indices (leap offsets, Eq. 6 / Table "Communication aggregation")
  const int M = g.Mu[j];
  const int ip = wrapi(i + 1, I), im = wrapi(i - 1, I);
  const int ie = wrapi(i + M, I), iw = wrapi(i - M, I);
  const int fE = wrapi(i + (M - 1) / 2, I), fE1 = wrapi(i + (M + 1) / 2, I);
  const int fW = wrapi(i - (M + 1) / 2, I), fW1 = wrapi(i - (M - 1) / 2, I);
  int Mv = 1, M1 = 1;
  if (hasS) {
    Mv = g.Mv[j];
    M1 = g.Mu[j + 1];
  }
  const int vie = wrapi(i + Mv, I), viw = wrapi(i - Mv, I);
  const int vfE = wrapi(i + (Mv - 1) / 2, I), vfW = wrapi(i - (Mv + 1) / 2, I);
  const int gE = wrapi(i + (M1 - 1) / 2, I), gW = wrapi(i - (M1 + 1) / 2, I);

  // ---- column state a2 from pi (level independent)
  auto mass = [&](int r, int c) { return g.pit[r + c] + pi[r + c]; };
  auto Pu_at = [&](int r, int c) { return sqrt_t(T(0.5) * (mass(r, c) + mass(r, wrapi(c + 1, I)))); };
  auto Pv_at = [&](int r, int c) { return sqrt_t(T(0.5) * (mass(r, c) + mass(r + I, c))); };
  const T one = T(1);
  const T rPc = one / sqrt_t(mass(rj, i));
  const T rPe = one / sqrt_t(mass(rj, ie)), rPw = one / sqrt_t(mass(rj, iw));
  const T rPE1 = one / sqrt_t(mass(rj, fE1)), rPW1 = one / sqrt_t(mass(rj, fW1));
  const T rPs = hasS ? one / sqrt_t(mass(rjp, i)) : T(0);
  const T rPn = hasN ? one / sqrt_t(mass(rjm, i)) : T(0);
  const T Puc = Pu_at(rj, i), rPuc = one / Puc;
  const T rPue = one / Pu_at(rj, ie), rPuw = one / Pu_at(rj, iw);
  const T rPum = one / Pu_at(rj, im);
  const T rPus = hasS ? one / Pu_at(rjp, i) : T(0), rPusm = hasS ? one / Pu_at(rjp, im) : T(0);
  const T rPun = hasN ? one / Pu_at(rjm, i) : T(0);
  const T PufE = Pu_at(rj, fE), PufE1 = Pu_at(rj, fE1), PufW = Pu_at(rj, fW), PufW1 = Pu_at(rj, fW1);
  const T Pvc = hasS ? Pv_at(rj, i) : T(0), Pvp = hasS ? Pv_at(rj, ip) : T(0);
  const T Pvn = hasN ? Pv_at(rjm, i) : T(0), Pvnp = hasN ? Pv_at(rjm, ip) : T(0);
  const T Pvs = hasSS ? Pv_at(rjp, i) : T(0);
  const T rPvc = hasS ? one / Pvc : T(0);
  const T rPve = hasS ? one / Pv_at(rj, vie) : T(0), rPvw = hasS ? one / Pv_at(rj, viw) : T(0);
  const T rPvn = hasN ? one / Pvn : T(0), rPvs = hasSS ? one / Pvs : T(0);
  const T PuvE = hasS ? Pu_at(rj, vfE) : T(0), PuvW = hasS ? Pu_at(rj, vfW) : T(0);
  const T PusvE = hasS ? Pu_at(rjp, vfE) : T(0), PusvW = hasS ? Pu_at(rjp, vfW) : T(0);
  const T PugE = hasS ? Pu_at(rjp, gE) : T(0), PugW = hasS ? Pu_at(rjp, gW) : T(0);
  // R T0 pi / pi~ at the columns of the two pressure-gradient pairs
  const T psE1 = g.rt0pit[rj + fE1] * pi[rj + fE1], psW1 = g.rt0pit[rj + fW1] * pi[rj + fW1];
  const T psc = g.rt0pit[rj + i] * pi[rj + i];
  const T pss = hasS ? g.rt0pit[rjp + i] * pi[rjp + i] : T(0);

  // ---- row geometry
  const T rdx = g.rdx[j], rdy = g.rdy[j], zf = g.zf[j], r2A = g.r2A[j], f0 = g.f0[j], cota = g.cota[j];
  const T svj = hasS ? g.sv[j] : T(0), svjm = hasN ? g.sv[j - 1] : T(0);
  const T yvj = hasS ? g.yv[j] : T(0), yvjm = hasN ? g.yv[j - 1] : T(0);
  const T yvjp = hasSS ? g.yv[j + 1] : T(0), svjp = hasSS ? g.sv[j + 1] : T(0);
  T rdxs = T(0), rdys = T(0), zfv = T(0), r2Av = T(0), cn = T(0), cs = T(0), f0s = T(0), cotas = T(0);
  if (hasS) {
    rdxs = g.rdx[j + 1];
    rdys = g.rdy[j + 1];
    zfv = g.zfv[j];
    r2Av = g.r2Av[j];
    cn = g.cn[j];
    cs = g.cs[j];
    f0s = g.f0[j + 1];
    cotas = g.cota[j + 1];
  }
  const T b = g.b, rady = g.rady;

  // ---- column integrals C (FP64) at the own column, i+1 and j+1
  const double Cc = ((double)PufE * Ubar[rj + fE] - (double)PufW * Ubar[rj + fW]) * (double)rdx +
                    ((hasS ? (double)svj * (double)Pvc * Vbar[rj + i] : 0.0) -
                     (hasN ? (double)svjm * (double)Pvn * Vbar[rjm + i] : 0.0)) * (double)rdy;
  const double Cp = ((double)PufE1 * Ubar[rj + fE1] - (double)PufW1 * Ubar[rj + fW1]) * (double)rdx +
                    ((hasS ? (double)svj * (double)Pvp * Vbar[rj + ip] : 0.0) -
                     (hasN ? (double)svjm * (double)Pvnp * Vbar[rjm + ip] : 0.0)) * (double)rdy;
  double Cs = 0.0;
  if (hasS)
    Cs = ((double)PugE * Ubar[rjp + gE] - (double)PugW * Ubar[rjp + gW]) * (double)rdxs +
         ((hasSS ? (double)svjp * (double)Pvs * Vbar[rjp + i] : 0.0) - (double)svj * (double)Pvc * Vbar[rj + i]) *
             (double)rdys;
  if (MODE == 0)
    pio[rj + i] = (T)(-Cc);
  else {
    const double pb = (MODE == 1) ? (double)pi[rj + i] : (double)pib[rj + i];
    pio[rj + i] = (T)(pb - (double)cdt * Cc);
  }
  const T Cf = (T)Cc, Cpf = (T)Cp, Csf = (T)Cs;

  // ---- carries
  T SD = 0, SDp = 0, SDs = 0;     // suffix sums of dsigma * D
  T dSU = 0, dSV = 0;             // suffix sums of the hydrostatic differences
  T Wb = 0, Wbp = 0, Wbs = 0;     // W at the bottom face of the current level
  T GsB = 0, GuB = 0, GvB = 0;    // G = F/P one level below
  T PPh = 0, PU = 0, PV = 0;      // partial tendencies of the level below
  double ubar = 0.0, vbar = 0.0;  // sum dsigma * out (next stage's C)

  for (int k = K - 1; k >= -1; --k) {
    T Gsc = 0, Guc = 0, Gvc = 0, Wt = 0, Wtp = 0, Wts = 0;
    T nPPh = 0, nPU = 0, nPV = 0;
    if (k >= 0) {
      const T* Uk = U + (size_t)k * plane;
      const T* Phk = Phi + (size_t)k * plane;
      const T* Vk = V + (size_t)k * vplane;
      const T dsk = g.ds[k], Hkk = g.Hkk[k], hk = g.hk[k], hkr = g.hk_rds[k], r2dsk = g.r2ds[k];
      const T onems = T(1.0 - g.shd[k]);
      // loads
      const T Phc = Phk[rj + i], Phe = Phk[rj + ie], Phw = Phk[rj + iw];
      const T PhE1 = Phk[rj + fE1], PhW1 = Phk[rj + fW1];
      const T Phs = hasS ? Phk[rjp + i] : T(0), Phn = hasN ? Phk[rjm + i] : T(0);
      const T Uc = Uk[rj + i], Ue = Uk[rj + ie], Uw = Uk[rj + iw], Um = Uk[rj + im];
      const T UfE = Uk[rj + fE], UfE1 = Uk[rj + fE1], UfW = Uk[rj + fW], UfW1 = Uk[rj + fW1];
      const T Us = hasS ? Uk[rjp + i] : T(0), Un = hasN ? Uk[rjm + i] : T(0);
      T Vc = 0, Vp = 0, Ve = 0, Vw = 0, Vn = 0, Vnp = 0, Vs = 0;
      if (hasS) {
        Vc = Vk[rj + i];
        Vp = Vk[rj + ip];
        Ve = Vk[rj + vie];
        Vw = Vk[rj + viw];
      }
      if (hasN) {
        Vn = Vk[rjm + i];
        Vnp = Vk[rjm + ip];
      }
      if (hasSS) Vs = Vk[rjp + i];
      // mass fluxes
      const T FlE = PufE * UfE, FlE1 = PufE1 * UfE1, FlW = PufW * UfW, FlW1 = PufW1 * UfW1;
      const T Ftc = Pvc * Vc, Ftp = Pvp * Vp, Ftn = Pvn * Vn, Ftnp = Pvnp * Vnp, Fts = Pvs * Vs;
      // leap divergence (a3) at the own column, i+1 and j+1
      const T D = (FlE - FlW) * rdx + (svj * Ftc - svjm * Ftn) * rdy;
      const T Dp = (FlE1 - FlW1) * rdx + (svj * Ftp - svjm * Ftnp) * rdy;
      T Ds = 0;
      if (hasS) Ds = (PugE * Uk[rjp + gE] - PugW * Uk[rjp + gW]) * rdxs + (svjp * Fts - svj * Ftc) * rdys;
      // a4: suffix sums -> W at the top face of level k
      SD += dsk * D;
      SDp += dsk * Dp;
      SDs += dsk * Ds;
      Wt = SD - onems * Cf;
      Wtp = SDp - onems * Cpf;
      Wts = SDs - onems * Csf;

      // ---- Phi cell: advection + Omega~ (a7, Q_k = C - SD_k)
      Gsc = Phc * rPc;
      {
        T hor = zf * (FlE * Phe * rPe - FlW * Phw * rPw);
        if (hasS) hor += yvj * Ftc * Phs * rPs;
        if (hasN) hor -= yvjm * Ftn * Phn * rPn;
        const T X = -(b * rPc) * (Hkk * D + hkr * (Cf - SD));
        nPPh = X - (hor * r2A + Wb * GsB * r2dsk) * rPc;
      }
      // ---- U cell
      Guc = Uc * rPuc;
      {
        const T ZE = zf * T(0.5) * (FlE + FlE1), ZW = zf * T(0.5) * (FlW + FlW1);
        T hor = ZE * Ue * rPue - ZW * Uw * rPuw;
        if (hasS) hor += T(0.5) * yvj * (Ftc + Ftp) * Us * rPus;
        if (hasN) hor -= T(0.5) * yvjm * (Ftn + Ftnp) * Un * rPun;
        const T WuB = T(0.5) * (Wb + Wbp);
        // a5/a6: psi difference over the (x+N, x-N+1) pair
        const T BE1 = b * rPE1 * PhE1, BW1 = b * rPW1 * PhW1;
        const T dpsi = Hkk * (BE1 - BW1) + dSU + (psE1 - psW1);
        dSU += hk * (BE1 - BW1);
        const T pgf = Puc * dpsi * rdx;
        const T fs = f0 + Guc * cota;
        const T vs = Vn + Vnp + Vc + Vp;
        nPU = -(hor * r2A + WuB * GuB * r2dsk) * rPuc - pgf - T(0.25) * fs * vs;
      }
      // ---- V cell
      if (hasS) {
        Gvc = Vc * rPvc;
        const T UvE = Uk[rj + vfE], UvW = Uk[rj + vfW], UsvE = Uk[rjp + vfE], UsvW = Uk[rjp + vfW];
        const T Usm = Uk[rjp + im];
        const T ZE = zfv * T(0.5) * (PuvE * UvE + PusvE * UsvE);
        const T ZW = zfv * T(0.5) * (PuvW * UvW + PusvW * UsvW);
        T hor = ZE * Ve * rPve - ZW * Vw * rPvw;
        if (hasSS) hor += T(0.5) * (yvj * Ftc + yvjp * Fts) * Vs * rPvs;
        if (hasN) hor -= T(0.5) * (yvjm * Ftn + yvj * Ftc) * Vn * rPvn;
        const T WvB = T(0.5) * (Wb + Wbs);
        const T Bs = b * rPs * Phs, Bc = b * rPc * Phc;
        const T dpsi = Hkk * (Bs - Bc) + dSV + (pss - psc);
        dSV += hk * (Bs - Bc);
        const T pgf = Pvc * dpsi * rady;
        const T cor = cn * ((f0 + Um * rPum * cota) * Um + (f0 + Uc * rPuc * cota) * Uc) +
                      cs * ((f0s + Usm * rPusm * cotas) * Usm + (f0s + Us * rPus * cotas) * Us);
        nPV = -(hor * r2Av + WvB * GvB * r2dsk) * rPvc - pgf + cor;
      }
    }
    // ---- complete level k+1 with its top-face vertical term (needs G_k) and write it
    if (k + 1 <= K - 1) {
      const int kk = k + 1;
      const T r2dsk1 = g.r2ds[kk];
      const T TPh = PPh + Wb * Gsc * r2dsk1 * rPc;
      const T TU = PU + T(0.5) * (Wb + Wbp) * Guc * r2dsk1 * rPuc;
      const size_t o = (size_t)kk * plane + rj + i;
      T bPh, bU;
      if (MODE == 0) {
        bPh = T(0);
        bU = T(0);
      } else if (MODE == 1) {
        bPh = Phi[o];
        bU = U[o];
      } else {
        bPh = Phib[o];
        bU = Ub[o];
      }
      const T oPh = bPh + cdt * TPh, oU = bU + cdt * TU;
      Phio[o] = oPh;
      Uo[o] = oU;
      const double dsk1 = g.dsd[kk];
      ubar += dsk1 * (double)oU;
      if (hasS) {
        const T TV = PV + T(0.5) * (Wb + Wbs) * Gvc * r2dsk1 * rPvc;
        const size_t ov = (size_t)kk * vplane + rj + i;
        const T bV = (MODE == 0) ? T(0) : (MODE == 1 ? V[ov] : Vb[ov]);
        const T oV = bV + cdt * TV;
        Vo[ov] = oV;
        vbar += dsk1 * (double)oV;
      }
    }
    PPh = nPPh;
    PU = nPU;
    PV = nPV;
    GsB = Gsc;
    GuB = Guc;
    GvB = Gvc;
    Wb = Wt;
    Wbp = Wtp;
    Wbs = Wts;
  }
  if (Ubar_o) {
    Ubar_o[rj + i] = ubar;
    if (hasS) Vbar_o[rj + i] = vbar;
  }
}

template <class T, int MODE>
__global__ void __launch_bounds__(kFusedBX * kFusedBY, sizeof(T) == 4 ? AGCM_FUSED_MINB : AGCM_FUSED_MINB64)
    k_fused_stage(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ Phi,
                  const T* __restrict__ pi, const double* __restrict__ Ubar, const double* __restrict__ Vbar,
                  const T* Ub, const T* Vb, const T* Phib, const T* pib, T* Uo, T* Vo, T* Phio, T* pio,
                  double* __restrict__ Ubar_o, double* __restrict__ Vbar_o, T cdt) {
  const int i = blockIdx.x * kFusedBX + threadIdx.x;
  const int j = kFusedBY == 1 ? (int)blockIdx.y : (int)(blockIdx.y * kFusedBY + threadIdx.y);
  if (i >= g.I || j >= g.J) return;
  fused_column<T, MODE>(g, i, j, U, V, Phi, pi, Ubar, Vbar, Ub, Vb, Phib, pib, Uo, Vo, Phio, pio, Ubar_o, Vbar_o,
                        cdt);
}

// Vertical means Ubar = sum_k dsigma_k U_k, Vbar likewise (FP64), of a state.
template <class T>
__global__ void __launch_bounds__(256) k_vsum(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                              double* __restrict__ Ubar, double* __restrict__ Vbar) {
  const int I = g.I, J = g.J, K = g.K;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const size_t plane = (size_t)J * I, vplane = (size_t)(J - 1) * I;
  double su = 0.0, sv = 0.0;
  const bool hasV = n < (J - 1) * I;
  for (int k = 0; k < K; ++k) {
    su += g.dsd[k] * (double)U[(size_t)k * plane + n];
    if (hasV) sv += g.dsd[k] * (double)V[(size_t)k * vplane + n];
  }
  Ubar[n] = su;
  if (hasV) Vbar[n] = sv;
}

}  // namespace agcm
