// agcm_fused.cuh — the production stage kernel: a whole stage in one pass over the levels.
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
//           beta_k' h_k' Phi_k' / P (the level coefficient beta of Eq. 1 sits
//           in the tables) between the two columns that enter each pressure
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
//
// A stage is two launches of k_fused_stage, run concurrently on two streams:
// the low-latitude band of rows whose strides M_j (scalar/U row j and row
// j+1, V row j) are all 1 — half of the rows under Eq. 7 — with the column
// body specialised to stride 1 (every leap offset is i or i +- 1, so
// coinciding loads and P factors are one value and the stencil needs 17
// instead of 31 loads per level, with no register spills), and the remaining
// rows with the general body.
#pragma once
#include "agcm_common.cuh"

namespace agcm {

// Launch shape of the stage kernel: one warp per block covering 32 columns of
// one row (the row index is then warp-uniform, so the row geometry and leap
// strides live in uniform registers), and a register cap from the number of
// resident blocks requested (measured on GB300 at 1440x720x30: 20 one-warp
// blocks per SM, i.e. <= 96 registers, is the fastest FP32 shape for the
// general body; FP64 is bound by the FP64 pipe and keeps more registers).
#ifndef AGCM_FUSED_MINB
#define AGCM_FUSED_MINB 20
#endif
// The stride-1 body needs fewer registers: 28 resident blocks (<= 72
// registers) measured fastest for it (0.594 ms per stage against 0.600 at 24
// and 0.627 with the two launches serialised on one stream, 0.653 for the
// general body over all rows).
#ifndef AGCM_FUSED_MINB_L1
#define AGCM_FUSED_MINB_L1 28
#endif
#ifndef AGCM_FUSED_MINB64
#define AGCM_FUSED_MINB64 8
#endif
constexpr int kTileX = 32;  // columns of one warp (one block) of the stage kernel

// The work of one thread: the column (j, i) through all levels of one stage.
// MODE 0: out = T(xs) (validation); MODE 1: base = xs (first stage);
// MODE 2: base given (later stages; may alias out).
// Ubar_b/Vbar_b: vertical means of the base state (FP32 path, MODE > 0): the
// output's means are base + sum_k dsigma_k (out_k - base_k), the increments
// being exact differences of stored floats, so no FP64 work runs per level.
// TERMS selects the term groups of Eq. 2: 1 = advection L (skew flux form,
// vertical advection), 2 = adaptation A (pressure gradient, Coriolis pair,
// Omega~ conversion, dpi/dt), 3 = both (the unsplit step).
// NL: Eq. 1's delta kappa Phi/P term is on; every Phi/P that enters psi or
// the Omega~ coefficient is scaled by 1 + rho_k Phi/P.
template <class T, int MODE, int TERMS = 3, bool NL = false, bool L1 = false>
__device__ __forceinline__ void fused_column(
    const Geom<T>& g, const int i, const int j, const T* __restrict__ U, const T* __restrict__ V,
    const T* __restrict__ Phi, const T* __restrict__ pi, const double* __restrict__ Ubar,
    const double* __restrict__ Vbar, const T* Ub, const T* Vb, const T* Phib, const T* pib, T* Uo, T* Vo, T* Phio,
    T* pio, double* Ubar_o, double* Vbar_o, const double* Ubar_b, const double* Vbar_b, const T cdt) {
  const int I = g.I, J = g.J, K = g.K;
  constexpr bool ADV = (TERMS & 1) != 0, ADA = (TERMS & 2) != 0;
  const bool hasS = L1 || j < J - 1;   // V row j exists, scalar row j+1 exists
  const bool hasN = L1 || j > 0;       // V row j-1 exists
  const bool hasSS = L1 || j + 1 < J - 1;  // V row j+1 exists
  const unsigned plane = (unsigned)J * I, vplane = (unsigned)(J - 1) * I;
  const int rj = j * I, rjm = hasN ? rj - I : rj, rjp = hasS ? rj + I : rj;

  // ---- level-independent indices (leap offsets, Eq. 6 / Table "Communication aggregation")
  // L1: every stride of the stencil is 1 and the row is interior, so the
  // leap offsets are i and i +- 1; the compiler then merges the loads and P
  // factors at coinciding points.  The operations are the same; their
  // contraction into FMAs may differ, so results agree with the general body
  // to rounding, not to the bit
  const int M = L1 ? 1 : g.Mu[j];
  const int ip = wrapi(i + 1, I), im = wrapi(i - 1, I);
  const int ie = L1 ? ip : wrapi(i + M, I), iw = L1 ? im : wrapi(i - M, I);
  const int fE = L1 ? i : wrapi(i + (M - 1) / 2, I), fE1 = L1 ? ip : wrapi(i + (M + 1) / 2, I);
  const int fW = L1 ? im : wrapi(i - (M + 1) / 2, I), fW1 = L1 ? i : wrapi(i - (M - 1) / 2, I);
  int Mv = 1, M1 = 1;
  if (hasS && !L1) {
    Mv = g.Mv[j];
    M1 = g.Mu[j + 1];
  }
  const int vie = L1 ? ip : wrapi(i + Mv, I), viw = L1 ? im : wrapi(i - Mv, I);
  const int vfE = L1 ? i : wrapi(i + (Mv - 1) / 2, I), vfW = L1 ? im : wrapi(i - (Mv + 1) / 2, I);
  const int gE = L1 ? i : wrapi(i + (M1 - 1) / 2, I), gW = L1 ? im : wrapi(i - (M1 + 1) / 2, I);

  // ---- indices of the level loads
  const int lr0 = rj, lrN = rjm, lrS = rjp;
  const int li = i, lie = ie, liw = iw, lfE = fE, lfE1 = fE1, lfW = fW, lfW1 = fW1, lip = ip, lim = im;
  const int lvie = vie, lviw = viw, lvfE = vfE, lvfW = vfW, lgE = gE, lgW = gW;

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
  // R T~_s pi / pi~ at the columns of the two pressure-gradient pairs
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
  const T rady = g.rady;

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
    pio[rj + i] = ADA ? (T)(-Cc) : T(0);
  else {
    const double pb = (MODE == 1) ? (double)pi[rj + i] : (double)pib[rj + i];
    pio[rj + i] = ADA ? (T)(pb - (double)cdt * Cc) : (T)pb;
  }
  const T Cf = (T)Cc, Cpf = (T)Cp, Csf = (T)Cs;

  // ---- carries
  T SD = 0, SDp = 0, SDs = 0;     // suffix sums of dsigma * D
  T dSU = 0, dSV = 0;             // suffix sums of the hydrostatic differences
  T Wb = 0, Wbp = 0, Wbs = 0;     // W at the bottom face of the current level
  T GsB = 0, GuB = 0, GvB = 0;    // G = F/P one level below
  T PPh = 0, PU = 0, PV = 0;      // partial tendencies of the level below
  // vertical means of the output (next stage's C): FP64 sums in the FP64
  // path; base + FP32 sum of increments in the FP32 path
  constexpr bool kInc = sizeof(T) == 4 && MODE != 0;
  double ubar = 0.0, vbar = 0.0;
  T dubar = T(0), dvbar = T(0);

  // software pipeline: the geometry of a level is loaded one iteration before
  // its level is computed, and the base state of a level one iteration before
  // that level is completed and written
  T q_ds = g.ds[K - 1], q_H = g.Hkk[K - 1], q_hk = g.hk[K - 1], q_hr = g.hk_rds[K - 1], q_r2 = g.r2ds[K - 1];
  T q_om = g.oms[K - 1];
  T q_rho = NL ? g.rho[K - 1] : T(0);
  double q_dsd = g.dsd[K - 1];
  T p_r2 = 0, p_ds = 0;   // level below: 1/(2 dsigma), dsigma
  double p_dsd = 0.0;
  T pbU = 0, pbV = 0, pbPh = 0;  // level below: base values
  const size_t o_own = (size_t)rj + i;
  int it = 0;
  for (int k = K - 1; k >= -1; --k, ++it) {
    T Gsc = 0, Guc = 0, Gvc = 0, Wt = 0, Wtp = 0, Wts = 0;
    T nPPh = 0, nPU = 0, nPV = 0;
    T c_r2 = 0, c_ds = 0, nbU = 0, nbV = 0, nbPh = 0;
    double c_dsd = 0.0;
    if (k >= 0) {
      if (MODE == 2) {  // base of this level, used when it is completed next iteration
        nbU = Ub[(size_t)k * plane + o_own];
        nbPh = Phib[(size_t)k * plane + o_own];
        if (hasS) nbV = Vb[(size_t)k * vplane + o_own];
      }
      const T* Uk = U + (size_t)k * plane;
      const T* Phk = Phi + (size_t)k * plane;
      const T* Vk = V + (size_t)k * vplane;
      const T dsk = q_ds, Hkk = q_H, hk = q_hk, hkr = q_hr, r2dsk = q_r2, onems = q_om, rho = q_rho;
      c_r2 = q_r2;
      c_ds = q_ds;
      c_dsd = q_dsd;
      if (k >= 1) {
        q_ds = g.ds[k - 1];
        q_H = g.Hkk[k - 1];
        q_hk = g.hk[k - 1];
        q_hr = g.hk_rds[k - 1];
        q_r2 = g.r2ds[k - 1];
        q_om = g.oms[k - 1];
        if (NL) q_rho = g.rho[k - 1];
        q_dsd = g.dsd[k - 1];
      }
      // loads
      const T Phc = Phk[lr0 + li], Phe = Phk[lr0 + lie], Phw = Phk[lr0 + liw];
      const T PhE1 = Phk[lr0 + lfE1], PhW1 = Phk[lr0 + lfW1];
      const T Phs = hasS ? Phk[lrS + li] : T(0), Phn = hasN ? Phk[lrN + li] : T(0);
      const T Uc = Uk[lr0 + li], Ue = Uk[lr0 + lie], Uw = Uk[lr0 + liw], Um = Uk[lr0 + lim];
      const T UfE = Uk[lr0 + lfE], UfE1 = Uk[lr0 + lfE1], UfW = Uk[lr0 + lfW], UfW1 = Uk[lr0 + lfW1];
      const T Us = hasS ? Uk[lrS + li] : T(0), Un = hasN ? Uk[lrN + li] : T(0);
      T Vc = 0, Vp = 0, Ve = 0, Vw = 0, Vn = 0, Vnp = 0, Vs = 0;
      if (hasS) {
        Vc = Vk[lr0 + li];
        Vp = Vk[lr0 + lip];
        Ve = Vk[lr0 + lvie];
        Vw = Vk[lr0 + lviw];
      }
      if (hasN) {
        Vn = Vk[lrN + li];
        Vnp = Vk[lrN + lip];
      }
      if (hasSS) Vs = Vk[lrS + li];
      if (MODE == 1) {
        nbU = Uc;
        nbPh = Phc;
        nbV = Vc;
      }
      // mass fluxes
      const T FlE = PufE * UfE, FlE1 = PufE1 * UfE1, FlW = PufW * UfW, FlW1 = PufW1 * UfW1;
      const T Ftc = Pvc * Vc, Ftp = Pvp * Vp, Ftn = Pvn * Vn, Ftnp = Pvnp * Vnp, Fts = Pvs * Vs;
      // leap divergence (a3) at the own column, i+1 and j+1
      const T D = (FlE - FlW) * rdx + (svj * Ftc - svjm * Ftn) * rdy;
      const T Dp = (FlE1 - FlW1) * rdx + (svj * Ftp - svjm * Ftnp) * rdy;
      T Ds = 0;
      if (hasS) Ds = (PugE * Uk[lrS + lgE] - PugW * Uk[lrS + lgW]) * rdxs + (svjp * Fts - svj * Ftc) * rdys;
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
        // Omega~ with Eq. 1's coefficient: Hkk, hkr carry beta_k; the
        // delta kappa Phi/P part scales it by 1 + rho_k Phi/P
        const T X = -(NL ? rPc * (one + rho * Gsc) : rPc) * (Hkk * D + hkr * (Cf - SD));
        nPPh = (ADA ? X : T(0)) - (ADV ? (hor * r2A + Wb * GsB * r2dsk) * rPc : T(0));
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
        T BE1 = rPE1 * PhE1, BW1 = rPW1 * PhW1;
        if (NL) {
          BE1 *= one + rho * BE1;
          BW1 *= one + rho * BW1;
        }
        const T dpsi = Hkk * (BE1 - BW1) + dSU + (psE1 - psW1);
        dSU += hk * (BE1 - BW1);
        const T pgf = Puc * dpsi * rdx;
        const T fs = f0 + Guc * cota;
        const T vs = Vn + Vnp + Vc + Vp;
        nPU = (ADV ? -(hor * r2A + WuB * GuB * r2dsk) * rPuc : T(0)) - (ADA ? pgf + T(0.25) * fs * vs : T(0));
      }
      // ---- V cell
      if (hasS) {
        Gvc = Vc * rPvc;
        const T UvE = Uk[lr0 + lvfE], UvW = Uk[lr0 + lvfW], UsvE = Uk[lrS + lvfE], UsvW = Uk[lrS + lvfW];
        const T Usm = Uk[lrS + lim];
        const T ZE = zfv * T(0.5) * (PuvE * UvE + PusvE * UsvE);
        const T ZW = zfv * T(0.5) * (PuvW * UvW + PusvW * UsvW);
        T hor = ZE * Ve * rPve - ZW * Vw * rPvw;
        if (hasSS) hor += T(0.5) * (yvj * Ftc + yvjp * Fts) * Vs * rPvs;
        if (hasN) hor -= T(0.5) * (yvjm * Ftn + yvj * Ftc) * Vn * rPvn;
        const T WvB = T(0.5) * (Wb + Wbs);
        T Bs = rPs * Phs, Bc = Gsc;
        if (NL) {
          Bs *= one + rho * Bs;
          Bc *= one + rho * Bc;
        }
        const T dpsi = Hkk * (Bs - Bc) + dSV + (pss - psc);
        dSV += hk * (Bs - Bc);
        const T pgf = Pvc * dpsi * rady;
        const T cor = cn * ((f0 + Um * rPum * cota) * Um + (f0 + Uc * rPuc * cota) * Uc) +
                      cs * ((f0s + Usm * rPusm * cotas) * Usm + (f0s + Us * rPus * cotas) * Us);
        nPV = (ADV ? -(hor * r2Av + WvB * GvB * r2dsk) * rPvc : T(0)) + (ADA ? cor - pgf : T(0));
      }
    }
    // ---- complete level k+1 with its top-face vertical term (needs G_k) and write it
    if (k + 1 <= K - 1) {
      const int kk = k + 1;
      const T r2dsk1 = p_r2;
      const T TPh = PPh + (ADV ? Wb * Gsc * r2dsk1 * rPc : T(0));
      const T TU = PU + (ADV ? T(0.5) * (Wb + Wbp) * Guc * r2dsk1 * rPuc : T(0));
      const size_t o = (size_t)kk * plane + rj + i;
      const T bPh = MODE == 0 ? T(0) : pbPh, bU = MODE == 0 ? T(0) : pbU;
      const T oPh = bPh + cdt * TPh, oU = bU + cdt * TU;
      Phio[o] = oPh;
      Uo[o] = oU;
      if (kInc) {
        dubar += p_ds * (oU - bU);
      } else {
        ubar += p_dsd * (double)oU;
      }
      if (hasS) {
        const T TV = PV + (ADV ? T(0.5) * (Wb + Wbs) * Gvc * r2dsk1 * rPvc : T(0));
        const size_t ov = (size_t)kk * vplane + rj + i;
        const T bV = MODE == 0 ? T(0) : pbV;
        const T oV = bV + cdt * TV;
        Vo[ov] = oV;
        if (kInc)
          dvbar += p_ds * (oV - bV);
        else
          vbar += p_dsd * (double)oV;
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
    p_r2 = c_r2;
    p_ds = c_ds;
    p_dsd = c_dsd;
    pbU = nbU;
    pbV = nbV;
    pbPh = nbPh;
  }
  if (Ubar_o) {
    if (kInc) {
      ubar = Ubar_b[rj + i] + (double)dubar;
      if (hasS) vbar = Vbar_b[rj + i] + (double)dvbar;
    }
    Ubar_o[rj + i] = ubar;
    if (hasS) Vbar_o[rj + i] = vbar;
  }
}

// One warp per block covering 32 columns of one row, loads from global
// memory (the row index is warp-uniform, so row tables sit in uniform
// registers); PART picks the rows of the launch: 0 every row, 1 the rows
// outside the stride-1 band [l1lo, l1hi), 2 the band, with the stride-1 body,
// 3 the rows g.rowc (those the row-segment kernel leaves).
template <class T, int MODE, int TERMS = 3, bool NL = false, int PART = 0>
__global__ void __launch_bounds__(kTileX, sizeof(T) == 4 ? (PART == 2 ? AGCM_FUSED_MINB_L1 : AGCM_FUSED_MINB)
                                                          : AGCM_FUSED_MINB64)
    k_fused_stage(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ Phi,
                  const T* __restrict__ pi, const double* __restrict__ Ubar, const double* __restrict__ Vbar,
                  const T* Ub, const T* Vb, const T* Phib, const T* pib, T* Uo, T* Vo, T* Phio, T* pio,
                  double* Ubar_o, double* Vbar_o, const double* Ubar_b, const double* Vbar_b, T cdt) {
  const int i = blockIdx.x * kTileX + threadIdx.x;
  int j = blockIdx.y;
  if (PART == 1 && j >= g.l1lo) j += g.l1hi - g.l1lo;
  if (PART == 2) j += g.l1lo;
  if (PART == 3) j = g.rowc[j];
  if (i < g.I)
    fused_column<T, MODE, TERMS, NL, PART == 2>(g, i, j, U, V, Phi, pi, Ubar, Vbar, Ub, Vb, Phib, pib, Uo, Vo, Phio,
                                                pio, Ubar_o, Vbar_o, Ubar_b, Vbar_b, cdt);
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
