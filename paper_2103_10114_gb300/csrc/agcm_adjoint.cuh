// agcm_adjoint.cuh — hand-written adjoint (vector-Jacobian product) of the
// spatial operator T at a state x, in gather form: every element of the
// result is formed by the one thread that owns it, as the sum over the
// tendency terms whose stencil reads it.  No two threads write the same
// element, so there are no atomics and the result does not depend on the
// order in which threads run (bit-identical from run to run).
//
//   k_colstate    (agcm_phases.cuh) phase A at x: m = pi~ + pi, P = sqrt(m) and
//                 its U/V-point values and reciprocals.
//   k_adj_col     32 columns x level groups per block: phase B at x (the
//                 leap divergence D_k of Eq. 6, its column sum C, the sigma
//                 mass flux W_h = sh_h C - sum_{k<h} ds_k D_k of Alg. 1 /
//                 Alg. 2, the Omega~ factor S_k and the hydrostatic psi)
//                 together with its transpose: the adjoints of W and psi
//                 gathered from the tendencies that read them, the
//                 transposed prefix / suffix scans and the adjoint Dbar_k of
//                 D_k.
//   k_adj_rows    one row segment per block, levels in a loop: the adjoints of
//                 the mass fluxes F = P^u U, P^v V, of G = U / P^u, V / P^v,
//                 Phi / P and of U, V through the Coriolis pair, each gathered
//                 from the tendency points that read it (from factors staged
//                 in shared memory), then the chain F = P U, G = F / P back to
//                 U, V, Phi and the level sums of the adjoints of the 2-D
//                 factors.  k_adj_gather does the same through L1 for the rows
//                 whose strides reach past a row segment's halo.
//   k_adj_colstate  m^u, m^v are stride-1 means of m: the adjoint of pi.
//
// The transposed stencil.  Every advection term is a face flux Z times the
// value G at the far end of a pair of points (x, x + M):  the tendency at x
// holds + Z G(x + M) and the tendency at x + M holds - Z G(x), both with the
// same face flux (Z at x + M/2; the skew form of the advection).  With
// hb(x) = dT(x) / d(hor)(x) * ybar(x) the adjoint of the face flux is
// hb(x) G(x + M) - hb(x + M) G(x), and the adjoint of G(x) is
// hb(x - M) Z(x - M/2) - hb(x + M) Z(x + M/2): the leap offsets of the
// forward stencil mirrored.  A face flux is a mean of one or two mass fluxes
// F, so F's adjoint sums the adjoints of the faces that average it.  The same
// holds meridionally (pairs of rows j, j + 1) and vertically (levels k, k + 1,
// face flux W).  The Coriolis pair and the pressure gradient are read at
// fixed neighbours and transposed the same way.
//
// Output: out = (accumulate ? out : 0) + scale * J(x)^T ybar, and optionally
// sum += scale * J(x)^T ybar in the same pass (the stage accumulation).
#pragma once
#include "agcm_common.cuh"
#include "agcm_phases.cuh"

namespace agcm {

// Outputs of k_adj_col (the inputs of the gather kernels).
template <class T>
struct AdjCol {
  T* W;      // (K+1)*J*I: the sigma mass flux at the half levels h = 1..K-1
  T* psi;    // K*J*I: hydrostatic psi
  T* Db;     // K*J*I: adjoint of the divergence D_k
  T* aPhi;   // K*J*I: adjoint of Phi through psi and the Omega~ term
  T* arP;    // J*I: adjoint of 1/P through the Omega~ term
  T* aPiD;   // J*I: adjoint of pi through the surface term of psi
};

// Phase B and its transpose.  Forward (per column):
//   D_k  = (F^u[i+(M-1)/2] - F^u[i-(M+1)/2]) rdx + (sv_j F^v_j - sv_{j-1} F^v_{j-1}) rdy
//   C    = sum_k ds_k D_k;  dpi/dt = -C
//   W_h  = sh_h C - sum_{k<h} ds_k D_k  =  sum_{k>=h} ds_k D_k - (1 - sh_h) C
//   G_k  = Phi_k / P;  c_k = 1 (+ rho_k G_k with the delta kappa Phi/P term)
//   B_k  = G_k c_k;  psi_k = Hkk_k B_k + sum_{k'>k} hk_k' B_k' + R T~_s pi / pi~
//   S_k  = Hkk_k D_k + hk_k / ds_k sum_{k'<k} ds_k' D_k';  Omega~ tendency -c_k S_k / P
//   (H carries the level coefficient beta of its source level)
// Transposed: the adjoint of psi_k (gathered from the pressure-gradient terms
// of the U and V points that read it) runs a prefix scan to the adjoint of
// B_k, hence of Phi_k and 1/P; the adjoint of W_h (gathered from the
// vertical advection of the levels h-1, h at the points whose face means hold
// W(j, i)) and of -C give Cbar and the suffix sums that form Dbar_k.
//
// Both forms below hold 32 columns per block and split each column's levels
// into groups (threadIdx.y): walk 1 forms a group's partial sums, the block
// exchanges them through shared memory (every sum in group order, so the
// result is the same on every run), and walk 2 forms each level's outputs
// with the prefix and suffix offsets of the other groups.  The sums run in
// the state's precision: FP64 issues at 1/64 of the FP32 rate on this GPU,
// and per level and column they would be the bulk of the pass.
//   k_adj_col    groups of at most kColL levels (K <= 8 kColL): walk 1
//                keeps each level's values in shared memory for walk 2;
//   k_adj_col_w  any K, kColG groups: walk 2 re-forms each level (its loads
//                hit L1).
#ifndef AGCM_COLL
#define AGCM_COLL 8
#endif
constexpr int kColL = AGCM_COLL;
#ifndef AGCM_COLG
#define AGCM_COLG 2
#endif
constexpr int kColG = AGCM_COLG;

// The per-column pieces shared by the two forms.  ST: the level tables are
// read from a copy in shared memory (8 values per level: ds, Hkk, hk, hk_rds,
// r2ds, 1 - sh, rho), else from the grid's tables in global memory.
enum { kLds, kLHkk, kLhk, kLhkr, kLr2ds, kLoms, kLrho, kLN = 8 };
template <class T>
__device__ __forceinline__ void col_tables(const Geom<T>& g, T* lt, int tid, int nthreads) {
  for (int k = tid; k < g.K; k += nthreads) {
    T* L = lt + kLN * k;
    L[kLds] = g.ds[k];
    L[kLHkk] = g.Hkk[k];
    L[kLhk] = g.hk[k];
    L[kLhkr] = g.hk_rds[k];
    L[kLr2ds] = g.r2ds[k];
    L[kLoms] = g.oms[k];
    L[kLrho] = g.nl ? g.rho[k] : T(0);
    L[7] = T(0);
  }
}
template <class T, bool ST>
struct ColCtx {
  const Geom<T>& g;
  const T* lt = nullptr;  // shared-memory level tables (ST)
  const T *U, *V, *Phi, *yU, *yV, *yPhi;
  // element offsets fit 32 bits: nlon * nlat * nlev <= 4e9
  unsigned plane, vplane, r2;
  int ic, ue, uw, im;
  bool hasS, hasN, nl;
  T rdx, rdy, rady, svS, svN, Pue, Puw, rPc, rPui, rPum, PvS, PvN, rPvS, rPvN;

  __device__ T tab(int k, int f) const {
    if constexpr (ST) {
      return lt[kLN * k + f];
    } else {
      const T* p = f == kLds ? g.ds : f == kLHkk ? g.Hkk : f == kLhk ? g.hk : f == kLhkr ? g.hk_rds
                 : f == kLr2ds ? g.r2ds : f == kLoms ? g.oms : g.rho;
      return ldg(p + k);
    }
  }
  __device__ ColCtx(const Geom<T>& g_, const T* lt_, const T* U_, const T* V_, const T* Phi_,
                    const ColState<T>& cs, const T* yU_, const T* yV_, const T* yPhi_, int i, int j)
      : g(g_), lt(lt_), U(U_), V(V_), Phi(Phi_), yU(yU_), yV(yV_), yPhi(yPhi_) {
    const int I = g.I, J = g.J;
    plane = (unsigned)J * (unsigned)I;
    vplane = (unsigned)(J - 1) * (unsigned)I;
    r2 = (unsigned)j * (unsigned)I;
    ic = i;
    hasS = j < J - 1;
    hasN = j > 0;
    nl = g.nl != 0;
    const int M = ldg(g.Mu + j);
    ue = wrapi(ic + (M - 1) / 2, I);
    uw = wrapi(ic - (M + 1) / 2, I);
    im = wrapi(ic - 1, I);
    rdx = ldg(g.rdx + j);
    rdy = ldg(g.rdy + j);
    rady = g.rady;
    svS = hasS ? ldg(g.sv + j) : T(0);
    svN = hasN ? ldg(g.sv + j - 1) : T(0);
    const unsigned n = r2 + ic;
    Pue = ldg(cs.Pu + r2 + ue);
    Puw = ldg(cs.Pu + r2 + uw);
    rPc = ldg(cs.rP + n);
    rPui = ldg(cs.rPu + n);
    rPum = ldg(cs.rPu + r2 + im);
    PvS = hasS ? ldg(cs.Pv + n) : T(0);
    PvN = hasN ? ldg(cs.Pv + n - I) : T(0);
    rPvS = hasS ? ldg(cs.rPv + n) : T(0);
    rPvN = hasN ? ldg(cs.rPv + n - I) : T(0);
  }
  // an L2 prefetch of the rows a level reads (no registers held: the level
  // is loaded one level later)
  __device__ void prefetch(int k) const {
    const unsigned o3 = (unsigned)k * plane + r2 + ic, ov = (unsigned)k * vplane + r2 + ic;
    const int I = g.I;
    auto pf = [](const T* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); };
    pf(U + o3);
    pf(yU + o3);
    pf(Phi + o3);
    pf(yPhi + o3);
    if (hasS) {
      pf(V + ov);
      pf(yV + ov);
    }
    if (hasN) {
      pf(V + ov - I);
      pf(yV + ov - I);
    }
  }
  // the values of one level: D, the adjoint of psi, Phi, ybar_Phi and the
  // products y / P, x / P of the five points whose vertical advection holds
  // W(j, i): Phi (j, i), U (j, i-1), U (j, i), V (j-1, i), V (j, i)
  struct Lev {
    T D, pb, ph, yx, q[5], x[5];
  };
  __device__ void level(int k, Lev& v) const {
    const int I = g.I;
    const unsigned o3 = (unsigned)k * plane + r2, ov = (unsigned)k * vplane + r2;
    const T* u = U + o3;
    const T* yu = yU + o3;
    const T* vv = V + ov;
    const T* yvv = yV + ov;
    const T VS = hasS ? ldg(vv + ic) : T(0), VN = hasN ? ldg(vv - I + ic) : T(0);
    const T yVS = hasS ? ldg(yvv + ic) : T(0), yVN = hasN ? ldg(yvv - I + ic) : T(0);
    v.D = (Pue * ldg(u + ue) - Puw * ldg(u + uw)) * rdx + (svS * PvS * VS - svN * PvN * VN) * rdy;
    // the pressure-gradient terms of the U points i - (M+1)/2, i + (M-1)/2
    // and the V points (j-1, i), (j, i) read psi(j, i)
    v.pb = rdx * (ldg(yu + ue) * Pue - ldg(yu + uw) * Puw) + rady * (yVS * PvS - yVN * PvN);
    v.ph = ldg(Phi + o3 + ic);
    v.yx = ldg(yPhi + o3 + ic);
    v.q[0] = v.yx * rPc;
    v.x[0] = v.ph * rPc;
    v.q[1] = ldg(yu + im) * rPum;
    v.x[1] = ldg(u + im) * rPum;
    v.q[2] = ldg(yu + ic) * rPui;
    v.x[2] = ldg(u + ic) * rPui;
    v.q[3] = yVN * rPvN;
    v.x[3] = VN * rPvN;
    v.q[4] = yVS * rPvS;
    v.x[4] = VS * rPvS;
  }
  // adjoint of W_k: vb(k-1) G(k) - vb(k) G(k-1) at the five points,
  // vb = -y r2ds / P (the U and V points hold W(j, i) in a face mean, weight 1/2)
  __device__ T adj_w(int k, const Lev& c, const Lev& p) const {
    const T r = tab(k, kLr2ds), rm = tab(k - 1, kLr2ds);
    const T aw = r * c.q[0] * p.x[0] - rm * p.q[0] * c.x[0];
    T h = 0;
#pragma unroll
    for (int q = 1; q < 5; ++q) h += r * c.q[q] * p.x[q] - rm * p.q[q] * c.x[q];
    return aw + T(0.5) * h;
  }
  __device__ T Bk(int k, T ph) const {
    T B = rPc * ph;
    if (nl) B *= T(1) + tab(k, kLrho) * B;
    return B;
  }
  // Omega~ carries c_k: its D-dependence is that of -c_k S_k / P
  __device__ T xbk(int k, T ph, T yx) const { return nl ? yx * (T(1) + tab(k, kLrho) * rPc * ph) : yx; }
  // the prefix quantities of level k: the adjoint of Phi, and arp += the
  // adjoint of 1/P (Q, pre: the prefix sums before level k)
  __device__ T adj_phi(int k, T D, T pb, T ph, T yx, T Q, T pre, T& arp) const {
    const T Hkk = tab(k, kLHkk);
    const T Sk = Hkk * D + tab(k, kLhkr) * Q;
    const T Bb = Hkk * pb + tab(k, kLhk) * pre;
    if (!nl) {
      arp += Bb * ph - yx * Sk;
      return Bb * rPc;
    }
    const T rho = tab(k, kLrho), G = rPc * ph;
    const T Gb = Bb * (T(1) + T(2) * rho * G) - yx * rPc * rho * Sk;  // dB/dG = 1 + 2 rho G
    arp += Gb * ph - yx * (T(1) + rho * G) * Sk;
    return Gb * rPc;
  }
};

__device__ __forceinline__ int gy_off(int gy, int lane) { return gy * 32 + lane; }

// Group sums of one column: sum ds D, sum pb, sum sh aW, sum aW, sum hk B, sum hk_rds xb.
template <class T>
struct ColSums {
  T Q, pre, C, Cb, psum, Rs, Ss, SXs, SWs;
};
template <class T>
__device__ __forceinline__ ColSums<T> col_exchange(T* red, int G, int gy, int lane, const T s[6]) {
  // red: [6][G][32]
#pragma unroll
  for (int q = 0; q < 6; ++q) red[(q * G + gy) * 32 + lane] = s[q];
  __syncthreads();
  ColSums<T> r{};
  for (int q = 0; q < G; ++q) {
    const T d = red[(0 * G + q) * 32 + lane], p = red[(1 * G + q) * 32 + lane];
    r.C += d;
    r.Cb += red[(2 * G + q) * 32 + lane];
    r.psum += p;
    if (q < gy) {
      r.Q += d;
      r.pre += p;
    } else if (q > gy) {
      r.Rs += d;
      r.SWs += red[(3 * G + q) * 32 + lane];
      r.Ss += red[(4 * G + q) * 32 + lane];
      r.SXs += red[(5 * G + q) * 32 + lane];
    }
  }
  return r;
}

// The suffix quantities of level k: W_k, psi_k, Dbar_k.  q*: this group's
// sums up to level k (qD before it, the others including it), s*: this
// group's totals, r: the other groups' offsets.
template <class T, bool ST>
__device__ __forceinline__ void col_suffix(const ColCtx<T, ST>& c, const AdjCol<T>& o, int k, unsigned q3, T D, T B,
                                           T xb, T qD, T qB, T qX, T qA, T sD, T sB, T sX, T sA,
                                           const ColSums<T>& r, T ps) {
  const T ds = c.tab(k, kLds), Hkk = c.tab(k, kLHkk);
  if (k > 0) o.W[q3] = r.Rs + (sD - qD) - c.tab(k, kLoms) * r.C;  // sum_{k' >= k} ds D - (1 - sh_k) C
  o.psi[q3] = Hkk * B + (r.Ss + (sB - qB)) + ps;
  const T SW = r.SWs + (sA - qA), SX = r.SXs + (sX - qX);
  o.Db[q3] = ds * (r.Cb - SW) - c.rPc * (Hkk * xb + ds * SX);
}

// Four 256-thread blocks per SM (64 registers; the FP64 form keeps two):
// at 720 x 360 x 30 FP32 0.124 ms against 0.159 ms for two blocks (106
// registers), the pass being bound by load latency.
#ifndef AGCM_COLB
#define AGCM_COLB 4
#endif
#ifndef AGCM_COLU
#define AGCM_COLU 8
#endif
constexpr int kColU = AGCM_COLU;
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? AGCM_COLB : 2) k_adj_col(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                                 const T* __restrict__ Phi, const T* __restrict__ pi, ColState<T> cs,
                                                 const T* __restrict__ yU, const T* __restrict__ yV,
                                                 const T* __restrict__ yPhi, const T* __restrict__ ypi,
                                                 AdjCol<T> o) {
  extern __shared__ __align__(16) unsigned char col_smem[];
  T* const red = reinterpret_cast<T*>(col_smem);  // [7][G][32]: group sums, then arp
  const int I = g.I, K = g.K, G = blockDim.y;
  // each level's D, psi adjoint, Phi, ybar_Phi and W adjoint: [5][kColL][G][32];
  // then the level tables [K][8]
  T* const lv = red + 7 * G * 32 + gy_off(threadIdx.y, threadIdx.x);
  T* const lt = red + (7 + 5 * kColL) * G * 32;
  const int lstride = G * 32;
  const int lane = threadIdx.x, gy = threadIdx.y;
  const int i = blockIdx.x * 32 + lane, j = blockIdx.y;
  const bool col = i < I;
  col_tables(g, lt, gy * 32 + lane, G * 32);
  __syncthreads();
  const ColCtx<T, true> c(g, lt, U, V, Phi, cs, yU, yV, yPhi, col ? i : 0, j);
  const int kb = min(K, gy * kColL), ke = min(K, kb + kColL);
  const unsigned n = c.r2 + c.ic;
  // ---- walk 1: every level's values into shared memory, and the group sums
  auto vD = [&](int l) -> T& { return lv[(0 * kColL + l) * lstride]; };
  auto vP = [&](int l) -> T& { return lv[(1 * kColL + l) * lstride]; };
  auto vPh = [&](int l) -> T& { return lv[(2 * kColL + l) * lstride]; };
  auto vY = [&](int l) -> T& { return lv[(3 * kColL + l) * lstride]; };
  auto vA = [&](int l) -> T& { return lv[(4 * kColL + l) * lstride]; };
  T s[6] = {0, 0, 0, 0, 0, 0};
  typename ColCtx<T, true>::Lev cv{}, pv{};
  if (kb > 0 && kb < ke) c.level(kb - 1, pv);
#pragma unroll kColU
  for (int l = 0; l < kColL; ++l) {
    const int k = kb + l;
    if (k < ke) {
      if (k + 1 < ke) c.prefetch(k + 1);
      c.level(k, cv);
      const T aw = k > 0 ? c.adj_w(k, cv, pv) : T(0);
      vD(l) = cv.D;
      vP(l) = cv.pb;
      vPh(l) = cv.ph;
      vY(l) = cv.yx;
      vA(l) = aw;
      s[0] += c.tab(k, kLds) * cv.D;
      s[1] += cv.pb;
      s[2] += (T(1) - c.tab(k, kLoms)) * aw;  // sh_k aW_k (aW = 0 at k = 0)
      s[3] += aw;
      s[4] += c.tab(k, kLhk) * c.Bk(k, cv.ph);
      s[5] += c.tab(k, kLhkr) * c.xbk(k, cv.ph, cv.yx);
      pv = cv;
    }
  }
  ColSums<T> r = col_exchange(red, G, gy, lane, s);
  // ---- walk 2: the outputs of every level, from shared memory (each thread
  // reads back only what it wrote)
  T arp = 0;
  if (col && kb < ke) {
    r.Cb -= ldg(ypi + n);
    const T ps = ldg(g.rt0pit + n) * ldg(pi + n);
    T qD = 0, qB = 0, qX = 0, qA = 0, Q = r.Q, pre = r.pre;
#pragma unroll kColU
    for (int l = 0; l < kColL; ++l) {
      const int k = kb + l;
      if (k < ke) {
        const unsigned q3 = (unsigned)k * c.plane + n;
        const T D = vD(l), pb = vP(l), ph = vPh(l), yx = vY(l);
        o.aPhi[q3] = c.adj_phi(k, D, pb, ph, yx, Q, pre, arp);
        const T dsk = c.tab(k, kLds);
        Q += dsk * D;
        pre += pb;
        const T B = c.Bk(k, ph), xb = c.xbk(k, ph, yx);
        const T qD0 = qD;
        qD += dsk * D;
        qB += c.tab(k, kLhk) * B;
        qX += c.tab(k, kLhkr) * xb;
        qA += vA(l);
        col_suffix(c, o, k, q3, D, B, xb, qD0, qB, qX, qA, s[0], s[4], s[5], s[3], r, ps);
      }
    }
  }
  T* const rarp = red + 6 * G * 32;
  rarp[gy * 32 + lane] = arp;
  __syncthreads();
  if (gy == 0 && col) {
    T a = 0;
    for (int q = 0; q < G; ++q) a += rarp[q * 32 + lane];
    o.arP[n] = a;
    o.aPiD[n] = r.psum * ldg(g.rt0pit + n);
  }
}

// Any K: kColG groups of L = ceil(K / kColG) levels; walk 2 re-forms each level.
template <class T>
__global__ void __launch_bounds__(32 * kColG) k_adj_col_w(Geom<T> g, const T* __restrict__ U, const T* __restrict__ V,
                                                          const T* __restrict__ Phi, const T* __restrict__ pi,
                                                          ColState<T> cs, const T* __restrict__ yU,
                                                          const T* __restrict__ yV, const T* __restrict__ yPhi,
                                                          const T* __restrict__ ypi, AdjCol<T> o) {
  __shared__ T red[7 * kColG * 32];
  const int I = g.I, K = g.K;
  const int lane = threadIdx.x, gy = threadIdx.y;
  const int i = blockIdx.x * 32 + lane, j = blockIdx.y;
  const bool col = i < I;
  const ColCtx<T, false> c(g, nullptr, U, V, Phi, cs, yU, yV, yPhi, col ? i : 0, j);
  const int L = (K + kColG - 1) / kColG;
  const int kb = min(K, gy * L), ke = min(K, kb + L);
  const unsigned n = c.r2 + c.ic;
  T s[6] = {0, 0, 0, 0, 0, 0};
  typename ColCtx<T, false>::Lev cv{}, pv{};
  if (kb < ke) {
    if (kb > 0) c.level(kb - 1, pv);
    for (int k = kb; k < ke; ++k) {
      c.level(k, cv);
      const T aw = k > 0 ? c.adj_w(k, cv, pv) : T(0);
      s[0] += ldg(g.ds + k) * cv.D;
      s[1] += cv.pb;
      s[2] += (T(1) - ldg(g.oms + k)) * aw;
      s[3] += aw;
      s[4] += ldg(g.hk + k) * c.Bk(k, cv.ph);
      s[5] += ldg(g.hk_rds + k) * c.xbk(k, cv.ph, cv.yx);
      pv = cv;
    }
  }
  ColSums<T> r = col_exchange(red, kColG, gy, lane, s);
  T arp = 0;
  if (col && kb < ke) {
    r.Cb -= ldg(ypi + n);
    const T ps = ldg(g.rt0pit + n) * ldg(pi + n);
    T qD = 0, qB = 0, qX = 0, qA = 0, Q = r.Q, pre = r.pre;
    if (kb > 0) c.level(kb - 1, pv);
    for (int k = kb; k < ke; ++k) {
      c.level(k, cv);
      const unsigned q3 = (unsigned)k * c.plane + n;
      o.aPhi[q3] = c.adj_phi(k, cv.D, cv.pb, cv.ph, cv.yx, Q, pre, arp);
      Q += ldg(g.ds + k) * cv.D;
      pre += cv.pb;
      const T B = c.Bk(k, cv.ph), xb = c.xbk(k, cv.ph, cv.yx);
      const T qD0 = qD;
      qD += ldg(g.ds + k) * cv.D;
      qB += ldg(g.hk + k) * B;
      qX += ldg(g.hk_rds + k) * xb;
      if (k > 0) qA += c.adj_w(k, cv, pv);
      col_suffix(c, o, k, q3, cv.D, B, xb, qD0, qB, qX, qA, s[0], s[4], s[5], s[3], r, ps);
      pv = cv;
    }
  }
  T* const rarp = red + 6 * kColG * 32;
  rarp[gy * 32 + lane] = arp;
  __syncthreads();
  if (gy == 0 && col) {
    T a = 0;
    for (int q = 0; q < kColG; ++q) a += rarp[q * 32 + lane];
    o.arP[n] = a;
    o.aPiD[n] = r.psum * ldg(g.rt0pit + n);
  }
}

// Output of the adjoint product and the optional stage accumulation.
template <class T>
struct AdjOut {
  T *oU, *oV, *oPhi, *opi;  // out = (accumulate ? out : 0) + scale * J^T ybar
  T *sU, *sV, *sPhi, *spi;  // sum = sum_in + scale * J^T ybar (when sU != nullptr)
  const T *rU, *rV, *rPhi, *rpi;  // sum_in: the sum itself, or another array
  T scale;
  int accumulate;
};

// Adjoints of the 2-D factors, summed over the levels by k_adj_gather.
template <class T>
struct AdjM {
  T *mub, *mvb, *mcb;
};

constexpr int kAdjTileX = 32, kAdjTileY = 4;

// An empty asm that the compiler must assume changes p: loads through the
// result cannot be hoisted out of the loop that calls it.
template <class P>
__device__ __forceinline__ P* opaque(P* p) {
  asm volatile("" : "+l"(p));
  return p;
}

// The gathered adjoint of one column (j, i) at the levels of one chunk of
// kAdjLevChunk levels (blockIdx.z): the U point (j, i), the Phi point (j, i)
// and, for j < J-1, the V point (j, i).  Each neighbour value is read through
// L1.  This is the general form for any stride; k_adj_rows below takes the
// rows whose strides are small, and this kernel the nrows rows in `rows`.
// The level sums of the 2-D factors' adjoints are written per chunk to
// part[3][nchunks][nrows][I] and added in chunk order by k_adj_fold.
constexpr int kAdjLevChunk = 4;
// Offsets in row j (stride M = Mu_j):  a0 = i - (M-1)/2, b0 = i + (M+1)/2 =
// a0 + M (the pair whose face flux is F^u(i) for a Phi point, one of the two
// for a U point), a1 = i - (M+1)/2, b1 = i + (M-1)/2 = a1 + M (the other U
// pair), iW = i - M, iE = i + M.
template <class T>
__global__ void __launch_bounds__(kAdjTileX* kAdjTileY, 4) k_adj_gather(
    Geom<T> g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ Phi, ColState<T> cs,
    const T* __restrict__ W, const T* __restrict__ psi, const T* __restrict__ Db, const T* __restrict__ aPhi,
    const T* __restrict__ arPcol, const T* __restrict__ yU, const T* __restrict__ yV, const T* __restrict__ yPhi,
    const int* __restrict__ rows, int nrows, T* __restrict__ part, AdjOut<T> o) {
  const int I = g.I, J = g.J, K = g.K;
  const int i = blockIdx.x * kAdjTileX + (int)(threadIdx.x % kAdjTileX);
  const int jq = blockIdx.y * kAdjTileY + (int)(threadIdx.x / kAdjTileX);
  if (i >= I || jq >= nrows) return;
  const int j = ldg(rows + jq);
  const int kb = blockIdx.z * kAdjLevChunk, ke = min(K, kb + kAdjLevChunk);
  const size_t plane = (size_t)J * I, vplane = (size_t)(J - 1) * I;
  const bool hasS = j < J - 1, hasN = j > 0, hasSS = j + 1 < J - 1;
  const int M = ldg(g.Mu + j);
  const int a0 = wrapi(i - (M - 1) / 2, I), b0 = wrapi(i + (M + 1) / 2, I);
  const int a1 = wrapi(i - (M + 1) / 2, I), b1 = wrapi(i + (M - 1) / 2, I);
  const int iE = wrapi(i + M, I), iW = wrapi(i - M, I), ip = wrapi(i + 1, I), im = wrapi(i - 1, I);
  const T zf = ldg(g.zf + j), r2A = ldg(g.r2A + j), rdx = ldg(g.rdx + j), f0 = ldg(g.f0 + j),
          cota = ldg(g.cota + j);
  const T r2AN = hasN ? ldg(g.r2A + j - 1) : T(0), r2AS = hasS ? ldg(g.r2A + j + 1) : T(0);
  const T yvS = hasS ? ldg(g.yv + j) : T(0), yvN = hasN ? ldg(g.yv + j - 1) : T(0),
          yvSS = hasSS ? ldg(g.yv + j + 1) : T(0);
  const T cnS = hasS ? ldg(g.cn + j) : T(0), csN = hasN ? ldg(g.cs + j - 1) : T(0);
  // V row j (stride Mv_j) and V row j-1 (stride Mv_{j-1})
  int cS = i, dS = i, vE = i, vW = i, fEv = i, fWv = i, cN = i, dN = i;
  T zfvS = 0, r2AvS = 0, r2AvSS = 0, r2AvN = 0, zfvN = 0, svS = 0, rdyS = 0, rdyS1 = 0, f0S = 0, cotaS = 0;
  if (hasS) {
    const int Mv = ldg(g.Mv + j);
    cS = wrapi(i - (Mv - 1) / 2, I);
    dS = wrapi(i + (Mv + 1) / 2, I);
    vE = wrapi(i + Mv, I);
    vW = wrapi(i - Mv, I);
    fEv = wrapi(i + (Mv - 1) / 2, I);
    fWv = wrapi(i - (Mv + 1) / 2, I);
    zfvS = ldg(g.zfv + j);
    r2AvS = ldg(g.r2Av + j);
    svS = ldg(g.sv + j);
    rdyS = ldg(g.rdy + j);
    rdyS1 = ldg(g.rdy + j + 1);
    f0S = ldg(g.f0 + j + 1);
    cotaS = ldg(g.cota + j + 1);
    if (hasSS) r2AvSS = ldg(g.r2Av + j + 1);
  }
  if (hasN) {
    const int Mv = ldg(g.Mv + j - 1);
    cN = wrapi(i - (Mv - 1) / 2, I);
    dN = wrapi(i + (Mv + 1) / 2, I);
    zfvN = ldg(g.zfv + j - 1);
    r2AvN = ldg(g.r2Av + j - 1);
  }
  const T rady = g.rady;
  const size_t r2 = (size_t)j * I, r2n = r2 - I, r2s = r2 + I;
  const T rPc = ldg(cs.rP + r2 + i), rPuc = ldg(cs.rPu + r2 + i), Puc = ldg(cs.Pu + r2 + i);
  const T rPvc = hasS ? ldg(cs.rPv + r2 + i) : T(0), Pvc = hasS ? ldg(cs.Pv + r2 + i) : T(0);
  // pointwise factors: hb = -ybar r2A / P (horizontal), G = x / P, F = P x
  auto hbP = [&](size_t r3x, size_t r2x, T r2Ax, int ii) { return -ldg(yPhi + r3x + ii) * r2Ax * ldg(cs.rP + r2x + ii); };
  auto hbU = [&](size_t r3x, size_t r2x, T r2Ax, int ii) { return -ldg(yU + r3x + ii) * r2Ax * ldg(cs.rPu + r2x + ii); };
  auto hbV = [&](size_t rvx, size_t r2x, T r2Ax, int ii) { return -ldg(yV + rvx + ii) * r2Ax * ldg(cs.rPv + r2x + ii); };
  auto Gs = [&](size_t r3x, size_t r2x, int ii) { return ldg(Phi + r3x + ii) * ldg(cs.rP + r2x + ii); };
  auto Gu = [&](size_t r3x, size_t r2x, int ii) { return ldg(U + r3x + ii) * ldg(cs.rPu + r2x + ii); };
  auto Gv = [&](size_t rvx, size_t r2x, int ii) { return ldg(V + rvx + ii) * ldg(cs.rPv + r2x + ii); };
  auto Fl = [&](size_t r3x, size_t r2x, int ii) { return ldg(cs.Pu + r2x + ii) * ldg(U + r3x + ii); };
  auto Ft = [&](size_t rvx, size_t r2x, int ii) { return ldg(cs.Pv + r2x + ii) * ldg(V + rvx + ii); };
  T aPu = 0, arPu = 0, aPv = 0, arPv = 0, arP = blockIdx.z == 0 ? ldg(arPcol + r2 + i) : T(0);
  for (int k = kb; k < ke; ++k) {
    // the 2-D factors are re-read at every level (L1 hits) rather than held
    // in registers across the loop: the pointers are made opaque per level
    cs.rP = opaque(cs.rP);
    cs.rPu = opaque(cs.rPu);
    cs.Pu = opaque(cs.Pu);
    cs.rPv = opaque(cs.rPv);
    cs.Pv = opaque(cs.Pv);
    const size_t r3 = (size_t)k * plane + r2, r3n = r3 - I, r3s = r3 + I;
    const size_t rv = (size_t)k * vplane + r2, rvn = rv - I, rvs = rv + I;
    const T r2ds = ldg(g.r2ds + k);
    const T r2dsU = k > 0 ? ldg(g.r2ds + k - 1) : T(0), r2dsD = k < K - 1 ? ldg(g.r2ds + k + 1) : T(0);
    const T Wt = k > 0 ? ldg(W + r3 + i) : T(0), Wb = k < K - 1 ? ldg(W + r3 + plane + i) : T(0);
    // ---------------- U point (j, i) and the zonal mass flux F^u(j, i)
    const T Fla0 = Fl(r3, r2, a0), Flb0 = Fl(r3, r2, b0), Fla1 = Fl(r3, r2, a1), Flb1 = Fl(r3, r2, b1);
    const T FtS = hasS ? Ft(rv, r2, i) : T(0), FtSp = hasS ? Ft(rv, r2, ip) : T(0);
    const T FtN = hasN ? Ft(rvn, r2n, i) : T(0), FtNp = hasN ? Ft(rvn, r2n, ip) : T(0);
    // adjoint of F^u(j, i): the Phi pair (a0, b0), the U pairs (a0, b0) and
    // (a1, b1), the V pairs of rows j and j-1 whose face means hold it, and
    // the divergence of the scalar points a0 and b0
    T aFl = zf * (hbP(r3, r2, r2A, a0) * Gs(r3, r2, b0) - hbP(r3, r2, r2A, b0) * Gs(r3, r2, a0));
    aFl += T(0.5) * zf *
           ((hbU(r3, r2, r2A, a0) * Gu(r3, r2, b0) - hbU(r3, r2, r2A, b0) * Gu(r3, r2, a0)) +
            (hbU(r3, r2, r2A, a1) * Gu(r3, r2, b1) - hbU(r3, r2, r2A, b1) * Gu(r3, r2, a1)));
    if (hasS) aFl += T(0.5) * zfvS * (hbV(rv, r2, r2AvS, cS) * Gv(rv, r2, dS) - hbV(rv, r2, r2AvS, dS) * Gv(rv, r2, cS));
    if (hasN)
      aFl += T(0.5) * zfvN * (hbV(rvn, r2n, r2AvN, cN) * Gv(rvn, r2n, dN) - hbV(rvn, r2n, r2AvN, dN) * Gv(rvn, r2n, cN));
    aFl += rdx * (ldg(Db + r3 + a0) - ldg(Db + r3 + b0));
    // adjoint of G^u(j, i): zonal pairs (i - M, i), (i, i + M), meridional
    // pairs with rows j-1 and j+1, vertical pairs with levels k-1 and k+1,
    // and the Coriolis terms of the U point itself and of the V points
    // (j, i), (j, i+1), (j-1, i), (j-1, i+1)
    const T ZEu = T(0.5) * zf * (Flb1 + Flb0), ZWu = T(0.5) * zf * (Fla1 + Fla0);
    const T YSu = T(0.5) * yvS * (FtS + FtSp), YNu = T(0.5) * yvN * (FtN + FtNp);
    const T WTu = k > 0 ? T(0.5) * (Wt + ldg(W + r3 + ip)) : T(0);
    const T WBu = k < K - 1 ? T(0.5) * (Wb + ldg(W + r3 + plane + ip)) : T(0);
    const T yUc = ldg(yU + r3 + i), Uc = ldg(U + r3 + i);
    const T yVS0 = hasS ? ldg(yV + rv + i) : T(0), yVS1 = hasS ? ldg(yV + rv + ip) : T(0);
    const T yVN0 = hasN ? ldg(yV + rvn + i) : T(0), yVN1 = hasN ? ldg(yV + rvn + ip) : T(0);
    const T VS0 = hasS ? ldg(V + rv + i) : T(0), VS1 = hasS ? ldg(V + rv + ip) : T(0);
    const T VN0 = hasN ? ldg(V + rvn + i) : T(0), VN1 = hasN ? ldg(V + rvn + ip) : T(0);
    const T Cu = cnS * (yVS0 + yVS1) + csN * (yVN0 + yVN1);
    T aGu = hbU(r3, r2, r2A, iW) * ZWu - hbU(r3, r2, r2A, iE) * ZEu;
    if (hasN) aGu += hbU(r3n, r2n, r2AN, i) * YNu;
    if (hasS) aGu -= hbU(r3s, r2s, r2AS, i) * YSu;
    if (k > 0) aGu -= ldg(yU + r3 - plane + i) * r2dsU * rPuc * WTu;
    if (k < K - 1) aGu += ldg(yU + r3 + plane + i) * r2dsD * rPuc * WBu;
    aGu += (T(-0.25) * yUc * (VN0 + VN1 + VS0 + VS1) + Cu * Uc) * cota;
    const T Guc = Uc * rPuc;
    const T aU = Cu * (f0 + Guc * cota);
    // the U point's own tendency: its factors 1/P^u and P^u
    T horU = ZEu * Gu(r3, r2, iE) - ZWu * Gu(r3, r2, iW);
    if (hasS) horU += YSu * Gu(r3s, r2s, i);
    if (hasN) horU -= YNu * Gu(r3n, r2n, i);
    T verU = 0;
    if (k < K - 1) verU += WBu * ldg(U + r3 + plane + i) * rPuc;
    if (k > 0) verU -= WTu * ldg(U + r3 - plane + i) * rPuc;
    const T tRPu = -yUc * (horU * r2A + verU * r2ds);
    const T tPu = -yUc * (ldg(psi + r3 + b0) - ldg(psi + r3 + a0)) * rdx;
    // F^u = P^u U, G^u = U / P^u
    const T bu = aU + aFl * Puc + aGu * rPuc;
    aPu += aFl * Uc + tPu;
    arPu += aGu * Uc + tRPu;
    {
      const size_t q = r3 + i;
      const T v = o.scale * bu;
      o.oU[q] = (o.accumulate ? o.oU[q] : T(0)) + v;
      if (o.sU) o.sU[q] = o.rU[q] + v;
    }
    // ---------------- Phi point (j, i)
    // adjoint of G^s(j, i): zonal pairs (i - M, i), (i, i + M) with face
    // fluxes F^u(a1), F^u(b1), meridional pairs, vertical pairs
    const T yPc = ldg(yPhi + r3 + i), Phc = ldg(Phi + r3 + i);
    T aGs = zf * (hbP(r3, r2, r2A, iW) * Fla1 - hbP(r3, r2, r2A, iE) * Flb1);
    if (hasN) aGs += hbP(r3n, r2n, r2AN, i) * yvN * FtN;
    if (hasS) aGs -= hbP(r3s, r2s, r2AS, i) * yvS * FtS;
    if (k > 0) aGs -= ldg(yPhi + r3 - plane + i) * r2dsU * rPc * Wt;
    if (k < K - 1) aGs += ldg(yPhi + r3 + plane + i) * r2dsD * rPc * Wb;
    // the Phi point's own tendency: its factor 1/P
    T horP = zf * (Flb1 * Gs(r3, r2, iE) - Fla1 * Gs(r3, r2, iW));
    if (hasS) horP += yvS * FtS * Gs(r3s, r2s, i);
    if (hasN) horP -= yvN * FtN * Gs(r3n, r2n, i);
    T verP = 0;
    if (k < K - 1) verP += Wb * ldg(Phi + r3 + plane + i) * rPc;
    if (k > 0) verP -= Wt * ldg(Phi + r3 - plane + i) * rPc;
    const T tRP = -yPc * (horP * r2A + verP * r2ds);
    const T bp = ldg(aPhi + r3 + i) + aGs * rPc;
    arP += aGs * Phc + tRP;
    {
      const size_t q = r3 + i;
      const T v = o.scale * bp;
      o.oPhi[q] = (o.accumulate ? o.oPhi[q] : T(0)) + v;
      if (o.sU) o.sPhi[q] = o.rPhi[q] + v;
    }
    // ---------------- V point (j, i)
    if (hasS) {
      const T yVc = yVS0, Vc = VS0;
      const T FtSS = hasSS ? Ft(rvs, r2s, i) : T(0);
      // adjoint of F^v(j, i): the Phi pair and the U pairs (i-1, i) of rows
      // (j, j+1), the V pairs (j-1, j) and (j, j+1), the divergence of the
      // scalar points (j, i) and (j+1, i)
      const T hbVc = -yVc * r2AvS * rPvc;
      const T GvS = Gv(rv, r2, i);
      const T aYP = hbP(r3, r2, r2A, i) * Gs(r3s, r2s, i) - hbP(r3s, r2s, r2AS, i) * Gs(r3, r2, i);
      const T aYU = (hbU(r3, r2, r2A, i) * Gu(r3s, r2s, i) - hbU(r3s, r2s, r2AS, i) * Gu(r3, r2, i)) +
                    (hbU(r3, r2, r2A, im) * Gu(r3s, r2s, im) - hbU(r3s, r2s, r2AS, im) * Gu(r3, r2, im));
      T aYV = 0;
      if (hasSS) aYV += hbVc * Gv(rvs, r2s, i) - hbV(rvs, r2s, r2AvSS, i) * GvS;
      if (hasN) aYV += hbV(rvn, r2n, r2AvN, i) * GvS - hbVc * Gv(rvn, r2n, i);
      T aFt = yvS * aYP + T(0.5) * yvS * (aYU + aYV);
      aFt += svS * (rdyS * ldg(Db + r3 + i) - rdyS1 * ldg(Db + r3s + i));
      // adjoint of G^v(j, i): zonal pairs (i - Mv, i), (i, i + Mv) with face
      // fluxes the means of F^u over rows j, j+1; meridional and vertical pairs
      const T ZEv = T(0.5) * zfvS * (Fl(r3, r2, fEv) + Fl(r3s, r2s, fEv));
      const T ZWv = T(0.5) * zfvS * (Fl(r3, r2, fWv) + Fl(r3s, r2s, fWv));
      const T YSv = hasSS ? T(0.5) * (yvS * FtS + yvSS * FtSS) : T(0);
      const T YNv = hasN ? T(0.5) * (yvN * FtN + yvS * FtS) : T(0);
      const T WTv = k > 0 ? T(0.5) * (Wt + ldg(W + r3s + i)) : T(0);
      const T WBv = k < K - 1 ? T(0.5) * (Wb + ldg(W + r3s + plane + i)) : T(0);
      T aGv = hbV(rv, r2, r2AvS, vW) * ZWv - hbV(rv, r2, r2AvS, vE) * ZEv;
      if (hasN) aGv += hbV(rvn, r2n, r2AvN, i) * YNv;
      if (hasSS) aGv -= hbV(rvs, r2s, r2AvSS, i) * YSv;
      if (k > 0) aGv -= ldg(yV + rv - vplane + i) * r2dsU * rPvc * WTv;
      if (k < K - 1) aGv += ldg(yV + rv + vplane + i) * r2dsD * rPvc * WBv;
      // adjoint of V(j, i): the Coriolis terms of the U points (j, i-1),
      // (j, i), (j+1, i-1), (j+1, i)
      const T aV = T(-0.25) * (ldg(yU + r3 + im) * (f0 + Gu(r3, r2, im) * cota) + yUc * (f0 + Guc * cota) +
                               ldg(yU + r3s + im) * (f0S + Gu(r3s, r2s, im) * cotaS) +
                               ldg(yU + r3s + i) * (f0S + Gu(r3s, r2s, i) * cotaS));
      // the V point's own tendency: its factors 1/P^v and P^v
      T horV = ZEv * Gv(rv, r2, vE) - ZWv * Gv(rv, r2, vW);
      if (hasSS) horV += YSv * Gv(rvs, r2s, i);
      if (hasN) horV -= YNv * Gv(rvn, r2n, i);
      T verV = 0;
      if (k < K - 1) verV += WBv * ldg(V + rv + vplane + i) * rPvc;
      if (k > 0) verV -= WTv * ldg(V + rv - vplane + i) * rPvc;
      const T tRPv = -yVc * (horV * r2AvS + verV * r2ds);
      const T tPv = -yVc * (ldg(psi + r3s + i) - ldg(psi + r3 + i)) * rady;
      const T bv = aV + aFt * Pvc + aGv * rPvc;
      aPv += aFt * Vc + tPv;
      arPv += aGv * Vc + tRPv;
      const size_t q = rv + i;
      const T v = o.scale * bv;
      o.oV[q] = (o.accumulate ? o.oV[q] : T(0)) + v;
      if (o.sU) o.sV[q] = o.rV[q] + v;
    }
  }
  // P^u = sqrt(m^u): dP^u/dm^u = 1/(2 P^u), d(1/P^u)/dm^u = -1/(2 P^u^3)
  const size_t cstride = (size_t)gridDim.z * nrows * I;
  const size_t n = ((size_t)blockIdx.z * nrows + jq) * I + i;
  part[n] = aPu * T(0.5) * rPuc - arPu * T(0.5) * rPuc * rPuc * rPuc;
  part[cstride + n] = hasS ? aPv * T(0.5) * rPvc - arPv * T(0.5) * rPvc * rPvc * rPvc : T(0);
  part[2 * cstride + n] = -arP * T(0.5) * rPc * rPc * rPc;
}

// The level-chunk partial sums of k_adj_gather, added in chunk order into
// the adjoints of m^u, m^v, m for its rows.
template <class T>
__global__ void __launch_bounds__(256) k_adj_fold(Geom<T> g, const int* __restrict__ rows, int nrows, int nchunks,
                                                  const T* __restrict__ part, AdjM<T> m) {
  const int I = g.I;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrows * I) return;
  const int jq = q / I, i = q - jq * I;
  const size_t cstride = (size_t)nchunks * nrows * I;
  T su = 0, sv = 0, sc = 0;
  for (int c = 0; c < nchunks; ++c) {
    const size_t n = ((size_t)c * nrows + jq) * I + i;
    su += part[n];
    sv += part[cstride + n];
    sc += part[2 * cstride + n];
  }
  const size_t n = (size_t)ldg(rows + jq) * I + i;
  m.mub[n] = su;
  m.mvb[n] = sv;
  m.mcb[n] = sc;
}

// ---------------------------------------------------------------------------
// Row-segment form of k_adj_gather.  A CTA of kAdjRowB threads takes one row
// j and a segment of `own` columns with a halo of H columns on each side
// (H = the widest offset at which the row's transposed stencil reads:
// max(M_j, Mv_j, (Mv_{j-1} + 1) / 2)).  Per level, every thread stages the
// pointwise factors of its column (y / P, x / P and P x of the U, Phi and V
// points of rows j-1, j, j+1, and three combinations for the Coriolis pair)
// into shared memory, then the owning threads gather the transposed stencil
// from there: each factor is formed once per CTA instead of once per reader,
// and every neighbour read is a shared-memory load at a fixed offset (the
// seam of the periodic row is resolved when staging).  The vertical
// neighbours are the thread's own column at levels k-1 and k+1: the previous
// level's raw values are kept in registers and the next level's are loaded
// one iteration ahead (they are also what the thread stages next).  Two
// shared buffers alternate between levels with one barrier per level: the
// buffer a level writes was last read two levels before, and every thread has
// passed the barrier between.
constexpr int kAdjRowB = 256;
constexpr int kAdjRowMaxH = 48;
enum AdjRowArr {
  kqP0, kGs0, kqU0, kGu0, kFl0, kqV0, kGv0, kFt0,  // row j, V row j
  kqP1, kGs1, kqU1, kGu1, kFl1, kqV1, kGv1, kFt1,  // row j+1, V row j+1
  kqPm, kGsm, kqUm, kGum, kqVm, kGvm, kFtm,        // row j-1, V row j-1
  kVs, kyC, kcUs,                                  // Coriolis combinations
  kAdjRowNA
};

// Halo of row j's adjoint stencil (Mv = 0 without a V row j, Mvm = 0 without
// a V row j-1) and its segments: nseg segments of at most S owned columns.
__host__ __device__ inline int adj_row_halo(int M, int Mv, int Mvm) {
  int h = M > Mv ? M : Mv;
  const int hm = (Mvm + 1) / 2;
  if (hm > h) h = hm;
  return h < 1 ? 1 : h;
}
__host__ __device__ inline void adj_row_segments(int I, int H, int* nseg, int* S) {
  const int w = kAdjRowB - 2 * H;
  *nseg = (I + w - 1) / w;
  *S = (I + *nseg - 1) / *nseg;
}
template <class T>
constexpr size_t adj_row_smem() {
  return (size_t)2 * kAdjRowNA * kAdjRowB * sizeof(T);
}

template <class T>
#ifndef AGCM_ADJROWB
#define AGCM_ADJROWB 2
#endif
__global__ void __launch_bounds__(kAdjRowB, sizeof(T) == 4 ? AGCM_ADJROWB : 1) k_adj_rows(
    Geom<T> g, const int* __restrict__ items, const T* __restrict__ U, const T* __restrict__ V,
    const T* __restrict__ Phi, ColState<T> cs, const T* __restrict__ W, const T* __restrict__ psi,
    const T* __restrict__ Db, const T* __restrict__ aPhi, const T* __restrict__ arPcol, const T* __restrict__ yU,
    const T* __restrict__ yV, const T* __restrict__ yPhi, AdjM<T> m, AdjOut<T> o) {
  extern __shared__ __align__(16) unsigned char adj_smem[];
  T* const sm = reinterpret_cast<T*>(adj_smem);
  const int I = g.I, J = g.J, K = g.K;
  const int item = ldg(items + blockIdx.x);
  const int j = item >> 8, seg = item & 255;
  const bool hasS = j < J - 1, hasN = j > 0, hasSS = j + 1 < J - 1;
  const int M = ldg(g.Mu + j), Mv = hasS ? ldg(g.Mv + j) : 0, Mvm = hasN ? ldg(g.Mv + j - 1) : 0;
  const int H = adj_row_halo(M, Mv, Mvm);
  int nseg, S;
  adj_row_segments(I, H, &nseg, &S);
  const int s0 = seg * S, own = min(S, I - s0);
  const int t = threadIdx.x;
  const bool active = t < own + 2 * H, owner = t >= H && t < H + own;
  int c = (s0 - H + t) % I;
  if (c < 0) c += I;
  // element offsets fit 32 bits: nlon * nlat * nlev <= 4e9
  const unsigned plane = (unsigned)J * (unsigned)I, vplane = (unsigned)(J - 1) * (unsigned)I;
  const unsigned r2 = (unsigned)j * (unsigned)I;
  // row tables
  const T zf = ldg(g.zf + j), r2A = ldg(g.r2A + j), rdx = ldg(g.rdx + j), f0 = ldg(g.f0 + j),
          cota = ldg(g.cota + j);
  const T r2AN = hasN ? ldg(g.r2A + j - 1) : T(0), r2AS = hasS ? ldg(g.r2A + j + 1) : T(0);
  const T yvS = hasS ? ldg(g.yv + j) : T(0), yvN = hasN ? ldg(g.yv + j - 1) : T(0),
          yvSS = hasSS ? ldg(g.yv + j + 1) : T(0);
  const T cnS = hasS ? ldg(g.cn + j) : T(0), csN = hasN ? ldg(g.cs + j - 1) : T(0);
  const T zfvS = hasS ? ldg(g.zfv + j) : T(0), r2AvS = hasS ? ldg(g.r2Av + j) : T(0);
  const T r2AvSS = hasSS ? ldg(g.r2Av + j + 1) : T(0);
  const T zfvN = hasN ? ldg(g.zfv + j - 1) : T(0), r2AvN = hasN ? ldg(g.r2Av + j - 1) : T(0);
  const T svS = hasS ? ldg(g.sv + j) : T(0), rdyS = hasS ? ldg(g.rdy + j) : T(0),
          rdyS1 = hasS ? ldg(g.rdy + j + 1) : T(0);
  const T f0S = hasS ? ldg(g.f0 + j + 1) : T(0), cotaS = hasS ? ldg(g.cota + j + 1) : T(0);
  const T rady = g.rady;
  // offsets of the stencil from an owned column
  const int oa0 = -(M - 1) / 2, ob0 = (M + 1) / 2, oa1 = -(M + 1) / 2, ob1 = (M - 1) / 2;
  const int ocS = -(Mv - 1) / 2, odS = (Mv + 1) / 2, ofEv = (Mv - 1) / 2, ofWv = -(Mv + 1) / 2;
  const int ocN = -(Mvm - 1) / 2, odN = (Mvm + 1) / 2;
  const int a0g = wrapi(c + oa0, I), b0g = wrapi(c + ob0, I), cp = wrapi(c + 1, I);
  // the 2-D factors of the staged column c, rows j-1, j, j+1 (V rows alike)
  const T rP0 = ldg(cs.rP + r2 + c), rPu0 = ldg(cs.rPu + r2 + c), Pu0 = ldg(cs.Pu + r2 + c);
  const T rP1 = hasS ? ldg(cs.rP + r2 + I + c) : T(0), rPu1 = hasS ? ldg(cs.rPu + r2 + I + c) : T(0),
          Pu1 = hasS ? ldg(cs.Pu + r2 + I + c) : T(0);
  const T rPm = hasN ? ldg(cs.rP + r2 - I + c) : T(0), rPum = hasN ? ldg(cs.rPu + r2 - I + c) : T(0);
  const T rPv0 = hasS ? ldg(cs.rPv + r2 + c) : T(0), Pv0 = hasS ? ldg(cs.Pv + r2 + c) : T(0);
  const T rPv1 = hasSS ? ldg(cs.rPv + r2 + I + c) : T(0), Pv1 = hasSS ? ldg(cs.Pv + r2 + I + c) : T(0);
  const T rPvm = hasN ? ldg(cs.rPv + r2 - I + c) : T(0), Pvm = hasN ? ldg(cs.Pv + r2 - I + c) : T(0);
  // raw values of column c at one level: row j, j+1, j-1 (Phi, U), V rows j, j+1, j-1
  struct Raw {
    T yP0, P0, yU0, U0, yV0, V0, yP1, P1, yU1, U1, yV1, V1, yPm, Pm, yUm, Um, yVm, Vm;
  };
  auto load_raw = [&](int k, Raw& r) {
    const unsigned r3 = (unsigned)k * plane + r2 + c, rv = (unsigned)k * vplane + r2 + c;
    r.yP0 = ldg(yPhi + r3);
    r.P0 = ldg(Phi + r3);
    r.yU0 = ldg(yU + r3);
    r.U0 = ldg(U + r3);
    r.yV0 = hasS ? ldg(yV + rv) : T(0);
    r.V0 = hasS ? ldg(V + rv) : T(0);
    r.yP1 = hasS ? ldg(yPhi + r3 + I) : T(0);
    r.P1 = hasS ? ldg(Phi + r3 + I) : T(0);
    r.yU1 = hasS ? ldg(yU + r3 + I) : T(0);
    r.U1 = hasS ? ldg(U + r3 + I) : T(0);
    r.yV1 = hasSS ? ldg(yV + rv + I) : T(0);
    r.V1 = hasSS ? ldg(V + rv + I) : T(0);
    r.yPm = hasN ? ldg(yPhi + r3 - I) : T(0);
    r.Pm = hasN ? ldg(Phi + r3 - I) : T(0);
    r.yUm = hasN ? ldg(yU + r3 - I) : T(0);
    r.Um = hasN ? ldg(U + r3 - I) : T(0);
    r.yVm = hasN ? ldg(yV + rv - I) : T(0);
    r.Vm = hasN ? ldg(V + rv - I) : T(0);
  };
  // the owner's other inputs at one level: psi and Dbar at the columns a0,
  // b0, i of row j and i of row j+1, and the adjoint of Phi from the column pass
  struct Own {
    T psa, psb, psc, pss, Dba, Dbb, Dbc, Dbs, aPh;
  };
  auto load_own = [&](int k, Own& w) {
    const unsigned r3 = (unsigned)k * plane + r2;
    w.psa = ldg(psi + r3 + a0g);
    w.psb = ldg(psi + r3 + b0g);
    w.psc = ldg(psi + r3 + c);
    w.pss = hasS ? ldg(psi + r3 + I + c) : T(0);
    w.Dba = ldg(Db + r3 + a0g);
    w.Dbb = ldg(Db + r3 + b0g);
    w.Dbc = ldg(Db + r3 + c);
    w.Dbs = hasS ? ldg(Db + r3 + I + c) : T(0);
    w.aPh = ldg(aPhi + r3 + c);
  };
  Raw cur{}, nxt{};
  Own ocur{}, onxt{};
  if (active) load_raw(0, cur);
  if (owner) load_own(0, ocur);
  // the array the owner reads back and adds to: the stage sum, or the
  // output itself when accumulating
  const T* const rmwU = o.sU ? o.rU : (o.accumulate ? o.oU : nullptr);
  const T* const rmwP = o.sU ? o.rPhi : (o.accumulate ? o.oPhi : nullptr);
  const T* const rmwV = o.sU ? o.rV : (o.accumulate ? o.oV : nullptr);
  // own column at level k-1 (row j, V row j)
  T yPp = 0, Pp = 0, yUp = 0, Up = 0, yVp = 0, Vp = 0;
  // W at level k (rows j, j+1; columns i, i+1), loaded one level ahead
  T Wt = 0, Wtp = 0, Wts = 0;
  T aPu = 0, arPu = 0, aPv = 0, arPv = 0, arP = owner ? ldg(arPcol + r2 + c) : T(0);
  const T rPc = rP0, rPuc = rPu0, Puc = Pu0, rPvc = rPv0, Pvc = Pv0;
  for (int k = 0; k < K; ++k) {
    T* const b = sm + (size_t)(k & 1) * kAdjRowNA * kAdjRowB;
    // this level's values to add to, loaded before the staging so that the
    // load is in flight across it
    T accU = 0, accP = 0, accV = 0;
    if (owner && rmwU) {
      const unsigned q = (unsigned)k * plane + r2 + c;
      accU = rmwU[q];
      accP = rmwP[q];
      if (hasS) accV = rmwV[(unsigned)k * vplane + r2 + c];
    }
    if (active) {
      T* const q = b + t;
      const Raw& r = cur;
      const T Gu0 = r.U0 * rPu0, Gu1 = r.U1 * rPu1;
      q[kqP0 * kAdjRowB] = r.yP0 * rP0;
      q[kGs0 * kAdjRowB] = r.P0 * rP0;
      q[kqU0 * kAdjRowB] = r.yU0 * rPu0;
      q[kGu0 * kAdjRowB] = Gu0;
      q[kFl0 * kAdjRowB] = Pu0 * r.U0;
      q[kqV0 * kAdjRowB] = r.yV0 * rPv0;
      q[kGv0 * kAdjRowB] = r.V0 * rPv0;
      q[kFt0 * kAdjRowB] = Pv0 * r.V0;
      q[kqP1 * kAdjRowB] = r.yP1 * rP1;
      q[kGs1 * kAdjRowB] = r.P1 * rP1;
      q[kqU1 * kAdjRowB] = r.yU1 * rPu1;
      q[kGu1 * kAdjRowB] = Gu1;
      q[kFl1 * kAdjRowB] = Pu1 * r.U1;
      q[kqV1 * kAdjRowB] = r.yV1 * rPv1;
      q[kGv1 * kAdjRowB] = r.V1 * rPv1;
      q[kFt1 * kAdjRowB] = Pv1 * r.V1;
      q[kqPm * kAdjRowB] = r.yPm * rPm;
      q[kGsm * kAdjRowB] = r.Pm * rPm;
      q[kqUm * kAdjRowB] = r.yUm * rPum;
      q[kGum * kAdjRowB] = r.Um * rPum;
      q[kqVm * kAdjRowB] = r.yVm * rPvm;
      q[kGvm * kAdjRowB] = r.Vm * rPvm;
      q[kFtm * kAdjRowB] = Pvm * r.Vm;
      // V(j-1) + V(j); cn yV(j) + cs yV(j-1); the Coriolis factor yU fs of rows j, j+1
      q[kVs * kAdjRowB] = r.V0 + r.Vm;
      q[kyC * kAdjRowB] = cnS * r.yV0 + csN * r.yVm;
      q[kcUs * kAdjRowB] = r.yU0 * (f0 + Gu0 * cota) + (hasS ? r.yU1 * (f0S + Gu1 * cotaS) : T(0));
      if (k + 1 < K) load_raw(k + 1, nxt);
    }
    if (owner && k + 1 < K) load_own(k + 1, onxt);
    T Wb = 0, Wbp = 0, Wbs = 0;
    if (owner && k + 1 < K) {
      const unsigned wq = (unsigned)(k + 1) * plane + r2;
      Wb = ldg(W + wq + c);
      Wbp = ldg(W + wq + cp);
      Wbs = hasS ? ldg(W + wq + I + c) : T(0);
    }
    __syncthreads();
    if (owner) {
      const T* const L = b + t;
      auto A = [&](int arr, int off) { return L[arr * kAdjRowB + off]; };
      const unsigned r3 = (unsigned)k * plane + r2, rv = (unsigned)k * vplane + r2;
      const T r2ds = ldg(g.r2ds + k);
      const T r2dsU = k > 0 ? ldg(g.r2ds + k - 1) : T(0), r2dsD = k + 1 < K ? ldg(g.r2ds + k + 1) : T(0);
      const bool up = k > 0, dn = k + 1 < K;
      // own column at levels k and k+1
      const T yPc = cur.yP0, Pc = cur.P0, yUc = cur.yU0, Uc = cur.U0, yVc = cur.yV0, Vc = cur.V0;
      const T yPn = dn ? nxt.yP0 : T(0), Pn = dn ? nxt.P0 : T(0), yUn = dn ? nxt.yU0 : T(0),
              Un = dn ? nxt.U0 : T(0), yVn = dn ? nxt.yV0 : T(0), Vn = dn ? nxt.V0 : T(0);
      // ---------------- U point and F^u
      const T Fla0 = A(kFl0, oa0), Flb0 = A(kFl0, ob0), Fla1 = A(kFl0, oa1), Flb1 = A(kFl0, ob1);
      T aFl = -zf * r2A * (A(kqP0, oa0) * A(kGs0, ob0) - A(kqP0, ob0) * A(kGs0, oa0));
      aFl -= T(0.5) * zf * r2A *
             ((A(kqU0, oa0) * A(kGu0, ob0) - A(kqU0, ob0) * A(kGu0, oa0)) +
              (A(kqU0, oa1) * A(kGu0, ob1) - A(kqU0, ob1) * A(kGu0, oa1)));
      if (hasS) aFl -= T(0.5) * zfvS * r2AvS * (A(kqV0, ocS) * A(kGv0, odS) - A(kqV0, odS) * A(kGv0, ocS));
      if (hasN) aFl -= T(0.5) * zfvN * r2AvN * (A(kqVm, ocN) * A(kGvm, odN) - A(kqVm, odN) * A(kGvm, ocN));
      aFl += rdx * (ocur.Dba - ocur.Dbb);
      const T FtS = A(kFt0, 0), FtSp = A(kFt0, 1), FtN = A(kFtm, 0), FtNp = A(kFtm, 1);
      const T ZEu = T(0.5) * zf * (Flb1 + Flb0), ZWu = T(0.5) * zf * (Fla1 + Fla0);
      const T YSu = T(0.5) * yvS * (FtS + FtSp), YNu = T(0.5) * yvN * (FtN + FtNp);
      const T WTu = up ? T(0.5) * (Wt + Wtp) : T(0), WBu = dn ? T(0.5) * (Wb + Wbp) : T(0);
      const T Cu = A(kyC, 0) + A(kyC, 1);
      T aGu = -r2A * (A(kqU0, -M) * ZWu - A(kqU0, M) * ZEu);
      if (hasN) aGu -= r2AN * A(kqUm, 0) * YNu;
      if (hasS) aGu += r2AS * A(kqU1, 0) * YSu;
      if (up) aGu -= r2dsU * yUp * rPuc * WTu;
      if (dn) aGu += r2dsD * yUn * rPuc * WBu;
      aGu += (T(-0.25) * yUc * (A(kVs, 0) + A(kVs, 1)) + Cu * Uc) * cota;
      const T aU = Cu * (f0 + Uc * rPuc * cota);
      T horU = ZEu * A(kGu0, M) - ZWu * A(kGu0, -M) + YSu * A(kGu1, 0) - YNu * A(kGum, 0);
      const T verU = (dn ? WBu * Un * rPuc : T(0)) - (up ? WTu * Up * rPuc : T(0));
      const T tRPu = -yUc * (horU * r2A + verU * r2ds);
      const T tPu = -yUc * (ocur.psb - ocur.psa) * rdx;
      const T bu = aU + aFl * Puc + aGu * rPuc;
      aPu += aFl * Uc + tPu;
      arPu += aGu * Uc + tRPu;
      {
        const unsigned q = r3 + c;
        const T v = o.scale * bu;
        if (o.sU) {
          o.oU[q] = v;
          o.sU[q] = accU + v;
        } else {
          o.oU[q] = accU + v;  // accU = 0 unless accumulating
        }
      }
      // ---------------- Phi point
      T aGs = -r2A * zf * (A(kqP0, -M) * Fla1 - A(kqP0, M) * Flb1);
      if (hasN) aGs -= r2AN * A(kqPm, 0) * yvN * FtN;
      if (hasS) aGs += r2AS * A(kqP1, 0) * yvS * FtS;
      if (up) aGs -= r2dsU * yPp * rPc * Wt;
      if (dn) aGs += r2dsD * yPn * rPc * Wb;
      const T horP = zf * (Flb1 * A(kGs0, M) - Fla1 * A(kGs0, -M)) + yvS * FtS * A(kGs1, 0) - yvN * FtN * A(kGsm, 0);
      const T verP = (dn ? Wb * Pn * rPc : T(0)) - (up ? Wt * Pp * rPc : T(0));
      const T tRP = -yPc * (horP * r2A + verP * r2ds);
      const T bp = ocur.aPh + aGs * rPc;
      arP += aGs * Pc + tRP;
      {
        const unsigned q = r3 + c;
        const T v = o.scale * bp;
        if (o.sU) {
          o.oPhi[q] = v;
          o.sPhi[q] = accP + v;
        } else {
          o.oPhi[q] = accP + v;
        }
      }
      // ---------------- V point
      if (hasS) {
        const T aYP = -r2A * A(kqP0, 0) * A(kGs1, 0) + r2AS * A(kqP1, 0) * A(kGs0, 0);
        const T aYU = (-r2A * A(kqU0, 0) * A(kGu1, 0) + r2AS * A(kqU1, 0) * A(kGu0, 0)) +
                      (-r2A * A(kqU0, -1) * A(kGu1, -1) + r2AS * A(kqU1, -1) * A(kGu0, -1));
        T aYV = 0;
        if (hasSS) aYV += -r2AvS * A(kqV0, 0) * A(kGv1, 0) + r2AvSS * A(kqV1, 0) * A(kGv0, 0);
        if (hasN) aYV += -r2AvN * A(kqVm, 0) * A(kGv0, 0) + r2AvS * A(kqV0, 0) * A(kGvm, 0);
        T aFt = yvS * aYP + T(0.5) * yvS * (aYU + aYV);
        aFt += svS * (rdyS * ocur.Dbc - rdyS1 * ocur.Dbs);
        const T ZEv = T(0.5) * zfvS * (A(kFl0, ofEv) + A(kFl1, ofEv));
        const T ZWv = T(0.5) * zfvS * (A(kFl0, ofWv) + A(kFl1, ofWv));
        const T FtSS = A(kFt1, 0);
        const T YSv = hasSS ? T(0.5) * (yvS * FtS + yvSS * FtSS) : T(0);
        const T YNv = hasN ? T(0.5) * (yvN * FtN + yvS * FtS) : T(0);
        const T WTv = up ? T(0.5) * (Wt + Wts) : T(0), WBv = dn ? T(0.5) * (Wb + Wbs) : T(0);
        T aGv = -r2AvS * (A(kqV0, -Mv) * ZWv - A(kqV0, Mv) * ZEv);
        if (hasN) aGv -= r2AvN * A(kqVm, 0) * YNv;
        if (hasSS) aGv += r2AvSS * A(kqV1, 0) * YSv;
        if (up) aGv -= r2dsU * yVp * rPvc * WTv;
        if (dn) aGv += r2dsD * yVn * rPvc * WBv;
        const T aV = T(-0.25) * (A(kcUs, -1) + A(kcUs, 0));
        const T horV = ZEv * A(kGv0, Mv) - ZWv * A(kGv0, -Mv) + YSv * A(kGv1, 0) - YNv * A(kGvm, 0);
        const T verV = (dn ? WBv * Vn * rPvc : T(0)) - (up ? WTv * Vp * rPvc : T(0));
        const T tRPv = -yVc * (horV * r2AvS + verV * r2ds);
        const T tPv = -yVc * (ocur.pss - ocur.psc) * rady;
        const T bv = aV + aFt * Pvc + aGv * rPvc;
        aPv += aFt * Vc + tPv;
        arPv += aGv * Vc + tRPv;
        const unsigned q = rv + c;
        const T v = o.scale * bv;
        if (o.sU) {
          o.oV[q] = v;
          o.sV[q] = accV + v;
        } else {
          o.oV[q] = accV + v;
        }
      }
      yPp = yPc; Pp = Pc; yUp = yUc; Up = Uc; yVp = yVc; Vp = Vc;
      Wt = Wb; Wtp = Wbp; Wts = Wbs;
    }
    cur = nxt;
    ocur = onxt;
  }
  if (owner) {
    const unsigned n = r2 + c;
    m.mub[n] = aPu * T(0.5) * rPuc - arPu * T(0.5) * rPuc * rPuc * rPuc;
    m.mvb[n] = hasS ? aPv * T(0.5) * rPvc - arPv * T(0.5) * rPvc * rPvc * rPvc : T(0);
    m.mcb[n] = -arP * T(0.5) * rPc * rPc * rPc;
  }
}

// pi-bar = direct psi part + m-bar, with m^u_i = (m_i + m_{i+1})/2 and
// m^v_j = (m_j + m_{j+1})/2 transposed as gathers.
template <class T>
__global__ void __launch_bounds__(256) k_adj_colstate(Geom<T> g, AdjM<T> m, const T* __restrict__ aPiD,
                                                      AdjOut<T> o) {
  const int I = g.I, J = g.J;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I * J) return;
  const int j = n / I, i = n - j * I;
  T mb = m.mcb[n] + T(0.5) * (m.mub[n] + m.mub[j * I + wrapi(i - 1, I)]);
  if (j < J - 1) mb += T(0.5) * m.mvb[n];
  if (j > 0) mb += T(0.5) * m.mvb[n - I];
  const T v = o.scale * (aPiD[n] + mb);
  o.opi[n] = (o.accumulate ? o.opi[n] : T(0)) + v;
  if (o.spi) o.spi[n] = o.rpi[n] + v;
}

}  // namespace agcm
