// agcm_row.cuh — the stage kernel on whole row segments staged in shared memory.
//
// One CTA owns a segment of one latitude row j: the columns [c0, c0 + S) of
// the scalar/Phi row, the U row and (j < J-1) the V row, plus a halo of H
// columns on each side, H > every leap stride that row's stencil uses (Mu_j,
// Mv_j, Mu_{j+1}; Eq. 6 / Eq. 7).  Thread t stands for the column
// c = c0 - H + t (periodic in longitude) and streams the levels from the
// surface (k = K-1) to the top.  Per level:
//   * the raw rows j-1, j, j+1 of U, Phi and V of the stage input (and row j
//     of the base state x_n in the later stages) arrive in a ring of shared
//     memory slots by 1-D bulk copies (cp.async.bulk, completing on one
//     mbarrier per slot), issued several levels ahead of their use from a
//     descriptor list built once per CTA;
//   * own column: each thread forms what its neighbours need — the mass
//     fluxes F = P U (Eq. 1's IAP fluxes), G = F/P of the skew advection,
//     f* U of the Coriolis pair — and the leap divergence D of its column at
//     rows j and j+1 (Table "Communication aggregation": the (x+N-1, x-N)
//     pair, read from the staged U rows), advances the column carries of
//     Alg. 1 / Alg. 2 read bottom-up (suffix sums SD of dsigma D, so
//     W_k = SD_k - (1 - sh_k) C) and of the hydrostatic integral (psi as a
//     suffix sum of H Phi/P, reading R7), and publishes all of it to one of
//     two shared-memory buffers;
//   * after one barrier, the owned columns assemble the Phi, U and V cells
//     (advection L, pressure gradient over the (x+N, x-N+1) pair, Coriolis
//     pair, Omega~ conversion) from their neighbours' published values; the
//     vertical advection of a level needs the level above, so each level is
//     completed and written one iteration later.
// Nothing is recomputed per neighbour and every stencil read is a 32-bit
// shared-memory offset fixed for the whole column, which is what the
// one-thread-per-column global-load kernel (agcm_fused.cuh) spent most of its
// instructions on.  The column integral C (dpi/dt = -C) comes from the FP64
// vertical means Ubar, Vbar of the stage input, as in that kernel, and each
// stage accumulates its output's means for the next stage.
//
// Rows whose halo would leave fewer than 32 owned columns in a CTA (the one
// or two rows nearest each pole at 0.25 deg) and grids whose rows are not
// 16-byte aligned run the global-load kernel instead.
#pragma once
#include <type_traits>

#include "agcm_common.cuh"

namespace agcm {

#ifndef AGCM_ROW_B
#define AGCM_ROW_B 256
#endif
constexpr int kRowB = AGCM_ROW_B;  // threads per CTA: the widest segment + halo
constexpr int kRowNP = 13;         // arrays each thread publishes per level
constexpr int kRowRaw = 12;        // staged rows per level: U, Phi, V at j-1, j, j+1 and x_n's U, Phi, V at j
constexpr int kRowDesc = 48;       // copy descriptors per CTA: 12 rows of at most 4 pieces
#ifndef AGCM_ROW_MINB
#define AGCM_ROW_MINB (768 / AGCM_ROW_B)  // resident CTAs per SM: 24 warps at <= 80 registers
#endif
// levels in flight: a ring of two slots (three measured slower), which the
// level loop pairs with the two published buffers
template <class T>
struct RowCfg {
  static constexpr int R = 2;
};

// Halo of row j: one more than the largest stride of its stencil, to a
// multiple of 4 columns (16-byte aligned bulk copies).
__host__ __device__ __forceinline__ int row_halo(int Mu, int Mv, int M1) {
  int m = Mu > Mv ? Mu : Mv;
  m = m > M1 ? m : M1;
  return (m + 1 + 3) & ~3;
}
// Segments of a row of I columns with halo H in CTAs of B threads: count and
// width (a multiple of 4).  count = 0: the row is left to the column kernel,
// because its halo would take more than half of a CTA (strides above 63 with
// B = 256: the three rows nearest each pole at 0.25 deg).
__host__ __device__ __forceinline__ void row_segments(int I, int H, int B, int* nseg, int* S) {
  const int smax = (B - 2 * H) & ~3;
  if (smax < B / 2) {
    *nseg = 0;
    *S = 0;
    return;
  }
  const int n = (I + smax - 1) / smax;
  *nseg = n;
  *S = (((I + n - 1) / n) + 3) & ~3;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a ring slot's copies: try_wait suspends the thread until the phase
// completes (or a hardware time limit passes), so the loop turns rarely; it
// gives up after about a second (2e9 clocks), setting the CTA's abort flag
// and the status word to AGCM_ETIMEOUT (4).  Once the flag is set every later
// wait of the CTA returns at once, so the kernel runs to its end (no thread
// leaves early, every barrier is still met).
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                                  int* err) {
  long long t0 = -1;
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return;
    const long long now = clock64();
    if (t0 < 0) t0 = now;
    if (now - t0 > 2000000000LL) {
      *abort_flag = 1;
      if (err) atomicExch(err, 4);
      return;
    }
  }
}
// Executed by a whole warp with warp-uniform operands: one elected lane
// issues the copy (or, with tx != 0, announces tx bytes on the barrier), so
// the warp does not diverge around it.
__device__ __forceinline__ void bulk_copy_g2s_warp(unsigned dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n"
      " @p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n}" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_warp(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n"
      " @p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
// Named barrier over the CTA's first n threads (n a multiple of 32): warps
// past the segment leave at the start and take no part.
__device__ __forceinline__ void row_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// Stage arguments shared with the launcher.
template <class T>
struct RowArgs {
  const T* U;
  const T* V;
  const T* Phi;
  const T* pi;
  const double* Ubar;
  const double* Vbar;
  const T* Ub;
  const T* Vb;
  const T* Phib;
  const T* pib;
  T* Uo;
  T* Vo;
  T* Phio;
  T* pio;
  double* Ubar_o;
  double* Vbar_o;
  const double* Ubar_b;
  const double* Vbar_b;
  T cdt;
  const int* rows;   // work items of this launch: row j << 8 | segment
  int* err;          // status word (AGCM_ETIMEOUT)
};

// One bulk copy of a level: a piece of a staged row, its source at level 0,
// the plane stride in elements, its destination offset in a ring slot
// (bytes) and its size in bytes.
struct RowDesc {
  const char* src0;
  unsigned long long plane_bytes;
  unsigned dst;
  unsigned bytes;
};

constexpr size_t kRowHead = 64 + (size_t)kRowDesc * sizeof(RowDesc);
// Bytes of dynamic shared memory for NTP columns per array and K levels.
template <class T>
__host__ __device__ constexpr size_t row_smem_bytes(int NTP, int K) {
  return kRowHead + sizeof(T) * (size_t)NTP * (RowCfg<T>::R * kRowRaw + 2 * kRowNP + 2) +
         (size_t)K * (8 * sizeof(T) + sizeof(double));
}

// The stage on one row segment.  MODE 0: out = T(x) (validation); MODE 1:
// base = x (first stage); MODE 2: base = x_n (later stages; may alias out).
// TERMS: 1 advection, 2 adaptation, 3 both (Eq. 2's split).  NL: Eq. 1's
// delta kappa Phi/P term (each Phi/P entering psi or the Omega~ coefficient
// is scaled by 1 + rho_k Phi/P).  MC > 0: every row of the launch has
// Mu_j = Mv_j = Mu_{j+1} = MC, so the partner offsets are compile-time
// constants; MC = 0: any strides.
//
// row_segment runs one work item (row j, segment seg) with the CTA's dynamic
// shared memory `smem`; fresh = false when an earlier item of the same CTA
// left its mbarriers initialised (a persistent CTA running item after item,
// with every thread of the CTA past the earlier item).  A `return` only ends
// the item for the threads that take it.
template <class T, int MODE, int TERMS, bool NL, int MC>
__device__ __forceinline__ void row_segment(const Geom<T>& g, const RowArgs<T>& a, const int j, const int seg,
                                            unsigned char* smem, const bool fresh) {
  constexpr int R = RowCfg<T>::R;
  constexpr bool ADV = (TERMS & 1) != 0, ADA = (TERMS & 2) != 0;
  constexpr bool kInc = sizeof(T) == 4 && MODE != 0;
  const int I = g.I, J = g.J, K = g.K;
  const bool hasV = MC > 0 || j < J - 1;  // V row j (and scalar row j+1) exist; the classes hold no last row
  const int Mu = MC ? MC : g.Mu[j];
  const int Mv = MC ? MC : (hasV ? g.Mv[j] : 1);
  const int M1 = MC ? MC : (hasV ? g.Mu[j + 1] : 1);
  const int H = row_halo(Mu, Mv, M1);
  int nseg, Sw;
  row_segments(I, H, kRowB, &nseg, &Sw);
  const int c0 = seg * Sw;
  if (seg >= nseg || c0 >= I) return;  // whole CTA, before any barrier (the host lists no such item)
  const int Sown = min(Sw, I - c0);
  const int NT = Sown + 2 * H;
  const int NTW = (NT + 31) & ~31;
  const int t = threadIdx.x;
  if (t >= NTW) return;  // whole warps past the segment
  constexpr int NTP = kRowB;  // array pitch
  const bool owned = t >= H && t < H + Sown;
  const int cstart = ((c0 - H) % I + I) % I;  // global column of thread 0
  int gc = cstart + t;                        // own global column
  while (gc >= I) gc -= I;

  // shared memory: ring mbarriers, abort flag, descriptor count; the copy
  // descriptors; the ring of staged raw rows; two buffers of the published
  // arrays; the P^u rows j and j+1; the level tables
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 8 * R);
  int* s_ndesc = reinterpret_cast<int*>(smem + 8 * R + 4);
  unsigned* s_tx = reinterpret_cast<unsigned*>(smem + 8 * R + 8);
  RowDesc* desc = reinterpret_cast<RowDesc*>(smem + 64);
  T* ring = reinterpret_cast<T*>(smem + kRowHead);
  T* dA = ring + (size_t)R * kRowRaw * NTP;            // 2 buffers x kRowNP arrays
  T* puR = dA + (size_t)2 * kRowNP * NTP;              // P^u of row j, then of row j+1
  T* lev = puR + (size_t)2 * NTP;                      // K x 8 level coefficients
  double* levd = reinterpret_cast<double*>(lev + (size_t)8 * K);  // K: dsigma in FP64
  double* q2 = reinterpret_cast<double*>(dA);          // prologue only: P^u Ubar at rows j, j+1

  // ---- set-up: level tables, mbarriers, copy descriptors, rows the copies never fill
  for (int k = t; k < K; k += NTW) {
    T* L = lev + 8 * k;
    L[0] = g.ds[k];
    L[1] = g.Hkk[k];
    L[2] = g.hk[k];
    L[3] = g.hk_rds[k];
    L[4] = g.r2ds[k];
    L[5] = g.oms[k];
    L[6] = NL ? g.rho[k] : T(0);
    L[7] = T(0);
    levd[k] = g.dsd[k];
  }
  const unsigned ring_s = smem_addr(ring);
  if (t == 0) {
    if (!fresh)
      for (int s = 0; s < R; ++s)
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar + s)) : "memory");
    for (int s = 0; s < R; ++s) mbar_init(bar + s, 1);
    *abort_flag = 0;
    // one descriptor per piece of every staged row that exists: q = 0..2 U
    // rows j-1, j, j+1; 3..5 Phi; 6..8 V; 9..11 x_n's U, Phi, V at row j
    int nd = 0;
    unsigned tx = 0;
    for (int q = 0; q < kRowRaw; ++q) {
      if (q >= 9 && MODE != 2) break;
      const int f = q < 9 ? q / 3 : q - 9;
      const int r = q < 9 ? j - 1 + q % 3 : j;
      const int nrows = f == 2 ? J - 1 : J;
      if (r < 0 || r >= nrows) continue;
      const T* fld = q < 9 ? (f == 0 ? a.U : (f == 1 ? a.Phi : a.V)) : (f == 0 ? a.Ub : (f == 1 ? a.Phib : a.Vb));
      const T* row = fld + (size_t)r * I;
      int pos = cstart, left = NT, off = 0;
      while (left > 0 && nd < kRowDesc) {
        const int len = left < I - pos ? left : I - pos;
        desc[nd].src0 = reinterpret_cast<const char*>(row + pos);
        desc[nd].plane_bytes = (unsigned long long)nrows * I * sizeof(T);
        desc[nd].dst = (unsigned)(((size_t)q * NTP + off) * sizeof(T));
        desc[nd].bytes = (unsigned)(len * sizeof(T));
        tx += desc[nd].bytes;
        ++nd;
        off += len;
        left -= len;
        pos = 0;
      }
    }
    *s_ndesc = nd;
    *s_tx = tx;
    mbar_fence_init();
  }
  for (int q = 0; q < kRowRaw; ++q) {
    // rows outside the grid stay zero: U/Phi rows j-1 (j = 0) and j+1 (j = J-1),
    // V rows j-1, j, j+1 outside 0..J-2, x_n's V row j (j = J-1)
    const int f = q < 9 ? q / 3 : q - 9;
    const int r = q < 9 ? j - 1 + q % 3 : j;
    const int nrows = f == 2 ? J - 1 : J;
    if (r >= 0 && r < nrows) continue;
    for (int s = 0; s < R; ++s) ring[((size_t)s * kRowRaw + q) * NTP + t] = T(0);
  }
  row_sync(NTW);
  // Copies of level kk into slot s: warp 0 announces the bytes, and warp w
  // issues descriptors w, w + nw, ... (nw = warps of the segment), so no warp
  // carries all the copies; the warp index is made warp-uniform so that the
  // loop and the copies run without divergence.
  const int nw = NTW >> 5;
  const int warp = __shfl_sync(0xffffffffu, t >> 5, 0);
  const int ndesc = *s_ndesc;
  const unsigned txb = *s_tx;
  // a warp's first two descriptors are read once, for every level; the
  // levels are issued from the surface up, one after the other, so their
  // sources step down one plane per level from one past the surface level
  RowDesc d0{nullptr, 0, 0, 0}, d1{nullptr, 0, 0, 0};
  if (warp < ndesc) d0 = desc[warp];
  if (warp + nw < ndesc) d1 = desc[warp + nw];
  const char* src0 = d0.src0 + (unsigned long long)K * d0.plane_bytes;
  const char* src1 = d1.src0 + (unsigned long long)K * d1.plane_bytes;
  auto issue_level = [&](int kk, int s) {
    if (warp == 0) mbar_expect_tx_warp(bar + s, txb);
    const unsigned base = ring_s + (unsigned)(s * kRowRaw * NTP * sizeof(T));
    src0 -= d0.plane_bytes;
    src1 -= d1.plane_bytes;
    if (d0.bytes) bulk_copy_g2s_warp(base + d0.dst, src0, d0.bytes, bar + s);
    if (d1.bytes) bulk_copy_g2s_warp(base + d1.dst, src1, d1.bytes, bar + s);
    for (int d = warp + 2 * nw; d < ndesc; d += nw) {  // segments of fewer than six warps
      const RowDesc e = desc[d];
      bulk_copy_g2s_warp(base + e.dst, e.src0 + (unsigned long long)kk * e.plane_bytes, e.bytes, bar + s);
    }
  };
  for (int s = 0; s < R && s < K; ++s) issue_level(K - 1 - s, s);

  // ---- level-independent column quantities of the own column (a2)
  const T one = T(1);
  auto mass = [&](int r, int c) -> T { return g.pit[(size_t)r * I + c] + a.pi[(size_t)r * I + c]; };
  const int gcp = gc + 1 < I ? gc + 1 : 0;
  const bool hasN = j > 0, hasS = hasV, hasSS = j + 1 < J - 1;
  T rPn = 0, rPc, rPs = 0, Puc, rPuc, Pus = 0, rPus = 0, rPun = 0;
  T Pvc = 0, rPvn = 0, rPvc = 0, rPvs = 0, sPvn = 0, sPvc = 0, sPvs = 0;
  {
    const T mc = mass(j, gc), mcp = mass(j, gcp);
    rPc = one / sqrt_t(mc);
    Puc = sqrt_t(T(0.5) * (mc + mcp));
    rPuc = one / Puc;
    T ms = 0;
    if (hasN) {
      const T mn = mass(j - 1, gc);
      rPn = one / sqrt_t(mn);
      rPun = one / sqrt_t(T(0.5) * (mn + mass(j - 1, gcp)));
      const T Pvn = sqrt_t(T(0.5) * (mn + mc));
      rPvn = one / Pvn;
      sPvn = g.sv[j - 1] * Pvn;
    }
    if (hasS) {
      ms = mass(j + 1, gc);
      rPs = one / sqrt_t(ms);
      Pus = sqrt_t(T(0.5) * (ms + mass(j + 1, gcp)));
      rPus = one / Pus;
      Pvc = sqrt_t(T(0.5) * (mc + ms));
      rPvc = one / Pvc;
      sPvc = g.sv[j] * Pvc;
    }
    if (hasSS) {
      const T Pvs = sqrt_t(T(0.5) * (ms + mass(j + 2, gc)));
      rPvs = one / Pvs;
      sPvs = g.sv[j + 1] * Pvs;
    }
  }
  // ---- row geometry (block-uniform)
  const T rdx = g.rdx[j], rdy = g.rdy[j], zf2 = T(0.5) * g.zf[j], zf = g.zf[j], r2A = g.r2A[j];
  const T f0 = g.f0[j], cota = g.cota[j], adl = g.adl, adl2 = T(0.5) * g.adl, rady = g.rady;
  T rdxs = 0, rdys = 0, zfv2 = 0, r2Av = 0, cn = 0, cs = 0, f0s = 0, cotas = 0;
  if (hasS) {
    rdxs = g.rdx[j + 1];
    rdys = g.rdy[j + 1];
    zfv2 = T(0.5) * g.zfv[j];
    r2Av = g.r2Av[j];
    cn = g.cn[j];
    cs = g.cs[j];
    f0s = g.f0[j + 1];
    cotas = g.cota[j + 1];
  }

  // ---- offsets of the leap partners, fixed for the column.  A halo
  // thread's partner may lie up to H - 1 columns outside the segment; such
  // reads land in the neighbouring arrays of the same allocation (the ring
  // before the published arrays, the P^u rows and level tables after them)
  // and feed only results that no owned column uses.
  const int dE = (Mu - 1) / 2, dW = -(Mu + 1) / 2;       // F^lambda pair of D (Eq. 6)
  const int dE1 = (Mu + 1) / 2, dW1 = -(Mu - 1) / 2;     // psi pair of the U gradient
  const int de = Mu, dw = -Mu;                           // advection partners +-M
  const int dvE = (Mv - 1) / 2, dvW = -(Mv + 1) / 2;     // V-cell zonal faces
  const int dve = Mv, dvw = -Mv;                         // V-cell partners +-Mv
  const int dgE = (M1 - 1) / 2, dgW = -(M1 + 1) / 2;     // D of row j+1

  // ---- column integrals C (FP64) of rows j and j+1 from the vertical means
  q2[t] = (double)Puc * a.Ubar[(size_t)j * I + gc];
  q2[NTP + t] = hasS ? (double)Pus * a.Ubar[(size_t)(j + 1) * I + gc] : 0.0;
  puR[t] = Puc;
  puR[NTP + t] = Pus;
  row_sync(NTW);
  const double vbn = hasN ? (double)sPvn * a.Vbar[(size_t)(j - 1) * I + gc] : 0.0;
  const double vbc = hasS ? (double)sPvc * a.Vbar[(size_t)j * I + gc] : 0.0;
  const double vbs = hasSS ? (double)sPvs * a.Vbar[(size_t)(j + 1) * I + gc] : 0.0;
  const double Cc = (q2[t + dE] - q2[t + dW]) * (double)rdx + (vbc - vbn) * (double)rdy;
  const double Cs =
      hasS ? (q2[NTP + t + dgE] - q2[NTP + t + dgW]) * (double)rdxs + (vbs - vbc) * (double)rdys : 0.0;
  if (owned) {
    const size_t o = (size_t)j * I + gc;
    if (MODE == 0)
      a.pio[o] = ADA ? (T)(-Cc) : T(0);
    else {
      const double pb = (MODE == 1) ? (double)a.pi[o] : (double)a.pib[o];
      a.pio[o] = ADA ? (T)(pb - (double)a.cdt * Cc) : (T)pb;
    }
  }
  const T Cf = (T)Cc, Csf = (T)Cs;
  // loop-invariant products of the per-column factors
  const T kPc = r2A * rPc, kPu = r2A * rPuc, kPv = r2Av * rPvc;  // horizontal flux sums -> tendencies
  const T gU = Puc * rdx, gV = Pvc * rady;                         // pressure-gradient factors
  const T cota4 = T(0.25) * cota, f04 = T(0.25) * f0;             // a quarter of f* at the U point
  // the P^u partners of the divergences, fixed for the column
  const T puE = puR[t + dE], puW = puR[t + dW], pusE = puR[NTP + t + dgE], pusW = puR[NTP + t + dgW];
  row_sync(NTW);  // q2 (in the published-array buffers) is free again

  // ---- carries down the column
  T SD = 0, SDs = 0;                       // suffix sums of dsigma D, rows j and j+1
  T S = (T)(g.rt0pit[(size_t)j * I + gc] * a.pi[(size_t)j * I + gc]);   // psi suffix + R T~_s pi / pi~
  T Ss = hasS ? (T)(g.rt0pit[(size_t)(j + 1) * I + gc] * a.pi[(size_t)(j + 1) * I + gc]) : T(0);
  T Wb = 0, Wbp = 0, Wbs = 0;              // W at the bottom face of the level: own, c+1, row j+1
  T GsB = 0, GuB = 0, GvB = 0;             // G of the level below
  T PPh = 0, PU = 0, PV = 0;               // partial tendencies of the level below
  T pbU = 0, pbV = 0, pbPh = 0;            // base values of the level below
  T p_wc = 0, p_wu = 0, p_wv = 0, p_ds = 0;  // level below: r2ds / P at the scalar point, halved at the U and V points; dsigma
  double p_dsd = 0.0;
  double ubar = 0.0, vbar = 0.0;
  T dubar = 0, dvbar = 0;
  const T cdt = a.cdt;
  // element offsets fit 32 bits: nlon * nlat * nlev <= 4e9
  const unsigned plane = (unsigned)J * (unsigned)I, vplane = (unsigned)(J - 1) * (unsigned)I;
  const unsigned o_own = (unsigned)j * (unsigned)I + (unsigned)gc;
  // outputs of the own column, stepped down one plane per completed level
  // (the levels complete from the surface up, one after the other)
  T* oPhp = a.Phio + (size_t)K * plane + o_own;
  T* oUp = a.Uo + (size_t)K * plane + o_own;
  T* oVp = hasV ? a.Vo + (size_t)K * vplane + o_own : nullptr;

  // Complete level kk (its partials, base and bottom-face W are the carries)
  // with the top-face vertical flux, which needs G of the level above.
  auto complete = [&](T Gsc, T Guc, T Gvc) {
    const T TPh = PPh + (ADV ? (Wb * Gsc) * p_wc : T(0));
    const T TU = PU + (ADV ? ((Wb + Wbp) * Guc) * p_wu : T(0));
    const T bPh = MODE == 0 ? T(0) : pbPh, bU = MODE == 0 ? T(0) : pbU;
    const T oPh = bPh + cdt * TPh, oU = bU + cdt * TU;
    oPhp -= plane;
    oUp -= plane;
    if (owned) {
      *oPhp = oPh;
      *oUp = oU;
    }
    if (kInc)
      dubar += p_ds * (oU - bU);
    else
      ubar += p_dsd * (double)oU;
    if (hasV) {
      const T TV = PV + (ADV ? ((Wb + Wbs) * Gvc) * p_wv : T(0));
      const T bV = MODE == 0 ? T(0) : pbV;
      const T oV = bV + cdt * TV;
      oVp -= vplane;
      if (owned) *oVp = oV;
      if (kInc)
        dvbar += p_ds * (oV - bV);
      else
        vbar += p_dsd * (double)oV;
    }
  };

  // The level loop runs in pairs: with two ring slots, the level of
  // iteration q uses slot q % 2 and published buffer q % 2, so each half of a
  // pair has its slot and buffer fixed at compile time and the carries pass
  // from one half to the other without copies.
  static_assert(R == 2, "the level loop pairs the two ring slots");
  unsigned ph = 0;  // parity of the current use of both slots
  auto level = [&](const int k, auto SL) {
    constexpr int slot = decltype(SL)::value, buf = slot;
    mbar_wait_bounded(bar + slot, ph, abort_flag, a.err);
    const T* rw = ring + (size_t)slot * kRowRaw * NTP;
    const T* raw = rw + t;
    T* A = dA + (size_t)buf * kRowNP * NTP + t;
    T dsk, Hkk, hk, hkr, r2dsk, onems, rho;
    if constexpr (sizeof(T) == 4) {
      const float4 l0 = reinterpret_cast<const float4*>(lev)[2 * k];
      const float4 l1 = reinterpret_cast<const float4*>(lev)[2 * k + 1];
      dsk = l0.x; Hkk = l0.y; hk = l0.z; hkr = l0.w; r2dsk = l1.x; onems = l1.y; rho = l1.z;
    } else {
      const double2 l0 = reinterpret_cast<const double2*>(lev)[4 * k];
      const double2 l1 = reinterpret_cast<const double2*>(lev)[4 * k + 1];
      const double2 l2 = reinterpret_cast<const double2*>(lev)[4 * k + 2];
      const double2 l3 = reinterpret_cast<const double2*>(lev)[4 * k + 3];
      dsk = l0.x; Hkk = l0.y; hk = l1.x; hkr = l1.y; r2dsk = l2.x; onems = l2.y; rho = l3.x;
    }
    const double dsd = levd[k];
    // ---- own column: the published quantities, D, W and psi
    const T Un = raw[0 * NTP], Uc = raw[1 * NTP], Us = raw[2 * NTP];
    const T Phn = raw[3 * NTP], Phc = raw[4 * NTP], Phs = raw[5 * NTP];
    const T Vn = raw[6 * NTP], Vc = raw[7 * NTP], Vs = raw[8 * NTP];
    T nbU = 0, nbPh = 0, nbV = 0;
    if (MODE == 2) {
      nbU = raw[9 * NTP];
      nbPh = raw[10 * NTP];
      nbV = raw[11 * NTP];
    } else if (MODE == 1) {
      nbU = Uc;
      nbPh = Phc;
      nbV = Vc;
    }
    const T Gsc = Phc * rPc, Gsn = Phn * rPn, Gss = Phs * rPs;
    const T Guc = Uc * rPuc, Gun = Un * rPun, Gus = Us * rPus;
    const T Gvc = Vc * rPvc, Gvn = Vn * rPvn, Gvs = Vs * rPvs;
    const T FTn = sPvn * Vn, FTc = sPvc * Vc, FTs = sPvs * Vs;
    // leap divergence (a3) of rows j and j+1 from the staged U rows
    const T FLe = puE * raw[1 * NTP + dE], FLw = puW * raw[1 * NTP + dW];
    const T FLc = Puc * Uc, FLs = Pus * Us;
    const T fUc = (f0 + Guc * cota) * Uc, fUs = (f0s + Gus * cotas) * Us;
    const T FLse = pusE * raw[2 * NTP + dgE], FLsw = pusW * raw[2 * NTP + dgW];
    const T D = (FLe - FLw) * rdx + (FTc - FTn) * rdy;
    const T Ds = (FLse - FLsw) * rdxs + (FTs - FTc) * rdys;
    // a4: suffix sums -> W at the top face; a5: psi
    SD += dsk * D;
    SDs += dsk * Ds;
    const T Wt = SD - onems * Cf, Wts = SDs - onems * Csf;
    T Bc = Gsc, Bs = Gss;
    if (NL) {
      Bc *= one + rho * Gsc;
      Bs *= one + rho * Gss;
    }
    const T psi = Hkk * Bc + S, psis = Hkk * Bs + Ss;
    S += hk * Bc;
    Ss += hk * Bs;
    // publish (threads past the segment write slots nobody reads)
    A[0 * NTP] = Gsc;                     // G = Phi/P, row j
    A[1 * NTP] = Guc;                     // G = U/P^u, row j
    A[2 * NTP] = Gvc;                     // G = V/P^v, V row j
    A[3 * NTP] = FLc;                     // F^lambda, row j
    A[4 * NTP] = FLs;                     // F^lambda, row j+1
    A[5 * NTP] = FTn;                     // sin(theta^v) P^v V, V row j-1
    A[6 * NTP] = FTc;                     // sin(theta^v) P^v V, V row j
    A[7 * NTP] = Vn;                      // V, V row j-1
    A[8 * NTP] = Vc;                      // V, V row j
    A[9 * NTP] = fUc;                     // f* U, row j
    A[10 * NTP] = fUs;                    // f* U, row j+1
    A[11 * NTP] = psi;                    // psi, row j
    A[12 * NTP] = Wt;                     // W at the top face, row j
    // the level below is complete now that G of this level is known
    if (k + 1 <= K - 1) complete(Gsc, Guc, Gvc);  // level k + 1
    const T wc = r2dsk * rPc, wu = T(0.5) * r2dsk * rPuc, wv = T(0.5) * r2dsk * rPvc;
    row_sync(NTW);
    // every thread is past its reads of this ring slot: fetch level k - R into it
    if (k - R >= 0) issue_level(k - R, slot);
    // ---- the cells, from the leap partners' published values
    T nPPh, nPU, nPV = 0;
    {  // Phi cell: advection + Omega~ (a7, with Q_k = C - SD_k)
      const T hor = zf * (FLe * A[0 * NTP + de] - FLw * A[0 * NTP + dw]) + adl * (FTc * Gss - FTn * Gsn);
      const T X = -(NL ? rPc * (one + rho * Gsc) : rPc) * (Hkk * D + hkr * (Cf - SD));
      nPPh = (ADA ? X : T(0)) - (ADV ? hor * kPc + (Wb * GsB) * wc : T(0));
    }
    const T Wtp = A[12 * NTP + 1];
    {  // U cell
      const T FLW1 = (MC == 1) ? FLc : A[3 * NTP + dW1];   // (x-N+1) with N = 1 is the own column
      const T psiW1 = (MC == 1) ? psi : A[11 * NTP + dW1];
      const T ZE = zf2 * (FLe + A[3 * NTP + dE1]), ZW = zf2 * (FLw + FLW1);
      const T hor = ZE * A[1 * NTP + de] - ZW * A[1 * NTP + dw] +
                    adl2 * ((FTc + A[6 * NTP + 1]) * Gus - (FTn + A[5 * NTP + 1]) * Gun);
      const T pgf = gU * (A[11 * NTP + dE1] - psiW1);
      const T fs4 = f04 + Guc * cota4;
      const T vs = Vn + A[7 * NTP + 1] + Vc + A[8 * NTP + 1];
      nPU = (ADV ? -(hor * kPu + ((Wb + Wbp) * GuB) * wu) : T(0)) - (ADA ? pgf + fs4 * vs : T(0));
    }
    if (hasV) {  // V cell
      // with equal strides the V-cell faces are the divergence pairs of rows j and j+1
      const T ZE = MC ? zfv2 * (FLe + FLse) : zfv2 * (A[3 * NTP + dvE] + A[4 * NTP + dvE]);
      const T ZW = MC ? zfv2 * (FLw + FLsw) : zfv2 * (A[3 * NTP + dvW] + A[4 * NTP + dvW]);
      const T hor = ZE * A[2 * NTP + dve] - ZW * A[2 * NTP + dvw] +
                    adl2 * ((FTc + FTs) * Gvs - (FTn + FTc) * Gvn);
      const T pgf = gV * (psis - psi);
      const T cor = cn * (A[9 * NTP - 1] + fUc) + cs * (A[10 * NTP - 1] + fUs);
      nPV = (ADV ? -(hor * kPv + ((Wb + Wbs) * GvB) * wv) : T(0)) + (ADA ? cor - pgf : T(0));
    }
    PPh = nPPh;
    PU = nPU;
    PV = nPV;
    Wbp = Wtp;
    GsB = Gsc;
    GuB = Guc;
    GvB = Gvc;
    Wb = Wt;
    Wbs = Wts;
    p_wc = wc;
    p_wu = wu;
    p_wv = wv;
    p_ds = dsk;
    p_dsd = dsd;
    pbU = nbU;
    pbV = nbV;
    pbPh = nbPh;
  };
  int k = K - 1;
  for (; k >= 1; k -= 2) {
    level(k, std::integral_constant<int, 0>{});
    level(k - 1, std::integral_constant<int, 1>{});
    ph ^= 1u;
  }
  if (k == 0) level(0, std::integral_constant<int, 0>{});
  // level 0 has no level above: its top-face flux W_0 G_{-1} is zero
  complete(T(0), T(0), T(0));
  if (owned && a.Ubar_o) {
    if (kInc) {
      ubar = a.Ubar_b[o_own] + (double)dubar;
      if (hasV) vbar = a.Vbar_b[o_own] + (double)dvbar;
    }
    a.Ubar_o[o_own] = ubar;
    if (hasV) a.Vbar_o[o_own] = vbar;
  }
  // after a timeout, wait (bounded) for the copies still in flight before the
  // CTA's shared memory is released: the last R levels' phases, then one more
  // millisecond (copies take microseconds)
  if (t == 0 && *abort_flag) {
    // the level of iteration q sits in slot q % R, use q / R; every level is
    // issued, the last at iteration K - 1
    for (int q = K - 1; q >= 0 && q > K - 1 - R; --q) {
      const long long t0 = clock64();
      while (!mbar_try(bar + q % R, (unsigned)((q / R) & 1)) && clock64() - t0 < 2000000000LL) {
      }
    }
    const long long t1 = clock64();
    while (clock64() - t1 < 2000000LL) {
    }
  }
}

// One work item per CTA: a.rows[blockIdx.x] = row j << 8 | segment.
template <class T, int MODE, int TERMS, bool NL, int MC>
__global__ void __launch_bounds__(kRowB, sizeof(T) == 4 ? AGCM_ROW_MINB : 2)
    k_row_stage(const Geom<T> g, const RowArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int item = a.rows[blockIdx.x];
  row_segment<T, MODE, TERMS, NL, MC>(g, a, item >> 8, item & 255, smem, true);
}

}  // namespace agcm
