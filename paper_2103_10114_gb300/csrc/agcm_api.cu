// agcm_api.cu — implementation of the C ABI declared in include/agcm.h.
//
// Host side: grid geometry (Eq. 7 leap strides, metric terms, sigma tables,
// the standard stratification), the CFL time step, device memory, the
// three-stage step driver (unsplit and split), the low-latitude filters, the
// adjoint driver, the diagnostics, ensembles and the allocation-free
// tendency.  Device side: the kernels in agcm_fused.cuh (the stage),
// agcm_phases.cuh / agcm_adjoint.cuh (the adjoint), agcm_diag.cuh,
// agcm_ensemble.cuh and agcm_filter.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/agcm.h"
#include "agcm_common.cuh"
#include "agcm_phases.cuh"
#include "agcm_fused.cuh"
#include "agcm_row.cuh"
#include "agcm_adjoint.cuh"
#include "agcm_diag.cuh"
#include "agcm_ensemble.cuh"
#include "agcm_filter.cuh"

namespace {

// ---------------------------------------------------------------- errors
thread_local std::string t_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) return fail(AGCM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

std::atomic<uint64_t> g_grid_uid{0};

// Stage kernel choice (agcm_set_stage_kernel): 0 = by grid, 1 = column kernel,
// 2 = row-segment kernel wherever the rows allow it.
std::atomic<int> g_stage_choice{0};

// Whether `items` row-segment CTAs make at least two waves on the current
// device (three resident CTAs per SM); smaller grids run the column kernel,
// whose one-warp blocks give more parallelism (measured on GB300: 720x360
// rows, 2.3 waves, 0.165 against 0.185 ms per FP32 stage; 256x128, half a
// wave, 0.072 against 0.043 ms).
inline int rows_fill_device(long long items) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return items >= 2LL * 3 * nsm ? 1 : 0;
}

// Guards every grid's lazily built device tables and its count of live
// states and ensembles, so that states may be created and destroyed from
// several host threads.
std::mutex g_grid_mu;

// ---------------------------------------------------------------- allocator
agcm_alloc_fn g_alloc = nullptr;
agcm_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc((uint64_t)bytes, g_alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(void* p) {
  if (!p) return;
  if (g_free)
    g_free(p, g_alloc_ctx);
  else
    cudaFree(p);
}

// ---------------------------------------------------------------- constants
// Reading R2: only the Earth radius is fixed by the paper (zonal grid-size table).
constexpr double kA = 6.371e6;
constexpr double kOmega = 7.292e-5;
constexpr double kR = 287.04;
constexpr double kCp = 1004.64;
constexpr double kT0 = 250.0;     // default isothermal standard stratification [K]
constexpr double kG = 9.80665;    // gravity, for the lapse-rate standard atmosphere
constexpr double kPi = 3.14159265358979323846;

// Eq. 7 with cos(90deg - theta) = sin(theta) and res = dlam, rounded up to an
// integer >= 1 (ratios within 1e-9 of an integer count as that integer) and
// then to the next odd number (U sits on half points, so the stride is odd).
int eq7_stride(double theta, double dlam) {
  const double ref = std::asin(std::sqrt(0.5) * std::sin(dlam));
  const double here = std::asin(std::sin(theta) * std::sin(dlam));
  int n = (int)std::ceil(ref / here - 1e-9);
  n = std::max(n, 1);
  return (n & 1) ? n : n + 1;
}

}  // namespace

// ---------------------------------------------------------------- objects
struct DevGeomBlob {
  void* blob = nullptr;
  bool ready = false;
};

struct agcm_grid {
  int I = 0, J = 0, K = 0;
  // process-unique id of the grid's tables, renewed when they change
  // (agcm_grid_set_thermo): the allocation-free tendency keeps the last
  // grid's device tables and rebuilds them only when this id changes
  uint64_t uid = 0;
  double dlam = 0, dth = 0;
  std::vector<double> s, c, cot, A, sv, Av, sh, ds, Hkk, hk, pit;
  // thermodynamics (agcm_grid_set_thermo): surface geopotential, the level
  // coefficients beta_k = (1 - delta_p)(1 + delta_c) b_k, beta2 = (1 - delta_p)
  // delta kappa, and R T~_s of each column
  std::vector<double> phis, beta, rts;
  double beta2 = 0;
  agcm_thermo_t th{0, kT0, 288.15, 6.5e-3, 216.65, 0.0, 0.0, 0.0};
  std::vector<int> Mu, Mv;
  // device copies of the tables, per precision (0 = FP64, 1 = FP32)
  DevGeomBlob dev[2];
  agcm::Geom<double> gd{};
  agcm::Geom<float> gf{};
  int device = -1;
  int refs = 0;
};

// Kernel ids for the per-kernel event timing.
enum KernelId : int {
  KID_COLSTATE = 0,
  KID_VSUM,
  KID_FUSED,
  KID_DIAG,
  KID_ADJ_COL,
  KID_ADJ_GATHER,
  KID_ADJ_COLSTATE,
  KID_ENSEMBLE,
  KID_FILTER,
  KID_COUNT
};
static const char* const kKernelNames[KID_COUNT] = {
    "k_colstate", "k_vsum", "k_fused_stage", "k_diag",
    "k_adj_col", "k_adj_gather", "k_adj_colstate", "k_ensemble", "k_filter"};

struct Profiler {
  bool on = false;
  struct Rec { int id; cudaEvent_t a, b; int nl; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[KID_COUNT] = {};
  int64_t n[KID_COUNT] = {};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int id, cudaStream_t st) {
    if (!on) return;
    Rec r{id, get(), get(), 1};
    cudaEventRecord(r.a, st);
    recs.push_back(r);
  }
  // nlaunch: kernel launches inside the bracket (a stage of the stage kernel
  // may be two concurrent launches)
  void end(cudaStream_t st, int nlaunch = 1) {
    if (!on || recs.empty()) return;
    cudaEventRecord(recs.back().b, st);
    recs.back().nl = nlaunch;
  }
  int drain() {
    for (auto& r : recs) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) return 1;
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.id] += t;
      n[r.id] += r.nl;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
    return 0;
  }
  void reset() {
    drain();
    for (int q = 0; q < KID_COUNT; ++q) { ms[q] = 0; n[q] = 0; }
  }
  ~Profiler() {
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

constexpr int kSide = 5;  // side streams of a state

struct agcm_state {
  Profiler prof;
  const agcm_grid* grid = nullptr;
  int stage_choice = 0;  // 0: the process's agcm_set_stage_kernel; 1 column; 2 row segments
  int prec = AGCM_FP64;
  size_t esz = 8;
  size_t n3 = 0, nv = 0, n2 = 0;
  // prognostic x_n and the stage states x1, x2 (U, V, Phi, pi packed)
  void* x[3][4] = {};
  // adjoint forward-recompute scratch (allocated with the adjoint workspace):
  // P, rP, Pu, rPu, Pv, rPv (2-D), W ((K+1) planes), psi
  void* col[6] = {};
  void* W = nullptr;
  void* psi = nullptr;
  // FP64 vertical means sum_k dsigma U_k and V_k of x[0..2] (J*I each), the
  // input of the fused stage kernel's column integral; bar_valid for x[0]
  double* ubar[3] = {};
  double* vbar[3] = {};
  bool bar_valid = false;
  // diagnostics partials
  double* diag = nullptr;
  int* err = nullptr;  // device status word: AGCM_ETIMEOUT if a bounded wait gave up
  // side streams for the launches of a stage (and of an adjoint product) that
  // run beside the one on the caller's stream: forked from it by ev_fork,
  // joined to it by ev_join[q]
  cudaStream_t aux[kSide] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
  std::vector<void*> owned;
  // adjoint workspace (allocated on the first agcm_step_adjoint call)
  bool adj_ready = false;
  void* adj3[2] = {};   // Db aPhi                                  (K*J*I)
  void* adj2[5] = {};   // arPcol aPiD mub mvb mcb                  (J*I)
  // rows of the adjoint gather: row-segment items (j << 8 | segment) of
  // k_adj_rows, and the rows left to k_adj_gather
  int* adj_items = nullptr;
  int n_adj_items = 0;
  int* adj_rows = nullptr;
  int n_adj_rows = 0;
  void* adj_part = nullptr;  // level-chunk partial sums of those rows (3 * chunks * rows * I)
  void* mu[2][4] = {};  // stage adjoints mu2, mu1
};

namespace {

// The longest run of rows j, 1 <= j <= J-3, whose stencil strides Mu_j, Mv_j
// and Mu_{j+1} are all 1 (the low-latitude band of Eq. 7): those rows run the
// stride-1 column body.  Empty (lo = hi = 0) when there is none.
inline void leap1_band(const agcm_grid* g, int* lo, int* hi) {
  int best_lo = 0, best_hi = 0;
  for (int j = 1; j <= g->J - 3;) {
    if (g->Mu[j] == 1 && g->Mv[j] == 1 && g->Mu[j + 1] == 1) {
      int e = j;
      while (e <= g->J - 3 && g->Mu[e] == 1 && g->Mv[e] == 1 && g->Mu[e + 1] == 1) ++e;
      if (e - j > best_hi - best_lo) {
        best_lo = j;
        best_hi = e;
      }
      j = e;
    } else {
      ++j;
    }
  }
  *lo = best_lo;
  *hi = best_hi;
}

// Work items of the row-segment stage kernel, j << 8 | segment, for every row
// whose halo leaves at least half of a CTA to owned columns (the grid's rows
// must be 16-byte aligned, i.e. nlon % 4 == 0), in three classes: rows whose
// strides Mu_j, Mv_j, Mu_{j+1} all equal kRowClsM[c] (1, 3, 5, 7), and the
// others (nk[c] items each, listed in that order); and the rows left to the
// column kernel.
inline void row_lists(const agcm_grid* g, std::vector<int>* rowk, std::vector<int>* rowc, int nk[agcm::kRowCls]) {
  std::vector<int> cls[agcm::kRowCls];
  rowc->clear();
  for (int j = 0; j < g->J; ++j) {
    const bool hv = j < g->J - 1;
    const int Mu = g->Mu[j], Mv = hv ? g->Mv[j] : Mu, M1 = hv ? g->Mu[j + 1] : Mu;
    const int H = agcm::row_halo(Mu, hv ? Mv : 1, hv ? M1 : 1);
    int n = 0, S = 0;
    agcm::row_segments(g->I, H, agcm::kRowB, &n, &S);
    if (g->I % 4 == 0 && n > 0 && n < 256) {
      // the last row has no V row: always the general class
      int c = agcm::kRowCls - 1;
      if (hv && Mu == Mv && Mu == M1)
        for (int q = 0; q + 1 < agcm::kRowCls; ++q)
          if (Mu == agcm::kRowClsM[q]) c = q;
      for (int q = 0; q < n; ++q)
        if (q * S < g->I) cls[c].push_back(j << 8 | q);
    } else {
      rowc->push_back(j);
    }
  }
  rowk->clear();
  for (int c = 0; c < agcm::kRowCls; ++c) {
    nk[c] = (int)cls[c].size();
    rowk->insert(rowk->end(), cls[c].begin(), cls[c].end());
  }
}

template <class T>
int upload_geom(const agcm_grid* g, void** blob_out, agcm::Geom<T>* geom_out) {
  const int I = g->I, J = g->J, K = g->K;
  // pack every table into one allocation
  std::vector<char> host;
  auto put = [&](const void* src, size_t bytes) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + bytes);
    std::memcpy(host.data() + off, src, bytes);
    return off;
  };
  auto putT = [&](const std::vector<double>& v) {
    std::vector<T> t(v.begin(), v.end());
    return put(t.data(), t.size() * sizeof(T));
  };
  auto putD = [&](const std::vector<double>& v) { return put(v.data(), v.size() * sizeof(double)); };
  auto putI = [&](const std::vector<int>& v) { return put(v.data(), v.size() * sizeof(int)); };

  std::vector<double> rdx(J), rdy(J), zf(J), r2A(J), f0(J), cota(J);
  for (int j = 0; j < J; ++j) {
    rdx[j] = 1.0 / (kA * g->s[j] * g->Mu[j] * g->dlam);
    rdy[j] = 1.0 / (kA * g->s[j] * g->dth);
    zf[j] = kA * g->dth / g->Mu[j];
    r2A[j] = 0.5 / g->A[j];
    f0[j] = 2.0 * kOmega * g->c[j];
    cota[j] = g->cot[j] / kA;
  }
  const int JV = J - 1;
  std::vector<double> yv(JV), zfv(JV), r2Av(JV), cn(JV), cs(JV);
  for (int j = 0; j < JV; ++j) {
    yv[j] = kA * g->dlam * g->sv[j];
    zfv[j] = kA * g->dth / g->Mv[j];
    r2Av[j] = 0.5 / g->Av[j];
    cn[j] = 0.25 * g->A[j] / g->Av[j];
    cs[j] = 0.25 * g->A[j + 1] / g->Av[j];
  }
  // the hydrostatic weights carry the level coefficient beta_k (Eq. 1's
  // (1 - delta_p) b (1 + delta_c)), so no kernel multiplies by b; rho_k =
  // beta2 / beta_k scales the delta kappa Phi/P part relative to it
  std::vector<double> r2ds(K), Hkkb(K), hkb(K), hk_rds(K), oms(K), rho(K);
  for (int k = 0; k < K; ++k) {
    r2ds[k] = 0.5 / g->ds[k];
    Hkkb[k] = g->beta[k] * g->Hkk[k];
    hkb[k] = g->beta[k] * g->hk[k];
    hk_rds[k] = g->beta[k] * g->hk[k] / g->ds[k];
    oms[k] = 1.0 - g->sh[k];
    rho[k] = g->beta[k] != 0.0 ? g->beta2 / g->beta[k] : 0.0;
  }
  // low-latitude filter bands (Table "Conventional Filtering scheme")
  auto band_of = [](double colat) {
    const double lat = std::fabs(90.0 - colat * 180.0 / kPi);
    return lat < 38.0 ? 1 : (lat <= 70.0 ? 2 : 0);
  };
  std::vector<int> filtU, filtV;  // the two-grid removal needs an even nlon
  for (int j = 0; j < J; ++j) {
    const int bnd = band_of((j + 0.5) * g->dth);
    if (bnd == 2 || (bnd == 1 && I % 2 == 0)) filtU.push_back(4 * j + bnd);
  }
  for (int j = 0; j < JV; ++j) {
    const int bnd = band_of((j + 1.0) * g->dth);
    if (bnd == 2 || (bnd == 1 && I % 2 == 0)) filtV.push_back(4 * j + bnd);
  }
  const int nfU = (int)filtU.size(), nfV = (int)filtV.size();
  filtU.push_back(0);
  filtV.push_back(0);
  std::vector<double> rt0pit((size_t)J * I);
  for (size_t n = 0; n < rt0pit.size(); ++n) rt0pit[n] = g->rts[n] / g->pit[n];

  size_t o_Mu = putI(g->Mu), o_rdx = putT(rdx), o_rdy = putT(rdy), o_zf = putT(zf), o_r2A = putT(r2A),
         o_f0 = putT(f0), o_cota = putT(cota);
  std::vector<int> MvPad(g->Mv);
  if (MvPad.empty()) MvPad.push_back(1);
  size_t o_Mv = putI(MvPad), o_sv = putT(g->sv.empty() ? std::vector<double>{0} : g->sv),
         o_yv = putT(yv.empty() ? std::vector<double>{0} : yv),
         o_zfv = putT(zfv.empty() ? std::vector<double>{0} : zfv),
         o_r2Av = putT(r2Av.empty() ? std::vector<double>{0} : r2Av),
         o_cn = putT(cn.empty() ? std::vector<double>{0} : cn),
         o_cs = putT(cs.empty() ? std::vector<double>{0} : cs);
  size_t o_ds = putT(g->ds), o_r2ds = putT(r2ds), o_hk = putT(hkb), o_Hkk = putT(Hkkb),
         o_hkr = putT(hk_rds), o_oms = putT(oms), o_rho = putT(rho), o_dsd = putD(g->ds), o_shd = putD(g->sh), o_Ad = putD(g->A),
         o_Avd = putD(g->Av.empty() ? std::vector<double>{0} : g->Av);
  size_t o_rt0 = putT(rt0pit), o_pit = putT(g->pit);
  size_t o_bu = putI(filtU), o_bv = putI(filtV);
  std::vector<int> rowk, rowc;
  int nk[agcm::kRowCls];
  row_lists(g, &rowk, &rowc, nk);
  const int nrowc = (int)rowc.size();
  rowk.push_back(0);
  rowc.push_back(0);
  size_t o_rk = putI(rowk), o_rc = putI(rowc);

  void* d = dev_alloc(host.size());
  if (!d) return fail(AGCM_ENOMEM, "device allocation of %zu bytes for the grid tables failed", host.size());
  if (cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    dev_free(d);
    return fail(AGCM_ECUDA, "copy of the grid tables failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  char* base = (char*)d;
  agcm::Geom<T> G{};
  G.I = I; G.J = J; G.K = K;
  G.Mu = (const int*)(base + o_Mu);
  G.rdx = (const T*)(base + o_rdx);
  G.rdy = (const T*)(base + o_rdy);
  G.zf = (const T*)(base + o_zf);
  G.r2A = (const T*)(base + o_r2A);
  G.f0 = (const T*)(base + o_f0);
  G.cota = (const T*)(base + o_cota);
  G.Mv = (const int*)(base + o_Mv);
  G.sv = (const T*)(base + o_sv);
  G.yv = (const T*)(base + o_yv);
  G.zfv = (const T*)(base + o_zfv);
  G.r2Av = (const T*)(base + o_r2Av);
  G.cn = (const T*)(base + o_cn);
  G.cs = (const T*)(base + o_cs);
  G.ds = (const T*)(base + o_ds);
  G.r2ds = (const T*)(base + o_r2ds);
  G.hk = (const T*)(base + o_hk);
  G.Hkk = (const T*)(base + o_Hkk);
  G.hk_rds = (const T*)(base + o_hkr);
  G.oms = (const T*)(base + o_oms);
  G.filtU = (const int*)(base + o_bu);
  G.filtV = (const int*)(base + o_bv);
  G.nfU = nfU;
  G.nfV = nfV;
  G.dsd = (const double*)(base + o_dsd);
  G.shd = (const double*)(base + o_shd);
  G.Ad = (const double*)(base + o_Ad);
  G.Avd = (const double*)(base + o_Avd);
  G.rt0pit = (const T*)(base + o_rt0);
  G.pit = (const T*)(base + o_pit);
  G.rho = (const T*)(base + o_rho);
  G.nl = g->beta2 != 0.0 && g->th.delta != 0.0;
  leap1_band(g, &G.l1lo, &G.l1hi);
  G.rady = (T)(1.0 / (kA * g->dth));
  G.adl = (T)(kA * g->dlam);
  G.rowk = (const int*)(base + o_rk);
  G.rowc = (const int*)(base + o_rc);
  long long nitems = 0;
  for (int c = 0; c < agcm::kRowCls; ++c) nitems += G.nk[c] = nk[c];
  G.nrowc = nrowc;
  G.rowfill = rows_fill_device(nitems);
  *blob_out = d;
  *geom_out = G;
  return AGCM_OK;
}

int ensure_geom(const agcm_grid* cg, int prec) {
  agcm_grid* g = const_cast<agcm_grid*>(cg);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g->dev[prec].ready) {
      if (g->device != dev)
        return fail(AGCM_EINVAL, "grid tables live on device %d, current device is %d", g->device, dev);
      return AGCM_OK;
    }
    if (g->device >= 0 && g->device != dev)
      return fail(AGCM_EINVAL, "grid tables live on device %d, current device is %d", g->device, dev);
  }
  // The upload allocates through the allocator hook, which may call back into
  // the embedding runtime (and from there into this library, e.g. a garbage
  // collector destroying another state): it runs without the lock held.
  void* blob = nullptr;
  agcm::Geom<double> gd{};
  agcm::Geom<float> gf{};
  int rc = prec == AGCM_FP64 ? upload_geom<double>(g, &blob, &gd) : upload_geom<float>(g, &blob, &gf);
  if (rc) return rc;
  bool lost = false;
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g->dev[prec].ready) {
      lost = true;  // another thread published first
    } else {
      g->device = dev;
      g->dev[prec].blob = blob;
      if (prec == AGCM_FP64)
        g->gd = gd;
      else
        g->gf = gf;
      g->dev[prec].ready = true;
    }
  }
  if (lost) dev_free(blob);
  return AGCM_OK;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline unsigned nblocks(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <class T>
const agcm::Geom<T>& geom_of(const agcm_state* s) {
  if constexpr (sizeof(T) == 8)
    return s->grid->gd;
  else
    return s->grid->gf;
}

// FP64 vertical means of x[0] (needed once after a load).
template <class T>
int ensure_bar(agcm_state* s, cudaStream_t st) {
  if (s->bar_valid) return AGCM_OK;
  const agcm::Geom<T>& G = geom_of<T>(s);
  s->prof.begin(KID_VSUM, st);
  agcm::k_vsum<T><<<nblocks(s->n2, 256), 256, 0, st>>>(G, (const T*)s->x[0][0], (const T*)s->x[0][1], s->ubar[0],
                                                       s->vbar[0]);
  s->prof.end(st);
  CUDA_TRY(cudaGetLastError());
  s->bar_valid = true;
  return AGCM_OK;
}

// One stage: out = base + cdt * T(x[in]) (MODE 1: base = x[in]; MODE 2:
// base = x[0]; MODE 0: out = T).  Writes the vertical means of out to
// bar[outb] (outb < 0: not written).
//
// Two designs of the stage kernel.  The row-segment kernel (agcm_row.cuh)
// takes every row whose leap halo fits a CTA, when the rows are 16-byte
// aligned; the few rows it leaves (the ones next to the poles on fine grids)
// run the column kernel (agcm_fused.cuh, PART 3).  Grids or buffers the
// row-segment kernel cannot take run the column kernel on every row, as the
// stride-1 band (PART 2, specialised body) and the other rows (PART 1).
// Given aux, evf and evj (kSide side streams, a fork event and one join event
// per side stream), launches other than the first run on side streams,
// forked from st after everything already queued there and joined back
// before st continues, so they overlap; without them they run one after the
// other on st.  *launched (optional) receives the number of kernel launches
// made.
#ifndef AGCM_ROW_KERNEL
#define AGCM_ROW_KERNEL 1
#endif
template <class T, int MODE, int TERMS = 3>
int launch_fused(const agcm::Geom<T>& G, const void* const xs[4], const double* ub, const double* vb,
                 const void* const xb[4], void* const out[4], double* ubo, double* vbo, const double* ubb,
                 const double* vbb, double cdt, int* err, cudaStream_t st, const cudaStream_t* aux = nullptr,
                 cudaEvent_t evf = nullptr, const cudaEvent_t* evj = nullptr, int* launched = nullptr,
                 int state_choice = 0) {
  if (launched) *launched = 1;
  const bool fork = aux && evf && evj;
  auto col_launch = [&](auto nl, auto part, int ny, cudaStream_t q) {
    const unsigned gx = (unsigned)((G.I + agcm::kTileX - 1) / agcm::kTileX);
    agcm::k_fused_stage<T, MODE, TERMS, decltype(nl)::value, decltype(part)::value>
        <<<dim3(gx, (unsigned)ny), agcm::kTileX, 0, q>>>(
            G, (const T*)xs[0], (const T*)xs[1], (const T*)xs[2], (const T*)xs[3], ub, vb, (const T*)xb[0],
            (const T*)xb[1], (const T*)xb[2], (const T*)xb[3], (T*)out[0], (T*)out[1], (T*)out[2], (T*)out[3],
            ubo, vbo, ubb, vbb, (T)cdt);
  };
  auto two = [&](auto first, auto second) -> int {  // first on aux[0] (forked), second on st
    if (fork) {
      CUDA_TRY(cudaEventRecord(evf, st));
      CUDA_TRY(cudaStreamWaitEvent(aux[0], evf, 0));
    }
    first(fork ? aux[0] : st);
    second(st);
    if (fork) {
      CUDA_TRY(cudaEventRecord(evj[0], aux[0]));
      CUDA_TRY(cudaStreamWaitEvent(st, evj[0], 0));
    }
    if (launched) *launched = 2;
    return AGCM_OK;
  };
  auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  // a state's own choice (agcm_state_set_stage_kernel), else the process's
  const int choice = state_choice > 0 ? state_choice : g_stage_choice.load(std::memory_order_relaxed);
  int nitems = 0;
  for (int c = 0; c < agcm::kRowCls; ++c) nitems += G.nk[c];
  bool rowpath = AGCM_ROW_KERNEL && choice != 1 && (choice == 2 || G.rowfill) && nitems > 0 &&
                 a16(xs[0]) && a16(xs[1]) && a16(xs[2]);
  if (MODE == 2) rowpath = rowpath && a16(xb[0]) && a16(xb[1]) && a16(xb[2]);
  const size_t smem = agcm::row_smem_bytes<T>(agcm::kRowB, G.K);
  if (smem > 227 * 1024) rowpath = false;
  auto rows = [&](auto nl) -> int {
    if (rowpath) {
      agcm::RowArgs<T> ra{(const T*)xs[0], (const T*)xs[1], (const T*)xs[2], (const T*)xs[3], ub, vb,
                          (const T*)xb[0], (const T*)xb[1], (const T*)xb[2], (const T*)xb[3], (T*)out[0],
                          (T*)out[1], (T*)out[2], (T*)out[3], ubo, vbo, ubb, vbb, (T)cdt, G.rowk, err};
      int nlaunch = 0;
      // one launch per stride class, or one over classes [c0, c1) (the
      // body for any strides); class c's items follow those of the classes before it
      auto cls_go = [&](auto mc, int c0, int c1, cudaStream_t q) -> int {
        int off = 0, n = 0;
        for (int c = 0; c < c1; ++c) (c < c0 ? off : n) += G.nk[c];
        if (n == 0) return AGCM_OK;
        auto kern = agcm::k_row_stage<T, MODE, TERMS, decltype(nl)::value, decltype(mc)::value>;
        static std::atomic<size_t> attr{0};  // per instantiation: the size set so far
        if (attr.load() < smem) {
          CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr.store(smem);
        }
        agcm::RowArgs<T> rc = ra;
        rc.rows = G.rowk + off;
        kern<<<(unsigned)n, agcm::kRowB, smem, q>>>(G, rc);
        ++nlaunch;
        return AGCM_OK;
      };
      // the launches run side by side: the stride-1 rows on st, the rows
      // next to the poles (column kernel), the stride-3, 5 and 7 rows and
      // the other rows each on a side stream (a launch of less than a
      // wave then no longer waits for another's last wave).  They are issued
      // longest block first (the column kernel's level walk, then the rows
      // with the widest halos), and the side streams' priorities keep that
      // order, so that the shortest blocks fill the last wave.  The stride-5
      // and 7 classes have bodies of their own in the stages of a step; the
      // tendency and the split term groups take them with the other rows.
      constexpr bool kSpec = MODE != 0 && TERMS == 3;
      constexpr int cAny = agcm::kRowCls - 1;
      const int cOther = kSpec ? cAny : 2;
      int nOther = 0;
      for (int c = cOther; c < agcm::kRowCls; ++c) nOther += G.nk[c];
      const bool side[kSide] = {G.nrowc > 0, G.nk[1] > 0, nOther > 0, kSpec && G.nk[2] > 0, kSpec && G.nk[3] > 0};
      if (fork) {
        CUDA_TRY(cudaEventRecord(evf, st));
        for (int q = 0; q < kSide; ++q)
          if (side[q]) CUDA_TRY(cudaStreamWaitEvent(aux[q], evf, 0));
      }
      if (G.nrowc > 0) {
        col_launch(nl, std::integral_constant<int, 3>{}, G.nrowc, fork ? aux[0] : st);
        ++nlaunch;
      }
      int rc = cls_go(std::integral_constant<int, 0>{}, cOther, agcm::kRowCls, fork ? aux[2] : st);
      if (!rc) rc = cls_go(std::integral_constant<int, 3>{}, 1, 2, fork ? aux[1] : st);
      if constexpr (kSpec) {
        if (!rc) rc = cls_go(std::integral_constant<int, 7>{}, 3, 4, fork ? aux[4] : st);
        if (!rc) rc = cls_go(std::integral_constant<int, 5>{}, 2, 3, fork ? aux[3] : st);
      }
      if (!rc) rc = cls_go(std::integral_constant<int, 1>{}, 0, 1, st);
      if (fork) {  // joined whatever rc says, so that no side stream is left forked
        for (int q = 0; q < kSide; ++q)
          if (side[q]) {
            CUDA_TRY(cudaEventRecord(evj[q], aux[q]));
            CUDA_TRY(cudaStreamWaitEvent(st, evj[q], 0));
          }
      }
      if (rc) return rc;
      if (launched) *launched = nlaunch;
    } else {
      const int nb = G.l1hi - G.l1lo;
      if (nb <= 0) {
        col_launch(nl, std::integral_constant<int, 0>{}, G.J, st);
      } else if (nb == G.J) {
        col_launch(nl, std::integral_constant<int, 2>{}, nb, st);
      } else {
        int rc = two([&](cudaStream_t q) { col_launch(nl, std::integral_constant<int, 2>{}, nb, q); },
                     [&](cudaStream_t q) { col_launch(nl, std::integral_constant<int, 1>{}, G.J - nb, q); });
        if (rc) return rc;
      }
    }
    CUDA_TRY(cudaGetLastError());
    return AGCM_OK;
  };
  // the delta kappa Phi/P term touches only the adaptation terms
  if constexpr ((TERMS & 2) != 0) {
    if (G.nl) return rows(std::true_type{});
  }
  return rows(std::false_type{});
}

template <class T, int MODE, int TERMS = 3>
int fused_stage(agcm_state* s, int in, void* const out[4], int outb, double cdt, cudaStream_t st) {
  const agcm::Geom<T>& G = geom_of<T>(s);
  s->prof.begin(KID_FUSED, st);
  int launched = 1;
  int rc = launch_fused<T, MODE, TERMS>(G, s->x[in], s->ubar[in], s->vbar[in], s->x[0], out,
                                 outb >= 0 ? s->ubar[outb] : nullptr, outb >= 0 ? s->vbar[outb] : nullptr,
                                 s->ubar[0], s->vbar[0], cdt, s->err, st, s->aux, s->ev_fork, s->ev_join,
                                 &launched, s->stage_choice);
  s->prof.end(st, launched);
  return rc;
}

template <class T>
int run_steps(agcm_state* s, int nsteps, double dt, cudaStream_t st) {
  if (sizeof(T) == 4) s->bar_valid = false;  // exact means once per call in FP32
  int rc = ensure_bar<T>(s, st);
  if (rc) return rc;
  for (int n = 0; n < nsteps; ++n) {
    if ((rc = fused_stage<T, 1>(s, 0, s->x[1], 1, 0.5 * dt, st))) return rc;
    if ((rc = fused_stage<T, 2>(s, 1, s->x[2], 2, 0.5 * dt, st))) return rc;
    if ((rc = fused_stage<T, 2>(s, 2, s->x[0], 0, dt, st))) return rc;
  }
  return AGCM_OK;
}

// Split stepping (Sec. "Optimizations": A_F is called 3 M times and L_F 3
// times per step, reading the labels as A = adaptation, L = advection): per
// step, msub three-stage steps of the adaptation terms with dt/msub, then one
// three-stage step of the advection terms with dt.
template <class T, int TERMS>
int three_stage(agcm_state* s, double dt, cudaStream_t st) {
  int rc;
  if ((rc = fused_stage<T, 1, TERMS>(s, 0, s->x[1], 1, 0.5 * dt, st))) return rc;
  if ((rc = fused_stage<T, 2, TERMS>(s, 1, s->x[2], 2, 0.5 * dt, st))) return rc;
  return fused_stage<T, 2, TERMS>(s, 2, s->x[0], 0, dt, st);
}

template <class T>
int run_steps_split(agcm_state* s, int nsteps, double dt, int msub, cudaStream_t st) {
  if (sizeof(T) == 4) s->bar_valid = false;
  int rc = ensure_bar<T>(s, st);
  if (rc) return rc;
  for (int n = 0; n < nsteps; ++n) {
    for (int m = 0; m < msub; ++m)
      if ((rc = three_stage<T, 2>(s, dt / msub, st))) return rc;
    if ((rc = three_stage<T, 1>(s, dt, st))) return rc;
  }
  return AGCM_OK;
}

template <class T>
int run_tendency(agcm_state* s, void* const out[4], cudaStream_t st) {
  int rc = ensure_bar<T>(s, st);
  if (rc) return rc;
  return fused_stage<T, 0>(s, 0, out, -1, 1.0, st);
}


template <class T>
int diagnostics(const agcm_state* s, double h[8], cudaStream_t st) {
  const agcm::Geom<double>& G = s->grid->gd;
  const int nb = agcm::kDiagPartials;
  agcm_state* sm = const_cast<agcm_state*>(s);
  sm->prof.begin(KID_DIAG, st);
  agcm::k_diag<T><<<nb, agcm::kDiagThreads, 0, st>>>(G, (const T*)s->x[0][0], (const T*)s->x[0][1],
                                                     (const T*)s->x[0][2], (const T*)s->x[0][3], s->diag);
  agcm::k_diag_final<<<1, agcm::kDiagThreads, 0, st>>>(s->diag, nb, s->diag + 8 * nb);
  sm->prof.end(st);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(h, s->diag + 8 * nb, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return AGCM_OK;
}

template <class T>
int adjoint_step(agcm_state* s, const void* const lam_in[4], void* const lam_out[4], double dt, cudaStream_t st);

}  // namespace

// ======================================================================= C ABI
extern "C" {

const char* agcm_last_error(void) { return t_err.c_str(); }

int agcm_version(void) { return 100; }

int agcm_set_allocator(agcm_alloc_fn alloc, agcm_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(AGCM_EINVAL, "alloc and free must both be set or both be NULL");
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return AGCM_OK;
}

// Standard stratification T~ at p/p0: isothermal, or a lapse-rate troposphere
// T~ = Ts0 (p/p0)^(R lapse/g) above an isothermal stratosphere at Ttrop.
static double std_temperature(const agcm_thermo_t& t, double p) {
  if (t.profile == 0) return t.T0;
  if (t.lapse == 0.0) return t.Ts0;
  return std::max(t.Ts0 * std::pow(p, kR * t.lapse / kG), t.Ttrop);
}

// Standard surface pressure / p0 and temperature under phis: hydrostatic
// balance of T~ from p0 at phi = 0 (closed forms of the two layers).
static void std_surface(const agcm_thermo_t& t, double phis, double& pit, double& Ts) {
  if (t.profile == 0 || t.lapse == 0.0) {
    Ts = t.profile == 0 ? t.T0 : t.Ts0;
    pit = std::exp(-phis / (kR * Ts));
    return;
  }
  const double z = phis / kG, n = kG / (kR * t.lapse), Tz = t.Ts0 - t.lapse * z;
  if (Tz >= t.Ttrop) {
    Ts = Tz;
    pit = std::pow(Tz / t.Ts0, n);
  } else {
    Ts = t.Ttrop;
    const double ztr = (t.Ts0 - t.Ttrop) / t.lapse;
    pit = std::pow(t.Ttrop / t.Ts0, n) * std::exp(-kG * (z - ztr) / (kR * t.Ttrop));
  }
}

// beta_k, beta2, pi~ and R T~_s of a grid from its thermodynamic settings.
static void thermo_tables(agcm_grid* g) {
  const agcm_thermo_t& t = g->th;
  const double kap = kR / kCp;
  g->beta.resize(g->K);
  for (int k = 0; k < g->K; ++k) {
    const double mid = 0.5 * (g->sh[k] + g->sh[k + 1]);
    g->beta[k] = (1.0 - t.delta_p) * (1.0 + t.delta_c) * std::sqrt(kap * kR * std_temperature(t, mid));
  }
  g->beta2 = (1.0 - t.delta_p) * t.delta * kap;
  g->pit.resize(g->phis.size());
  g->rts.resize(g->phis.size());
  for (size_t n = 0; n < g->phis.size(); ++n) {
    double Ts = 0.0;
    std_surface(t, g->phis[n], g->pit[n], Ts);
    g->rts[n] = kR * Ts;
  }
}

int agcm_grid_set_thermo(agcm_grid_t* g, const agcm_thermo_t* t) {
  if (!g) return fail(AGCM_EINVAL, "null grid");
  std::lock_guard<std::mutex> lk(g_grid_mu);
  if (g->dev[0].blob || g->dev[1].blob || g->refs > 0)
    return fail(AGCM_EINVAL, "agcm_grid_set_thermo: the grid already has device tables (call it before the first state)");
  agcm_thermo_t v{0, kT0, 288.15, 6.5e-3, 216.65, 0.0, 0.0, 0.0};
  if (t) v = *t;
  if ((v.profile != 0 && v.profile != 1) || !(v.T0 > 0) || !(v.Ts0 > 0) || !(v.Ttrop > 0) || v.Ttrop > v.Ts0 ||
      !(v.lapse >= 0) || !std::isfinite(v.lapse) || !std::isfinite(v.delta) || !(v.delta_c > -1.0) ||
      !std::isfinite(v.delta_c) || !(v.delta_p >= 0.0 && v.delta_p <= 1.0) || !std::isfinite(v.T0) ||
      !std::isfinite(v.Ts0))
    return fail(AGCM_EINVAL, "agcm_grid_set_thermo: value out of range");
  g->th = v;
  thermo_tables(g);
  g->uid = ++g_grid_uid;
  return AGCM_OK;
}

int agcm_grid_create(int nlon, int nlat, int nlev, const double* sigma_half, const int32_t* leap_u,
                     const int32_t* leap_v, const double* phis, agcm_grid_t** out) {
  if (!out) return fail(AGCM_EINVAL, "out is NULL");
  *out = nullptr;
  if (nlon < 3 || nlat < 2 || nlev < 1)
    return fail(AGCM_EINVAL, "need nlon >= 3, nlat >= 2, nlev >= 1 (got %d, %d, %d)", nlon, nlat, nlev);
  if ((double)nlon * nlat * nlev > 4.0e9)
    return fail(AGCM_EINVAL, "grid of %d x %d x %d points is too large", nlon, nlat, nlev);
  // column indices are 32-bit and the stage launch has one grid row per latitude
  if ((double)nlon * nlat > 1073741824.0 || nlat > 65535)
    return fail(AGCM_EINVAL, "nlon * nlat must be at most 2^30 and nlat at most 65535 (got %d x %d)", nlon, nlat);
  agcm_grid* g = new agcm_grid;
  const int I = nlon, J = nlat, K = nlev;
  g->I = I; g->J = J; g->K = K;
  g->dlam = 2.0 * kPi / I;
  g->dth = kPi / J;
  g->s.resize(J); g->c.resize(J); g->cot.resize(J); g->A.resize(J); g->Mu.resize(J);
  for (int j = 0; j < J; ++j) {
    const double th = (j + 0.5) * g->dth;
    g->s[j] = std::sin(th);
    g->c[j] = std::cos(th);
    g->cot[j] = g->c[j] / g->s[j];
    g->A[j] = kA * kA * g->s[j] * g->dth * g->dlam;
    g->Mu[j] = leap_u ? leap_u[j] : eq7_stride(th, g->dlam);
  }
  g->sv.resize(J - 1); g->Av.resize(J - 1); g->Mv.resize(J - 1);
  for (int j = 0; j < J - 1; ++j) {
    const double th = (j + 1.0) * g->dth;
    g->sv[j] = std::sin(th);
    g->Av[j] = kA * kA * g->sv[j] * g->dth * g->dlam;
    g->Mv[j] = leap_v ? leap_v[j] : eq7_stride(th, g->dlam);
  }
  for (int j = 0; j < J; ++j)
    if (g->Mu[j] < 1 || (g->Mu[j] & 1) == 0 || 2 * g->Mu[j] >= I) {
      int m = g->Mu[j];
      delete g;
      return fail(AGCM_EINVAL, "leap_u[%d] = %d: strides must be odd, >= 1 and below nlon/2", j, m);
    }
  for (int j = 0; j < J - 1; ++j)
    if (g->Mv[j] < 1 || (g->Mv[j] & 1) == 0 || 2 * g->Mv[j] >= I) {
      int m = g->Mv[j];
      delete g;
      return fail(AGCM_EINVAL, "leap_v[%d] = %d: strides must be odd, >= 1 and below nlon/2", j, m);
    }
  g->sh.resize(K + 1);
  for (int h = 0; h <= K; ++h) g->sh[h] = sigma_half ? sigma_half[h] : (double)h / K;
  if (g->sh[0] != 0.0 || g->sh[K] != 1.0) {
    delete g;
    return fail(AGCM_EINVAL, "sigma_half must start at 0 and end at 1");
  }
  g->ds.resize(K); g->Hkk.resize(K); g->hk.resize(K);
  for (int k = 0; k < K; ++k) {
    g->ds[k] = g->sh[k + 1] - g->sh[k];
    if (!(g->ds[k] > 0.0)) {
      delete g;
      return fail(AGCM_EINVAL, "sigma_half must increase strictly (level %d)", k);
    }
    const double mid = 0.5 * (g->sh[k] + g->sh[k + 1]);
    g->Hkk[k] = std::log(g->sh[k + 1] / mid);
    g->hk[k] = k > 0 ? std::log(g->sh[k + 1] / g->sh[k]) : 0.0;
  }
  g->phis.assign((size_t)J * I, 0.0);
  for (size_t n = 0; n < g->phis.size(); ++n) {
    const double p = phis ? phis[n] : 0.0;
    if (!std::isfinite(p)) {
      delete g;
      return fail(AGCM_EINVAL, "phis[%zu] is not finite", n);
    }
    g->phis[n] = p;
  }
  thermo_tables(g);  // the default isothermal 250 K atmosphere
  g->uid = ++g_grid_uid;
  *out = g;
  return AGCM_OK;
}

int agcm_grid_destroy(agcm_grid_t* g) {
  if (!g) return AGCM_OK;
  void* blobs[2] = {nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g->refs > 0) return fail(AGCM_EINVAL, "grid still has %d live states", g->refs);
    for (int p = 0; p < 2; ++p) blobs[p] = g->dev[p].blob;
  }
  for (void* b : blobs)
    if (b) dev_free(b);  // outside the lock: the free hook may call back into the library
  delete g;
  return AGCM_OK;
}

int agcm_grid_leap(const agcm_grid_t* g, int32_t* lu, int32_t* lv) {
  if (!g || !lu || (!lv && g->J > 1)) return fail(AGCM_EINVAL, "null argument");
  for (int j = 0; j < g->J; ++j) lu[j] = g->Mu[j];
  for (int j = 0; j < g->J - 1; ++j) lv[j] = g->Mv[j];
  return AGCM_OK;
}

int agcm_grid_dt(const agcm_grid_t* g, double umax, double* dt) {
  if (!g || !dt || !(umax >= 0.0)) return fail(AGCM_EINVAL, "bad argument");
  const int K = g->K;
  // S = D^{1/2} (H B^2 D^-1 H^T D + R T~_s 1 1^T D) D^{-1/2}, D = diag(dsigma),
  // B = diag(beta_k):
  // symmetric and positive semi-definite with the eigenvalues of the column
  // operator; its largest eigenvalue by power iteration.
  std::vector<double> H((size_t)K * K, 0.0);
  for (int k = 0; k < K; ++k) {
    H[(size_t)k * K + k] = g->Hkk[k];
    for (int kk = k + 1; kk < K; ++kk) H[(size_t)k * K + kk] = g->hk[kk];
  }
  std::vector<double> S((size_t)K * K, 0.0);
  double rt = 0.0;
  for (double v : g->rts) rt = std::max(rt, v);
  for (int p = 0; p < K; ++p)
    for (int q = 0; q < K; ++q) {
      double acc = 0.0;
      for (int m = 0; m < K; ++m)
        acc += H[(size_t)p * K + m] * g->beta[m] * g->beta[m] * H[(size_t)q * K + m] / g->ds[m];
      S[(size_t)p * K + q] = std::sqrt(g->ds[p] * g->ds[q]) * (acc + rt);
    }
  std::vector<double> v(K, 1.0), w(K);
  double lam = 0.0;
  for (int it = 0; it < 10000; ++it) {
    double nrm = 0.0;
    for (int p = 0; p < K; ++p) {
      double acc = 0.0;
      for (int q = 0; q < K; ++q) acc += S[(size_t)p * K + q] * v[q];
      w[p] = acc;
      nrm += acc * acc;
    }
    nrm = std::sqrt(nrm);
    double dot = 0.0;
    for (int p = 0; p < K; ++p) dot += v[p] * w[p];
    double vn = 0.0;
    for (int p = 0; p < K; ++p) vn += v[p] * v[p];
    const double est = dot / vn;
    for (int p = 0; p < K; ++p) v[p] = w[p] / nrm;
    if (it > 10 && std::fabs(est - lam) <= 1e-15 * std::fabs(est)) {
      lam = est;
      break;
    }
    lam = est;
  }
  const double cmax = std::sqrt(lam);
  const double kx = 2.0 / (kA * std::sqrt(0.5) * g->dlam), ky = 2.0 / (kA * g->dth);
  *dt = 1.6 / ((cmax + umax) * std::sqrt(kx * kx + ky * ky));
  return AGCM_OK;
}

static void release_streams(agcm_state* s) {
  for (int q = 0; q < kSide; ++q) {
    if (s->ev_join[q]) cudaEventDestroy(s->ev_join[q]);
    if (s->aux[q]) cudaStreamDestroy(s->aux[q]);
    s->ev_join[q] = nullptr;
    s->aux[q] = nullptr;
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  s->ev_fork = nullptr;
}

int agcm_state_create(const agcm_grid_t* g, int precision, int nmembers, agcm_state_t** out) {
  if (!g || !out) return fail(AGCM_EINVAL, "null argument");
  *out = nullptr;
  if (precision != AGCM_FP64 && precision != AGCM_FP32) return fail(AGCM_EINVAL, "precision must be AGCM_FP64 or AGCM_FP32");
  if (nmembers != 1) return fail(AGCM_EINVAL, "nmembers must be 1; ensembles use agcm_ensemble_*");
  int rc = ensure_geom(g, AGCM_FP64);
  if (!rc && precision == AGCM_FP32) rc = ensure_geom(g, AGCM_FP32);
  if (rc) return rc;
  agcm_state* s = new agcm_state;
  s->grid = g;
  s->prec = precision;
  s->esz = precision == AGCM_FP64 ? 8 : 4;
  const size_t I = g->I, J = g->J, K = g->K;
  s->n3 = K * J * I;
  s->nv = K * (J - 1) * I;
  s->n2 = J * I;
  auto get = [&](size_t bytes) -> void* {
    void* p = dev_alloc(bytes);
    if (p) s->owned.push_back(p);
    return p;
  };
  bool ok = true;
  for (int c = 0; c < 3 && ok; ++c) {
    ok = ok && (s->x[c][0] = get(s->n3 * s->esz));
    ok = ok && (s->x[c][1] = get(std::max<size_t>(s->nv, 1) * s->esz));
    ok = ok && (s->x[c][2] = get(s->n3 * s->esz));
    ok = ok && (s->x[c][3] = get(s->n2 * s->esz));
  }
  for (int c = 0; c < 3 && ok; ++c) {
    ok = ok && (s->ubar[c] = (double*)get(s->n2 * sizeof(double)));
    ok = ok && (s->vbar[c] = (double*)get(s->n2 * sizeof(double)));
  }
  ok = ok && (s->diag = (double*)get((agcm::kDiagPartials + 1) * 8 * sizeof(double)));
  ok = ok && (s->err = (int*)get(256));
  if (ok) cudaMemset(s->err, 0, sizeof(int));
  if (!ok) {
    for (void* p : s->owned) dev_free(p);
    delete s;
    return fail(AGCM_ENOMEM, "device allocation for a %zu x %zu x %zu state failed", I, J, K);
  }
  for (int c = 0; c < 3; ++c)
    for (int f = 0; f < 4; ++f) {
      size_t n = f == 1 ? std::max<size_t>(s->nv, 1) : (f == 3 ? s->n2 : s->n3);
      cudaMemset(s->x[c][f], 0, n * s->esz);
    }
  // side stream priorities: the rows next to the poles and the rows of any
  // strides (the widest halos, the longest blocks) first, then the stride-3,
  // 5 and 7 classes; the stride-1 class runs on the caller's stream
  int prio_least = 0, prio_greatest = 0;
  bool side_ok = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) == cudaSuccess &&
                 cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  const int prio_mid = (prio_least + prio_greatest) / 2;
  const int prio[kSide] = {prio_greatest, prio_mid, prio_greatest, prio_mid, prio_mid};
  for (int q = 0; q < kSide && side_ok; ++q)
    side_ok = cudaStreamCreateWithPriority(&s->aux[q], cudaStreamNonBlocking, prio[q]) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->ev_join[q], cudaEventDisableTiming) == cudaSuccess;
  if (!side_ok || cudaDeviceSynchronize() != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    release_streams(s);
    for (void* p : s->owned) dev_free(p);
    delete s;
    return fail(AGCM_ECUDA, "state initialisation failed: %s", cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    const_cast<agcm_grid*>(g)->refs++;
  }
  *out = s;
  return AGCM_OK;
}

int agcm_state_destroy(agcm_state_t* s) {
  if (!s) return AGCM_OK;
  cudaDeviceSynchronize();
  release_streams(s);
  for (void* p : s->owned) dev_free(p);
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    const_cast<agcm_grid*>(s->grid)->refs--;
  }
  delete s;
  return AGCM_OK;
}

int agcm_state_load(agcm_state_t* s, const void* U, const void* V, const void* Phi, const void* pi,
                    int on_device, void* stream) {
  if (!s || !U || !Phi || !pi || (!V && s->nv)) return fail(AGCM_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(s->x[0][0], U, s->n3 * s->esz, kind, st));
  if (s->nv) CUDA_TRY(cudaMemcpyAsync(s->x[0][1], V, s->nv * s->esz, kind, st));
  CUDA_TRY(cudaMemcpyAsync(s->x[0][2], Phi, s->n3 * s->esz, kind, st));
  CUDA_TRY(cudaMemcpyAsync(s->x[0][3], pi, s->n2 * s->esz, kind, st));
  s->bar_valid = false;
  return AGCM_OK;
}

int agcm_state_store(const agcm_state_t* s, void* U, void* V, void* Phi, void* pi, int on_device,
                     void* stream) {
  if (!s || !U || !Phi || !pi || (!V && s->nv)) return fail(AGCM_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(U, s->x[0][0], s->n3 * s->esz, kind, st));
  if (s->nv) CUDA_TRY(cudaMemcpyAsync(V, s->x[0][1], s->nv * s->esz, kind, st));
  CUDA_TRY(cudaMemcpyAsync(Phi, s->x[0][2], s->n3 * s->esz, kind, st));
  CUDA_TRY(cudaMemcpyAsync(pi, s->x[0][3], s->n2 * s->esz, kind, st));
  return AGCM_OK;
}

int agcm_step(agcm_state_t* s, int nsteps, double dt, void* stream) {
  if (!s || nsteps < 0 || !std::isfinite(dt)) return fail(AGCM_EINVAL, "bad argument");
  if (nsteps == 0) return AGCM_OK;
  cudaStream_t st = as_stream(stream);
  return s->prec == AGCM_FP64 ? run_steps<double>(s, nsteps, dt, st) : run_steps<float>(s, nsteps, dt, st);
}

int agcm_filter(agcm_state_t* s, double r, void* stream) {
  if (!s || !(r > 0.0) || r > 0.25) return fail(AGCM_EINVAL, "filter weight r must be in (0, 1/4]");
  cudaStream_t st = as_stream(stream);
  const agcm_grid* g = s->grid;
  const int I = g->I, J = g->J, K = g->K;
  auto run = [&](auto tag, auto vw) -> int {
    using T = decltype(tag);
    constexpr int VW = decltype(vw)::value;
    const agcm::Geom<T>& G = geom_of<T>(s);
    const long long items = (long long)(2 * K + 1) * G.nfU + (long long)K * G.nfV;
    if (items == 0) return AGCM_OK;
    const size_t row_bytes = ((size_t)I * sizeof(T) + 15) & ~size_t(15);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / row_bytes));
    const size_t smem = (size_t)wpb * row_bytes;
    auto kern = agcm::k_filter<T, VW>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem));
    const long long want = (items + wpb - 1) / wpb;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(want, (long long)std::max(occ, 1) * nsm));
    agcm::FiltArgs<T> a{(T*)s->x[0][0], (T*)s->x[0][1], (T*)s->x[0][2], (T*)s->x[0][3],
                        G.filtU, G.filtV, G.nfU, G.nfV, I, J, K, (int)row_bytes, items, (T)r};
    s->prof.begin(KID_FILTER, st);
    kern<<<grid, wpb * 32, smem, st>>>(a);
    s->prof.end(st);
    CUDA_TRY(cudaGetLastError());
    return AGCM_OK;
  };
  if ((size_t)I * 8 > 96 * 1024) return fail(AGCM_EINVAL, "nlon too large for the row filter");
  s->bar_valid = false;  // the filtered state needs fresh vertical means
  using V1 = std::integral_constant<int, 1>;
  using V2 = std::integral_constant<int, 2>;
  using V4 = std::integral_constant<int, 4>;
  auto aligned = [&](size_t a) {  // vector rows need every field base on the vector size
    for (int f = 0; f < 4; ++f)
      if ((uintptr_t)s->x[0][f] % a) return false;
    return true;
  };
  if (s->prec == AGCM_FP64) return I % 2 == 0 && aligned(16) ? run(double(0), V2{}) : run(double(0), V1{});
  return I % 4 == 0 && aligned(16) ? run(float(0), V4{}) : run(float(0), V1{});
}

int agcm_step_split(agcm_state_t* s, int nsteps, double dt, int msub, void* stream) {
  if (!s || nsteps < 0 || msub < 1 || msub > 64 || !std::isfinite(dt)) return fail(AGCM_EINVAL, "bad argument");
  if (nsteps == 0) return AGCM_OK;
  cudaStream_t st = as_stream(stream);
  return s->prec == AGCM_FP64 ? run_steps_split<double>(s, nsteps, dt, msub, st)
                              : run_steps_split<float>(s, nsteps, dt, msub, st);
}

int agcm_grid_dt_split(const agcm_grid_t* g, double umax, double* dt, int* msub) {
  if (!g || !dt || !msub || !(umax > 0.0)) return fail(AGCM_EINVAL, "bad argument");
  // adaptation alone: the gravity-wave bound (c_max only); advection alone:
  // the same wavenumber bound with the flow speed umax only
  double dt_grav = 0.0;
  int rc = agcm_grid_dt(g, 0.0, &dt_grav);
  if (rc) return rc;
  const double kx = 2.0 / (kA * std::sqrt(0.5) * g->dlam), ky = 2.0 / (kA * g->dth);
  const double dtl = 1.6 / (umax * std::sqrt(kx * kx + ky * ky));
  *dt = dtl;
  *msub = (int)std::ceil(dtl / dt_grav - 1e-9);
  if (*msub < 1) *msub = 1;
  return AGCM_OK;
}

int agcm_tendency(agcm_state_t* s, void* tU, void* tV, void* tPhi, void* tpi, void* stream) {
  if (!s || !tU || !tPhi || !tpi || (!tV && s->nv)) return fail(AGCM_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  void* out[4] = {tU, tV, tPhi, tpi};
  return s->prec == AGCM_FP64 ? run_tendency<double>(s, out, st) : run_tendency<float>(s, out, st);
}

int agcm_step_adjoint(agcm_state_t* s, const void* const lam_in[4], void* const lam_out[4], double dt,
                      void* stream) {
  if (!s || !lam_in || !lam_out || !std::isfinite(dt)) return fail(AGCM_EINVAL, "bad argument");
  for (int f = 0; f < 4; ++f)
    if ((!lam_in[f] || !lam_out[f]) && !(f == 1 && s->nv == 0)) return fail(AGCM_EINVAL, "null adjoint buffer %d", f);
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < 4; ++q)
      if (lam_in[f] && lam_in[f] == lam_out[q]) return fail(AGCM_EINVAL, "lam_in and lam_out alias (buffer %d)", f);
  cudaStream_t st = as_stream(stream);
  return s->prec == AGCM_FP64 ? adjoint_step<double>(s, lam_in, lam_out, dt, st)
                              : adjoint_step<float>(s, lam_in, lam_out, dt, st);
}

int agcm_diagnostics(const agcm_state_t* s, agcm_diag_t* out, void* stream) {
  if (!s || !out) return fail(AGCM_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  double h[8];
  int rc = s->prec == AGCM_FP64 ? diagnostics<double>(s, h, st) : diagnostics<float>(s, h, st);
  if (rc) return rc;
  out->mass = h[0];
  out->e_kin = h[1];
  out->e_pot = h[2];
  out->e_ps = h[3];
  out->energy = h[1] + h[2] + h[3];
  out->max_u = h[4];
  out->max_v = h[5];
  out->finite = h[6] == 0.0 ? 1 : 0;
  out->reserved = 0;
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == AGCM_ETIMEOUT) return fail(AGCM_ETIMEOUT, "a bounded wait in the stage kernel gave up");
  if (!out->finite) return fail(AGCM_ENONFINITE, "state holds %g non-finite values", h[6]);
  return AGCM_OK;
}

int agcm_profile_enable(agcm_state_t* s, int enable) {
  if (!s) return fail(AGCM_EINVAL, "null state");
  s->prof.reset();
  s->prof.on = enable != 0;
  return AGCM_OK;
}

int agcm_profile_read(agcm_state_t* s, double* ms_total, int64_t* launches) {
  if (!s || !ms_total || !launches) return fail(AGCM_EINVAL, "null argument");
  if (s->prof.drain()) return fail(AGCM_ECUDA, "event synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
  for (int q = 0; q < KID_COUNT; ++q) {
    ms_total[q] = s->prof.ms[q];
    launches[q] = s->prof.n[q];
  }
  return AGCM_OK;
}

int agcm_kernel_count(void) { return KID_COUNT; }

int agcm_set_stage_kernel(int choice) {
  if (choice < 0 || choice > 2) return fail(AGCM_EINVAL, "stage kernel choice must be 0, 1 or 2");
  g_stage_choice.store(choice);
  return AGCM_OK;
}

int agcm_state_set_stage_kernel(agcm_state_t* s, int choice) {
  if (!s) return fail(AGCM_EINVAL, "null state");
  if (choice < 0 || choice > 2) return fail(AGCM_EINVAL, "stage kernel choice must be 0, 1 or 2");
  s->stage_choice = choice;
  return AGCM_OK;
}

const char* agcm_kernel_name(int id) { return (id >= 0 && id < KID_COUNT) ? kKernelNames[id] : ""; }

}  // extern "C"

// ------------------------------------------------------------------ adjoint
namespace {

int ensure_adj(agcm_state* s) {
  if (s->adj_ready) return AGCM_OK;
  const size_t e = s->esz, n3 = s->n3 * e, nv = std::max<size_t>(s->nv, 1) * e, n2 = s->n2 * e;
  const size_t nw = (size_t)(s->grid->K + 1) * s->grid->J * s->grid->I * e;
  bool ok = true;
  auto get = [&](size_t bytes) -> void* {
    void* p = dev_alloc(bytes);
    if (p) s->owned.push_back(p);
    else ok = false;
    return p;
  };
  // forward recompute (phases A, B) at the stage states
  for (auto& p : s->col) p = get(n2);
  s->W = get(nw);
  s->psi = get(n3);
  for (auto& p : s->adj3) p = get(n3);
  for (auto& p : s->adj2) p = get(n2);
  // rows whose adjoint halo fits a row segment go to k_adj_rows
  const agcm_grid* g = s->grid;
  std::vector<int> items, rows;
  for (int j = 0; j < g->J; ++j) {
    const int H = agcm::adj_row_halo(g->Mu[j], j < g->J - 1 ? g->Mv[j] : 0, j > 0 ? g->Mv[j - 1] : 0);
    int nseg = 0, S = 0;
    if (H <= agcm::kAdjRowMaxH && H < g->I) agcm::adj_row_segments(g->I, H, &nseg, &S);
    if (nseg > 0 && nseg <= 256) {
      for (int q = 0; q < nseg; ++q)
        if (q * S < g->I) items.push_back(j << 8 | q);
    } else {
      rows.push_back(j);
    }
  }
  auto put_ints = [&](const std::vector<int>& v) -> int* {
    if (v.empty()) return nullptr;
    int* d = (int*)get(v.size() * sizeof(int));
    if (d && cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    return d;
  };
  s->adj_items = put_ints(items);
  s->n_adj_items = (int)items.size();
  s->adj_rows = put_ints(rows);
  s->n_adj_rows = (int)rows.size();
  if (!rows.empty()) {
    const size_t nch = (size_t)(g->K + agcm::kAdjLevChunk - 1) / agcm::kAdjLevChunk;
    s->adj_part = get(3 * nch * rows.size() * g->I * e);
  }
  for (int c = 0; c < 2; ++c) {
    s->mu[c][0] = get(n3);
    s->mu[c][1] = get(nv);
    s->mu[c][2] = get(n3);
    s->mu[c][3] = get(n2);
  }
  if (!ok) return fail(AGCM_ENOMEM, "device allocation of the adjoint workspace failed");
  s->adj_ready = true;
  return AGCM_OK;
}

// out = (accumulate ? out : 0) + scale * J(x)^T y, J the Jacobian of T at x;
// with sum != nullptr also sum = sum_in + scale * J(x)^T y (sum_in defaults
// to sum itself).  No atomics and no
// zeroing: the P family, the column pass (phase B at x and its transpose),
// the gathered adjoint of every point (row segments, and the rows past their
// halo on the second stream), the adjoint of pi.
template <class T>
int vjp(agcm_state* s, void* const x[4], const void* const y[4], void* const out[4], double scale, int accumulate,
        cudaStream_t st, void* const* sum = nullptr, const void* const* sum_in = nullptr) {
  if (!sum_in) sum_in = sum;
  const agcm::Geom<T>& G = geom_of<T>(s);
  const size_t n2 = s->n2;
  agcm::ColState<T> cs{(T*)s->col[0], (T*)s->col[1], (T*)s->col[2], (T*)s->col[3], (T*)s->col[4], (T*)s->col[5]};
  s->prof.begin(KID_COLSTATE, st);
  agcm::k_colstate<T><<<nblocks(n2, 256), 256, 0, st>>>(G, (const T*)x[3], cs);
  s->prof.end(st);
  const agcm::AdjCol<T> c{(T*)s->W, (T*)s->psi, (T*)s->adj3[0], (T*)s->adj3[1], (T*)s->adj2[0], (T*)s->adj2[1]};
  s->prof.begin(KID_ADJ_COL, st);
  const dim3 cgrid((unsigned)((G.I + 31) / 32), (unsigned)G.J);
  // level groups of at most kColL levels, 32 x ng threads (the kernel's bound is 256)
  const int ng = (G.K + agcm::kColL - 1) / agcm::kColL;
  if (ng <= 8) {
    const size_t smem = ((7 + 5 * agcm::kColL) * ng * 32 + agcm::kLN * G.K) * sizeof(T);
    static std::atomic<size_t> attr{0};  // the size set so far
    if (attr.load() < smem) {
      CUDA_TRY(cudaFuncSetAttribute(agcm::k_adj_col<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr.store(smem);
    }
    agcm::k_adj_col<T><<<cgrid, dim3(32, ng), smem, st>>>(
        G, (const T*)x[0], (const T*)x[1], (const T*)x[2], (const T*)x[3], cs, (const T*)y[0], (const T*)y[1],
        (const T*)y[2], (const T*)y[3], c);
  } else {
    agcm::k_adj_col_w<T><<<cgrid, dim3(32, agcm::kColG), 0, st>>>(
        G, (const T*)x[0], (const T*)x[1], (const T*)x[2], (const T*)x[3], cs, (const T*)y[0], (const T*)y[1],
        (const T*)y[2], (const T*)y[3], c);
  }
  s->prof.end(st);
  const agcm::AdjM<T> m{(T*)s->adj2[2], (T*)s->adj2[3], (T*)s->adj2[4]};
  const agcm::AdjOut<T> o{(T*)out[0], (T*)out[1], (T*)out[2], (T*)out[3],
                          sum ? (T*)sum[0] : nullptr, sum ? (T*)sum[1] : nullptr,
                          sum ? (T*)sum[2] : nullptr, sum ? (T*)sum[3] : nullptr,
                          sum ? (const T*)sum_in[0] : nullptr, sum ? (const T*)sum_in[1] : nullptr,
                          sum ? (const T*)sum_in[2] : nullptr, sum ? (const T*)sum_in[3] : nullptr, (T)scale,
                          accumulate};
  s->prof.begin(KID_ADJ_GATHER, st);
  // the rows of the L1 form run on the state's second stream beside the
  // row-segment kernel (they write other rows)
  const bool fork = s->n_adj_items > 0 && s->n_adj_rows > 0 && s->aux[0];
  if (fork) {
    CUDA_TRY(cudaEventRecord(s->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(s->aux[0], s->ev_fork, 0));
  }
  if (s->n_adj_rows > 0) {
    cudaStream_t q = fork ? s->aux[0] : st;
    const int nch = (G.K + agcm::kAdjLevChunk - 1) / agcm::kAdjLevChunk;
    const dim3 agrid((unsigned)((G.I + agcm::kAdjTileX - 1) / agcm::kAdjTileX),
                     (unsigned)((s->n_adj_rows + agcm::kAdjTileY - 1) / agcm::kAdjTileY), (unsigned)nch);
    agcm::k_adj_gather<T><<<agrid, agcm::kAdjTileX * agcm::kAdjTileY, 0, q>>>(
        G, (const T*)x[0], (const T*)x[1], (const T*)x[2], cs, (const T*)s->W, (const T*)s->psi,
        (const T*)s->adj3[0], (const T*)s->adj3[1], (const T*)s->adj2[0], (const T*)y[0], (const T*)y[1],
        (const T*)y[2], s->adj_rows, s->n_adj_rows, (T*)s->adj_part, o);
    agcm::k_adj_fold<T><<<nblocks((size_t)s->n_adj_rows * G.I, 256), 256, 0, q>>>(
        G, s->adj_rows, s->n_adj_rows, nch, (const T*)s->adj_part, m);
  }
  if (s->n_adj_items > 0) {
    constexpr size_t smem = agcm::adj_row_smem<T>();
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
      CUDA_TRY(cudaFuncSetAttribute(agcm::k_adj_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr.store(true);
    }
    agcm::k_adj_rows<T><<<(unsigned)s->n_adj_items, agcm::kAdjRowB, smem, st>>>(
        G, s->adj_items, (const T*)x[0], (const T*)x[1], (const T*)x[2], cs, (const T*)s->W, (const T*)s->psi,
        (const T*)s->adj3[0], (const T*)s->adj3[1], (const T*)s->adj2[0], (const T*)y[0], (const T*)y[1],
        (const T*)y[2], m, o);
  }
  if (fork) {
    CUDA_TRY(cudaEventRecord(s->ev_join[0], s->aux[0]));
    CUDA_TRY(cudaStreamWaitEvent(st, s->ev_join[0], 0));
  }
  s->prof.end(st);
  s->prof.begin(KID_ADJ_COLSTATE, st);
  agcm::k_adj_colstate<T><<<nblocks(n2, 256), 256, 0, st>>>(G, m, (const T*)s->adj2[1], o);
  s->prof.end(st);
  CUDA_TRY(cudaGetLastError());
  return AGCM_OK;
}

// One step x3 = xn + dt T(x2), x2 = xn + dt/2 T(x1), x1 = xn + dt/2 T(xn):
// lam_n = lam3 + mu2 + mu1 + dt/2 J(xn)^T mu1, mu2 = dt J(x2)^T lam3,
// mu1 = dt/2 J(x1)^T mu2.  The stage states are recomputed from xn.
template <class T>
int adjoint_step(agcm_state* s, const void* const lam_in[4], void* const lam_out[4], double dt, cudaStream_t st) {
  int rc;
  if ((rc = ensure_adj(s))) return rc;
  if ((rc = ensure_bar<T>(s, st))) return rc;
  if ((rc = fused_stage<T, 1>(s, 0, s->x[1], 1, 0.5 * dt, st))) return rc;
  if ((rc = fused_stage<T, 2>(s, 1, s->x[2], 2, 0.5 * dt, st))) return rc;
  void* const* mu2 = s->mu[0];
  void* const* mu1 = s->mu[1];
  // each product also adds itself to lam_out (no separate accumulation
  // pass); the first forms lam_out = lam_in + mu2 (no copy of lam_in)
  if ((rc = vjp<T>(s, s->x[2], lam_in, mu2, dt, 0, st, lam_out, lam_in))) return rc;
  if ((rc = vjp<T>(s, s->x[1], mu2, mu1, 0.5 * dt, 0, st, lam_out))) return rc;
  return vjp<T>(s, s->x[0], mu1, lam_out, 0.5 * dt, 1, st);
}

}  // namespace

// ======================================= allocation-free tendency (static scratch)
//
// agcm_tendency_static computes T(x) like agcm_tendency, but without a state
// object and without allocating device memory: its scratch (the grid's device
// tables and the FP64 vertical means Ubar/Vbar) lives in one file-scope
// __device__ array of fixed size that every GPU holds from the moment this
// library is loaded until the process exits.  It serves callers that cannot
// call cudaMalloc: an application running under a fixed device-memory budget
// that forbids new allocations, and embedders whose allocator owns all device
// memory and hands the library only input and output buffers.
namespace {

constexpr size_t kStaticCols = 262144;  // nlat * nlon at most (e.g. 720 x 360)
constexpr int kStaticRows = 4096;       // nlat at most
constexpr int kStaticLevels = 256;      // nlev at most
constexpr int kStaticMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
// byte layout of the scratch array
constexpr size_t kRowB = al256(kStaticRows * 8), kLevB = al256((kStaticLevels + 1) * 8),
                 kColB = al256(kStaticCols * 8);
constexpr size_t kOffRaw = 0;                        // 6 row arrays s c cot A sv Av (double)
constexpr size_t kOffRawLev = kOffRaw + 6 * kRowB;   // sh ds Hkk hk beta (double)
constexpr size_t kOffPitRaw = kOffRawLev + 5 * kLevB;  // pi~, R T~_s (double)
constexpr size_t kOffInt = kOffPitRaw + 2 * kColB;   // Mu Mv (int)
constexpr size_t kOffRowT = kOffInt + 2 * kRowB;     // 12 typed row arrays
constexpr size_t kOffLevT = kOffRowT + 12 * kRowB;   // 7 typed level arrays
constexpr size_t kOffColT = kOffLevT + 7 * kLevB;    // pit, rt0pit (typed)
constexpr size_t kOffBar = kOffColT + 2 * kColB;     // Ubar, Vbar (double)
constexpr size_t kOffRowL = kOffBar + 2 * kColB;     // row-segment items, then column-kernel rows (int)
constexpr size_t kItemB = al256((kStaticCols / 128 + kStaticRows) * 4);  // at most ceil(nlon/128) items a row
constexpr size_t kOffErr = kOffRowL + kItemB + al256(kStaticRows * 4);  // status word of the stage kernel
constexpr size_t kStaticBytes = kOffErr + 256;       // about 13 MB

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};
// per device: the grid id and precision whose tables the array holds (0: none)
uint64_t g_static_uid[kStaticMaxDevices] = {};
int g_static_prec[kStaticMaxDevices] = {};

// Typed device tables from the raw FP64 ones (same formulas as the state path).
template <class T>
__global__ void k_static_geom(int I, int J, int K, const double* raw, const double* rawlev, const double* pitraw,
                              const int* Mu, const int* Mv, T* rowT, T* levT, T* colT, size_t rowStride,
                              size_t levStride, size_t colStride, double beta2) {
  const double* s = raw;
  const double* c = raw + rowStride;
  const double* cot = raw + 2 * rowStride;
  const double* A = raw + 3 * rowStride;
  const double* sv = raw + 4 * rowStride;
  const double* Av = raw + 5 * rowStride;
  const double* ds = rawlev + levStride;
  const double* hk = rawlev + 3 * levStride;
  const double* beta = rawlev + 4 * levStride;
  const double dlam = 2.0 * kPi / I, dth = kPi / J;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  // one pass covers the columns, the rows and the levels, whichever is longest
  // (a grid may have more levels than columns)
  const size_t ncol = (size_t)I * J, nall = ncol > (size_t)K ? ncol : (size_t)K;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < nall; n += stride) {
    if (n < (size_t)J) {
      const int j = (int)n;
      rowT[0 * rowStride + j] = (T)(1.0 / (kA * s[j] * Mu[j] * dlam));
      rowT[1 * rowStride + j] = (T)(1.0 / (kA * s[j] * dth));
      rowT[2 * rowStride + j] = (T)(kA * dth / Mu[j]);
      rowT[3 * rowStride + j] = (T)(0.5 / A[j]);
      rowT[4 * rowStride + j] = (T)(2.0 * kOmega * c[j]);
      rowT[5 * rowStride + j] = (T)(cot[j] / kA);
      if (j < J - 1) {
        rowT[6 * rowStride + j] = (T)sv[j];
        rowT[7 * rowStride + j] = (T)(kA * dlam * sv[j]);
        rowT[8 * rowStride + j] = (T)(kA * dth / Mv[j]);
        rowT[9 * rowStride + j] = (T)(0.5 / Av[j]);
        rowT[10 * rowStride + j] = (T)(0.25 * A[j] / Av[j]);
        rowT[11 * rowStride + j] = (T)(0.25 * A[j + 1] / Av[j]);
      }
    }
    if (n < (size_t)K) {
      const int k = (int)n;
      levT[0 * levStride + k] = (T)ds[k];
      levT[1 * levStride + k] = (T)(0.5 / ds[k]);
      levT[2 * levStride + k] = (T)(beta[k] * hk[k]);
      levT[3 * levStride + k] = (T)(beta[k] * rawlev[2 * levStride + k]);
      levT[4 * levStride + k] = (T)(beta[k] * hk[k] / ds[k]);
      levT[5 * levStride + k] = (T)(1.0 - rawlev[k]);
      levT[6 * levStride + k] = (T)(beta[k] != 0.0 ? beta2 / beta[k] : 0.0);
    }
    if (n < ncol) {
      colT[n] = (T)pitraw[n];
      colT[colStride + n] = (T)(pitraw[colStride + n] / pitraw[n]);
    }
  }
}

// tables: upload the grid's tables and build the typed ones (false when the
// array already holds this grid's tables in this precision).
template <class T>
int tendency_static(const agcm_grid* g, char* base, bool tables, const void* U, const void* V, const void* Phi,
                    const void* pi, void* tU, void* tV, void* tPhi, void* tpi, cudaStream_t st) {
  const int I = g->I, J = g->J, K = g->K;
  const size_t rS = kRowB / 8, lS = kLevB / 8, cS = kColB / 8;  // strides in elements of 8 bytes
  double* raw = (double*)(base + kOffRaw);
  double* rawlev = (double*)(base + kOffRawLev);
  double* pitraw = (double*)(base + kOffPitRaw);
  int* Mu = (int*)(base + kOffInt);
  int* Mv = (int*)(base + kOffInt + kRowB);
  // typed tables are indexed with the element strides rS/lS/cS of the raw
  // (8-byte) tables, so a float table uses the first half of its region
  T* rowT = (T*)(base + kOffRowT);
  T* levT = (T*)(base + kOffLevT);
  T* colT = (T*)(base + kOffColT);
  if (tables) {
  const std::vector<double>* rows[6] = {&g->s, &g->c, &g->cot, &g->A, &g->sv, &g->Av};
  for (int q = 0; q < 6; ++q)
    if (!rows[q]->empty())
      CUDA_TRY(cudaMemcpyAsync(raw + q * rS, rows[q]->data(), rows[q]->size() * 8, cudaMemcpyHostToDevice, st));
  const std::vector<double>* levs[5] = {&g->sh, &g->ds, &g->Hkk, &g->hk, &g->beta};
  for (int q = 0; q < 5; ++q)
    CUDA_TRY(cudaMemcpyAsync(rawlev + q * lS, levs[q]->data(), levs[q]->size() * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(pitraw, g->pit.data(), g->pit.size() * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(pitraw + cS, g->rts.data(), g->rts.size() * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(Mu, g->Mu.data(), g->Mu.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!g->Mv.empty())
    CUDA_TRY(cudaMemcpyAsync(Mv, g->Mv.data(), g->Mv.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  {
    std::vector<int> rk, rc;
    int nk[agcm::kRowCls];
    row_lists(g, &rk, &rc, nk);
    if (!rk.empty())
      CUDA_TRY(cudaMemcpyAsync(base + kOffRowL, rk.data(), rk.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!rc.empty())
      CUDA_TRY(cudaMemcpyAsync(base + kOffRowL + kItemB, rc.data(), rc.size() * sizeof(int),
                               cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(base + kOffErr, 0, sizeof(int), st));
  }
  k_static_geom<T><<<nblocks(std::max<size_t>((size_t)I * J, (size_t)K), 256), 256, 0, st>>>(
      I, J, K, raw, rawlev, pitraw, Mu, Mv, rowT, levT, colT, rS, lS, cS, g->beta2);
  CUDA_TRY(cudaGetLastError());
  }
  agcm::Geom<T> G{};
  G.I = I; G.J = J; G.K = K;
  G.Mu = Mu;
  G.Mv = Mv;
  G.rdx = rowT + 0 * rS; G.rdy = rowT + 1 * rS; G.zf = rowT + 2 * rS; G.r2A = rowT + 3 * rS;
  G.f0 = rowT + 4 * rS; G.cota = rowT + 5 * rS; G.sv = rowT + 6 * rS; G.yv = rowT + 7 * rS;
  G.zfv = rowT + 8 * rS; G.r2Av = rowT + 9 * rS; G.cn = rowT + 10 * rS; G.cs = rowT + 11 * rS;
  G.ds = levT + 0 * lS; G.r2ds = levT + 1 * lS; G.hk = levT + 2 * lS; G.Hkk = levT + 3 * lS;
  G.hk_rds = levT + 4 * lS;
  G.oms = levT + 5 * lS;
  G.rho = levT + 6 * lS;
  G.nl = g->beta2 != 0.0 && g->th.delta != 0.0;
  leap1_band(g, &G.l1lo, &G.l1hi);  // no second stream here: the two launches run in order
  G.dsd = rawlev + 1 * lS;
  G.shd = rawlev + 0 * lS;
  G.Ad = raw + 3 * rS;
  G.Avd = raw + 5 * rS;
  G.pit = colT;
  G.rt0pit = colT + cS;
  G.rady = (T)(1.0 / (kA * g->dth));
  G.adl = (T)(kA * g->dlam);
  {
    std::vector<int> rk, rc;
    row_lists(g, &rk, &rc, G.nk);  // host only: counts (the lists were copied with the tables)
    G.nrowc = (int)rc.size();
    long long nitems = 0;
    for (int c = 0; c < agcm::kRowCls; ++c) nitems += G.nk[c];
    G.rowfill = rows_fill_device(nitems);
    G.rowk = (const int*)(base + kOffRowL);
    G.rowc = (const int*)(base + kOffRowL + kItemB);
  }
  double* ubar = (double*)(base + kOffBar);
  double* vbar = (double*)(base + kOffBar + kColB);
  agcm::k_vsum<T><<<nblocks((size_t)I * J, 256), 256, 0, st>>>(G, (const T*)U, (const T*)V, ubar, vbar);
  const void* xs[4] = {U, V, Phi, pi};
  const void* none[4] = {nullptr, nullptr, nullptr, nullptr};
  void* out[4] = {tU, tV, tPhi, tpi};
  return launch_fused<T, 0>(G, xs, ubar, vbar, none, out, nullptr, nullptr, nullptr, nullptr, 1.0,
                            (int*)(base + kOffErr), st);
}

}  // namespace

extern "C" int agcm_tendency_static(const agcm_grid_t* g, int precision, const void* U, const void* V,
                                    const void* Phi, const void* pi, void* tU, void* tV, void* tPhi, void* tpi,
                                    void* stream) {
  if (!g || !U || !V || !Phi || !pi || !tU || !tV || !tPhi || !tpi) return fail(AGCM_EINVAL, "null argument");
  if (precision != AGCM_FP64 && precision != AGCM_FP32)
    return fail(AGCM_EINVAL, "precision must be AGCM_FP64 or AGCM_FP32");
  if ((size_t)g->I * g->J > kStaticCols || g->J > kStaticRows || g->K > kStaticLevels)
    return fail(AGCM_EINVAL,
                "agcm_tendency_static: grid %d x %d x %d exceeds the static scratch limit "
                "(nlon*nlat <= %zu, nlat <= %d, nlev <= %d)",
                g->I, g->J, g->K, kStaticCols, kStaticRows, kStaticLevels);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(AGCM_EINVAL, "device ordinal %d not supported", dev);
  void* base = nullptr;
  bool tables = true;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    // once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(AGCM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  base = g_static_ptr[dev];
  // the array keeps the last call's tables: rebuild them only for another
  // grid (or the same grid after agcm_grid_set_thermo) or precision
  tables = g_static_uid[dev] != g->uid || g_static_prec[dev] != precision;
  g_static_uid[dev] = 0;  // stays 0 if this call fails part-way
  cudaStream_t st = as_stream(stream);
  const int rc = precision == AGCM_FP64
                     ? tendency_static<double>(g, (char*)base, tables, U, V, Phi, pi, tU, tV, tPhi, tpi, st)
                     : tendency_static<float>(g, (char*)base, tables, U, V, Phi, pi, tU, tV, tPhi, tpi, st);
  if (rc == AGCM_OK) {
    g_static_uid[dev] = g->uid;
    g_static_prec[dev] = precision;
  }
  return rc;
}

// ================================================================ ensembles
struct agcm_ensemble {
  int prec = AGCM_FP32;
  std::vector<agcm_state*> members;
  std::vector<char> host_desc;   // EnsMember<T>[n]
  void* d_desc = nullptr;
  agcm::EnsSync* d_sync = nullptr;
  int queue_cap = 0;             // steps per launch
  int nitems = 0;
  int warps_per_block = 1;
  int blocks_per_sm = 0;         // 0: as many as fit
  int rows_per_item = 1;         // row tile of a work item
  double timeout_s = 1.0;
  int test_missing = 0;
  bool desc_dirty = true;
  // work items of the row-segment persistent launch (warps_per_block = 8)
  std::vector<int> host_items;   // int2 pairs
  void* d_items = nullptr;
  int nitems_rows = 0;
  size_t rows_smem = 0;          // dynamic shared memory of that launch
  std::vector<double> last_dt;
  Profiler prof;
};

namespace {

template <class T>
void fill_desc(agcm_ensemble* e) {
  e->host_desc.assign(e->members.size() * sizeof(agcm::EnsMember<T>), 0);
  auto* d = reinterpret_cast<agcm::EnsMember<T>*>(e->host_desc.data());
  int begin = 0;
  for (size_t m = 0; m < e->members.size(); ++m) {
    agcm_state* s = e->members[m];
    d[m].g = geom_of<T>(s);
    for (int c = 0; c < 3; ++c) {
      for (int f = 0; f < 4; ++f) d[m].x[c][f] = (T*)s->x[c][f];
      d[m].ubar[c] = s->ubar[c];
      d[m].vbar[c] = s->vbar[c];
    }
    d[m].nbx = (s->grid->I + 31) / 32;
    d[m].item_begin = begin;
    d[m].dt = (T)0;
    begin += d[m].nbx * ((s->grid->J + e->rows_per_item - 1) / e->rows_per_item);
  }
  e->nitems = begin;
  // row-segment persistent launch: every member's row-segment items (any
  // stride class), then 256-column chunks of the rows left to the column body
  e->host_items.clear();
  e->rows_smem = 0;
  for (size_t m = 0; m < e->members.size(); ++m) {
    const agcm_grid* g = e->members[m]->grid;
    std::vector<int> rk, rc;
    int nk[agcm::kRowCls];
    row_lists(g, &rk, &rc, nk);
    for (int it : rk) {
      e->host_items.push_back((int)m);
      e->host_items.push_back(it);
    }
    for (int j : rc)
      for (int c = 0; c * agcm::kRowB < g->I; ++c) {
        e->host_items.push_back((int)m | (1 << 16));
        e->host_items.push_back(j << 8 | c);
      }
    e->rows_smem = std::max(e->rows_smem, agcm::row_smem_bytes<T>(agcm::kRowB, g->K));
  }
  e->nitems_rows = (int)(e->host_items.size() / 2);
}

template <class T>
int ensemble_step(agcm_ensemble* e, int nsteps, const double* dt, cudaStream_t st) {
  auto* d = reinterpret_cast<agcm::EnsMember<T>*>(e->host_desc.data());
  const size_t n = e->members.size();
  bool changed = e->desc_dirty;
  for (size_t m = 0; m < n; ++m)
    if (e->last_dt.size() != n || e->last_dt[m] != dt[m]) changed = true;
  if (changed) {
    e->last_dt.assign(dt, dt + n);
    for (size_t m = 0; m < n; ++m) d[m].dt = (T)dt[m];
    CUDA_TRY(cudaMemcpyAsync(e->d_desc, e->host_desc.data(), e->host_desc.size(), cudaMemcpyHostToDevice, st));
    e->desc_dirty = false;
  }
  for (agcm_state* s : e->members) {
    if (sizeof(T) == 4 && nsteps > 0) s->bar_valid = false;  // exact means once per call in FP32
    int rc = ensure_bar<T>(s, st);
    if (rc) return rc;
  }
  if (nsteps == 0) return AGCM_OK;  // prepared: dt uploaded, vertical means valid
  int dev = 0, nsm = 0, clock_khz = 0, occ = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  const int threads = 32 * e->warps_per_block;
  if (e->warps_per_block == 8) {  // the row-segment persistent launch
    auto kr = agcm::k_ensemble_rows<T>;
    if (e->rows_smem > 227 * 1024) return fail(AGCM_EINVAL, "ensemble member with too many levels for the row launch");
    CUDA_TRY(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->rows_smem));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kr, agcm::kRowB, e->rows_smem));
    if (occ < 1) return fail(AGCM_EINVAL, "row-segment ensemble kernel does not fit");
    const int per_sm = e->blocks_per_sm > 0 ? std::min(e->blocks_per_sm, occ) : occ;
    const unsigned grid = (unsigned)(per_sm * nsm);
    const long long limit = (long long)(e->timeout_s * (double)clock_khz * 1000.0);
    const size_t sync_bytes = sizeof(agcm::EnsSync) + sizeof(unsigned) * (size_t)e->queue_cap * 3;
    for (int done = 0; done < nsteps; done += e->queue_cap) {
      const int chunk = std::min(e->queue_cap, nsteps - done);
      CUDA_TRY(cudaMemsetAsync(e->d_sync, 0, sync_bytes, st));
      e->prof.begin(KID_ENSEMBLE, st);
      kr<<<grid, agcm::kRowB, e->rows_smem, st>>>((const agcm::EnsMember<T>*)e->d_desc, (const int2*)e->d_items,
                                                 e->nitems_rows, chunk, e->d_sync, grid + (unsigned)e->test_missing,
                                                 limit);
      e->prof.end(st);
      CUDA_TRY(cudaGetLastError());
    }
    for (agcm_state* s : e->members) s->bar_valid = true;
    return AGCM_OK;
  }
  auto kern = e->rows_per_item == 4 ? agcm::k_ensemble<T, 4>
                                    : (e->rows_per_item == 2 ? agcm::k_ensemble<T, 2> : agcm::k_ensemble<T, 1>);
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0));
  if (occ < 1) return fail(AGCM_EINVAL, "ensemble kernel does not fit with %d threads per block", threads);
  const int per_sm = e->blocks_per_sm > 0 ? std::min(e->blocks_per_sm, occ) : occ;
  const unsigned grid = (unsigned)(per_sm * nsm);
  const long long limit = (long long)(e->timeout_s * (double)clock_khz * 1000.0);
  const size_t sync_bytes = sizeof(agcm::EnsSync) + sizeof(unsigned) * (size_t)e->queue_cap * 3;
  for (int done = 0; done < nsteps; done += e->queue_cap) {
    const int chunk = std::min(e->queue_cap, nsteps - done);
    CUDA_TRY(cudaMemsetAsync(e->d_sync, 0, sync_bytes, st));
    e->prof.begin(KID_ENSEMBLE, st);
    kern<<<grid, threads, 0, st>>>((const agcm::EnsMember<T>*)e->d_desc, (int)n, e->nitems, chunk, e->d_sync,
                                   grid + (unsigned)e->test_missing, limit);
    e->prof.end(st);
    CUDA_TRY(cudaGetLastError());
  }
  for (agcm_state* s : e->members) s->bar_valid = true;
  return AGCM_OK;
}

}  // namespace

extern "C" {

int agcm_ensemble_create(agcm_state_t* const* members, int n, agcm_ensemble_t** out) {
  if (!members || n < 1 || !out) return fail(AGCM_EINVAL, "need n >= 1 members and an output pointer");
  *out = nullptr;
  agcm_ensemble* e = new agcm_ensemble;
  e->prec = members[0]->prec;
  for (int m = 0; m < n; ++m) {
    if (!members[m] || members[m]->prec != e->prec) {
      delete e;
      return fail(AGCM_EINVAL, "member %d is null or has another precision", m);
    }
    if (members[m]->grid->beta2 != 0.0 && members[m]->grid->th.delta != 0.0) {
      delete e;
      return fail(AGCM_EINVAL, "member %d: ensembles do not cover the nonlinear delta kappa Phi/P term", m);
    }
    for (int q = 0; q < m; ++q)
      if (members[q] == members[m]) {
        delete e;
        return fail(AGCM_EINVAL, "member %d appears twice", m);
      }
    e->members.push_back(members[m]);
  }
  if (e->prec == AGCM_FP64)
    fill_desc<double>(e);
  else
    fill_desc<float>(e);
  e->queue_cap = 1024;
  e->d_desc = dev_alloc(e->host_desc.size());
  e->d_items = dev_alloc(std::max<size_t>(e->host_items.size(), 2) * sizeof(int));
  if (e->d_items && !e->host_items.empty() &&
      cudaMemcpy(e->d_items, e->host_items.data(), e->host_items.size() * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    dev_free(e->d_items);
    e->d_items = nullptr;
  }
  e->d_sync = (agcm::EnsSync*)dev_alloc(sizeof(agcm::EnsSync) + sizeof(unsigned) * (size_t)e->queue_cap * 3);
  if (!e->d_desc || !e->d_sync || !e->d_items) {
    dev_free(e->d_desc);
    dev_free(e->d_sync);
    dev_free(e->d_items);
    delete e;
    return fail(AGCM_ENOMEM, "device allocation for the ensemble failed");
  }
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    for (agcm_state* s : e->members) const_cast<agcm_grid*>(s->grid)->refs++;
  }
  *out = e;
  return AGCM_OK;
}

int agcm_ensemble_destroy(agcm_ensemble_t* e) {
  if (!e) return AGCM_OK;
  cudaDeviceSynchronize();
  dev_free(e->d_desc);
  dev_free(e->d_sync);
  dev_free(e->d_items);
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    for (agcm_state* s : e->members) const_cast<agcm_grid*>(s->grid)->refs--;
  }
  delete e;
  return AGCM_OK;
}

int agcm_ensemble_configure(agcm_ensemble_t* e, int warps_per_block, int blocks_per_sm) {
  if (!e || (warps_per_block != 1 && warps_per_block != 8) || blocks_per_sm < 0)
    return fail(AGCM_EINVAL, "warps_per_block must be 1 or 8 and blocks_per_sm >= 0");
  e->warps_per_block = warps_per_block;
  e->blocks_per_sm = blocks_per_sm;
  return AGCM_OK;
}

int agcm_ensemble_tile(agcm_ensemble_t* e, int rows_per_item) {
  if (!e || (rows_per_item != 1 && rows_per_item != 2 && rows_per_item != 4))
    return fail(AGCM_EINVAL, "rows_per_item must be 1, 2 or 4");
  if (rows_per_item == e->rows_per_item) return AGCM_OK;
  e->rows_per_item = rows_per_item;
  // item ranges change; the descriptor (with its dt) is uploaded again at the next step
  const std::vector<char> old = e->host_desc;
  if (e->prec == AGCM_FP64)
    fill_desc<double>(e);
  else
    fill_desc<float>(e);
  const size_t n = e->members.size();
  if (e->prec == AGCM_FP64) {
    for (size_t m = 0; m < n; ++m)
      reinterpret_cast<agcm::EnsMember<double>*>(e->host_desc.data())[m].dt =
          reinterpret_cast<const agcm::EnsMember<double>*>(old.data())[m].dt;
  } else {
    for (size_t m = 0; m < n; ++m)
      reinterpret_cast<agcm::EnsMember<float>*>(e->host_desc.data())[m].dt =
          reinterpret_cast<const agcm::EnsMember<float>*>(old.data())[m].dt;
  }
  e->desc_dirty = true;
  return AGCM_OK;
}

int agcm_ensemble_set_timeout(agcm_ensemble_t* e, double seconds, int test_missing_blocks) {
  if (!e || !(seconds > 0.0) || seconds > 60.0 || test_missing_blocks < 0)
    return fail(AGCM_EINVAL, "timeout must be in (0, 60] s and test_missing_blocks >= 0");
  e->timeout_s = seconds;
  e->test_missing = test_missing_blocks;
  return AGCM_OK;
}

int agcm_ensemble_step(agcm_ensemble_t* e, int nsteps, const double* dt, void* stream) {
  if (!e || nsteps < 0 || !dt) return fail(AGCM_EINVAL, "bad argument");
  for (size_t m = 0; m < e->members.size(); ++m)
    if (!std::isfinite(dt[m])) return fail(AGCM_EINVAL, "dt[%zu] is not finite", m);
  cudaStream_t st = as_stream(stream);
  return e->prec == AGCM_FP64 ? ensemble_step<double>(e, nsteps, dt, st) : ensemble_step<float>(e, nsteps, dt, st);
}

int agcm_ensemble_status(agcm_ensemble_t* e, void* stream) {
  if (!e) return fail(AGCM_EINVAL, "null ensemble");
  int status = 0;
  cudaStream_t st = as_stream(stream);
  CUDA_TRY(cudaMemcpyAsync(&status, &e->d_sync->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (status == AGCM_ETIMEOUT)
    return fail(AGCM_ETIMEOUT, "a grid barrier of the ensemble kernel gave up waiting (not all blocks resident?)");
  return AGCM_OK;
}

int agcm_ensemble_profile(agcm_ensemble_t* e, int enable, double* ms_total, int64_t* launches) {
  if (!e) return fail(AGCM_EINVAL, "null ensemble");
  if (ms_total && launches) {
    if (e->prof.drain()) return fail(AGCM_ECUDA, "event synchronisation failed");
    *ms_total = e->prof.ms[KID_ENSEMBLE];
    *launches = e->prof.n[KID_ENSEMBLE];
  }
  if (enable >= 0) {
    e->prof.reset();
    e->prof.on = enable != 0;
  }
  return AGCM_OK;
}

}  // extern "C"
