/*
 * agcm.h — C ABI of the GB300 leap-format dynamical-core step (arXiv 2103.10114).
 *
 * The library (libagcm.so, CUDA sm_103a) advances the IAP-transformed
 * primitive equations (Eq. 1, split as Eq. 2 into advection L and adaptation
 * A) on a latitude–longitude–sigma Arakawa C grid.  Every zonal difference on
 * row j spans an odd stride M_j (Eq. 6), chosen by Eq. 7 so that the zonal
 * spacing never falls below the 45-degree spacing; this replaces the polar
 * filter.  The vertical sums of Alg. 1 / Alg. 2 (sigma velocity, surface
 * pressure tendency) and the hydrostatic integral run as in-kernel column scans.
 *
 * Conventions shared by every call
 *  - Grid: I = nlon, J = nlat, K = nlev.  Scalar (Phi, pi) and U rows
 *    j = 0..J-1 sit at colatitude (j+1/2)*pi/J; V rows j = 0..J-2 at
 *    (j+1)*pi/J; V is zero on the pole edges.  U index i sits at longitude
 *    (i+1/2)*2pi/I, scalars and V at i*2pi/I.  V points toward increasing
 *    colatitude (south).
 *  - Layout: SoA, row-major [k][j][i] with i (longitude) contiguous.
 *    U, Phi: K*J*I values; V: K*(J-1)*I; pi: J*I (= p'_sa / p0, the surface
 *    pressure anomaly over the grid's standard surface pressure pi~, which
 *    is exp(-phi_s/(R*250 K)) by default; see agcm_grid_set_thermo).
 *  - Element type: double for AGCM_FP64 states, float for AGCM_FP32 states.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = default
 *    stream).  Calls that take a stream are asynchronous on it unless stated.
 *    A state also owns five internal streams, created with stream
 *    priorities (the launches with the longest blocks highest): each stage
 *    of agcm_step, agcm_step_split, agcm_tendency and agcm_step_adjoint forks
 *    some of its launches onto them after the work already queued on
 *    `stream` and joins them back before `stream` continues, so ordering on
 *    `stream` (and capture of `stream` into a CUDA graph) is as for one
 *    launch.
 *  - Errors: every call returns AGCM_OK (0) or a negative-free positive code
 *    below; agcm_last_error() returns a message for the calling thread.  The
 *    library never aborts the process and never traps on the device.
 *  - Ownership: pointers passed in are borrowed for the duration of the call;
 *    the library copies what it keeps.  Objects returned through `out`
 *    pointers are owned by the caller and released with the matching destroy.
 */
#ifndef AGCM_H_
#define AGCM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum agcm_status {
  AGCM_OK = 0,
  AGCM_EINVAL = 1,      /* invalid argument (sizes, tables, null pointers) */
  AGCM_ENOMEM = 2,      /* device allocation failed */
  AGCM_ECUDA = 3,       /* a CUDA runtime call failed; message has the CUDA text */
  AGCM_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  AGCM_ENONFINITE = 5   /* the state holds NaN or Inf (reported by diagnostics) */
};

enum agcm_precision { AGCM_FP64 = 0, AGCM_FP32 = 1 };

typedef struct agcm_grid agcm_grid_t;
typedef struct agcm_state agcm_state_t;

/* Message for the last failing call on this thread ("" if none). */
const char* agcm_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int agcm_version(void);

/*
 * Device memory hook.  By default the library calls cudaMalloc/cudaFree.
 * A caller may route every allocation through its own allocator (the Python
 * binding routes them through PyTorch's caching allocator).  `alloc` returns
 * NULL on failure, which the library reports as AGCM_ENOMEM.  Pass NULLs to
 * restore the default.  Not thread-safe against concurrent state creation.
 */
typedef void* (*agcm_alloc_fn)(uint64_t bytes, void* ctx);
typedef void (*agcm_free_fn)(void* ptr, void* ctx);
int agcm_set_allocator(agcm_alloc_fn alloc, agcm_free_fn free_fn, void* ctx);

/*
 * agcm_grid_create — the geometry of one grid (host only; no device work).
 * Eq. 6 (leap-format centred difference) and Eq. 7 (N_leap from the
 * 45-degree reference spacing) define the stride tables.
 *   nlon >= 3, nlat >= 2, nlev >= 1; nlon*nlat <= 2^30, nlat <= 65535 and
 *   nlon*nlat*nlev <= 4e9.
 *   sigma_half: nlev+1 half levels, sigma_half[0] = 0, sigma_half[nlev] = 1,
 *               strictly increasing; NULL = uniform.
 *   leap_u:     nlat strides for the scalar/U rows; NULL = Eq. 7 raised to
 *               the next odd number (N = max(1, ceil(r - 1e-9))).
 *   leap_v:     nlat-1 strides for the V rows; NULL = Eq. 7 at the V rows.
 *               Every stride must be odd, >= 1 and satisfy 2*M < nlon.
 *   phis:       nlat*nlon surface geopotential [m^2/s^2]; NULL = flat.
 * Returns AGCM_EINVAL for any violation, with the offending row in the message.
 */
int agcm_grid_create(int nlon, int nlat, int nlev, const double* sigma_half, const int32_t* leap_u,
                     const int32_t* leap_v, const double* phis, agcm_grid_t** out);
int agcm_grid_destroy(agcm_grid_t* grid);

/*
 * agcm_grid_set_thermo — the standard stratification and the switches of
 * Eq. 1's Phi equation, (1 - delta_p)[b(1 + delta_c) + delta kappa Phi/P]
 * times the Omega~ term.  The paper defines neither T~(p) nor the deltas;
 * this library reads them as follows (host only, no device work):
 *   profile 0: isothermal T~ = T0 (the default: T0 = 250 K, every delta 0);
 *   profile 1: T~(p) = Ts0 (p/p0)^(R lapse/g), not below Ttrop (a lapse-rate
 *              troposphere under an isothermal stratosphere), g = 9.80665.
 *   b_k = sqrt(kappa R T~(sigma_k)) at each layer's mid sigma; the standard
 *   surface pressure pi~ and temperature T~_s under phis follow from the
 *   hydrostatic column of T~ starting at p0 where phi = 0, and the surface
 *   part of the pressure gradient is R T~_s pi / pi~.  The coefficient c
 *   above multiplies Phi/P in the hydrostatic integral as well as the Omega~
 *   conversion, so the spatial operator stays energy neutral.
 *   Ranges: profile 0 or 1; T0, Ts0, Ttrop > 0; Ttrop <= Ts0; lapse >= 0;
 *   delta finite; delta_c > -1; 0 <= delta_p <= 1.  NULL restores the
 *   default.  Must be called before the first state on the grid is created
 *   (the device tables are built then): AGCM_EINVAL afterwards.
 *   With delta != 0 (the nonlinear delta kappa Phi/P term) ensembles return
 *   AGCM_EINVAL; the step, the tendency and the adjoint step cover it.
 */
typedef struct agcm_thermo {
  int profile;
  double T0, Ts0, lapse, Ttrop;
  double delta, delta_c, delta_p;
} agcm_thermo_t;
int agcm_grid_set_thermo(agcm_grid_t* grid, const agcm_thermo_t* thermo);

/* Copy the stride tables out (leap_u: nlat values, leap_v: nlat-1 values). */
int agcm_grid_leap(const agcm_grid_t* grid, int32_t* leap_u, int32_t* leap_v);

/*
 * Time step from the gravity-wave bound (the paper gives no dt; Sec.
 * "Filtering" only states the CFL condition dt <= dx / U):
 * dt = 1.6 / ((c_max + umax) * sqrt((2/(a cos45 dlam))^2 + (2/(a dth))^2)),
 * c_max^2 the largest eigenvalue of the linear column operator with the
 * level coefficients (1 - delta_p)(1 + delta_c) b_k and the largest R T~_s of
 * the grid.  Host only.
 */
int agcm_grid_dt(const agcm_grid_t* grid, double umax, double* dt);

/*
 * agcm_state_create — device storage for one prognostic state on `grid`
 * (Eq. 1's U, V, Phi and p'_sa/p0) plus the stage buffers of the three-stage
 * step.  precision: AGCM_FP64 or AGCM_FP32 (FP32 keeps the column integral of
 * the surface-pressure tendency in FP64).  nmembers must be 1 (ensembles of
 * uneven grids use agcm_ensemble_*).  The state keeps a reference to `grid`;
 * destroy the state before the grid.
 */
int agcm_state_create(const agcm_grid_t* grid, int precision, int nmembers, agcm_state_t** out);
int agcm_state_destroy(agcm_state_t* state);

/*
 * Load or store the prognostic fields: the forecast variables of Eq. 1 after
 * the IAP transform and the subtraction of the standard stratification
 * (Sec. "Governing equations": U, V, Phi and p'_sa / p0; Eq. 2's F), here
 * U and V (the IAP wind P u, P v), Phi and pi = p'_sa / p0.  Pointers hold
 * the state's element type in the layout above; on_device = 1 for device
 * pointers, 0 for host pointers (pinned host memory gives asynchronous
 * copies).  Asynchronous on `stream`.
 */
int agcm_state_load(agcm_state_t* state, const void* U, const void* V, const void* Phi,
                    const void* pi, int on_device, void* stream);
int agcm_state_store(const agcm_state_t* state, void* U, void* V, void* Phi, void* pi,
                     int on_device, void* stream);

/*
 * agcm_step — advance `nsteps` steps of length dt seconds with the
 * three-stage scheme x1 = xn + dt/2 T(xn), x2 = xn + dt/2 T(x1),
 * x_{n+1} = xn + dt T(x2) (three calls per step: Sec. "Optimizations").
 * T is the full spatial operator of Eq. 1 with the grid's thermodynamics:
 * leap advection, pressure gradient, Coriolis, Omega~ conversion and the
 * column-integrated divergence (Alg. 1 / Alg. 2).  nsteps >= 0 (0 does
 * nothing), dt finite, else AGCM_EINVAL.
 * Asynchronous; launch errors are returned, device-side non-finite values
 * show up in agcm_diagnostics.
 */
int agcm_step(agcm_state_t* state, int nsteps, double dt, void* stream);

/*
 * agcm_filter — the low-latitude filters the leap format keeps (Table
 * "Conventional Filtering scheme"), applied in place to x_n, each zonal row by
 * its latitude: |lat| < 38 deg removes the two-grid-interval wave (the
 * printed sum read as that projection; skipped when nlon is odd);
 * 38..70 deg applies F + r (F_{x-1} - 2F + F_{x+1}) with 0 < r <= 1/4 (the
 * paper's r_j is not given; 1/4 removes the two-grid wave); poleward of 70
 * deg nothing.  Every row sum is kept, so mass is kept.  Asynchronous.
 */
int agcm_filter(agcm_state_t* state, double r, void* stream);

/*
 * agcm_step_split — split time stepping (Sec. "Optimizations": per step the
 * adaptation process is called 3*M times and the advection process 3 times;
 * reading the labels as A = adaptation, L = advection): each of the nsteps
 * steps runs msub three-stage steps of the adaptation terms (pressure
 * gradient, Coriolis pair, Omega~ conversion, dpi/dt) with dt/msub, then one
 * three-stage step of the advection terms with dt.  1 <= msub <= 64.
 * agcm_grid_dt_split: dt from the advective bound alone (flow speed umax) and
 * msub = ceil(dt / gravity-wave dt).  Host only.
 */
int agcm_step_split(agcm_state_t* state, int nsteps, double dt, int msub, void* stream);
int agcm_grid_dt_split(const agcm_grid_t* grid, double umax, double* dt, int* msub);

/*
 * agcm_tendency — T(x) of the current state (Eq. 2: -L + A) into
 * caller-owned device buffers of the state's layout and element type; the
 * state is not modified.  For validation.
 */
int agcm_tendency(agcm_state_t* state, void* tU, void* tV, void* tPhi, void* tpi, void* stream);

/*
 * agcm_step_adjoint — vector-Jacobian product of ONE step at the state x_n
 * currently held by `xn` (not modified): lam_out = (d x_{n+1} / d x_n)^T lam_in,
 * the step being the three-stage scheme over Eq. 1's spatial operator.
 * lam_in[4] / lam_out[4] are caller-owned device buffers {U, V, Phi, pi} of the
 * state's element type and layout; lam_in and lam_out must not alias
 * (AGCM_EINVAL when a lam_in buffer is a lam_out buffer).  The stage states are
 * recomputed from x_n.  Exact transpose of the linearised step, hand-written
 * (no automatic differentiation): every element of the result is formed by one
 * thread from the terms whose stencil reads it, so the result is the same bit
 * for bit on every call.  The first call allocates the state's adjoint
 * workspace (about ten field-sized arrays; AGCM_ENOMEM if that fails).
 * Asynchronous on `stream`.
 */
int agcm_step_adjoint(agcm_state_t* xn, const void* const lam_in[4], void* const lam_out[4], double dt,
                      void* stream);

/*
 * Diagnostics: FP64 global sums and maxima of x_n.  The energy is the total
 * effective energy of Sec. "Validation" (the energy-conservation figure):
 * kinetic plus available potential plus available surface potential energy,
 * in the IAP variables, whose sum the spatial operator conserves exactly;
 * mass is the area sum of the surface pressure.  Synchronises `stream`.
 */
typedef struct agcm_diag {
  double mass;      /* sum_j A_j (pi~ + pi)  [p0 m^2] */
  double e_kin;     /* 1/2 sum dsigma (A U^2 + Av V^2) */
  double e_pot;     /* 1/2 sum dsigma A Phi^2 (available potential) */
  double e_ps;      /* 1/2 sum A (R T~_s / pi~) pi^2 (available surface potential) */
  double energy;    /* e_kin + e_pot + e_ps */
  double max_u;     /* max |U| */
  double max_v;     /* max |V| */
  int32_t finite;   /* 1 if every value is finite, else 0 */
  int32_t reserved;
} agcm_diag_t;
int agcm_diagnostics(const agcm_state_t* state, agcm_diag_t* out, void* stream);

/*
 * Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the library launches for `state` (no effect on results).
 * agcm_profile_enable(state, 1) clears the counters and starts recording;
 * agcm_profile_read synchronises the recorded events and returns, per kernel
 * id 0..agcm_kernel_count()-1, the summed milliseconds and the launch count.
 * The events bracket a whole stage of the stage kernel, which is one launch
 * or several concurrent ones (the row-segment kernel once per stride class,
 * the column kernel for the rows next to the poles; or the column kernel's
 * stride-1 row band and the other rows): its milliseconds are per stage, its
 * count is of launches.
 * ms_total and launches hold at least agcm_kernel_count() entries.
 */
int agcm_profile_enable(agcm_state_t* state, int enable);
/*
 * agcm_set_stage_kernel — which of the library's two designs of the stage
 * kernel runs the steps, tendencies and adjoint recomputes of every state
 * (process-wide; results agree to rounding, both match the oracle).
 *   0 (default): the row-segment kernel (whole latitude-row segments staged in
 *     shared memory) when the grid's rows are 16-byte aligned (nlon % 4 == 0)
 *     and its row segments make at least two waves of CTAs on the GPU, else
 *     the column kernel (one thread per column, stencil read through L1);
 *   1: always the column kernel;
 *   2: the row-segment kernel wherever the rows allow it, on any grid size.
 * Rows whose leap stride exceeds 63 (next to the poles on fine grids) always
 * run the column kernel.  Other values return AGCM_EINVAL.  Host only.
 */
int agcm_set_stage_kernel(int choice);
/*
 * agcm_state_set_stage_kernel — the same choice for one state only: 1 the
 * column kernel, 2 the row-segment kernel wherever the rows allow it, 0 (the
 * default) the process's agcm_set_stage_kernel.  An ensemble of many states
 * stepped side by side on several streams can run its small members on the
 * row-segment kernel, which a state alone would not choose (its segments would
 * not fill the GPU).  Other values or a null state return AGCM_EINVAL.  Host
 * only; takes effect at the state's next launch.
 */
int agcm_state_set_stage_kernel(agcm_state_t* state, int choice);
int agcm_profile_read(agcm_state_t* state, double* ms_total, int64_t* launches);
int agcm_kernel_count(void);
const char* agcm_kernel_name(int id);

/*
 * Ensembles (many members, uneven resolutions, one persistent launch).
 * agcm_ensemble_create: members are existing states, all of one precision,
 * each on its own grid; the ensemble borrows their buffers (destroy it before
 * them).  agcm_ensemble_step advances every member nsteps steps of the
 * three-stage scheme (dt[m] seconds for member m) in one kernel launch whose
 * blocks pull (member, row segment) work items from a device queue; member m
 * does the same arithmetic as agcm_step on it (results agree to about one
 * rounding: the two kernels may contract multiply-adds differently).  Stages are separated
 * by grid barriers whose waits are bounded by the timeout (default 1 s): if a
 * wait runs out the kernel stops and agcm_ensemble_status reports
 * AGCM_ETIMEOUT (this happens only if not all blocks can be resident at once,
 * e.g. when other work occupies the GPU).  The launch can be captured in a
 * CUDA graph once a first call has uploaded the dt values (nsteps = 0 only
 * prepares: it uploads dt and the members' vertical means without stepping).
 * agcm_ensemble_configure sets the launch shape: warps per block 1 (one-warp
 * blocks running the column body on items of 32 columns) or 8 (256-thread
 * blocks running the row-segment body on (member, row segment) items, the
 * rows it leaves on the column body), and blocks per SM (0 = as many as
 * fit); agcm_ensemble_tile sets the row tile of a one-warp work item (1, 2 or
 * 4 consecutive rows of 32 columns, taken by one warp in order); an
 * autotuner picks among them (ensemble.py).  Set both before capturing
 * a graph: a replay keeps the shape it was captured with.
 * agcm_ensemble_set_timeout: barrier timeout in seconds; test_missing_blocks
 * > 0 makes every barrier wait for blocks that do not exist, to exercise the
 * timeout path (tests only).  agcm_ensemble_profile: enable (1) / disable (0)
 * CUDA-event timing of the ensemble launches, or read it (-1 keeps the state)
 * into ms_total / launches when those are non-NULL.
 */
typedef struct agcm_ensemble agcm_ensemble_t;
int agcm_ensemble_create(agcm_state_t* const* members, int n, agcm_ensemble_t** out);
int agcm_ensemble_destroy(agcm_ensemble_t* ens);
int agcm_ensemble_configure(agcm_ensemble_t* ens, int warps_per_block, int blocks_per_sm);
int agcm_ensemble_tile(agcm_ensemble_t* ens, int rows_per_item);
int agcm_ensemble_set_timeout(agcm_ensemble_t* ens, double seconds, int test_missing_blocks);
int agcm_ensemble_step(agcm_ensemble_t* ens, int nsteps, const double* dt, void* stream);
int agcm_ensemble_status(agcm_ensemble_t* ens, void* stream);
int agcm_ensemble_profile(agcm_ensemble_t* ens, int enable, double* ms_total, int64_t* launches);

/*
 * agcm_tendency_static — T(x) like agcm_tendency, for callers that cannot
 * allocate device memory: an application running under a fixed device-memory
 * budget that forbids new allocations, or an embedder whose allocator owns
 * all device memory and lends the library only its buffers.  The paper has no
 * counterpart; this is a deployment convenience.
 *   grid:   created with agcm_grid_create (host only); nlon*nlat <= 262144,
 *           nlat <= 4096, nlev <= 256 — larger grids return AGCM_EINVAL.
 *   U, V, Phi, pi: caller-owned device input (layout above, element type of
 *           `precision`); tU, tV, tPhi, tpi: caller-owned device output.
 * The call allocates nothing: its scratch (the grid's device tables and the
 * FP64 vertical means, about 13 MB) is one fixed array that every GPU holds
 * from library load until process exit.  Every call overwrites the vertical
 * means in that array, and a call on another grid (or precision) rebuilds the
 * tables in it (a call on the grid of the previous call on that device
 * reuses them), so calls whose kernels overlap on a GPU (other streams,
 * other threads) race; serialise them.  The first call on a device looks up
 * the array's device address (set-up, once per device, with that device
 * current); make that first call before any stream capture.  Asynchronous on
 * `stream`.
 */
int agcm_tendency_static(const agcm_grid_t* grid, int precision, const void* U, const void* V, const void* Phi,
                         const void* pi, void* tU, void* tV, void* tPhi, void* tpi, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AGCM_H_ */
