// Oracle for the leap-format IAP dynamical-core step (arXiv 2103.10114).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 CPU statement of
// the discrete scheme.  Only the test-suite, the smoke check and the timed CPU
// baseline may load it; the product library never links, calls or includes
// anything here, and nothing here comes from the product library.
//
// Every quantity follows the paper's notation where the paper has one:
//   Eq. 1   IAP-transformed tendencies of U, V, Phi and p'_sa/p0 (called pi here)
//   Eq. 2   dF/dt = -L_F + A_F, with L the advection part (read: Sec. "Optimizations",
//           which calls L_F the advection process)
//   Eq. 5   the ordinary centred zonal difference
//   Eq. 6   the leap-format centred difference over N_leap points
//   Eq. 7   N_leap from the 45-degree reference spacing
//   Table "Communication aggregation of leap-format difference variables":
//           staggered pairs span an odd stride M, centred pairs span +-M
//   Alg. 1 / Alg. 2   vertical sum and prefix sum that give the sigma velocity
// Where the paper is silent the code takes a reading (R1..R11, F1..F4,
// T1..T4); each is stated at the place it is used.
//
// Parity status: pinned by the tests under tests/ (energy and mass
// conservation, piecewise skewness, reduction to Eq. 5, closed forms of the
// stride-M differences, reflection symmetries, brute-force spectra of the
// linearisation, the printed Eq. 7 values and the zonal grid-size table).
// Agreement with the authors' own IAP-AGCM code is unpinned: the paper prints
// neither the full discrete equations nor their coefficients.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---- constants (reading R2; only the Earth radius is fixed by the paper,
//      through the zonal grid-size table) --------------------------------
const double kA = 6.371e6;        // Earth radius [m]
const double kOmega = 7.292e-5;   // rotation rate [1/s]
const double kR = 287.04;         // gas constant of dry air
const double kCp = 1004.64;       // heat capacity at constant pressure
const double kT0 = 250.0;         // default isothermal standard stratification [K] (reading R2)
const double kPi = 3.14159265358979323846;
const double kG = 9.80665;        // gravity, for the standard atmosphere's lapse rate [m/s^2]

// ---- forward-mode dual number: value + one directional derivative --------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double sqrt(double a) { return std::sqrt(a); }

// ---- operation counter: a double that tallies the arithmetic it takes part
// in (one count per add/subtract, multiply, divide, square root).  Used only
// to state the scheme's operations per grid point; results are bit-identical
// to the plain double instantiation.
struct OpTally {
  unsigned long long add = 0, mul = 0, div = 0, sqrt = 0;
};
static OpTally g_tally;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_tally.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_tally.add; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_tally.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_tally.div; return Cnt(a.v / b.v); }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, Cnt b) { return Cnt(a) + b; }
inline Cnt operator-(Cnt a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, Cnt b) { return Cnt(a) - b; }
inline Cnt operator*(Cnt a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, Cnt b) { return Cnt(a) * b; }
inline Cnt operator/(Cnt a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, Cnt b) { return Cnt(a) / b; }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt sqrt(Cnt a) { ++g_tally.sqrt; return Cnt(std::sqrt(a.v)); }

// ---- Eq. 7 ------------------------------------------------------------
// ratio of the 45-degree zonal spacing to the spacing at colatitude theta;
// cos(90deg - theta) = sin(theta) and res = the zonal grid step.
double leap_ratio(double theta, double dlam) {
  return std::asin(std::cos(kPi / 4.0) * std::sin(dlam)) /
         std::asin(std::sin(theta) * std::sin(dlam));
}

// Reading R3: N = max(1, ceil(ratio)); a ratio within 1e-9 of an integer
// counts as that integer, so the reference latitude itself keeps stride 1.
// The operator stride M is N raised to the next odd number, because U sits on
// half points (Sec. "Leap-Format Difference Scheme": N_leap must be odd).
int leap_stride(double theta, double dlam) {
  double r = leap_ratio(theta, dlam);
  int n = (int)std::ceil(r - 1e-9);
  if (n < 1) n = 1;
  if (n % 2 == 0) n += 1;
  return n;
}

// ---- standard stratification and the Eq. 1 coefficient of Omega~ ----------
// Eq. 1 subtracts a standard stratification T~(p) and scales the Omega~ term
// of the Phi equation by (1 - delta_p)[b(1 + delta_c) + delta kappa Phi / P];
// the paper defines neither T~ nor the deltas (readings T1..T4).
struct Thermo {
  int profile = 0;     // 0: isothermal T0; 1: lapse rate to a tropopause, isothermal above (T1)
  double T0 = kT0;     // isothermal temperature [K]
  double Ts0 = 288.15, lapse = 6.5e-3, Ttrop = 216.65;  // profile 1: T at p0, -dT/dz, tropopause T
  double delta = 0.0, delta_c = 0.0, delta_p = 0.0;    // Eq. 1's switches (T4)
};

// T~ at p / p0 (T1): profile 1 is T = Ts0 (p/p0)^(R lapse / g), not below Ttrop.
double std_temp(const Thermo& t, double p) {
  if (t.profile == 0) return t.T0;
  if (t.lapse == 0.0) return t.Ts0;
  return std::fmax(t.Ts0 * std::pow(p, kR * t.lapse / kG), t.Ttrop);
}

// Standard surface pressure / p0 and temperature under surface geopotential
// phis: the hydrostatic column of T~ from p0 at phi = 0 (T3).
void std_surface(const Thermo& t, double phis, double* pit, double* Ts) {
  if (t.profile == 0) {
    *pit = std::exp(-phis / (kR * t.T0));
    *Ts = t.T0;
    return;
  }
  if (t.lapse == 0.0) {
    *pit = std::exp(-phis / (kR * t.Ts0));
    *Ts = t.Ts0;
    return;
  }
  const double z = phis / kG, ex = kG / (kR * t.lapse);
  const double T = t.Ts0 - t.lapse * z;
  if (T >= t.Ttrop) {
    *pit = std::pow(T / t.Ts0, ex);
    *Ts = T;
  } else {
    const double ztr = (t.Ts0 - t.Ttrop) / t.lapse;
    *pit = std::pow(t.Ttrop / t.Ts0, ex) * std::exp(-kG * (z - ztr) / (kR * t.Ttrop));
    *Ts = t.Ttrop;
  }
}

struct Grid {
  int I = 0, J = 0, K = 0;
  double dlam = 0, dth = 0;
  // scalar/U rows j = 0..J-1 at colatitude (j+1/2) dth   (reading R1)
  std::vector<double> s, c, cot, A;
  // V rows j = 0..J-2 at colatitude (j+1) dth; V = 0 on the pole edges
  std::vector<double> sv, Av;
  std::vector<int> Mu, Mv;
  // sigma: half levels sh[0..K] with sh[0] = 0 (model top) and sh[K] = 1
  std::vector<double> sh, ds, H;  // H is K x K, row-major
  std::vector<double> pit;        // standard surface pressure / p0, J x I
  std::vector<double> rts;        // R T~_s of each column, J x I (T3)
  std::vector<double> phis;       // surface geopotential, J x I
  std::vector<double> beta;       // (1 - delta_p)(1 + delta_c) b_k, b_k = sqrt(kappa R T~(sigma_k)) (T2)
  double beta2 = 0;               // (1 - delta_p) delta kappa: the Phi-dependent part of the coefficient
  Thermo th;
};

// The thermodynamic tables of a grid from its Thermo (T1..T4).
void apply_thermo(Grid& g) {
  const Thermo& t = g.th;
  const double kap = kR / kCp;
  g.beta.resize(g.K);
  for (int k = 0; k < g.K; ++k) {
    const double sig = 0.5 * (g.sh[k] + g.sh[k + 1]);
    g.beta[k] = (1.0 - t.delta_p) * (1.0 + t.delta_c) * std::sqrt(kap * kR * std_temp(t, sig));
  }
  g.beta2 = (1.0 - t.delta_p) * t.delta * kap;
  g.pit.resize((size_t)g.J * g.I);
  g.rts.resize(g.pit.size());
  for (size_t n = 0; n < g.pit.size(); ++n) {
    double Ts = 0;
    std_surface(t, g.phis[n], &g.pit[n], &Ts);
    g.rts[n] = kR * Ts;
  }
}

// ---- storage helpers ---------------------------------------------------
struct Ix {
  int I, J, K;
  size_t s3(int k, int j, int i) const { return ((size_t)k * J + j) * I + i; }
  size_t v3(int k, int j, int i) const { return ((size_t)k * (J - 1) + j) * I + i; }
  size_t s2(int j, int i) const { return (size_t)j * I + i; }
  size_t h3(int h, int j, int i) const { return ((size_t)h * J + j) * I + i; }
  int w(int i) const {
    int r = i % I;
    return r < 0 ? r + I : r;
  }
};

enum : unsigned {
  TERM_ADV = 1u,      // advection L_1 + L_2 + L_3 of U, V, Phi
  TERM_COR = 2u,      // Coriolis pair with f* = 2 Omega cos(theta) + u cot(theta)/a
  TERM_PGF_PI = 4u,   // R T0 pi / pi~ part of the pressure gradient, and dpi/dt
  TERM_PGF_PHI = 8u,  // hydrostatic phi' part of the pressure gradient, and Omega~
  TERM_ALL = 15u
};

// ---- the spatial operator T(x) = -L(x) + A(x) of Eq. 2 -------------------
template <class T>
void tendency(const Grid& g, const T* U, const T* V, const T* Ph, const T* pi, T* tU,
              T* tV, T* tPh, T* tpi, unsigned terms) {
  const int I = g.I, J = g.J, K = g.K, JV = J - 1;
  const Ix x{I, J, K};
  const double a = kA, dlam = g.dlam, dth = g.dth;

  // a2: mass m = p_es/p0 = pi~ + pi, P = sqrt(m); P at U and V points from
  //     the stride-1 mean of m (reading: P^2 at a face is the mean mass).
  std::vector<T> m((size_t)J * I), P((size_t)J * I), Pu((size_t)J * I), Pv((size_t)JV * I);
  for (int j = 0; j < J; ++j)
    for (int i = 0; i < I; ++i) {
      m[x.s2(j, i)] = g.pit[x.s2(j, i)] + pi[x.s2(j, i)];
      P[x.s2(j, i)] = sqrt(m[x.s2(j, i)]);
    }
  for (int j = 0; j < J; ++j)
    for (int u = 0; u < I; ++u)
      Pu[x.s2(j, u)] = sqrt(0.5 * (m[x.s2(j, u)] + m[x.s2(j, x.w(u + 1))]));
  for (int j = 0; j < JV; ++j)
    for (int i = 0; i < I; ++i)
      Pv[x.s2(j, i)] = sqrt(0.5 * (m[x.s2(j, i)] + m[x.s2(j + 1, i)]));

  // a3: mass fluxes and the leap-format divergence (Eq. 6 applied to the
  //     staggered zonal flux, stride M_j; ordinary difference in latitude).
  const size_t n3 = (size_t)K * J * I, nv = (size_t)K * JV * I;
  std::vector<T> Fl(n3), Ft(nv), D(n3);
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < J; ++j)
      for (int u = 0; u < I; ++u) Fl[x.s3(k, j, u)] = Pu[x.s2(j, u)] * U[x.s3(k, j, u)];
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < JV; ++j)
      for (int i = 0; i < I; ++i) Ft[x.v3(k, j, i)] = Pv[x.s2(j, i)] * V[x.v3(k, j, i)];
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < J; ++j) {
      const int M = g.Mu[j];
      for (int i = 0; i < I; ++i) {
        T zonal = (Fl[x.s3(k, j, x.w(i + (M - 1) / 2))] - Fl[x.s3(k, j, x.w(i - (M + 1) / 2))]) /
                  (a * g.s[j] * M * dlam);
        T south = (j < JV) ? g.sv[j] * Ft[x.v3(k, j, i)] : T(0.0);
        T north = (j > 0) ? g.sv[j - 1] * Ft[x.v3(k, j - 1, i)] : T(0.0);
        D[x.s3(k, j, i)] = zonal + (south - north) / (a * g.s[j] * dth);
      }
    }

  // a4: column integrals (Alg. 1 / Alg. 2): C = sum_k dsigma_k D_k gives
  //     dpi/dt = -C; the vertical mass flux at half level h is
  //     W_h = sh_h C - sum_{k<h} dsigma_k D_k, zero at the top and the bottom.
  std::vector<T> C((size_t)J * I);
  std::vector<T> W((size_t)(K + 1) * J * I);
  for (int j = 0; j < J; ++j)
    for (int i = 0; i < I; ++i) {
      T sum = 0.0;
      for (int k = 0; k < K; ++k) sum += g.ds[k] * D[x.s3(k, j, i)];
      C[x.s2(j, i)] = sum;
      W[x.h3(0, j, i)] = 0.0;
      W[x.h3(K, j, i)] = 0.0;
      for (int h = 1; h < K; ++h) {
        T part = 0.0;
        for (int k = 0; k < h; ++k) part += g.ds[k] * D[x.s3(k, j, i)];
        W[x.h3(h, j, i)] = g.sh[h] * sum - part;
      }
    }

  // Eq. 1's coefficient of Omega~ at (k, j, i): c = beta_k + beta2 Phi / P
  //     (reading T4; beta2 = 0 unless the delta kappa Phi / P term is on).
  auto coef = [&](int k, int j, int i) -> T {
    if (g.beta2 == 0.0) return T(g.beta[k]);
    return g.beta[k] + g.beta2 * Ph[x.s3(k, j, i)] / P[x.s2(j, i)];
  };

  // a5: psi = phi' + R T~_s pi / pi~, with phi'_k = sum_k' H[k][k'] (c/P) Phi_k'
  //     (hydrostatic integral from the surface, reading R7; isothermal
  //     T~ = T0 gives c = b).
  std::vector<T> psi(n3);
  for (int j = 0; j < J; ++j)
    for (int i = 0; i < I; ++i) {
      const T ps = g.rts[x.s2(j, i)] * pi[x.s2(j, i)] / g.pit[x.s2(j, i)];
      for (int k = 0; k < K; ++k) {
        T phi = 0.0;
        for (int kk = 0; kk < K; ++kk)
          phi += g.H[(size_t)k * K + kk] * ((coef(kk, j, i) / P[x.s2(j, i)]) * Ph[x.s3(kk, j, i)]);
        T val = 0.0;
        if (terms & TERM_PGF_PHI) val += phi;
        if (terms & TERM_PGF_PI) val += ps;
        psi[x.s3(k, j, i)] = val;
      }
    }

  for (size_t n = 0; n < n3; ++n) { tU[n] = 0.0; tPh[n] = 0.0; }
  for (size_t n = 0; n < nv; ++n) tV[n] = 0.0;
  for (size_t n = 0; n < (size_t)J * I; ++n) tpi[n] = 0.0;

  // a6: pressure gradient  -P^u (psi[i+(M+1)/2] - psi[i-(M-1)/2]) / (a sin M dlam)
  //     at U points and -P^v (psi_{j+1} - psi_j) / (a dth) at V points.
  if (terms & (TERM_PGF_PI | TERM_PGF_PHI)) {
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < J; ++j) {
        const int M = g.Mu[j];
        for (int u = 0; u < I; ++u) {
          T grad = (psi[x.s3(k, j, x.w(u + (M + 1) / 2))] - psi[x.s3(k, j, x.w(u - (M - 1) / 2))]) /
                   (a * g.s[j] * M * dlam);
          tU[x.s3(k, j, u)] -= Pu[x.s2(j, u)] * grad;
        }
      }
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < JV; ++j)
        for (int i = 0; i < I; ++i) {
          T grad = (psi[x.s3(k, j + 1, i)] - psi[x.s3(k, j, i)]) / (a * dth);
          tV[x.v3(k, j, i)] -= Pv[x.s2(j, i)] * grad;
        }
  }
  // a7: Omega~ conversion, the exact H-transpose of a5 with the same c:
  //     dPhi_k/dt += -(c/P) (1/dsigma_k) sum_k' H[k'][k] dsigma_k' D_k'.
  if (terms & TERM_PGF_PHI) {
    for (int j = 0; j < J; ++j)
      for (int i = 0; i < I; ++i) {
        for (int k = 0; k < K; ++k) {
          T acc = 0.0;
          for (int kk = 0; kk < K; ++kk) acc += g.H[(size_t)kk * K + k] * (g.ds[kk] * D[x.s3(kk, j, i)]);
          tPh[x.s3(k, j, i)] -= (coef(k, j, i) / P[x.s2(j, i)]) * acc / g.ds[k];
        }
      }
  }
  if (terms & TERM_PGF_PI)
    for (int j = 0; j < J; ++j)
      for (int i = 0; i < I; ++i) tpi[x.s2(j, i)] = -C[x.s2(j, i)];

  // a8: Coriolis pair.  Each (U, V) pair touching at a cell corner carries
  //     B = 1/4 A_j f*(U point) U V; U_t = -(1/A_j) dB/dU, V_t = +(1/Av) dB/dV
  //     with f* frozen inside the form (reading R8), so the pair is energy neutral.
  if (terms & TERM_COR) {
    auto fstar = [&](int k, int j, int u) -> T {
      return 2.0 * kOmega * g.c[j] + (U[x.s3(k, j, u)] / Pu[x.s2(j, u)]) * g.cot[j] / a;
    };
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < J; ++j)
        for (int u = 0; u < I; ++u) {
          T vs = 0.0;
          if (j > 0) vs += V[x.v3(k, j - 1, u)] + V[x.v3(k, j - 1, x.w(u + 1))];
          if (j < JV) vs += V[x.v3(k, j, u)] + V[x.v3(k, j, x.w(u + 1))];
          tU[x.s3(k, j, u)] -= 0.25 * fstar(k, j, u) * vs;
        }
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < JV; ++j)
        for (int i = 0; i < I; ++i) {
          const int im = x.w(i - 1);
          T up = g.A[j] * (fstar(k, j, im) * U[x.s3(k, j, im)] + fstar(k, j, i) * U[x.s3(k, j, i)]);
          T dn = g.A[j + 1] *
                 (fstar(k, j + 1, im) * U[x.s3(k, j + 1, im)] + fstar(k, j + 1, i) * U[x.s3(k, j + 1, i)]);
          tV[x.v3(k, j, i)] += 0.25 * (up + dn) / g.Av[j];
        }
  }

  // a9: advection in the skew form L(F)_c = 1/(2 A_c P_c) sum_faces flux_f G_n,
  //     G = F/P, pairs across every face; zonal partners at +-M (Table
  //     "Communication aggregation": the centred pattern x +- (2N-1)).
  if (terms & TERM_ADV) {
    std::vector<T> Gs(n3), Gu(n3), Gv(nv);
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < J; ++j)
        for (int i = 0; i < I; ++i) {
          Gs[x.s3(k, j, i)] = Ph[x.s3(k, j, i)] / P[x.s2(j, i)];
          Gu[x.s3(k, j, i)] = U[x.s3(k, j, i)] / Pu[x.s2(j, i)];
        }
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < JV; ++j)
        for (int i = 0; i < I; ++i) Gv[x.v3(k, j, i)] = V[x.v3(k, j, i)] / Pv[x.s2(j, i)];

    // scalar (Phi) cells
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < J; ++j) {
        const int M = g.Mu[j];
        for (int i = 0; i < I; ++i) {
          T ZE = (a * dth / M) * Fl[x.s3(k, j, x.w(i + (M - 1) / 2))];
          T ZW = (a * dth / M) * Fl[x.s3(k, j, x.w(i - (M + 1) / 2))];
          T hor = ZE * Gs[x.s3(k, j, x.w(i + M))] - ZW * Gs[x.s3(k, j, x.w(i - M))];
          if (j < JV) hor += (a * dlam * g.sv[j]) * Ft[x.v3(k, j, i)] * Gs[x.s3(k, j + 1, i)];
          if (j > 0) hor -= (a * dlam * g.sv[j - 1]) * Ft[x.v3(k, j - 1, i)] * Gs[x.s3(k, j - 1, i)];
          T ver = 0.0;
          if (k < K - 1) ver += W[x.h3(k + 1, j, i)] * Gs[x.s3(k + 1, j, i)];
          if (k > 0) ver -= W[x.h3(k, j, i)] * Gs[x.s3(k - 1, j, i)];
          const T Pc = P[x.s2(j, i)];
          T L = hor / (2.0 * g.A[j] * Pc) + ver / (2.0 * g.ds[k] * Pc);
          tPh[x.s3(k, j, i)] -= L;
        }
      }
    // U cells: fluxes are stride-1 means of the scalar-cell fluxes; the zonal
    // face toward the partner u+-M sits at the scalar point midway.
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < J; ++j) {
        const int M = g.Mu[j];
        for (int u = 0; u < I; ++u) {
          const int iE = u + (M + 1) / 2, iW = u - (M - 1) / 2;
          T ZE = (a * dth / M) * 0.5 * (Fl[x.s3(k, j, x.w(iE - 1))] + Fl[x.s3(k, j, x.w(iE))]);
          T ZW = (a * dth / M) * 0.5 * (Fl[x.s3(k, j, x.w(iW - 1))] + Fl[x.s3(k, j, x.w(iW))]);
          T hor = ZE * Gu[x.s3(k, j, x.w(u + M))] - ZW * Gu[x.s3(k, j, x.w(u - M))];
          if (j < JV) {
            T YS = 0.5 * a * dlam * g.sv[j] * (Ft[x.v3(k, j, u)] + Ft[x.v3(k, j, x.w(u + 1))]);
            hor += YS * Gu[x.s3(k, j + 1, u)];
          }
          if (j > 0) {
            T YN = 0.5 * a * dlam * g.sv[j - 1] * (Ft[x.v3(k, j - 1, u)] + Ft[x.v3(k, j - 1, x.w(u + 1))]);
            hor -= YN * Gu[x.s3(k, j - 1, u)];
          }
          T ver = 0.0;
          if (k < K - 1) {
            T Wb = 0.5 * (W[x.h3(k + 1, j, u)] + W[x.h3(k + 1, j, x.w(u + 1))]);
            ver += Wb * Gu[x.s3(k + 1, j, u)];
          }
          if (k > 0) {
            T Wt = 0.5 * (W[x.h3(k, j, u)] + W[x.h3(k, j, x.w(u + 1))]);
            ver -= Wt * Gu[x.s3(k - 1, j, u)];
          }
          const T Pc = Pu[x.s2(j, u)];
          T L = hor / (2.0 * g.A[j] * Pc) + ver / (2.0 * g.ds[k] * Pc);
          tU[x.s3(k, j, u)] -= L;
        }
      }
    // V cells: zonal faces at the U longitude midway to the partner i+-Mv,
    // flux = mean of the two adjacent scalar rows' zonal fluxes there.
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < JV; ++j) {
        const int M = g.Mv[j];
        for (int i = 0; i < I; ++i) {
          const int uE = x.w(i + (M - 1) / 2), uW = x.w(i - (M + 1) / 2);
          T ZE = (a * dth / M) * 0.5 * (Fl[x.s3(k, j, uE)] + Fl[x.s3(k, j + 1, uE)]);
          T ZW = (a * dth / M) * 0.5 * (Fl[x.s3(k, j, uW)] + Fl[x.s3(k, j + 1, uW)]);
          T hor = ZE * Gv[x.v3(k, j, x.w(i + M))] - ZW * Gv[x.v3(k, j, x.w(i - M))];
          if (j + 1 < JV) {
            T YS = 0.5 * a * dlam * (g.sv[j] * Ft[x.v3(k, j, i)] + g.sv[j + 1] * Ft[x.v3(k, j + 1, i)]);
            hor += YS * Gv[x.v3(k, j + 1, i)];
          }
          if (j > 0) {
            T YN = 0.5 * a * dlam * (g.sv[j - 1] * Ft[x.v3(k, j - 1, i)] + g.sv[j] * Ft[x.v3(k, j, i)]);
            hor -= YN * Gv[x.v3(k, j - 1, i)];
          }
          T ver = 0.0;
          if (k < K - 1) {
            T Wb = 0.5 * (W[x.h3(k + 1, j, i)] + W[x.h3(k + 1, j + 1, i)]);
            ver += Wb * Gv[x.v3(k + 1, j, i)];
          }
          if (k > 0) {
            T Wt = 0.5 * (W[x.h3(k, j, i)] + W[x.h3(k, j + 1, i)]);
            ver -= Wt * Gv[x.v3(k - 1, j, i)];
          }
          const T Pc = Pv[x.s2(j, i)];
          T L = hor / (2.0 * g.Av[j] * Pc) + ver / (2.0 * g.ds[k] * Pc);
          tV[x.v3(k, j, i)] -= L;
        }
      }
  }
}

// a10: three-stage step (reading R9; "3 calls" per process per step):
//   x1 = xn + dt/2 T(xn);  x2 = xn + dt/2 T(x1);  x_{n+1} = xn + dt T(x2)
template <class T>
void step(const Grid& g, T* U, T* V, T* Ph, T* pi, double dt, int nsteps, unsigned terms) {
  const size_t n3 = (size_t)g.K * g.J * g.I, nv = (size_t)g.K * (g.J - 1) * g.I,
               n2 = (size_t)g.J * g.I;
  std::vector<T> sU(n3), sV(nv), sP(n3), sp(n2), tU(n3), tV(nv), tP(n3), tp(n2);
  const double coef[3] = {0.5 * dt, 0.5 * dt, dt};
  for (int n = 0; n < nsteps; ++n) {
    for (size_t q = 0; q < n3; ++q) { sU[q] = U[q]; sP[q] = Ph[q]; }
    for (size_t q = 0; q < nv; ++q) sV[q] = V[q];
    for (size_t q = 0; q < n2; ++q) sp[q] = pi[q];
    for (int st = 0; st < 3; ++st) {
      tendency<T>(g, sU.data(), sV.data(), sP.data(), sp.data(), tU.data(), tV.data(), tP.data(),
                  tp.data(), terms);
      for (size_t q = 0; q < n3; ++q) { sU[q] = U[q] + coef[st] * tU[q]; sP[q] = Ph[q] + coef[st] * tP[q]; }
      for (size_t q = 0; q < nv; ++q) sV[q] = V[q] + coef[st] * tV[q];
      for (size_t q = 0; q < n2; ++q) sp[q] = pi[q] + coef[st] * tp[q];
    }
    for (size_t q = 0; q < n3; ++q) { U[q] = sU[q]; Ph[q] = sP[q]; }
    for (size_t q = 0; q < nv; ++q) V[q] = sV[q];
    for (size_t q = 0; q < n2; ++q) pi[q] = sp[q];
  }
}

}  // namespace

// ---- low-latitude filters (Table "Conventional Filtering scheme") ---------
// Band by latitude phi = 90deg - colatitude: 1 = "simplified" filter for
// |phi| < 38deg, read as removing the two-grid-interval zonal wave exactly
// (the printed sum is garbled: F_x - (-1)^x (1/I) sum_x' (-1)^x' F_x');
// 2 = the 3-point operator F_x + r (F_{x-1} - 2 F_x + F_{x+1}) for
// 38deg <= |phi| <= 70deg; 0 = none (the leap format covers |phi| > 70deg).
int filter_band(double colat) {
  const double lat = std::fabs(90.0 - colat * 180.0 / kPi);
  if (lat < 38.0) return 1;
  if (lat <= 70.0) return 2;
  return 0;
}

void filter_row(double* F, int I, int band, double r) {
  if (band == 1) {
    if (I % 2 != 0) return;  // no two-grid wave on an odd circle
    double alt = 0.0;
    for (int x = 0; x < I; ++x) alt += (x % 2 == 0 ? 1.0 : -1.0) * F[x];
    const double a = alt / I;
    for (int x = 0; x < I; ++x) F[x] -= (x % 2 == 0 ? 1.0 : -1.0) * a;
  } else if (band == 2) {
    std::vector<double> old(F, F + I);
    for (int x = 0; x < I; ++x) {
      const double l = old[(x - 1 + I) % I], c = old[x], rr = old[(x + 1) % I];
      F[x] = c + r * (l - 2.0 * c + rr);
    }
  }
}

// ======================= C interface for the tests =========================
extern "C" {

double orc_leap_ratio(double theta, double dlam) { return leap_ratio(theta, dlam); }

// zonal grid size a sin(theta) dlam (Table "zonal grid size in different resolutions")
double orc_zonal_dx(double theta, double dlam) { return kA * std::sin(theta) * dlam; }

void orc_leap_table(int I, int J, int32_t* Mu, int32_t* Mv) {
  const double dlam = 2.0 * kPi / I, dth = kPi / J;
  for (int j = 0; j < J; ++j) Mu[j] = leap_stride((j + 0.5) * dth, dlam);
  for (int j = 0; j + 1 < J; ++j) Mv[j] = leap_stride((j + 1.0) * dth, dlam);
}

// Build a grid; NULL tables select the defaults (uniform sigma, Eq. 7 strides,
// flat terrain).  Returns NULL when an argument is invalid.
void* orc_create(int I, int J, int K, const double* sigma_half, const int32_t* Mu,
                 const int32_t* Mv, const double* phis) {
  if (I < 3 || J < 2 || K < 1) return nullptr;
  Grid* g = new Grid;
  g->I = I; g->J = J; g->K = K;
  g->dlam = 2.0 * kPi / I;
  g->dth = kPi / J;
  g->s.resize(J); g->c.resize(J); g->cot.resize(J); g->A.resize(J); g->Mu.resize(J);
  g->sv.resize(J - 1); g->Av.resize(J - 1); g->Mv.resize(J - 1);
  for (int j = 0; j < J; ++j) {
    const double th = (j + 0.5) * g->dth;
    g->s[j] = std::sin(th);
    g->c[j] = std::cos(th);
    g->cot[j] = g->c[j] / g->s[j];
    g->A[j] = kA * kA * g->s[j] * g->dth * g->dlam;
    g->Mu[j] = Mu ? Mu[j] : leap_stride(th, g->dlam);
  }
  for (int j = 0; j + 1 < J; ++j) {
    const double th = (j + 1.0) * g->dth;
    g->sv[j] = std::sin(th);
    g->Av[j] = kA * kA * g->sv[j] * g->dth * g->dlam;
    g->Mv[j] = Mv ? Mv[j] : leap_stride(th, g->dlam);
  }
  for (int j = 0; j < J; ++j)
    if (g->Mu[j] < 1 || g->Mu[j] % 2 == 0 || 2 * g->Mu[j] >= I) { delete g; return nullptr; }
  for (int j = 0; j + 1 < J; ++j)
    if (g->Mv[j] < 1 || g->Mv[j] % 2 == 0 || 2 * g->Mv[j] >= I) { delete g; return nullptr; }
  g->sh.resize(K + 1);
  for (int h = 0; h <= K; ++h) g->sh[h] = sigma_half ? sigma_half[h] : (double)h / K;
  if (g->sh[0] != 0.0 || g->sh[K] != 1.0) { delete g; return nullptr; }
  g->ds.resize(K);
  for (int k = 0; k < K; ++k) {
    g->ds[k] = g->sh[k + 1] - g->sh[k];
    if (!(g->ds[k] > 0.0)) { delete g; return nullptr; }
  }
  // reading R7: H[k][k] = ln(sh_{k+1}/sigma_k) with sigma_k the layer midpoint,
  // H[k][k'] = ln(sh_{k'+1}/sh_{k'}) for k' below k, zero above.
  g->H.assign((size_t)K * K, 0.0);
  for (int k = 0; k < K; ++k) {
    const double sig = 0.5 * (g->sh[k] + g->sh[k + 1]);
    g->H[(size_t)k * K + k] = std::log(g->sh[k + 1] / sig);
    for (int kk = k + 1; kk < K; ++kk) g->H[(size_t)k * K + kk] = std::log(g->sh[kk + 1] / g->sh[kk]);
  }
  // reading R2: by default pi~ = exp(-phi_s / (R T0)), the isothermal standard
  // surface pressure, and b = sqrt(kappa R T0) on every level
  g->phis.assign((size_t)J * I, 0.0);
  if (phis) g->phis.assign(phis, phis + (size_t)J * I);
  apply_thermo(*g);
  return g;
}

void orc_destroy(void* h) { delete static_cast<Grid*>(h); }

// p = {profile, T0, Ts0, lapse, Ttrop, delta, delta_c, delta_p}; returns 0, or
// -1 for values outside their range (the grid is then unchanged).
int orc_set_thermo(void* h, const double* p) {
  Thermo t;
  t.profile = (int)p[0];
  t.T0 = p[1]; t.Ts0 = p[2]; t.lapse = p[3]; t.Ttrop = p[4];
  t.delta = p[5]; t.delta_c = p[6]; t.delta_p = p[7];
  if ((t.profile != 0 && t.profile != 1) || !(t.T0 > 0) || !(t.Ts0 > 0) || !(t.lapse >= 0) || !(t.Ttrop > 0) ||
      t.Ttrop > t.Ts0 || !(t.delta_c > -1) || !(t.delta_p >= 0 && t.delta_p <= 1) || !std::isfinite(t.delta))
    return -1;
  Grid& g = *static_cast<Grid*>(h);
  g.th = t;
  apply_thermo(g);
  return 0;
}

double orc_std_temp(const double* p, double p_over_p0) {
  Thermo t;
  t.profile = (int)p[0]; t.T0 = p[1]; t.Ts0 = p[2]; t.lapse = p[3]; t.Ttrop = p[4];
  return std_temp(t, p_over_p0);
}

void orc_std_surface(const double* p, double phis, double* out) {
  Thermo t;
  t.profile = (int)p[0]; t.T0 = p[1]; t.Ts0 = p[2]; t.lapse = p[3]; t.Ttrop = p[4];
  std_surface(t, phis, out, out + 1);
}

void orc_get_leap(void* h, int32_t* Mu, int32_t* Mv) {
  const Grid* g = static_cast<Grid*>(h);
  for (int j = 0; j < g->J; ++j) Mu[j] = g->Mu[j];
  for (int j = 0; j + 1 < g->J; ++j) Mv[j] = g->Mv[j];
}

void orc_tendency(void* h, const double* U, const double* V, const double* Ph, const double* pi,
                  double* tU, double* tV, double* tPh, double* tpi, unsigned terms) {
  tendency<double>(*static_cast<Grid*>(h), U, V, Ph, pi, tU, tV, tPh, tpi, terms);
}

// The tendency through the counting type: writes the tendency (identical to
// orc_tendency) and ops[4] = adds, multiplies, divides, square roots of one
// evaluation on state values (geometry-only products are table work, not
// counted).
void orc_tendency_opcount(void* h, const double* U, const double* V, const double* Ph, const double* pi,
                          double* tU, double* tV, double* tPh, double* tpi, unsigned terms,
                          unsigned long long* ops) {
  const Grid& g = *static_cast<Grid*>(h);
  const size_t n3 = (size_t)g.K * g.J * g.I, nv = (size_t)g.K * (g.J - 1) * g.I, n2 = (size_t)g.J * g.I;
  std::vector<Cnt> u(U, U + n3), v(V, V + nv), p(Ph, Ph + n3), q(pi, pi + n2);
  std::vector<Cnt> tu(n3), tv(std::max<size_t>(nv, 1)), tp(n3), tq(n2);
  g_tally = OpTally();
  tendency<Cnt>(g, u.data(), v.data(), p.data(), q.data(), tu.data(), tv.data(), tp.data(), tq.data(), terms);
  ops[0] = g_tally.add;
  ops[1] = g_tally.mul;
  ops[2] = g_tally.div;
  ops[3] = g_tally.sqrt;
  for (size_t n = 0; n < n3; ++n) { tU[n] = tu[n].v; tPh[n] = tp[n].v; }
  for (size_t n = 0; n < nv; ++n) tV[n] = tv[n].v;
  for (size_t n = 0; n < n2; ++n) tpi[n] = tq[n].v;
}

void orc_step(void* h, double* U, double* V, double* Ph, double* pi, double dt, int nsteps,
              unsigned terms) {
  step<double>(*static_cast<Grid*>(h), U, V, Ph, pi, dt, nsteps, terms);
}

// Jacobian-vector products: the derivative of the tendency (or of nsteps
// steps) at x along dx, by forward-mode dual numbers through the same code.
static void pack(const double* x, const double* dx, size_t n, std::vector<Dual>& out) {
  out.resize(n);
  for (size_t q = 0; q < n; ++q) out[q] = Dual(x[q], dx[q]);
}
static void unpack(const std::vector<Dual>& in, double* x, double* dx) {
  for (size_t q = 0; q < in.size(); ++q) {
    if (x) x[q] = in[q].v;
    dx[q] = in[q].d;
  }
}

void orc_tendency_jvp(void* h, const double* U, const double* V, const double* Ph, const double* pi,
                      const double* dU, const double* dV, const double* dPh, const double* dpi,
                      double* jU, double* jV, double* jPh, double* jpi, unsigned terms) {
  const Grid& g = *static_cast<Grid*>(h);
  const size_t n3 = (size_t)g.K * g.J * g.I, nv = (size_t)g.K * (g.J - 1) * g.I, n2 = (size_t)g.J * g.I;
  std::vector<Dual> xU, xV, xP, xp, tU(n3), tV(nv), tP(n3), tp(n2);
  pack(U, dU, n3, xU); pack(V, dV, nv, xV); pack(Ph, dPh, n3, xP); pack(pi, dpi, n2, xp);
  tendency<Dual>(g, xU.data(), xV.data(), xP.data(), xp.data(), tU.data(), tV.data(), tP.data(),
                 tp.data(), terms);
  unpack(tU, nullptr, jU); unpack(tV, nullptr, jV); unpack(tP, nullptr, jPh); unpack(tp, nullptr, jpi);
}

// In/out: (U,V,Ph,pi) advance nsteps; (dU,dV,dPh,dpi) become J^nsteps applied to them.
void orc_step_jvp(void* h, double* U, double* V, double* Ph, double* pi, double* dU, double* dV,
                  double* dPh, double* dpi, double dt, int nsteps, unsigned terms) {
  const Grid& g = *static_cast<Grid*>(h);
  const size_t n3 = (size_t)g.K * g.J * g.I, nv = (size_t)g.K * (g.J - 1) * g.I, n2 = (size_t)g.J * g.I;
  std::vector<Dual> xU, xV, xP, xp;
  pack(U, dU, n3, xU); pack(V, dV, nv, xV); pack(Ph, dPh, n3, xP); pack(pi, dpi, n2, xp);
  step<Dual>(g, xU.data(), xV.data(), xP.data(), xp.data(), dt, nsteps, terms);
  unpack(xU, U, dU); unpack(xV, V, dV); unpack(xP, Ph, dPh); unpack(xp, pi, dpi);
}

int orc_filter_band(double colat) { return filter_band(colat); }

// Apply the low-latitude filters in place to every row of U, Phi, pi (scalar
// rows) and V (V rows), each row by its own latitude band.
void orc_filter(void* h, double* U, double* V, double* Ph, double* pi, double r) {
  const Grid& g = *static_cast<Grid*>(h);
  const int I = g.I, J = g.J, K = g.K;
  for (int j = 0; j < J; ++j) {
    const int band = filter_band((j + 0.5) * g.dth);
    for (int k = 0; k < K; ++k) {
      filter_row(U + ((size_t)k * J + j) * I, I, band, r);
      filter_row(Ph + ((size_t)k * J + j) * I, I, band, r);
    }
    filter_row(pi + (size_t)j * I, I, band, r);
  }
  for (int j = 0; j + 1 < J; ++j) {
    const int band = filter_band((j + 1.0) * g.dth);
    for (int k = 0; k < K; ++k) filter_row(V + ((size_t)k * (J - 1) + j) * I, I, band, r);
  }
}

// a11: out[0] mass = sum A_j (pi~ + pi) [p0 m^2]; out[1] kinetic, out[2]
// available potential, out[3] available surface potential energy (reading R4,
// all as 1/2 <x, x>_W pieces); out[4] total; out[5] max|U|; out[6] max|V|;
// out[7] 1 if every value is finite.
void orc_diagnostics(void* h, const double* U, const double* V, const double* Ph, const double* pi,
                     double* out) {
  const Grid& g = *static_cast<Grid*>(h);
  const int I = g.I, J = g.J, K = g.K, JV = J - 1;
  const Ix x{I, J, K};
  double mass = 0, ek = 0, ep = 0, eps = 0, mu = 0, mv = 0;
  bool finite = true;
  for (int j = 0; j < J; ++j)
    for (int i = 0; i < I; ++i) {
      const double p = pi[x.s2(j, i)];
      mass += g.A[j] * (g.pit[x.s2(j, i)] + p);
      eps += 0.5 * g.A[j] * (g.rts[x.s2(j, i)] / g.pit[x.s2(j, i)]) * p * p;
      finite = finite && std::isfinite(p);
    }
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < J; ++j)
      for (int i = 0; i < I; ++i) {
        const double u = U[x.s3(k, j, i)], f = Ph[x.s3(k, j, i)];
        ek += 0.5 * g.ds[k] * g.A[j] * u * u;
        ep += 0.5 * g.ds[k] * g.A[j] * f * f;
        mu = std::fmax(mu, std::fabs(u));
        finite = finite && std::isfinite(u) && std::isfinite(f);
      }
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < JV; ++j)
      for (int i = 0; i < I; ++i) {
        const double v = V[x.v3(k, j, i)];
        ek += 0.5 * g.ds[k] * g.Av[j] * v * v;
        mv = std::fmax(mv, std::fabs(v));
        finite = finite && std::isfinite(v);
      }
  out[0] = mass; out[1] = ek; out[2] = ep; out[3] = eps; out[4] = ek + ep + eps;
  out[5] = mu; out[6] = mv; out[7] = finite ? 1.0 : 0.0;
}

}  // extern "C"
