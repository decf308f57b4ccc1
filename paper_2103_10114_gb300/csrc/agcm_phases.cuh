// agcm_phases.cuh — phase A of the spatial operator T(x) for the adjoint's
// forward recompute:
//
//  phase A (colstate): m = pi~ + pi, P = sqrt(m) and its U/V-point values and
//                      reciprocals (2-D, one thread per column).
// Phase B (the leap divergence, the column sum C, the sigma mass flux W, the
// Omega~ factor and the hydrostatic psi) is recomputed by the adjoint's
// column kernel together with its transpose, and phase C (advection,
// pressure gradient, Coriolis) is reversed by the gather kernels; both are in
// agcm_adjoint.cuh.  The forward step computes all three phases inside its
// stage kernels (agcm_row.cuh, agcm_fused.cuh).
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

}  // namespace agcm
