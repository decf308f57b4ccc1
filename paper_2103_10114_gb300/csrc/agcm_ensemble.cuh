// agcm_ensemble.cuh — many members of uneven resolution in one persistent launch.
//
// Each member is a state on its own grid.  A work item is a row tile of one
// member: 32 columns of `rows` consecutive rows (the warp takes the rows one
// after the other, so a row's stencil rows are still in L1 for the next); each
// warp pulls items from a per-(step, stage)
// device counter and runs the same column body as the single-state stage
// kernel (fused_column), so a member advanced in an ensemble does the same
// arithmetic as alone; the two kernels are compiled separately, so the
// compiler may contract multiply-adds differently (results agree to about
// one FP32 / FP64 rounding, not to the bit).  Stages are separated by a grid-wide barrier whose
// wait is bounded in time: if it runs out, the kernel records AGCM_ETIMEOUT in
// the status word and every block returns; nothing spins forever and nothing
// traps.  The launch is sized so that every block is resident at once.
#pragma once
#include "agcm_common.cuh"
#include "agcm_fused.cuh"
#include "agcm_row.cuh"

namespace agcm {

template <class T>
struct EnsMember {
  Geom<T> g;
  T* x[3][4];         // x_n, x_1, x_2: U, V, Phi, pi
  double* ubar[3];    // FP64 vertical means of x[c]
  double* vbar[3];
  T dt;
  int nbx;            // 32-column blocks per row
  int item_begin;     // first global item of this member (nbx * ceil(J / rows) items)
};

struct EnsSync {
  unsigned int count;       // barrier arrivals
  unsigned int gen;         // barrier generation
  int status;               // 0 or AGCM_ETIMEOUT (4)
  int pad;
  unsigned int queue[1];    // nsteps*3 item counters (flexible)
};

// Grid barrier with a bounded wait.  `expected` blocks must arrive; the wait
// gives up after `limit` clock cycles and records the timeout.
__device__ __forceinline__ bool ens_barrier(EnsSync* sy, unsigned expected, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &sy->gen;
    volatile int* vst = &sy->status;
    const unsigned int g0 = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&sy->count, 1u) + 1u;
    if (arrived == expected) {
      sy->count = 0u;
      __threadfence();
      atomicAdd(&sy->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g0 && *vst == 0) {
        if (clock64() - t0 > limit) {
          atomicExch(&sy->status, 4);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&sy->status) == 0;
}

template <class T>
__device__ __forceinline__ int ens_member_of(const EnsMember<T>* mem, int nmem, int item) {
  int lo = 0, hi = nmem - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mem[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One warp per block (the stage kernel's shape); the register cap of 12
// resident blocks per SM (168 registers) measured fastest for the 64-member
// mix on GB300 (20 -> 18.1 ms/step, 16 -> 14.4, 12 -> 12.6); the autotuner
// varies the number of resident blocks per SM.
#ifndef AGCM_ENS_MINB
#define AGCM_ENS_MINB 12
#endif
// ROWS: the row tile of a work item (a compile-time count, so that the
// one-row kernel carries no row loop).
template <class T, int ROWS>
__global__ void __launch_bounds__(32, sizeof(T) == 4 ? AGCM_ENS_MINB : 8)
    k_ensemble(const EnsMember<T>* __restrict__ mem, int nmem, int nitems, int nsteps, EnsSync* sy,
               unsigned expected_blocks, long long limit) {
  const int lane = threadIdx.x & 31;
  // the current member's descriptor, copied to shared memory per work item so
  // that its pointers are re-read cheaply instead of held in registers
  __shared__ __align__(16) unsigned long long sdesc[(sizeof(EnsMember<T>) + 7) / 8];
  const EnsMember<T>& e = *reinterpret_cast<const EnsMember<T>*>(sdesc);
  int cur = -1;
  for (int step = 0; step < nsteps; ++step) {
    for (int stage = 0; stage < 3; ++stage) {
      unsigned int* q = &sy->queue[step * 3 + stage];
      while (true) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(q, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        const int m = ens_member_of(mem, nmem, item);
        if (m != cur) {
          __syncwarp();
          const unsigned long long* src = reinterpret_cast<const unsigned long long*>(mem + m);
          for (int w = lane; w < (int)((sizeof(EnsMember<T>) + 7) / 8); w += 32) sdesc[w] = src[w];
          __syncwarp();
          cur = m;
        }
        const int local = item - e.item_begin;
        const int jt = local / e.nbx;
        const int i = (local - jt * e.nbx) * 32 + lane;
#pragma unroll 1
        for (int r = 0; r < ROWS; ++r) {
          const int j = jt * ROWS + r;
          if (j >= e.g.J) break;  // warp-uniform
          if (i < e.g.I) {
            const Geom<T>& g = e.g;
            // stage 1: x_n -> x1 (dt/2); stage 2: x1 -> x2 (dt/2); stage 3: x2 -> x_n
            // in place (dt); the base is x_n in all three (stage 1 reads it
            // as base instead of reusing its own values: the same arithmetic)
            const int a = stage, b = stage == 0 ? 1 : (stage == 1 ? 2 : 0);
            const T c = stage == 2 ? e.dt : T(0.5) * e.dt;
            fused_column<T, 2>(g, i, j, e.x[a][0], e.x[a][1], e.x[a][2], e.x[a][3], e.ubar[a], e.vbar[a],
                                      e.x[0][0], e.x[0][1], e.x[0][2], e.x[0][3], e.x[b][0], e.x[b][1],
                                      e.x[b][2], e.x[b][3], e.ubar[b], e.vbar[b], e.ubar[0], e.vbar[0], c);
          }
        }
      }
      __threadfence();
      if (!ens_barrier(sy, expected_blocks, limit)) return;
    }
  }
}

// The column body for the few rows the row-segment body leaves, out of line
// so that its registers do not burden the row-segment body.
template <class T>
__device__ __noinline__ void ens_column_item(const EnsMember<T>& e, int i, int j, int a, int b, T c) {
  fused_column<T, 2>(e.g, i, j, e.x[a][0], e.x[a][1], e.x[a][2], e.x[a][3], e.ubar[a], e.vbar[a], e.x[0][0],
                     e.x[0][1], e.x[0][2], e.x[0][3], e.x[b][0], e.x[b][1], e.x[b][2], e.x[b][3], e.ubar[b],
                     e.vbar[b], e.ubar[0], e.vbar[0], c);
}

// The row-segment form of the persistent launch: CTAs of kRowB threads (the
// single-state row-segment kernel's shape, AGCM_ROW_MINB resident per SM)
// pull work items of every member from the stage's queue:
//   kind 0: (member, row j, segment) — the row-segment body, stride class 0
//           (any strides), with the member's tables from its descriptor;
//   kind 1: (member, row j, 256-column chunk) — rows the row-segment body
//           leaves (strides above 63, rows not 16-byte aligned): each warp runs
//           the column body on 32 columns of the chunk.
// Items are int2 {member | kind << 16, j << 8 | segment-or-chunk}.  Every
// stage uses x_n as its base (stage 1 reads it as input and base), the three
// stages of a step as in agcm_step; a bounded grid barrier separates them.
template <class T>
__global__ void __launch_bounds__(kRowB, sizeof(T) == 4 ? AGCM_ROW_MINB : 2)
    k_ensemble_rows(const EnsMember<T>* __restrict__ mem, const int2* __restrict__ items, int nitems, int nsteps,
                    EnsSync* sy, unsigned expected_blocks, long long limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  // the current member's descriptor, copied to shared memory when it changes
  __shared__ __align__(16) unsigned long long sdesc[(sizeof(EnsMember<T>) + 7) / 8];
  __shared__ int s_item;
  // the stage's arguments for the row-segment body, kept in shared memory so
  // that the body reads its pointers from there rather than holding them
  __shared__ __align__(16) unsigned long long sargs[(sizeof(RowArgs<T>) + 7) / 8];
  RowArgs<T>& ra = *reinterpret_cast<RowArgs<T>*>(sargs);
  const EnsMember<T>& e = *reinterpret_cast<const EnsMember<T>*>(sdesc);
  const int t = threadIdx.x;
  int cur = -1;
  bool fresh = true;  // the row-segment body's mbarriers are not initialised yet
  for (int step = 0; step < nsteps; ++step) {
    for (int stage = 0; stage < 3; ++stage) {
      unsigned int* q = &sy->queue[step * 3 + stage];
      while (true) {
        __syncthreads();  // every thread is past the previous item
        if (t == 0) s_item = (int)atomicAdd(q, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 w = items[it];
        const int m = w.x & 0xffff, kind = w.x >> 16;
        // stage 1: x_n -> x1 (dt/2); stage 2: x1 -> x2 (dt/2); stage 3: x2 -> x_n (dt)
        const int a = stage, b = stage == 0 ? 1 : (stage == 1 ? 2 : 0);
        if (m != cur) {
          const unsigned long long* src = reinterpret_cast<const unsigned long long*>(mem + m);
          for (int q2 = t; q2 < (int)((sizeof(EnsMember<T>) + 7) / 8); q2 += blockDim.x) sdesc[q2] = src[q2];
          __syncthreads();
          if (t == 0)
            ra = RowArgs<T>{e.x[a][0], e.x[a][1], e.x[a][2], e.x[a][3], e.ubar[a], e.vbar[a],
                            e.x[0][0], e.x[0][1], e.x[0][2], e.x[0][3], e.x[b][0], e.x[b][1], e.x[b][2], e.x[b][3],
                            e.ubar[b], e.vbar[b], e.ubar[0], e.vbar[0],
                            stage == 2 ? e.dt : T(0.5) * e.dt, nullptr, &sy->status};
          __syncthreads();
          cur = m;
        }
        const T c = stage == 2 ? e.dt : T(0.5) * e.dt;
        if (kind == 0) {
          row_segment<T, 2, 3, false, 0>(e.g, ra, w.y >> 8, w.y & 255, smem, fresh);
          fresh = false;
        } else {
          const int i = (w.y & 255) * kRowB + t;
          if (i < e.g.I) ens_column_item<T>(e, i, w.y >> 8, a, b, c);
        }
      }
      cur = -1;  // the next stage rebuilds the member's arguments
      __threadfence();
      if (!ens_barrier(sy, expected_blocks, limit)) return;
    }
  }
}

}  // namespace agcm
