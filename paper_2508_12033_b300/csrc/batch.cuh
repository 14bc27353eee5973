// Batched propagation of several systems in one persistent launch.
//
// Every system of a batch keeps its own handle (system tables, walker and cache
// blocks, branching buffers).  One launch propagates the walkers of all systems
// with one persistent CTA per resident slot: a CTA repeatedly takes the next
// item (system k, walkers [w0, w0 + count)) from a global counter, copies system
// k's descriptor into its shared memory, partitions the rest of its shared
// memory into count regions of system k's per-walker size and runs one walker
// per warp with the same per-walker interval as the single-system kernels.
// Small systems therefore run many warps per SM, inside the same launch; count
// is chosen by the host as the number of system-k regions that fit in the
// CTA's shared memory.  A system of which fewer than a few walkers would fit
// (its O(N^2) caches already in global memory) instead keeps every walker's
// working set in global memory (gsm_buf, gsm_stride doubles per warp of the
// grid) and runs one walker on each of the CTA's warps.  The item order is chosen by the host
// (systems in order, or the most expensive systems first so that the longest
// items start early and the queue drains evenly).
#pragma once

#include "walker.cuh"
#include "walker_mixed.cuh"

namespace lrdmc {

// One system of a batched propagation (a whole number of 16-byte words, so
// that a CTA copies it as doubles into 16-byte aligned shared memory).
struct alignas(16) PropJob {
  DevSys S;
  Layout L;
  LayoutM M;
  StepParams P;
  double* state;
  double* cache;
  int n_w;
  int region;   // shared doubles per walker (even)
  int gsm;      // 1: the walkers' working sets live in global memory (system too large to share a CTA)
};
constexpr int JOB_WORDS = (int)(sizeof(PropJob) / sizeof(double));
static_assert(sizeof(PropJob) % 16 == 0, "PropJob must be a whole number of 16-byte words");

// PREC 0: FP64 kernels, 1: mixed.  items[k] = (system, first walker, count,
// unused), count <= warps per CTA; counter is zeroed before the launch;
// scratch_per_warp = global scratch doubles per warp of the grid.
template <int PREC>
__global__ void k_propagate_batch(const PropJob* __restrict__ jobs, const int4* __restrict__ items, int n_items,
                                  unsigned* __restrict__ counter, double* __restrict__ scratch,
                                  size_t scratch_per_warp, double* gsm_buf, size_t gsm_stride) {
  extern __shared__ double smem[];
  __shared__ int s_item;
  // the exponential table is the same constant table in every system image
  const double* T = stage_table(jobs[0].S, smem);
  PropJob* J = reinterpret_cast<PropJob*>(smem + EXP_TAB);
  double* regions = smem + EXP_TAB + JOB_WORDS;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* wscr = scratch + ((size_t)blockIdx.x * (blockDim.x >> 5) + wib) * scratch_per_warp;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int idx = s_item;
    if (idx >= n_items) break;
    const int4 it = items[idx];
    const double* src = reinterpret_cast<const double*>(jobs + it.x);
    for (int o = threadIdx.x; o < JOB_WORDS; o += blockDim.x) reinterpret_cast<double*>(J)[o] = src[o];
    __syncthreads();
    if (wib < it.z) {
      const int w = it.y + wib;
      if (J->gsm) {
        double* sm = gsm_buf + ((size_t)blockIdx.x * (blockDim.x >> 5) + wib) * gsm_stride;
        if (PREC == 0) {
          const Scr ws = warp_scratch_at(J->L, J->S.n_nuc, wscr);
          propagate_walker_impl<false, true>(J->S, J->L, J->state, J->cache, w, J->P, T, sm, ws, lane);
        } else {
          const ScrM ws = warp_scratch_m_at(J->L, J->M, wscr);
          propagate_walker_m(J->S, J->L, J->M, J->state, J->cache, w, J->P, T, reinterpret_cast<float*>(sm), ws,
                             lane);
        }
      } else {
        double* sm = regions + (size_t)wib * J->region;
        if (PREC == 0) {
          const Scr ws = warp_scratch_at(J->L, J->S.n_nuc, wscr);
          propagate_walker<false>(J->S, J->L, J->state, J->cache, w, J->P, T, sm, ws, lane);
        } else {
          const ScrM ws = warp_scratch_m_at(J->L, J->M, wscr);
          propagate_walker_m(J->S, J->L, J->M, J->state, J->cache, w, J->P, T, reinterpret_cast<float*>(sm), ws,
                             lane);
        }
      }
    }
    __syncthreads();   // the descriptor and s_item are rewritten for the next item
  }
}

}  // namespace lrdmc
