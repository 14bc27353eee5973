// Branching (reconfiguration) kernels, Sec. II.A of the paper.
//
//  branch_reduce_body per-interval sums in a fixed order (deterministic):
//                    sum w, sum w e_L, sum f, sum f e_L with f = w/(W - E_0),
//                    max w, OR of status bits, hop statistics
//  k_reconfigure     integer comb: q_b = floor(w_b / w_max 2^S), exact uint64
//                    prefix sum, and for every slot alpha the first b with
//                    (xi32 + alpha 2^32) Q_total < N 2^32 Q_b (128-bit test)
//  slot_body         where each copy is stored (selected walkers keep their slots)
//  k_gather_slots    in place: unselected slots receive a copy of their source, w = 1
//
// A single system's branching spreads the per-walker FP64 work over the grid
// (k_branch_partials, k_branch_combine, k_quantise) and keeps the integer scan,
// comb and slot assignment in one CTA (k_reconfigure_q); the one-CTA bodies
// serve the batched path (one CTA per system) and the comb entry points.  The
// gather moves the walker blocks and is HBM-bound.
#pragma once

#include "common.cuh"

namespace lrdmc {

constexpr int BR_THREADS = 1024;

enum BranchStat : int {
  BS_SUMW = 0, BS_SUMWE = 1, BS_SUMF = 2, BS_SUMFE = 3, BS_WMAX = 4, BS_STATUS = 5,
  BS_MOVES = 6, BS_MOVESMAX = 7, BS_BAD = 8, BS_SURV = 9, BS_COUNT = 16
};

// One CTA of BR_THREADS threads.  Each thread accumulates a strided subset in
// index order; the partials are combined by a fixed tree: xor-shuffles within
// each warp, then the warps' results by the first warp.
__device__ void branch_reduce_body(const Layout& L, const double* __restrict__ state, int n_w, double E0, int lb,
                                   double* __restrict__ out) {
  constexpr int NW = BR_THREADS / 32;
  __shared__ double s_part[6][NW];
  __shared__ unsigned s_or[NW];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // w, w e, f, f e, moves, max moves
  unsigned orv = 0u;
  for (int a = t; a < n_w; a += BR_THREADS) {
    const double* sc = state + (size_t)a * L.g_stride + L.g_sc;
    const double w = sc[SC_W], e = sc[SC_EL];
    acc[0] += w;
    if (w != 0.0) {
      // a walker of zero weight is no longer part of the population: it adds
      // nothing to the averages, also when its e_L or W is not finite (the
      // load-balanced step sets w = 0 where W - E_0 <= 0 or W is NaN)
      acc[1] += w * e;
      const double f = lb ? w / (sc[SC_WDIAG] - E0) : w;
      acc[2] += f;
      acc[3] += f * e;
    }
    acc[4] += sc[SC_MOVES];
    acc[5] = fmax(acc[5], sc[SC_MOVES]);
    orv |= (unsigned)sc[SC_STATUS];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += __shfl_xor_sync(FULL, acc[k], o);
    acc[5] = fmax(acc[5], __shfl_xor_sync(FULL, acc[5], o));
    orv |= __shfl_xor_sync(FULL, orv, o);
  }
  if (lane == 0) {
    for (int k = 0; k < 6; ++k) s_part[k][wid] = acc[k];
    s_or[wid] = orv;
  }
  __syncthreads();
  if (wid == 0) {
    double r[6];
    for (int k = 0; k < 6; ++k) r[k] = lane < NW ? s_part[k][lane] : 0.0;
    unsigned ro = lane < NW ? s_or[lane] : 0u;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 5; ++k) r[k] += __shfl_xor_sync(FULL, r[k], o);
      r[5] = fmax(r[5], __shfl_xor_sync(FULL, r[5], o));
      ro |= __shfl_xor_sync(FULL, ro, o);
    }
    if (lane == 0) {
      out[BS_SUMW] = r[0];
      out[BS_SUMWE] = r[1];
      out[BS_SUMF] = r[2];
      out[BS_SUMFE] = r[3];
      out[BS_MOVES] = r[4];
      out[BS_MOVESMAX] = r[5];
      out[BS_STATUS] = (double)ro;
    }
  }
}

// Comb over the inclusive prefix sums Q of the quantised weights (total tot):
// src[alpha] = the first b with (xi32 + alpha 2^32) tot < n 2^32 Q_b, for
// the slots [lo, hi) of this thread; then the number of distinct survivors
// and the status words.
__device__ void comb_body(int n, uint32_t xi32, const unsigned long long* __restrict__ Q, unsigned long long tot,
                          int lo, int hi, int32_t* __restrict__ src, int32_t* __restrict__ status,
                          double* __restrict__ stats_out, double wmax) {
  __shared__ int s_cnt[BR_THREADS];
  const int t = threadIdx.x;
  // (3) comb: first b with (xi32 + alpha 2^32) tot < n 2^32 Q_b.  Thread t
  // takes the contiguous slots [lo, hi): a binary search for the first, then,
  // since the answer does not decrease with alpha, a forward walk for the rest.
  const unsigned __int128 n32 = (unsigned __int128)(unsigned)n << 32;
  {
    int b = 0;
    for (int al = lo; al < hi; ++al) {
      const unsigned __int128 lhs = ((unsigned __int128)xi32 + ((unsigned __int128)(unsigned)al << 32)) *
                                    (unsigned __int128)tot;
      if (al == lo) {
        int b0 = 0, b1 = n - 1;   // condition holds at b = n - 1
        while (b0 < b1) {
          const int mid = (b0 + b1) >> 1;
          if (lhs < n32 * (unsigned __int128)Q[mid]) b1 = mid; else b0 = mid + 1;
        }
        b = b0;
      } else {
        while (b < n - 1 && !(lhs < n32 * (unsigned __int128)Q[b])) ++b;
      }
      src[al] = b;
    }
  }
  __syncthreads();
  // (4) distinct survivors (src is non-decreasing)
  int cnt = 0;
  for (int al = t; al < n; al += BR_THREADS) cnt += (al == 0 || src[al] != src[al - 1]) ? 1 : 0;
  s_cnt[t] = cnt;
  __syncthreads();
  for (int s = BR_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) s_cnt[t] += s_cnt[t + s];
    __syncthreads();
  }
  if (t == 0) {
    if (status) { status[0] = 0; status[1] = s_cnt[0]; }
    if (stats_out) { stats_out[BS_BAD] = 0.0; stats_out[BS_WMAX] = wmax; stats_out[BS_SURV] = s_cnt[0]; }
  }
}

// Integer comb.  Weights are read as w[a * w_stride]; Q is uint64 scratch of
// n entries.  status[0] = 0 ok / 1 invalid weights; status[1] = survivors.
__device__ void reconfigure_body(const double* __restrict__ w, int w_stride, int n, uint32_t xi32,
                                 unsigned long long* __restrict__ Q, int32_t* __restrict__ src,
                                 int32_t* __restrict__ status, double* __restrict__ stats_out) {
  __shared__ double s_max[BR_THREADS];
  __shared__ int s_bad[BR_THREADS];
  __shared__ unsigned long long s_sum[BR_THREADS];
  const int t = threadIdx.x;
  // (1) max weight and validity
  double m = 0.0;
  int bad = 0;
  for (int a = t; a < n; a += BR_THREADS) {
    const double v = w[(size_t)a * w_stride];
    if (!isfinite(v) || v < 0.0) bad = 1;
    m = fmax(m, v);
  }
  s_max[t] = m;
  s_bad[t] = bad;
  __syncthreads();
  for (int s = BR_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) {
      s_max[t] = fmax(s_max[t], s_max[t + s]);
      s_bad[t] |= s_bad[t + s];
    }
    __syncthreads();
  }
  const double wmax = s_max[0];
  if (s_bad[0] || !(wmax > 0.0)) {
    if (t == 0 && status) { status[0] = 1; status[1] = 0; }
    if (t == 0 && stats_out) { stats_out[BS_BAD] = 1.0; stats_out[BS_WMAX] = wmax; }
    return;
  }
  // (2) quantise and scan: thread t owns the contiguous chunk [lo, hi)
  int nbits = 0;
  for (int v = n; v; v >>= 1) ++nbits;
  const double scale = ldexp(1.0, 62 - nbits);
  const int chunk = (n + BR_THREADS - 1) / BR_THREADS;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  unsigned long long loc = 0ull;
  for (int a = lo; a < hi; ++a) loc += (unsigned long long)floor((w[(size_t)a * w_stride] / wmax) * scale);
  s_sum[t] = loc;
  __syncthreads();
  // inclusive Hillis-Steele scan of the chunk totals (integers: order-free)
  for (int off = 1; off < BR_THREADS; off <<= 1) {
    const unsigned long long v = t >= off ? s_sum[t - off] : 0ull;
    __syncthreads();
    s_sum[t] += v;
    __syncthreads();
  }
  unsigned long long run = t ? s_sum[t - 1] : 0ull;
  for (int a = lo; a < hi; ++a) {
    run += (unsigned long long)floor((w[(size_t)a * w_stride] / wmax) * scale);
    Q[a] = run;
  }
  __syncthreads();
  const unsigned long long tot = s_sum[BR_THREADS - 1];
  comb_body(n, xi32, Q, tot, lo, hi, src, status, stats_out, wmax);
}

// Exclusive prefix count over the block of the flags f(i), i in [0, n), in
// contiguous per-thread chunks: returns this thread's chunk [lo, hi) and the
// number of flagged items before lo; s_cnt is BR_THREADS ints of scratch.
template <typename F>
__device__ __forceinline__ int chunk_offset(int n, F f, int* s_cnt, int& lo, int& hi) {
  const int t = threadIdx.x, chunk = (n + BR_THREADS - 1) / BR_THREADS;
  lo = min(n, t * chunk);
  hi = min(n, lo + chunk);
  int c = 0;
  for (int i = lo; i < hi; ++i) c += f(i) ? 1 : 0;
  s_cnt[t] = c;
  __syncthreads();
  for (int off = 1; off < BR_THREADS; off <<= 1) {
    const int v = t >= off ? s_cnt[t - off] : 0;
    __syncthreads();
    s_cnt[t] += v;
    __syncthreads();
  }
  const int before = s_cnt[t] - c;
  __syncthreads();
  return before;
}

// Where the copies of the comb are stored: src (comb order, non-decreasing)
// becomes slot -> source walker.  A selected walker keeps its own slot for its
// first copy; its further copies, in comb order, fill the slots of the walkers
// that were not selected, in increasing slot order.  So only those slots need
// a copy.  scratch holds 2 n ints.  Nothing happens when status[0] != 0.
__device__ void slot_body(int n, int32_t* __restrict__ src, int32_t* __restrict__ scratch,
                          const int32_t* __restrict__ status) {
  __shared__ int s_cnt[BR_THREADS];
  if (status && status[0] != 0) return;
  int32_t* A = scratch;        // selected flags, then slot -> source
  int32_t* X = scratch + n;    // further copies' sources, in comb order
  const int t = threadIdx.x;
  for (int k = t; k < n; k += BR_THREADS) A[k] = 0;
  __syncthreads();
  for (int al = t; al < n; al += BR_THREADS) A[CHK(src[al], n)] = 1;
  __syncthreads();
  // further copies in comb order
  int lo, hi;
  int r = chunk_offset(n, [&](int al) { return al > 0 && src[al] == src[al - 1]; }, s_cnt, lo, hi);
  for (int al = lo; al < hi; ++al)
    if (al > 0 && src[al] == src[al - 1]) X[r++] = src[al];
  __syncthreads();
  // unselected slots in increasing order, listed in src (no longer needed)
  r = chunk_offset(n, [&](int k) { return A[k] == 0; }, s_cnt, lo, hi);
  for (int k = lo; k < hi; ++k)
    if (A[k] == 0) src[r++] = k;
  const int n_free = s_cnt[BR_THREADS - 1];
  __syncthreads();
  for (int k = t; k < n; k += BR_THREADS) A[k] = A[k] ? k : -1;
  __syncthreads();
  for (int j = t; j < n_free; j += BR_THREADS) A[CHK(src[j], n)] = X[j];
  __syncthreads();
  for (int k = t; k < n; k += BR_THREADS) src[k] = A[k];
}

// With slots set, src leaves as slot -> source walker (slot_body), else as
// the comb's indices.
__global__ void __launch_bounds__(BR_THREADS) k_reconfigure(const double* __restrict__ w, int w_stride,
                                                            int n, uint32_t xi32,
                                                            unsigned long long* __restrict__ Q,
                                                            int32_t* __restrict__ src,
                                                            int32_t* __restrict__ status,
                                                            double* __restrict__ stats_out, int slots) {
  reconfigure_body(w, w_stride, n, xi32, Q, src, status, stats_out);
  if (!slots) return;
  __syncthreads();
  slot_body(n, src, reinterpret_cast<int32_t*>(Q), status);
}

// ------------------------------------------------------------ grid-wide passes
// A single system's branching at large N_w: the per-walker FP64 work (the
// load-balanced weight w / (W - E_0) in the sums, w_b / w_max in the
// quantisation) exceeds what one SM's FP64 pipe does in a few microseconds,
// so it is spread over the grid and the one-CTA kernel keeps only integer work:
//  k_branch_partials  CTA c reduces the contiguous walkers [c C, (c + 1) C)
//                     in a fixed order (same quantities as branch_reduce_body,
//                     plus max w and the invalid-weight flag)
//  k_branch_combine   one warp adds the CTA partials in index order
//  k_quantise         q_b = floor(w_b / w_max 2^S) for every walker, into Q
//  k_reconfigure_q    prefix sums of q, comb, survivors, slot assignment
// q_b, its prefix sums and the comb are the integers reconfigure_body forms
// (max and integer sums do not depend on order, q_b is the same expression);
// the FP64 sums are deterministic, in their own fixed order.
constexpr int BP_THREADS = 256;
constexpr int BP_MAX_CTAS = 1024;
constexpr int BP_STRIDE = 16;   // doubles per CTA partial
enum BranchPart : int {
  BP_SUMW = 0, BP_SUMWE = 1, BP_SUMF = 2, BP_SUMFE = 3, BP_MOVES = 4, BP_MOVESMAX = 5, BP_STATUS = 6,
  BP_WMAX = 7, BP_BAD = 8
};

__host__ __device__ inline int branch_part_ctas(int n) {
  const int c = (n + BP_THREADS - 1) / BP_THREADS;
  return c < 1 ? 1 : (c > BP_MAX_CTAS ? BP_MAX_CTAS : c);
}

__global__ void __launch_bounds__(BP_THREADS) k_branch_partials(Layout L, const double* __restrict__ state,
                                                                int n_w, double E0, int lb,
                                                                double* __restrict__ part) {
  constexpr int NW = BP_THREADS / 32;
  __shared__ double s_part[8][NW];
  __shared__ unsigned s_or[NW], s_bad[NW];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int C = (n_w + gridDim.x - 1) / gridDim.x;
  const int lo = min(n_w, (int)blockIdx.x * C), hi = min(n_w, lo + C);
  // w, w e, f, f e, moves, max moves, (unused), max w
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  unsigned orv = 0u, bad = 0u;
  for (int a = lo + t; a < hi; a += BP_THREADS) {
    const double* sc = state + (size_t)a * L.g_stride + L.g_sc;
    const double w = sc[SC_W], e = sc[SC_EL];
    acc[0] += w;
    if (w != 0.0) {
      // a walker of zero weight is no longer part of the population: it adds
      // nothing to the averages, also when its e_L or W is not finite (the
      // load-balanced step sets w = 0 where W - E_0 <= 0 or W is NaN)
      acc[1] += w * e;
      const double f = lb ? w / (sc[SC_WDIAG] - E0) : w;
      acc[2] += f;
      acc[3] += f * e;
    }
    acc[4] += sc[SC_MOVES];
    acc[5] = fmax(acc[5], sc[SC_MOVES]);
    orv |= (unsigned)sc[SC_STATUS];
    if (!isfinite(w) || w < 0.0) bad = 1u;
    acc[7] = fmax(acc[7], w);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += __shfl_xor_sync(FULL, acc[k], o);
    acc[5] = fmax(acc[5], __shfl_xor_sync(FULL, acc[5], o));
    acc[7] = fmax(acc[7], __shfl_xor_sync(FULL, acc[7], o));
    orv |= __shfl_xor_sync(FULL, orv, o);
    bad |= __shfl_xor_sync(FULL, bad, o);
  }
  if (lane == 0) {
    for (int k = 0; k < 8; ++k) s_part[k][wid] = acc[k];
    s_or[wid] = orv;
    s_bad[wid] = bad;
  }
  __syncthreads();
  if (t == 0) {
    double r[8];
    unsigned ro = 0u, rb = 0u;
    for (int k = 0; k < 8; ++k) r[k] = s_part[k][0];
    for (int v = 1; v < NW; ++v) {
      for (int k = 0; k < 5; ++k) r[k] += s_part[k][v];
      r[5] = fmax(r[5], s_part[5][v]);
      r[7] = fmax(r[7], s_part[7][v]);
    }
    for (int v = 0; v < NW; ++v) { ro |= s_or[v]; rb |= s_bad[v]; }
    double* out = part + (size_t)blockIdx.x * BP_STRIDE;
    for (int k = 0; k < 6; ++k) out[k] = r[k];
    out[BP_STATUS] = (double)ro;
    out[BP_WMAX] = r[7];
    out[BP_BAD] = (double)rb;
  }
}

// One warp: the n_part CTA partials, lane l taking l, l + 32, ... in order,
// then a fixed xor tree.  Writes the branching statistics, w_max and the
// invalid-weight flag (negative or non-finite weights, or all zero).
__global__ void __launch_bounds__(32) k_branch_combine(const double* __restrict__ part, int n_part,
                                                       double* __restrict__ out) {
  const int lane = threadIdx.x;
  double r[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double wm = 0.0;
  unsigned ro = 0u, rb = 0u;
  for (int c = lane; c < n_part; c += 32) {
    const double* p = part + (size_t)c * BP_STRIDE;
    for (int k = 0; k < 5; ++k) r[k] += p[k];
    r[5] = fmax(r[5], p[BP_MOVESMAX]);
    wm = fmax(wm, p[BP_WMAX]);
    ro |= (unsigned)p[BP_STATUS];
    rb |= p[BP_BAD] != 0.0 ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) r[k] += __shfl_xor_sync(FULL, r[k], o);
    r[5] = fmax(r[5], __shfl_xor_sync(FULL, r[5], o));
    wm = fmax(wm, __shfl_xor_sync(FULL, wm, o));
    ro |= __shfl_xor_sync(FULL, ro, o);
    rb |= __shfl_xor_sync(FULL, rb, o);
  }
  if (lane == 0) {
    out[BS_SUMW] = r[0];
    out[BS_SUMWE] = r[1];
    out[BS_SUMF] = r[2];
    out[BS_SUMFE] = r[3];
    out[BS_MOVES] = r[4];
    out[BS_MOVESMAX] = r[5];
    out[BS_STATUS] = (double)ro;
    out[BS_WMAX] = wm;
    out[BS_BAD] = (rb || !(wm > 0.0)) ? 1.0 : 0.0;
  }
}

// Q[b] = floor(w_b / w_max 2^S), S = 62 - bitlength(n); nothing when the
// weights are invalid.
__global__ void __launch_bounds__(BP_THREADS) k_quantise(const double* __restrict__ w, int w_stride, int n,
                                                         const double* __restrict__ stats,
                                                         unsigned long long* __restrict__ Q) {
  if (stats[BS_BAD] != 0.0) return;
  const double wmax = stats[BS_WMAX];
  int nbits = 0;
  for (int v = n; v; v >>= 1) ++nbits;
  const double scale = ldexp(1.0, 62 - nbits);
  for (int a = blockIdx.x * BP_THREADS + threadIdx.x; a < n; a += gridDim.x * BP_THREADS)
    Q[a] = (unsigned long long)floor((w[(size_t)a * w_stride] / wmax) * scale);
}

// One CTA: Q holds q_b on entry and the inclusive prefix sums after the scan;
// then the comb and, as in k_reconfigure with slots set, the slot assignment.
// Q doubles as the slot assignment's scratch.
__global__ void __launch_bounds__(BR_THREADS) k_reconfigure_q(int n, uint32_t xi32,
                                                              unsigned long long* __restrict__ Q,
                                                              int32_t* __restrict__ src,
                                                              int32_t* __restrict__ status,
                                                              double* __restrict__ stats) {
  __shared__ unsigned long long s_sum[BR_THREADS];
  const int t = threadIdx.x;
  if (stats[BS_BAD] != 0.0) {
    if (t == 0) { status[0] = 1; status[1] = 0; }
    return;
  }
  const int chunk = (n + BR_THREADS - 1) / BR_THREADS;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  unsigned long long loc = 0ull;
  for (int a = lo; a < hi; ++a) loc += Q[a];
  s_sum[t] = loc;
  __syncthreads();
  for (int off = 1; off < BR_THREADS; off <<= 1) {
    const unsigned long long v = t >= off ? s_sum[t - off] : 0ull;
    __syncthreads();
    s_sum[t] += v;
    __syncthreads();
  }
  unsigned long long run = t ? s_sum[t - 1] : 0ull;
  for (int a = lo; a < hi; ++a) {
    run += Q[a];
    Q[a] = run;
  }
  __syncthreads();
  comb_body(n, xi32, Q, s_sum[BR_THREADS - 1], lo, hi, src, status, stats, stats[BS_WMAX]);
  __syncthreads();
  slot_body(n, src, reinterpret_cast<int32_t*>(Q), status);
}

// new[alpha] = old[src[alpha]], weight reset to 1; skipped when status[0] != 0.
// The walker's cache block (when the layout has one) moves with it.  Threads
// tid, tid + nth, ... of the launch take the copies.  In place (new == old,
// src a slot assignment of slot_body) only the slots with src[alpha] != alpha
// are written; they are never the source of a copy.
__device__ void gather_body(const Layout& L, const double* old_state, double* new_state,
                            const double* old_cache, double* new_cache,
                            const int32_t* __restrict__ src, int n_w, const int32_t* __restrict__ status,
                            size_t tid, size_t nth) {
  if (status[0] != 0) return;
  const bool inplace = new_state == old_state;
  const int per = L.g_stride / 2;   // double2 per walker block (stride is a multiple of 16 doubles)
  const double2* o2 = reinterpret_cast<const double2*>(old_state);
  double2* n2 = reinterpret_cast<double2*>(new_state);
  const size_t total = (size_t)n_w * per;
  for (size_t idx = tid; idx < total; idx += nth) {
    const int a = (int)(idx / per);
    const int o = (int)(idx - (size_t)a * per);
    const int sa = CHK(src[a], n_w);
    if (inplace && sa == a) continue;
    double2 v = o2[(size_t)sa * per + o];
    if (2 * o == L.g_sc + SC_W) v.x = 1.0;
    n2[idx] = v;
  }
  if (inplace)
    for (size_t a = tid; a < (size_t)n_w; a += nth)
      if (src[a] == (int)a) new_state[a * L.g_stride + L.g_sc + SC_W] = 1.0;
  if (!old_cache || L.c_stride == 0) return;
  const int cper = L.c_stride / 2;
  const double2* oc = reinterpret_cast<const double2*>(old_cache);
  double2* nc = reinterpret_cast<double2*>(new_cache);
  const size_t ctotal = (size_t)n_w * cper;
  for (size_t idx = tid; idx < ctotal; idx += nth) {
    const int a = (int)(idx / cper);
    const int sa = CHK(src[a], n_w);
    if (inplace && sa == a) continue;
    nc[idx] = oc[(size_t)sa * cper + (idx - (size_t)a * cper)];
  }
}

// In-place gather after slot_body: one CTA per slot; the slot of a selected
// walker only has its weight reset, the slot of an unselected one receives a
// copy of its source's walker and cache blocks (weight 1).  Sources are always
// selected walkers, so no source is overwritten.
__global__ void k_gather_slots(Layout L, double* state, double* cache, const int32_t* __restrict__ src,
                               const int32_t* __restrict__ status) {
  if (status[0] != 0) return;
  const int a = blockIdx.x, sa = CHK(src[a], (int)gridDim.x);   // one CTA per walker slot
  if (sa == a) {
    if (threadIdx.x == 0) state[(size_t)a * L.g_stride + L.g_sc + SC_W] = 1.0;
    return;
  }
  const int per = L.g_stride / 2;
  const double2* o2 = reinterpret_cast<const double2*>(state + (size_t)sa * L.g_stride);
  double2* n2 = reinterpret_cast<double2*>(state + (size_t)a * L.g_stride);
  for (int o = threadIdx.x; o < per; o += blockDim.x) {
    double2 v = o2[o];
    if (2 * o == L.g_sc + SC_W) v.x = 1.0;
    n2[o] = v;
  }
  if (!cache || L.c_stride == 0) return;
  const int cper = L.c_stride / 2;
  const double2* oc = reinterpret_cast<const double2*>(cache + (size_t)sa * L.c_stride);
  double2* nc = reinterpret_cast<double2*>(cache + (size_t)a * L.c_stride);
  for (int o = threadIdx.x; o < cper; o += blockDim.x) nc[o] = oc[o];
}


// ------------------------------------------------------------ batches
// One system of a batch at branching time.
struct BranchJob {
  Layout L;
  const double* state;
  double* alt;
  const double* cache;
  double* cache_alt;
  int n_w, lb;
  double E0;
  uint32_t xi32;
  unsigned long long* Q;
  int32_t* src;
  int32_t* status;   // [2] per job
  double* stats;     // [BS_COUNT] per job
};

// Block b reduces, or reconfigures, system b; the gather takes blockIdx.y as
// the system.
__global__ void __launch_bounds__(BR_THREADS) k_branch_reduce_batch(const BranchJob* __restrict__ jobs) {
  const BranchJob& J = jobs[blockIdx.x];
  branch_reduce_body(J.L, J.state, J.n_w, J.E0, J.lb, J.stats);
}

__global__ void __launch_bounds__(BR_THREADS) k_reconfigure_batch(const BranchJob* __restrict__ jobs) {
  const BranchJob& J = jobs[blockIdx.x];
  reconfigure_body(J.state + J.L.g_sc + SC_W, J.L.g_stride, J.n_w, J.xi32, J.Q, J.src, J.status, J.stats);
  __syncthreads();
  slot_body(J.n_w, J.src, reinterpret_cast<int32_t*>(J.Q), J.status);
}

__global__ void k_gather_batch(const BranchJob* __restrict__ jobs) {
  const BranchJob& J = jobs[blockIdx.y];
  gather_body(J.L, J.state, J.alt, J.cache, J.cache_alt, J.src, J.n_w, J.status,
              blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

}  // namespace lrdmc
