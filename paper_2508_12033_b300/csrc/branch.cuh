// Branching (reconfiguration) kernels, Sec. II.A of the paper.
//
//  k_branch_reduce   per-interval sums in a fixed order (deterministic):
//                    sum w, sum w e_L, sum f, sum f e_L with f = w/(W - E_0),
//                    max w, OR of status bits, hop statistics
//  k_reconfigure     integer comb: q_b = floor(w_b / w_max 2^S), exact uint64
//                    prefix sum, and for every slot alpha the first b with
//                    (xi32 + alpha 2^32) Q_total < N 2^32 Q_b (128-bit test)
//  k_gather          new walker alpha = copy of old walker s(alpha), w = 1
//
// The reduction and the comb run in one CTA: N_w is at most a few 10^5 and the
// work is O(N_w) integer/FP64 operations, far below one microsecond per 10^4
// walkers; the gather moves the walker blocks and is HBM-bound.
#pragma once

#include "common.cuh"

namespace lrdmc {

constexpr int BR_THREADS = 1024;

enum BranchStat : int {
  BS_SUMW = 0, BS_SUMWE = 1, BS_SUMF = 2, BS_SUMFE = 3, BS_WMAX = 4, BS_STATUS = 5,
  BS_MOVES = 6, BS_MOVESMAX = 7, BS_BAD = 8, BS_SURV = 9, BS_COUNT = 16
};

// One CTA of BR_THREADS threads.  Each thread accumulates a strided subset in
// index order, then the partials are combined by a fixed tree.
__device__ void branch_reduce_body(const Layout& L, const double* __restrict__ state, int n_w, double E0, int lb,
                                   double* __restrict__ out) {
  __shared__ double s_buf[BR_THREADS];
  __shared__ unsigned s_or[BR_THREADS];
  const int t = threadIdx.x;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // w, w e, f, f e, moves, max moves
  unsigned orv = 0u;
  for (int a = t; a < n_w; a += BR_THREADS) {
    const double* sc = state + (size_t)a * L.g_stride + L.g_sc;
    const double w = sc[SC_W], e = sc[SC_EL];
    acc[0] += w;
    acc[1] += w * e;
    const double f = lb ? w / (sc[SC_WDIAG] - E0) : w;
    acc[2] += f;
    acc[3] += f * e;
    acc[4] += sc[SC_MOVES];
    acc[5] = fmax(acc[5], sc[SC_MOVES]);
    orv |= (unsigned)sc[SC_STATUS];
  }
  double res[6];
  for (int k = 0; k < 6; ++k) {
    s_buf[t] = acc[k];
    __syncthreads();
    for (int s = BR_THREADS / 2; s > 0; s >>= 1) {
      if (t < s) s_buf[t] = (k == 5) ? fmax(s_buf[t], s_buf[t + s]) : s_buf[t] + s_buf[t + s];
      __syncthreads();
    }
    res[k] = s_buf[0];
    __syncthreads();
  }
  s_or[t] = orv;
  __syncthreads();
  for (int s = BR_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) s_or[t] |= s_or[t + s];
    __syncthreads();
  }
  if (t == 0) {
    out[BS_SUMW] = res[0];
    out[BS_SUMWE] = res[1];
    out[BS_SUMF] = res[2];
    out[BS_SUMFE] = res[3];
    out[BS_MOVES] = res[4];
    out[BS_MOVESMAX] = res[5];
    out[BS_STATUS] = (double)s_or[0];
  }
}

__global__ void __launch_bounds__(BR_THREADS) k_branch_reduce(Layout L, const double* __restrict__ state,
                                                              int n_w, double E0, int lb,
                                                              double* __restrict__ out) {
  branch_reduce_body(L, state, n_w, E0, lb, out);
}

// Integer comb.  Weights are read as w[a * w_stride]; Q is uint64 scratch of
// n entries.  status[0] = 0 ok / 1 invalid weights; status[1] = survivors.
__device__ void reconfigure_body(const double* __restrict__ w, int w_stride, int n, uint32_t xi32,
                                 unsigned long long* __restrict__ Q, int32_t* __restrict__ src,
                                 int32_t* __restrict__ status, double* __restrict__ stats_out) {
  __shared__ double s_max[BR_THREADS];
  __shared__ int s_bad[BR_THREADS];
  __shared__ unsigned long long s_sum[BR_THREADS];
  __shared__ int s_cnt[BR_THREADS];
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
  // (3) comb: first b with (xi32 + alpha 2^32) tot < n 2^32 Q_b
  const unsigned __int128 n32 = (unsigned __int128)(unsigned)n << 32;
  for (int al = t; al < n; al += BR_THREADS) {
    const unsigned __int128 lhs = ((unsigned __int128)xi32 + ((unsigned __int128)(unsigned)al << 32)) *
                                  (unsigned __int128)tot;
    int b0 = 0, b1 = n - 1;   // condition holds at b = n - 1
    while (b0 < b1) {
      const int mid = (b0 + b1) >> 1;
      if (lhs < n32 * (unsigned __int128)Q[mid]) b1 = mid; else b0 = mid + 1;
    }
    src[al] = b0;
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

__global__ void __launch_bounds__(BR_THREADS) k_reconfigure(const double* __restrict__ w, int w_stride,
                                                            int n, uint32_t xi32,
                                                            unsigned long long* __restrict__ Q,
                                                            int32_t* __restrict__ src,
                                                            int32_t* __restrict__ status,
                                                            double* __restrict__ stats_out) {
  reconfigure_body(w, w_stride, n, xi32, Q, src, status, stats_out);
}

// new[alpha] = old[src[alpha]], weight reset to 1; skipped when status[0] != 0.
// The walker's cache block (when the layout has one) moves with it.  Threads
// tid, tid + nth, ... of the launch take the copies.
__device__ void gather_body(const Layout& L, const double* __restrict__ old_state, double* __restrict__ new_state,
                            const double* __restrict__ old_cache, double* __restrict__ new_cache,
                            const int32_t* __restrict__ src, int n_w, const int32_t* __restrict__ status,
                            size_t tid, size_t nth) {
  if (status[0] != 0) return;
  const int per = L.g_stride / 2;   // double2 per walker block (stride is a multiple of 16 doubles)
  const double2* o2 = reinterpret_cast<const double2*>(old_state);
  double2* n2 = reinterpret_cast<double2*>(new_state);
  const size_t total = (size_t)n_w * per;
  for (size_t idx = tid; idx < total; idx += nth) {
    const int a = (int)(idx / per);
    const int o = (int)(idx - (size_t)a * per);
    double2 v = o2[(size_t)src[a] * per + o];
    if (2 * o == L.g_sc + SC_W) v.x = 1.0;
    n2[idx] = v;
  }
  if (!old_cache || L.c_stride == 0) return;
  const int cper = L.c_stride / 2;
  const double2* oc = reinterpret_cast<const double2*>(old_cache);
  double2* nc = reinterpret_cast<double2*>(new_cache);
  const size_t ctotal = (size_t)n_w * cper;
  for (size_t idx = tid; idx < ctotal; idx += nth) {
    const int a = (int)(idx / cper);
    nc[idx] = oc[(size_t)src[a] * cper + (idx - (size_t)a * cper)];
  }
}

__global__ void k_gather(Layout L, const double* __restrict__ old_state, double* __restrict__ new_state,
                         const double* __restrict__ old_cache, double* __restrict__ new_cache,
                         const int32_t* __restrict__ src, int n_w, const int32_t* __restrict__ status) {
  gather_body(L, old_state, new_state, old_cache, new_cache, src, n_w, status,
              blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
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
}

__global__ void k_gather_batch(const BranchJob* __restrict__ jobs) {
  const BranchJob& J = jobs[blockIdx.y];
  gather_body(J.L, J.state, J.alt, J.cache, J.cache_alt, J.src, J.n_w, J.status,
              blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

}  // namespace lrdmc
