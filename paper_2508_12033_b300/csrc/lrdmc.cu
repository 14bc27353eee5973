// Host side of the LRDMC library: handle, workspace layout, launches and the
// branching-history energy estimator.  See include/lrdmc.h for the ABI.
#include "lrdmc.h"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "batch.cuh"
#include "branch.cuh"
#include "common.cuh"
#include "walker.cuh"
#include "walker_mixed.cuh"

using namespace lrdmc;

namespace {

constexpr size_t ALIGN = 256;
constexpr int MAX_WALKERS = 1 << 24;
// Upper bound of resident warps that get per-warp scratch (148 SMs x 32 warps);
// the launch grid is clamped to it.
constexpr int SCRATCH_WARPS_CAP = 148 * 32;
// Status words (int32) of a handle: [0, 2) reconfiguration status, DSTAT_NEXT
// the propagate kernels' work counter.
constexpr int DSTAT_NEXT = 8;
// status word DSTAT_DRIFT: drift-triggered re-inversions since creation
constexpr int DSTAT_DRIFT = 9;
// Default tolerance of the Sherman-Morrison drift check (lrdmc_set_drift_tol):
// an inverse residual delta perturbs the hop ratios of the spin block by
// about delta relative, so 1e-11 keeps them an order of magnitude inside the
// 1e-10 relative agreement the FP64 path is held to.
constexpr double DRIFT_TOL_DEFAULT = 1e-11;
// The gradient kernel keeps its working sets in global memory when shared
// memory would hold fewer than this many of them per SM.
constexpr int ADJ_MIN_WARPS = 8;
// A batched system of which fewer walkers than this fit in a CTA's shared
// memory (and whose O(N^2) caches are in global memory) runs with its working
// sets in global memory, one walker on each of the CTA's warps.
constexpr int BATCH_GSM_FIT = 4;
// Single-system propagation keeps the working sets in global memory when
// shared memory (SMEM_PER_SM per SM) would hold fewer than PROP_MIN_WARPS of them.
constexpr int PROP_MIN_WARPS = 8;
constexpr size_t SMEM_PER_SM = 227 * 1024;
// Walkers whose shared-memory layout would exceed these sizes keep their O(N^2)
// caches in the cache block (see make_plan).  Measured on water-methane: the
// FP64 kernel, bound by the FP64 pipe, is faster with its geometry in shared
// memory (17.9 M against 14.8 M walker-steps/s); the latency-bound mixed kernel
// is faster with more resident warps and its O(N^2) arrays in global memory
// (38.9 M against 32.7 M).
constexpr size_t GEO_GLOBAL_BYTES = 32 * 1024;
constexpr size_t GEO_GLOBAL_BYTES_MIXED = 8 * 1024;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// F(t) = erf(sqrt t) / sqrt t in long double, for t >= -1 (F is entire:
// F(t) = (2/sqrt pi) sum_n (-t)^n / (n! (2n + 1)), used for |t| < 2).
long double erf_ratio_ld(long double t) {
  if (fabsl(t) < 2.0L) {
    long double term = 1.0L, sum = 0.0L;   // term = (-t)^n / n!
    for (int n = 0; n < 60; ++n) {
      sum += term / (2 * n + 1);
      term *= -t / (n + 1);
    }
    return sum * 1.12837916709551257389615890312154517L;   // 2 / sqrt(pi)
  }
  const long double r = sqrtl(t);
  return erfl(r) / r;
}

// Coefficients of the erf_over_r table (fp64math.cuh): for interval k, the
// degree-(ERF_NC - 1) polynomial in u = t - k/2, |u| <= 1/4, that interpolates
// F at the ERF_NC Chebyshev points of the interval; computed in long double
// (Chebyshev coefficients by the discrete cosine sums, then rewritten in powers
// of u through the three-term recurrence of the Chebyshev polynomials).
void erf_ratio_table(double* out) {
  const int N = ERF_NC;
  const long double pi = 3.14159265358979323846264338327950288L, h = 0.25L;
  for (int k = 0; k < ERF_INT; ++k) {
    const long double c = 0.5L * k;
    long double f[ERF_NC], a[ERF_NC];
    for (int i = 0; i < N; ++i) f[i] = erf_ratio_ld(c + h * cosl(pi * (i + 0.5L) / N));
    for (int j = 0; j < N; ++j) {
      long double sum = 0.0L;
      for (int i = 0; i < N; ++i) sum += f[i] * cosl(pi * j * (i + 0.5L) / N);
      a[j] = (j == 0 ? 1.0L : 2.0L) * sum / N;
    }
    // power-basis coefficients in x = u / h: sum_j a_j T_j(x)
    long double px[ERF_NC] = {0}, tm[ERF_NC] = {0}, t0[ERF_NC] = {0}, t1[ERF_NC] = {0};
    t0[0] = 1.0L;   // T_0
    t1[1] = 1.0L;   // T_1
    for (int i = 0; i < N; ++i) px[i] += a[0] * t0[i];
    if (N > 1)
      for (int i = 0; i < N; ++i) px[i] += a[1] * t1[i];
    for (int j = 2; j < N; ++j) {
      for (int i = 0; i < N; ++i) tm[i] = (i ? 2.0L * t1[i - 1] : 0.0L) - t0[i];   // T_j = 2 x T_{j-1} - T_{j-2}
      for (int i = 0; i < N; ++i) { px[i] += a[j] * tm[i]; t0[i] = t1[i]; t1[i] = tm[i]; }
    }
    long double sc = 1.0L;
    for (int i = 0; i < N; ++i) {
      out[k * N + i] = (double)(px[i] * sc);
      sc /= h;
    }
  }
}

// Everything derived from the inputs before any device work.
struct Plan {
  int n_nuc = 0, n_shell = 0, n_prim = 0, n_bf = 0, n_orb = 0, n_up = 0, n_dn = 0, n_e = 0, n_max = 0;
  int n_w = 0;
  Layout L{};
  LayoutM M{};
  int precision = 0;
  size_t smem_per_warp = 0;
  // workspace offsets (bytes)
  size_t o_sys = 0, sys_bytes = 0, o_state = 0, o_alt = 0, state_bytes = 0, o_cache = 0, o_cache_alt = 0,
         cache_bytes = 0, o_stats = 0, o_part = 0, o_q = 0, o_src = 0, o_dstat = 0, o_stamps = 0, o_scr = 0, o_gsm = 0,
         total = 0;
  int scratch_warps = 0;
  bool gsm = false;   // propagate with the working sets in global memory (large systems)
  // system image offsets (bytes, inside the sys block)
  size_t i_R, i_Z, i_rc, i_irc, i_j1A, i_j1B, i_exps, i_coefs, i_C, i_kind, i_atom, i_l, i_nprim, i_off, i_bf, i_ash,
      i_tab, i_f_R, i_f_Z, i_f_rc, i_f_j1A, i_f_j1B, i_f_exps, i_f_coefs, i_f_C, i_irc2, i_erf, i_ord;
  std::string err;
};

bool make_plan(const lrdmc_system* sys, const lrdmc_trial_wf* wf, const lrdmc_params* prm, Plan& P) {
  if (!sys || !wf || !prm) { P.err = "NULL argument"; return false; }
  if (sys->n_nuc < 1 || !sys->R || !sys->Z || !sys->pot_kind || !sys->r_c) { P.err = "bad nuclei"; return false; }
  if (sys->n_up < 0 || sys->n_dn < 0 || sys->n_up + sys->n_dn < 1) { P.err = "bad electron counts"; return false; }
  if (wf->n_shell < 1 || !wf->shell_atom || !wf->shell_l || !wf->shell_nprim || !wf->exps || !wf->coefs || !wf->C ||
      !wf->j1_A || !wf->j1_B) { P.err = "bad trial wavefunction arrays"; return false; }
  if (!(prm->a > 0.0) || prm->n_w < 1 || prm->n_w > MAX_WALKERS || prm->reinv_period < 1 ||
      prm->node_rule < -1 || prm->node_rule > 2 || prm->p_gbar < 0 || prm->n_equil < 0) {
    P.err = "bad run parameters"; return false;
  }
  if (prm->precision < 0 || prm->precision > 4) {
    P.err = "precision must be 0 (FP64), 1 (mixed), 2 (mixed, TF32 tensor cores), 3 (mixed, BF16 tensor cores) "
            "or 4 (mixed, split-TF32 tensor cores)";
    return false;
  }
  P.precision = prm->precision;
  P.n_nuc = sys->n_nuc;
  P.n_up = sys->n_up;
  P.n_dn = sys->n_dn;
  P.n_e = P.n_up + P.n_dn;
  P.n_max = std::max(P.n_up, P.n_dn);
  P.n_shell = wf->n_shell;
  P.n_w = prm->n_w;
  for (int I = 0; I < P.n_nuc; ++I) {
    if (sys->pot_kind[I] != 0 && sys->pot_kind[I] != 1) { P.err = "pot_kind must be 0 or 1"; return false; }
    if (sys->pot_kind[I] == 1 && !(sys->r_c[I] > 0.0)) { P.err = "r_c must be > 0"; return false; }
  }
  for (int s = 0; s < P.n_shell; ++s) {
    const int l = wf->shell_l[s];
    if (l < -1 || l > 1) { P.err = "shell_l must be -1, 0 or 1"; return false; }
    if (wf->shell_atom[s] < 0 || wf->shell_atom[s] >= P.n_nuc) { P.err = "shell_atom out of range"; return false; }
    if (wf->shell_nprim[s] < 1) { P.err = "shell_nprim must be >= 1"; return false; }
    P.n_prim += wf->shell_nprim[s];
    P.n_bf += (l == 1) ? 3 : 1;
  }
  P.n_orb = wf->n_orb;
  if (P.n_orb < P.n_max) { P.err = "n_orb < max(n_up, n_dn)"; return false; }
  // walker block in global memory
  Layout& L = P.L;
  L.n_e = P.n_e; L.n_up = P.n_up; L.n_dn = P.n_dn; L.n_max = P.n_max; L.n_bf = P.n_bf; L.n_hop = 6 * P.n_e;
  const int nbt = P.n_up * P.n_up + P.n_dn * P.n_dn;
  L.g_x = 0;
  L.g_bt = 3 * P.n_e;
  L.g_cache = L.g_bt + nbt;
  L.g_rat = L.g_cache + 5 * P.n_max * P.n_e;
  L.g_pot = L.g_rat + L.n_hop;
  L.g_sc = round_up(L.g_pot + 2 * P.n_e, 16);
  L.g_stride = round_up(L.g_sc + SC_COUNT, 16);
  // per-warp shared memory; a large FP64 system keeps its electron-nucleus
  // geometry and pair distances (O(N_e N_nuc + N_e^2)) in the cache block
  // instead, so that several of its walkers share an SM
  auto fp64_layout = [&](int geo_glob) {
    L.geo_glob = geo_glob;
    L.s_x = 0;
    L.s_bt = 3 * P.n_e;
    L.s_rat = L.s_bt + nbt;
    L.s_ep = L.s_rat + L.n_hop;
    L.s_ej = L.s_ep + 2 * P.n_e;
    L.s_dd = L.s_ej + 6 * P.n_e;
    L.s_geo = L.s_dd + 4 * P.n_e;
    L.s_pr2 = L.s_geo + (geo_glob ? 0 : 4 * P.n_e * P.n_nuc);
    L.s_hd = L.s_pr2 + (geo_glob ? 0 : P.n_e * P.n_e);
    L.s_hj1 = L.s_hd + L.n_hop;
    L.s_hj2 = L.s_hj1 + L.n_hop;
    L.s_tmp = L.s_hj2 + L.n_hop;
    L.s_phi5 = L.s_tmp + std::max(6 * (P.n_e - 1 + P.n_nuc), 6 * P.n_bf);
    L.s_u = L.s_phi5 + 5 * P.n_max;
    L.s_row = L.s_u + P.n_max;
    L.s_xo = L.s_row + P.n_max;
    L.s_v = L.s_xo + 4;
    L.s_sc = L.s_v + 12;
    L.s_stride = round_up(L.s_sc + SC_COUNT, 4);
    // per-walker cache block
    L.c_mir = 0;
    L.c_g = round_up(L.s_tmp - L.s_ej, 4);
    L.c_chi = L.c_g + P.n_e * P.n_bf;
    L.c_u2 = L.c_chi + P.n_bf * L.n_hop;
    L.c_pt = L.c_u2 + P.n_e * L.n_hop;
    L.c_geo = L.c_pt + 4 * P.n_e * P.n_e;
    L.c_pr2 = L.c_geo + (geo_glob ? 4 * P.n_e * P.n_nuc : 0);
    L.c_stride = round_up(L.c_pr2 + (geo_glob ? P.n_e * P.n_e : 0), 16);
  };
  fp64_layout(0);
  if (P.precision == 0 && (size_t)L.s_stride * sizeof(double) > GEO_GLOBAL_BYTES) fp64_layout(1);
  P.M = layout_mixed(L, P.n_nuc, P.n_prim);
  // a large mixed-precision system keeps its O(N^2) arrays in global memory
  if (P.precision != 0 && (size_t)P.M.stride * sizeof(float) > GEO_GLOBAL_BYTES_MIXED)
    P.M = layout_mixed(L, P.n_nuc, P.n_prim, 1);
  // precision 2 / 3 / 4: the FP32 orbital contractions on the tensor cores
  // (TF32 / BF16 / three TF32 products of split operands)
  P.M.tc = P.precision >= 2 ? P.precision - 1 : 0;
  if (P.precision != 0) L.c_stride = round_up((P.M.c_floats + 1) / 2, 16);
  P.smem_per_warp = P.precision == 0 ? (size_t)L.s_stride * sizeof(double) : (size_t)P.M.stride * sizeof(float);
  if (P.smem_per_warp + EXP_TAB * sizeof(double) > 200 * 1024) { P.err = "system too large for the per-warp shared-memory layout"; return false; }
  // system image
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) / 16 * 16; return r; };
  P.i_R = take(sizeof(double) * 3 * P.n_nuc);
  P.i_Z = take(sizeof(double) * P.n_nuc);
  P.i_rc = take(sizeof(double) * P.n_nuc);
  P.i_irc = take(sizeof(double) * P.n_nuc);
  P.i_j1A = take(sizeof(double) * P.n_nuc);
  P.i_j1B = take(sizeof(double) * P.n_nuc);
  P.i_exps = take(sizeof(double) * P.n_prim);
  P.i_coefs = take(sizeof(double) * P.n_prim);
  P.i_C = take(sizeof(double) * (size_t)P.n_orb * P.n_bf);
  P.i_kind = take(sizeof(int) * P.n_nuc);
  P.i_atom = take(sizeof(int) * P.n_shell);
  P.i_l = take(sizeof(int) * P.n_shell);
  P.i_nprim = take(sizeof(int) * P.n_shell);
  P.i_off = take(sizeof(int) * P.n_shell);
  P.i_bf = take(sizeof(int) * P.n_shell);
  P.i_ash = take(sizeof(int) * (P.n_nuc + 1));
  P.i_ord = take(sizeof(int) * P.n_shell);
  P.i_tab = take(sizeof(double) * EXP_TAB);
  P.i_irc2 = take(sizeof(double) * P.n_nuc);
  P.i_erf = take(sizeof(double) * ERF_INT * ERF_NC);
  P.i_f_R = take(sizeof(float) * 3 * P.n_nuc);
  P.i_f_Z = take(sizeof(float) * P.n_nuc);
  P.i_f_rc = take(sizeof(float) * P.n_nuc);
  P.i_f_j1A = take(sizeof(float) * P.n_nuc);
  P.i_f_j1B = take(sizeof(float) * P.n_nuc);
  P.i_f_exps = take(sizeof(float) * P.n_prim);
  P.i_f_coefs = take(sizeof(float) * P.n_prim);
  P.i_f_C = take(sizeof(float) * (size_t)P.n_orb * P.n_bf);
  P.sys_bytes = o;
  // workspace
  size_t w = 0;
  P.o_sys = w; w += align_up(P.sys_bytes);
  P.state_bytes = (size_t)P.n_w * L.g_stride * sizeof(double);
  P.o_state = w; w += align_up(P.state_bytes);
  P.o_alt = w; w += align_up(P.state_bytes);
  P.cache_bytes = (size_t)P.n_w * L.c_stride * sizeof(double);
  P.o_cache = w; w += align_up(P.cache_bytes);
  P.o_cache_alt = w; w += align_up(P.cache_bytes);
  P.o_stats = w; w += align_up(sizeof(double) * BS_COUNT);
  P.o_part = w; w += align_up(sizeof(double) * BP_STRIDE * (size_t)branch_part_ctas(P.n_w));
  P.o_q = w; w += align_up(sizeof(unsigned long long) * P.n_w);
  P.o_src = w; w += align_up(sizeof(int32_t) * P.n_w);
  P.o_dstat = w; w += align_up(sizeof(int32_t) * 16);
  P.o_stamps = w; w += align_up(sizeof(unsigned long long) * 3 * (size_t)P.n_w);
  // scratch for at least ceil(n / wpb) CTAs of wpb <= 8 warps (n = min(n_w, cap)), so
  // that a launch of one walker per warp never leaves a walker for a second round
  P.scratch_warps = round_up(std::min(P.n_w, SCRATCH_WARPS_CAP) + 7, 4);
  const size_t per_warp = P.precision == 0 ? scratch_doubles(L, P.n_nuc) : scratch_doubles_m(L, P.M);
  P.o_scr = w; w += align_up(sizeof(double) * per_warp * (size_t)P.scratch_warps);
  // a system whose shared layout leaves fewer than PROP_MIN_WARPS warps per SM
  // (and whose O(N^2) caches are already in global memory) is propagated with
  // the working sets in global memory, one region per scratch warp
  const bool glob = P.precision == 0 ? L.geo_glob != 0 : P.M.glob != 0;
  P.gsm = glob && P.smem_per_warp * PROP_MIN_WARPS > SMEM_PER_SM;
  if (P.gsm) { P.o_gsm = w; w += align_up(P.smem_per_warp * (size_t)P.scratch_warps); }
  P.total = w;
  return true;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

double estimate(const std::vector<double>& wbar, const std::vector<double>& ebar, int p, int n0, double* err) {
  const int n = (int)wbar.size();
  std::vector<double> lg(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = std::max(0, k - p); j < k; ++j) s += std::log(wbar[j]);
    lg[k] = s;
  }
  const int m = n - n0;
  if (err) *err = NAN;
  if (m <= 0) return NAN;
  double lmax = -INFINITY;
  for (int k = n0; k < n; ++k) lmax = std::max(lmax, lg[k]);
  std::vector<double> g(m), e(m);
  double num = 0.0, den = 0.0;
  for (int k = 0; k < m; ++k) {
    g[k] = std::exp(lg[n0 + k] - lmax);
    e[k] = ebar[n0 + k];
    num += g[k] * e[k];
    den += g[k];
  }
  if (err && m >= 16) {
    double best = 0.0;
    for (int B = 1; m / B >= 8; B *= 2) {
      const int nb = m / B;
      std::vector<double> bn(nb, 0.0), bd(nb, 0.0);
      for (int b = 0; b < nb; ++b)
        for (int k = b * B; k < (b + 1) * B; ++k) { bn[b] += g[k] * e[k]; bd[b] += g[k]; }
      double tn = 0.0, td = 0.0;
      for (int b = 0; b < nb; ++b) { tn += bn[b]; td += bd[b]; }
      std::vector<double> jk(nb);
      double mean = 0.0;
      for (int b = 0; b < nb; ++b) { jk[b] = (tn - bn[b]) / (td - bd[b]); mean += jk[b]; }
      mean /= nb;
      double var = 0.0;
      for (int b = 0; b < nb; ++b) var += (jk[b] - mean) * (jk[b] - mean);
      var *= (double)(nb - 1) / nb;
      best = std::max(best, std::sqrt(var));
    }
    *err = best;
  }
  return num / den;
}

}  // namespace

struct lrdmc_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns = false;
  Plan P;
  DevSys S{};
  lrdmc_params prm{};
  double* state = nullptr;
  double* alt = nullptr;
  double* cache = nullptr;       // per-walker cache blocks (layout of the precision in use)
  std::vector<double> hR, hZ, hA, hB;   // host copies of the differentiable system parameters
  double* gscr = nullptr;        // per-warp scratch of the adjoint kernel (allocated on first use)
  size_t gscr_per_warp = 0;
  // adjoint launch shape; with adj_gsm set the working sets live in global
  // memory (adj_gsm, with their own per-warp scratch adj_scr)
  int adj_grid = 0, adj_wpb = 0;
  int sm_warps = 0;              // working sets per SM that shared memory holds (launch shape of create)
  int prop_grid = 0, prop_wpb = 0;   // propagate launch shape (differs from grid/wpb with P.gsm)
  void* gsm = nullptr;           // P.gsm: the propagate kernels' working sets
  double* adj_gsm = nullptr;
  double* adj_scr = nullptr;
  double* adj_blk = nullptr;     // per-warp walker blocks of the gradient kernel
  double* cache_alt = nullptr;
  double* stats = nullptr;
  double* part = nullptr;        // branching: per-CTA partial sums
  unsigned long long* Q = nullptr;
  int32_t* src = nullptr;
  int32_t* dstat = nullptr;
  unsigned long long* stamps = nullptr;
  double* scr = nullptr;
  bool timing = false;
  int wpb = 4, grid = 1, num_sms = 1;
  double E0 = 0.0;
  uint32_t interval = 0;
  int last_kind = 1;
  double drift_tol = DRIFT_TOL_DEFAULT;
  std::vector<double> wbar, ebar, e0h, mmean;
  std::vector<int> mmax, surv;
  std::vector<uint32_t> stor;
  std::vector<char> img;         // host copy of the device system image (kept current by set_params)
  int64_t launches = 0;
  std::string err;
};

static lrdmc_status fail(lrdmc_handle h, lrdmc_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

static lrdmc_status cuda_fail(lrdmc_handle h, const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return fail(h, LRDMC_ERR_CUDA, buf);
}

#define CK(h, call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, #call, e_); \
  } while (0)

#define LAUNCHED(h)                                          \
  do {                                                       \
    ++(h)->launches;                                         \
    cudaError_t e_ = cudaGetLastError();                     \
    if (e_ != cudaSuccess) return cuda_fail(h, "kernel launch", e_); \
  } while (0)

// Shared memory of a walker kernel's CTA: the exponential table (FP64 kernels
// only; the mixed kernels read it through L1) and one working set per warp.
static int table_bytes(const Plan& P) { return P.precision == 0 ? (int)(EXP_TAB * sizeof(double)) : 0; }

static int smem_bytes(lrdmc_handle h) {
  return (int)(table_bytes(h->P) + h->wpb * h->P.smem_per_warp);
}

// The dynamic shared-memory limit is a per-kernel attribute shared by every
// handle in the process, so it is raised to the device's opt-in maximum (it
// permits, it reserves nothing); each launch still requests only its own size.
static lrdmc_status set_kernel_smem(lrdmc_handle h, int optin) {
  CK(h, cudaFuncSetAttribute(k_propagate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_propagate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_init_walkers, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_eval_configs, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_eloc_grad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_propagate_m<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_propagate_m<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_init_walkers_m, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  CK(h, cudaFuncSetAttribute(k_eval_configs_m, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  return LRDMC_OK;
}

static int walker_grid(lrdmc_handle h, int n) {
  const int need = (n + h->wpb - 1) / h->wpb;
  return std::max(1, std::min(need, h->grid));
}

// Place walkers from host arrays and evaluate (x staged through the alternate buffer).
static lrdmc_status place_walkers(lrdmc_handle h, const double* x, const double* w) {
  const Plan& P = h->P;
  const size_t xbytes = sizeof(double) * (size_t)P.n_w * 3 * P.n_e;
  double* dx = h->alt;
  double* dw = nullptr;
  CK(h, cudaMemcpyAsync(dx, x, xbytes, cudaMemcpyHostToDevice, h->stream));
  if (w) {
    dw = h->alt + (size_t)P.n_w * 3 * P.n_e;
    CK(h, cudaMemcpyAsync(dw, w, sizeof(double) * P.n_w, cudaMemcpyHostToDevice, h->stream));
  }
  const int smem = smem_bytes(h);
  if (P.precision == 0)
    k_init_walkers<<<walker_grid(h, P.n_w), h->wpb * 32, smem, h->stream>>>(h->S, P.L, h->state, h->cache, dx, dw,
                                                                            P.n_w, h->prm.a, h->prm.node_rule,
                                                                            h->scr);
  else
    k_init_walkers_m<<<walker_grid(h, P.n_w), h->wpb * 32, smem, h->stream>>>(h->S, P.L, P.M, h->state, h->cache, dx, dw,
                                                                              P.n_w, h->prm.a, h->prm.node_rule,
                                                                              h->scr);
  LAUNCHED(h);
  CK(h, cudaStreamSynchronize(h->stream));
  return LRDMC_OK;
}

// Copy the requested walker fields to host memory (any pointer may be null):
// one gather kernel into the alternate buffer, one copy per field straight
// into the caller's buffer, then a synchronisation.
static lrdmc_status fetch(lrdmc_handle h, double* x, double* w, double* ev, double* ratios, uint32_t* status,
                          int32_t* moves) {
  const Plan& P = h->P;
  const size_t nx = (size_t)P.n_w * 3 * P.n_e, nr = (size_t)P.n_w * P.L.n_hop, nw = P.n_w;
  double* b = h->alt;
  double* dx = x ? b : nullptr;
  double* dw = w ? b + nx : nullptr;
  double* dev = ev ? b + nx + nw : nullptr;
  double* drat = ratios ? b + nx + 5 * nw : nullptr;
  uint32_t* dst = status ? (uint32_t*)(b + nx + 5 * nw + nr) : nullptr;
  int32_t* dmv = moves ? (int32_t*)(b + nx + 5 * nw + nr) + nw : nullptr;
  const size_t tot = (x ? nx : 0) + (ratios ? nr : 0) + nw;
  k_extract<<<std::max(1, std::min(1024, (int)((tot + 255) / 256))), 256, 0, h->stream>>>(P.L, h->state, P.n_w, dx,
                                                                                        dw, dev, drat, dst, dmv);
  LAUNCHED(h);
  if (x) CK(h, cudaMemcpyAsync(x, dx, sizeof(double) * nx, cudaMemcpyDeviceToHost, h->stream));
  if (w) CK(h, cudaMemcpyAsync(w, dw, sizeof(double) * nw, cudaMemcpyDeviceToHost, h->stream));
  if (ev) CK(h, cudaMemcpyAsync(ev, dev, sizeof(double) * 4 * nw, cudaMemcpyDeviceToHost, h->stream));
  if (ratios) CK(h, cudaMemcpyAsync(ratios, drat, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->stream));
  if (status) CK(h, cudaMemcpyAsync(status, dst, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost, h->stream));
  if (moves) CK(h, cudaMemcpyAsync(moves, dmv, sizeof(int32_t) * nw, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return LRDMC_OK;
}

// Host side of a branching after the statistics hs of the handle's population
// are read back: swap in the gathered population (swap: gathered into the
// alternate buffers; else in place), extend the history, advance the interval
// and (load-balanced) update E_0.
static lrdmc_status finish_branch(lrdmc_handle h, const double* hs, bool swap) {
  const Plan& P = h->P;
  if (hs[BS_BAD] != 0.0)
    return fail(h, LRDMC_ERR_NONFINITE, "weights negative, non-finite or all zero: population unchanged");
  const int lb = h->last_kind == LRDMC_LOAD_BALANCED;
  if (swap) {
    std::swap(h->state, h->alt);
    std::swap(h->cache, h->cache_alt);
  }
  h->wbar.push_back(hs[BS_SUMW] / (double)P.n_w);
  h->ebar.push_back(hs[BS_SUMFE] / hs[BS_SUMF]);
  h->e0h.push_back(h->E0);
  h->mmean.push_back(hs[BS_MOVES] / (double)P.n_w);
  h->mmax.push_back((int)hs[BS_MOVESMAX]);
  h->surv.push_back((int)hs[BS_SURV]);
  h->stor.push_back((uint32_t)hs[BS_STATUS]);
  ++h->interval;
  if (lb) h->E0 = estimate(h->wbar, h->ebar, h->prm.p_gbar, 0, nullptr);
  return LRDMC_OK;
}

// Step parameters of one interval of handle h under schedule sch.
static StepParams step_params(lrdmc_handle h, const lrdmc_schedule* sch) {
  StepParams sp;
  sp.kind = sch->kind;
  sp.n_proj = sch->n_proj;
  sp.tau = sch->tau;
  sp.max_moves = sch->max_moves;
  sp.E0 = h->E0;
  sp.seed = h->prm.seed;
  sp.interval = h->interval;
  sp.a = h->prm.a;
  sp.node_rule = h->prm.node_rule;
  sp.reinv_period = h->prm.reinv_period;
  sp.drift_tol = h->drift_tol;
  sp.drift_count = h->dstat + DSTAT_DRIFT;
  sp.stamps = h->timing ? h->stamps : nullptr;
  sp.rotate = sch->rotate != 0;
  sp.next = nullptr;
  return sp;
}

// Schedule arguments shared by the single and batched entry points.
static const char* check_schedule(const lrdmc_schedule* sch) {
  if (!sch) return "NULL schedule";
  if (sch->kind != LRDMC_CONVENTIONAL && sch->kind != LRDMC_LOAD_BALANCED) return "schedule kind must be 0 or 1";
  if (sch->kind == LRDMC_LOAD_BALANCED && sch->n_proj < 0) return "n_proj < 0";
  if (sch->kind == LRDMC_CONVENTIONAL && (!(sch->tau > 0.0) || sch->max_moves < 1))
    return "conventional schedule needs tau > 0 and max_moves >= 1";
  return nullptr;
}

// ------------------------------------------------------------------ batches
struct lrdmc_batch_s {
  std::vector<lrdmc_handle> h;
  int precision = 0, device = 0, num_sms = 1, smem_optin = 0;
  int max_threads = 1024;        // of the batched kernel (its register use)
  cudaStream_t stream = nullptr;
  int policy = 1;
  size_t cta_dyn = 0;            // dynamic shared bytes per CTA of the current launch shape
  int wmax = 1, grid = 1;        // warps per CTA, CTAs
  std::vector<int> fit;          // walkers per item, per system, for the current shape
  std::vector<int> gsm;          // per system: working sets in global memory (current shape)
  double* d_gsm = nullptr;       // those working sets: grid x wmax warps x gsm_stride doubles
  size_t gsm_stride = 0, gsm_cap = 0;
  size_t scratch_per_warp = 0;   // global scratch doubles per warp
  size_t scratch_warps = 0;      // warps the scratch is sized for
  int total = 0, n_items = 0;    // walkers over all systems; items of the current shape
  PropJob* d_jobs = nullptr;
  BranchJob* d_bjobs = nullptr;
  int4* d_items = nullptr;
  unsigned* d_counter = nullptr;
  double* d_scratch = nullptr;
  double* d_stats = nullptr;     // [n][BS_COUNT]
  int32_t* d_status = nullptr;   // [n][2]
  std::vector<PropJob> jobs;
  std::vector<BranchJob> bjobs;
  bool timing = false;
  int64_t launches = 0;
  std::string err;
};

static lrdmc_status bfail(lrdmc_batch b, lrdmc_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

#define BCK(b, call)                                                   \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      char buf_[512];                                                  \
      snprintf(buf_, sizeof buf_, "%s: %s", #call, cudaGetErrorString(e_)); \
      return bfail(b, LRDMC_ERR_CUDA, buf_);                           \
    }                                                                  \
  } while (0)

#define BLAUNCHED(b)                                                   \
  do {                                                                 \
    ++(b)->launches;                                                   \
    cudaError_t e_ = cudaGetLastError();                               \
    if (e_ != cudaSuccess) return bfail(b, LRDMC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// Shared doubles one walker of handle h needs in a batched CTA.
static int batch_region(lrdmc_handle h) {
  const Plan& P = h->P;
  return round_up(P.precision == 0 ? P.L.s_stride : (P.M.stride + 1) / 2, 2);
}

// Launch shape for cta_dyn dynamic shared bytes per CTA: walkers per item of
// every system, warps per CTA and CTAs per SM.  *ok = false when a system
// does not fit or the kernel does not fit on an SM.
static lrdmc_status batch_shape(lrdmc_batch b, size_t cta_dyn, bool* ok, std::vector<int>& fit, int* wmax,
                                int* bps, std::vector<int>* gsm = nullptr) {
  *ok = false;
  const long avail = (long)cta_dyn / (long)sizeof(double) - EXP_TAB - JOB_WORDS;
  const int cap = std::max(1, b->max_threads / 32);
  fit.assign(b->h.size(), 0);
  if (gsm) gsm->assign(b->h.size(), 0);
  int w = 0;
  for (size_t k = 0; k < b->h.size(); ++k) {
    const Plan& P = b->h[k]->P;
    const long n = avail / batch_region(b->h[k]);
    const bool glob = P.precision == 0 ? P.L.geo_glob != 0 : P.M.glob != 0;
    if (n < BATCH_GSM_FIT && glob) {
      // too large to share a CTA's shared memory: global working sets, one walker per warp
      fit[k] = std::min(cap, P.n_w);
      if (gsm) (*gsm)[k] = 1;
    } else {
      if (n < 1) return LRDMC_OK;
      fit[k] = (int)std::min<long>(std::min<long>(n, cap), P.n_w);
    }
    w = std::max(w, fit[k]);
  }
  *wmax = w;
  if (b->precision == 0)
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_propagate_batch<0>, w * 32, cta_dyn));
  else
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_propagate_batch<1>, w * 32, cta_dyn));
  *ok = *bps >= 1;
  return LRDMC_OK;
}

// Work items (system, first walker, count) in the order of the current policy.
static lrdmc_status batch_items(lrdmc_batch b) {
  const int n = (int)b->h.size();
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  if (b->policy == 1) {
    auto cost = [&](int k) {
      const Plan& P = b->h[k]->P;
      return (double)P.n_e * (double)(P.n_bf + P.n_nuc + P.n_e);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  }
  std::vector<int4> items;
  for (int k : order)
    for (int w0 = 0; w0 < b->h[k]->P.n_w; w0 += b->fit[k])
      items.push_back(make_int4(k, w0, std::min(b->fit[k], b->h[k]->P.n_w - w0), 0));
  b->n_items = (int)items.size();
  BCK(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return LRDMC_OK;
}

// Adopt the launch shape for cta_dyn bytes (it must fit) and rebuild the items.
static lrdmc_status batch_use(lrdmc_batch b, size_t cta_dyn) {
  bool ok = false;
  std::vector<int> fit, gsm;
  int w = 0, bps = 0;
  lrdmc_status st = batch_shape(b, cta_dyn, &ok, fit, &w, &bps, &gsm);
  if (st != LRDMC_OK) return st;
  if (!ok) return bfail(b, LRDMC_ERR_UNSUPPORTED, "batched launch shape does not fit");
  const int grid = std::max(1, std::min(bps * b->num_sms, (int)(b->scratch_warps / w)));
  // global working sets of the systems that do not share a CTA (grown, never shrunk)
  size_t stride = 0;
  for (size_t k = 0; k < b->h.size(); ++k)
    if (gsm[k]) stride = std::max(stride, (size_t)batch_region(b->h[k]));
  const size_t need = stride * (size_t)grid * w;
  if (need > b->gsm_cap) {
    BCK(b, cudaStreamSynchronize(b->stream));
    if (b->d_gsm) BCK(b, cudaFree(b->d_gsm));
    b->d_gsm = nullptr;
    b->gsm_cap = 0;
    BCK(b, cudaMalloc(&b->d_gsm, sizeof(double) * need));
    b->gsm_cap = need;
  }
  b->gsm_stride = stride;
  b->cta_dyn = cta_dyn;
  b->fit = fit;
  b->gsm = gsm;
  b->wmax = w;
  b->grid = grid;
  return batch_items(b);
}

// Candidate shapes: the CTA's dynamic shared memory is the opt-in maximum or
// its half, third or quarter (one to four CTAs per SM).
static size_t batch_candidate(lrdmc_batch b, int c) {
  const size_t top = (size_t)b->smem_optin - 1024;   // room for the static shared word
  return top / (size_t)(c + 1) / 16 * 16;
}

static void batch_free(lrdmc_batch b) {
  cudaFree(b->d_jobs);
  cudaFree(b->d_bjobs);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_scratch);
  cudaFree(b->d_stats);
  cudaFree(b->d_status);
  cudaFree(b->d_gsm);
  for (lrdmc_handle h : b->h) lrdmc_destroy(h);
  b->h.clear();
}

// One batched interval with the current launch shape (no argument checks).
static lrdmc_status batch_launch(lrdmc_batch b, const lrdmc_schedule* sch) {
  const int n = (int)b->h.size();
  for (int k = 0; k < n; ++k) {
    lrdmc_handle h = b->h[k];
    PropJob& J = b->jobs[k];
    J.S = h->S;
    J.L = h->P.L;
    J.M = h->P.M;
    J.P = step_params(h, sch);
    J.state = h->state;
    J.cache = h->cache;
    J.n_w = h->P.n_w;
    J.region = batch_region(h);
    J.gsm = b->gsm[k];
    h->last_kind = sch->kind;
  }
  BCK(b, cudaMemcpyAsync(b->d_jobs, b->jobs.data(), sizeof(PropJob) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), b->stream));
  if (b->precision == 0)
    k_propagate_batch<0><<<b->grid, b->wmax * 32, b->cta_dyn, b->stream>>>(
        b->d_jobs, b->d_items, b->n_items, b->d_counter, b->d_scratch, b->scratch_per_warp, b->d_gsm, b->gsm_stride);
  else
    k_propagate_batch<1><<<b->grid, b->wmax * 32, b->cta_dyn, b->stream>>>(
        b->d_jobs, b->d_items, b->n_items, b->d_counter, b->d_scratch, b->scratch_per_warp, b->d_gsm, b->gsm_stride);
  BLAUNCHED(b);
  return LRDMC_OK;
}

extern "C" {

const char* lrdmc_status_string(lrdmc_status s) {
  switch (s) {
    case LRDMC_OK: return "ok";
    case LRDMC_ERR_ARG: return "invalid argument";
    case LRDMC_ERR_CUDA: return "CUDA error";
    case LRDMC_ERR_NONFINITE: return "non-finite or invalid weights";
    case LRDMC_ERR_NEG_DIAG: return "W - E0 <= 0";
    case LRDMC_ERR_STEP_CAP: return "step cap reached";
    case LRDMC_ERR_SINGULAR: return "singular Slater matrix";
    case LRDMC_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

const char* lrdmc_last_error(lrdmc_handle h) { return h ? h->err.c_str() : "NULL handle"; }

void lrdmc_philox4x32(uint64_t seed, const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  for (int k = 0; k < 4; ++k) out[k] = c[k];
}

lrdmc_status lrdmc_workspace_bytes(const lrdmc_system* sys, const lrdmc_trial_wf* wf, const lrdmc_params* prm,
                                   size_t* bytes) {
  Plan P;
  if (!bytes) return LRDMC_ERR_ARG;
  if (!make_plan(sys, wf, prm, P))
    return P.err.find("too large") != std::string::npos ? LRDMC_ERR_UNSUPPORTED : LRDMC_ERR_ARG;
  *bytes = P.total;
  return LRDMC_OK;
}

lrdmc_status lrdmc_create(const lrdmc_system* sys, const lrdmc_trial_wf* wf, const lrdmc_params* prm,
                          const double* x0, void* workspace, size_t workspace_bytes, void* stream,
                          lrdmc_handle* out) {
  if (!out) return LRDMC_ERR_ARG;
  *out = nullptr;
  lrdmc_handle h = new lrdmc_s();
  if (!make_plan(sys, wf, prm, h->P) || !x0) {
    lrdmc_status s = (h->P.err.find("too large") != std::string::npos) ? LRDMC_ERR_UNSUPPORTED : LRDMC_ERR_ARG;
    *out = h;   // keep the handle so the caller can read the message; destroy frees it
    if (!x0) h->err = "x0 is NULL"; else h->err = h->P.err;
    return s;
  }
  const Plan& P = h->P;
  h->prm = *prm;
  h->stream = (cudaStream_t)stream;
  *out = h;
  CK(h, cudaGetDevice(&h->device));
  CK(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  if (workspace) {
    if (workspace_bytes < P.total) return fail(h, LRDMC_ERR_ARG, "workspace too small");
    if ((uintptr_t)workspace % ALIGN) return fail(h, LRDMC_ERR_ARG, "workspace not 256-byte aligned");
    h->ws = workspace;
    h->ws_bytes = workspace_bytes;
  } else {
    CK(h, cudaMalloc(&h->ws, P.total));
    h->owns = true;
    h->ws_bytes = P.total;
  }
  char* base = (char*)h->ws;
  // system image
  std::vector<char> img(P.sys_bytes, 0);
  auto putd = [&](size_t off, const double* src, size_t n) { if (n) memcpy(img.data() + off, src, n * sizeof(double)); };
  auto puti = [&](size_t off, const int* src, size_t n) { if (n) memcpy(img.data() + off, src, n * sizeof(int)); };
  putd(P.i_R, sys->R, 3 * (size_t)P.n_nuc);
  putd(P.i_Z, sys->Z, P.n_nuc);
  putd(P.i_rc, sys->r_c, P.n_nuc);
  {
    std::vector<double> irc(P.n_nuc);
    for (int I = 0; I < P.n_nuc; ++I) irc[I] = sys->pot_kind[I] == 1 ? 1.0 / sys->r_c[I] : 0.0;
    putd(P.i_irc, irc.data(), irc.size());
    for (int I = 0; I < P.n_nuc; ++I)
      irc[I] = sys->pot_kind[I] == 1 ? (double)(1.0L / ((long double)sys->r_c[I] * sys->r_c[I])) : 0.0;
    putd(P.i_irc2, irc.data(), irc.size());
  }
  {
    std::vector<double> et(ERF_INT * ERF_NC);
    erf_ratio_table(et.data());
    putd(P.i_erf, et.data(), et.size());
  }
  putd(P.i_j1A, wf->j1_A, P.n_nuc);
  putd(P.i_j1B, wf->j1_B, P.n_nuc);
  putd(P.i_exps, wf->exps, P.n_prim);
  putd(P.i_coefs, wf->coefs, P.n_prim);
  putd(P.i_C, wf->C, (size_t)P.n_orb * P.n_bf);
  puti(P.i_kind, sys->pot_kind, P.n_nuc);
  // shells grouped by nucleus (stable); each keeps its primitive and basis offsets
  std::vector<int> off(P.n_shell), bf(P.n_shell);
  for (int s = 0, po = 0, bo = 0; s < P.n_shell; ++s) {
    off[s] = po; bf[s] = bo;
    po += wf->shell_nprim[s];
    bo += wf->shell_l[s] == 1 ? 3 : 1;
  }
  std::vector<int> order(P.n_shell);
  for (int s = 0; s < P.n_shell; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return wf->shell_atom[x] < wf->shell_atom[y]; });
  std::vector<int> r_atom(P.n_shell), r_l(P.n_shell), r_np(P.n_shell), r_off(P.n_shell), r_bf(P.n_shell);
  std::vector<int> ash(P.n_nuc + 1, 0);
  for (int k = 0; k < P.n_shell; ++k) {
    const int s = order[k];
    r_atom[k] = wf->shell_atom[s]; r_l[k] = wf->shell_l[s]; r_np[k] = wf->shell_nprim[s];
    r_off[k] = off[s]; r_bf[k] = bf[s];
    ash[r_atom[k] + 1]++;
  }
  for (int I = 0; I < P.n_nuc; ++I) ash[I + 1] += ash[I];
  puti(P.i_atom, r_atom.data(), P.n_shell);
  puti(P.i_l, r_l.data(), P.n_shell);
  puti(P.i_nprim, r_np.data(), P.n_shell);
  puti(P.i_off, r_off.data(), P.n_shell);
  puti(P.i_bf, r_bf.data(), P.n_shell);
  puti(P.i_ash, ash.data(), P.n_nuc + 1);
  {
    // shells in the order the per-hop basis pass takes them: non-p first, so
    // that lanes of one warp pass mostly share a shell kind
    std::vector<int> ord;
    for (int k = 0; k < P.n_shell; ++k)
      if (r_l[k] != 1) ord.push_back(k);
    h->S.n_shell_np = (int)ord.size();
    for (int k = 0; k < P.n_shell; ++k)
      if (r_l[k] == 1) ord.push_back(k);
    puti(P.i_ord, ord.data(), ord.size());
  }
  double tab[EXP_TAB];
  for (int j = 0; j < EXP_TAB; ++j) tab[j] = (double)exp2l((long double)j / EXP_TAB);
  putd(P.i_tab, tab, EXP_TAB);
  auto putf = [&](size_t off, const double* src, size_t n) {
    for (size_t k = 0; k < n; ++k) {
      const float v = (float)src[k];
      memcpy(img.data() + off + k * sizeof(float), &v, sizeof(float));
    }
  };
  putf(P.i_f_R, sys->R, 3 * (size_t)P.n_nuc);
  putf(P.i_f_Z, sys->Z, P.n_nuc);
  putf(P.i_f_rc, sys->r_c, P.n_nuc);
  putf(P.i_f_j1A, wf->j1_A, P.n_nuc);
  putf(P.i_f_j1B, wf->j1_B, P.n_nuc);
  putf(P.i_f_exps, wf->exps, P.n_prim);
  putf(P.i_f_coefs, wf->coefs, P.n_prim);
  putf(P.i_f_C, wf->C, (size_t)P.n_orb * P.n_bf);
  char* dsys = base + P.o_sys;
  h->img = img;
  CK(h, cudaMemcpyAsync(dsys, h->img.data(), P.sys_bytes, cudaMemcpyHostToDevice, h->stream));
  DevSys& S = h->S;
  S.n_nuc = P.n_nuc; S.n_shell = P.n_shell; S.n_prim = P.n_prim; S.n_bf = P.n_bf; S.n_orb = P.n_orb;
  S.n_up = P.n_up; S.n_dn = P.n_dn; S.n_e = P.n_e; S.n_max = P.n_max;
  S.R = (const double*)(dsys + P.i_R);
  S.Z = (const double*)(dsys + P.i_Z);
  S.rc = (const double*)(dsys + P.i_rc);
  S.irc = (const double*)(dsys + P.i_irc);
  S.j1A = (const double*)(dsys + P.i_j1A);
  S.j1B = (const double*)(dsys + P.i_j1B);
  S.exps = (const double*)(dsys + P.i_exps);
  S.coefs = (const double*)(dsys + P.i_coefs);
  S.C = (const double*)(dsys + P.i_C);
  S.kind = (const int*)(dsys + P.i_kind);
  S.sh_atom = (const int*)(dsys + P.i_atom);
  S.sh_l = (const int*)(dsys + P.i_l);
  S.sh_nprim = (const int*)(dsys + P.i_nprim);
  S.sh_off = (const int*)(dsys + P.i_off);
  S.sh_bf = (const int*)(dsys + P.i_bf);
  S.atom_sh = (const int*)(dsys + P.i_ash);
  S.sh_ord = (const int*)(dsys + P.i_ord);
  S.exptab = (const double*)(dsys + P.i_tab);
  S.irc2 = (const double*)(dsys + P.i_irc2);
  S.erftab = (const double*)(dsys + P.i_erf);
  S.Rf = (const float*)(dsys + P.i_f_R);
  S.Zf = (const float*)(dsys + P.i_f_Z);
  S.rcf = (const float*)(dsys + P.i_f_rc);
  S.j1Af = (const float*)(dsys + P.i_f_j1A);
  S.j1Bf = (const float*)(dsys + P.i_f_j1B);
  S.expsf = (const float*)(dsys + P.i_f_exps);
  S.coefsf = (const float*)(dsys + P.i_f_coefs);
  S.Cf = (const float*)(dsys + P.i_f_C);
  S.j2_anti = wf->j2_anti;
  S.j2_par = wf->j2_par;
  S.j2_b = wf->j2_b;
  S.j2_antif = (float)S.j2_anti;
  S.j2_parf = (float)S.j2_par;
  S.j2_bf = (float)S.j2_b;
  double vii = 0.0;
  for (int I = 0; I < P.n_nuc; ++I)
    for (int J = I + 1; J < P.n_nuc; ++J) {
      const double dx = sys->R[3 * I] - sys->R[3 * J], dy = sys->R[3 * I + 1] - sys->R[3 * J + 1],
                   dz = sys->R[3 * I + 2] - sys->R[3 * J + 2];
      vii += sys->Z[I] * sys->Z[J] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
  S.v_ii = vii;
  h->hR.assign(sys->R, sys->R + 3 * (size_t)P.n_nuc);
  h->hZ.assign(sys->Z, sys->Z + P.n_nuc);
  h->hA.assign(wf->j1_A, wf->j1_A + P.n_nuc);
  h->hB.assign(wf->j1_B, wf->j1_B + P.n_nuc);
  h->state = (double*)(base + P.o_state);
  h->alt = (double*)(base + P.o_alt);
  h->cache = P.cache_bytes ? (double*)(base + P.o_cache) : nullptr;
  h->cache_alt = P.cache_bytes ? (double*)(base + P.o_cache_alt) : nullptr;
  h->stats = (double*)(base + P.o_stats);
  h->part = (double*)(base + P.o_part);
  h->Q = (unsigned long long*)(base + P.o_q);
  h->src = (int32_t*)(base + P.o_src);
  h->dstat = (int32_t*)(base + P.o_dstat);
  h->stamps = (unsigned long long*)(base + P.o_stamps);
  h->scr = (double*)(base + P.o_scr);
  h->gsm = P.gsm ? (void*)(base + P.o_gsm) : nullptr;
  CK(h, cudaMemsetAsync(h->dstat, 0, sizeof(int32_t) * 16, h->stream));
  // launch geometry: up to 4 walkers (warps) per CTA within the shared-memory budget
  int smem_optin = 0;
  CK(h, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  lrdmc_status st = set_kernel_smem(h, smem_optin);
  if (st != LRDMC_OK) return st;
  // walkers (warps) per CTA: the count that keeps the most warps resident per
  // SM (shared memory is the limit; ties go to larger CTAs, fewer table copies)
  int best_warps = 0, best_wpb = 1, best_bps = 0;
  for (int wpb = 1; wpb <= 8; ++wpb) {
    h->wpb = wpb;
    if ((size_t)smem_bytes(h) > (size_t)smem_optin) break;
    int bps = 0;
    if (P.precision == 0)
      CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_propagate<false>, wpb * 32, smem_bytes(h)));
    else
      CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &bps, P.M.glob ? k_propagate_m<false, 1> : k_propagate_m<false, 0>, wpb * 32, smem_bytes(h)));
    if (bps >= 1 && bps * wpb >= best_warps) {
      best_warps = bps * wpb;
      best_wpb = wpb;
      best_bps = bps;
    }
  }
  if (best_warps == 0) return fail(h, LRDMC_ERR_UNSUPPORTED, "walker working set exceeds shared memory");
  h->wpb = best_wpb;
  h->sm_warps = best_warps;
  h->grid = std::max(1, std::min(best_bps * h->num_sms, P.scratch_warps / h->wpb));
  h->prop_wpb = h->wpb;
  h->prop_grid = h->grid;
  if (P.gsm) {
    // working sets in global memory: as many 4-warp CTAs as the registers allow
    int bps = 0;
    h->prop_wpb = 4;
    if (P.precision == 0)
      CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_propagate_g<false>, 4 * 32,
                                                          EXP_TAB * sizeof(double)));
    else
      CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_propagate_m<true, -1>, 4 * 32, 0));
    if (bps < 1) return fail(h, LRDMC_ERR_UNSUPPORTED, "propagate kernel does not fit an SM");
    h->prop_grid = std::max(1, std::min(bps * h->num_sms, P.scratch_warps / h->prop_wpb));
  }
  st = place_walkers(h, x0, nullptr);
  if (st != LRDMC_OK) return st;
  std::vector<double> ev(4 * (size_t)P.n_w);
  st = fetch(h, nullptr, nullptr, ev.data(), nullptr, nullptr, nullptr);
  if (st != LRDMC_OK) return st;
  double s = 0.0;
  for (int a = 0; a < P.n_w; ++a) s += ev[4 * (size_t)a + 3];
  h->E0 = s / (double)P.n_w;
  return LRDMC_OK;
}

lrdmc_status lrdmc_destroy(lrdmc_handle h) {
  if (!h) return LRDMC_ERR_ARG;
  if (h->owns && h->ws) {
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
  }
  if (h->gscr) {
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->gscr);
  }
  if (h->adj_gsm || h->adj_blk) {
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->adj_gsm) cudaFree(h->adj_gsm);
    if (h->adj_blk) cudaFree(h->adj_blk);
  }
  delete h;
  return LRDMC_OK;
}

lrdmc_status lrdmc_propagate(lrdmc_handle h, const lrdmc_schedule* sch) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  if (const char* bad = check_schedule(sch)) return fail(h, LRDMC_ERR_ARG, bad);
  if (sch->rotate && h->P.precision != 0)
    return fail(h, LRDMC_ERR_UNSUPPORTED, "the randomised lattice is implemented for precision 0 only");
  DeviceGuard g(h->device);
  StepParams sp = step_params(h, sch);
  // dynamic walker assignment: the work counter (status word 8) starts at zero
  sp.next = (unsigned*)(h->dstat + DSTAT_NEXT);
  CK(h, cudaMemsetAsync(sp.next, 0, sizeof(unsigned), h->stream));
  const Plan& P = h->P;
  const int grid = std::max(1, std::min(h->prop_grid, (P.n_w + h->prop_wpb - 1) / h->prop_wpb));
  const int threads = h->prop_wpb * 32;
  const int smem = P.gsm ? table_bytes(P) : smem_bytes(h);
  double* gd = (double*)h->gsm;
  float* gf = (float*)h->gsm;
  if (P.precision == 0) {
    if (sp.rotate) {
      if (P.gsm)
        k_propagate_g<true><<<grid, threads, smem, h->stream>>>(h->S, P.L, h->state, h->cache, P.n_w, sp, h->scr,
                                                                gd);
      else
        k_propagate<true><<<grid, threads, smem, h->stream>>>(h->S, P.L, h->state, h->cache, P.n_w, sp, h->scr);
    } else {
      if (P.gsm)
        k_propagate_g<false><<<grid, threads, smem, h->stream>>>(h->S, P.L, h->state, h->cache, P.n_w, sp, h->scr,
                                                                 gd);
      else
        k_propagate<false><<<grid, threads, smem, h->stream>>>(h->S, P.L, h->state, h->cache, P.n_w, sp, h->scr);
    }
  } else {
    if (P.gsm)
      k_propagate_m<true, -1><<<grid, threads, smem, h->stream>>>(h->S, P.L, P.M, h->state, h->cache, P.n_w, sp,
                                                                  h->scr, gf);
    else if (P.M.glob)
      k_propagate_m<false, 1><<<grid, threads, smem, h->stream>>>(h->S, P.L, P.M, h->state, h->cache, P.n_w, sp,
                                                                  h->scr, nullptr);
    else
      k_propagate_m<false, 0><<<grid, threads, smem, h->stream>>>(h->S, P.L, P.M, h->state, h->cache, P.n_w, sp,
                                                                  h->scr, nullptr);
  }
  LAUNCHED(h);
  h->last_kind = sch->kind;
  return LRDMC_OK;
}

lrdmc_status lrdmc_branch(lrdmc_handle h) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  const Plan& P = h->P;
  const int lb = h->last_kind == LRDMC_LOAD_BALANCED;
  // per-walker FP64 work over the grid, the integer comb in one CTA
  const int nc = branch_part_ctas(P.n_w);
  k_branch_partials<<<nc, BP_THREADS, 0, h->stream>>>(P.L, h->state, P.n_w, h->E0, lb, h->part);
  LAUNCHED(h);
  k_branch_combine<<<1, 32, 0, h->stream>>>(h->part, nc, h->stats);
  LAUNCHED(h);
  k_quantise<<<nc, BP_THREADS, 0, h->stream>>>(h->state + P.L.g_sc + SC_W, P.L.g_stride, P.n_w, h->stats, h->Q);
  LAUNCHED(h);
  const uint32_t xi = branch_offset32(h->prm.seed, h->interval);
  k_reconfigure_q<<<1, BR_THREADS, 0, h->stream>>>(P.n_w, xi, h->Q, h->src, h->dstat, h->stats);
  LAUNCHED(h);
  // in place: only the slots of walkers the comb did not select receive a copy
  k_gather_slots<<<P.n_w, 256, 0, h->stream>>>(P.L, h->state, h->cache, h->src, h->dstat);
  LAUNCHED(h);
  double hs[BS_COUNT];
  CK(h, cudaMemcpyAsync(hs, h->stats, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return finish_branch(h, hs, false);
}

lrdmc_status lrdmc_energy(lrdmc_handle h, double* E, double* err) {
  if (!h || !E) return LRDMC_ERR_ARG;
  *E = estimate(h->wbar, h->ebar, h->prm.p_gbar, h->prm.n_equil, err);
  return LRDMC_OK;
}

lrdmc_status lrdmc_estimate(int n, const double* wbar, const double* ebar, int p_gbar, int n_equil, double* E,
                            double* err) {
  if (n < 0 || (n > 0 && (!wbar || !ebar)) || p_gbar < 0 || n_equil < 0 || !E) return LRDMC_ERR_ARG;
  for (int k = 0; k < n; ++k)
    if (!(wbar[k] > 0.0) || !std::isfinite(wbar[k]) || !std::isfinite(ebar[k])) return LRDMC_ERR_ARG;
  const std::vector<double> wb(wbar, wbar + n), eb(ebar, ebar + n);
  *E = estimate(wb, eb, p_gbar, n_equil, err);
  return LRDMC_OK;
}

lrdmc_status lrdmc_extrapolate_a(int n, const double* a, const double* E, const double* err, int order,
                                 double* coef, double* cov, double* chi2) {
  if (!a || !E || !err || !coef || order < 1 || order > 3 || n < order + 1) return LRDMC_ERR_ARG;
  const int m = order + 1;
  for (int k = 0; k < n; ++k)
    if (!(std::isfinite(a[k]) && a[k] > 0.0 && std::isfinite(err[k]) && err[k] > 0.0 && std::isfinite(E[k])))
      return LRDMC_ERR_ARG;
  // weighted design X[k][j] = a_k^(2j) / err_k and right-hand side E_k / err_k
  std::vector<double> X((size_t)n * m), y(n);
  for (int k = 0; k < n; ++k) {
    double p = 1.0;
    for (int j = 0; j < m; ++j) {
      X[(size_t)k * m + j] = p / err[k];
      p *= a[k] * a[k];
    }
    y[k] = E[k] / err[k];
  }
  // Householder QR: column j is reflected onto e_j; the same reflections act on y
  std::vector<double> R((size_t)m * m, 0.0);
  double scale = 0.0;
  for (int j = 0; j < m; ++j)
    for (int k = 0; k < n; ++k) scale = std::max(scale, std::fabs(X[(size_t)k * m + j]));
  for (int j = 0; j < m; ++j) {
    double norm = 0.0;
    for (int k = j; k < n; ++k) norm += X[(size_t)k * m + j] * X[(size_t)k * m + j];
    norm = std::sqrt(norm);
    if (!(norm > 1e-13 * scale)) return LRDMC_ERR_ARG;
    const double alpha = X[(size_t)j * m + j] > 0.0 ? -norm : norm;
    std::vector<double> v(n, 0.0);
    for (int k = j; k < n; ++k) v[k] = X[(size_t)k * m + j];
    v[j] -= alpha;
    double vv = 0.0;
    for (int k = j; k < n; ++k) vv += v[k] * v[k];
    for (int c = j; c < m; ++c) {
      double d = 0.0;
      for (int k = j; k < n; ++k) d += v[k] * X[(size_t)k * m + c];
      const double f = 2.0 * d / vv;
      for (int k = j; k < n; ++k) X[(size_t)k * m + c] -= f * v[k];
    }
    double d = 0.0;
    for (int k = j; k < n; ++k) d += v[k] * y[k];
    const double f = 2.0 * d / vv;
    for (int k = j; k < n; ++k) y[k] -= f * v[k];
  }
  for (int j = 0; j < m; ++j)
    for (int c = j; c < m; ++c) R[(size_t)j * m + c] = X[(size_t)j * m + c];
  // back substitution R coef = (Q^T y)[0..m)
  for (int j = m - 1; j >= 0; --j) {
    double s = y[j];
    for (int c = j + 1; c < m; ++c) s -= R[(size_t)j * m + c] * coef[c];
    coef[j] = s / R[(size_t)j * m + j];
  }
  if (chi2) {
    double r2 = 0.0;
    for (int k = m; k < n; ++k) r2 += y[k] * y[k];
    *chi2 = r2;
  }
  if (cov) {
    // cov = R^-1 R^-T
    std::vector<double> Ri((size_t)m * m, 0.0);
    for (int c = 0; c < m; ++c) {
      for (int j = m - 1; j >= 0; --j) {
        double s = (j == c) ? 1.0 : 0.0;
        for (int q = j + 1; q < m; ++q) s -= R[(size_t)j * m + q] * Ri[(size_t)q * m + c];
        Ri[(size_t)j * m + c] = s / R[(size_t)j * m + j];
      }
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += Ri[(size_t)i * m + q] * Ri[(size_t)j * m + q];
        cov[(size_t)i * m + j] = s;
      }
  }
  return LRDMC_OK;
}

lrdmc_status lrdmc_history(lrdmc_handle h, int cap, int* n, double* wbar, double* ebar, double* e0,
                           double* moves_mean, int* moves_max, int* survivors, uint32_t* status_or) {
  if (!h) return LRDMC_ERR_ARG;
  const int m = (int)h->wbar.size();
  if (n) *n = m;
  const int k = std::min(std::max(cap, 0), m);
  for (int i = 0; i < k; ++i) {
    if (wbar) wbar[i] = h->wbar[i];
    if (ebar) ebar[i] = h->ebar[i];
    if (e0) e0[i] = h->e0h[i];
    if (moves_mean) moves_mean[i] = h->mmean[i];
    if (moves_max) moves_max[i] = h->mmax[i];
    if (survivors) survivors[i] = h->surv[i];
    if (status_or) status_or[i] = h->stor[i];
  }
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_e0(lrdmc_handle h, double* e0) {
  if (!h || !e0) return LRDMC_ERR_ARG;
  *e0 = h->E0;
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_e0(lrdmc_handle h, double e0) {
  if (!h || !std::isfinite(e0)) return LRDMC_ERR_ARG;
  h->E0 = e0;
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_walkers(lrdmc_handle h, double* x, double* w, double* ev, double* ratios, uint32_t* status,
                               int32_t* moves) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  return fetch(h, x, w, ev, ratios, status, moves);
}

lrdmc_status lrdmc_set_walkers(lrdmc_handle h, const double* x, const double* w) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  if (!x) return fail(h, LRDMC_ERR_ARG, "x is NULL");
  DeviceGuard g(h->device);
  return place_walkers(h, x, w);
}

lrdmc_status lrdmc_clear_status(lrdmc_handle h) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  k_set_scalar<<<std::max(1, std::min(1024, (h->P.n_w + 255) / 256)), 256, 0, h->stream>>>(h->P.L, h->state,
                                                                                           h->P.n_w, SC_STATUS, 0.0);
  LAUNCHED(h);
  return LRDMC_OK;
}

namespace {
constexpr uint64_t CKPT_MAGIC = 0x4c52444d43434b32ull;   // "LRDMCCK2"

struct CkptHeader {
  uint64_t magic;
  int32_t n_w, n_e, g_stride, precision, n_hist, c_stride;
  uint64_t seed;
  double a, E0;
  uint32_t interval, last_kind;
  int32_t node_rule, n_up;
  uint64_t fingerprint;   // FNV-1a of the system image and the pair Jastrow parameters
};
// Bytes of one branching-history record in the file (wbar, ebar, E0, mean
// moves, max moves, survivors, stored slots).
constexpr size_t CKPT_HIST_BYTES = 4 * sizeof(double) + 2 * sizeof(int) + sizeof(uint32_t);

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t k = 0; k < n; ++k) { h ^= c[k]; h *= 0x100000001b3ull; }
  return h;
}

// Fingerprint of what the cached walker evaluations depend on besides a and
// the node rule: nuclei, potentials, basis, orbitals and every Jastrow
// parameter (the system image holds all but the pair Jastrow constants).
uint64_t system_fingerprint(lrdmc_handle h) {
  uint64_t f = fnv1a(0xcbf29ce484222325ull, h->img.data(), h->img.size());
  const double j2[3] = {h->S.j2_anti, h->S.j2_par, h->S.j2_b};
  return fnv1a(f, j2, sizeof j2);
}
}  // namespace

lrdmc_status lrdmc_save(lrdmc_handle h, const char* path) {
  if (!h || !h->state || !path) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  const Plan& P = h->P;
  std::vector<double> st((size_t)P.n_w * P.L.g_stride), cs((size_t)P.n_w * P.L.c_stride);
  CK(h, cudaMemcpyAsync(st.data(), h->state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, h->stream));
  if (!cs.empty())
    CK(h, cudaMemcpyAsync(cs.data(), h->cache, sizeof(double) * cs.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CkptHeader hd{};
  hd.magic = CKPT_MAGIC;
  hd.n_w = P.n_w; hd.n_e = P.n_e; hd.g_stride = P.L.g_stride; hd.precision = P.precision;
  hd.c_stride = P.L.c_stride;
  hd.n_hist = (int32_t)h->wbar.size();
  hd.seed = h->prm.seed; hd.a = h->prm.a; hd.E0 = h->E0; hd.interval = h->interval; hd.last_kind = h->last_kind;
  hd.node_rule = h->prm.node_rule; hd.n_up = P.n_up;
  hd.fingerprint = system_fingerprint(h);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(h, LRDMC_ERR_ARG, std::string("cannot open ") + path);
  bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(st.data(), sizeof(double), st.size(), f) == st.size() &&
            fwrite(cs.data(), sizeof(double), cs.size(), f) == cs.size();
  const size_t m = h->wbar.size();
  if (m) {
    ok = ok && fwrite(h->wbar.data(), sizeof(double), m, f) == m && fwrite(h->ebar.data(), sizeof(double), m, f) == m &&
         fwrite(h->e0h.data(), sizeof(double), m, f) == m && fwrite(h->mmean.data(), sizeof(double), m, f) == m &&
         fwrite(h->mmax.data(), sizeof(int), m, f) == m && fwrite(h->surv.data(), sizeof(int), m, f) == m &&
         fwrite(h->stor.data(), sizeof(uint32_t), m, f) == m;
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? LRDMC_OK : fail(h, LRDMC_ERR_ARG, "checkpoint write failed");
}

lrdmc_status lrdmc_load(lrdmc_handle h, const char* path) {
  if (!h || !h->state || !path) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  const Plan& P = h->P;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(h, LRDMC_ERR_ARG, std::string("cannot open ") + path);
  CkptHeader hd{};
  bool ok = fread(&hd, sizeof hd, 1, f) == 1;
  if (!ok || hd.magic != CKPT_MAGIC || hd.n_w != P.n_w || hd.n_e != P.n_e || hd.n_up != P.n_up ||
      hd.g_stride != P.L.g_stride || hd.c_stride != P.L.c_stride || hd.precision != P.precision ||
      hd.n_hist < 0) {
    fclose(f);
    return fail(h, LRDMC_ERR_ARG, "checkpoint does not match this handle's layout");
  }
  // the cached ratios, W and e_L of every walker belong to one Hamiltonian:
  // refuse a checkpoint of another lattice spacing, node rule, system or
  // trial function
  if (memcmp(&hd.a, &h->prm.a, sizeof(double)) != 0 || hd.node_rule != h->prm.node_rule ||
      hd.fingerprint != system_fingerprint(h)) {
    fclose(f);
    return fail(h, LRDMC_ERR_ARG, "checkpoint was written for another lattice spacing, node rule, system or "
                                  "trial wavefunction");
  }
  const size_t nst = (size_t)P.n_w * P.L.g_stride, ncs = (size_t)P.n_w * P.L.c_stride;
  const size_t m = (size_t)hd.n_hist;
  {
    // the history length must agree with the file's size before it sizes any buffer
    long here = ftell(f);
    if (here < 0 || fseek(f, 0, SEEK_END) != 0) { fclose(f); return fail(h, LRDMC_ERR_ARG, "checkpoint not seekable"); }
    const long end = ftell(f);
    if (end < here || fseek(f, here, SEEK_SET) != 0) { fclose(f); return fail(h, LRDMC_ERR_ARG, "checkpoint not seekable"); }
    const size_t rest = (size_t)(end - here), need = sizeof(double) * (nst + ncs);
    if (rest < need || (rest - need) != m * CKPT_HIST_BYTES) {
      fclose(f);
      return fail(h, LRDMC_ERR_ARG, "checkpoint size does not match its header");
    }
  }
  std::vector<double> st, cs, wb, eb, e0, mm;
  std::vector<int> mx, sv;
  std::vector<uint32_t> so;
  try {
    st.resize(nst); cs.resize(ncs);
    wb.resize(m); eb.resize(m); e0.resize(m); mm.resize(m); mx.resize(m); sv.resize(m); so.resize(m);
  } catch (const std::bad_alloc&) {
    fclose(f);
    return fail(h, LRDMC_ERR_ARG, "checkpoint too large for host memory");
  }
  ok = fread(st.data(), sizeof(double), st.size(), f) == st.size() &&
       fread(cs.data(), sizeof(double), cs.size(), f) == cs.size();
  if (m) {
    ok = ok && fread(wb.data(), sizeof(double), m, f) == m && fread(eb.data(), sizeof(double), m, f) == m &&
         fread(e0.data(), sizeof(double), m, f) == m && fread(mm.data(), sizeof(double), m, f) == m &&
         fread(mx.data(), sizeof(int), m, f) == m && fread(sv.data(), sizeof(int), m, f) == m &&
         fread(so.data(), sizeof(uint32_t), m, f) == m;
  }
  fclose(f);
  if (!ok) return fail(h, LRDMC_ERR_ARG, "checkpoint truncated");
  CK(h, cudaMemcpyAsync(h->state, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, h->stream));
  if (!cs.empty())
    CK(h, cudaMemcpyAsync(h->cache, cs.data(), sizeof(double) * cs.size(), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->prm.seed = hd.seed;
  h->E0 = hd.E0;
  h->interval = hd.interval;
  h->last_kind = (int)hd.last_kind;
  h->wbar = wb; h->ebar = eb; h->e0h = e0; h->mmean = mm; h->mmax = mx; h->surv = sv; h->stor = so;
  return LRDMC_OK;
}

lrdmc_status lrdmc_eval_configs(lrdmc_handle h, int n, const double* x, double* ratios, double* ev, int32_t* n_node) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  if (n < 0 || n > h->P.n_w) return fail(h, LRDMC_ERR_ARG, "n must be in [0, n_w]");
  if (n == 0) return LRDMC_OK;
  if (!x || !ratios || !ev) return fail(h, LRDMC_ERR_ARG, "NULL device pointer");
  DeviceGuard g(h->device);
  const int smem = smem_bytes(h);
  if (h->P.precision == 0)
    k_eval_configs<<<walker_grid(h, n), h->wpb * 32, smem, h->stream>>>(h->S, h->P.L, h->alt, x, n, h->prm.a,
                                                                        h->prm.node_rule, ratios, ev, n_node, h->scr);
  else
    k_eval_configs_m<<<walker_grid(h, n), h->wpb * 32, smem, h->stream>>>(h->S, h->P.L, h->P.M, h->alt, x, n,
                                                                          h->prm.a, h->prm.node_rule, ratios, ev,
                                                                          n_node, h->scr);
  LAUNCHED(h);
  return LRDMC_OK;
}

size_t lrdmc_reconfigure_scratch_bytes(int n) {
  if (n < 1) return 0;
  return align_up(sizeof(unsigned long long) * (size_t)n) + ALIGN;
}

lrdmc_status lrdmc_reconfigure_indices(int n, const double* w, uint32_t xi32, int32_t* src, void* scratch,
                                       size_t scratch_bytes, int32_t* status_out, void* stream) {
  if (n < 1 || n > MAX_WALKERS || !w || !src || !scratch) return LRDMC_ERR_ARG;
  if (scratch_bytes < lrdmc_reconfigure_scratch_bytes(n) || (uintptr_t)scratch % ALIGN) return LRDMC_ERR_ARG;
  unsigned long long* Q = (unsigned long long*)scratch;
  int32_t* st = (int32_t*)((char*)scratch + align_up(sizeof(unsigned long long) * (size_t)n));
  k_reconfigure<<<1, BR_THREADS, 0, (cudaStream_t)stream>>>(w, 1, n, xi32, Q, src, st, nullptr, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return LRDMC_ERR_CUDA;
  if (status_out) {
    e = cudaMemcpyAsync(status_out, st, 2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return LRDMC_ERR_CUDA;
  }
  return LRDMC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free reconfiguration indices.  Scratch lives in one file-scope
// device array (Q words followed by two status words); its device address is
// looked up once per device with cudaGetSymbolAddress.  The host-side symbol
// name is not a device address and is never passed to a kernel.
}  // extern "C"

namespace {
constexpr int NOALLOC_Q_WORDS = LRDMC_NOALLOC_MAX_WALKERS;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_Q_WORDS + 32];
constexpr int NOALLOC_MAX_DEVICES = 64;
std::atomic<unsigned long long*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;

// Device address of this device's scratch array (set up on first use).
cudaError_t noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  unsigned long long* p = g_noalloc_ptr[dev].load();
  if (!p) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    p = g_noalloc_ptr[dev].load();
    if (!p) {
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) return e;
      p = (unsigned long long*)addr;
      g_noalloc_ptr[dev].store(p);
    }
  }
  *out = p;
  return cudaSuccess;
}
}  // namespace

extern "C" {

lrdmc_status lrdmc_reconfigure_indices_noalloc(int n, const double* w, uint32_t xi32, int32_t* src,
                                               int32_t* status_out, void* stream) {
  if (n > LRDMC_NOALLOC_MAX_WALKERS) return LRDMC_ERR_UNSUPPORTED;
  if (n < 1 || !w || !src) return LRDMC_ERR_ARG;
  unsigned long long* q = nullptr;
  if (noalloc_scratch(&q) != cudaSuccess) return LRDMC_ERR_CUDA;
  int32_t* st = (int32_t*)(q + NOALLOC_Q_WORDS);
  k_reconfigure<<<1, BR_THREADS, 0, (cudaStream_t)stream>>>(w, 1, n, xi32, q, src, st, nullptr, 0);
  if (cudaGetLastError() != cudaSuccess) return LRDMC_ERR_CUDA;
  if (status_out &&
      cudaMemcpyAsync(status_out, st, 2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream) !=
          cudaSuccess)
    return LRDMC_ERR_CUDA;
  return LRDMC_OK;
}

}  // extern "C"

namespace {
// Per-device constant table of a testing aid, built on the device's first
// call.  The table pointer is published (under a lock) only after its copy
// succeeded, so a failed set-up leaves no pointer to uninitialised memory and
// the next call tries again.
std::mutex g_tab_mutex;
cudaError_t device_table(double* (&slot)[64], const std::vector<double>& host, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  if (!slot[dev]) {
    double* d = nullptr;
    e = cudaMalloc(&d, sizeof(double) * host.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return e;
    }
    slot[dev] = d;
  }
  *out = slot[dev];
  return cudaSuccess;
}
double* g_exp_tab[64] = {nullptr};
double* g_erf_tab[64] = {nullptr};
}  // namespace

extern "C" {

lrdmc_status lrdmc_fp64math(int n, const double* x, double* exp_out, double* rcp_out, double* rsqrt_out,
                            void* stream) {
  if (n < 0 || (n > 0 && !x)) return LRDMC_ERR_ARG;
  if (n == 0) return LRDMC_OK;
  std::vector<double> tab(EXP_TAB);
  for (int j = 0; j < EXP_TAB; ++j) tab[j] = (double)exp2l((long double)j / EXP_TAB);
  double* d_tab = nullptr;
  if (device_table(g_exp_tab, tab, &d_tab) != cudaSuccess) return LRDMC_ERR_CUDA;
  k_fp64math<<<std::min(1024, (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, x, exp_out, rcp_out, rsqrt_out,
                                                                                d_tab);
  return cudaGetLastError() == cudaSuccess ? LRDMC_OK : LRDMC_ERR_CUDA;
}

lrdmc_status lrdmc_erf_ratio_table(double* out, int* n_int, int* n_coef) {
  if (n_int) *n_int = ERF_INT;
  if (n_coef) *n_coef = ERF_NC;
  if (out) erf_ratio_table(out);
  return LRDMC_OK;
}

lrdmc_status lrdmc_erf_over_r(int n, const double* s, double r_c, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!s || !out)) || !(r_c > 0.0)) return LRDMC_ERR_ARG;
  if (n == 0) return LRDMC_OK;
  std::vector<double> tab(ERF_INT * ERF_NC);
  erf_ratio_table(tab.data());
  double* d_tab = nullptr;
  if (device_table(g_erf_tab, tab, &d_tab) != cudaSuccess) return LRDMC_ERR_CUDA;
  const double irc2 = (double)(1.0L / ((long double)r_c * r_c));
  k_erf_over_r<<<std::min(1024, (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, s, 1.0 / r_c, irc2, out,
                                                                                  d_tab);
  return cudaGetLastError() == cudaSuccess ? LRDMC_OK : LRDMC_ERR_CUDA;
}

lrdmc_status lrdmc_param_count(lrdmc_handle h, int* n) {
  if (!h || !n) return LRDMC_ERR_ARG;
  *n = param_count(h->P.n_nuc);
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_params(lrdmc_handle h, double* theta) {
  if (!h || !theta) return LRDMC_ERR_ARG;
  const int nn = h->P.n_nuc;
  for (int k = 0; k < 3 * nn; ++k) theta[k] = h->hR[k];
  theta[3 * nn] = h->S.j2_anti;
  theta[3 * nn + 1] = h->S.j2_par;
  theta[3 * nn + 2] = h->S.j2_b;
  for (int I = 0; I < nn; ++I) {
    theta[3 * nn + 3 + I] = h->hA[I];
    theta[4 * nn + 3 + I] = h->hB[I];
  }
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_params(lrdmc_handle h, const double* theta) {
  if (!h || !h->state || !theta) return LRDMC_ERR_ARG;
  const Plan& P = h->P;
  const int nn = P.n_nuc;
  for (int k = 0; k < param_count(nn); ++k)
    if (!std::isfinite(theta[k])) return fail(h, LRDMC_ERR_ARG, "non-finite parameter");
  DeviceGuard g(h->device);
  std::vector<double> x((size_t)P.n_w * 3 * P.n_e), w(P.n_w);
  {
    lrdmc_status st = fetch(h, x.data(), w.data(), nullptr, nullptr, nullptr, nullptr);   // synchronises
    if (st != LRDMC_OK) return st;
  }
  h->hR.assign(theta, theta + 3 * nn);
  h->S.j2_anti = theta[3 * nn];
  h->S.j2_par = theta[3 * nn + 1];
  h->S.j2_b = theta[3 * nn + 2];
  h->S.j2_antif = (float)h->S.j2_anti;
  h->S.j2_parf = (float)h->S.j2_par;
  h->S.j2_bf = (float)h->S.j2_b;
  h->hA.assign(theta + 3 * nn + 3, theta + 4 * nn + 3);
  h->hB.assign(theta + 4 * nn + 3, theta + 5 * nn + 3);
  std::vector<float> fR(3 * nn), fA(nn), fB(nn);
  for (int k = 0; k < 3 * nn; ++k) fR[k] = (float)h->hR[k];
  for (int I = 0; I < nn; ++I) { fA[I] = (float)h->hA[I]; fB[I] = (float)h->hB[I]; }
  char* dsys = (char*)h->ws + P.o_sys;
  memcpy(h->img.data() + P.i_R, h->hR.data(), sizeof(double) * 3 * nn);
  memcpy(h->img.data() + P.i_j1A, h->hA.data(), sizeof(double) * nn);
  memcpy(h->img.data() + P.i_j1B, h->hB.data(), sizeof(double) * nn);
  memcpy(h->img.data() + P.i_f_R, fR.data(), sizeof(float) * 3 * nn);
  memcpy(h->img.data() + P.i_f_j1A, fA.data(), sizeof(float) * nn);
  memcpy(h->img.data() + P.i_f_j1B, fB.data(), sizeof(float) * nn);
  CK(h, cudaMemcpyAsync(dsys + P.i_R, h->hR.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dsys + P.i_j1A, h->hA.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dsys + P.i_j1B, h->hB.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dsys + P.i_f_R, fR.data(), sizeof(float) * 3 * nn, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dsys + P.i_f_j1A, fA.data(), sizeof(float) * nn, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dsys + P.i_f_j1B, fB.data(), sizeof(float) * nn, cudaMemcpyHostToDevice, h->stream));
  double vii = 0.0;
  for (int I = 0; I < nn; ++I)
    for (int J = I + 1; J < nn; ++J) {
      const double dx = h->hR[3 * I] - h->hR[3 * J], dy = h->hR[3 * I + 1] - h->hR[3 * J + 1],
                   dz = h->hR[3 * I + 2] - h->hR[3 * J + 2];
      vii += h->hZ[I] * h->hZ[J] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
  h->S.v_ii = vii;
  CK(h, cudaStreamSynchronize(h->stream));
  return place_walkers(h, x.data(), w.data());
}

lrdmc_status lrdmc_local_energy_grad(lrdmc_handle h, int n, const double* x, double* eL, double* logpsi,
                                     double* grad_eL, double* grad_logpsi) {
  if (!h || !h->state) return LRDMC_ERR_ARG;
  if (h->P.precision != 0) return fail(h, LRDMC_ERR_UNSUPPORTED, "gradients are implemented for precision 0");
  if (n < 0) return fail(h, LRDMC_ERR_ARG, "n < 0");
  if (n == 0) return LRDMC_OK;
  if (!x) return fail(h, LRDMC_ERR_ARG, "NULL device pointer");
  DeviceGuard g(h->device);
  const Plan& P = h->P;
  if (!h->gscr) {
    h->gscr_per_warp = (adj_scratch_doubles(P.L, P.n_shell) + 1) / 2 * 2;
    if (h->sm_warps < ADJ_MIN_WARPS) {
      // fewer than ADJ_MIN_WARPS shared-memory working sets per SM: working
      // sets in global memory, as many warps as the registers allow
      int bps = 0;
      h->adj_wpb = 4;
      CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_eloc_grad<true>, h->adj_wpb * 32,
                                                          EXP_TAB * sizeof(double)));
      if (bps < 1) return fail(h, LRDMC_ERR_UNSUPPORTED, "gradient kernel does not fit an SM");
      h->adj_grid = bps * h->num_sms;
      const size_t nw = (size_t)h->adj_grid * h->adj_wpb;
      // the kernel addresses working sets at slot * s_stride and scratch at
      // slot * scratch_doubles
      CK(h, cudaMalloc(&h->adj_gsm, sizeof(double) * nw * ((size_t)P.L.s_stride + scratch_doubles(P.L, P.n_nuc))));
      h->adj_scr = h->adj_gsm + nw * (size_t)P.L.s_stride;
    } else {
      h->adj_grid = h->grid;
      h->adj_wpb = h->wpb;
    }
    const size_t nw = (size_t)h->adj_grid * h->adj_wpb;
    CK(h, cudaMalloc(&h->adj_blk, sizeof(double) * nw * (size_t)P.L.g_stride));
    CK(h, cudaMalloc(&h->gscr, sizeof(double) * h->gscr_per_warp * nw));
  }
  // one launch; each warp evaluates its configurations in its own walker block
  const int grid = std::max(1, std::min(h->adj_grid, (n + h->adj_wpb - 1) / h->adj_wpb));
  if (h->adj_gsm)
    k_eloc_grad<true><<<grid, h->adj_wpb * 32, EXP_TAB * sizeof(double), h->stream>>>(
        h->S, P.L, h->adj_blk, x, n, h->prm.a, h->prm.node_rule, h->adj_scr, h->gscr, h->gscr_per_warp, eL, logpsi,
        grad_eL, grad_logpsi, h->adj_gsm);
  else
    k_eloc_grad<false><<<grid, h->adj_wpb * 32, smem_bytes(h), h->stream>>>(
        h->S, P.L, h->adj_blk, x, n, h->prm.a, h->prm.node_rule, h->scr, h->gscr, h->gscr_per_warp, eL, logpsi,
        grad_eL, grad_logpsi, nullptr);
  LAUNCHED(h);
  return LRDMC_OK;
}

lrdmc_status lrdmc_weighted_rows(lrdmc_handle h, int n, int m, const double* rows, const double* w, double* out) {
  if (!h || n < 0 || m < 1 || !rows || !w || !out) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  k_weighted_rows<<<std::max(1, std::min(1024, (m + 255) / 256)), 256, 0, h->stream>>>(n, m, rows, w, out);
  LAUNCHED(h);
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_timing(lrdmc_handle h, int enable) {
  if (!h) return LRDMC_ERR_ARG;
  h->timing = enable != 0;
  return LRDMC_OK;
}

lrdmc_status lrdmc_interval_timing(lrdmc_handle h, double out[6]) {
  if (!h || !out || !h->state) return LRDMC_ERR_ARG;
  if (!h->timing) return fail(h, LRDMC_ERR_ARG, "timing is not enabled");
  DeviceGuard g(h->device);
  const int n = h->P.n_w;
  std::vector<unsigned long long> st(3 * (size_t)n);
  CK(h, cudaMemcpyAsync(st.data(), h->stamps, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost,
                        h->stream));
  std::vector<int32_t> mvs(n);
  lrdmc_status s = fetch(h, nullptr, nullptr, nullptr, nullptr, nullptr, mvs.data());   // synchronises
  if (s != LRDMC_OK) return s;
  unsigned long long t0 = ~0ull, t1 = 0;
  double sum = 0.0, mx = 0.0;
  for (int a = 0; a < n; ++a) {
    t0 = std::min(t0, st[3 * a]);
    t1 = std::max(t1, st[3 * a + 1]);
    const double d = (double)(st[3 * a + 1] - st[3 * a]) * 1e-6;
    sum += d;
    mx = std::max(mx, d);
  }
  const double span = (double)(t1 - t0) * 1e-6;
  const int resident = std::min(n, h->prop_grid * h->prop_wpb);
  double mv = 0.0, mvmax = 0.0;
  for (int a = 0; a < n; ++a) {
    const double m = mvs[a];
    mv += m;
    mvmax = std::max(mvmax, m);
  }
  out[0] = span;
  out[1] = sum / n;
  out[2] = mx;
  out[3] = span > 0 ? sum / (span * resident) : 0.0;
  out[4] = mv / n;
  out[5] = mvmax;
  return LRDMC_OK;
}

}  // extern "C"

namespace {
#ifdef LRDMC_CHECKED
__device__ int g_chk_selftest_out;
// Testing aid of the checked build: one thread evaluates CHK(i, n).
__global__ void k_check_selftest(int i, int n) { g_chk_selftest_out = CHK(i, n); }
#endif
}  // namespace

extern "C" {

int lrdmc_checked_build(void) {
#ifdef LRDMC_CHECKED
  return 1;
#else
  return 0;
#endif
}

lrdmc_status lrdmc_check_word(uint64_t* word, int clear) {
#ifdef LRDMC_CHECKED
  if (!word) return LRDMC_ERR_ARG;
  unsigned long long v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return LRDMC_ERR_CUDA;
  if (cudaMemcpyFromSymbol(&v, g_lrdmc_check, sizeof v) != cudaSuccess) return LRDMC_ERR_CUDA;
  *word = v;
  if (clear) {
    const unsigned long long z = 0;
    if (cudaMemcpyToSymbol(g_lrdmc_check, &z, sizeof z) != cudaSuccess) return LRDMC_ERR_CUDA;
  }
  return LRDMC_OK;
#else
  (void)word;
  (void)clear;
  return LRDMC_ERR_UNSUPPORTED;
#endif
}

lrdmc_status lrdmc_check_selftest(int i, int n, int* result) {
#ifdef LRDMC_CHECKED
  if (!result) return LRDMC_ERR_ARG;
  k_check_selftest<<<1, 1>>>(i, n);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return LRDMC_ERR_CUDA;
  if (cudaMemcpyFromSymbol(result, g_chk_selftest_out, sizeof(int)) != cudaSuccess) return LRDMC_ERR_CUDA;
  return LRDMC_OK;
#else
  (void)i;
  (void)n;
  (void)result;
  return LRDMC_ERR_UNSUPPORTED;
#endif
}

lrdmc_status lrdmc_set_drift_tol(lrdmc_handle h, double tol) {
  if (!h || !(tol >= 0.0)) return LRDMC_ERR_ARG;
  h->drift_tol = tol;
  return LRDMC_OK;
}

lrdmc_status lrdmc_drift_reinversions(lrdmc_handle h, int64_t* n) {
  if (!h || !h->dstat || !n) return LRDMC_ERR_ARG;
  DeviceGuard g(h->device);
  int32_t v = 0;
  CK(h, cudaMemcpyAsync(&v, h->dstat + DSTAT_DRIFT, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  *n = v;
  return LRDMC_OK;
}

lrdmc_status lrdmc_launch_count(lrdmc_handle h, int64_t* n) {
  if (!h || !n) return LRDMC_ERR_ARG;
  *n = h->launches;
  return LRDMC_OK;
}

lrdmc_status lrdmc_stream(lrdmc_handle h, void** stream) {
  if (!h || !stream) return LRDMC_ERR_ARG;
  *stream = (void*)h->stream;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_create(int n_sys, const lrdmc_system* sys, const lrdmc_trial_wf* wf,
                                const lrdmc_params* prm, const double* const* x0, void* stream, lrdmc_batch* out) {
  if (!out) return LRDMC_ERR_ARG;
  *out = nullptr;
  if (n_sys < 1 || !sys || !wf || !prm || !x0) return LRDMC_ERR_ARG;
  for (int k = 1; k < n_sys; ++k)
    if (prm[k].precision != prm[0].precision) return LRDMC_ERR_ARG;
  lrdmc_batch b = new lrdmc_batch_s();
  *out = b;   // kept on failure so that the caller can read the message; destroy frees it
  b->stream = (cudaStream_t)stream;
  b->precision = prm[0].precision;
  BCK(b, cudaGetDevice(&b->device));
  BCK(b, cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
  BCK(b, cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  for (int k = 0; k < n_sys; ++k) {
    lrdmc_handle h = nullptr;
    const lrdmc_status st = lrdmc_create(&sys[k], &wf[k], &prm[k], x0[k], nullptr, 0, stream, &h);
    if (st != LRDMC_OK) {
      const std::string msg = "system " + std::to_string(k) + ": " + (h ? h->err : std::string("create failed"));
      if (h) lrdmc_destroy(h);
      return bfail(b, st, msg);
    }
    b->h.push_back(h);
    const Plan& P = h->P;
    b->total += P.n_w;
    b->scratch_per_warp =
        std::max(b->scratch_per_warp, P.precision == 0 ? scratch_doubles(P.L, P.n_nuc) : scratch_doubles_m(P.L, P.M));
  }
  b->scratch_per_warp = (b->scratch_per_warp + 1) / 2 * 2;
  BCK(b, cudaFuncSetAttribute(k_propagate_batch<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batch_candidate(b, 0)));
  BCK(b, cudaFuncSetAttribute(k_propagate_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batch_candidate(b, 0)));
  cudaFuncAttributes fa{};
  if (b->precision == 0) BCK(b, cudaFuncGetAttributes(&fa, k_propagate_batch<0>));
  else BCK(b, cudaFuncGetAttributes(&fa, k_propagate_batch<1>));
  b->max_threads = fa.maxThreadsPerBlock;
  // scratch for the largest grid x warps of any candidate shape; default shape:
  // the candidate with the most resident warps
  int best = -1, best_warps = 0;
  for (int c = 0; c < 4; ++c) {
    bool ok = false;
    std::vector<int> fit;
    int w = 0, bps = 0;
    lrdmc_status st = batch_shape(b, batch_candidate(b, c), &ok, fit, &w, &bps);
    if (st != LRDMC_OK) return st;
    if (!ok) continue;
    b->scratch_warps = std::max(b->scratch_warps, (size_t)bps * b->num_sms * w);
    if (bps * w > best_warps) { best_warps = bps * w; best = c; }
  }
  if (best < 0) return bfail(b, LRDMC_ERR_UNSUPPORTED, "largest system exceeds a CTA's shared memory");
  b->jobs.resize(n_sys);
  b->bjobs.resize(n_sys);
  BCK(b, cudaMalloc(&b->d_jobs, sizeof(PropJob) * n_sys));
  BCK(b, cudaMalloc(&b->d_bjobs, sizeof(BranchJob) * n_sys));
  BCK(b, cudaMalloc(&b->d_items, sizeof(int4) * (size_t)b->total));
  BCK(b, cudaMalloc(&b->d_counter, sizeof(unsigned)));
  BCK(b, cudaMalloc(&b->d_scratch, sizeof(double) * b->scratch_per_warp * b->scratch_warps));
  BCK(b, cudaMalloc(&b->d_stats, sizeof(double) * BS_COUNT * n_sys));
  BCK(b, cudaMalloc(&b->d_status, sizeof(int32_t) * 2 * n_sys));
  BCK(b, cudaMemsetAsync(b->d_status, 0, sizeof(int32_t) * 2 * n_sys, b->stream));
  return batch_use(b, batch_candidate(b, best));
}

lrdmc_status lrdmc_batch_destroy(lrdmc_batch b) {
  if (!b) return LRDMC_ERR_ARG;
  {
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    batch_free(b);
  }
  delete b;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_handle(lrdmc_batch b, int k, lrdmc_handle* h) {
  if (!b || !h || k < 0 || k >= (int)b->h.size()) return LRDMC_ERR_ARG;
  *h = b->h[k];
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_propagate(lrdmc_batch b, const lrdmc_schedule* sch) {
  if (!b || b->h.empty()) return LRDMC_ERR_ARG;
  if (const char* bad = check_schedule(sch)) return bfail(b, LRDMC_ERR_ARG, bad);
  if (sch->rotate) return bfail(b, LRDMC_ERR_UNSUPPORTED, "the randomised lattice is not batched");
  DeviceGuard g(b->device);
  return batch_launch(b, sch);
}

lrdmc_status lrdmc_batch_branch(lrdmc_batch b) {
  if (!b || b->h.empty()) return LRDMC_ERR_ARG;
  DeviceGuard g(b->device);
  const int n = (int)b->h.size();
  size_t most = 1;
  for (int k = 0; k < n; ++k) {
    lrdmc_handle h = b->h[k];
    const Plan& P = h->P;
    BranchJob& J = b->bjobs[k];
    J.L = P.L;
    J.state = h->state;
    J.alt = h->state;           // in place: only unselected slots receive a copy
    J.cache = h->cache;
    J.cache_alt = h->cache;
    J.n_w = P.n_w;
    J.lb = h->last_kind == LRDMC_LOAD_BALANCED;
    J.E0 = h->E0;
    J.xi32 = branch_offset32(h->prm.seed, h->interval);
    J.Q = h->Q;
    J.src = h->src;
    J.status = b->d_status + 2 * k;
    J.stats = b->d_stats + (size_t)BS_COUNT * k;
    most = std::max(most, (size_t)P.n_w * std::max(P.L.g_stride, P.L.c_stride) / 2);
  }
  BCK(b, cudaMemcpyAsync(b->d_bjobs, b->bjobs.data(), sizeof(BranchJob) * n, cudaMemcpyHostToDevice, b->stream));
  k_branch_reduce_batch<<<n, BR_THREADS, 0, b->stream>>>(b->d_bjobs);
  BLAUNCHED(b);
  k_reconfigure_batch<<<n, BR_THREADS, 0, b->stream>>>(b->d_bjobs);
  BLAUNCHED(b);
  const int gx = (int)std::max<size_t>(1, std::min<size_t>((most + 255) / 256, (size_t)b->num_sms * 8));
  k_gather_batch<<<dim3(gx, n), 256, 0, b->stream>>>(b->d_bjobs);
  BLAUNCHED(b);
  std::vector<double> hs((size_t)BS_COUNT * n);
  BCK(b, cudaMemcpyAsync(hs.data(), b->d_stats, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  lrdmc_status worst = LRDMC_OK;
  std::string msg;
  for (int k = 0; k < n; ++k) {
    const lrdmc_status st = finish_branch(b->h[k], hs.data() + (size_t)BS_COUNT * k, false);
    if (st != LRDMC_OK) {
      if (worst == LRDMC_OK) worst = st;
      msg += "system " + std::to_string(k) + ": " + b->h[k]->err + "; ";
    }
  }
  if (worst != LRDMC_OK) return bfail(b, worst, msg);
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_set_order(lrdmc_batch b, int policy) {
  if (!b || (policy != 0 && policy != 1)) return LRDMC_ERR_ARG;
  DeviceGuard g(b->device);
  b->policy = policy;
  return batch_items(b);
}

lrdmc_status lrdmc_batch_tune(lrdmc_batch b, const lrdmc_schedule* sch, double times_ms[4], int* best_ctas) {
  if (!b || b->h.empty()) return LRDMC_ERR_ARG;
  if (const char* bad = check_schedule(sch)) return bfail(b, LRDMC_ERR_ARG, bad);
  if (sch->rotate) return bfail(b, LRDMC_ERR_UNSUPPORTED, "the randomised lattice is not batched");
  DeviceGuard g(b->device);
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 1e30f;
  lrdmc_status st = LRDMC_OK;
  for (int c = 0; c < 4 && st == LRDMC_OK; ++c) {
    if (times_ms) times_ms[c] = 0.0;
    bool ok = false;
    std::vector<int> fit;
    int w = 0, bps = 0;
    st = batch_shape(b, batch_candidate(b, c), &ok, fit, &w, &bps);
    if (st != LRDMC_OK || !ok) continue;
    st = batch_use(b, batch_candidate(b, c));
    if (st != LRDMC_OK) break;
    // keep every walker (and its caches) to restore after the trial
    for (lrdmc_handle h : b->h) {
      if (cudaMemcpyAsync(h->alt, h->state, h->P.state_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
          cudaMemcpyAsync(h->cache_alt, h->cache, h->P.cache_bytes, cudaMemcpyDeviceToDevice, b->stream) !=
              cudaSuccess) {
        st = bfail(b, LRDMC_ERR_CUDA, "snapshot copy failed");
        break;
      }
    }
    if (st != LRDMC_OK) break;
    cudaEventRecord(e0, b->stream);
    st = batch_launch(b, sch);
    cudaEventRecord(e1, b->stream);
    if (st != LRDMC_OK) break;
    for (lrdmc_handle h : b->h) {
      if (cudaMemcpyAsync(h->state, h->alt, h->P.state_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
          cudaMemcpyAsync(h->cache, h->cache_alt, h->P.cache_bytes, cudaMemcpyDeviceToDevice, b->stream) !=
              cudaSuccess) {
        st = bfail(b, LRDMC_ERR_CUDA, "restore copy failed");
        break;
      }
    }
    if (st != LRDMC_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = bfail(b, LRDMC_ERR_CUDA, "tuning launch failed"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (times_ms) times_ms[c] = ms;
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LRDMC_OK) return st;
  if (best < 0) return bfail(b, LRDMC_ERR_UNSUPPORTED, "no launch shape fits");
  if (best_ctas) *best_ctas = best + 1;
  return batch_use(b, batch_candidate(b, best));
}

lrdmc_status lrdmc_batch_set_timing(lrdmc_batch b, int enable) {
  if (!b) return LRDMC_ERR_ARG;
  b->timing = enable != 0;
  for (lrdmc_handle h : b->h) h->timing = b->timing;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_timing(lrdmc_batch b, double out[8]) {
  if (!b || !out || b->h.empty()) return LRDMC_ERR_ARG;
  if (!b->timing) return bfail(b, LRDMC_ERR_ARG, "timing is not enabled");
  DeviceGuard g(b->device);
  unsigned long long t0 = ~0ull, t1 = 0;
  double sum = 0.0, mx = 0.0;
  std::vector<std::vector<std::pair<unsigned long long, unsigned long long>>> per_sm(b->num_sms);
  double slot_busy = 0.0, slot_cap = 0.0;
  int n_items = 0;
  for (size_t k = 0; k < b->h.size(); ++k) {
    lrdmc_handle h = b->h[k];
    const int n = h->P.n_w;
    std::vector<unsigned long long> st(3 * (size_t)n);
    BCK(b, cudaMemcpyAsync(st.data(), h->stamps, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int a = 0; a < n; ++a) {
      t0 = std::min(t0, st[3 * a]);
      t1 = std::max(t1, st[3 * a + 1]);
      const double d = (double)(st[3 * a + 1] - st[3 * a]) * 1e-6;
      sum += d;
      mx = std::max(mx, d);
      const unsigned sm = (unsigned)st[3 * a + 2];
      if (sm < per_sm.size()) per_sm[sm].push_back({st[3 * a], st[3 * a + 1]});
    }
    // items of this system: fit[k] consecutive walkers run together in one CTA
    for (int w0 = 0; w0 < n; w0 += b->fit[k]) {
      const int c = std::min(b->fit[k], n - w0);
      unsigned long long s0 = ~0ull, s1 = 0;
      for (int a = w0; a < w0 + c; ++a) {
        s0 = std::min(s0, st[3 * a]);
        s1 = std::max(s1, st[3 * a + 1]);
        slot_busy += (double)(st[3 * a + 1] - st[3 * a]);
      }
      slot_cap += (double)c * (double)(s1 - s0);
      ++n_items;
    }
  }
  const double span = t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
  // per SM: time covered by at least one walker, and the idle tail after its last walker
  double covered = 0.0, tail = 0.0;
  for (auto& v : per_sm) {
    if (v.empty()) { tail += span; continue; }
    std::sort(v.begin(), v.end());
    unsigned long long cs = v[0].first, ce = v[0].second, busy = 0, last = 0;
    for (const auto& iv : v) {
      if (iv.first > ce) { busy += ce - cs; cs = iv.first; ce = iv.second; }
      else ce = std::max(ce, iv.second);
      last = std::max(last, iv.second);
    }
    busy += ce - cs;
    covered += (double)busy * 1e-6;
    tail += (double)(t1 - last) * 1e-6;
  }
  out[0] = span;
  out[1] = sum / b->total;
  out[2] = mx;
  out[3] = span > 0.0 ? 1.0 - covered / (span * per_sm.size()) : 0.0;
  out[4] = tail / per_sm.size();
  out[5] = slot_cap > 0.0 ? slot_busy / slot_cap : 0.0;
  out[6] = b->total;
  out[7] = n_items;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_launch_count(lrdmc_batch b, int64_t* n) {
  if (!b || !n) return LRDMC_ERR_ARG;
  *n = b->launches;
  return LRDMC_OK;
}

const char* lrdmc_batch_last_error(lrdmc_batch b) { return b ? b->err.c_str() : "NULL batch"; }

}  // extern "C"
