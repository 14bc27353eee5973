// Warp-per-walker FP64 kernels of the LRDMC projection step.
//
// One warp owns one walker at a time.  Its working set (positions, the
// transposed inverse Slater matrices B^T, the 6 N_e hop ratios and their
// determinant / Jastrow parts, per-electron Jastrow / potential terms and the
// electron-nucleus / electron-electron geometry of the current configuration)
// lives in shared memory for a whole branching interval (in global memory for
// systems too large for that).  The walker's cache block in global memory
// keeps, across intervals, the orbital value/gradient/Laplacian rows of every
// electron, g_i = C^T B[:, i], the basis values at every hop and the pair
// Jastrow terms of every hop and of every pair.  The FP64 pipe is the bound,
// so the formulation minimises FP64 work:
//   * determinant ratio of hop (i, d) = chi(r') . g_i (one N_bf dot per hop);
//     g is updated by the same rank-1 factors as B after each hop;
//   * every hop re-evaluates only what depends on the moved electron; the
//     other electrons' pair terms with it are swapped from the caches;
//   * |r' - R|^2 = (|r - R|^2 + a^2) + 2 (+-a) (r - R)_axis: distances are
//     formed once per (electron, nucleus) and per electron pair and shared by
//     the 6 hops and all shells on a nucleus;
//   * the pseudopotential of an electron is recomputed only when it hops;
//   * Sherman-Morrison keeps B = A^{-1} current, with a from-scratch
//     Gauss-Jordan inversion every reinv_period hops;
//   * exp / rsqrt / reciprocal / erf(r/r_c)/r use the reduced-slot forms of
//     fp64math.cuh.
#pragma once

#include "common.cuh"
#include "fp64math.cuh"

namespace lrdmc {

// ------------------------------------------------------------ basis functions
// Value, gradient and Laplacian of the functions of shell s at offset d from
// its nucleus (r2 = |d|^2): out[c * n_bf + mu], c = 0 value, 1..3 gradient,
// 4 Laplacian.
__device__ __forceinline__ void shell_derivs(const DevSys& S, int s, const double d[3], double r2,
                                             double* __restrict__ out, int n_bf, const double* T) {
  const int l = __ldg(S.sh_l + s);
  const int np = __ldg(S.sh_nprim + s);
  const int off = __ldg(S.sh_off + s);
  const int bf = CHK(__ldg(S.sh_bf + s), n_bf);
  // h = c exp(-z r) for the Slater 1s kind, c exp(-a r^2) for Gaussians;
  // s0 = sum h, s1 = sum c1 h, s2 = sum c2 h with
  //   Slater: c1 = -z, c2 = z^2 - 2 z / r           (h' and lap h)
  //   s:      c1 = -2a, c2 = 4 a^2 r^2 - 6 a        (grad = c1 h d, lap h)
  //   p:      c1 = -2a, c2 = 4 a^2 r^2 - 10 a       (d_m times the radial part)
  // The Gaussian kinds share one primitive loop; the Slater kind has a loop of
  // its own, which a warp without Slater shells (the usual case) skips.
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (l == -1) {
    // Slater 1s (a branch of its own: a warp without Slater shells skips it)
    const double ir = rsqrt_nr(r2);
    const double r = r2 * ir;
    for (int q = 0; q < np; ++q) {
      const double z = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp_tab(-z * r, T);
      s0 += h;
      s1 = fma(-z, h, s1);
      s2 = fma(z * z - 2.0 * z * ir, h, s2);
    }
    s1 *= ir;   // grad = h' d / r
  } else {
    const double k6 = l == 1 ? 10.0 : 6.0;
    for (int q = 0; q < np; ++q) {
      const double z = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp_tab(-z * r2, T);
      s0 += h;
      s1 = fma(-2.0 * z, h, s1);
      s2 = fma(4.0 * z * z * r2 - k6 * z, h, s2);
    }
  }
  if (l != 1) {
    // s and Slater: grad = s1 d
    out[bf] = s0;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = s1 * d[m];
    out[4 * n_bf + bf] = s2;
  } else {
    // d_m h: grad_n = delta_mn h - 2a d_m d_n h, lap = d_m (4a^2 r^2 - 10 a) h;
    // with t_m = d_m s1 the gradient takes one operation per component
    for (int m = 0; m < 3; ++m) {
      const double t = d[m] * s1;
      out[bf + m] = d[m] * s0;
      for (int n = 0; n < 3; ++n) out[(1 + n) * n_bf + bf + m] = m == n ? fma(d[n], t, s0) : d[n] * t;
      out[4 * n_bf + bf + m] = d[m] * s2;
    }
  }
}

// Lanes per dot product when n_out dot products of length len are spread over
// a warp: S in {1, 2, 4, 8} lanes take consecutive slices of one dot and are
// combined by shuffles; chosen to minimise (warp passes) x (slice length) +
// (shuffle levels), the FP64 instruction count of the warp.
__device__ __forceinline__ int split_factor(int n_out, int len) {
  int best = 1, cost = 1 << 30;
  for (int c = 1, lv = 0; c <= 8; c <<= 1, ++lv) {
    const int k = ((n_out * c + WARP - 1) / WARP) * ((len + c - 1) / c) + lv;
    if (k < cost) { cost = k; best = c; }
  }
  return best;
}

// Warp sums of several values per lane by recursive halving: at each of the
// first levels a lane keeps half of its values, adds the partner's copy of that
// half and hands over the other half, so that k values cost k - 1 additions
// plus one per remaining level instead of k per level.
// warp_sum8: lane l returns the warp total of v[(l >> 2) & 7].
__device__ __forceinline__ double warp_sum8(const double v[8], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
  double w[4], u[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double keep = h4 ? v[j + 4] : v[j], give = h4 ? v[j] : v[j + 4];
    w[j] = keep + __shfl_xor_sync(FULL, give, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double keep = h3 ? w[j + 2] : w[j], give = h3 ? w[j] : w[j + 2];
    u[j] = keep + __shfl_xor_sync(FULL, give, 8);
  }
  double t = (h2 ? u[1] : u[0]) + __shfl_xor_sync(FULL, h2 ? u[0] : u[1], 4);
  t += __shfl_xor_sync(FULL, t, 2);
  t += __shfl_xor_sync(FULL, t, 1);
  return t;
}
// warp_sum4: lane l returns the warp total of v[(l >> 3) & 3].
__device__ __forceinline__ double warp_sum4(const double v[4], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8;
  double w[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double keep = h4 ? v[j + 2] : v[j], give = h4 ? v[j] : v[j + 2];
    w[j] = keep + __shfl_xor_sync(FULL, give, 16);
  }
  double t = (h3 ? w[1] : w[0]) + __shfl_xor_sync(FULL, h3 ? w[0] : w[1], 8);
  t += __shfl_xor_sync(FULL, t, 4);
  t += __shfl_xor_sync(FULL, t, 2);
  t += __shfl_xor_sync(FULL, t, 1);
  return t;
}

// Orbital value/gradient/Laplacian of the first n_sig orbitals at point q:
// phi5[c * n_max + k].  Warp-cooperative; chi5 is scratch of 5 n_bf doubles.
__device__ void orbital_derivs(const DevSys& S, const Layout& L, const double q[3], int n_sig, double* chi5,
                               double* phi5, const double* T, int lane) {
  for (int s = lane; s < S.n_shell; s += WARP) {
    const int atom = CHK(__ldg(S.sh_atom + s), S.n_nuc);
    const double d[3] = {q[0] - __ldg(S.R + 3 * atom), q[1] - __ldg(S.R + 3 * atom + 1),
                         q[2] - __ldg(S.R + 3 * atom + 2)};
    shell_derivs(S, s, d, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], chi5, L.n_bf, T);
  }
  __syncwarp();
  const int n_out = 5 * n_sig, G = split_factor(n_out, L.n_bf);
  const int chunk = (L.n_bf + G - 1) / G, n_task = n_out * G;
  for (int base = 0; base < n_task; base += WARP) {
    const int task = base + lane, o = task / G, part = task - o * G;
    double acc = 0.0;
    if (task < n_task) {
      const int c = o / n_sig, k = o - c * n_sig;
      const double* crow = S.C + (size_t)k * L.n_bf;
      const double* x = chi5 + c * L.n_bf;
      const int mu1 = min(L.n_bf, (part + 1) * chunk);
      for (int mu = part * chunk; mu < mu1; ++mu) acc = fma(__ldg(crow + mu), x[mu], acc);
    }
    for (int sh = 1; sh < G; sh <<= 1) acc += __shfl_xor_sync(FULL, acc, sh);
    if (task < n_task && part == 0) phi5[(o / n_sig) * L.n_max + (o % n_sig)] = acc;
  }
  __syncwarp();
}

// Bare and capped electron-nucleus potentials of one electron (Appendix D:
// nu_ei and nu^a_ei), warp-cooperative over nuclei; result valid in all lanes.
// 1/r from the refined reciprocal square root; ia = 1/a.
__device__ void electron_potentials(const DevSys& S, const double q[3], double a, double ia, int lane, double& nu,
                                    double& nucap) {
  nu = 0.0;
  nucap = 0.0;
  for (int I = lane; I < S.n_nuc; I += WARP) {
    const double dx = q[0] - __ldg(S.R + 3 * I), dy = q[1] - __ldg(S.R + 3 * I + 1),
                 dz = q[2] - __ldg(S.R + 3 * I + 2);
    const double s = fma(dz, dz, fma(dy, dy, dx * dx));
    const double ir = rsqrt_nr(s);
    const double Z = __ldg(S.Z + I);
    if (__ldg(S.kind + I) == 0) {
      nu -= Z * ir;
      nucap -= s >= a * a ? Z * ir : Z * ia;   // Z / max(r, a)
    } else {
      const double v = -Z * erf_over_r(s, ir, __ldg(S.irc + I), __ldg(S.irc2 + I), S.erftab);
      nu += v;
      nucap += v;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    nu += __shfl_xor_sync(FULL, nu, o);
    nucap += __shfl_xor_sync(FULL, nucap, o);
  }
}

// Bare and capped potentials of every electron (ep[2 i], ep[2 i + 1]): G lanes
// per electron (the largest power of two with n_e G <= 32), each taking every
// G-th nucleus, combined by shuffles.
__device__ void all_potentials(const DevSys& S, const Layout& L, const double* x, double* ep, double a, double ia,
                               int lane) {
  const int ne = L.n_e;
  int G = 1;
  while (G < WARP && ne * 2 * G <= WARP) G <<= 1;
  const double a2 = a * a;
  for (int base = 0; base < ne; base += WARP / G) {
    const int e = base + lane / G, sub = lane % G;
    double nu = 0.0, nucap = 0.0;
    if (e < ne)
      for (int I = sub; I < S.n_nuc; I += G) {
        const double dx = x[3 * e] - __ldg(S.R + 3 * I), dy = x[3 * e + 1] - __ldg(S.R + 3 * I + 1),
                     dz = x[3 * e + 2] - __ldg(S.R + 3 * I + 2);
        const double s = fma(dz, dz, fma(dy, dy, dx * dx));
        const double ir = rsqrt_nr(s);
        const double Z = __ldg(S.Z + I);
        if (__ldg(S.kind + I) == 0) {
          nu -= Z * ir;
          nucap -= dge_nonneg(s, a2) ? Z * ir : Z * ia;
        } else {
          const double v = -Z * erf_over_r(s, ir, __ldg(S.irc + I), __ldg(S.irc2 + I), S.erftab);
          nu += v;
          nucap += v;
        }
      }
    for (int o = G >> 1; o; o >>= 1) {
      nu += __shfl_xor_sync(FULL, nu, o);
      nucap += __shfl_xor_sync(FULL, nucap, o);
    }
    if (e < ne && sub == 0) {
      ep[2 * e] = nu;
      ep[2 * e + 1] = nucap;
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------ Gauss-Jordan
// In-place inversion of the N x N matrix held as the left half of M = [A | I]
// (N x 2N, row-major) with partial pivoting; afterwards the right half is
// A^{-1}.  Returns true on a zero (or non-finite) pivot.  With logdet set,
// adds log|det A| (the sum of log|pivot|) to it.  f is scratch of N doubles:
// the elimination factors of a column are recorded first, so that all rows are
// then updated in one pass over (row, column) pairs.  The pivot search
// compares |a| on the integer images of the doubles (a NaN never wins; the
// lowest row wins ties), over as many butterfly levels as the candidate lanes
// need, and 1/pivot is the refined reciprocal, so that the FP64 pipe sees only
// the row scaling and the elimination.
__device__ bool warp_gauss_jordan(double* M, int N, int lane, double* f, double* logdet = nullptr) {
  const int W2 = 2 * N;
  int npad = 1;
  while (npad < N && npad < WARP) npad <<= 1;
  constexpr long long ABS = 0x7fffffffffffffffll, INF = 0x7ff0000000000000ll;
  for (int c = 0; c < N; ++c) {
    long long best = -1;   // |a| as a non-negative integer image; -1: no candidate
    int bi = N;
    for (int r = c + lane; r < N; r += WARP) {
      const long long v = __double_as_longlong(M[r * W2 + c]) & ABS;
      if (v <= INF && (v > best || (v == best && r < bi))) { best = v; bi = r; }
    }
    for (int o = npad >> 1; o; o >>= 1) {
      const long long ob = __shfl_xor_sync(FULL, best, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    best = __shfl_sync(FULL, best, 0);
    bi = __shfl_sync(FULL, bi, 0);
    if (best <= 0 || best >= INF) return true;    // zero, no candidate or infinite
    if (bi != c) {
      for (int j = lane; j < W2; j += WARP) {
        const double t = M[c * W2 + j];
        M[c * W2 + j] = M[bi * W2 + j];
        M[bi * W2 + j] = t;
      }
    }
    __syncwarp();
    const double piv = M[c * W2 + c];
    // refined reciprocal inside the normal range, the division outside it
    const int ex = (int)(best >> 52);
    const double inv = ex > 24 && ex < 2000 ? rcp_nr(piv) : 1.0 / piv;
    if (logdet) *logdet += log(fabs(piv));
    __syncwarp();
    // scale the pivot row; record the other rows' factors (other rows: no conflict)
    for (int j = lane; j < W2; j += WARP) M[c * W2 + j] *= inv;
    for (int r = lane; r < N; r += WARP) f[r] = r == c ? 0.0 : M[r * W2 + c];
    __syncwarp();
    for (int t = lane; t < N * W2; t += WARP) {
      const int r = t / W2, j = t - r * W2;
      const double fr = f[r];
      if ((__double_as_longlong(fr) << 1) != 0) M[t] -= fr * M[c * W2 + j];   // fr != 0
    }
    __syncwarp();
  }
  return false;
}

// Global-memory working arrays of one walker evaluation.  In the propagate
// and initialisation kernels g, chi, u2 and pt point into the walker's cache
// block; configuration evaluation uses per-warp scratch for g and keeps no
// hop caches (chi, u2, pt null).  gj is per-warp scratch (the Gauss-Jordan
// work matrix [n_max][2 n_max]).
struct Scr {
  double* g;     // [n_e][n_bf]   g_i = C^T B[:, i]
  double* chi;   // [n_bf][6 n_e] basis values at every hop (mu-major: lanes on consecutive hops read consecutive words)
  double* u2;    // [n_e][6 n_e]  u2[j][p]: pair Jastrow term of hop p with partner j
  double* pt;    // [n_e][n_e][4] pair terms at the current positions: u, u'/r, u'' + 2u'/r, 1/(2r)
  double* gj;
  double* geo;   // global geometry and pair distances of a large system (null: shared memory)
  double* pr2;
};
__host__ __device__ inline size_t geo_doubles(const Layout& L, int n_nuc) {
  return L.geo_glob ? 4 * (size_t)L.n_e * n_nuc + (size_t)L.n_e * L.n_e : 0;
}
__host__ __device__ inline size_t scratch_doubles(const Layout& L, int n_nuc) {
  return (size_t)L.n_e * L.n_bf + 2 * (size_t)L.n_max * L.n_max + geo_doubles(L, n_nuc);
}
// Per-warp scratch starting at base (a region of scratch_doubles(L) doubles).
__device__ __forceinline__ Scr warp_scratch_at(const Layout& L, int n_nuc, double* base) {
  Scr s;
  s.g = base;
  s.gj = s.g + (size_t)L.n_e * L.n_bf;
  s.chi = s.u2 = s.pt = nullptr;
  s.geo = L.geo_glob ? s.gj + 2 * (size_t)L.n_max * L.n_max : nullptr;
  s.pr2 = L.geo_glob ? s.geo + 4 * (size_t)L.n_e * n_nuc : nullptr;
  return s;
}
__device__ __forceinline__ Scr warp_scratch(const Layout& L, int n_nuc, double* base, int slot) {
  return warp_scratch_at(L, n_nuc, base + (size_t)slot * scratch_doubles(L, n_nuc));
}
__device__ __forceinline__ Scr walker_scratch(const Layout& L, double* cblk, const Scr& warp) {
  Scr s;
  s.g = cblk + L.c_g;
  s.chi = cblk + L.c_chi;
  s.u2 = cblk + L.c_u2;
  s.pt = cblk + L.c_pt;
  s.gj = warp.gj;
  s.geo = L.geo_glob ? cblk + L.c_geo : nullptr;
  s.pr2 = L.geo_glob ? cblk + L.c_pr2 : nullptr;
  return s;
}

// Squared distance written with explicit FMAs so that every call site rounds
// identically (incremental updates subtract exactly what was added).
__device__ __forceinline__ double sqdist(double dx, double dy, double dz) {
  return fma(dz, dz, fma(dy, dy, dx * dx));
}

// B^T of both spin blocks from the cached orbital values A[i][k] = phi_k(r_i)
// (walker block in global memory).  Returns true if a block is singular.
__device__ bool reinvert(const Layout& L, const double* __restrict__ gblk, double* sm, double* scratch, int lane,
                         double* logdet = nullptr) {
  bool sing = false;
  const double* cache = gblk + L.g_cache;
  double* bt = sm + L.s_bt;
  // the work matrix in the per-hop scratch region of the working set when it
  // fits (free between hops), else in the global scratch
  if (2 * L.n_max * L.n_max <= L.s_phi5 - L.s_tmp) scratch = sm + L.s_tmp;
  for (int blk = 0; blk < 2; ++blk) {
    const int n = blk ? L.n_dn : L.n_up;
    const int e0 = blk ? L.n_up : 0;
    const int bto = blk ? L.n_up * L.n_up : 0;
    if (n == 0) continue;
    for (int o = lane; o < n * 2 * n; o += WARP) {
      const int r = o / (2 * n), c = o - r * 2 * n;
      scratch[o] = c < n ? cache[(e0 + r) * 5 * L.n_max + c] : (c - n == r ? 1.0 : 0.0);
    }
    __threadfence_block();
    __syncwarp();
    sing |= warp_gauss_jordan(scratch, n, lane, sm + L.s_row, logdet);
    for (int o = lane; o < n * n; o += WARP) {
      const int i = o / n, k = o - i * n;
      bt[bto + o] = scratch[k * 2 * n + n + i];
    }
    __threadfence_block();
    __syncwarp();
  }
  return sing;
}

// g_i = C^T B[:, i] for electrons [e0, e1).
__device__ void compute_g(const DevSys& S, const Layout& L, const double* sm, double* g, int e0, int e1, int lane) {
  const double* bt = sm + L.s_bt;
  for (int o = lane + e0 * L.n_bf; o < e1 * L.n_bf; o += WARP) {
    const int i = o / L.n_bf, mu = o - i * L.n_bf;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc = fma(__ldg(S.C + (size_t)k * L.n_bf + mu), brow[k], acc);
    g[o] = acc;
  }
  __threadfence_block();
  __syncwarp();
}

// ------------------------------------------------------------ evaluation
struct EvalOut {
  double bbar, vsf, W, eL;
  double kept;   // sum of the kept (positive) hop ratios
  int n_node;
};

// Pade pair term u = c r/(1 + b r) and its radial derivatives from s = r^2,
// written with 1/r: u = c q, q = 1/(1/r + b), and 1/(1 + b r) = q / r.
struct Pair {
  double u, up, upp, ir;
};
__device__ __forceinline__ Pair pade_ir(double ir, double c, double b) {
  Pair p;
  p.ir = ir;
  const double q = rcp_nr(p.ir + b);
  const double t = p.ir * q;
  p.u = c * q;
  p.up = c * t * t;
  p.upp = -2.0 * b * p.up * t;
  return p;
}
__device__ __forceinline__ Pair pade(double s, double c, double b) { return pade_ir(rsqrt_nr(s), c, b); }
__device__ __forceinline__ double pade_value(double s, double c, double b) { return c * rcp_nr(rsqrt_nr(s) + b); }

// Component of (xi - xj) along hop axis ax: the Cartesian component, or the
// projection on versor ax of a randomised lattice.
template <bool ROT>
__device__ __forceinline__ double proj(const double* xi, const double* xj, const double* V, int ax) {
  if (!ROT) return xi[ax] - xj[ax];
  const double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
  return fma(dz, V[3 * ax + 2], fma(dy, V[3 * ax + 1], dx * V[3 * ax]));
}

// Unordered pair q (0 <= q < n (n - 1) / 2, row-major over i < j) -> (i, j).
__device__ __forceinline__ void pair_index(int q, int n, int& i, int& j) {
  const float b = 2.f * n - 1.f;
  int r = (int)((b - sqrtf(fmaxf(b * b - 8.f * q, 0.f))) * 0.5f);
  r = max(0, min(r, n - 2));
  while (r > 0 && r * (2 * n - r - 1) / 2 > q) --r;
  while (r < n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= q) ++r;
  i = r;
  j = q - r * (2 * n - r - 1) / 2 + r + 1;
}

// Jastrow pair constant for electrons i, j.
__device__ __forceinline__ double pair_c(const DevSys& S, const Layout& L, int i, int j) {
  return ((i < L.n_up) == (j < L.n_up)) ? S.j2_par : S.j2_anti;
}

// (4) fixed-node split and regularised potential per electron, from the hop
// ratios, the Jastrow and determinant derivatives and the potentials.  G lanes
// share an electron (G = 2 when n_e <= 16): each sums 6/G of its hop ratios,
// the pair combines the node test and the ratio sum, and both evaluate the
// electron's potential terms (one adds them).  For the per-configuration node
// rule both the capped and the plain sums are kept and chosen at the end.
__device__ EvalOut assemble(const DevSys& S, const Layout& L, const double* sm, double ia2, int node_rule,
                            int lane) {
  const int ne = L.n_e;
  const double* rat = sm + L.s_rat;
  const double* ej = sm + L.s_ej;
  const double* ep = sm + L.s_ep;
  const double* dd = sm + L.s_dd;
  const int G = ne <= WARP / 2 ? 2 : 1, per_pass = WARP / G, sub = lane % G, nd = 6 / G;
  double kept = 0.0, negs = 0.0, nuopt = 0.0, nuplain = 0.0, vee = 0.0;
  int nnode = 0;
  bool any_node = false;
  for (int base = 0; base < ne; base += per_pass) {
    const int i = base + lane / G;
    const bool valid = i < ne;
    double sr = 0.0;
    bool node = false;
    if (valid)
      for (int d = sub * nd; d < (sub + 1) * nd; ++d) {
        const double r = rat[6 * i + d];
        const long long b = __double_as_longlong(r);
        sr += r;
        if (b > 0) kept += r;                               // r > 0
        if (b < 0 && (b << 1) != 0) { negs -= r; node = true; }   // r < 0 (not -0)
      }
    if (G == 2) {
      sr += __shfl_xor_sync(FULL, sr, 1);
      node |= __shfl_xor_sync(FULL, (int)node, 1) != 0;
    }
    any_node |= __any_sync(FULL, node);
    if (valid && sub == 0) {
      const double* q = ej + 6 * i;
      const double* dv = dd + 4 * i;
      const double lap = dv[3] + 2.0 * (dv[0] * q[1] + dv[1] * q[2] + dv[2] * q[3]) + q[4] +
                         (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      const double nu_zv = ep[2 * i] + 0.5 * ((sr - 6.0) * ia2 - lap);
      const double nu_cap = fmax(nu_zv, ep[2 * i + 1]);
      bool apply;
      if (node_rule == 0) apply = node;
      else apply = node_rule >= 1;       // rule 1: capped sum, chosen below
      nuopt += apply ? nu_cap : nu_zv;
      nuplain += nu_zv;
      vee += q[5];
    }
    nnode += __popc(__ballot_sync(FULL, valid && sub == 0 && node));
  }
  {
    const double v[4] = {kept, negs, nuopt, vee};
    const double t = warp_sum4(v, lane);
    kept = __shfl_sync(FULL, t, 0);
    negs = __shfl_sync(FULL, t, 8);
    nuopt = __shfl_sync(FULL, t, 16);
    vee = __shfl_sync(FULL, t, 24);
  }
  if (node_rule == 1 && !any_node) {
#pragma unroll
    for (int o = 16; o; o >>= 1) nuplain += __shfl_xor_sync(FULL, nuplain, o);
    nuopt = nuplain;
  }
  EvalOut e;
  const double i2a2 = 0.5 * ia2;
  e.kept = kept;
  e.bbar = kept * i2a2;
  e.vsf = negs * i2a2;
  e.W = 3.0 * ne * ia2 + nuopt + vee + S.v_ii + e.vsf;
  e.eL = e.W - e.bbar;
  e.n_node = nnode;
  return e;
}

// Determinant derivatives grad_i D/D, lap_i D/D for electrons [e0, e1).
__device__ void det_derivs(const Layout& L, const double* __restrict__ gblk, double* sm, int e0, int e1, int lane) {
  const double* bt = sm + L.s_bt;
  const double* cache = gblk + L.g_cache;
  double* dd = sm + L.s_dd;
  for (int o = lane + 4 * e0; o < 4 * e1; o += WARP) {
    const int i = o >> 2, c = o & 3;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    const double* ce = cache + i * 5 * L.n_max + (c + 1) * L.n_max;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc = fma(ce[k], brow[k], acc);
    dd[o] = acc;
  }
}

// Full evaluation at the walker's current configuration (Appendix D): every
// hop ratio, b_bar, V_sf, W, e_L.  Requires x, B^T and potentials in shared
// memory, the orbital cache in the walker block and g current in scr.g.
// Fills the incremental caches: geometry, pair distances, per-electron
// Jastrow sums and derivatives, per-hop determinant ratio and Jastrow sums,
// and (when scr.chi is set) the basis values at every hop.
template <bool ROT, bool GG>
__device__ EvalOut eval_full(const DevSys& S, const Layout& L, const double* __restrict__ gblk, double* sm, Scr scr,
                             double a, int node_rule, const double* T, int lane) {
  const int ne = L.n_e, nbf = L.n_bf, nn = S.n_nuc, P = L.n_hop;
  const double* x = sm + L.s_x;
  const double* g = scr.g;
  double* rat = sm + L.s_rat;
  double* ej = sm + L.s_ej;
  // GG: a large system's geometry caches in global memory (compile-time
  // choice, so that the shared-memory form keeps shared-memory accesses)
  double* geo = GG ? scr.geo : sm + L.s_geo;
  double* pr2 = GG ? scr.pr2 : sm + L.s_pr2;
  double* hD = sm + L.s_hd;
  double* hJ1 = sm + L.s_hj1;
  double* hJ2 = sm + L.s_hj2;
  const double* V = sm + L.s_v;
  const double a2 = a * a;
  // (1) current-configuration Jastrow sums/derivatives and geometry; G lanes
  // share one electron, each taking every G-th partner (electrons, then nuclei)
  {
    int npad = 1;
    while (npad < ne) npad <<= 1;
    const int G = npad >= WARP ? 1 : WARP / npad;
    const int per = ne - 1 + nn;
    for (int base = 0; base < ne; base += WARP / G) {
      const int e = base + lane / G, sub = lane % G;
      double U = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, LJ = 0.0, vee = 0.0;
      if (e < ne) {
        const double xe = x[3 * e], ye = x[3 * e + 1], ze = x[3 * e + 2];
        for (int t = sub; t < per; t += G) {
          if (t < ne - 1) {
            const int j = t < e ? t : t + 1;
            const double dx = xe - x[3 * j], dy = ye - x[3 * j + 1], dz = ze - x[3 * j + 2];
            const double s = sqdist(dx, dy, dz);
            pr2[e * ne + j] = s + a2;
            const Pair p = pade(s, pair_c(S, L, e, j), S.j2_b);
            const double f = p.up * p.ir, lap = p.upp + 2.0 * f, hir = 0.5 * p.ir;
            U += p.u;
            gx = fma(f, dx, gx); gy = fma(f, dy, gy); gz = fma(f, dz, gz);
            LJ += lap;
            vee += hir;
            if (scr.pt) {
              double* pt = scr.pt + CHK(4 * (e * ne + j), 4 * ne * ne);
              pt[0] = p.u; pt[1] = f; pt[2] = lap; pt[3] = hir;
            }
          } else {
            const int I = t - (ne - 1);
            const double dx = xe - __ldg(S.R + 3 * I), dy = ye - __ldg(S.R + 3 * I + 1),
                         dz = ze - __ldg(S.R + 3 * I + 2);
            const double s = sqdist(dx, dy, dz);
            double* gg = geo + (e * nn + I) * 4;
            gg[0] = s + a2;
            if (ROT) {
              for (int k = 0; k < 3; ++k) gg[1 + k] = fma(dz, V[3 * k + 2], fma(dy, V[3 * k + 1], dx * V[3 * k]));
            } else {
              gg[1] = dx; gg[2] = dy; gg[3] = dz;
            }
            const double A = __ldg(S.j1A + I);
            if (A != 0.0) {
              const Pair p = pade(s, -A, __ldg(S.j1B + I));
              const double f = p.up * p.ir;
              U += p.u;
              gx = fma(f, dx, gx); gy = fma(f, dy, gy); gz = fma(f, dz, gz);
              LJ += p.upp + 2.0 * f;
            }
          }
        }
      }
      for (int o = G >> 1; o; o >>= 1) {
        U += __shfl_xor_sync(FULL, U, o);
        gx += __shfl_xor_sync(FULL, gx, o);
        gy += __shfl_xor_sync(FULL, gy, o);
        gz += __shfl_xor_sync(FULL, gz, o);
        LJ += __shfl_xor_sync(FULL, LJ, o);
        vee += __shfl_xor_sync(FULL, vee, o);
      }
      if (e < ne && sub == 0) {
        double* q = ej + 6 * e;
        q[0] = U; q[1] = gx; q[2] = gy; q[3] = gz; q[4] = LJ; q[5] = vee;
      }
    }
  }
  det_derivs(L, gblk, sm, 0, ne, lane);
  __syncwarp();
  // (3a) with hop caches: the pair Jastrow term of every hop, each unordered
  // pair once (the term of hop (i, d) with partner j is the term of hop
  // (j, d ^ 1) with i, bit for bit), into scr.u2
  if (scr.u2) {
    const int n_task = 3 * ne * (ne - 1);
    for (int t = lane; t < n_task; t += WARP) {
      const int q = t / 6, d = t - 6 * q, ax = d >> 1;
      int i, j;
      pair_index(q, ne, i, j);
      const double sa = (d & 1) ? -a : a;
      const double v =
          pade_value(fma(sa + sa, proj<ROT>(x + 3 * i, x + 3 * j, V, ax), pr2[i * ne + j]), pair_c(S, L, i, j), S.j2_b);
      scr.u2[CHK((size_t)j * P + 6 * i + d, (size_t)ne * P)] = v;
      scr.u2[CHK((size_t)i * P + 6 * j + (d ^ 1), (size_t)ne * P)] = v;
    }
    __threadfence_block();
    __syncwarp();
  }
  // (3) every hop: basis values (kept in scr.chi), determinant ratio
  // chi(r') . g_i, one-body and pair Jastrow sums
  for (int p = lane; p < P; p += WARP) {
    const int i = p / 6, d = p - 6 * i, ax = d >> 1;
    const double sa = (d & 1) ? -a : a;
    const double s2a = sa + sa;
    const double* gi = g + i * nbf;
    double det = 0.0, J1 = 0.0, J2 = 0.0;
    for (int I = 0; I < nn; ++I) {
      const double* gg = geo + (i * nn + I) * 4;
      const double s = fma(s2a, gg[1 + ax], gg[0]);   // |r' - R_I|^2
      double dv[3];
      if (ROT) {
        for (int k = 0; k < 3; ++k) dv[k] = fma(sa, V[3 * ax + k], x[3 * i + k] - __ldg(S.R + 3 * I + k));
      } else {
        dv[0] = gg[1]; dv[1] = gg[2]; dv[2] = gg[3];
        dv[ax] += sa;
      }
      const double A = __ldg(S.j1A + I);
      if (A != 0.0) J1 += pade_value(s, -A, __ldg(S.j1B + I));
      for (int sh = CHK(__ldg(S.atom_sh + I), S.n_shell); sh < CHK(__ldg(S.atom_sh + I + 1), S.n_shell + 1); ++sh) {
        const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh),
                  bf = __ldg(S.sh_bf + sh);
        const double arg = l == -1 ? s * rsqrt_nr(s) : s;
        double rad = 0.0;
        for (int q = 0; q < np; ++q) rad = fma(__ldg(S.coefs + off + q), exp_tab(-__ldg(S.exps + off + q) * arg, T), rad);
        if (l != 1) {
          det = fma(rad, gi[bf], det);
          if (scr.chi) scr.chi[CHK((size_t)bf * P + p, (size_t)nbf * P)] = rad;
        } else {
          const double c0 = dv[0] * rad, c1 = dv[1] * rad, c2 = dv[2] * rad;
          det = fma(c0, gi[bf], fma(c1, gi[bf + 1], fma(c2, gi[bf + 2], det)));
          if (scr.chi) {
            scr.chi[CHK((size_t)bf * P + p, (size_t)nbf * P)] = c0;
            scr.chi[CHK((size_t)(bf + 1) * P + p, (size_t)nbf * P)] = c1;
            scr.chi[CHK((size_t)(bf + 2) * P + p, (size_t)nbf * P)] = c2;
          }
        }
      }
    }
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      J2 += scr.u2 ? scr.u2[(size_t)j * P + p]
                   : pade_value(fma(s2a, proj<ROT>(x + 3 * i, x + 3 * j, V, ax), pr2[i * ne + j]), pair_c(S, L, i, j),
                                S.j2_b);
    }
    hD[p] = det;
    hJ1[p] = J1;
    hJ2[p] = J2;
    rat[p] = det * exp_tab(J1 + J2 - ej[6 * i], T);
  }
  __threadfence_block();
  __syncwarp();
  return assemble(S, L, sm, 1.0 / (a * a), node_rule, lane);
}

// Incremental evaluation after electron m hopped from xo (kept at s_xo) to its
// position in x.  Everything that does not depend on electron m keeps its
// cached value: the basis values at the other electrons' hops, their one-body
// Jastrow sums and, outside m's spin block, their determinant ratios.  With
// all_blocks (after a from-scratch inversion changed B of both blocks) the
// determinant ratios and derivatives of every electron are refreshed from the
// cached basis values.  Pair terms with m are swapped, not recomputed: the old
// term comes from the caches (scr.pt for the current positions, scr.u2 for
// the hops) and the new term of hop d of electron i with m equals the term of
// m's opposite hop (d ^ 1) with i, since r_i + s a e - r_m = -(r_m - s a e - r_i).
// Electron m's bare and capped potentials are evaluated here too, on the lanes
// that hold its distances to the nuclei (ia = 1/a).
template <bool ROT, bool GG>
__device__ EvalOut eval_incr(const DevSys& S, const Layout& L, const double* __restrict__ gblk, double* sm, Scr scr,
                             int m, bool all_blocks, double a, double ia, int node_rule, const double* T, int lane) {
  const int ne = L.n_e, nbf = L.n_bf, nn = S.n_nuc, P = L.n_hop;
  const double* x = sm + L.s_x;
  const double* xo = sm + L.s_xo;
  const double* g = scr.g;
  double* rat = sm + L.s_rat;
  double* ej = sm + L.s_ej;
  // GG: a large system's geometry caches in global memory (compile-time
  // choice, so that the shared-memory form keeps shared-memory accesses)
  double* geo = GG ? scr.geo : sm + L.s_geo;
  double* pr2 = GG ? scr.pr2 : sm + L.s_pr2;
  double* hD = sm + L.s_hd;
  double* hJ1 = sm + L.s_hj1;
  double* hJ2 = sm + L.s_hj2;
  double* tmp = sm + L.s_tmp;
  const double* V = sm + L.s_v;
  const double a2 = a * a;
  const int per = ne - 1 + nn;
  const double xm = x[3 * m], ym = x[3 * m + 1], zm = x[3 * m + 2];
  // (A) electron m: geometry, its Jastrow sums and its bare and capped
  // potentials from scratch, one partner (electron, then nucleus) per lane;
  // (B) the partner electron's sums swap their term with m (old term from
  // scr.pt)
  {
    const double xo0 = xo[0], xo1 = xo[1], xo2 = xo[2];
    // U, grad (3), lap, e-e, nu, nu capped
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = lane; t < per; t += WARP) {
      const bool pair = t < ne - 1;
      const int j = t < m ? t : t + 1, I = t - (ne - 1);
      double px, py, pz, c, b;
      if (pair) {
        px = x[3 * j]; py = x[3 * j + 1]; pz = x[3 * j + 2];
        c = pair_c(S, L, m, j);
        b = S.j2_b;
      } else {
        px = __ldg(S.R + 3 * I); py = __ldg(S.R + 3 * I + 1); pz = __ldg(S.R + 3 * I + 2);
        c = -__ldg(S.j1A + I);
        b = __ldg(S.j1B + I);
      }
      const double dx = xm - px, dy = ym - py, dz = zm - pz;
      const double s = sqdist(dx, dy, dz);
      const double ir = rsqrt_nr(s);
      // one Pade evaluation for both kinds; a nucleus without one-body term
      // (c = 0) contributes zeros and is evaluated at a dummy distance
      const Pair p = pade_ir(pair || dnonzero(c) ? ir : 1.0, c, b);
      const double f = p.up * p.ir, lap = p.upp + 2.0 * f;
      acc[0] += p.u;
      acc[1] = fma(f, dx, acc[1]); acc[2] = fma(f, dy, acc[2]); acc[3] = fma(f, dz, acc[3]);
      acc[4] += lap;
      if (pair) {
        const double hir = 0.5 * p.ir;
        acc[5] += hir;
        pr2[m * ne + j] = s + a2;
        pr2[j * ne + m] = s + a2;
        double* pm = scr.pt + CHK(4 * (m * ne + j), 4 * ne * ne);
        double* pj = scr.pt + CHK(4 * (j * ne + m), 4 * ne * ne);
        const double ou = pm[0], of = pm[1], ol = pm[2], oh = pm[3];
        const double ox = px - xo0, oy = py - xo1, oz = pz - xo2;
        double* q = ej + 6 * j;
        q[0] += p.u - ou;
        q[1] += f * -dx - of * ox;
        q[2] += f * -dy - of * oy;
        q[3] += f * -dz - of * oz;
        q[4] += lap - ol;
        q[5] += hir - oh;
        pm[0] = p.u; pm[1] = f; pm[2] = lap; pm[3] = hir;
        pj[0] = p.u; pj[1] = f; pj[2] = lap; pj[3] = hir;
      } else {
        double* gg = geo + (m * nn + I) * 4;
        gg[0] = s + a2;
        if (ROT) {
          for (int k = 0; k < 3; ++k) gg[1 + k] = fma(dz, V[3 * k + 2], fma(dy, V[3 * k + 1], dx * V[3 * k]));
        } else {
          gg[1] = dx; gg[2] = dy; gg[3] = dz;
        }
        // nu_ei and nu^a_ei (Appendix D): -Z/r and -Z/max(r, a), or the
        // screened -Z erf(r/r_c)/r for both, as -Z v and -Z v_cap (only the
        // screened kind spends FP64 work in its branch)
        const double Z = __ldg(S.Z + I);
        double v, vcap;
        if (__ldg(S.kind + I) == 0) {
          v = ir;
          vcap = dge_nonneg(s, a2) ? ir : ia;
        } else {
          v = erf_over_r(s, ir, __ldg(S.irc + I), __ldg(S.irc2 + I), S.erftab);
          vcap = v;
        }
        acc[6] = fma(-Z, v, acc[6]);
        acc[7] = fma(-Z, vcap, acc[7]);
      }
    }
    const double tot = warp_sum8(acc, lane);
    const int k = (lane >> 2) & 7;
    if ((lane & 3) == 0) {
      if (k < 6) ej[6 * m + k] = tot;
      else sm[L.s_ep + 2 * m + (k - 6)] = tot;
    }
  }
  // (C) determinant derivatives of the refreshed spin block(s)
  const SpinRef srm = spin_ref(L, m);
  const int b0 = all_blocks ? 0 : m - srm.ii, b1 = all_blocks ? ne : m - srm.ii + srm.n;
  det_derivs(L, gblk, sm, b0, b1, lane);
  __threadfence_block();
  __syncwarp();
  // (D) basis values at m's six hops.  A Gaussian primitive factors over the
  // hop: with g = gg[1 + k] the component of r_m - R along hop versor k,
  // |r_m +- a v_k - R|^2 = (|r_m - R|^2 + a^2) +- 2 a g, so
  // exp(-z |r' - R|^2) = E0 t^(+-1), E0 = exp(-z (|r_m - R|^2 + a^2)),
  // t = exp(-2 z a |g|) <= 1: the hop away from the nucleus takes E0 t, the
  // hop towards it E0 / t.  One lane per shell; a primitive costs 4
  // exponentials and 3 reciprocals instead of 6 exponentials.  The radial
  // values of p shells go to the per-hop scratch (free until the Jastrow pass
  // below) and their Cartesian factors are applied in a second, uniform pass
  // over (p shell, component, hop).  Slater 1s shells (not separable) evaluate
  // their six hops directly, as does a hop towards a nucleus more than
  // 650 / (2 z a) bohr away (t would underflow).
  {
    double* radp = tmp;   // [n_shell][6]
    for (int sh = lane; sh < S.n_shell; sh += WARP) {
      const int I = CHK(__ldg(S.sh_atom + sh), nn);
      const double* gg = geo + (m * nn + I) * 4;
      const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = CHK(__ldg(S.sh_off + sh), S.n_prim),
                bf = CHK(__ldg(S.sh_bf + sh), nbf);
      double rad[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (l == -1) {
        for (int d = 0; d < 6; ++d) {
          const double sa = (d & 1) ? -a : a;
          const double s = fma(sa + sa, gg[1 + (d >> 1)], gg[0]);
          const double r = s * rsqrt_nr(s);
          for (int q = 0; q < np; ++q)
            rad[d] = fma(__ldg(S.coefs + off + q), exp_tab(-__ldg(S.exps + off + q) * r, T), rad[d]);
        }
      } else {
        const double g3[3] = {gg[1], gg[2], gg[3]};
        for (int q = 0; q < np; ++q) {
          const double z = __ldg(S.exps + off + q);
          const double e0 = __ldg(S.coefs + off + q) * exp_tab(-z * gg[0], T);
          const double tza = -(a + a) * z;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double x = tza * fabs(g3[k]);
            const double t = exp_tab(x, T);
            const double away = e0 * t;
            double toward;
            // |x| < 650 and g >= 0 are tested on the integer images (no FP64 compare)
            if ((__double_as_longlong(x) & 0x7fffffffffffffffll) < 0x4084500000000000ll) {
              toward = e0 * rcp_nr(t);
            } else {
              toward = __ldg(S.coefs + off + q) * exp_tab(-z * fma(-(a + a), fabs(g3[k]), gg[0]), T);
            }
            // hop 2k moves by +a along v_k, hop 2k + 1 by -a (g = -0 counts as
            // negative: both hops then take e0)
            const bool pos = __double_as_longlong(g3[k]) >= 0;
            rad[2 * k] += pos ? away : toward;
            rad[2 * k + 1] += pos ? toward : away;
          }
        }
      }
      if (l == 1) {
        for (int d = 0; d < 6; ++d) radp[CHK(6 * sh + d, L.s_phi5 - L.s_tmp)] = rad[d];
      } else {
        for (int d = 0; d < 6; ++d) scr.chi[CHK((size_t)bf * P + 6 * m + d, (size_t)nbf * P)] = rad[d];
      }
    }
    __syncwarp();
    const int n_pt = 18 * (S.n_shell - S.n_shell_np);
    for (int o = lane; o < n_pt; o += WARP) {
      const int kk = o / 18, r = o - 18 * kk, k = r / 6, d = r - 6 * k, ax = d >> 1;
      const int sh = CHK(__ldg(S.sh_ord + S.n_shell_np + kk), S.n_shell);
      const int I = CHK(__ldg(S.sh_atom + sh), nn), bf = CHK(__ldg(S.sh_bf + sh), nbf - 2);
      const double sa = (d & 1) ? -a : a;
      const double* gg = geo + (m * nn + I) * 4;
      const double dk = ROT ? fma(sa, V[3 * ax + k], x[3 * m + k] - __ldg(S.R + 3 * I + k))
                            : gg[1 + k] + (k == ax ? sa : 0.0);
      scr.chi[CHK((size_t)(bf + k) * P + 6 * m + d, (size_t)nbf * P)] = dk * radp[CHK(6 * sh + d, L.s_phi5 - L.s_tmp)];
    }
    __syncwarp();
  }
  for (int o = lane; o < 6 * per; o += WARP) {
    const int d = o / per, t = o - d * per, ax = d >> 1;
    const double sa = (d & 1) ? -a : a;
    const bool pair = t < ne - 1;
    const int j = t < m ? t : t + 1, I = t - (ne - 1);
    double s, c, b;
    if (pair) {
      s = fma(sa + sa, proj<ROT>(x + 3 * m, x + 3 * j, V, ax), pr2[m * ne + j]);
      c = pair_c(S, L, m, j);
      b = S.j2_b;
    } else {
      const double* gg = geo + (m * nn + I) * 4;
      c = -__ldg(S.j1A + I);
      b = __ldg(S.j1B + I);
      s = dnonzero(c) ? fma(sa + sa, gg[1 + ax], gg[0]) : 1.0;
    }
    const double v = pade_value(s, c, b);
    tmp[CHK(o, L.s_phi5 - L.s_tmp)] = v;
    if (pair) scr.u2[CHK((size_t)j * P + 6 * m + d, (size_t)ne * P)] = v;
  }
  __threadfence_block();
  __syncwarp();
  {
    // sums over partners of each of m's hops: four lanes per hop
    const int d = lane >> 2, sub = lane & 3;
    double J1 = 0.0, J2 = 0.0;
    if (d < 6) {
      for (int t = sub; t < ne - 1; t += 4) J2 += tmp[d * per + t];
      for (int t = ne - 1 + sub; t < per; t += 4) J1 += tmp[d * per + t];
    }
    J1 += __shfl_xor_sync(FULL, J1, 1);
    J2 += __shfl_xor_sync(FULL, J2, 1);
    J1 += __shfl_xor_sync(FULL, J1, 2);
    J2 += __shfl_xor_sync(FULL, J2, 2);
    if (d < 6 && sub == 0) {
      hJ1[6 * m + d] = J1;
      hJ2[6 * m + d] = J2;
    }
  }
  // (E) determinant ratios of the refreshed block(s) from the cached basis
  // values, each dot product split over G lanes
  {
    const int n_out = 6 * (b1 - b0), G = split_factor(n_out, nbf);
    const int chunk = (nbf + G - 1) / G, n_task = n_out * G;
    for (int base = 0; base < n_task; base += WARP) {
      const int task = base + lane, o = task / G, part = task - o * G;
      const int p = 6 * b0 + o;
      double det = 0.0;
      if (task < n_task) {
        const double* gi = g + (p / 6) * nbf;
        const int mu1 = min(nbf, (part + 1) * chunk);
        for (int mu = part * chunk; mu < mu1; ++mu) det = fma(scr.chi[CHK((size_t)mu * P + p, (size_t)nbf * P)], gi[mu], det);
      }
      for (int sh = 1; sh < G; sh <<= 1) det += __shfl_xor_sync(FULL, det, sh);
      if (task < n_task && part == 0) hD[p] = det;
    }
  }
  // (F) pair Jastrow sums of the other electrons' hops: swap the term with m.
  // Up to four old terms per lane are loaded before any store, so that their
  // global-memory latencies overlap (a store through one pointer could alias
  // the next load, which would otherwise serialise them).
  {
    double* um = scr.u2 + (size_t)m * P;
    for (int base = 0; base < P; base += 4 * WARP) {
      double vn[4], uo[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = base + k * WARP + lane, i = p / 6;
        const bool ok = p < P && i != m;
        vn[k] = ok ? tmp[((p - 6 * i) ^ 1) * per + (i < m ? i : i - 1)] : 0.0;
        uo[k] = ok ? um[p] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = base + k * WARP + lane, i = p / 6;
        if (p < P && i != m) {
          hJ2[p] += vn[k] - uo[k];
          um[p] = vn[k];
        }
      }
    }
  }
  __threadfence_block();
  __syncwarp();
  // (G) all hop ratios
  for (int p = lane; p < P; p += WARP) rat[p] = hD[p] * exp_tab(hJ1[p] + hJ2[p] - ej[6 * (p / 6)], T);
  __threadfence_block();
  __syncwarp();
  return assemble(S, L, sm, ia * ia, node_rule, lane);
}

// Build the orbital cache and potentials at every electron, invert both
// Slater blocks and evaluate.  x must already be in shared memory.
__device__ EvalOut init_walker(const DevSys& S, const Layout& L, double* __restrict__ gblk, double* sm, Scr scr,
                               double a, int node_rule, const double* T, int lane, bool& singular,
                               double* logdet = nullptr) {
  double* chi5 = sm + L.s_tmp;     // scratch while no evaluation is in progress
  double* phi5 = sm + L.s_phi5;
  double* cache = gblk + L.g_cache;
  const double* x = sm + L.s_x;
  double* ep = sm + L.s_ep;
  const double ia = 1.0 / a;
  for (int i = 0; i < L.n_e; ++i) {
    const int n = i < L.n_up ? L.n_up : L.n_dn;
    const double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    orbital_derivs(S, L, q, n, chi5, phi5, T, lane);
    for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
    __syncwarp();
  }
  all_potentials(S, L, x, ep, a, ia, lane);
  __threadfence_block();
  singular = reinvert(L, gblk, sm, scr.gj, lane, logdet);
  compute_g(S, L, sm, scr.g, 0, L.n_e, lane);
  return L.geo_glob ? eval_full<false, true>(S, L, gblk, sm, scr, a, node_rule, T, lane)
                    : eval_full<false, false>(S, L, gblk, sm, scr, a, node_rule, T, lane);
}

// Heat-bath choice over the kept hops (r > 0) in the order p = 6 i + d: the
// first p whose running sum exceeds u * total (total = the sum of the kept
// ratios taken by the evaluation); the last kept hop if rounding leaves none;
// -1 without kept hops.  Each lane owns a contiguous run of hops: lane sums,
// one warp scan of them, then each lane continues the running sum over its own
// hops.  Signs and the comparisons of non-negative sums are taken on the
// integer images (the order of non-negative doubles is that of their bits), so
// the FP64 pipe sees only the additions.
__device__ __forceinline__ bool positive(double r) { return __double_as_longlong(r) > 0; }

__device__ int choose_hop(const double* rat, int n_hop, double u, double total, int lane) {
  if (!dpos(total)) return -1;
  const long long t = __double_as_longlong(u * total);
  const int per = (n_hop + WARP - 1) / WARP, p0 = lane * per, p1 = min(n_hop, p0 + per);
  double own = 0.0;
  for (int p = p0; p < p1; ++p) {
    const double r = rat[p];
    if (positive(r)) own += r;
  }
  double incl = own;
#pragma unroll
  for (int o = 1; o < WARP; o <<= 1) {
    const double v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  double run = __shfl_up_sync(FULL, incl, 1);
  if (lane == 0) run = 0.0;
  int hit = -1, last = -1;
  for (int p = p0; p < p1; ++p) {
    const double r = rat[p];
    if (positive(r)) {
      run += r;
      last = p;
      if (hit < 0 && __double_as_longlong(run) > t) hit = p;
    }
  }
  const unsigned hm = __ballot_sync(FULL, hit >= 0);
  if (hm) return __shfl_sync(FULL, hit, __ffs(hm) - 1);
  const unsigned km = __ballot_sync(FULL, last >= 0);
  return km ? __shfl_sync(FULL, last, 31 - __clz(km)) : -1;
}

// Apply hop p: orbital derivatives at the moved electron, Sherman-Morrison
// update of its spin block and of g by the same factors, cache and position
// update (the old position goes to s_xo), and with pots the moved electron's
// potentials (otherwise the incremental evaluation that follows sets them).
template <bool ROT>
__device__ void apply_hop(const DevSys& S, const Layout& L, double* __restrict__ gblk, double* sm, Scr scr, int p,
                          double a, double ia, bool pots, const double* T, int lane) {
  double* x = sm + L.s_x;
  double* bt = sm + L.s_bt;
  double* cache = gblk + L.g_cache;
  double* phi5 = sm + L.s_phi5;
  double* f = sm + L.s_u;
  double* row = sm + L.s_row;
  double* chi5 = sm + L.s_tmp;     // per-hop scratch, refilled by the next evaluation
  double* g = scr.g;
  double* grow = chi5 + 5 * L.n_bf;
  p = CHK(p, L.n_hop);
  const int i = p / 6, d = p - 6 * i;
  double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  const double sa = (d & 1) ? -a : a;
  if (ROT) {
    const double* V = sm + L.s_v;
    for (int k = 0; k < 3; ++k) q[k] = fma(sa, V[3 * (d >> 1) + k], q[k]);
  } else {
    q[d >> 1] += sa;
  }
  const SpinRef sr = spin_ref(L, i);
  orbital_derivs(S, L, q, sr.n, chi5, phi5, T, lane);
  double* B = bt + sr.bt_off;   // B^T of the spin block: B[j * n + k] = (A^{-1})_{k j}
  const int n = sr.n;
  // u_j = phi(r') . B[:, j]; the determinant ratio is u_ii.  Each dot is split
  // over G lanes (consecutive slices of k) and combined by shuffles.
  {
    const int G = split_factor(n, n), chunk = (n + G - 1) / G, n_task = n * G;
    for (int base = 0; base < n_task; base += WARP) {
      const int task = base + lane, j = task / G, part = task - j * G;
      double acc = 0.0;
      if (task < n_task) {
        const int k1 = min(n, (part + 1) * chunk);
        for (int k = part * chunk; k < k1; ++k) acc = fma(phi5[k], B[j * n + k], acc);
      }
      for (int sh = 1; sh < G; sh <<= 1) acc += __shfl_xor_sync(FULL, acc, sh);
      if (task < n_task && part == 0) f[j] = acc;
    }
  }
  for (int k = lane; k < n; k += WARP) row[k] = B[sr.ii * n + k];
  for (int mu = lane; mu < L.n_bf; mu += WARP) grow[mu] = g[i * L.n_bf + mu];
  __threadfence_block();
  __syncwarp();
  const double invR = rcp_nr(f[sr.ii]);   // u_ii > 0: the chosen hop is a kept one
  __syncwarp();
  // A' = A + e_i (phi' - phi)^T  =>  B' = B - B e_i (u - e_i)^T / u_i
  for (int j = lane; j < n; j += WARP) f[j] = (f[j] - (j == sr.ii ? 1.0 : 0.0)) * invR;
  __syncwarp();
  for (int o = lane; o < n * n; o += WARP) {
    const int j = o / n, k = o - j * n;
    B[o] = fma(-row[k], f[j], B[o]);
  }
  // g_j -= f_j g_i over the spin block's rows (element o = j n_bf + mu), four
  // loads per lane issued before their stores (overlapped latencies)
  {
    double* gb = g + (i - sr.ii) * L.n_bf;
    const int nt = n * L.n_bf;
    for (int base = 0; base < nt; base += 4 * WARP) {
      double gv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int o = base + k * WARP + lane;
        gv[k] = o < nt ? gb[o] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int o = base + k * WARP + lane;
        if (o < nt) {
          const int j = o / L.n_bf, mu = o - j * L.n_bf;
          gb[o] = fma(-grow[mu], f[j], gv[k]);
        }
      }
    }
  }
  for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
  double nu = 0.0, nucap = 0.0;
  if (pots) electron_potentials(S, q, a, ia, lane, nu, nucap);
  if (lane == 0) {
    double* xo = sm + L.s_xo;
    xo[0] = x[3 * i]; xo[1] = x[3 * i + 1]; xo[2] = x[3 * i + 2];
    x[3 * i] = q[0];
    x[3 * i + 1] = q[1];
    x[3 * i + 2] = q[2];
    if (pots) {
      sm[L.s_ep + 2 * i] = nu;
      sm[L.s_ep + 2 * i + 1] = nucap;
    }
  }
  __threadfence_block();
  __syncwarp();
}

// ------------------------------------------------------------ kernels
struct StepParams {
  int kind;          // 0 conventional, 1 load-balanced
  int n_proj;
  double tau;
  int max_moves;
  double E0;
  uint64_t seed;
  uint32_t interval;
  double a;
  int node_rule;
  int reinv_period;
  unsigned long long* stamps;   // optional: per walker (start ns, end ns, SM id)
  int rotate;                   // randomised lattice: new versors every interval
  unsigned* next;               // optional: zeroed work counter; warps past their first walker take the next
                                // unclaimed one from it (dynamic assignment), else walkers go round-robin
  double drift_tol;             // > 0: re-invert when the inverse residual after a hop exceeds it
  int* drift_count;             // optional: device counter of drift-triggered re-inversions
};

// Drift of the Sherman-Morrison inverse after electron i hopped: the largest
// |(A B)_rj - delta_rj| over the columns j of the spin block, for the row r
// of the next electron of the block (cyclically; the moved electron itself in
// a one-electron block), with A's rows the FP64 orbital values
// val[e * vstride + k] and B from B^T in shared memory.  Between from-scratch
// inversions B accumulates the rounding of every rank-1 update; the product
// with a row of A that the update did not touch exposes that drift.  Each
// dot product is split over G lanes (G the largest power of two with n G <=
// 32, at most 8); the maximum is taken on the integer images of the
// non-negative residuals (a NaN ranks above every number), so only the dot
// products use the FP64 pipe.  Result valid in all lanes.  Kept out of line:
// it runs on one hop in four, and inlined it would add registers to the whole
// hop loop.
__device__ __noinline__ double inverse_residual(const Layout& L, const double* val, int vstride,
                                                   const double* bt, int i, int lane) {
  const SpinRef sr = spin_ref(L, i);
  const int n = sr.n, e0 = i - sr.ii, rr = (sr.ii + 1) % n;
  const double* B = bt + sr.bt_off;   // B[j * n + k] = (A^{-1})_{k j}
  const double* arow = val + (size_t)(e0 + rr) * vstride;
  int G = 1;
  while (G < 8 && n * G * 2 <= WARP) G <<= 1;
  const int chunk = (n + G - 1) / G;
  long long worst = 0;
  for (int base = 0; base < n * G; base += WARP) {
    const int task = base + lane, j = task / G, part = task - j * G;
    double acc = 0.0;
    if (j < n) {
      const int k1 = min(n, (part + 1) * chunk);
      for (int k = part * chunk; k < k1; ++k) acc = fma(arow[k], B[j * n + k], acc);
    }
    for (int o = 1; o < G; o <<= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (j < n) {
      const long long r = __double_as_longlong(acc - (rr == j ? 1.0 : 0.0)) & 0x7fffffffffffffffll;
      worst = r > worst ? r : worst;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const long long v = __shfl_xor_sync(FULL, worst, o);
    worst = v > worst ? v : worst;
  }
  return __longlong_as_double(worst);
}

// The drift check runs on every DRIFT_EVERY-th hop since the last inversion
// (drift grows gradually; a check per hop would cost a few percent).
constexpr int DRIFT_EVERY = 4;

// Next walker of a warp after w: from the work counter (first-come order,
// which evens out walkers of unequal cost) or round-robin.
__device__ __forceinline__ int next_walker(const StepParams& P, int w, int nwarps, int lane) {
  if (!P.next) return w + nwarps;
  unsigned v = 0;
  if (lane == 0) v = atomicAdd(P.next, 1u);
  return nwarps + (int)__shfl_sync(FULL, v, 0);
}

// Hop versors of walker slot w in an interval (rows of V): one uniformly random
// rotation of the Cartesian axes (Shoemake, "Uniform random rotations",
// Graphics Gems III, 1992) from three Philox uniforms: counter
// (w, 2^32-1, interval, 2) words 0-1 and 2-3, counter (w, 2^32-1, interval, 3)
// words 0-1.
__host__ __device__ inline void interval_versors(uint64_t seed, uint32_t w, uint32_t interval, double V[9]) {
  uint32_t c[4] = {w, 0xFFFFFFFFu, interval, 2u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = uniform53(c[0], c[1]), u2 = uniform53(c[2], c[3]);
  uint32_t e[4] = {w, 0xFFFFFFFFu, interval, 3u};
  philox4x32_10(e, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u3 = uniform53(e[0], e[1]);
  const double ta = sqrt(1.0 - u1), tb = sqrt(u1);
  const double twopi = 6.283185307179586476925286766559;
  const double qx = ta * sin(twopi * u2), qy = ta * cos(twopi * u2);
  const double qz = tb * sin(twopi * u3), qw = tb * cos(twopi * u3);
  // rotation matrix R of the unit quaternion; versor k (row k of V) = R e_k
  const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                       2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                       2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) V[3 * k + j] = R[3 * j + k];
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned sm_id() {
  unsigned id;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
  return id;
}

// The exponential table sits at the start of dynamic shared memory, the
// per-warp regions after it.
__device__ __forceinline__ double* stage_table(const DevSys& S, double* smem) {
  for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) smem[j] = S.exptab[j];
  __syncthreads();
  return smem;
}

__device__ __forceinline__ void load_block(const Layout& L, const double* __restrict__ g, double* sm, int lane) {
  for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = g[L.g_x + o];
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) sm[L.s_bt + o] = g[L.g_bt + o];
  for (int o = lane; o < L.n_hop; o += WARP) sm[L.s_rat + o] = g[L.g_rat + o];
  for (int o = lane; o < 2 * L.n_e; o += WARP) sm[L.s_ep + o] = g[L.g_pot + o];
  for (int o = lane; o < SC_COUNT; o += WARP) sm[L.s_sc + o] = g[L.g_sc + o];
  __syncwarp();
}

__device__ __forceinline__ void store_block(const Layout& L, double* __restrict__ g, const double* sm, int lane) {
  __syncwarp();
  for (int o = lane; o < 3 * L.n_e; o += WARP) g[L.g_x + o] = sm[L.s_x + o];
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) g[L.g_bt + o] = sm[L.s_bt + o];
  for (int o = lane; o < L.n_hop; o += WARP) g[L.g_rat + o] = sm[L.s_rat + o];
  for (int o = lane; o < 2 * L.n_e; o += WARP) g[L.g_pot + o] = sm[L.s_ep + o];
  for (int o = lane; o < SC_COUNT; o += WARP) g[L.g_sc + o] = sm[L.s_sc + o];
}

// Shared-memory caches [s_ej, s_tmp) from / to the walker's cache block.
__device__ __forceinline__ void load_mirror(const Layout& L, const double* __restrict__ c, double* sm, int lane) {
  const int n = L.s_tmp - L.s_ej;
  for (int o = lane; o < n; o += WARP) sm[L.s_ej + o] = c[L.c_mir + o];
  __syncwarp();
}

__device__ __forceinline__ void store_mirror(const Layout& L, double* __restrict__ c, const double* sm, int lane) {
  __syncwarp();
  const int n = L.s_tmp - L.s_ej;
  for (int o = lane; o < n; o += WARP) c[L.c_mir + o] = sm[L.s_ej + o];
}

// Place walkers at x_in (n x n_e x 3), build caches, invert and evaluate.
__global__ void k_init_walkers(DevSys S, Layout L, double* __restrict__ state, double* __restrict__ cache,
                               const double* __restrict__ x_in, const double* __restrict__ w_in, int n, double a,
                               int node_rule, double* scratch) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + EXP_TAB + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const Scr wscr = warp_scratch(L, S.n_nuc, scratch, slot);
  for (int w = slot; w < n; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    double* cblk = cache + (size_t)w * L.c_stride;
    const Scr scr = walker_scratch(L, cblk, wscr);
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, gblk, sm, scr, a, node_rule, T, lane, sing);
    if (lane == 0) {
      double* sc = sm + L.s_sc;
      for (int k = 0; k < SC_COUNT; ++k) sc[k] = 0.0;
      sc[SC_W] = w_in ? w_in[w] : 1.0;
      sc[SC_BBAR] = e.bbar;
      sc[SC_VSF] = e.vsf;
      sc[SC_WDIAG] = e.W;
      sc[SC_EL] = e.eL;
      sc[SC_NNODE] = e.n_node;
      sc[SC_STATUS] = sing ? (double)ST_SINGULAR : 0.0;
      sc[SC_CACHE] = sing ? 0.0 : 1.0;
      sc[SC_KEPT] = e.kept;
    }
    store_block(L, gblk, sm, lane);
    store_mirror(L, cblk, sm, lane);
  }
}

// Evaluate arbitrary configurations without touching the walkers (the orbital
// cache of each configuration goes to scratch walker blocks).
__global__ void k_eval_configs(DevSys S, Layout L, double* __restrict__ blocks, const double* __restrict__ x_in, int n,
                               double a, int node_rule, double* __restrict__ ratios, double* __restrict__ ev,
                               int32_t* __restrict__ n_node, double* scratch) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + EXP_TAB + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const Scr scr = warp_scratch(L, S.n_nuc, scratch, slot);
  for (int w = slot; w < n; w += nwarps) {
    double* gblk = blocks + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, gblk, sm, scr, a, node_rule, T, lane, sing);
    for (int o = lane; o < L.n_hop; o += WARP) ratios[(size_t)w * L.n_hop + o] = sm[L.s_rat + o];
    if (lane == 0) {
      ev[4 * (size_t)w] = e.bbar;
      ev[4 * (size_t)w + 1] = e.vsf;
      ev[4 * (size_t)w + 2] = e.W;
      ev[4 * (size_t)w + 3] = e.eL;
      if (n_node) n_node[w] = sing ? -1 : e.n_node;
    }
    __syncwarp();
  }
}

// One branching interval for every walker (Algorithm 2 for kind 1,
// Algorithm 1 for kind 0).  The walker state stays in shared memory for the
// whole interval.  On the fixed lattice the caches of the incremental
// evaluation persist in the walker's cache block from one interval to the
// next, so every hop is evaluated incrementally; without valid caches (new
// walkers after a failed inversion, or a stored evaluation from a randomised
// lattice) the first hop evaluates in full.  A randomised interval draws new
// versors and evaluates in full at its start.
// One walker's interval (the body of k_propagate, also run by the batched
// kernel): w is the walker index within its system, sm the warp's region.
template <bool ROT, bool GG>
__device__ void propagate_walker_impl(const DevSys& S, const Layout& L, double* __restrict__ state,
                                      double* __restrict__ cache, int w, const StepParams& P, const double* T,
                                      double* sm, const Scr& wscr, int lane) {
  double* sc = sm + L.s_sc;
  const double ia = 1.0 / P.a;
  {
    const unsigned long long t_start = global_ns();
    double* gblk = state + (size_t)w * L.g_stride;
    double* cblk = cache + (size_t)w * L.c_stride;
    const Scr scr = walker_scratch(L, cblk, wscr);
    load_block(L, gblk, sm, lane);
    const bool rotated_before = sc[SC_ROTATED] != 0.0;
    bool cached = !ROT && !rotated_before && sc[SC_CACHE] != 0.0;
    if (cached) load_mirror(L, cblk, sm, lane);
    bool g_valid = cached;
    if (ROT || rotated_before) {
      // new versors (or the Cartesian axes again): the stored evaluation used others
      if (ROT && lane == 0) interval_versors(P.seed, (uint32_t)w, P.interval, sm + L.s_v);
      __syncwarp();
      compute_g(S, L, sm, scr.g, 0, L.n_e, lane);
      const EvalOut e0 = eval_full<ROT, GG>(S, L, gblk, sm, scr, P.a, P.node_rule, T, lane);
      g_valid = cached = true;
      if (lane == 0) {
        sc[SC_BBAR] = e0.bbar;
        sc[SC_VSF] = e0.vsf;
        sc[SC_WDIAG] = e0.W;
        sc[SC_EL] = e0.eL;
        sc[SC_NNODE] = e0.n_node;
        sc[SC_KEPT] = e0.kept;
      }
      __syncwarp();
    }
    double weight = 1.0, tau_left = P.tau;
    double bbar = sc[SC_BBAR], Wd = sc[SC_WDIAG], eL = sc[SC_EL], kept = sc[SC_KEPT];
    uint32_t status = (uint32_t)sc[SC_STATUS];
    int moves = 0, since = (int)sc[SC_SINCE];
    for (int k = 0;; ++k) {
      if (P.kind == 1 && k >= P.n_proj) break;
      double u_tau, u_move;
      step_uniforms(P.seed, (uint32_t)w, (uint32_t)k, P.interval, u_tau, u_move);
      if (P.kind == 1) {
        // w <- w b_x, b_x = b_bar / (W - E_0)
        const double den = Wd - P.E0;
        if (dpos(den)) {
          // refined reciprocal (a few ulp) instead of the FP64 division's longer sequence
          weight *= dge_nonneg(den, 0x1p-1000) ? bbar * rcp_nr(den) : bbar / den;
        } else {
          weight *= 0.0;
          status |= ST_NEG_DIAG;
        }
      } else {
        // tau_xi = min(-ln(1 - xi) / b_bar, tau_left); w <- w exp(-tau_xi e_L)
        double t = -log(1.0 - u_tau) / bbar;
        const bool clipped = !(t < tau_left);
        if (clipped) t = tau_left;
        weight *= exp_tab(-t * eL, T);
        tau_left -= t;
        if (clipped) break;
      }
      const int p = choose_hop(sm + L.s_rat, L.n_hop, u_move, kept, lane);
      if (p < 0) {
        status |= ST_STUCK;
      } else {
        if (!g_valid) {
          compute_g(S, L, sm, scr.g, 0, L.n_e, lane);
          g_valid = true;
        }
        apply_hop<ROT>(S, L, gblk, sm, scr, p, P.a, ia, !cached, T, lane);
        ++moves;
        bool reinv = false;
        // drift check between the periodic inversions (the moved row of A is
        // already in the cache)
        const bool drift = P.drift_tol > 0.0 && since + 1 < P.reinv_period && (since + 1) % DRIFT_EVERY == 0 &&
                           !(inverse_residual(L, gblk + L.g_cache, 5 * L.n_max, sm + L.s_bt, p / 6, lane) <=
                             P.drift_tol);
        if (++since >= P.reinv_period || drift) {
          if (reinvert(L, gblk, sm, scr.gj, lane)) status |= ST_SINGULAR;
          compute_g(S, L, sm, scr.g, 0, L.n_e, lane);
          since = 0;
          reinv = true;
          if (drift) {
            status |= ST_DRIFT;
            if (lane == 0 && P.drift_count) atomicAdd(P.drift_count, 1);
          }
        }
        EvalOut e;
        if (!cached) {
          e = eval_full<ROT, GG>(S, L, gblk, sm, scr, P.a, P.node_rule, T, lane);
          cached = true;
        } else {
          e = eval_incr<ROT, GG>(S, L, gblk, sm, scr, p / 6, reinv, P.a, ia, P.node_rule, T, lane);
        }
        bbar = e.bbar;
        Wd = e.W;
        eL = e.eL;
        kept = e.kept;
        if (lane == 0) {
          sc[SC_BBAR] = e.bbar;
          sc[SC_VSF] = e.vsf;
          sc[SC_WDIAG] = e.W;
          sc[SC_EL] = e.eL;
          sc[SC_NNODE] = e.n_node;
          sc[SC_KEPT] = e.kept;
        }
      }
      if (P.kind == 0 && k + 1 >= P.max_moves) {
        status |= ST_STEP_CAP;
        break;
      }
    }
    if (!isfinite(weight) || !isfinite(eL)) status |= ST_NONFINITE;
    const bool keep = !ROT && cached && !(status & ST_SINGULAR);
    if (lane == 0) {
      sc[SC_W] = weight;
      sc[SC_STATUS] = (double)status;
      sc[SC_MOVES] = moves;
      sc[SC_SINCE] = since;
      sc[SC_CACHE] = keep ? 1.0 : 0.0;
      sc[SC_ROTATED] = ROT ? 1.0 : 0.0;
    }
    store_block(L, gblk, sm, lane);
    if (keep) store_mirror(L, cblk, sm, lane);
    if (P.stamps && lane == 0) {
      P.stamps[3 * (size_t)w] = t_start;
      P.stamps[3 * (size_t)w + 1] = global_ns();
      P.stamps[3 * (size_t)w + 2] = sm_id();
    }
  }
}

template <bool ROT>
__device__ __forceinline__ void propagate_walker(const DevSys& S, const Layout& L, double* __restrict__ state,
                                                 double* __restrict__ cache, int w, const StepParams& P,
                                                 const double* T, double* sm, const Scr& wscr, int lane) {
  if (L.geo_glob) propagate_walker_impl<ROT, true>(S, L, state, cache, w, P, T, sm, wscr, lane);
  else propagate_walker_impl<ROT, false>(S, L, state, cache, w, P, T, sm, wscr, lane);
}

// Body of the propagate kernels.  GSM: the warps' working sets live in global
// memory (gsm + slot * s_stride) instead of shared memory; used for systems
// whose shared layout would let only a few warps share an SM (their O(N^2)
// caches are in global memory too).
template <bool ROT, bool GSM>
__device__ __forceinline__ void propagate_kernel_body(const DevSys& S, const Layout& L, double* __restrict__ state,
                                                      double* __restrict__ cache, int n_w, const StepParams& P,
                                                      double* scratch, double* gsm) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  double* sm = GSM ? gsm + (size_t)slot * L.s_stride : smem + EXP_TAB + wib * L.s_stride;
  const Scr wscr = warp_scratch(L, S.n_nuc, scratch, slot);
  for (int w = slot; w < n_w; w = next_walker(P, w, nwarps, lane))
    propagate_walker<ROT>(S, L, state, cache, w, P, T, sm, wscr, lane);
}

template <bool ROT>
__global__ void k_propagate(DevSys S, Layout L, double* __restrict__ state, double* __restrict__ cache, int n_w,
                            StepParams P, double* scratch) {
  propagate_kernel_body<ROT, false>(S, L, state, cache, n_w, P, scratch, nullptr);
}

// Working sets in global memory: 4-warp CTAs, as many as the registers allow;
// at most 128 registers per thread keep 4 CTAs (16 warps) per SM.
template <bool ROT>
__global__ void __maxnreg__(128) k_propagate_g(DevSys S, Layout L, double* __restrict__ state,
                                               double* __restrict__ cache, int n_w, StepParams P, double* scratch,
                                               double* gsm) {
  propagate_kernel_body<ROT, true>(S, L, state, cache, n_w, P, scratch, gsm);
}

// Compact copies of walker fields (for host readback); a null output is skipped.
__global__ void k_extract(Layout L, const double* __restrict__ state, int n_w, double* __restrict__ x,
                          double* __restrict__ w, double* __restrict__ ev, double* __restrict__ rat,
                          uint32_t* __restrict__ st, int32_t* __restrict__ mv) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  if (x)
    for (int idx = tid; idx < n_w * 3 * L.n_e; idx += nth) {
      const int a = idx / (3 * L.n_e), o = idx - a * 3 * L.n_e;
      x[idx] = state[(size_t)a * L.g_stride + L.g_x + o];
    }
  if (rat)
    for (int idx = tid; idx < n_w * L.n_hop; idx += nth) {
      const int a = idx / L.n_hop, o = idx - a * L.n_hop;
      rat[idx] = state[(size_t)a * L.g_stride + L.g_rat + o];
    }
  for (int a = tid; a < n_w; a += nth) {
    const double* sc = state + (size_t)a * L.g_stride + L.g_sc;
    if (w) w[a] = sc[SC_W];
    if (ev) {
      ev[4 * a] = sc[SC_BBAR];
      ev[4 * a + 1] = sc[SC_VSF];
      ev[4 * a + 2] = sc[SC_WDIAG];
      ev[4 * a + 3] = sc[SC_EL];
    }
    if (st) st[a] = (uint32_t)sc[SC_STATUS];
    if (mv) mv[a] = (int32_t)sc[SC_MOVES];
  }
}

__global__ void k_fp64math(int n, const double* __restrict__ x, double* __restrict__ e, double* __restrict__ r,
                           double* __restrict__ q, const double* __restrict__ tab) {
  __shared__ double T[EXP_TAB];
  for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) T[j] = tab[j];
  __syncthreads();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double v = x[k];
    if (e) e[k] = exp_tab(v, T);
    if (r) r[k] = rcp_nr(v);
    if (q) q[k] = rsqrt_nr(v);
  }
}

// erf(r/r_c)/r at s = r^2 through the table of erf_over_r (testing aid).
__global__ void k_erf_over_r(int n, const double* __restrict__ s, double irc, double irc2, double* __restrict__ out,
                             const double* __restrict__ C) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = erf_over_r(s[k], rsqrt_nr(s[k]), irc, irc2, C);
}

// Set walker scalar idx of every walker to v.
__global__ void k_set_scalar(Layout L, double* __restrict__ state, int n_w, int idx, double v) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_w; a += gridDim.x * blockDim.x)
    state[(size_t)a * L.g_stride + L.g_sc + idx] = v;
}

}  // namespace lrdmc
