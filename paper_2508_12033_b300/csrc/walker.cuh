// Warp-per-walker FP64 kernels of the LRDMC projection step.
//
// One warp owns one walker at a time.  Its working set (positions, the
// transposed inverse Slater matrices B^T, the per-electron orbital
// value/gradient/Laplacian cache, the 6 N_e hop ratios, per-electron
// Jastrow/potential terms and scratch) lives in shared memory for a whole
// branching interval; HBM is touched only when the walker is loaded and
// stored.  The FP64 pipe is the bound, so the formulation minimises FP64
// operations:
//   * the determinant ratio of hop (i, d) is chi(r') . g_i with
//     g_i = C^T B[:, i] precomputed once per electron (N_bf dot per hop
//     instead of an N_bf x N_orb contraction followed by an N_orb dot);
//   * the Jastrow ratio needs only the displaced electron's pair terms;
//   * Sherman-Morrison keeps B = A^{-1} current after each hop, with a
//     from-scratch Gauss-Jordan inversion every reinv_period hops.
#pragma once

#include "common.cuh"

namespace lrdmc {

// ------------------------------------------------------------ basis functions
// Sum over basis functions of chi_mu(p) * g[mu] for one point.
__device__ __forceinline__ double basis_dot(const DevSys& S, double px, double py, double pz,
                                            const double* __restrict__ g) {
  double acc = 0.0;
  for (int s = 0; s < S.n_shell; ++s) {
    const int atom = __ldg(S.sh_atom + s);
    const int l = __ldg(S.sh_l + s);
    const int np = __ldg(S.sh_nprim + s);
    const int off = __ldg(S.sh_off + s);
    const int bf = __ldg(S.sh_bf + s);
    const double dx = px - __ldg(S.R + 3 * atom);
    const double dy = py - __ldg(S.R + 3 * atom + 1);
    const double dz = pz - __ldg(S.R + 3 * atom + 2);
    const double r2 = dx * dx + dy * dy + dz * dz;
    double rad = 0.0;
    if (l == -1) {
      const double r = sqrt(r2);
      for (int q = 0; q < np; ++q) rad += __ldg(S.coefs + off + q) * exp(-__ldg(S.exps + off + q) * r);
      acc += rad * g[bf];
    } else {
      for (int q = 0; q < np; ++q) rad += __ldg(S.coefs + off + q) * exp(-__ldg(S.exps + off + q) * r2);
      if (l == 0)
        acc += rad * g[bf];
      else
        acc += rad * (dx * g[bf] + dy * g[bf + 1] + dz * g[bf + 2]);
    }
  }
  return acc;
}

// Value, gradient and Laplacian of the functions of shell s at a point:
// out[c * n_bf + mu], c = 0 value, 1..3 gradient, 4 Laplacian.
__device__ __forceinline__ void shell_derivs(const DevSys& S, int s, double px, double py,
                                             double pz, double* __restrict__ out, int n_bf) {
  const int atom = __ldg(S.sh_atom + s);
  const int l = __ldg(S.sh_l + s);
  const int np = __ldg(S.sh_nprim + s);
  const int off = __ldg(S.sh_off + s);
  const int bf = __ldg(S.sh_bf + s);
  const double d[3] = {px - __ldg(S.R + 3 * atom), py - __ldg(S.R + 3 * atom + 1),
                       pz - __ldg(S.R + 3 * atom + 2)};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (l == -1) {
    // h = c exp(-z r): grad = h' d / r, lap = (z^2 - 2 z / r) h
    const double r = sqrt(r2);
    double v = 0.0, dr = 0.0, lp = 0.0;
    for (int q = 0; q < np; ++q) {
      const double z = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp(-z * r);
      v += h;
      dr += -z * h;
      lp += (z * z - 2.0 * z / r) * h;
    }
    out[bf] = v;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = dr * d[m] / r;
    out[4 * n_bf + bf] = lp;
  } else if (l == 0) {
    // h = c exp(-a r^2): grad = -2a d h, lap = (4 a^2 r^2 - 6 a) h
    double v = 0.0, gs = 0.0, lp = 0.0;
    for (int q = 0; q < np; ++q) {
      const double al = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp(-al * r2);
      v += h;
      gs += -2.0 * al * h;
      lp += (4.0 * al * al * r2 - 6.0 * al) * h;
    }
    out[bf] = v;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = gs * d[m];
    out[4 * n_bf + bf] = lp;
  } else {
    // d_m h: grad_n = delta_mn h - 2a d_m d_n h, lap = d_m (4a^2 r^2 - 10 a) h
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int q = 0; q < np; ++q) {
      const double al = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp(-al * r2);
      s0 += h;
      s1 += -2.0 * al * h;
      s2 += (4.0 * al * al * r2 - 10.0 * al) * h;
    }
    for (int m = 0; m < 3; ++m) {
      out[bf + m] = d[m] * s0;
      for (int n = 0; n < 3; ++n)
        out[(1 + n) * n_bf + bf + m] = (m == n ? s0 : 0.0) + d[m] * d[n] * s1;
      out[4 * n_bf + bf + m] = d[m] * s2;
    }
  }
}

// Orbital value/gradient/Laplacian of the first n_sig orbitals at one point:
// phi5[c * n_max + k].  Warp-cooperative; chi5 is scratch of 5 * n_bf doubles.
__device__ void orbital_derivs(const DevSys& S, const Layout& L, double px, double py, double pz,
                               int n_sig, double* chi5, double* phi5, int lane) {
  for (int s = lane; s < S.n_shell; s += WARP) shell_derivs(S, s, px, py, pz, chi5, L.n_bf);
  __syncwarp();
  for (int o = lane; o < 5 * n_sig; o += WARP) {
    const int c = o / n_sig, k = o - c * n_sig;
    const double* crow = S.C + (size_t)k * L.n_bf;
    const double* x = chi5 + c * L.n_bf;
    double acc = 0.0;
    for (int mu = 0; mu < L.n_bf; ++mu) acc += __ldg(crow + mu) * x[mu];
    phi5[c * L.n_max + k] = acc;
  }
  __syncwarp();
}

// ------------------------------------------------------------ Gauss-Jordan
// In-place inversion of the N x N matrix held as the left half of M = [A | I]
// (N x 2N, row-major) with partial pivoting; afterwards the right half is
// A^{-1}.  Returns true on a zero (or non-finite) pivot.
__device__ bool warp_gauss_jordan(double* M, int N, int lane) {
  const int W2 = 2 * N;
  for (int c = 0; c < N; ++c) {
    double best = -1.0;
    int bi = N;
    for (int r = c + lane; r < N; r += WARP) {
      const double v = fabs(M[r * W2 + c]);
      if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(FULL, best, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > 0.0) || !isfinite(best)) return true;
    if (bi != c) {
      for (int j = lane; j < W2; j += WARP) {
        const double t = M[c * W2 + j];
        M[c * W2 + j] = M[bi * W2 + j];
        M[bi * W2 + j] = t;
      }
    }
    __syncwarp();
    const double inv = 1.0 / M[c * W2 + c];
    __syncwarp();
    for (int j = lane; j < W2; j += WARP) M[c * W2 + j] *= inv;
    __syncwarp();
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = M[r * W2 + c];
      __syncwarp();
      if (f != 0.0)
        for (int j = lane; j < W2; j += WARP) M[r * W2 + j] -= f * M[c * W2 + j];
      __syncwarp();
    }
  }
  return false;
}

// B^T of both spin blocks from the cached orbital values A[i][k] = phi_k(r_i).
// scratch: >= 2 n_max^2 doubles.  Returns true if a block is singular.
__device__ bool reinvert(const Layout& L, double* sm, double* scratch, int lane) {
  bool sing = false;
  const double* cache = sm + L.s_cache;
  double* bt = sm + L.s_bt;
  for (int blk = 0; blk < 2; ++blk) {
    const int n = blk ? L.n_dn : L.n_up;
    const int e0 = blk ? L.n_up : 0;
    const int bto = blk ? L.n_up * L.n_up : 0;
    if (n == 0) continue;
    for (int o = lane; o < n * 2 * n; o += WARP) {
      const int r = o / (2 * n), c = o - r * 2 * n;
      scratch[o] = c < n ? cache[(e0 + r) * 5 * L.n_max + c] : (c - n == r ? 1.0 : 0.0);
    }
    __syncwarp();
    sing |= warp_gauss_jordan(scratch, n, lane);
    // B = right half; B^T[i][k] = B[k][i]
    for (int o = lane; o < n * n; o += WARP) {
      const int i = o / n, k = o - i * n;
      bt[bto + o] = scratch[k * 2 * n + n + i];
    }
    __syncwarp();
  }
  return sing;
}

// ------------------------------------------------------------ evaluation
struct EvalOut {
  double bbar, vsf, W, eL;
  int n_node;
};

// Evaluate the lattice-regularised FN Hamiltonian at the walker's current
// configuration (Appendix D): all hop ratios, b_bar, V_sf, W and e_L.
// Requires x, B^T and the orbital cache in shared memory; writes the ratios.
__device__ EvalOut eval_walker(const DevSys& S, const Layout& L, double* sm, double a,
                               int node_rule, int lane) {
  const int ne = L.n_e, nbf = L.n_bf, nmax = L.n_max;
  const double* x = sm + L.s_x;
  const double* bt = sm + L.s_bt;
  const double* cache = sm + L.s_cache;
  double* g = sm + L.s_g;
  double* rat = sm + L.s_rat;
  double* ej = sm + L.s_ej;   // per electron: U_i (Jastrow sum), lap_i Psi/Psi
  double* ep = sm + L.s_ep;   // per electron: nu_ei, nu^a_ei, half e-e sum

  // (1) per-electron Jastrow sums and derivatives, potentials, lap Psi / Psi
  for (int i = lane; i < ne; i += WARP) {
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const bool up_i = i < L.n_up;
    double U = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, LJ = 0.0, vee = 0.0;
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      const double dx = xi - x[3 * j], dy = yi - x[3 * j + 1], dz = zi - x[3 * j + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double c = (up_i == (j < L.n_up)) ? S.j2_par : S.j2_anti;
      const double t = 1.0 / (1.0 + S.j2_b * r);
      U += c * r * t;
      const double up = c * t * t;
      const double upp = -2.0 * S.j2_b * c * t * t * t;
      const double ir = 1.0 / r;
      gx += up * ir * dx; gy += up * ir * dy; gz += up * ir * dz;
      LJ += upp + 2.0 * up * ir;
      vee += 0.5 * ir;
    }
    double nu = 0.0, nucap = 0.0;
    for (int I = 0; I < S.n_nuc; ++I) {
      const double dx = xi - __ldg(S.R + 3 * I), dy = yi - __ldg(S.R + 3 * I + 1),
                   dz = zi - __ldg(S.R + 3 * I + 2);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double A = __ldg(S.j1A + I), B = __ldg(S.j1B + I);
      const double t = 1.0 / (1.0 + B * r);
      U -= A * r * t;
      const double vp = -A * t * t;
      const double vpp = 2.0 * A * B * t * t * t;
      const double ir = 1.0 / r;
      gx += vp * ir * dx; gy += vp * ir * dy; gz += vp * ir * dz;
      LJ += vpp + 2.0 * vp * ir;
      const double Z = __ldg(S.Z + I);
      if (__ldg(S.kind + I) == 0) {
        nu -= Z * ir;
        nucap -= Z / fmax(r, a);
      } else {
        const double v = -Z * erf(r / __ldg(S.rc + I)) * ir;
        nu += v;
        nucap += v;
      }
    }
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    const double* ce = cache + i * 5 * nmax;
    double dgx = 0.0, dgy = 0.0, dgz = 0.0, dl = 0.0;
    for (int k = 0; k < sr.n; ++k) {
      const double b = brow[k];
      dgx += ce[1 * nmax + k] * b;
      dgy += ce[2 * nmax + k] * b;
      dgz += ce[3 * nmax + k] * b;
      dl += ce[4 * nmax + k] * b;
    }
    const double lap = dl + 2.0 * (dgx * gx + dgy * gy + dgz * gz) + LJ + (gx * gx + gy * gy + gz * gz);
    ej[2 * i] = U;
    ej[2 * i + 1] = lap;
    ep[3 * i] = nu;
    ep[3 * i + 1] = nucap;
    ep[3 * i + 2] = vee;
  }
  // (2) g_i = C^T B[:, i]
  for (int o = lane; o < ne * nbf; o += WARP) {
    const int i = o / nbf, mu = o - i * nbf;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc += __ldg(S.C + (size_t)k * nbf + mu) * brow[k];
    g[o] = acc;
  }
  __syncwarp();
  // (3) every hop: determinant ratio chi(r') . g_i times the Jastrow ratio
  for (int p = lane; p < 6 * ne; p += WARP) {
    const int i = p / 6, d = p - 6 * i;
    double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    q[d >> 1] += (d & 1) ? -a : a;
    const double det = basis_dot(S, q[0], q[1], q[2], g + i * nbf);
    const bool up_i = i < L.n_up;
    double Up = 0.0;
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      const double dx = q[0] - x[3 * j], dy = q[1] - x[3 * j + 1], dz = q[2] - x[3 * j + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double c = (up_i == (j < L.n_up)) ? S.j2_par : S.j2_anti;
      Up += c * r / (1.0 + S.j2_b * r);
    }
    for (int I = 0; I < S.n_nuc; ++I) {
      const double dx = q[0] - __ldg(S.R + 3 * I), dy = q[1] - __ldg(S.R + 3 * I + 1),
                   dz = q[2] - __ldg(S.R + 3 * I + 2);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      Up -= __ldg(S.j1A + I) * r / (1.0 + __ldg(S.j1B + I) * r);
    }
    rat[p] = det * exp(Up - ej[2 * i]);
  }
  __syncwarp();
  // (4) fixed-node split and regularised potential per electron
  bool has_node = false;
  for (int i = lane; i < ne; i += WARP)
    for (int d = 0; d < 6; ++d) has_node |= rat[6 * i + d] < 0.0;
  const bool any_node = __any_sync(FULL, has_node);
  double kept = 0.0, negs = 0.0, nuopt = 0.0, vee = 0.0;
  int nn = 0;
  const double ia2 = 1.0 / (a * a);
  for (int i = lane; i < ne; i += WARP) {
    double sr = 0.0;
    bool node = false;
    for (int d = 0; d < 6; ++d) {
      const double r = rat[6 * i + d];
      sr += r;
      if (r > 0.0) kept += r;
      if (r < 0.0) { negs -= r; node = true; }
    }
    const double nu_zv = ep[3 * i] + 0.5 * ((sr - 6.0) * ia2 - ej[2 * i + 1]);
    bool apply;
    if (node_rule == 0) apply = node;
    else if (node_rule == 1) apply = any_node;
    else if (node_rule == 2) apply = true;
    else apply = false;
    nuopt += apply ? fmax(nu_zv, ep[3 * i + 1]) : nu_zv;
    vee += ep[3 * i + 2];
    nn += node ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kept += __shfl_xor_sync(FULL, kept, o);
    negs += __shfl_xor_sync(FULL, negs, o);
    nuopt += __shfl_xor_sync(FULL, nuopt, o);
    vee += __shfl_xor_sync(FULL, vee, o);
    nn += __shfl_xor_sync(FULL, nn, o);
  }
  EvalOut e;
  const double i2a2 = 0.5 * ia2;
  e.bbar = kept * i2a2;
  e.vsf = negs * i2a2;
  e.W = 3.0 * ne * ia2 + nuopt + vee + S.v_ii + e.vsf;
  e.eL = e.W - e.bbar;
  e.n_node = nn;
  return e;
}

// Build the orbital cache at every electron, invert both Slater blocks and
// evaluate.  x must already be in shared memory.
__device__ EvalOut init_walker(const DevSys& S, const Layout& L, double* sm, double a,
                               int node_rule, int lane, bool& singular) {
  double* chi5 = sm + L.s_chi5;
  double* phi5 = sm + L.s_phi5;
  double* cache = sm + L.s_cache;
  const double* x = sm + L.s_x;
  for (int i = 0; i < L.n_e; ++i) {
    const int n = i < L.n_up ? L.n_up : L.n_dn;
    orbital_derivs(S, L, x[3 * i], x[3 * i + 1], x[3 * i + 2], n, chi5, phi5, lane);
    for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
    __syncwarp();
  }
  singular = reinvert(L, sm, sm + L.s_g, lane);
  return eval_walker(S, L, sm, a, node_rule, lane);
}

// Heat-bath choice over the kept hops (r > 0) in the order p = 6 i + d: the
// first p whose running sum exceeds u * total; the last kept hop if rounding
// leaves none; -1 without kept hops.  Sequential sum, as the method states it.
__device__ int choose_hop(const double* rat, int n_hop, double u, int lane) {
  int choice = -1;
  if (lane == 0) {
    double total = 0.0;
    for (int p = 0; p < n_hop; ++p) total += rat[p] > 0.0 ? rat[p] : 0.0;
    if (total > 0.0) {
      const double t = u * total;
      double run = 0.0;
      int last = -1;
      for (int p = 0; p < n_hop; ++p) {
        const double k = rat[p] > 0.0 ? rat[p] : 0.0;
        if (k > 0.0) last = p;
        run += k;
        if (run > t) { choice = p; break; }
      }
      if (choice < 0) choice = last;
    }
  }
  return __shfl_sync(FULL, choice, 0);
}

// Apply hop p: new orbital derivatives at the moved electron, Sherman-Morrison
// update of its spin block, cache and position update.
__device__ void apply_hop(const DevSys& S, const Layout& L, double* sm, int p, double a, int lane) {
  double* x = sm + L.s_x;
  double* bt = sm + L.s_bt;
  double* cache = sm + L.s_cache;
  double* phi5 = sm + L.s_phi5;
  double* u = sm + L.s_u;
  double* row = sm + L.s_row;
  const int i = p / 6, d = p - 6 * i;
  double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  q[d >> 1] += (d & 1) ? -a : a;
  const SpinRef sr = spin_ref(L, i);
  orbital_derivs(S, L, q[0], q[1], q[2], sr.n, sm + L.s_chi5, phi5, lane);
  double* B = bt + sr.bt_off;   // B^T of the spin block: B[j * n + k] = (A^{-1})_{k j}
  const int n = sr.n;
  // u_j = phi(r') . B[:, j]; the determinant ratio is u_ii
  for (int j = lane; j < n; j += WARP) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += phi5[k] * B[j * n + k];
    u[j] = acc;
  }
  for (int k = lane; k < n; k += WARP) row[k] = B[sr.ii * n + k];
  __syncwarp();
  // A' = A + e_i (phi' - phi)^T  =>  B' = B - B e_i (u - e_i)^T / u_i
  const double invR = 1.0 / u[sr.ii];
  for (int o = lane; o < n * n; o += WARP) {
    const int j = o / n, k = o - j * n;
    const double f = (u[j] - (j == sr.ii ? 1.0 : 0.0)) * invR;
    B[o] -= row[k] * f;
  }
  for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
  if (lane == 0) {
    x[3 * i] = q[0];
    x[3 * i + 1] = q[1];
    x[3 * i + 2] = q[2];
  }
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
};

__device__ __forceinline__ void load_block(const Layout& L, const double* __restrict__ g, double* sm,
                                           int lane) {
  for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = g[L.g_x + o];
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) sm[L.s_bt + o] = g[L.g_bt + o];
  for (int o = lane; o < 5 * L.n_max * L.n_e; o += WARP) sm[L.s_cache + o] = g[L.g_cache + o];
  for (int o = lane; o < L.n_hop; o += WARP) sm[L.s_rat + o] = g[L.g_rat + o];
  for (int o = lane; o < SC_COUNT; o += WARP) sm[L.s_sc + o] = g[L.g_sc + o];
  __syncwarp();
}

__device__ __forceinline__ void store_block(const Layout& L, double* __restrict__ g, const double* sm,
                                            int lane) {
  __syncwarp();
  for (int o = lane; o < 3 * L.n_e; o += WARP) g[L.g_x + o] = sm[L.s_x + o];
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) g[L.g_bt + o] = sm[L.s_bt + o];
  for (int o = lane; o < 5 * L.n_max * L.n_e; o += WARP) g[L.g_cache + o] = sm[L.s_cache + o];
  for (int o = lane; o < L.n_hop; o += WARP) g[L.g_rat + o] = sm[L.s_rat + o];
  for (int o = lane; o < SC_COUNT; o += WARP) g[L.g_sc + o] = sm[L.s_sc + o];
}

// Place walkers at x_in (n x n_e x 3), build caches, invert and evaluate.
__global__ void k_init_walkers(DevSys S, Layout L, double* __restrict__ state,
                               const double* __restrict__ x_in, const double* __restrict__ w_in,
                               int n, double a, int node_rule) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, sm, a, node_rule, lane, sing);
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
    }
    store_block(L, state + (size_t)w * L.g_stride, sm, lane);
  }
}

// Evaluate arbitrary configurations without touching the walkers.
__global__ void k_eval_configs(DevSys S, Layout L, const double* __restrict__ x_in, int n, double a,
                               int node_rule, double* __restrict__ ratios, double* __restrict__ ev,
                               int32_t* __restrict__ n_node) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, sm, a, node_rule, lane, sing);
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
// whole interval.
__global__ void k_propagate(DevSys S, Layout L, double* __restrict__ state, int n_w, StepParams P) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + wib * L.s_stride;
  double* sc = sm + L.s_sc;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n_w; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    load_block(L, gblk, sm, lane);
    double weight = 1.0, tau_left = P.tau;
    double bbar = sc[SC_BBAR], Wd = sc[SC_WDIAG], eL = sc[SC_EL];
    uint32_t status = (uint32_t)sc[SC_STATUS];
    int moves = 0, since = (int)sc[SC_SINCE];
    for (int k = 0;; ++k) {
      if (P.kind == 1 && k >= P.n_proj) break;
      double u_tau, u_move;
      step_uniforms(P.seed, (uint32_t)w, (uint32_t)k, P.interval, u_tau, u_move);
      if (P.kind == 1) {
        // w <- w b_x, b_x = b_bar / (W - E_0)
        const double den = Wd - P.E0;
        if (den > 0.0) {
          weight *= bbar / den;
        } else {
          weight *= 0.0;
          status |= ST_NEG_DIAG;
        }
      } else {
        // tau_xi = min(-ln(1 - xi) / b_bar, tau_left); w <- w exp(-tau_xi e_L)
        double t = -log(1.0 - u_tau) / bbar;
        const bool clipped = !(t < tau_left);
        if (clipped) t = tau_left;
        weight *= exp(-t * eL);
        tau_left -= t;
        if (clipped) break;
      }
      const int p = choose_hop(sm + L.s_rat, L.n_hop, u_move, lane);
      if (p < 0) {
        status |= ST_STUCK;
      } else {
        apply_hop(S, L, sm, p, P.a, lane);
        ++moves;
        if (++since >= P.reinv_period) {
          if (reinvert(L, sm, sm + L.s_g, lane)) status |= ST_SINGULAR;
          since = 0;
        }
        const EvalOut e = eval_walker(S, L, sm, P.a, P.node_rule, lane);
        bbar = e.bbar;
        Wd = e.W;
        eL = e.eL;
        if (lane == 0) {
          sc[SC_BBAR] = e.bbar;
          sc[SC_VSF] = e.vsf;
          sc[SC_WDIAG] = e.W;
          sc[SC_EL] = e.eL;
          sc[SC_NNODE] = e.n_node;
        }
      }
      if (P.kind == 0 && k + 1 >= P.max_moves) {
        status |= ST_STEP_CAP;
        break;
      }
    }
    if (!isfinite(weight) || !isfinite(eL)) status |= ST_NONFINITE;
    if (lane == 0) {
      sc[SC_W] = weight;
      sc[SC_STATUS] = (double)status;
      sc[SC_MOVES] = moves;
      sc[SC_SINCE] = since;
    }
    store_block(L, gblk, sm, lane);
  }
}

// Compact copies of walker fields (for host readback).
__global__ void k_extract(Layout L, const double* __restrict__ state, int n_w, double* __restrict__ x,
                          double* __restrict__ w, double* __restrict__ ev, double* __restrict__ rat,
                          double* __restrict__ st, double* __restrict__ mv) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int idx = tid; idx < n_w * 3 * L.n_e; idx += nth) {
    const int a = idx / (3 * L.n_e), o = idx - a * 3 * L.n_e;
    x[idx] = state[(size_t)a * L.g_stride + L.g_x + o];
  }
  for (int idx = tid; idx < n_w * L.n_hop; idx += nth) {
    const int a = idx / L.n_hop, o = idx - a * L.n_hop;
    rat[idx] = state[(size_t)a * L.g_stride + L.g_rat + o];
  }
  for (int a = tid; a < n_w; a += nth) {
    const double* sc = state + (size_t)a * L.g_stride + L.g_sc;
    w[a] = sc[SC_W];
    ev[4 * a] = sc[SC_BBAR];
    ev[4 * a + 1] = sc[SC_VSF];
    ev[4 * a + 2] = sc[SC_WDIAG];
    ev[4 * a + 3] = sc[SC_EL];
    st[a] = sc[SC_STATUS];
    mv[a] = sc[SC_MOVES];
  }
}

__global__ void k_clear_status(Layout L, double* __restrict__ state, int n_w) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_w; a += gridDim.x * blockDim.x)
    state[(size_t)a * L.g_stride + L.g_sc + SC_STATUS] = 0.0;
}

}  // namespace lrdmc
