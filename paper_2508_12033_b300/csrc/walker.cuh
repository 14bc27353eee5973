// Warp-per-walker FP64 kernels of the LRDMC projection step.
//
// One warp owns one walker at a time.  Its working set (positions, the
// transposed inverse Slater matrices B^T, g_i = C^T B[:, i] for every
// electron, the 6 N_e hop ratios, per-electron Jastrow/potential terms and the
// electron-nucleus / electron-electron geometry of the current configuration)
// lives in shared memory for a whole branching interval.  The orbital
// value/gradient/Laplacian cache stays in the walker's global block (L2
// resident during the interval).  The FP64 pipe is the bound, so the
// formulation minimises FP64 work:
//   * determinant ratio of hop (i, d) = chi(r') . g_i (one N_bf dot per hop);
//     g is updated by the same rank-1 factors as B after each hop;
//   * |r' - R|^2 = (|r - R|^2 + a^2) + 2 (+-a) (r - R)_axis: distances are
//     formed once per (electron, nucleus) and per electron pair and shared by
//     the 6 hops and all shells on a nucleus;
//   * only the hopping electron's Jastrow pair terms enter its ratio;
//   * the pseudopotential of an electron is recomputed only when it hops;
//   * Sherman-Morrison keeps B = A^{-1} current, with a from-scratch
//     Gauss-Jordan inversion every reinv_period hops;
//   * exp / sqrt / reciprocal use the reduced-slot forms of fp64math.cuh.
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
  const int bf = __ldg(S.sh_bf + s);
  if (l == -1) {
    // h = c exp(-z r): grad = h' d / r, lap = (z^2 - 2 z / r) h
    const double ir = rsqrt_nr(r2);
    const double r = r2 * ir;
    double v = 0.0, dr = 0.0, lp = 0.0;
    for (int q = 0; q < np; ++q) {
      const double z = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp_tab(-z * r, T);
      v += h;
      dr += -z * h;
      lp += (z * z - 2.0 * z * ir) * h;
    }
    out[bf] = v;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = dr * d[m] * ir;
    out[4 * n_bf + bf] = lp;
  } else if (l == 0) {
    // h = c exp(-a r^2): grad = -2a d h, lap = (4 a^2 r^2 - 6 a) h
    double v = 0.0, gs = 0.0, lp = 0.0;
    for (int q = 0; q < np; ++q) {
      const double al = __ldg(S.exps + off + q);
      const double h = __ldg(S.coefs + off + q) * exp_tab(-al * r2, T);
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
      const double h = __ldg(S.coefs + off + q) * exp_tab(-al * r2, T);
      s0 += h;
      s1 += -2.0 * al * h;
      s2 += (4.0 * al * al * r2 - 10.0 * al) * h;
    }
    for (int m = 0; m < 3; ++m) {
      out[bf + m] = d[m] * s0;
      for (int n = 0; n < 3; ++n) out[(1 + n) * n_bf + bf + m] = (m == n ? s0 : 0.0) + d[m] * d[n] * s1;
      out[4 * n_bf + bf + m] = d[m] * s2;
    }
  }
}

// Orbital value/gradient/Laplacian of the first n_sig orbitals at point q:
// phi5[c * n_max + k].  Warp-cooperative; chi5 is scratch of 5 n_bf doubles.
__device__ void orbital_derivs(const DevSys& S, const Layout& L, const double q[3], int n_sig, double* chi5,
                               double* phi5, const double* T, int lane) {
  for (int s = lane; s < S.n_shell; s += WARP) {
    const int atom = __ldg(S.sh_atom + s);
    const double d[3] = {q[0] - __ldg(S.R + 3 * atom), q[1] - __ldg(S.R + 3 * atom + 1),
                         q[2] - __ldg(S.R + 3 * atom + 2)};
    shell_derivs(S, s, d, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], chi5, L.n_bf, T);
  }
  __syncwarp();
  for (int o = lane; o < 5 * n_sig; o += WARP) {
    const int c = o / n_sig, k = o - c * n_sig;
    const double* crow = S.C + (size_t)k * L.n_bf;
    const double* x = chi5 + c * L.n_bf;
    double acc = 0.0;
    for (int mu = 0; mu < L.n_bf; ++mu) acc = fma(__ldg(crow + mu), x[mu], acc);
    phi5[c * L.n_max + k] = acc;
  }
  __syncwarp();
}

// Bare and capped electron-nucleus potentials of one electron (Appendix D:
// nu_ei and nu^a_ei), warp-cooperative over nuclei; result valid in all lanes.
__device__ void electron_potentials(const DevSys& S, const double q[3], double a, int lane, double& nu,
                                    double& nucap) {
  nu = 0.0;
  nucap = 0.0;
  for (int I = lane; I < S.n_nuc; I += WARP) {
    const double dx = q[0] - __ldg(S.R + 3 * I), dy = q[1] - __ldg(S.R + 3 * I + 1),
                 dz = q[2] - __ldg(S.R + 3 * I + 2);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double Z = __ldg(S.Z + I);
    if (__ldg(S.kind + I) == 0) {
      nu -= Z / r;
      nucap -= Z / fmax(r, a);
    } else {
      const double v = -Z * erf(r / __ldg(S.rc + I)) / r;
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

// B^T of both spin blocks from the cached orbital values A[i][k] = phi_k(r_i)
// (walker block in global memory).  scratch: >= 2 n_max^2 doubles.  Returns
// true if a block is singular.
__device__ bool reinvert(const Layout& L, const double* __restrict__ gblk, double* sm, double* scratch, int lane) {
  bool sing = false;
  const double* cache = gblk + L.g_cache;
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
    for (int o = lane; o < n * n; o += WARP) {
      const int i = o / n, k = o - i * n;
      bt[bto + o] = scratch[k * 2 * n + n + i];
    }
    __syncwarp();
  }
  return sing;
}

// g_i = C^T B[:, i] for every electron.
__device__ void compute_g(const DevSys& S, const Layout& L, double* sm, int lane) {
  const double* bt = sm + L.s_bt;
  double* g = sm + L.s_g;
  for (int o = lane; o < L.n_e * L.n_bf; o += WARP) {
    const int i = o / L.n_bf, mu = o - i * L.n_bf;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc = fma(__ldg(S.C + (size_t)k * L.n_bf + mu), brow[k], acc);
    g[o] = acc;
  }
  __syncwarp();
}

// ------------------------------------------------------------ evaluation
struct EvalOut {
  double bbar, vsf, W, eL;
  int n_node;
};

// Pade pair term u = c r/(1 + b r) and its radial derivatives from s = r^2.
struct Pair {
  double u, up, upp, ir;
};
__device__ __forceinline__ Pair pade(double s, double c, double b) {
  Pair p;
  p.ir = rsqrt_nr(s);
  const double r = s * p.ir;
  const double t = rcp_nr(fma(b, r, 1.0));
  p.u = c * r * t;
  p.up = c * t * t;
  p.upp = -2.0 * b * p.up * t;
  return p;
}
__device__ __forceinline__ double pade_value(double s, double c, double b) {
  const double r = s * rsqrt_nr(s);
  return c * r * rcp_nr(fma(b, r, 1.0));
}

// Evaluate the lattice-regularised FN Hamiltonian at the walker's current
// configuration (Appendix D): all hop ratios, b_bar, V_sf, W and e_L.
// Requires x, B^T, the per-electron potentials in shared memory, the orbital
// cache in the global block, and g (recomputed here unless g_valid).
__device__ EvalOut eval_walker(const DevSys& S, const Layout& L, const double* __restrict__ gblk, double* sm,
                               double a, int node_rule, bool g_valid, const double* T, int lane) {
  const int ne = L.n_e, nbf = L.n_bf, nmax = L.n_max, nn = S.n_nuc;
  const double* x = sm + L.s_x;
  const double* bt = sm + L.s_bt;
  const double* cache = gblk + L.g_cache;
  double* g = sm + L.s_g;
  double* rat = sm + L.s_rat;
  double* ej = sm + L.s_ej;     // per electron: U_i, grad J (3), lap J, half e-e sum
  double* ep = sm + L.s_ep;     // per electron: nu_ei, nu^a_ei (kept across hops)
  double* geo = sm + L.s_geo;   // per (electron, nucleus): d (3), |d|^2 + a^2
  double* pr2 = sm + L.s_pr2;   // per electron pair: |r_i - r_j|^2 + a^2
  double* dd = sm + L.s_dd;     // per electron: grad D / D (3), lap D / D
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
        const bool up_e = e < L.n_up;
        for (int t = sub; t < per; t += G) {
          if (t < ne - 1) {
            const int j = t < e ? t : t + 1;
            const double dx = xe - x[3 * j], dy = ye - x[3 * j + 1], dz = ze - x[3 * j + 2];
            const double s = dx * dx + dy * dy + dz * dz;
            pr2[e * ne + j] = s + a2;
            const double c = (up_e == (j < L.n_up)) ? S.j2_par : S.j2_anti;
            const Pair p = pade(s, c, S.j2_b);
            const double f = p.up * p.ir;
            U += p.u;
            gx = fma(f, dx, gx); gy = fma(f, dy, gy); gz = fma(f, dz, gz);
            LJ += p.upp + 2.0 * f;
            vee = fma(0.5, p.ir, vee);
          } else {
            const int I = t - (ne - 1);
            const double dx = xe - __ldg(S.R + 3 * I), dy = ye - __ldg(S.R + 3 * I + 1),
                         dz = ze - __ldg(S.R + 3 * I + 2);
            const double s = dx * dx + dy * dy + dz * dz;
            double* gg = geo + (e * nn + I) * 4;
            gg[0] = dx; gg[1] = dy; gg[2] = dz; gg[3] = s + a2;
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
  // (1b) determinant derivatives grad_i D/D, lap_i D/D from the orbital cache
  for (int o = lane; o < 4 * ne; o += WARP) {
    const int i = o >> 2, c = o & 3;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    const double* ce = cache + i * 5 * nmax + (c + 1) * nmax;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc = fma(ce[k], brow[k], acc);
    dd[o] = acc;
  }
  // (2) g_i = C^T B[:, i] unless kept current by the rank-1 updates
  if (!g_valid) compute_g(S, L, sm, lane);
  __syncwarp();
  // (3) every hop: determinant ratio chi(r') . g_i times the Jastrow ratio
  for (int p = lane; p < 6 * ne; p += WARP) {
    const int i = p / 6, d = p - 6 * i, ax = d >> 1;
    const double sa = (d & 1) ? -a : a;
    const double s2a = sa + sa;
    const double* gi = g + i * nbf;
    double det = 0.0, Up = 0.0;
    for (int I = 0; I < nn; ++I) {
      const double* gg = geo + (i * nn + I) * 4;
      const double s = fma(s2a, gg[ax], gg[3]);            // |r' - R_I|^2
      double dv[3] = {gg[0], gg[1], gg[2]};
      dv[ax] += sa;
      const double A = __ldg(S.j1A + I);
      if (A != 0.0) Up += pade_value(s, -A, __ldg(S.j1B + I));
      for (int sh = __ldg(S.atom_sh + I); sh < __ldg(S.atom_sh + I + 1); ++sh) {
        const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh),
                  bf = __ldg(S.sh_bf + sh);
        double rad = 0.0;
        if (l == -1) {
          const double r = s * rsqrt_nr(s);
          for (int q = 0; q < np; ++q) rad = fma(__ldg(S.coefs + off + q), exp_tab(-__ldg(S.exps + off + q) * r, T), rad);
          det = fma(rad, gi[bf], det);
        } else {
          for (int q = 0; q < np; ++q) rad = fma(__ldg(S.coefs + off + q), exp_tab(-__ldg(S.exps + off + q) * s, T), rad);
          if (l == 0)
            det = fma(rad, gi[bf], det);
          else
            det = fma(rad, fma(dv[0], gi[bf], fma(dv[1], gi[bf + 1], dv[2] * gi[bf + 2])), det);
        }
      }
    }
    const bool up_i = i < L.n_up;
    const double xia = x[3 * i + ax];
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      const double s = fma(s2a, xia - x[3 * j + ax], pr2[i * ne + j]);
      const double c = (up_i == (j < L.n_up)) ? S.j2_par : S.j2_anti;
      Up += pade_value(s, c, S.j2_b);
    }
    rat[p] = det * exp_tab(Up - ej[6 * i], T);
  }
  __syncwarp();
  // (4) fixed-node split and regularised potential per electron
  bool has_node = false;
  for (int i = lane; i < ne; i += WARP)
    for (int d = 0; d < 6; ++d) has_node |= rat[6 * i + d] < 0.0;
  const bool any_node = __any_sync(FULL, has_node);
  double kept = 0.0, negs = 0.0, nuopt = 0.0, vee = 0.0;
  int nnode = 0;
  const double ia2 = 1.0 / a2;
  for (int i = lane; i < ne; i += WARP) {
    double sr = 0.0;
    bool node = false;
    for (int d = 0; d < 6; ++d) {
      const double r = rat[6 * i + d];
      sr += r;
      if (r > 0.0) kept += r;
      if (r < 0.0) { negs -= r; node = true; }
    }
    const double* q = ej + 6 * i;
    const double* dv = dd + 4 * i;
    const double lap = dv[3] + 2.0 * (dv[0] * q[1] + dv[1] * q[2] + dv[2] * q[3]) + q[4] +
                       (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double nu_zv = ep[2 * i] + 0.5 * ((sr - 6.0) * ia2 - lap);
    bool apply;
    if (node_rule == 0) apply = node;
    else if (node_rule == 1) apply = any_node;
    else if (node_rule == 2) apply = true;
    else apply = false;
    nuopt += apply ? fmax(nu_zv, ep[2 * i + 1]) : nu_zv;
    vee += q[5];
    nnode += node ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kept += __shfl_xor_sync(FULL, kept, o);
    negs += __shfl_xor_sync(FULL, negs, o);
    nuopt += __shfl_xor_sync(FULL, nuopt, o);
    vee += __shfl_xor_sync(FULL, vee, o);
    nnode += __shfl_xor_sync(FULL, nnode, o);
  }
  EvalOut e;
  const double i2a2 = 0.5 * ia2;
  e.bbar = kept * i2a2;
  e.vsf = negs * i2a2;
  e.W = 3.0 * ne * ia2 + nuopt + vee + S.v_ii + e.vsf;
  e.eL = e.W - e.bbar;
  e.n_node = nnode;
  return e;
}

// Build the orbital cache and potentials at every electron, invert both
// Slater blocks and evaluate.  x must already be in shared memory.
__device__ EvalOut init_walker(const DevSys& S, const Layout& L, double* __restrict__ gblk, double* sm, double a,
                               int node_rule, const double* T, int lane, bool& singular) {
  double* chi5 = sm + L.s_geo;     // scratch while no evaluation is in progress
  double* phi5 = sm + L.s_phi5;
  double* cache = gblk + L.g_cache;
  const double* x = sm + L.s_x;
  double* ep = sm + L.s_ep;
  for (int i = 0; i < L.n_e; ++i) {
    const int n = i < L.n_up ? L.n_up : L.n_dn;
    const double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    orbital_derivs(S, L, q, n, chi5, phi5, T, lane);
    for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
    double nu, nucap;
    electron_potentials(S, q, a, lane, nu, nucap);
    if (lane == 0) {
      ep[2 * i] = nu;
      ep[2 * i + 1] = nucap;
    }
    __syncwarp();
  }
  __threadfence_block();
  singular = reinvert(L, gblk, sm, sm + L.s_g, lane);
  return eval_walker(S, L, gblk, sm, a, node_rule, false, T, lane);
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

// Apply hop p: orbital derivatives at the moved electron, Sherman-Morrison
// update of its spin block (and of g by the same factors when g_valid),
// cache, potential and position update.
__device__ void apply_hop(const DevSys& S, const Layout& L, double* __restrict__ gblk, double* sm, int p, double a,
                          bool g_valid, const double* T, int lane) {
  double* x = sm + L.s_x;
  double* bt = sm + L.s_bt;
  double* cache = gblk + L.g_cache;
  double* phi5 = sm + L.s_phi5;
  double* f = sm + L.s_u;
  double* row = sm + L.s_row;
  double* chi5 = sm + L.s_geo;     // geometry is rebuilt by the next evaluation
  double* g = sm + L.s_g;
  double* grow = chi5 + 5 * L.n_bf;
  const int i = p / 6, d = p - 6 * i;
  double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  q[d >> 1] += (d & 1) ? -a : a;
  const SpinRef sr = spin_ref(L, i);
  orbital_derivs(S, L, q, sr.n, chi5, phi5, T, lane);
  double* B = bt + sr.bt_off;   // B^T of the spin block: B[j * n + k] = (A^{-1})_{k j}
  const int n = sr.n;
  // u_j = phi(r') . B[:, j]; the determinant ratio is u_ii
  for (int j = lane; j < n; j += WARP) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(phi5[k], B[j * n + k], acc);
    f[j] = acc;
  }
  for (int k = lane; k < n; k += WARP) row[k] = B[sr.ii * n + k];
  if (g_valid)
    for (int mu = lane; mu < L.n_bf; mu += WARP) grow[mu] = g[i * L.n_bf + mu];
  __syncwarp();
  const double invR = 1.0 / f[sr.ii];
  __syncwarp();
  // A' = A + e_i (phi' - phi)^T  =>  B' = B - B e_i (u - e_i)^T / u_i
  for (int j = lane; j < n; j += WARP) f[j] = (f[j] - (j == sr.ii ? 1.0 : 0.0)) * invR;
  __syncwarp();
  for (int o = lane; o < n * n; o += WARP) {
    const int j = o / n, k = o - j * n;
    B[o] = fma(-row[k], f[j], B[o]);
  }
  if (g_valid) {
    const int e0 = i - sr.ii;
    for (int o = lane; o < n * L.n_bf; o += WARP) {
      const int j = o / L.n_bf, mu = o - j * L.n_bf;
      double* gj = g + (e0 + j) * L.n_bf + mu;
      *gj = fma(-grow[mu], f[j], *gj);
    }
  }
  for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
  double nu, nucap;
  electron_potentials(S, q, a, lane, nu, nucap);
  if (lane == 0) {
    x[3 * i] = q[0];
    x[3 * i + 1] = q[1];
    x[3 * i + 2] = q[2];
    sm[L.s_ep + 2 * i] = nu;
    sm[L.s_ep + 2 * i + 1] = nucap;
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
};

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

// Place walkers at x_in (n x n_e x 3), build caches, invert and evaluate.
__global__ void k_init_walkers(DevSys S, Layout L, double* __restrict__ state, const double* __restrict__ x_in,
                               const double* __restrict__ w_in, int n, double a, int node_rule) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + EXP_TAB + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, gblk, sm, a, node_rule, T, lane, sing);
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
    store_block(L, gblk, sm, lane);
  }
}

// Evaluate arbitrary configurations without touching the walkers (the orbital
// cache of each configuration goes to scratch walker blocks).
__global__ void k_eval_configs(DevSys S, Layout L, double* __restrict__ scratch, const double* __restrict__ x_in,
                               int n, double a, int node_rule, double* __restrict__ ratios, double* __restrict__ ev,
                               int32_t* __restrict__ n_node) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + EXP_TAB + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    double* gblk = scratch + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker(S, L, gblk, sm, a, node_rule, T, lane, sing);
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
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = smem + EXP_TAB + wib * L.s_stride;
  double* sc = sm + L.s_sc;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n_w; w += nwarps) {
    const unsigned long long t_start = global_ns();
    double* gblk = state + (size_t)w * L.g_stride;
    load_block(L, gblk, sm, lane);
    double weight = 1.0, tau_left = P.tau;
    double bbar = sc[SC_BBAR], Wd = sc[SC_WDIAG], eL = sc[SC_EL];
    uint32_t status = (uint32_t)sc[SC_STATUS];
    int moves = 0, since = (int)sc[SC_SINCE];
    bool g_valid = false;
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
        if (!g_valid) {
          compute_g(S, L, sm, lane);
          g_valid = true;
        }
        apply_hop(S, L, gblk, sm, p, P.a, g_valid, T, lane);
        ++moves;
        if (++since >= P.reinv_period) {
          if (reinvert(L, gblk, sm, sm + L.s_g, lane)) status |= ST_SINGULAR;
          since = 0;
          g_valid = false;
        }
        const EvalOut e = eval_walker(S, L, gblk, sm, P.a, P.node_rule, g_valid, T, lane);
        g_valid = true;
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
    if (P.stamps && lane == 0) {
      P.stamps[3 * (size_t)w] = t_start;
      P.stamps[3 * (size_t)w + 1] = global_ns();
      P.stamps[3 * (size_t)w + 2] = sm_id();
    }
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

__global__ void k_clear_status(Layout L, double* __restrict__ state, int n_w) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_w; a += gridDim.x * blockDim.x)
    state[(size_t)a * L.g_stride + L.g_sc + SC_STATUS] = 0.0;
}

}  // namespace lrdmc
