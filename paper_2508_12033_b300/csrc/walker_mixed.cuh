// Mixed-precision (FP32 evaluation, FP64 accumulation) warp-per-walker kernels.
//
// Same method and walker layout as walker.cuh; what changes is where each
// quantity lives:
//   FP64  positions (lattice hops stay exact), weights, the b_bar / V_sf / W /
//         e_L accumulators, potentials as stored, Gauss-Jordan re-inversion;
//   FP32  B^T (Sherman-Morrison updates), g_i, orbital cache, every hop ratio,
//         Jastrow and basis values.
// Every hop ratio is produced directly as r - 1 ("delta form"), so that the
// kinetic sums of Appendix D never subtract two O(3 N_e / a^2) numbers in FP32:
//   * determinant: chi(r_i) . g_i = 1 exactly, so det - 1 = sum_mu
//     [chi_mu(r') - chi_mu(r_i)] g_mu, with every Gaussian difference formed as
//     h (exp(-alpha delta) - 1), delta = |r'-R|^2 - |r_i-R|^2 = 2 (+-a) d_axis + a^2;
//   * Jastrow: u(r') - u(r) = c delta t t' / (r' + r), t = 1/(1 + b r),
//     delta = 2 (+-a) (r_i - r_j)_axis + a^2, and exp(dJ) - 1 by expm1f;
//   * r - 1 = D + J + D J.
// The walker block's B^T and cache regions hold floats (first half of each).
#pragma once

#include "common.cuh"
#include "walker.cuh"

namespace lrdmc {

// Shared-memory layout of one warp for the mixed kernels (offsets in floats;
// the double arrays x and sc sit at even offsets).
struct LayoutM {
  int x, xf, bt, g, dl, ej, ep, dd, geo, rt1, pair, hcur, chi5, phi5, f, row, grow, sc, stride;
};

__host__ __device__ inline LayoutM layout_mixed(const Layout& L, int n_nuc, int n_prim) {
  LayoutM M;
  const int ne = L.n_e, nbt = L.n_up * L.n_up + L.n_dn * L.n_dn;
  int o = 0;
  M.sc = o; o += 2 * SC_COUNT;                         // doubles
  M.x = o; o += 2 * 3 * ne;                            // doubles
  M.xf = o; o += 3 * ne;
  M.bt = o; o += nbt;
  o = round_up(o, 2);
  const int gsz = ne * L.n_bf > 4 * L.n_max * L.n_max ? ne * L.n_bf : 4 * L.n_max * L.n_max;
  M.g = o; o += gsz;                                   // also FP64 Gauss-Jordan scratch
  M.dl = o; o += 6 * ne;
  M.ej = o; o += 5 * ne;
  M.ep = o; o += 2 * ne;
  M.dd = o; o += 4 * ne;
  M.geo = o; o += 4 * ne * n_nuc;
  M.rt1 = o; o += 2 * ne * n_nuc;
  M.pair = o; o += 3 * ne * ne;
  M.hcur = o; o += ne * n_prim;
  M.chi5 = o; o += 5 * L.n_bf;
  M.phi5 = o; o += 5 * L.n_max;
  M.f = o; o += L.n_max;
  M.row = o; o += L.n_max;
  M.grow = o; o += L.n_bf;
  M.stride = round_up(o, 4);
  return M;
}

__device__ __forceinline__ float* bt_f(const Layout& L, double* gblk) { return (float*)(gblk + L.g_bt); }
__device__ __forceinline__ float* cache_f(const Layout& L, double* gblk) { return (float*)(gblk + L.g_cache); }

// FP32 value/gradient/Laplacian of shell s at offset d (r2 = |d|^2).
__device__ __forceinline__ void shell_derivs_f(const DevSys& S, int s, const float d[3], float r2,
                                               float* __restrict__ out, int n_bf) {
  const int l = __ldg(S.sh_l + s), np = __ldg(S.sh_nprim + s), off = __ldg(S.sh_off + s), bf = __ldg(S.sh_bf + s);
  if (l == -1) {
    const float ir = rsqrtf(r2), r = r2 * ir;
    float v = 0.f, dr = 0.f, lp = 0.f;
    for (int q = 0; q < np; ++q) {
      const float z = (float)__ldg(S.exps + off + q);
      const float h = (float)__ldg(S.coefs + off + q) * __expf(-z * r);
      v += h;
      dr -= z * h;
      lp += (z * z - 2.f * z * ir) * h;
    }
    out[bf] = v;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = dr * d[m] * ir;
    out[4 * n_bf + bf] = lp;
  } else if (l == 0) {
    float v = 0.f, gs = 0.f, lp = 0.f;
    for (int q = 0; q < np; ++q) {
      const float al = (float)__ldg(S.exps + off + q);
      const float h = (float)__ldg(S.coefs + off + q) * __expf(-al * r2);
      v += h;
      gs -= 2.f * al * h;
      lp += (4.f * al * al * r2 - 6.f * al) * h;
    }
    out[bf] = v;
    for (int m = 0; m < 3; ++m) out[(1 + m) * n_bf + bf] = gs * d[m];
    out[4 * n_bf + bf] = lp;
  } else {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int q = 0; q < np; ++q) {
      const float al = (float)__ldg(S.exps + off + q);
      const float h = (float)__ldg(S.coefs + off + q) * __expf(-al * r2);
      s0 += h;
      s1 -= 2.f * al * h;
      s2 += (4.f * al * al * r2 - 10.f * al) * h;
    }
    for (int m = 0; m < 3; ++m) {
      out[bf + m] = d[m] * s0;
      for (int n = 0; n < 3; ++n) out[(1 + n) * n_bf + bf + m] = (m == n ? s0 : 0.f) + d[m] * d[n] * s1;
      out[4 * n_bf + bf + m] = d[m] * s2;
    }
  }
}

__device__ void orbital_derivs_f(const DevSys& S, const Layout& L, const float q[3], int n_sig, float* chi5,
                                 float* phi5, int lane) {
  for (int s = lane; s < S.n_shell; s += WARP) {
    const int atom = __ldg(S.sh_atom + s);
    const float d[3] = {q[0] - (float)__ldg(S.R + 3 * atom), q[1] - (float)__ldg(S.R + 3 * atom + 1),
                        q[2] - (float)__ldg(S.R + 3 * atom + 2)};
    shell_derivs_f(S, s, d, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], chi5, L.n_bf);
  }
  __syncwarp();
  for (int o = lane; o < 5 * n_sig; o += WARP) {
    const int c = o / n_sig, k = o - c * n_sig;
    const double* crow = S.C + (size_t)k * L.n_bf;
    const float* x = chi5 + c * L.n_bf;
    float acc = 0.f;
    for (int mu = 0; mu < L.n_bf; ++mu) acc = fmaf((float)__ldg(crow + mu), x[mu], acc);
    phi5[c * L.n_max + k] = acc;
  }
  __syncwarp();
}

__device__ void electron_potentials_f(const DevSys& S, const float q[3], float a, int lane, float& nu,
                                      float& nucap) {
  nu = 0.f;
  nucap = 0.f;
  for (int I = lane; I < S.n_nuc; I += WARP) {
    const float dx = q[0] - (float)__ldg(S.R + 3 * I), dy = q[1] - (float)__ldg(S.R + 3 * I + 1),
                dz = q[2] - (float)__ldg(S.R + 3 * I + 2);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float Z = (float)__ldg(S.Z + I);
    if (__ldg(S.kind + I) == 0) {
      nu -= Z / r;
      nucap -= Z / fmaxf(r, a);
    } else {
      const float v = -Z * erff(r / (float)__ldg(S.rc + I)) / r;
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

// FP64 re-inversion of the FP32 orbital values; B^T stored back as floats.
__device__ bool reinvert_m(const Layout& L, const LayoutM& M, double* gblk, float* sm, int lane) {
  bool sing = false;
  const float* cache = cache_f(L, gblk);
  float* bt = sm + M.bt;
  double* scratch = (double*)(sm + M.g);
  for (int blk = 0; blk < 2; ++blk) {
    const int n = blk ? L.n_dn : L.n_up;
    const int e0 = blk ? L.n_up : 0;
    const int bto = blk ? L.n_up * L.n_up : 0;
    if (n == 0) continue;
    for (int o = lane; o < n * 2 * n; o += WARP) {
      const int r = o / (2 * n), c = o - r * 2 * n;
      scratch[o] = c < n ? (double)cache[(e0 + r) * 5 * L.n_max + c] : (c - n == r ? 1.0 : 0.0);
    }
    __syncwarp();
    sing |= warp_gauss_jordan(scratch, n, lane);
    for (int o = lane; o < n * n; o += WARP) {
      const int i = o / n, k = o - i * n;
      bt[bto + o] = (float)scratch[k * 2 * n + n + i];
    }
    __syncwarp();
  }
  return sing;
}

__device__ void compute_g_m(const DevSys& S, const Layout& L, const LayoutM& M, float* sm, int lane) {
  const float* bt = sm + M.bt;
  float* g = sm + M.g;
  for (int o = lane; o < L.n_e * L.n_bf; o += WARP) {
    const int i = o / L.n_bf, mu = o - i * L.n_bf;
    const SpinRef sr = spin_ref(L, i);
    const float* brow = bt + sr.bt_off + sr.ii * sr.n;
    float acc = 0.f;
    for (int k = 0; k < sr.n; ++k) acc = fmaf((float)__ldg(S.C + (size_t)k * L.n_bf + mu), brow[k], acc);
    g[o] = acc;
  }
  __syncwarp();
}

// Evaluate at the current configuration: hop ratios as r - 1 (FP32) and the
// FP64 accumulators.
__device__ EvalOut eval_walker_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm,
                                 double a, int node_rule, bool g_valid, int lane) {
  const int ne = L.n_e, nbf = L.n_bf, nmax = L.n_max, nn = S.n_nuc;
  const float af = (float)a, a2f = af * af;
  const float* xf = sm + M.xf;
  const float* bt = sm + M.bt;
  const float* cache = cache_f(L, gblk);
  float* g = sm + M.g;
  float* dl = sm + M.dl;
  float* ej = sm + M.ej;     // grad J (3), lap J, half e-e sum
  const float* ep = sm + M.ep;
  float* dd = sm + M.dd;
  float* geo = sm + M.geo;   // per (electron, nucleus): d (3), |d|^2
  float* rt1 = sm + M.rt1;   // per (electron, nucleus): r, 1/(1 + B r)
  float* pair = sm + M.pair; // per electron pair: |d|^2, r, 1/(1 + b r)
  float* hcur = sm + M.hcur; // per (electron, primitive): coef exp(-alpha |d|^2)
  const float bj = (float)S.j2_b, cpar = (float)S.j2_par, canti = (float)S.j2_anti;
  // (1) current configuration: Jastrow derivatives, geometry, primitive values
  {
    int npad = 1;
    while (npad < ne) npad <<= 1;
    const int G = npad >= WARP ? 1 : WARP / npad;
    const int per = ne - 1 + nn;
    for (int base = 0; base < ne; base += WARP / G) {
      const int e = base + lane / G, sub = lane % G;
      float gx = 0.f, gy = 0.f, gz = 0.f, LJ = 0.f, vee = 0.f;
      if (e < ne) {
        const float xe = xf[3 * e], ye = xf[3 * e + 1], ze = xf[3 * e + 2];
        const bool up_e = e < L.n_up;
        for (int t = sub; t < per; t += G) {
          if (t < ne - 1) {
            const int j = t < e ? t : t + 1;
            const float dx = xe - xf[3 * j], dy = ye - xf[3 * j + 1], dz = ze - xf[3 * j + 2];
            const float s = dx * dx + dy * dy + dz * dz;
            const float ir = rsqrtf(s), r = s * ir;
            const float c = (up_e == (j < L.n_up)) ? cpar : canti;
            const float tt = __fdividef(1.f, fmaf(bj, r, 1.f));
            float* pp = pair + 3 * (e * ne + j);
            pp[0] = s; pp[1] = r; pp[2] = tt;
            const float up = c * tt * tt, upp = -2.f * bj * up * tt, f = up * ir;
            gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
            LJ += upp + 2.f * f;
            vee = fmaf(0.5f, ir, vee);
          } else {
            const int I = t - (ne - 1);
            const float dx = xe - (float)__ldg(S.R + 3 * I), dy = ye - (float)__ldg(S.R + 3 * I + 1),
                        dz = ze - (float)__ldg(S.R + 3 * I + 2);
            const float s = dx * dx + dy * dy + dz * dz;
            float* gg = geo + 4 * (e * nn + I);
            gg[0] = dx; gg[1] = dy; gg[2] = dz; gg[3] = s;
            for (int sh = __ldg(S.atom_sh + I); sh < __ldg(S.atom_sh + I + 1); ++sh) {
              const int np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh);
              const bool sto = __ldg(S.sh_l + sh) == -1;
              const float arg = sto ? sqrtf(s) : s;
              for (int q = 0; q < np; ++q)
                hcur[e * S.n_prim + off + q] = (float)__ldg(S.coefs + off + q) * __expf(-(float)__ldg(S.exps + off + q) * arg);
            }
            const float A = (float)__ldg(S.j1A + I);
            const float ir = rsqrtf(s), r = s * ir;
            const float B = (float)__ldg(S.j1B + I);
            const float tt = __fdividef(1.f, fmaf(B, r, 1.f));
            rt1[2 * (e * nn + I)] = r;
            rt1[2 * (e * nn + I) + 1] = tt;
            if (A != 0.f) {
              const float vp = -A * tt * tt, vpp = -2.f * B * vp * tt, f = vp * ir;
              gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
              LJ += vpp + 2.f * f;
            }
          }
        }
      }
      for (int o = G >> 1; o; o >>= 1) {
        gx += __shfl_xor_sync(FULL, gx, o);
        gy += __shfl_xor_sync(FULL, gy, o);
        gz += __shfl_xor_sync(FULL, gz, o);
        LJ += __shfl_xor_sync(FULL, LJ, o);
        vee += __shfl_xor_sync(FULL, vee, o);
      }
      if (e < ne && sub == 0) {
        float* q = ej + 5 * e;
        q[0] = gx; q[1] = gy; q[2] = gz; q[3] = LJ; q[4] = vee;
      }
    }
  }
  for (int o = lane; o < 4 * ne; o += WARP) {
    const int i = o >> 2, c = o & 3;
    const SpinRef sr = spin_ref(L, i);
    const float* brow = bt + sr.bt_off + sr.ii * sr.n;
    const float* ce = cache + i * 5 * nmax + (c + 1) * nmax;
    float acc = 0.f;
    for (int k = 0; k < sr.n; ++k) acc = fmaf(ce[k], brow[k], acc);
    dd[o] = acc;
  }
  if (!g_valid) compute_g_m(S, L, M, sm, lane);
  __syncwarp();
  // (3) every hop, as r - 1
  for (int p = lane; p < 6 * ne; p += WARP) {
    const int i = p / 6, d = p - 6 * i, ax = d >> 1;
    const float sa = (d & 1) ? -af : af;
    const float s2a = sa + sa;
    const float* gi = g + i * nbf;
    float D = 0.f, dJ = 0.f;
    for (int I = 0; I < nn; ++I) {
      const float* gg = geo + 4 * (i * nn + I);
      const float del = fmaf(s2a, gg[ax], a2f);           // |r'-R|^2 - |r-R|^2
      const float sp = gg[3] + del;
      const float A = (float)__ldg(S.j1A + I);
      const float r = rt1[2 * (i * nn + I)], tt = rt1[2 * (i * nn + I) + 1];
      const float rp = sp * rsqrtf(sp);
      if (A != 0.f) {
        const float tp = __fdividef(1.f, fmaf((float)__ldg(S.j1B + I), rp, 1.f));
        dJ -= A * del * tt * __fdividef(tp, rp + r);
      }
      for (int sh = __ldg(S.atom_sh + I); sh < __ldg(S.atom_sh + I + 1); ++sh) {
        const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh),
                  bf = __ldg(S.sh_bf + sh);
        float rd = 0.f, rn = 0.f;   // sum of (h' - h) and of h'
        for (int q = 0; q < np; ++q) {
          const float h = hcur[i * S.n_prim + off + q];
          const float al = (float)__ldg(S.exps + off + q);
          // the clamp only acts where h has already underflowed to 0
          const float dh = h * expm1f(fminf(l == -1 ? -al * __fdividef(del, rp + r) : -al * del, 80.f));
          rd += dh;
          rn += h + dh;
        }
        if (l != 1) {
          D = fmaf(rd, gi[bf], D);
        } else {
          const float* g3 = gi + bf;
          D = fmaf(rd, fmaf(gg[0], g3[0], fmaf(gg[1], g3[1], gg[2] * g3[2])), D);
          D = fmaf(sa * rn, g3[ax], D);
        }
      }
    }
    const bool up_i = i < L.n_up;
    const float xia = xf[3 * i + ax];
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      const float* pp = pair + 3 * (i * ne + j);
      const float del = fmaf(s2a, xia - xf[3 * j + ax], a2f);
      const float sp = pp[0] + del;
      const float rp = sp * rsqrtf(sp);
      const float tp = __fdividef(1.f, fmaf(bj, rp, 1.f));
      const float c = (up_i == (j < L.n_up)) ? cpar : canti;
      dJ = fmaf(c * del * pp[2], __fdividef(tp, rp + pp[1]), dJ);
    }
    const float J = expm1f(dJ);
    dl[p] = fmaf(D, J, D + J);
  }
  __syncwarp();
  // (4) fixed-node split and regularised potential per electron, FP64 sums
  bool has_node = false;
  for (int i = lane; i < ne; i += WARP)
    for (int d = 0; d < 6; ++d) has_node |= dl[6 * i + d] < -1.f;
  const bool any_node = __any_sync(FULL, has_node);
  double kept = 0.0, negs = 0.0, nuopt = 0.0, vee = 0.0;
  int nnode = 0;
  const double ia2 = 1.0 / (a * a);
  for (int i = lane; i < ne; i += WARP) {
    double sd = 0.0;
    bool node = false;
    for (int d = 0; d < 6; ++d) {
      const double x1 = (double)dl[6 * i + d];     // r - 1
      sd += x1;
      if (x1 > -1.0) kept += 1.0 + x1;
      if (x1 < -1.0) { negs -= 1.0 + x1; node = true; }
    }
    const float* q = ej + 5 * i;
    const float* dv = dd + 4 * i;
    const float lap = dv[3] + 2.f * (dv[0] * q[0] + dv[1] * q[1] + dv[2] * q[2]) + q[3] +
                      (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    const double nu_zv = (double)ep[2 * i] + 0.5 * (sd * ia2 - (double)lap);
    bool apply;
    if (node_rule == 0) apply = node;
    else if (node_rule == 1) apply = any_node;
    else if (node_rule == 2) apply = true;
    else apply = false;
    nuopt += apply ? fmax(nu_zv, (double)ep[2 * i + 1]) : nu_zv;
    vee += (double)q[4];
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

__device__ EvalOut init_walker_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm,
                                 double a, int node_rule, int lane, bool& singular) {
  float* chi5 = sm + M.chi5;
  float* phi5 = sm + M.phi5;
  float* cache = cache_f(L, gblk);
  const double* x = (const double*)(sm + M.x);
  float* xf = sm + M.xf;
  float* ep = sm + M.ep;
  for (int o = lane; o < 3 * L.n_e; o += WARP) xf[o] = (float)x[o];
  __syncwarp();
  for (int i = 0; i < L.n_e; ++i) {
    const int n = i < L.n_up ? L.n_up : L.n_dn;
    const float q[3] = {xf[3 * i], xf[3 * i + 1], xf[3 * i + 2]};
    orbital_derivs_f(S, L, q, n, chi5, phi5, lane);
    for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
    float nu, nucap;
    electron_potentials_f(S, q, (float)a, lane, nu, nucap);
    if (lane == 0) {
      ep[2 * i] = nu;
      ep[2 * i + 1] = nucap;
    }
    __syncwarp();
  }
  __threadfence_block();
  singular = reinvert_m(L, M, gblk, sm, lane);
  return eval_walker_m(S, L, M, gblk, sm, a, node_rule, false, lane);
}

// Heat-bath choice from r - 1 values (same order and rule as the FP64 path).
__device__ int choose_hop_m(const float* dl, int n_hop, double u, int lane) {
  int choice = -1;
  if (lane == 0) {
    double total = 0.0;
    for (int p = 0; p < n_hop; ++p) total += dl[p] > -1.f ? 1.0 + (double)dl[p] : 0.0;
    if (total > 0.0) {
      const double t = u * total;
      double run = 0.0;
      int last = -1;
      for (int p = 0; p < n_hop; ++p) {
        const double k = dl[p] > -1.f ? 1.0 + (double)dl[p] : 0.0;
        if (k > 0.0) last = p;
        run += k;
        if (run > t) { choice = p; break; }
      }
      if (choice < 0) choice = last;
    }
  }
  return __shfl_sync(FULL, choice, 0);
}

__device__ void apply_hop_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm, int p,
                            double a, bool g_valid, int lane) {
  double* x = (double*)(sm + M.x);
  float* xf = sm + M.xf;
  float* bt = sm + M.bt;
  float* cache = cache_f(L, gblk);
  float* phi5 = sm + M.phi5;
  float* f = sm + M.f;
  float* row = sm + M.row;
  float* g = sm + M.g;
  float* grow = sm + M.grow;
  const int i = p / 6, d = p - 6 * i;
  double qd[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  qd[d >> 1] += (d & 1) ? -a : a;
  const float q[3] = {(float)qd[0], (float)qd[1], (float)qd[2]};
  const SpinRef sr = spin_ref(L, i);
  orbital_derivs_f(S, L, q, sr.n, sm + M.chi5, phi5, lane);
  float* B = bt + sr.bt_off;
  const int n = sr.n;
  for (int j = lane; j < n; j += WARP) {
    float acc = 0.f;
    for (int k = 0; k < n; ++k) acc = fmaf(phi5[k], B[j * n + k], acc);
    f[j] = acc;
  }
  for (int k = lane; k < n; k += WARP) row[k] = B[sr.ii * n + k];
  if (g_valid)
    for (int mu = lane; mu < L.n_bf; mu += WARP) grow[mu] = g[i * L.n_bf + mu];
  __syncwarp();
  const float invR = 1.f / f[sr.ii];
  __syncwarp();
  for (int j = lane; j < n; j += WARP) f[j] = (f[j] - (j == sr.ii ? 1.f : 0.f)) * invR;
  __syncwarp();
  for (int o = lane; o < n * n; o += WARP) {
    const int j = o / n, k = o - j * n;
    B[o] = fmaf(-row[k], f[j], B[o]);
  }
  if (g_valid) {
    const int e0 = i - sr.ii;
    for (int o = lane; o < n * L.n_bf; o += WARP) {
      const int j = o / L.n_bf, mu = o - j * L.n_bf;
      float* gj = g + (e0 + j) * L.n_bf + mu;
      *gj = fmaf(-grow[mu], f[j], *gj);
    }
  }
  for (int o = lane; o < 5 * L.n_max; o += WARP) cache[i * 5 * L.n_max + o] = phi5[o];
  float nu, nucap;
  electron_potentials_f(S, q, (float)a, lane, nu, nucap);
  if (lane == 0) {
    x[3 * i] = qd[0]; x[3 * i + 1] = qd[1]; x[3 * i + 2] = qd[2];
    xf[3 * i] = q[0]; xf[3 * i + 1] = q[1]; xf[3 * i + 2] = q[2];
    sm[M.ep + 2 * i] = nu;
    sm[M.ep + 2 * i + 1] = nucap;
  }
  __threadfence_block();
  __syncwarp();
}

__device__ __forceinline__ void load_block_m(const Layout& L, const LayoutM& M, const double* __restrict__ g,
                                             float* sm, int lane) {
  double* x = (double*)(sm + M.x);
  double* sc = (double*)(sm + M.sc);
  for (int o = lane; o < 3 * L.n_e; o += WARP) {
    x[o] = g[L.g_x + o];
    sm[M.xf + o] = (float)g[L.g_x + o];
  }
  const float* btg = (const float*)(g + L.g_bt);
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) sm[M.bt + o] = btg[o];
  for (int o = lane; o < L.n_hop; o += WARP) sm[M.dl + o] = (float)(g[L.g_rat + o] - 1.0);
  for (int o = lane; o < 2 * L.n_e; o += WARP) sm[M.ep + o] = (float)g[L.g_pot + o];
  for (int o = lane; o < SC_COUNT; o += WARP) sc[o] = g[L.g_sc + o];
  __syncwarp();
}

__device__ __forceinline__ void store_block_m(const Layout& L, const LayoutM& M, double* __restrict__ g,
                                              const float* sm, int lane) {
  __syncwarp();
  const double* x = (const double*)(sm + M.x);
  const double* sc = (const double*)(sm + M.sc);
  for (int o = lane; o < 3 * L.n_e; o += WARP) g[L.g_x + o] = x[o];
  float* btg = (float*)(g + L.g_bt);
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) btg[o] = sm[M.bt + o];
  for (int o = lane; o < L.n_hop; o += WARP) g[L.g_rat + o] = 1.0 + (double)sm[M.dl + o];
  for (int o = lane; o < 2 * L.n_e; o += WARP) g[L.g_pot + o] = (double)sm[M.ep + o];
  for (int o = lane; o < SC_COUNT; o += WARP) g[L.g_sc + o] = sc[o];
}

__global__ void k_init_walkers_m(DevSys S, Layout L, LayoutM M, double* __restrict__ state,
                                 const double* __restrict__ x_in, const double* __restrict__ w_in, int n, double a,
                                 int node_rule) {
  extern __shared__ float smf[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sm = smf + wib * M.stride;
  double* x = (double*)(sm + M.x);
  double* sc = (double*)(sm + M.sc);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) x[o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker_m(S, L, M, gblk, sm, a, node_rule, lane, sing);
    if (lane == 0) {
      for (int k = 0; k < SC_COUNT; ++k) sc[k] = 0.0;
      sc[SC_W] = w_in ? w_in[w] : 1.0;
      sc[SC_BBAR] = e.bbar;
      sc[SC_VSF] = e.vsf;
      sc[SC_WDIAG] = e.W;
      sc[SC_EL] = e.eL;
      sc[SC_NNODE] = e.n_node;
      sc[SC_STATUS] = sing ? (double)ST_SINGULAR : 0.0;
    }
    store_block_m(L, M, gblk, sm, lane);
  }
}

__global__ void k_eval_configs_m(DevSys S, Layout L, LayoutM M, double* __restrict__ scratch,
                                 const double* __restrict__ x_in, int n, double a, int node_rule,
                                 double* __restrict__ ratios, double* __restrict__ ev, int32_t* __restrict__ n_node) {
  extern __shared__ float smf[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sm = smf + wib * M.stride;
  double* x = (double*)(sm + M.x);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n; w += nwarps) {
    double* gblk = scratch + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) x[o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker_m(S, L, M, gblk, sm, a, node_rule, lane, sing);
    for (int o = lane; o < L.n_hop; o += WARP) ratios[(size_t)w * L.n_hop + o] = 1.0 + (double)sm[M.dl + o];
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

__global__ void k_propagate_m(DevSys S, Layout L, LayoutM M, double* __restrict__ state, int n_w, StepParams P) {
  extern __shared__ float smf[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sm = smf + wib * M.stride;
  double* sc = (double*)(sm + M.sc);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < n_w; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    load_block_m(L, M, gblk, sm, lane);
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
        const double den = Wd - P.E0;
        if (den > 0.0) {
          weight *= bbar / den;
        } else {
          weight *= 0.0;
          status |= ST_NEG_DIAG;
        }
      } else {
        double t = -log(1.0 - u_tau) / bbar;
        const bool clipped = !(t < tau_left);
        if (clipped) t = tau_left;
        weight *= exp(-t * eL);
        tau_left -= t;
        if (clipped) break;
      }
      const int p = choose_hop_m(sm + M.dl, L.n_hop, u_move, lane);
      if (p < 0) {
        status |= ST_STUCK;
      } else {
        if (!g_valid) {
          compute_g_m(S, L, M, sm, lane);
          g_valid = true;
        }
        apply_hop_m(S, L, M, gblk, sm, p, P.a, g_valid, lane);
        ++moves;
        if (++since >= P.reinv_period) {
          if (reinvert_m(L, M, gblk, sm, lane)) status |= ST_SINGULAR;
          since = 0;
          g_valid = false;
        }
        const EvalOut e = eval_walker_m(S, L, M, gblk, sm, P.a, P.node_rule, g_valid, lane);
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
    store_block_m(L, M, gblk, sm, lane);
  }
}

}  // namespace lrdmc
