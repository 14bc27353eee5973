// Mixed-precision warp-per-walker kernels: FP32 hop evaluation, FP64 where
// conditioning demands it.
//
// Same method and walker layout as walker.cuh; what changes is where each
// quantity lives:
//   FP64  positions (lattice hops stay exact), the orbital values phi_k(r_i)
//         (rows of A), B = A^{-1} with its Sherman-Morrison updates and the
//         Gauss-Jordan re-inversion, the determinant derivatives grad/lap D/D,
//         weights and the b_bar / V_sf / W / e_L accumulators.  Near a node A
//         is ill-conditioned and an FP32 A or B would carry cond(A) * 1e-7
//         relative errors into every ratio; in FP64 they stay negligible.
//   FP32  every hop ratio (6 N_e per step, the bulk of the work): basis and
//         Jastrow differences, the orbital differences of every hop, an FP32
//         copy of B for the hop determinants, the orbital gradient/Laplacian
//         rows, potentials, heat-bath sums.
// Each hop ratio is produced directly as r - 1 ("delta form") so that the
// kinetic sums of Appendix D never subtract two O(3 N_e / a^2) numbers in FP32:
//   * determinant: phi(r_i) . B[:, i] = 1 exactly, so det - 1 = sum_k
//     [phi_k(r') - phi_k(r_i)] B_ki, the orbital differences contracted from
//     basis differences, every Gaussian difference formed as
//     h (exp(-alpha delta) - 1), delta = |r'-R|^2 - |r_i-R|^2 = 2 (+-a) d_axis + a^2;
//   * Jastrow: u(r') - u(r) = c delta t t' / (r' + r), t = 1/(1 + b r),
//     delta = 2 (+-a) (r_i - r_j)_axis + a^2;
//   * r - 1 = D + J + D J with J = exp(dJ) - 1.
// exp(x) - 1 in FP32: Taylor polynomial of degree 6 for |x| < 1/4 (truncation
// < 2e-8 relative), exp(x) - 1 from the hardware exponential otherwise.
// Walker block: B^T as doubles (as in the FP64 layout); the cache region holds
// the FP64 orbital values [n_e][n_max] followed by the gradient/Laplacian
// rows [n_e][4][n_max] (evaluated in FP32, stored as doubles so that the FP64
// determinant derivatives read them without conversions).  As in the FP64
// kernels, the caches of the incremental evaluation persist in a per-walker
// cache block across branching intervals, and pair terms are swapped from
// cached values rather than recomputed.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "walker.cuh"

namespace lrdmc {

// Shared-memory layout of one warp for the mixed kernels, in floats (double
// arrays at even offsets).  Per-electron float rows are padded by one word so
// that lanes working on different electrons hit different banks.  The range
// [mir, mir_end) holds everything the incremental evaluation keeps between
// hops and is copied to / from the walker's cache block.
struct LayoutM {
  int sc, x, bt, phiv, chiv, u, row, xo;                               // doubles
  int dd;                                                              // doubles, kept
  int dl, ej, ep, geo, rt1, pair, hcur, hdm, hj1, hj2, dph;            // floats, kept
  int xf, xfo, b32, chi5, phi5, tmp;                                   // floats
  int geo_st, rt1_st, pair_st, hcur_st, stride;
  int mir, mir_end;
  // walker cache block, in floats: the shared-memory copy, the pair Jastrow
  // difference of every hop with every partner [n_e][6 n_e] and the pair
  // derivative terms at the current positions [n_e][n_e][3]
  int c_u2, c_pt, c_floats;
  // large systems (glob): the O(N^2) arrays geo, rt1, pair, hcur and dph live
  // in global memory (the cache block at c_big, or per-warp scratch for
  // configuration evaluation) at offsets g_* from that base, big_floats in all;
  // their shared-memory extents are then zero
  int glob, c_big, g_geo, g_rt1, g_pair, g_hcur, g_dph, big_floats;
  // FP32 orbital contractions (basis rows x C^T): 0 FP32 FMA on the CUDA
  // cores, 1 TF32 tensor-core MMA, 2 BF16 tensor-core MMA, 3 three TF32 MMAs
  // per step on split operands (FP32 accumulation in all)
  int tc;
};

__host__ __device__ inline LayoutM layout_mixed(const Layout& L, int n_nuc, int n_prim, int glob = 0) {
  LayoutM M;
  M.glob = glob;
  M.tc = 0;
  const int ne = L.n_e, nbt = L.n_up * L.n_up + L.n_dn * L.n_dn, nm = L.n_max, nbf = L.n_bf, P = L.n_hop;
  const int per = ne - 1 + n_nuc;
  int o = 0;
  M.sc = o; o += 2 * SC_COUNT;
  M.x = o; o += 2 * 3 * ne;
  M.bt = o; o += 2 * nbt;
  M.phiv = o; o += 2 * nm;
  M.chiv = o; o += 2 * nbf;
  M.u = o; o += 2 * nm;
  M.row = o; o += 2 * nm;
  M.xo = o; o += 2 * 4;
  M.mir = o;
  M.dd = o; o += 2 * 4 * ne;
  M.dl = o; o += P;
  M.ej = o; o += 5 * ne;
  M.ep = o; o += 2 * ne;
  M.geo_st = 4 * n_nuc + 1;
  M.rt1_st = 2 * n_nuc + 1;
  M.pair_st = 2 * ne + 1;
  M.hcur_st = n_prim + 1;
  const int sz_geo = ne * M.geo_st, sz_rt1 = ne * M.rt1_st, sz_pair = ne * M.pair_st, sz_hcur = ne * M.hcur_st;
  const int sz_dph = P * nm;   // orbital differences at every hop [6 n_e][n_max]
  M.g_geo = 0;
  M.g_rt1 = M.g_geo + sz_geo;
  M.g_pair = M.g_rt1 + sz_rt1;
  M.g_hcur = M.g_pair + sz_pair;
  M.g_dph = M.g_hcur + sz_hcur;
  M.big_floats = glob ? round_up(M.g_dph + sz_dph, 4) : 0;
  M.geo = o; o += glob ? 0 : sz_geo;
  M.rt1 = o; o += glob ? 0 : sz_rt1;
  M.pair = o; o += glob ? 0 : sz_pair;
  M.hcur = o; o += glob ? 0 : sz_hcur;
  M.hdm = o; o += P;
  M.hj1 = o; o += P;
  M.hj2 = o; o += P;
  M.dph = o; o += glob ? 0 : sz_dph;
  o = round_up(o, 2);
  M.mir_end = o;
  M.xf = o; o += 3 * ne;
  M.xfo = o; o += 4;
  M.b32 = o; o += nbt;         // FP32 copy of B^T
  // move scratch (basis rows), the basis differences at the moved electron's
  // six hops [n_bf][6] and the per-hop Jastrow scratch of an evaluation share
  // one region: they are never live together
  int sh = 6 * nbf > 6 * per ? 6 * nbf : 6 * per;
  M.chi5 = o; o += sh;
  M.tmp = M.chi5;
  M.phi5 = o; o += 5 * nm;
  M.stride = round_up(o, 4);
  int c = round_up(M.mir_end - M.mir, 4);
  M.c_u2 = c; c += round_up(ne * P, 4);
  M.c_pt = c; c += round_up(3 * ne * ne, 4);
  M.c_big = c; c += M.big_floats;
  M.c_floats = c;
  return M;
}

// Per-warp global scratch of the mixed kernels: the basis differences at every
// hop [n_bf][6 n_e] floats (live only during a full evaluation) and the FP64
// Gauss-Jordan work matrix [n_max][2 n_max].
__host__ __device__ inline size_t scratch_doubles_m(const Layout& L, const LayoutM& M) {
  return ((size_t)L.n_bf * L.n_hop + 1) / 2 + 2 * (size_t)L.n_max * L.n_max + ((size_t)M.big_floats + 1) / 2;
}

// Global working arrays of one mixed evaluation (see LayoutM for the layouts);
// u2 and pt are null for configuration evaluation; big is the base of the
// global O(N^2) arrays of a large system (null otherwise).
struct ScrM {
  float* dchi;   // per-warp scratch of a full evaluation
  float* u2;
  float* pt;
  double* gj;
  float* big;
};
__device__ __forceinline__ ScrM warp_scratch_m_at(const Layout& L, const LayoutM& M, double* base) {
  ScrM s;
  s.dchi = (float*)base;
  s.gj = base + ((size_t)L.n_bf * L.n_hop + 1) / 2;
  s.u2 = s.pt = nullptr;
  s.big = M.glob ? (float*)(s.gj + 2 * (size_t)L.n_max * L.n_max) : nullptr;
  return s;
}
__device__ __forceinline__ ScrM warp_scratch_m(const Layout& L, const LayoutM& M, double* scratch, int slot) {
  return warp_scratch_m_at(L, M, scratch + (size_t)slot * scratch_doubles_m(L, M));
}
__device__ __forceinline__ ScrM walker_scratch_m(const LayoutM& M, double* cblk, const ScrM& warp) {
  ScrM s;
  float* c = (float*)cblk;
  s.dchi = warp.dchi;
  s.u2 = c + M.c_u2;
  s.pt = c + M.c_pt;
  s.gj = warp.gj;
  s.big = M.glob ? c + M.c_big : nullptr;
  return s;
}

// Where the O(N^2) arrays of one walker are: shared memory or global.  BIG
// fixes the placement at compile time (1 global, 0 shared), so that the
// compiler sees plain global or shared accesses that cannot alias the
// shared-memory scratch of the same loop; -1 decides at run time.
struct MArr {
  float* geo;
  float* rt1;
  float* pair;
  float* hcur;
  float* dph;
};
template <int BIG = -1>
__device__ __forceinline__ MArr marr(const LayoutM& M, float* sm, const ScrM& scr) {
  MArr A;
  if (BIG == 1 || (BIG < 0 && scr.big)) {
    A.geo = scr.big + M.g_geo;
    A.rt1 = scr.big + M.g_rt1;
    A.pair = scr.big + M.g_pair;
    A.hcur = scr.big + M.g_hcur;
    A.dph = scr.big + M.g_dph;
  } else {
    A.geo = sm + M.geo;
    A.rt1 = sm + M.rt1;
    A.pair = sm + M.pair;
    A.hcur = sm + M.hcur;
    A.dph = sm + M.dph;
  }
  return A;
}

__device__ __forceinline__ double* cache_val(const Layout& L, double* gblk) { return gblk + L.g_cache; }
__device__ __forceinline__ double* cache_der(const Layout& L, double* gblk) {
  return gblk + L.g_cache + L.n_e * L.n_max;
}

// exp(x) - 1 in FP32 (see the header comment).
__device__ __forceinline__ float expm1_fast(float x) {
  float p = fmaf(x, 1.f / 720.f, 1.f / 120.f);
  p = fmaf(x, p, 1.f / 24.f);
  p = fmaf(x, p, 1.f / 6.f);
  p = fmaf(x, p, 0.5f);
  p = fmaf(x, p, 1.f);
  const float small = x * p;
  const float big = __expf(x) - 1.f;
  return fabsf(x) < 0.25f ? small : big;
}

// FP32 value/gradient/Laplacian of shell s at offset d (r2 = |d|^2).
__device__ __forceinline__ void shell_derivs_f(const DevSys& S, int s, const float d[3], float r2,
                                               float* __restrict__ out, int n_bf) {
  const int l = __ldg(S.sh_l + s), np = __ldg(S.sh_nprim + s), off = __ldg(S.sh_off + s), bf = __ldg(S.sh_bf + s);
  if (l == -1) {
    const float ir = rsqrtf(r2), r = r2 * ir;
    float v = 0.f, dr = 0.f, lp = 0.f;
    for (int q = 0; q < np; ++q) {
      const float z = __ldg(S.expsf + off + q);
      const float h = __ldg(S.coefsf + off + q) * __expf(-z * r);
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
      const float al = __ldg(S.expsf + off + q);
      const float h = __ldg(S.coefsf + off + q) * __expf(-al * r2);
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
      const float al = __ldg(S.expsf + off + q);
      const float h = __ldg(S.coefsf + off + q) * __expf(-al * r2);
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

// FP32 Jastrow pair constant for electrons i, j.
__device__ __forceinline__ float pair_cf(const DevSys& S, const Layout& L, int i, int j) {
  return ((i < L.n_up) == (j < L.n_up)) ? S.j2_parf : S.j2_antif;
}

// FP64 values of the functions of shell s (for the rows of A).
__device__ __forceinline__ void shell_values_d(const DevSys& S, int s, const double d[3], double r2,
                                               double* __restrict__ out, const double* T) {
  const int l = __ldg(S.sh_l + s), np = __ldg(S.sh_nprim + s), off = __ldg(S.sh_off + s), bf = __ldg(S.sh_bf + s);
  const double arg = l == -1 ? r2 * rsqrt_nr(r2) : r2;
  double rad = 0.0;
  for (int q = 0; q < np; ++q) rad = fma(__ldg(S.coefs + off + q), exp_tab(-__ldg(S.exps + off + q) * arg, T), rad);
  if (l == 1) {
    out[bf] = d[0] * rad;
    out[bf + 1] = d[1] * rad;
    out[bf + 2] = d[2] * rad;
  } else {
    out[bf] = rad;
  }
}

// ------------------------------------------------------------ tensor cores
// Warp-level tensor-core form of the FP32 orbital contractions: D[r][k] =
// sum_mu A(r, mu) C[k][mu] for rows r < nr and orbitals k < nk, with
// A(r, mu) = a[r * rs + mu * ms] in shared memory and C the FP32 copy of the
// MO coefficients (n_orb x n_bf, read through L1).  The rows go through the
// 16-row M dimension of mma.sync, the orbitals through its 8-column N
// dimension and the basis functions through K; rows, orbitals and basis
// functions past the ends are zero operands.  tc = 1: m16n8k8 with both
// operands rounded to TF32 (cvt.rna, 10 explicit mantissa bits); tc = 2:
// m16n8k16 with BF16 operands (round to nearest even, 7 bits).  Accumulation
// is FP32 in both.  tc = 3: each FP32 operand x is split into TF32 parts
// hi = tf32(x), lo = tf32(x - hi) and the product formed as
// lo_a hi_b + hi_a lo_b + hi_a hi_b (three m16n8k8 MMAs, the small terms
// first; lo_a lo_b ~ 2^-22 |a b| is dropped), which restores close to FP32
// accuracy on the tensor cores.  Fragment layouts (g = lane / 4, t = lane % 4):
//   TF32 A: (g, t) (g + 8, t) (g, t + 4) (g + 8, t + 4); B: (k = t, n = g) (t + 4, g)
//   BF16 A: pairs (g, 2t..2t+1) (g + 8, 2t..) (g, 2t+8..2t+9) (g + 8, 2t+8..);
//        B: pairs (k = 2t..2t+1, n = g) (2t+8..2t+9, g), the lower k in the low half
//   D (both): (g, 2t) (g, 2t + 1) (g + 8, 2t) (g + 8, 2t + 1)
// store(r, k, v) receives every (r < nr, k < nk) result once.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float& d0, float& d1, float& d2, float& d3, const uint32_t a[4],
                                         const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <class Store>
__device__ __forceinline__ void tc_contract(int tc, const float* a, int rs, int ms, int nr, const float* __restrict__ Cf,
                                            int nbf, int nk, int lane, Store store) {
  const int g = lane >> 2, t = lane & 3;
  auto A = [&](int r, int mu) { return (r < nr && mu < nbf) ? a[r * rs + mu * ms] : 0.f; };
  auto B = [&](int k, int mu) { return (k < nk && mu < nbf) ? __ldg(Cf + (size_t)k * nbf + mu) : 0.f; };
  for (int r0 = 0; r0 < nr; r0 += 16) {
    for (int n0 = 0; n0 < nk; n0 += 8) {
      float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
      if (tc == 1) {
        for (int k0 = 0; k0 < nbf; k0 += 8) {
          const uint32_t av[4] = {to_tf32(A(r0 + g, k0 + t)), to_tf32(A(r0 + g + 8, k0 + t)),
                                  to_tf32(A(r0 + g, k0 + t + 4)), to_tf32(A(r0 + g + 8, k0 + t + 4))};
          const uint32_t bv[2] = {to_tf32(B(n0 + g, k0 + t)), to_tf32(B(n0 + g, k0 + t + 4))};
          mma_tf32(d0, d1, d2, d3, av, bv);
        }
      } else if (tc == 3) {
        for (int k0 = 0; k0 < nbf; k0 += 8) {
          const float af[4] = {A(r0 + g, k0 + t), A(r0 + g + 8, k0 + t), A(r0 + g, k0 + t + 4),
                               A(r0 + g + 8, k0 + t + 4)};
          const float bf[2] = {B(n0 + g, k0 + t), B(n0 + g, k0 + t + 4)};
          uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            ah[j] = to_tf32(af[j]);
            al[j] = to_tf32(af[j] - __uint_as_float(ah[j]));
          }
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            bh[j] = to_tf32(bf[j]);
            bl[j] = to_tf32(bf[j] - __uint_as_float(bh[j]));
          }
          mma_tf32(d0, d1, d2, d3, al, bh);
          mma_tf32(d0, d1, d2, d3, ah, bl);
          mma_tf32(d0, d1, d2, d3, ah, bh);
        }
      } else {
        for (int k0 = 0; k0 < nbf; k0 += 16) {
          const int c0 = k0 + 2 * t, c1 = k0 + 2 * t + 8;
          const uint32_t a0 = pack_bf16(A(r0 + g, c0), A(r0 + g, c0 + 1)),
                         a1 = pack_bf16(A(r0 + g + 8, c0), A(r0 + g + 8, c0 + 1)),
                         a2 = pack_bf16(A(r0 + g, c1), A(r0 + g, c1 + 1)),
                         a3 = pack_bf16(A(r0 + g + 8, c1), A(r0 + g + 8, c1 + 1));
          const uint32_t b0 = pack_bf16(B(n0 + g, c0), B(n0 + g, c0 + 1)),
                         b1 = pack_bf16(B(n0 + g, c1), B(n0 + g, c1 + 1));
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
              "{%0, %1, %2, %3};"
              : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
              : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
      }
      const int ra = r0 + g, rb = r0 + g + 8, ka = n0 + 2 * t, kb = n0 + 2 * t + 1;
      if (ra < nr && ka < nk) store(ra, ka, d0);
      if (ra < nr && kb < nk) store(ra, kb, d1);
      if (rb < nr && ka < nk) store(rb, ka, d2);
      if (rb < nr && kb < nk) store(rb, kb, d3);
    }
  }
}

// Orbital rows at one point q: FP64 values phiv[k] and FP32 gradient /
// Laplacian phi5[(c-1) * n_max + k], c = 1..4, for the first n_sig orbitals.
__device__ void orbital_rows_m(const DevSys& S, const Layout& L, const LayoutM& M, const double q[3], int n_sig,
                               float* sm, const double* T, int lane) {
  double* chiv = (double*)(sm + M.chiv);
  double* phiv = (double*)(sm + M.phiv);
  float* chi5 = sm + M.chi5;
  float* phi5 = sm + M.phi5;
  for (int s = lane; s < S.n_shell; s += WARP) {
    const int atom = __ldg(S.sh_atom + s);
    const double d[3] = {q[0] - __ldg(S.R + 3 * atom), q[1] - __ldg(S.R + 3 * atom + 1),
                         q[2] - __ldg(S.R + 3 * atom + 2)};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    shell_values_d(S, s, d, r2, chiv, T);
    const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    shell_derivs_f(S, s, df, (float)r2, chi5, L.n_bf);
  }
  __syncwarp();
  // FP64 values: n_sig orbitals x n_bf terms spread over all lanes in groups
  // of G lanes per orbital (strided partial sums, fixed-order xor reduction)
  {
    int G = 1;
    while (G * 2 * n_sig <= WARP) G *= 2;
    for (int base = 0; base < n_sig; base += WARP / G) {
      const int k = base + lane / G, sub = lane % G;
      double acc = 0.0;
      if (k < n_sig) {
        const double* crow = S.C + (size_t)k * L.n_bf;
        for (int mu = sub; mu < L.n_bf; mu += G) acc = fma(__ldg(crow + mu), chiv[mu], acc);
      }
      for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (k < n_sig && sub == 0) phiv[k] = acc;
    }
  }
  if (M.tc) {
    // the four derivative rows (chi5 rows 1..4) as one tensor-core tile
    tc_contract(M.tc, chi5 + L.n_bf, L.n_bf, 1, 4, S.Cf, L.n_bf, n_sig, lane,
                [&](int r, int k, float v) { phi5[r * L.n_max + k] = v; });
  } else {
    for (int o = lane; o < 4 * n_sig; o += WARP) {
      const int c = 1 + o / n_sig, k = o - (c - 1) * n_sig;
      const float* crow = S.Cf + (size_t)k * L.n_bf;
      const float* x = chi5 + c * L.n_bf;
      float acc = 0.f;
      for (int mu = 0; mu < L.n_bf; ++mu) acc = fmaf(__ldg(crow + mu), x[mu], acc);
      phi5[(c - 1) * L.n_max + k] = acc;
    }
  }
  __syncwarp();
}

__device__ void electron_potentials_f(const DevSys& S, const float q[3], float a, int lane, float& nu,
                                      float& nucap) {
  nu = 0.f;
  nucap = 0.f;
  for (int I = lane; I < S.n_nuc; I += WARP) {
    const float dx = q[0] - __ldg(S.Rf + 3 * I), dy = q[1] - __ldg(S.Rf + 3 * I + 1),
                dz = q[2] - __ldg(S.Rf + 3 * I + 2);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float Z = __ldg(S.Zf + I);
    if (__ldg(S.kind + I) == 0) {
      nu -= Z / r;
      nucap -= Z / fmaxf(r, a);
    } else {
      const float v = -Z * erff(r / __ldg(S.rcf + I)) / r;
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

// FP64 re-inversion of the FP64 orbital values (both spin blocks).
__device__ bool reinvert_m(const Layout& L, const LayoutM& M, double* gblk, float* sm, double* scratch, int lane) {
  bool sing = false;
  const double* val = cache_val(L, gblk);
  double* bt = (double*)(sm + M.bt);
  // the work matrix in the move scratch region (free between hops) when it fits
  // and is 8-byte aligned, else in the global scratch
  if ((M.chi5 & 1) == 0 && 4 * L.n_max * L.n_max <= M.phi5 - M.chi5) scratch = (double*)(sm + M.chi5);
  for (int blk = 0; blk < 2; ++blk) {
    const int n = blk ? L.n_dn : L.n_up;
    const int e0 = blk ? L.n_up : 0;
    const int bto = blk ? L.n_up * L.n_up : 0;
    if (n == 0) continue;
    for (int o = lane; o < n * 2 * n; o += WARP) {
      const int r = o / (2 * n), c = o - r * 2 * n;
      scratch[o] = c < n ? val[(e0 + r) * L.n_max + c] : (c - n == r ? 1.0 : 0.0);
    }
    __threadfence_block();
    __syncwarp();
    sing |= warp_gauss_jordan(scratch, n, lane, (double*)(sm + M.row));
    for (int o = lane; o < n * n; o += WARP) {
      const int i = o / n, k = o - i * n;
      bt[bto + o] = scratch[k * 2 * n + n + i];
    }
    __syncwarp();
  }
  return sing;
}

// FP32 copy of B^T for the spin blocks of electrons [e0, e1) (whole blocks).
__device__ void refresh_b32(const Layout& L, const LayoutM& M, float* sm, int e0, int e1, int lane) {
  const double* bt = (const double*)(sm + M.bt);
  float* b32 = sm + M.b32;
  const int o0 = e0 < L.n_up ? 0 : L.n_up * L.n_up;
  const int o1 = e1 <= L.n_up ? L.n_up * L.n_up : L.n_up * L.n_up + L.n_dn * L.n_dn;
  for (int o = o0 + lane; o < o1; o += WARP) b32[o] = (float)bt[o];
  __syncwarp();
}

// Orbital differences dph[p][k] = sum_mu C_k,mu dchi_mu(p) of the hops
// p = p0 + c, c in [0, n_hops), read from dchi[mu * ld + c]; k over the
// electron's spin block, each dot split over G lanes.
__device__ void orbital_diffs(const DevSys& S, const Layout& L, float* dph, const float* dchi, int ld, int p0,
                              int n_hops, int lane, int tc = 0) {
  const int nm = L.n_max, nbf = L.n_bf;
  if (tc) {
    // hops through the M dimension (16 per tile), orbitals of the larger spin
    // block through N; orbitals past a hop's own block are stored as zeros
    tc_contract(tc, dchi, 1, ld, n_hops, S.Cf, nbf, nm, lane, [&](int c, int k, float v) {
      const int p = p0 + c;
      const int nsig = (p / 6) < L.n_up ? L.n_up : L.n_dn;
      dph[p * nm + k] = k < nsig ? v : 0.f;
    });
    __syncwarp();
    return;
  }
  const int n_out = n_hops * nm, G = split_factor(n_out, nbf);
  const int chunk = (nbf + G - 1) / G, n_task = n_out * G;
  for (int base = 0; base < n_task; base += WARP) {
    const int task = base + lane, o = task / G, part = task - o * G;
    const int c = o / nm, k = o - c * nm;
    const int p = p0 + c;
    const int nsig = (p / 6) < L.n_up ? L.n_up : L.n_dn;
    float acc = 0.f;
    if (task < n_task && k < nsig) {
      const float* crow = S.Cf + (size_t)k * nbf;
      const int mu1 = min(nbf, (part + 1) * chunk);
      for (int mu = part * chunk; mu < mu1; ++mu) acc = fmaf(__ldg(crow + mu), dchi[(size_t)mu * ld + c], acc);
    }
    for (int sh = 1; sh < G; sh <<= 1) acc += __shfl_xor_sync(FULL, acc, sh);
    if (task < n_task && part == 0) dph[p * nm + k] = acc;
  }
  __syncwarp();
}

// Determinant ratio minus one of hops [p0, p1): dph[p] . B[:, i] (FP32 B).
__device__ void det_diffs(const Layout& L, const LayoutM& M, float* sm, const float* dph, int p0, int p1, int lane) {
  const float* b32 = sm + M.b32;
  float* hdm = sm + M.hdm;
  for (int p = p0 + lane; p < p1; p += WARP) {
    const SpinRef sr = spin_ref(L, p / 6);
    const float* brow = b32 + sr.bt_off + sr.ii * sr.n;
    const float* f = dph + p * L.n_max;
    float D = 0.f;
    for (int k = 0; k < sr.n; ++k) D = fmaf(f[k], brow[k], D);
    hdm[p] = D;
  }
  __syncwarp();
}

// ------------------------------------------------------------ evaluation
// FP32 pair geometry and Pade helpers, written with explicit FMAs so that every
// call site rounds identically (the incremental swaps subtract exactly the
// term that was added).
__device__ __forceinline__ float sqdistf(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }
// Jastrow difference of a hop, u(r') - u(r) = c del t t' / (r' + r), from the
// current r, t = 1/(1 + b r) and del = r'^2 - r^2 (r'^2 formed as r r + del).
__device__ __forceinline__ float pade_delta(float r, float t, float del, float c, float b) {
  const float sp = fmaf(r, r, del);
  const float rp = sp * rsqrtf(sp);
  const float tp = __fdividef(1.f, fmaf(b, rp, 1.f));
  return c * del * t * __fdividef(tp, rp + r);
}

// Assembly (FP64) from the r - 1 values, Jastrow and determinant derivatives.
__device__ EvalOut assemble_m(const DevSys& S, const Layout& L, const LayoutM& M, const float* sm, double ia2,
                              int node_rule, int lane) {
  const int ne = L.n_e;
  const float* dl = sm + M.dl;
  const float* ej = sm + M.ej;
  const float* ep = sm + M.ep;
  const double* dd = (const double*)(sm + M.dd);
  bool has_node = false;
  for (int i = lane; i < ne; i += WARP)
    for (int d = 0; d < 6; ++d) has_node |= dl[6 * i + d] < -1.f;
  const bool any_node = __any_sync(FULL, has_node);
  // FP64 accumulators: kept ratios, node-crossing ratios, and the potential
  // part of W (sum of nu_opt and the e-e terms)
  double kept = 0.0, negs = 0.0, pot = 0.0;
  int nnode = 0, nkept = 0;
  for (int i = lane; i < ne; i += WARP) {
    float sd = 0.f, skd = 0.f, sneg = 0.f;
    int nk = 0;
    bool node = false;
    for (int d = 0; d < 6; ++d) {
      const float x1 = dl[6 * i + d];     // r - 1
      sd += x1;
      if (x1 > -1.f) { skd += x1; ++nk; }
      if (x1 < -1.f) { sneg -= 1.f + x1; node = true; }
    }
    nkept += nk;
    kept += (double)skd;
    negs += (double)sneg;
    const float* q = ej + 5 * i;
    const double* dv = dd + 4 * i;
    // Jastrow part of the Laplacian in FP32, determinant parts in FP64
    const float jl = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3])));
    const double cross = dv[0] * (double)q[0] + dv[1] * (double)q[1] + dv[2] * (double)q[2];
    const double lap = dv[3] + 2.0 * cross + (double)jl;
    const double nu_zv = (double)ep[2 * i] + 0.5 * ((double)sd * ia2 - lap);
    bool apply;
    if (node_rule == 0) apply = node;
    else if (node_rule == 1) apply = any_node;
    else if (node_rule == 2) apply = true;
    else apply = false;
    pot += (apply ? fmax(nu_zv, (double)ep[2 * i + 1]) : nu_zv) + (double)q[4];
    nnode += node ? 1 : 0;
  }
  {
    const double v[4] = {kept, negs, pot, 0.0};
    const double t = warp_sum4(v, lane);
    kept = __shfl_sync(FULL, t, 0);
    negs = __shfl_sync(FULL, t, 8);
    pot = __shfl_sync(FULL, t, 16);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    nnode += __shfl_xor_sync(FULL, nnode, o);
    nkept += __shfl_xor_sync(FULL, nkept, o);
  }
  kept += (double)nkept;
  EvalOut e;
  const double i2a2 = 0.5 * ia2;
  e.kept = kept;
  e.bbar = kept * i2a2;
  e.vsf = negs * i2a2;
  e.W = 3.0 * ne * ia2 + pot + S.v_ii + e.vsf;
  e.eL = e.W - e.bbar;
  e.n_node = nnode;
  return e;
}

// FP64 determinant derivatives for electrons [e0, e1) from the FP32
// derivative cache and FP64 B.
__device__ void det_derivs_m(const Layout& L, const LayoutM& M, double* gblk, float* sm, int e0, int e1, int lane) {
  const double* bt = (const double*)(sm + M.bt);
  const double* der = cache_der(L, gblk);
  double* dd = (double*)(sm + M.dd);
  for (int o = lane + 4 * e0; o < 4 * e1; o += WARP) {
    const int i = o >> 2, c = o & 3;
    const SpinRef sr = spin_ref(L, i);
    const double* brow = bt + sr.bt_off + sr.ii * sr.n;
    const double* ce = der + (i * 4 + c) * L.n_max;
    double acc = 0.0;
    for (int k = 0; k < sr.n; ++k) acc = fma(ce[k], brow[k], acc);
    dd[o] = acc;
  }
}

// Geometry, pair data, primitive values and Jastrow derivative sums of one
// electron e against partner t (an electron for t < n_e - 1, else a nucleus);
// accumulates into gx, gy, gz, LJ, vee.  With pt set, the pair's derivative
// terms (u'/r, u'' + 2u'/r, 1/(2r)) go to pt[e][j].
__device__ __forceinline__ void partner_terms(const DevSys& S, const Layout& L, const LayoutM& M, float* sm,
                                              const MArr& AR, int e, int t, float* pt, float& gx, float& gy, float& gz,
                                              float& LJ, float& vee) {
  const int ne = L.n_e;
  const float* xf = sm + M.xf;
  const float bj = S.j2_bf;
  const float xe = xf[3 * e], ye = xf[3 * e + 1], ze = xf[3 * e + 2];
  if (t < ne - 1) {
    const int j = t < e ? t : t + 1;
    const float dx = xe - xf[3 * j], dy = ye - xf[3 * j + 1], dz = ze - xf[3 * j + 2];
    const float s = sqdistf(dx, dy, dz);
    const float ir = rsqrtf(s), r = s * ir;
    const float c = pair_cf(S, L, e, j);
    const float tt = __fdividef(1.f, fmaf(bj, r, 1.f));
    float* pp = AR.pair + e * M.pair_st + 2 * j;
    pp[0] = r; pp[1] = tt;
    const float up = c * tt * tt, upp = -2.f * bj * up * tt, f = up * ir;
    const float lap = upp + 2.f * f, hir = 0.5f * ir;
    gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
    LJ += lap;
    vee += hir;
    if (pt) {
      float* q = pt + 3 * (e * ne + j);
      q[0] = f; q[1] = lap; q[2] = hir;
    }
  } else {
    const int I = t - (ne - 1);
    const float dx = xe - __ldg(S.Rf + 3 * I), dy = ye - __ldg(S.Rf + 3 * I + 1), dz = ze - __ldg(S.Rf + 3 * I + 2);
    const float s = sqdistf(dx, dy, dz);
    float* gg = AR.geo + e * M.geo_st + 4 * I;
    gg[0] = dx; gg[1] = dy; gg[2] = dz; gg[3] = s;
    const float ir = rsqrtf(s), r = s * ir;
    float* hc = AR.hcur + e * M.hcur_st;
    for (int sh = __ldg(S.atom_sh + I); sh < __ldg(S.atom_sh + I + 1); ++sh) {
      const int np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh);
      const float arg = __ldg(S.sh_l + sh) == -1 ? r : s;
      for (int q = 0; q < np; ++q) hc[off + q] = __ldg(S.coefsf + off + q) * __expf(-__ldg(S.expsf + off + q) * arg);
    }
    const float A = __ldg(S.j1Af + I), B = __ldg(S.j1Bf + I);
    const float tt = __fdividef(1.f, fmaf(B, r, 1.f));
    AR.rt1[e * M.rt1_st + 2 * I] = r;
    AR.rt1[e * M.rt1_st + 2 * I + 1] = tt;
    if (A != 0.f) {
      const float vp = -A * tt * tt, vpp = -2.f * B * vp * tt, f = vp * ir;
      gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
      LJ += vpp + 2.f * f;
    }
  }
}

// Full evaluation: every hop ratio as r - 1 (FP32), the FP64 accumulators and
// every cache of the incremental update (the pair caches in scr when set).
// Requires the FP32 copy of B current.
template <int BIG = -1>
__device__ EvalOut eval_full_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm,
                               const ScrM& scr, double a, int node_rule, int lane) {
  const int ne = L.n_e, nn = S.n_nuc, P = L.n_hop;
  const float af = (float)a, a2f = af * af;
  const float* xf = sm + M.xf;
  float* dchi = scr.dchi;
  float* dl = sm + M.dl;
  float* ej = sm + M.ej;
  const MArr AR = marr<BIG>(M, sm, scr);
  const float* geo = AR.geo;
  const float* rt1 = AR.rt1;
  const float* pair = AR.pair;
  const float* hcur = AR.hcur;
  float* hdm = sm + M.hdm;
  float* hj1 = sm + M.hj1;
  float* hj2 = sm + M.hj2;
  const float bj = S.j2_bf;
  // (1) current configuration, G lanes per electron
  {
    int npad = 1;
    while (npad < ne) npad <<= 1;
    const int G = npad >= WARP ? 1 : WARP / npad;
    const int per = ne - 1 + nn;
    for (int base = 0; base < ne; base += WARP / G) {
      const int e = base + lane / G, sub = lane % G;
      float gx = 0.f, gy = 0.f, gz = 0.f, LJ = 0.f, vee = 0.f;
      if (e < ne)
        for (int t = sub; t < per; t += G) partner_terms(S, L, M, sm, AR, e, t, scr.pt, gx, gy, gz, LJ, vee);
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
  det_derivs_m(L, M, gblk, sm, 0, ne, lane);
  __syncwarp();
  // (3) every hop: basis differences (to scratch) and the one-body / pair
  // Jastrow differences
  for (int p = lane; p < P; p += WARP) {
    const int i = p / 6, d = p - 6 * i, ax = d >> 1;
    const float sa = (d & 1) ? -af : af;
    const float s2a = sa + sa;
    const float* hc = hcur + i * M.hcur_st;
    float J1 = 0.f;
    for (int I = 0; I < nn; ++I) {
      const float* gg = geo + i * M.geo_st + 4 * I;
      const float del = fmaf(s2a, gg[ax], a2f);             // |r'-R|^2 - |r-R|^2
      const float r = rt1[i * M.rt1_st + 2 * I];
      const float A = __ldg(S.j1Af + I);
      if (A != 0.f) J1 += pade_delta(r, rt1[i * M.rt1_st + 2 * I + 1], del, -A, __ldg(S.j1Bf + I));
      const float sp = gg[3] + del;
      const float rp = sp * rsqrtf(sp);
      for (int sh = __ldg(S.atom_sh + I); sh < __ldg(S.atom_sh + I + 1); ++sh) {
        const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = __ldg(S.sh_off + sh),
                  bf = __ldg(S.sh_bf + sh);
        const float arg = l == -1 ? __fdividef(del, rp + r) : del;
        float rd = 0.f, rn = 0.f;   // sums of h' - h and of h'
        for (int q = 0; q < np; ++q) {
          const float h = hc[off + q];
          // the clamp only acts where h has already underflowed to 0
          const float dh = h * expm1_fast(fminf(-__ldg(S.expsf + off + q) * arg, 80.f));
          rd += dh;
          rn += h + dh;
        }
        if (l != 1) {
          dchi[(size_t)bf * P + p] = rd;
        } else {
          for (int k = 0; k < 3; ++k) dchi[(size_t)(bf + k) * P + p] = fmaf(gg[k], rd, k == ax ? sa * rn : 0.f);
        }
      }
    }
    const float xia = xf[3 * i + ax];
    const float* pr = pair + i * M.pair_st;
    float J2 = 0.f;
    for (int j = 0; j < ne; ++j) {
      if (j == i) continue;
      const float del = fmaf(s2a, xia - xf[3 * j + ax], a2f);
      const float v = pade_delta(pr[2 * j], pr[2 * j + 1], del, pair_cf(S, L, i, j), bj);
      J2 += v;
      if (scr.u2) scr.u2[(size_t)j * P + p] = v;
    }
    hj1[p] = J1;
    hj2[p] = J2;
  }
  __threadfence_block();
  __syncwarp();
  // (4) orbital differences of every hop and the determinant ratios
  orbital_diffs(S, L, AR.dph, dchi, P, 0, P, lane, M.tc);
  det_diffs(L, M, sm, AR.dph, 0, P, lane);
  for (int p = lane; p < P; p += WARP) {
    const float D = hdm[p];
    const float J = expm1_fast(hj1[p] + hj2[p]);
    dl[p] = fmaf(D, J, D + J);
  }
  __syncwarp();
  return assemble_m(S, L, M, sm, 1.0 / (a * a), node_rule, lane);
}

// Incremental evaluation after electron m hopped (old position at xo/xfo),
// mirroring eval_incr of the FP64 kernel: m's terms from scratch, the other
// electrons' pair terms with m swapped using the cached old terms (scr.pt for
// the derivative sums, scr.u2 for the hop differences; the new difference of
// hop d of electron i with m is m's opposite hop d ^ 1 with i).
template <int BIG = -1>
__device__ EvalOut eval_incr_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm,
                               const ScrM& scr, int m, bool all_blocks, double a, double ia2, int node_rule,
                               int lane) {
  const int ne = L.n_e, nn = S.n_nuc, P = L.n_hop;
  const int per = ne - 1 + nn;
  const float af = (float)a, a2f = af * af;
  const float* xf = sm + M.xf;
  const float* xfo = sm + M.xfo;
  float* dc6 = sm + M.chi5;     // basis differences at m's hops [n_bf][6]
  float* dl = sm + M.dl;
  float* ej = sm + M.ej;
  const MArr AR = marr<BIG>(M, sm, scr);
  const float* geo = AR.geo;
  const float* rt1 = AR.rt1;
  float* pair = AR.pair;
  float* hdm = sm + M.hdm;
  float* hj1 = sm + M.hj1;
  float* hj2 = sm + M.hj2;
  float* tmp = sm + M.tmp;
  const float bj = S.j2_bf;
  // (A) electron m from scratch (geometry, pair data both ways, primitives,
  // Jastrow sums); (B) the partner electron's sums swap their term with m
  {
    const float xm = xf[3 * m], ym = xf[3 * m + 1], zm = xf[3 * m + 2];
    const float xo0 = xfo[0], xo1 = xfo[1], xo2 = xfo[2];
    float gx = 0.f, gy = 0.f, gz = 0.f, LJ = 0.f, vee = 0.f;
    for (int t = lane; t < per; t += WARP) {
      if (t < ne - 1) {
        const int j = t < m ? t : t + 1;
        // the old pair terms first: the stores below could alias them
        float* pm = scr.pt + 3 * (m * ne + j);
        float* pj = scr.pt + 3 * (j * ne + m);
        const float of = pm[0], ol = pm[1], oh = pm[2];
        const float pxj = xf[3 * j], pyj = xf[3 * j + 1], pzj = xf[3 * j + 2];
        const float dx = xm - pxj, dy = ym - pyj, dz = zm - pzj;
        const float s = sqdistf(dx, dy, dz);
        const float ir = rsqrtf(s), r = s * ir;
        const float c = pair_cf(S, L, m, j);
        const float tt = __fdividef(1.f, fmaf(bj, r, 1.f));
        float* pp = pair + m * M.pair_st + 2 * j;
        float* pq = pair + j * M.pair_st + 2 * m;
        pp[0] = r; pp[1] = tt;
        pq[0] = r; pq[1] = tt;
        const float up = c * tt * tt, upp = -2.f * bj * up * tt, f = up * ir;
        const float lap = upp + 2.f * f, hir = 0.5f * ir;
        gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
        LJ += lap;
        vee += hir;
        const float ox = pxj - xo0, oy = pyj - xo1, oz = pzj - xo2;
        float* q = ej + 5 * j;
        q[0] += f * -dx - of * ox;
        q[1] += f * -dy - of * oy;
        q[2] += f * -dz - of * oz;
        q[3] += lap - ol;
        q[4] += hir - oh;
        pm[0] = f; pm[1] = lap; pm[2] = hir;
        pj[0] = f; pj[1] = lap; pj[2] = hir;
      } else {
        partner_terms(S, L, M, sm, AR, m, t, nullptr, gx, gy, gz, LJ, vee);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      gx += __shfl_xor_sync(FULL, gx, o);
      gy += __shfl_xor_sync(FULL, gy, o);
      gz += __shfl_xor_sync(FULL, gz, o);
      LJ += __shfl_xor_sync(FULL, LJ, o);
      vee += __shfl_xor_sync(FULL, vee, o);
    }
    if (lane == 0) {
      float* q = ej + 5 * m;
      q[0] = gx; q[1] = gy; q[2] = gz; q[3] = LJ; q[4] = vee;
    }
  }
  // (C) determinant derivatives of the refreshed block(s)
  const SpinRef srm = spin_ref(L, m);
  const int b0 = all_blocks ? 0 : m - srm.ii, b1 = all_blocks ? ne : m - srm.ii + srm.n;
  det_derivs_m(L, M, gblk, sm, b0, b1, lane);
  __threadfence_block();
  __syncwarp();
  // (D) basis differences at m's six hops, one (hop, shell) per lane, and m's
  // Jastrow differences, one (hop, partner) per lane
  const float* hc = AR.hcur + m * M.hcur_st;
  for (int o = lane; o < 6 * S.n_shell; o += WARP) {
    const int d = o / S.n_shell, sh = o - d * S.n_shell, ax = d >> 1;
    const float sa = (d & 1) ? -af : af;
    const int I = CHK(__ldg(S.sh_atom + sh), S.n_nuc);
    const float* gg = geo + m * M.geo_st + 4 * I;
    const float del = fmaf(sa + sa, gg[ax], a2f);
    const float r = rt1[m * M.rt1_st + 2 * I];
    const int l = __ldg(S.sh_l + sh), np = __ldg(S.sh_nprim + sh), off = CHK(__ldg(S.sh_off + sh), S.n_prim),
              bf = CHK(__ldg(S.sh_bf + sh), L.n_bf - (l == 1 ? 2 : 0));
    const float sp = gg[3] + del;
    const float arg = l == -1 ? __fdividef(del, sp * rsqrtf(sp) + r) : del;
    float rd = 0.f, rn = 0.f;
    for (int q = 0; q < np; ++q) {
      const float h = hc[off + q];
      const float dh = h * expm1_fast(fminf(-__ldg(S.expsf + off + q) * arg, 80.f));
      rd += dh;
      rn += h + dh;
    }
    if (l != 1) {
      dc6[bf * 6 + d] = rd;
    } else {
      for (int k = 0; k < 3; ++k) dc6[(bf + k) * 6 + d] = fmaf(gg[k], rd, k == ax ? sa * rn : 0.f);
    }
  }
  __syncwarp();
  orbital_diffs(S, L, AR.dph, dc6, 6, 6 * m, 6, lane, M.tc);
  for (int o = lane; o < 6 * per; o += WARP) {
    const int d = o / per, t = o - d * per, ax = d >> 1;
    const float sa = (d & 1) ? -af : af;
    float v = 0.f;
    if (t < ne - 1) {
      const int j = t < m ? t : t + 1;
      const float* pp = pair + m * M.pair_st + 2 * j;
      const float del = fmaf(sa + sa, xf[3 * m + ax] - xf[3 * j + ax], a2f);
      v = pade_delta(pp[0], pp[1], del, pair_cf(S, L, m, j), bj);
      scr.u2[CHK((size_t)j * P + 6 * m + d, (size_t)ne * P)] = v;
    } else {
      const int I = t - (ne - 1);
      const float A = __ldg(S.j1Af + I);
      const float* gg = geo + m * M.geo_st + 4 * I;
      if (A != 0.f)
        v = pade_delta(rt1[m * M.rt1_st + 2 * I], rt1[m * M.rt1_st + 2 * I + 1], fmaf(sa + sa, gg[ax], a2f), -A,
                       __ldg(S.j1Bf + I));
    }
    tmp[CHK(o, M.phi5 - M.chi5)] = v;
  }
  __threadfence_block();
  __syncwarp();
  {
    // sums over partners of each of m's hops: four lanes per hop
    const int d = lane >> 2, sub = lane & 3;
    float J1 = 0.f, J2 = 0.f;
    if (d < 6)
      for (int t = sub; t < per; t += 4) {
        const float v = tmp[d * per + t];
        if (t < ne - 1) J2 += v;
        else J1 += v;
      }
    J1 += __shfl_xor_sync(FULL, J1, 1);
    J2 += __shfl_xor_sync(FULL, J2, 1);
    J1 += __shfl_xor_sync(FULL, J1, 2);
    J2 += __shfl_xor_sync(FULL, J2, 2);
    if (d < 6 && sub == 0) {
      hj1[6 * m + d] = J1;
      hj2[6 * m + d] = J2;
    }
  }
  // (E) determinant differences of the refreshed block(s) from the cached
  // orbital differences
  det_diffs(L, M, sm, AR.dph, 6 * b0, 6 * b1, lane);
  // (F) pair Jastrow differences of the other electrons' hops: swap the term
  // with m; up to four old terms per lane loaded before any store (overlapped
  // global-memory latencies)
  {
    float* um = scr.u2 + (size_t)m * P;
    for (int base = 0; base < P; base += 4 * WARP) {
      float vn[4], uo[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = base + k * WARP + lane, i = p / 6;
        const bool ok = p < P && i != m;
        vn[k] = ok ? tmp[((p - 6 * i) ^ 1) * per + (i < m ? i : i - 1)] : 0.f;
        uo[k] = ok ? um[p] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = base + k * WARP + lane, i = p / 6;
        if (p < P && i != m) {
          hj2[p] += vn[k] - uo[k];
          um[p] = vn[k];
        }
      }
    }
  }
  __threadfence_block();
  __syncwarp();
  // (G) all hops, as r - 1
  for (int p = lane; p < P; p += WARP) {
    const float D = hdm[p];
    const float J = expm1_fast(hj1[p] + hj2[p]);
    dl[p] = fmaf(D, J, D + J);
  }
  __threadfence_block();
  __syncwarp();
  return assemble_m(S, L, M, sm, ia2, node_rule, lane);
}

__device__ EvalOut init_walker_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm,
                                 const ScrM& scr, double a, int node_rule, const double* T, int lane, bool& singular) {
  double* val = cache_val(L, gblk);
  double* der = cache_der(L, gblk);
  const double* x = (const double*)(sm + M.x);
  float* xf = sm + M.xf;
  float* ep = sm + M.ep;
  const double* phiv = (const double*)(sm + M.phiv);
  const float* phi5 = sm + M.phi5;
  for (int o = lane; o < 3 * L.n_e; o += WARP) xf[o] = (float)x[o];
  __syncwarp();
  for (int i = 0; i < L.n_e; ++i) {
    const int n = i < L.n_up ? L.n_up : L.n_dn;
    const double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    orbital_rows_m(S, L, M, q, n, sm, T, lane);
    for (int o = lane; o < L.n_max; o += WARP) val[i * L.n_max + o] = phiv[o];
    for (int o = lane; o < 4 * L.n_max; o += WARP) der[i * 4 * L.n_max + o] = phi5[o];
    float nu, nucap;
    const float qf[3] = {xf[3 * i], xf[3 * i + 1], xf[3 * i + 2]};
    electron_potentials_f(S, qf, (float)a, lane, nu, nucap);
    if (lane == 0) {
      ep[2 * i] = nu;
      ep[2 * i + 1] = nucap;
    }
    __syncwarp();
  }
  __threadfence_block();
  singular = reinvert_m(L, M, gblk, sm, scr.gj, lane);
  refresh_b32(L, M, sm, 0, L.n_e, lane);
  return eval_full_m(S, L, M, gblk, sm, scr, a, node_rule, lane);
}

// Heat-bath choice from r - 1 values: same order and rule as the FP64 path
// (first hop whose running sum of kept ratios exceeds u * total, last kept hop
// if rounding leaves none), with the running sums formed by warp scans over
// chunks of 32 hops in FP32; total is the evaluation's sum of kept ratios.
__device__ int choose_hop_m(const float* dl, int n_hop, double u, double total, int lane) {
  if (!dpos(total)) return -1;
  const float t = (float)(u * total);
  float base = 0.f;
  int last = -1;
  for (int c = 0; c < n_hop; c += WARP) {
    const int p = c + lane;
    const float k = (p < n_hop && dl[p] > -1.f) ? 1.f + dl[p] : 0.f;
    float incl = k;
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
      const float v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned hit = __ballot_sync(FULL, base + incl > t);
    if (hit) return c + __ffs(hit) - 1;
    const unsigned kept = __ballot_sync(FULL, k > 0.f);
    if (kept) last = c + 31 - __clz(kept);
    base += __shfl_sync(FULL, incl, WARP - 1);
  }
  return last;
}

// Apply hop p: FP64 orbital value row and Sherman-Morrison update of B, FP32
// derivative rows, g of the moved spin block, potentials and position; the
// old position goes to xo / xfo.
__device__ void apply_hop_m(const DevSys& S, const Layout& L, const LayoutM& M, double* gblk, float* sm, int p,
                            double a, const double* T, int lane) {
  double* x = (double*)(sm + M.x);
  float* xf = sm + M.xf;
  double* bt = (double*)(sm + M.bt);
  double* val = cache_val(L, gblk);
  double* der = cache_der(L, gblk);
  const double* phiv = (const double*)(sm + M.phiv);
  const float* phi5 = sm + M.phi5;
  double* f = (double*)(sm + M.u);
  double* row = (double*)(sm + M.row);
  p = CHK(p, L.n_hop);
  const int i = p / 6, d = p - 6 * i;
  double q[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  q[d >> 1] += (d & 1) ? -a : a;
  const SpinRef sr = spin_ref(L, i);
  orbital_rows_m(S, L, M, q, sr.n, sm, T, lane);
  double* B = bt + sr.bt_off;
  const int n = sr.n;
  {
    // u_j = phi(r') . B[:, j], each dot split over G lanes
    const int G = split_factor(n, n), chunk = (n + G - 1) / G, n_task = n * G;
    for (int base = 0; base < n_task; base += WARP) {
      const int task = base + lane, j = task / G, part = task - j * G;
      double acc = 0.0;
      if (task < n_task) {
        const int k1 = min(n, (part + 1) * chunk);
        for (int k = part * chunk; k < k1; ++k) acc = fma(phiv[k], B[j * n + k], acc);
      }
      for (int sh = 1; sh < G; sh <<= 1) acc += __shfl_xor_sync(FULL, acc, sh);
      if (task < n_task && part == 0) f[j] = acc;
    }
  }
  for (int k = lane; k < n; k += WARP) row[k] = B[sr.ii * n + k];
  __syncwarp();
  const double invR = rcp_nr(f[sr.ii]);   // u_ii > 0: the chosen hop is a kept one
  __syncwarp();
  for (int j = lane; j < n; j += WARP) f[j] = (f[j] - (j == sr.ii ? 1.0 : 0.0)) * invR;
  __syncwarp();
  // B and its FP32 copy (same layout) in one pass
  float* b32 = sm + M.b32 + sr.bt_off;
  for (int o = lane; o < n * n; o += WARP) {
    const int j = o / n, k = o - j * n;
    const double nb = fma(-row[k], f[j], B[o]);
    B[o] = nb;
    b32[o] = (float)nb;
  }
  for (int o = lane; o < L.n_max; o += WARP) val[i * L.n_max + o] = phiv[o];
  for (int o = lane; o < 4 * L.n_max; o += WARP) der[i * 4 * L.n_max + o] = phi5[o];
  const float qf[3] = {(float)q[0], (float)q[1], (float)q[2]};
  float nu, nucap;
  electron_potentials_f(S, qf, (float)a, lane, nu, nucap);
  if (lane == 0) {
    double* xo = (double*)(sm + M.xo);
    float* xfo = sm + M.xfo;
    xo[0] = x[3 * i]; xo[1] = x[3 * i + 1]; xo[2] = x[3 * i + 2];
    xfo[0] = xf[3 * i]; xfo[1] = xf[3 * i + 1]; xfo[2] = xf[3 * i + 2];
    x[3 * i] = q[0]; x[3 * i + 1] = q[1]; x[3 * i + 2] = q[2];
    xf[3 * i] = qf[0]; xf[3 * i + 1] = qf[1]; xf[3 * i + 2] = qf[2];
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
  double* bt = (double*)(sm + M.bt);
  for (int o = lane; o < 3 * L.n_e; o += WARP) {
    x[o] = g[L.g_x + o];
    sm[M.xf + o] = (float)g[L.g_x + o];
  }
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) bt[o] = g[L.g_bt + o];
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
  const double* bt = (const double*)(sm + M.bt);
  for (int o = lane; o < 3 * L.n_e; o += WARP) g[L.g_x + o] = x[o];
  for (int o = lane; o < L.n_up * L.n_up + L.n_dn * L.n_dn; o += WARP) g[L.g_bt + o] = bt[o];
  for (int o = lane; o < L.n_hop; o += WARP) g[L.g_rat + o] = 1.0 + (double)sm[M.dl + o];
  for (int o = lane; o < 2 * L.n_e; o += WARP) g[L.g_pot + o] = (double)sm[M.ep + o];
  for (int o = lane; o < SC_COUNT; o += WARP) g[L.g_sc + o] = sc[o];
}

// Shared-memory caches [mir, mir_end) from / to the walker's cache block.
__device__ __forceinline__ void load_mirror_m(const LayoutM& M, const double* __restrict__ c, float* sm, int lane) {
  double* d = (double*)(sm + M.mir);
  const int n = (M.mir_end - M.mir) / 2;
  for (int o = lane; o < n; o += WARP) d[o] = c[o];
  __syncwarp();
}

__device__ __forceinline__ void store_mirror_m(const LayoutM& M, double* __restrict__ c, const float* sm, int lane) {
  __syncwarp();
  const double* d = (const double*)(sm + M.mir);
  const int n = (M.mir_end - M.mir) / 2;
  for (int o = lane; o < n; o += WARP) c[o] = d[o];
}

__global__ void k_init_walkers_m(DevSys S, Layout L, LayoutM M, double* __restrict__ state, double* __restrict__ cache,
                                 const double* __restrict__ x_in, const double* __restrict__ w_in, int n, double a,
                                 int node_rule, double* scratch) {
  extern __shared__ double smem[];
  const double* T = S.exptab;   // few FP64 exponentials: the table is read through L1
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sm = (float*)smem + wib * M.stride;
  double* x = (double*)(sm + M.x);
  double* sc = (double*)(sm + M.sc);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const ScrM wscr = warp_scratch_m(L, M, scratch, slot);
  for (int w = slot; w < n; w += nwarps) {
    double* gblk = state + (size_t)w * L.g_stride;
    double* cblk = cache + (size_t)w * L.c_stride;
    const ScrM scr = walker_scratch_m(M, cblk, wscr);
    for (int o = lane; o < 3 * L.n_e; o += WARP) x[o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker_m(S, L, M, gblk, sm, scr, a, node_rule, T, lane, sing);
    if (lane == 0) {
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
    store_block_m(L, M, gblk, sm, lane);
    store_mirror_m(M, cblk, sm, lane);
  }
}

__global__ void k_eval_configs_m(DevSys S, Layout L, LayoutM M, double* __restrict__ blocks,
                                 const double* __restrict__ x_in, int n, double a, int node_rule,
                                 double* __restrict__ ratios, double* __restrict__ ev, int32_t* __restrict__ n_node,
                                 double* scratch) {
  extern __shared__ double smem[];
  const double* T = S.exptab;   // few FP64 exponentials: the table is read through L1
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sm = (float*)smem + wib * M.stride;
  double* x = (double*)(sm + M.x);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const ScrM scr = warp_scratch_m(L, M, scratch, slot);
  for (int w = slot; w < n; w += nwarps) {
    double* gblk = blocks + (size_t)w * L.g_stride;
    for (int o = lane; o < 3 * L.n_e; o += WARP) x[o] = x_in[(size_t)w * 3 * L.n_e + o];
    __syncwarp();
    bool sing = false;
    const EvalOut e = init_walker_m(S, L, M, gblk, sm, scr, a, node_rule, T, lane, sing);
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

// One branching interval for every walker (mixed precision); the caches of
// the incremental evaluation persist in the walker's cache block.
// One walker's interval (the body of k_propagate_m, also run by the batched
// kernel).
template <int BIG = -1>
__device__ void propagate_walker_m(const DevSys& S, const Layout& L, const LayoutM& M, double* __restrict__ state,
                                   double* __restrict__ cache, int w, const StepParams& P, const double* T, float* sm,
                                   const ScrM& wscr, int lane) {
  double* sc = (double*)(sm + M.sc);
  const double ia2 = 1.0 / (P.a * P.a);
  {
    const unsigned long long t_start = global_ns();
    double* gblk = state + (size_t)w * L.g_stride;
    double* cblk = cache + (size_t)w * L.c_stride;
    const ScrM scr = walker_scratch_m(M, cblk, wscr);
    load_block_m(L, M, gblk, sm, lane);
    bool cached = sc[SC_CACHE] != 0.0;
    if (cached) load_mirror_m(M, cblk, sm, lane);
    refresh_b32(L, M, sm, 0, L.n_e, lane);
    double weight = 1.0, tau_left = P.tau;
    double bbar = sc[SC_BBAR], Wd = sc[SC_WDIAG], eL = sc[SC_EL], kept = sc[SC_KEPT];
    uint32_t status = (uint32_t)sc[SC_STATUS];
    int moves = 0, since = (int)sc[SC_SINCE];
    if (cached && since > 0 && P.drift_tol > 0.0) {
      // Sherman-Morrison drift check of the FP64 inverse, once per interval
      // before the first hop (inside the hop loop it would raise this
      // kernel's register pressure): one row of A B - I per spin block,
      // rotating with the interval.  Past the tolerance the walker re-inverts
      // now and, its hop caches then being stale, evaluates in full after its
      // first hop (the first step's weight uses the stored evaluation, as it
      // would without the check)
      bool drift = false;
      for (int blk = 0; blk < 2; ++blk) {
        const int nb = blk ? L.n_dn : L.n_up;
        if (nb == 0) continue;
        const int i = (blk ? L.n_up : 0) + (int)(P.interval % (unsigned)nb);
        drift |= !(inverse_residual(L, cache_val(L, gblk), L.n_max, (const double*)(sm + M.bt), i, lane) <=
                   P.drift_tol);
      }
      if (drift) {
        if (reinvert_m(L, M, gblk, sm, scr.gj, lane)) status |= ST_SINGULAR;
        refresh_b32(L, M, sm, 0, L.n_e, lane);
        since = 0;
        cached = false;
        status |= ST_DRIFT;
        if (lane == 0 && P.drift_count) atomicAdd(P.drift_count, 1);
      }
    }
    for (int k = 0;; ++k) {
      if (P.kind == 1 && k >= P.n_proj) break;
      double u_tau, u_move;
      step_uniforms(P.seed, (uint32_t)w, (uint32_t)k, P.interval, u_tau, u_move);
      if (P.kind == 1) {
        const double den = Wd - P.E0;
        if (dpos(den)) {
          // refined reciprocal (a few ulp) instead of the FP64 division's longer sequence
          weight *= dge_nonneg(den, 0x1p-1000) ? bbar * rcp_nr(den) : bbar / den;
        } else {
          weight *= 0.0;
          status |= ST_NEG_DIAG;
        }
      } else {
        double t = -log(1.0 - u_tau) / bbar;
        const bool clipped = !(t < tau_left);
        if (clipped) t = tau_left;
        weight *= exp_tab(-t * eL, T);
        tau_left -= t;
        if (clipped) break;
      }
      const int p = choose_hop_m(sm + M.dl, L.n_hop, u_move, kept, lane);
      if (p < 0) {
        status |= ST_STUCK;
      } else {
        apply_hop_m(S, L, M, gblk, sm, p, P.a, T, lane);
        ++moves;
        bool reinv = false;
        if (++since >= P.reinv_period) {
          if (reinvert_m(L, M, gblk, sm, scr.gj, lane)) status |= ST_SINGULAR;
          refresh_b32(L, M, sm, 0, L.n_e, lane);
          since = 0;
          reinv = true;
        }
        EvalOut e;
        if (!cached) {
          e = eval_full_m<BIG>(S, L, M, gblk, sm, scr, P.a, P.node_rule, lane);
          cached = true;
        } else {
          e = eval_incr_m<BIG>(S, L, M, gblk, sm, scr, p / 6, reinv, P.a, ia2, P.node_rule, lane);
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
    const bool keep = cached && !(status & ST_SINGULAR);
    if (lane == 0) {
      sc[SC_W] = weight;
      sc[SC_STATUS] = (double)status;
      sc[SC_MOVES] = moves;
      sc[SC_SINCE] = since;
      sc[SC_CACHE] = keep ? 1.0 : 0.0;
    }
    store_block_m(L, M, gblk, sm, lane);
    if (keep) store_mirror_m(M, cblk, sm, lane);
    if (P.stamps && lane == 0) {
      P.stamps[3 * (size_t)w] = t_start;
      P.stamps[3 * (size_t)w + 1] = global_ns();
      P.stamps[3 * (size_t)w + 2] = sm_id();
    }
  }
}

// At most 72 registers per thread (8 bytes spilled): the kernel is latency
// bound, and 28 resident warps per SM (4096 walkers in one wave on 148 SMs)
// run it faster than the 20 that its unconstrained 94 registers allow.
// GSM: working sets in global memory (gsm + slot * M.stride floats), as in
// the FP64 kernel.  BIG: placement of the O(N^2) arrays (LayoutM::glob; -1:
// decided at run time).
template <bool GSM, int BIG>
__global__ void __maxnreg__(72) k_propagate_m(DevSys S, Layout L, LayoutM M, double* __restrict__ state,
                                              double* __restrict__ cache, int n_w, StepParams P, double* scratch,
                                              float* gsm) {
  extern __shared__ double smem[];
  const double* T = S.exptab;   // few FP64 exponentials: the table is read through L1
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  float* sm = GSM ? gsm + (size_t)slot * M.stride : (float*)smem + wib * M.stride;
  const ScrM wscr = warp_scratch_m(L, M, scratch, slot);
  for (int w = slot; w < n_w; w = next_walker(P, w, nwarps, lane))
    propagate_walker_m<BIG>(S, L, M, state, cache, w, P, T, sm, wscr, lane);
}

}  // namespace lrdmc
