// Shared definitions of the LRDMC CUDA library: device-side system tables,
// per-walker memory layout, status bits and the Philox4x32-10 generator.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace lrdmc {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP = 32;

// Checked build (compiled with -DLRDMC_CHECKED into a library of its own):
// CHK(i, n) tests a data-derived index against its extent [0, n).  A failure
// records the first violation in the device word g_lrdmc_check (source line in
// the high 32 bits, the offending index in the low 32; later failures keep the
// first) and returns 0, so the access stays inside the array and nothing
// traps; the host reads and clears the word with lrdmc_check_word.  In the
// normal build CHK(i, n) is i.
#ifdef LRDMC_CHECKED
__device__ unsigned long long g_lrdmc_check;
__device__ __forceinline__ long long chk_index(long long i, long long n, int line) {
  if (i < 0 || i >= n) {
    atomicCAS(&g_lrdmc_check, 0ull, ((unsigned long long)(unsigned)line << 32) | (unsigned long long)(unsigned)i);
    return 0;
  }
  return i;
}
#define CHK(i, n) ((std::decay_t<decltype(i)>)::lrdmc::chk_index((long long)(i), (long long)(n), __LINE__))
#else
#define CHK(i, n) (i)
#endif

// per-walker status bits (mirror LRDMC_WALKER_* in lrdmc.h)
constexpr uint32_t ST_NEG_DIAG = 1u;
constexpr uint32_t ST_NONFINITE = 2u;
constexpr uint32_t ST_STEP_CAP = 4u;
constexpr uint32_t ST_STUCK = 8u;
constexpr uint32_t ST_SINGULAR = 16u;
constexpr uint32_t ST_DRIFT = 32u;      // a Sherman-Morrison drift check triggered a re-inversion

// Scalars kept at the end of every walker block (doubles; integer-valued
// fields are exact in double up to 2^53).
enum Scalar : int {
  SC_W = 0,       // weight accumulated in the current interval
  SC_BBAR = 1,    // b_bar(x): sum of kept hop ratios / (2 a^2)
  SC_VSF = 2,     // spin-flip term V_sf(x)
  SC_WDIAG = 3,   // W(x): diagonal of the FN lattice Hamiltonian
  SC_EL = 4,      // e_L(x) = W(x) - b_bar(x)
  SC_NNODE = 5,   // electrons with at least one node-crossing hop
  SC_STATUS = 6,  // sticky status bits
  SC_MOVES = 7,   // hops made in the last interval
  SC_SINCE = 8,   // hops since the last from-scratch inversion
  SC_CACHE = 9,   // 1: the walker's cache block matches x and B on the fixed lattice
  SC_ROTATED = 10,  // 1: the stored evaluation was taken on a randomised lattice
  SC_KEPT = 11,   // sum of the kept hop ratios (2 a^2 b_bar before rounding)
  SC_COUNT = 16
};

// System and trial-wavefunction tables in device memory (read-only).
struct DevSys {
  int n_nuc, n_shell, n_prim, n_bf, n_orb, n_up, n_dn, n_e, n_max;
  int n_shell_np;         // shells that are not p shells (sh_ord lists them first)
  const double* R;       // n_nuc x 3
  const double* Z;       // n_nuc
  const double* rc;      // n_nuc
  const double* irc;     // n_nuc: 1 / rc (erf-screened nuclei)
  const double* irc2;    // n_nuc: 1 / rc^2
  const int* kind;       // n_nuc: 0 bare Coulomb, 1 erf-screened
  const double* j1A;     // n_nuc
  const double* j1B;     // n_nuc
  const int* sh_atom;    // n_shell
  const int* sh_l;       // n_shell: 0 s, 1 p, -1 Slater 1s
  const int* sh_nprim;   // n_shell
  const int* sh_off;     // n_shell: first primitive
  const int* sh_bf;      // n_shell: first basis function
  const int* atom_sh;    // n_nuc + 1: shells are grouped by nucleus, atom I owns [atom_sh[I], atom_sh[I+1])
  const int* sh_ord;     // n_shell: shell indices, every non-p shell before every p shell
  const double* exptab;  // EXP_TAB = 256 entries 2^(j/256) for the table-driven exponential
  const double* erftab;  // ERF_INT x ERF_NC: polynomials of erf(sqrt t)/sqrt t (fp64math.cuh)
  const double* exps;    // n_prim
  const double* coefs;   // n_prim
  const double* C;       // n_orb x n_bf
  // FP32 copies for the mixed-precision kernels (no per-use conversion)
  const float* Rf;
  const float* Zf;
  const float* rcf;
  const float* j1Af;
  const float* j1Bf;
  const float* expsf;
  const float* coefsf;
  const float* Cf;
  double j2_anti, j2_par, j2_b;
  float j2_antif, j2_parf, j2_bf;   // FP32 copies (mixed kernels)
  double v_ii;           // nucleus-nucleus repulsion
};

// Offsets (in doubles) of the walker block in global memory and of the
// per-warp working set in shared memory.
struct Layout {
  int n_e, n_up, n_dn, n_max, n_bf, n_hop;
  // global walker block: positions, B^T, orbital cache [n_e][5][n_max], hop
  // ratios, per-electron potentials (nu_ei, nu^a_ei), scalars
  int g_x, g_bt, g_cache, g_rat, g_pot, g_sc, g_stride;
  // shared memory per warp (FP64 kernels): positions, B^T, hop ratios,
  // potentials [2 per electron], per-electron Jastrow terms [6],
  // determinant derivatives [4], electron-nucleus geometry [4 per (electron,
  // nucleus): |d|^2 + a^2 and the components of d along the three hop
  // versors], pair distances, per-hop determinant ratio and one-body / pair
  // Jastrow sums, per-hop scratch (also the moved electron's basis scratch),
  // orbital rows, rank-1 factors, old position of the moved electron, hop
  // versors [3][3], scalars
  int s_x, s_bt, s_rat, s_ej, s_ep, s_dd, s_geo, s_pr2, s_hd, s_hj1, s_hj2, s_tmp, s_phi5, s_u, s_row, s_xo,
      s_v, s_sc, s_stride;
  // per-walker cache block in global memory (FP64 kernels), kept across
  // branching intervals: a copy of the shared-memory caches [s_ej, s_tmp),
  // g_i = C^T B[:, i] [n_e][n_bf], the basis values at every hop [n_bf][6 n_e],
  // the pair Jastrow term of every hop with every partner [n_e][6 n_e] and the
  // pair terms at the current positions [n_e][n_e][4]
  int c_mir, c_g, c_chi, c_u2, c_pt, c_stride;
  // large systems: the electron-nucleus geometry [n_e][n_nuc][4] and the pair
  // distances [n_e][n_e] live in the cache block (c_geo, c_pr2) instead of
  // shared memory (s_geo, s_pr2 then have no extent)
  int geo_glob, c_geo, c_pr2;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Slater block of electron i: offset of its B^T block, index inside the spin
// block and the block order.
struct SpinRef {
  int bt_off, ii, n;
};
__host__ __device__ inline SpinRef spin_ref(const Layout& L, int i) {
  SpinRef s;
  if (i < L.n_up) {
    s.bt_off = 0; s.ii = i; s.n = L.n_up;
  } else {
    s.bt_off = L.n_up * L.n_up; s.ii = i - L.n_up; s.n = L.n_dn;
  }
  return s;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (X0,X1,X2,X3) -> (hi(M1 X2) ^ X1 ^ K0, lo(M1 X2), hi(M0 X0) ^ X3 ^ K1, lo(M0 X0))
// with the key bumped by the Weyl increments between rounds.
constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

__host__ __device__ inline void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  hi = __umulhi(a, b);
  lo = a * b;
#else
  uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
#endif
}

__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(PHILOX_M0, c[0], hi0, lo0);
    mulhilo32(PHILOX_M1, c[2], hi1, lo1);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Uniform in [0,1): top 32 bits from hi, next 21 from the top of lo, times 2^-53.
// On the device the exact value is assembled from bits: 0.5 + x 2^-53 has the
// bit pattern 0x3FE0000000000000 + x for x < 2^52, so v 2^-53 is that pattern
// with x = v - 2^52 when v >= 2^52, else that pattern with x = v, minus 0.5
// (exact by Sterbenz's lemma); one FP64 addition at most instead of an
// integer-to-double conversion and a multiplication.
__host__ __device__ inline double uniform53(uint32_t hi, uint32_t lo) {
  uint64_t v = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
#ifdef __CUDA_ARCH__
  const double h = __longlong_as_double((long long)(0x3FE0000000000000ull + (v & 0xFFFFFFFFFFFFFull)));
  return (v >> 52) ? h : h - 0.5;
#else
  return (double)v * 0x1p-53;
#endif
}

// Stream layout: counter (walker slot, step, interval, 0) gives the persistence
// time uniform from words 0-1 and the heat-bath uniform from words 2-3;
// counter (0, 0, interval, 1) word 0 is the reconfiguration comb offset.
__host__ __device__ inline void step_uniforms(uint64_t seed, uint32_t walker, uint32_t step,
                                              uint32_t interval, double& u_tau, double& u_move) {
  uint32_t c[4] = {walker, step, interval, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  u_tau = uniform53(c[0], c[1]);
  u_move = uniform53(c[2], c[3]);
}

__host__ __device__ inline uint32_t branch_offset32(uint64_t seed, uint32_t interval) {
  uint32_t c[4] = {0u, 0u, interval, 1u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return c[0];
}

}  // namespace lrdmc
