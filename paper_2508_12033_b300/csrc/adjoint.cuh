// Hand-written adjoint (reverse mode) of the lattice-regularised local energy
// e_L = W - b_bar (Appendix D) and of log|Psi_G| with respect to the nuclear
// coordinates R_I and the Jastrow parameters (c_anti, c_par, b, A_I, B_I), one
// configuration per warp, FP64.
//
// With S_i = sum_d r_{i,d} the six hop ratios of electron i, the regularised
// potential nu_zv,i = nu_i + ((S_i - 6)/a^2 - L_i)/2 enters W next to
// -b_bar + V_sf = -sum_p r_p/(2a^2), so electron i contributes
//   nu_i - L_i / 2                           where nu_opt,i = nu_zv,i,
//   nu^a_i + 3/a^2 - S_i/(2a^2)              where the cap nu^a_i is taken,
// plus V_ee + V_ii.  L_i = lap_i Psi/Psi = lD_i + 2 gD_i.gJ_i + lJ_i + |gJ_i|^2
// with gD_i = sum_k grad phi_k(r_i) B_ki, lD_i = sum_k lap phi_k(r_i) B_ki.
// The reverse pass carries adjoints back through
//   * the Jastrow gradient / Laplacian sums (pair and one-body radial terms);
//   * the determinant derivatives: B_bar_ki = gD_bar_i . grad phi_k(r_i) +
//     lD_bar_i lap phi_k(r_i), and for capped electrons the hop determinants
//     (R_bar phi_k(r')); then A_bar = -B^T B_bar B^T (dB = -B dA B);
//   * the orbitals to the basis functions, whose centre derivatives are minus
//     their position derivatives: grad chi, its Hessian and grad lap chi;
//   * the capped electrons' hop Jastrow differences;
//   * the potentials nu_i, nu^a_i and V_ii.
// log|Psi_G| = log|det A_up| + log|det A_dn| + J: d log|det|/d A = B^T, so
// d log|det| / d R_I = -sum_j sum_{mu on I} g_j[mu] grad chi_mu(r_j - R_I)
// with g_j = C^T B[:, j].
//
// Parameter order of every gradient row: R (n_nuc x 3), c_anti, c_par, b,
// A (n_nuc), B (n_nuc).
#pragma once

#include "walker.cuh"

namespace lrdmc {

__host__ __device__ inline int param_count(int n_nuc) { return 5 * n_nuc + 3; }

// Per-warp global scratch of the adjoint kernel (doubles).
__host__ __device__ inline size_t adj_scratch_doubles(const Layout& L, int n_shell) {
  const size_t nbt = (size_t)L.n_up * L.n_up + (size_t)L.n_dn * L.n_dn;
  return 3 * nbt + 10 * (size_t)L.n_e + 6 * (size_t)n_shell + L.n_bf + 2 * (size_t)L.n_max + 8;
}

// Centre-derivative contribution of the functions of shell s at offset d from
// its nucleus: sum_f [wv_f grad chi_f + Hess chi_f . wg + wl_f grad lap chi_f],
// where wg = gw * wgs_f (gw a 3-vector shared by the shell, wgs_f per function).
// The caller subtracts it from R_bar (d chi(r - R)/dR = -grad chi).
__device__ void shell_center_terms(const DevSys& S, int s, const double d[3], const double* wv, const double* wgs,
                                   const double gw[3], const double* wl, double out[3]) {
  const int l = __ldg(S.sh_l + s), np = __ldg(S.sh_nprim + s), off = __ldg(S.sh_off + s);
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  out[0] = out[1] = out[2] = 0.0;
  if (l == -1) {
    const double r = sqrt(r2), ir = 1.0 / r;
    const double u[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    double f1 = 0.0, f2 = 0.0, f3 = 0.0;   // radial derivatives of the contraction
    for (int q = 0; q < np; ++q) {
      const double z = __ldg(S.exps + off + q);
      const double f = __ldg(S.coefs + off + q) * exp(-z * r);
      f1 += -z * f;
      f2 += z * z * f;
      f3 += -z * z * z * f;
    }
    const double ug = u[0] * gw[0] + u[1] * gw[1] + u[2] * gw[2];
    const double lp = f3 + 2.0 * f2 * ir - 2.0 * f1 * ir * ir;   // d/dr of lap chi
    for (int k = 0; k < 3; ++k)
      out[k] = wv[0] * f1 * u[k] + wgs[0] * (f2 * ug * u[k] + f1 * ir * (gw[k] - ug * u[k])) + wl[0] * lp * u[k];
    return;
  }
  const double dg = d[0] * gw[0] + d[1] * gw[1] + d[2] * gw[2];
  for (int q = 0; q < np; ++q) {
    const double al = __ldg(S.exps + off + q);
    const double h = __ldg(S.coefs + off + q) * exp(-al * r2);
    if (l == 0) {
      const double g1 = -2.0 * al * h;                                  // grad chi = g1 d
      const double t3 = (20.0 * al * al - 8.0 * al * al * al * r2) * h;   // grad lap chi = t3 d
      for (int k = 0; k < 3; ++k)
        out[k] += wv[0] * g1 * d[k] + wgs[0] * (4.0 * al * al * d[k] * dg - 2.0 * al * gw[k]) * h +
                  wl[0] * t3 * d[k];
    } else {
      const double c2 = 4.0 * al * al * r2 - 10.0 * al, c3 = 28.0 * al * al - 8.0 * al * al * al * r2;
      for (int m = 0; m < 3; ++m) {
        for (int k = 0; k < 3; ++k) {
          const double dmk = (m == k) ? 1.0 : 0.0;
          const double grad = (dmk - 2.0 * al * d[m] * d[k]) * h;
          const double hess = (-2.0 * al * (d[k] * gw[m] + d[m] * gw[k] + dmk * dg) +
                               4.0 * al * al * d[m] * d[k] * dg) * h;
          const double gl = (dmk * c2 + d[m] * d[k] * c3) * h;
          out[k] += wv[m] * grad + wgs[m] * hess + wl[m] * gl;
        }
      }
    }
  }
}

// Basis values of every function at point q (chi[mu]).
__device__ void basis_values_at(const DevSys& S, const Layout& L, const double q[3], double* chi, int lane) {
  for (int s = lane; s < S.n_shell; s += WARP) {
    const int I = __ldg(S.sh_atom + s), l = __ldg(S.sh_l + s), np = __ldg(S.sh_nprim + s), off = __ldg(S.sh_off + s),
              bf = __ldg(S.sh_bf + s);
    const double d[3] = {q[0] - __ldg(S.R + 3 * I), q[1] - __ldg(S.R + 3 * I + 1), q[2] - __ldg(S.R + 3 * I + 2)};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double arg = l == -1 ? sqrt(r2) : r2;
    double rad = 0.0;
    for (int k = 0; k < np; ++k) rad += __ldg(S.coefs + off + k) * exp(-__ldg(S.exps + off + k) * arg);
    if (l == 1) {
      for (int m = 0; m < 3; ++m) chi[bf + m] = d[m] * rad;
    } else {
      chi[bf] = rad;
    }
  }
  __syncwarp();
}


// Partner-pair radial Jastrow terms: t = 1/(1 + b r).
//   u' = c t^2, u'' = -2 b c t^3;  du/dc = r t, du/db = -c r^2 t^2
//   du'/dc = t^2, du''/dc = -2 b t^3, du'/db = -2 c r t^3, du''/db = -2 c t^3 + 6 b c r t^4

// One configuration per warp: e_L, log|Psi_G| and their gradient rows.
// GSM: the warp's working set (the shared-memory layout of the propagate
// kernels) lives in global memory at gsm + slot * s_stride instead of shared
// memory.  Large systems use it: a 128-electron working set fills an SM's
// shared memory for a single warp, while from global memory (L1 / L2 resident)
// as many warps share an SM as their registers allow: at most 128 registers
// per thread (16 bytes spilled) let 16 warps share an SM, against 9 with the
// 216 the kernel takes unconstrained.
template <bool GSM>
__global__ void __maxnreg__(128) k_eloc_grad(DevSys S, Layout L, double* __restrict__ blocks, const double* __restrict__ x_in, int n,
                            double a, int node_rule, double* scratch, double* gscr, size_t gscr_per_warp,
                            double* __restrict__ eL_out, double* __restrict__ lp_out, double* __restrict__ ge_out,
                            double* __restrict__ gl_out, double* gsm) {
  extern __shared__ double smem[];
  const double* T = stage_table(S, smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* sm = GSM ? gsm + (size_t)(blockIdx.x * (blockDim.x >> 5) + wib) * L.s_stride
                   : smem + EXP_TAB + wib * L.s_stride;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const Scr scr = warp_scratch(L, S.n_nuc, scratch, slot);
  const int ne = L.n_e, nn = S.n_nuc, nbf = L.n_bf, np = param_count(nn), nsh = S.n_shell;
  const int nbt = L.n_up * L.n_up + L.n_dn * L.n_dn;
  // per-warp scratch
  double* gw = gscr + (size_t)slot * gscr_per_warp;
  double* Bb = gw;                  // B_bar per spin block, stored like B^T: Bb[i][k] = adjoint of B_ki
  double* Tm = Bb + nbt;
  double* Ab = Tm + nbt;            // A_bar [i][k] per spin block
  double* eadj = Ab + nbt;          // per electron: gD_bar (3), lD_bar, gJ_bar (3), lJ_bar, S_bar, capped
  double* shacc = eadj + 10 * ne;   // per shell: R_bar contributions (3 for e_L, 3 for log|Psi|)
  double* chih = shacc + 6 * nsh;   // basis values at one hop
  double* phih = chih + nbf;        // orbital values at one hop
  const double ia2 = 1.0 / (a * a), s_bar = -0.5 * ia2;
  for (int w = slot; w < n; w += nwarps) {
    double* gblk = blocks + (size_t)slot * L.g_stride;   // the warp's own walker block
    double* ge = ge_out ? ge_out + (size_t)w * np : nullptr;
    double* gl = gl_out ? gl_out + (size_t)w * np : nullptr;
    for (int o = lane; o < 3 * ne; o += WARP) sm[L.s_x + o] = x_in[(size_t)w * 3 * ne + o];
    __syncwarp();
    bool sing = false;
    double logdet = 0.0;
    const EvalOut ev = init_walker(S, L, gblk, sm, scr, a, node_rule, T, lane, sing, &logdet);
    const double* x = sm + L.s_x;
    const double* bt = sm + L.s_bt;
    const double* rat = sm + L.s_rat;
    const double* ej = sm + L.s_ej;
    const double* ep = sm + L.s_ep;
    const double* dd = sm + L.s_dd;
    const double* cache = gblk + L.g_cache;
    for (int o = lane; o < np; o += WARP) {
      if (ge) ge[o] = 0.0;
      if (gl) gl[o] = 0.0;
    }
    for (int o = lane; o < 6 * nsh; o += WARP) shacc[o] = 0.0;
    for (int o = lane; o < nbt; o += WARP) Bb[o] = 0.0;
    // (1) per electron: cap decision and adjoints of L_i, S_i, nu_i, nu^a_i
    bool any_node = false;
    for (int i = lane; i < ne; i += WARP)
      for (int d = 0; d < 6; ++d) any_node |= rat[6 * i + d] < 0.0;
    any_node = __any_sync(FULL, any_node);
    for (int i = lane; i < ne; i += WARP) {
      double si = 0.0;
      bool node = false;
      for (int d = 0; d < 6; ++d) {
        si += rat[6 * i + d];
        node |= rat[6 * i + d] < 0.0;
      }
      const double* q = ej + 6 * i;
      const double* dv = dd + 4 * i;
      const double lap = dv[3] + 2.0 * (dv[0] * q[1] + dv[1] * q[2] + dv[2] * q[3]) + q[4] +
                         (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      const double nu_zv = ep[2 * i] + 0.5 * ((si - 6.0) * ia2 - lap);
      bool apply;
      if (node_rule == 0) apply = node;
      else if (node_rule == 1) apply = any_node;
      else if (node_rule == 2) apply = true;
      else apply = false;
      const bool capped = apply && ep[2 * i + 1] > nu_zv;
      const double Lb = capped ? 0.0 : -0.5;
      double* e = eadj + 10 * i;
      for (int k = 0; k < 3; ++k) {
        e[k] = 2.0 * Lb * q[1 + k];                    // gD_bar
        e[4 + k] = 2.0 * Lb * (dv[k] + q[1 + k]);      // gJ_bar
      }
      e[3] = Lb;                                       // lD_bar
      e[7] = Lb;                                       // lJ_bar
      e[8] = capped ? s_bar : 0.0;                     // S_bar
      e[9] = capped ? 1.0 : 0.0;
    }
    __syncwarp();
    // (2) pair Jastrow: e_L through gJ_i, lJ_i (ordered pairs); log|Psi| through J
    {
      double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // e_L: c_anti, c_par, b; log|Psi|: same
      double Jp = 0.0;
      const double b = S.j2_b;
      for (int o = lane; o < ne * ne; o += WARP) {
        const int i = o / ne, j = o - i * ne;
        if (i == j) continue;
        const bool par = (i < L.n_up) == (j < L.n_up);
        const double c = par ? S.j2_par : S.j2_anti;
        const double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), ir = 1.0 / r;
        const double t = 1.0 / (1.0 + b * r), t2 = t * t, t3 = t2 * t, t4 = t3 * t;
        const double* e = eadj + 10 * i;
        const double gd = (e[4] * d[0] + e[5] * d[1] + e[6] * d[2]) * ir;   // gJ_bar . d / r
        // d/dc and d/db of u' / r d and of u'' + 2 u'/r
        const double dc = gd * t2 + e[7] * (-2.0 * b * t3 + 2.0 * t2 * ir);
        const double db = gd * (-2.0 * c * r * t3) + e[7] * (-2.0 * c * t3 + 6.0 * b * c * r * t4 - 4.0 * c * t3);
        acc[par ? 1 : 0] += dc;
        acc[2] += db;
        if (i < j) {
          Jp += c * r * t;
          acc[3 + (par ? 1 : 0)] += r * t;
          acc[5] += -c * r * r * t2;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        for (int k = 0; k < 6; ++k) acc[k] += __shfl_xor_sync(FULL, acc[k], o);
        Jp += __shfl_xor_sync(FULL, Jp, o);
      }
      if (lane == 0) {
        if (ge) { ge[3 * nn] += acc[0]; ge[3 * nn + 1] += acc[1]; ge[3 * nn + 2] += acc[2]; }
        if (gl) { gl[3 * nn] += acc[3]; gl[3 * nn + 1] += acc[4]; gl[3 * nn + 2] += acc[5]; }
      }
      logdet += Jp;
    }
    __syncwarp();
    // (3) one-body Jastrow, potentials and V_ii: one nucleus per lane, electrons in order
    {
      double J1 = 0.0;
      for (int I = lane; I < nn; I += WARP) {
        const double RI[3] = {__ldg(S.R + 3 * I), __ldg(S.R + 3 * I + 1), __ldg(S.R + 3 * I + 2)};
        const double A = __ldg(S.j1A + I), B = __ldg(S.j1B + I), Z = __ldg(S.Z + I);
        const int kind = __ldg(S.kind + I);
        double gR[3] = {0.0, 0.0, 0.0}, lR[3] = {0.0, 0.0, 0.0};
        double gA = 0.0, gB = 0.0, lA = 0.0, lB = 0.0;
        for (int i = 0; i < ne; ++i) {
          const double d[3] = {x[3 * i] - RI[0], x[3 * i + 1] - RI[1], x[3 * i + 2] - RI[2]};
          const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), ir = 1.0 / r;
          const double u[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
          const double* e = eadj + 10 * i;
          // one-body term v = -A r t, t = 1/(1 + B r)
          const double t = 1.0 / (1.0 + B * r), t2 = t * t, t3 = t2 * t, t4 = t3 * t;
          const double v1 = -A * t2, v2 = 2.0 * A * B * t3, v3 = -6.0 * A * B * B * t4;
          const double ug = u[0] * e[4] + u[1] * e[5] + u[2] * e[6];
          // d gJ_i / d R_I = -Hess v; d lJ_i / d R_I = -(v''' + 2 v''/r - 2 v'/r^2) u
          const double lpr = v3 + 2.0 * v2 * ir - 2.0 * v1 * ir * ir;
          for (int k = 0; k < 3; ++k)
            gR[k] -= v2 * ug * u[k] + v1 * ir * (e[4 + k] - ug * u[k]) + e[7] * lpr * u[k];
          // d/dA, d/dB of v'/r d and of v'' + 2 v'/r
          const double gd = ug;   // gJ_bar . u
          gA += gd * (-t2) + e[7] * (2.0 * B * t3 - 2.0 * t2 * ir);
          gB += gd * (2.0 * A * r * t3) + e[7] * (2.0 * A * t3 - 6.0 * A * B * r * t4 + 4.0 * A * t3);
          // potentials: d nu(|x - R|)/dR = -nu'(r) u
          double vp, vpc;
          if (kind == 0) {
            vp = Z * ir * ir;
            vpc = r > a ? Z * ir * ir : 0.0;
          } else {
            const double irc = __ldg(S.irc + I);
            const double y = r * irc;
            vp = -Z * (1.1283791670955126 * exp(-y * y) * irc * ir - erf(y) * ir * ir);
            vpc = vp;
          }
          const double wpot = (e[9] != 0.0) ? vpc : vp;   // nu_bar = 1 uncapped, nu^a_bar = 1 capped
          for (int k = 0; k < 3; ++k) gR[k] -= wpot * u[k];
          // log|Psi|: J_1 = sum_i v(|x_i - R_I|)
          J1 += -A * r * t;
          lA += -r * t;
          lB += A * r * r * t2;
          for (int k = 0; k < 3; ++k) lR[k] -= v1 * u[k];
        }
        // V_ii
        for (int J = 0; J < nn; ++J) {
          if (J == I) continue;
          const double D[3] = {RI[0] - __ldg(S.R + 3 * J), RI[1] - __ldg(S.R + 3 * J + 1), RI[2] - __ldg(S.R + 3 * J + 2)};
          const double R2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
          const double f = -Z * __ldg(S.Z + J) / (R2 * sqrt(R2));
          for (int k = 0; k < 3; ++k) gR[k] += f * D[k];
        }
        if (ge) {
          for (int k = 0; k < 3; ++k) ge[3 * I + k] += gR[k];
          ge[3 * nn + 3 + I] += gA;
          ge[4 * nn + 3 + I] += gB;
        }
        if (gl) {
          for (int k = 0; k < 3; ++k) gl[3 * I + k] += lR[k];
          gl[3 * nn + 3 + I] += lA;
          gl[4 * nn + 3 + I] += lB;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) J1 += __shfl_xor_sync(FULL, J1, o);
      logdet += J1;
    }
    __syncwarp();
    // (4) capped electrons: their hop ratios r = R_det exp(dJ) enter e_L through S_i
    for (int i = 0; i < ne; ++i) {
      if (eadj[10 * i + 9] == 0.0) continue;   // warp-uniform
      const SpinRef sr = spin_ref(L, i);
      const double* gi = scr.g + (size_t)i * nbf;
      for (int d = 0; d < 6; ++d) {
        const int p = 6 * i + d, ax = d >> 1;
        const double q[3] = {x[3 * i] + (ax == 0 ? ((d & 1) ? -a : a) : 0.0),
                             x[3 * i + 1] + (ax == 1 ? ((d & 1) ? -a : a) : 0.0),
                             x[3 * i + 2] + (ax == 2 ? ((d & 1) ? -a : a) : 0.0)};
        const double eJ = exp(sm[L.s_hj1 + p] + sm[L.s_hj2 + p] - ej[6 * i]);
        const double Rb = s_bar * eJ;           // adjoint of the determinant ratio
        const double Jb = s_bar * rat[p];       // adjoint of the Jastrow difference
        basis_values_at(S, L, q, chih, lane);
        for (int k = lane; k < sr.n; k += WARP) {
          double acc = 0.0;
          for (int mu = 0; mu < nbf; ++mu) acc = fma(__ldg(S.C + (size_t)k * nbf + mu), chih[mu], acc);
          phih[k] = acc;
        }
        __syncwarp();
        for (int k = lane; k < sr.n; k += WARP) Bb[sr.bt_off + sr.ii * sr.n + k] += Rb * phih[k];
        // basis centres at the hop: R_bar -= Rb g_i[mu] grad chi_mu(q - R)
        for (int s = lane; s < nsh; s += WARP) {
          const int I = __ldg(S.sh_atom + s), bf = __ldg(S.sh_bf + s), nf = __ldg(S.sh_l + s) == 1 ? 3 : 1;
          const double dq[3] = {q[0] - __ldg(S.R + 3 * I), q[1] - __ldg(S.R + 3 * I + 1), q[2] - __ldg(S.R + 3 * I + 2)};
          double wv[3] = {0.0, 0.0, 0.0}, z3[3] = {0.0, 0.0, 0.0}, out[3];
          for (int m = 0; m < nf; ++m) wv[m] = Rb * gi[bf + m];
          shell_center_terms(S, s, dq, wv, z3, z3, z3, out);
          for (int k = 0; k < 3; ++k) shacc[6 * s + k] -= out[k];
        }
        // Jastrow difference: pair terms (parameters) and one-body terms (parameters, centres)
        double pc[3] = {0.0, 0.0, 0.0};
        for (int j = lane; j < ne; j += WARP) {
          if (j == i) continue;
          const bool par = (i < L.n_up) == (j < L.n_up);
          const double c = par ? S.j2_par : S.j2_anti, b = S.j2_b;
          const double r1 = sqrt((q[0] - x[3 * j]) * (q[0] - x[3 * j]) + (q[1] - x[3 * j + 1]) * (q[1] - x[3 * j + 1]) +
                                 (q[2] - x[3 * j + 2]) * (q[2] - x[3 * j + 2]));
          const double r0 = sqrt((x[3 * i] - x[3 * j]) * (x[3 * i] - x[3 * j]) +
                                 (x[3 * i + 1] - x[3 * j + 1]) * (x[3 * i + 1] - x[3 * j + 1]) +
                                 (x[3 * i + 2] - x[3 * j + 2]) * (x[3 * i + 2] - x[3 * j + 2]));
          const double t1 = 1.0 / (1.0 + b * r1), t0 = 1.0 / (1.0 + b * r0);
          pc[par ? 1 : 0] += Jb * (r1 * t1 - r0 * t0);
          pc[2] += Jb * (-c * r1 * r1 * t1 * t1 + c * r0 * r0 * t0 * t0);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
          for (int k = 0; k < 3; ++k) pc[k] += __shfl_xor_sync(FULL, pc[k], o);
        if (lane == 0 && ge) { ge[3 * nn] += pc[0]; ge[3 * nn + 1] += pc[1]; ge[3 * nn + 2] += pc[2]; }
        for (int I = lane; I < nn; I += WARP) {
          const double A = __ldg(S.j1A + I), B = __ldg(S.j1B + I);
          const double RI[3] = {__ldg(S.R + 3 * I), __ldg(S.R + 3 * I + 1), __ldg(S.R + 3 * I + 2)};
          double gA = 0.0, gB = 0.0, gR[3] = {0.0, 0.0, 0.0};
          for (int side = 0; side < 2; ++side) {          // +v at q, -v at r_i
            const double sg = side == 0 ? 1.0 : -1.0;
            const double dd3[3] = {(side == 0 ? q[0] : x[3 * i]) - RI[0], (side == 0 ? q[1] : x[3 * i + 1]) - RI[1],
                                   (side == 0 ? q[2] : x[3 * i + 2]) - RI[2]};
            const double r = sqrt(dd3[0] * dd3[0] + dd3[1] * dd3[1] + dd3[2] * dd3[2]);
            const double t = 1.0 / (1.0 + B * r);
            gA += sg * (-r * t);
            gB += sg * (A * r * r * t * t);
            const double v1 = -A * t * t;
            for (int k = 0; k < 3; ++k) gR[k] += sg * (-v1 * dd3[k] / r);
          }
          if (ge) {
            ge[3 * nn + 3 + I] += Jb * gA;
            ge[4 * nn + 3 + I] += Jb * gB;
            for (int k = 0; k < 3; ++k) ge[3 * I + k] += Jb * gR[k];
          }
        }
        __syncwarp();
      }
    }
    // (5) B_bar from the determinant derivatives at the electrons
    for (int o = lane; o < ne * L.n_max; o += WARP) {
      const int i = o / L.n_max, k = o - i * L.n_max;
      const SpinRef sr = spin_ref(L, i);
      if (k >= sr.n) continue;
      const double* e = eadj + 10 * i;
      const double* ce = cache + (size_t)i * 5 * L.n_max;
      Bb[sr.bt_off + sr.ii * sr.n + k] += e[0] * ce[L.n_max + k] + e[1] * ce[2 * L.n_max + k] +
                                          e[2] * ce[3 * L.n_max + k] + e[3] * ce[4 * L.n_max + k];
    }
    __syncwarp();
    // (6) A_bar = -B^T B_bar B^T per spin block: Tm[k'][k] = sum_i Bb[i][k'] bt[i][k], Ab[j][k] = -sum_k' bt[j][k'] Tm[k'][k]
    for (int blk = 0; blk < 2; ++blk) {
      const int nb = blk ? L.n_dn : L.n_up, off = blk ? L.n_up * L.n_up : 0;
      for (int o = lane; o < nb * nb; o += WARP) {
        const int kp = o / nb, k = o - kp * nb;
        double acc = 0.0;
        for (int i2 = 0; i2 < nb; ++i2) acc = fma(Bb[off + i2 * nb + kp], bt[off + i2 * nb + k], acc);
        Tm[off + o] = acc;
      }
      __syncwarp();
      for (int o = lane; o < nb * nb; o += WARP) {
        const int j = o / nb, k = o - j * nb;
        double acc = 0.0;
        for (int kp = 0; kp < nb; ++kp) acc = fma(bt[off + j * nb + kp], Tm[off + kp * nb + k], acc);
        Ab[off + o] = -acc;
      }
      __syncwarp();
    }
    // (7) basis centres at the electrons: one shell per lane, electrons in order
    for (int s = lane; s < nsh; s += WARP) {
      const int I = __ldg(S.sh_atom + s), bf = __ldg(S.sh_bf + s), nf = __ldg(S.sh_l + s) == 1 ? 3 : 1;
      const double RI[3] = {__ldg(S.R + 3 * I), __ldg(S.R + 3 * I + 1), __ldg(S.R + 3 * I + 2)};
      double ae[3] = {0.0, 0.0, 0.0}, al[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < ne; ++i) {
        const SpinRef sr = spin_ref(L, i);
        const double* gi = scr.g + (size_t)i * nbf;
        const double* e = eadj + 10 * i;
        const double* abr = Ab + sr.bt_off + sr.ii * sr.n;
        const double d[3] = {x[3 * i] - RI[0], x[3 * i + 1] - RI[1], x[3 * i + 2] - RI[2]};
        double wv[3] = {0.0, 0.0, 0.0}, wg[3] = {0.0, 0.0, 0.0}, wl[3] = {0.0, 0.0, 0.0}, out[3];
        for (int m = 0; m < nf; ++m) {
          double acc = 0.0;   // chi_bar = sum_k C[k][mu] A_bar[i][k]
          for (int k = 0; k < sr.n; ++k) acc = fma(__ldg(S.C + (size_t)k * nbf + bf + m), abr[k], acc);
          wv[m] = acc;
          wg[m] = gi[bf + m];
          wl[m] = e[3] * gi[bf + m];
        }
        const double gwv[3] = {e[0], e[1], e[2]};
        shell_center_terms(S, s, d, wv, wg, gwv, wl, out);
        for (int k = 0; k < 3; ++k) ae[k] -= out[k];
        double z3[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < nf; ++m) wv[m] = gi[bf + m];
        shell_center_terms(S, s, d, wv, z3, z3, z3, out);
        for (int k = 0; k < 3; ++k) al[k] -= out[k];
      }
      for (int k = 0; k < 3; ++k) {
        shacc[6 * s + k] += ae[k];
        shacc[6 * s + 3 + k] += al[k];
      }
    }
    __syncwarp();
    for (int I = lane; I < nn; I += WARP) {
      double se[3] = {0.0, 0.0, 0.0}, sl[3] = {0.0, 0.0, 0.0};
      for (int s = __ldg(S.atom_sh + I); s < __ldg(S.atom_sh + I + 1); ++s)
        for (int k = 0; k < 3; ++k) {
          se[k] += shacc[6 * s + k];
          sl[k] += shacc[6 * s + 3 + k];
        }
      for (int k = 0; k < 3; ++k) {
        if (ge) ge[3 * I + k] += se[k];
        if (gl) gl[3 * I + k] += sl[k];
      }
    }
    if (lane == 0) {
      if (eL_out) eL_out[w] = sing ? nan("") : ev.eL;
      if (lp_out) lp_out[w] = sing ? nan("") : logdet;
    }
    __syncwarp();
  }
}

// out[j] = sum_k w[k] rows[k * m + j] in the order k = 0, 1, ... (one column per thread).
__global__ void k_weighted_rows(int n, int m, const double* __restrict__ rows, const double* __restrict__ w,
                                double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(w[k], rows[(size_t)k * m + j], acc);
    out[j] = acc;
  }
}

}  // namespace lrdmc
