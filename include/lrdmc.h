/*
 * lrdmc.h — C ABI of the B300 (sm_103a) LRDMC walker-propagation library.
 *
 * Implements the data-parallel hot path of lattice-regularised diffusion Monte
 * Carlo as described in Nakano, Sorella, Casula, "Load-Balanced Diffusion Monte
 * Carlo Method with Lattice Regularization" (arXiv 2508.12033):
 *   - the projection steps of all N_w walkers between two branchings, under the
 *     conventional fixed-projection-time schedule (Algorithm 1; Sec. II.B, the
 *     persistence time and continuous-time weight update) and the load-balanced
 *     fixed-N_proj schedule (Algorithm 2; Sec. II.C, the modified Green's function
 *     and its partition b_x, b_bar_x, p_{x',x});
 *   - the lattice-regularised fixed-node Hamiltonian those steps sample
 *     (Appendix D: 6 N_e single-electron hops of length a, spin-flip term,
 *     regularised local potential, per-electron nodal/nuclear cap);
 *   - the reconfiguration (branching) step with the correlated comb of Sec. II.A
 *     and the global-population-factor energy estimator of Sec. II.A.
 *
 * Conventions shared by every entry point
 *   - Every function returns an lrdmc_status; none aborts, none traps on the
 *     device.  After a failure lrdmc_last_error() describes it.
 *   - Inputs passed by host pointer are copied before the call returns; the
 *     caller keeps ownership.  A handle owns its device state unless the caller
 *     supplied the workspace (then the caller owns that memory and must keep it
 *     alive until lrdmc_destroy).
 *   - Device pointers (marked "device") must be CUDA device (or managed)
 *     allocations visible from the handle's device, 8-byte aligned.
 *   - All work is enqueued on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  Calls marked "synchronises" wait for that stream.
 *   - Electrons 0..n_up-1 are spin up, n_up..n_up+n_dn-1 spin down; positions are
 *     row-major [walker][electron][xyz] in bohr, energies in hartree.
 *   - Hop order of the 6 N_e lattice neighbours: p = 6 i + d with
 *     d = 0..5 -> (+x, -x, +y, -y, +z, -z) displacements of electron i by a.
 */
#ifndef LRDMC_H
#define LRDMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrdmc_s* lrdmc_handle;

typedef enum {
    LRDMC_OK = 0,
    LRDMC_ERR_ARG = 1,          /* invalid argument (sizes, NULL, out of range)     */
    LRDMC_ERR_CUDA = 2,         /* a CUDA runtime call failed                        */
    LRDMC_ERR_NONFINITE = 3,    /* a walker weight or local energy became non-finite */
    LRDMC_ERR_NEG_DIAG = 4,     /* W(x) - E_0 <= 0 met in a load-balanced step       */
    LRDMC_ERR_STEP_CAP = 5,     /* a conventional walker reached max_moves           */
    LRDMC_ERR_SINGULAR = 6,     /* a Slater matrix had a zero pivot                  */
    LRDMC_ERR_UNSUPPORTED = 7   /* system too large for the kernels' on-chip layout  */
} lrdmc_status;

/* Per-walker status bits (sticky until lrdmc_clear_status). */
#define LRDMC_WALKER_NEG_DIAG  1u   /* W - E_0 <= 0: the step weight was set to 0    */
#define LRDMC_WALKER_NONFINITE 2u
#define LRDMC_WALKER_STEP_CAP  4u
#define LRDMC_WALKER_STUCK     8u   /* no hop kept by the fixed-node rule (b_bar = 0) */
#define LRDMC_WALKER_SINGULAR  16u
#define LRDMC_WALKER_DRIFT     32u  /* re-inverted early: the inverse residual exceeded the drift tolerance */

/* Nuclei and electron counts (Appendix D: V_loc = sum nu_ei + sum nu_ee + V_ii). */
typedef struct {
    int n_nuc;
    const double* R;         /* host, n_nuc x 3                                      */
    const double* Z;         /* host, n_nuc: charge (valence charge for pseudo)      */
    const int* pot_kind;     /* host, n_nuc: 0 bare -Z/r, 1 screened -Z erf(r/r_c)/r */
    const double* r_c;       /* host, n_nuc: screening radius (kind 1 only)          */
    int n_up, n_dn;
} lrdmc_system;

/* Slater-Jastrow guiding function Psi_G = det A_up det A_dn exp(J).
 * Shell s: type shell_l[s] (0 = s, 1 = p with functions x,y,z, -1 = Slater 1s
 * exp(-zeta r)), centred on nucleus shell_atom[s], primitives
 * exps/coefs[off_s .. off_s + shell_nprim[s]) with off_s the running sum of
 * shell_nprim.  A contracted function is angular(d) * sum_g coefs_g exp(-exps_g |d|^2)
 * (Slater type: sum_g coefs_g exp(-exps_g |d|)); coefficients are used as given.
 * Orbitals phi_k = sum_mu C[k][mu] chi_mu; both spins use orbitals 0..n_sigma-1.
 * J = sum_{i<j} c r_ij/(1 + j2_b r_ij) - sum_{i,I} j1_A[I] r_iI/(1 + j1_B[I] r_iI),
 * c = j2_anti for opposite spins, j2_par for equal spins. */
typedef struct {
    int n_shell;
    const int* shell_atom;
    const int* shell_l;
    const int* shell_nprim;
    const double* exps;
    const double* coefs;
    int n_orb;
    const double* C;         /* host, n_orb x n_bf, row-major                         */
    double j2_anti, j2_par, j2_b;
    const double* j1_A;      /* host, n_nuc                                           */
    const double* j1_B;      /* host, n_nuc                                           */
} lrdmc_trial_wf;

typedef enum { LRDMC_CONVENTIONAL = 0, LRDMC_LOAD_BALANCED = 1 } lrdmc_kind;

/* One branching interval.  LOAD_BALANCED: every walker makes n_proj hops
 * (Algorithm 2).  CONVENTIONAL: every walker runs until its projection time tau
 * is used up (Algorithm 1), at most max_moves hops.
 * rotate != 0: randomised lattice (Appendix D): for this interval every walker
 * hops along its own uniformly random rotation of the three axes (drawn from
 * Philox counter (walker, 2^32-1, interval, 2..3)); every walker is re-evaluated
 * with the new versors before its first step.  Precision 0 only (the mixed
 * path returns LRDMC_ERR_UNSUPPORTED). */
typedef struct {
    int kind;
    int n_proj;
    double tau;
    int max_moves;
    int rotate;
} lrdmc_schedule;

/* Run parameters.
 *   a            lattice spacing (Appendix D)
 *   n_w          number of walkers (fixed by reconfiguration)
 *   seed         Philox4x32-10 key; streams are keyed by (walker slot, step,
 *                interval) so every call is reproducible
 *   node_rule    0: cap nu_zv,i by nu^a_ei only for electrons with a node-crossing
 *                hop (the paper's rule, per electron); 1: for all electrons when any
 *                hop crosses; 2: always; -1: never
 *   reinv_period Slater matrices are re-inverted from scratch every this many
 *                accepted hops of a walker (Sherman-Morrison in between)
 *   p_gbar       length p of the global population factor (Sec. II.A)
 *   n_equil      branchings discarded by lrdmc_energy
 *   precision    0 = FP64 throughout; 1 = mixed: FP32 evaluation of every hop
 *                ratio (as r - 1: basis and orbital differences, Jastrow
 *                differences) and of the orbital derivative cache; FP64
 *                positions, orbital values (rows of A), B = A^-1 with its
 *                Sherman-Morrison updates and Gauss-Jordan re-inversion every
 *                reinv_period hops, determinant derivatives, weights and the
 *                b_bar / W / e_L accumulators; 2 and 3 = mixed with the two
 *                FP32 orbital contractions against the MO coefficients (the
 *                moved electron's gradient/Laplacian rows and the orbital
 *                differences of its six hops, rows x N_bf x N_orb) on the tensor
 *                cores: warp-level mma.sync with TF32 (2) or BF16 (3) operands
 *                and FP32 accumulation; 4 =
 *                as 2 with each FP32 operand split into two TF32 parts and
 *                three MMAs per product (hi*hi + hi*lo + lo*hi), close to
 *                FP32 accuracy on the tensor cores                            */
typedef struct {
    double a;
    int n_w;
    uint64_t seed;
    int node_rule;
    int reinv_period;
    int p_gbar;
    int n_equil;
    int precision;
} lrdmc_params;

/* Device bytes a handle needs for this system and parameters (no allocation). */
lrdmc_status lrdmc_workspace_bytes(const lrdmc_system* sys, const lrdmc_trial_wf* wf,
                                   const lrdmc_params* prm, size_t* bytes);

/* Create a handle: copies the system and trial function to the device, places
 * the walkers at x0 (host, n_w x n_e x 3), inverts every Slater matrix from
 * scratch, evaluates the Hamiltonian at every walker and sets E_0 to the mean
 * local energy (the initial configurations of Algorithms 1 and 2).
 * workspace: device memory of at least lrdmc_workspace_bytes, 256-byte aligned,
 * or NULL to let the library allocate (and free) it.  stream: cudaStream_t or
 * NULL.  Synchronises. */
lrdmc_status lrdmc_create(const lrdmc_system* sys, const lrdmc_trial_wf* wf,
                          const lrdmc_params* prm, const double* x0,
                          void* workspace, size_t workspace_bytes, void* stream,
                          lrdmc_handle* out);

lrdmc_status lrdmc_destroy(lrdmc_handle h);

/* One interval: propagate all walkers between two branchings with the given
 * schedule (weights restart at 1).  Asynchronous. */
lrdmc_status lrdmc_propagate(lrdmc_handle h, const lrdmc_schedule* sch);

/* Branching step: records wbar_n = sum w / N_w and the walker-averaged local
 * energy ebar_n (Sec. II.A Eq. for ebar with weights w for the conventional
 * schedule, Sec. II.C form with weights w/(W - E_0) for the load-balanced one,
 * selected by the kind of the last lrdmc_propagate), reconfigures the
 * population with the integer comb (bit-exact, see lrdmc_reconfigure_indices),
 * resets every weight to 1 and, for the load-balanced schedule, sets E_0 to the
 * estimator over the history so far.  Synchronises (reads back a few scalars).
 * Returns LRDMC_ERR_NONFINITE, leaving the population and history unchanged,
 * when a weight is negative or non-finite or all weights are zero; the other
 * per-walker conditions (NEG_DIAG, STEP_CAP, STUCK, SINGULAR) do not stop the
 * run and are reported through the status bits and lrdmc_history. */
lrdmc_status lrdmc_branch(lrdmc_handle h);

/* Energy estimator E = sum_n Gbar_n^p ebar_n / sum_n Gbar_n^p over branchings
 * n >= n_equil, Gbar_n^p = prod_{j=1..p} wbar_{n-j}, with a block-jackknife error
 * (largest over block lengths 1, 2, 4, ... with >= 8 blocks; NaN if too few). */
lrdmc_status lrdmc_energy(lrdmc_handle h, double* E, double* err);

/* The estimator of lrdmc_energy over a caller-supplied branching history
 * (Sec. II.A: Gbar_n^p-weighted mean of ebar_n; the same block-jackknife
 * error), host arrays, no handle and no device work.
 *   wbar, ebar  n mean weights (> 0, finite) and walker-averaged local
 *               energies (finite) of consecutive branchings
 *   p_gbar      factors of Gbar_n^p; n_equil  branchings discarded
 *   E           out: the estimate (NaN if n <= n_equil)
 *   err         out or NULL: the error bar (NaN with fewer than 16 kept branchings)
 * LRDMC_ERR_ARG: n < 0, NULL arrays with n > 0, negative p_gbar or n_equil,
 * a non-positive or non-finite wbar, a non-finite ebar. */
lrdmc_status lrdmc_estimate(int n, const double* wbar, const double* ebar, int p_gbar, int n_equil, double* E,
                            double* err);

/* ------------------------------------------------------------ derivatives
 * Parameters differentiated by lrdmc_local_energy_grad, as one vector theta of
 * lrdmc_param_count = 5 n_nuc + 3 values: R (n_nuc x 3, bohr), j2_anti,
 * j2_par, j2_b, j1_A (n_nuc), j1_B (n_nuc). */
lrdmc_status lrdmc_param_count(lrdmc_handle h, int* n);
lrdmc_status lrdmc_get_params(lrdmc_handle h, double* theta);

/* Replace the handle's nuclear positions and Jastrow parameters (host theta);
 * V_ii is recomputed and every walker is re-placed at its current position
 * and weight (re-inverted and re-evaluated).  Synchronises. */
lrdmc_status lrdmc_set_params(lrdmc_handle h, const double* theta);

/* Hand-written adjoint of the lattice-regularised local energy e_L = W - b_bar
 * (Appendix D, the handle's node rule) and of log|Psi_G| at n configurations
 * (device x, n x n_e x 3; one launch, each warp evaluating its configurations
 * in a walker block of its own; large systems keep the per-warp working set in
 * global memory, allocated with that scratch on the first call), with
 * respect to theta:
 *   eL, logpsi          device, n (or NULL)
 *   grad_eL, grad_logpsi device, n x lrdmc_param_count (or NULL)
 * A configuration with a singular Slater matrix gets NaN values.  Precision 0
 * only (LRDMC_ERR_UNSUPPORTED otherwise).  Does not touch the walkers.
 * Asynchronous. */
lrdmc_status lrdmc_local_energy_grad(lrdmc_handle h, int n, const double* x, double* eL, double* logpsi,
                                     double* grad_eL, double* grad_logpsi);

/* out[j] = sum_k w[k] rows[k m + j] (device arrays; summation in the order
 * k = 0, 1, ...): the vector-Jacobian product of per-configuration gradient
 * rows.  Asynchronous. */
lrdmc_status lrdmc_weighted_rows(lrdmc_handle h, int n, int m, const double* rows, const double* w, double* out);

/* Lattice-space extrapolation (Sec. II: the LRDMC energy carries an O(a^2)
 * bias and is extrapolated to a -> 0 from runs at several spacings).  Weighted
 * least-squares fit of E(a) = sum_{j=0..order} coef[j] a^(2j) to the n points
 * (a[k], E[k]) with standard errors err[k] (weights 1/err^2), by Householder QR
 * of the weighted design matrix.  coef[0] is the a -> 0 energy.  Host-only
 * arrays, no handle and no device work.
 *   order   1 (E_0 + c a^2) to 3
 *   coef    out, order + 1 values
 *   cov     out or NULL, (order + 1)^2 covariance of coef, row-major
 *           (sqrt(cov[0]) is the standard error of the a -> 0 energy)
 *   chi2    out or NULL, weighted residual sum of squares
 * LRDMC_ERR_ARG: NULL inputs, order outside 1..3, n < order + 1, a non-finite
 * or non-positive a or err, non-finite E, or a rank-deficient design (fewer
 * than order + 1 distinct spacings). */
lrdmc_status lrdmc_extrapolate_a(int n, const double* a, const double* E, const double* err, int order,
                                 double* coef, double* cov, double* chi2);

/* Branching history: up to cap entries of wbar_n, ebar_n, the E_0 used in
 * interval n, the mean and max hops per walker, the number of distinct walkers
 * that survived reconfiguration and the OR of all walkers' status bits before
 * it.  *n receives the number of branchings so far.  Any pointer may be NULL. */
lrdmc_status lrdmc_history(lrdmc_handle h, int cap, int* n, double* wbar, double* ebar,
                           double* e0, double* moves_mean, int* moves_max, int* survivors,
                           uint32_t* status_or);

lrdmc_status lrdmc_get_e0(lrdmc_handle h, double* e0);
lrdmc_status lrdmc_set_e0(lrdmc_handle h, double e0);

/* Copy walker state to the host (synchronises).  Any pointer may be NULL, and
 * a NULL field is neither gathered nor copied; each requested field is copied
 * straight into the caller's buffer (pinned buffers take the fast DMA path).
 *   x (n_w x n_e x 3), w (n_w), ev (n_w x 4: b_bar, V_sf, W, e_L at the current
 *   configuration), ratios (n_w x 6 n_e: Psi_G(x_p)/Psi_G(x)), status (n_w),
 *   moves (n_w: hops in the last interval). */
lrdmc_status lrdmc_get_walkers(lrdmc_handle h, double* x, double* w, double* ev,
                               double* ratios, uint32_t* status, int32_t* moves);

/* Replace all walkers (host arrays; w may be NULL for all ones), re-invert and
 * re-evaluate from scratch.  Synchronises. */
lrdmc_status lrdmc_set_walkers(lrdmc_handle h, const double* x, const double* w);

lrdmc_status lrdmc_clear_status(lrdmc_handle h);

/* Checkpoint / resume (the paper is silent; library facility).  lrdmc_save
 * writes the complete walker state, E_0, the interval counter and the branching
 * history to a file (synchronises); lrdmc_load restores them into a handle
 * created for the same system, trial function and parameters.  Because every
 * random number is keyed by (seed, walker slot, step, interval), a run resumed
 * from a checkpoint continues bit for bit like the uninterrupted run.
 * The file records the lattice spacing a, the node rule and a 64-bit FNV-1a
 * fingerprint of the system and trial wavefunction (nuclei, potentials, basis,
 * orbital coefficients, Jastrow parameters): the stored walkers' cached
 * ratios, W and e_L belong to that Hamiltonian, so lrdmc_load returns
 * LRDMC_ERR_ARG, and leaves the handle unchanged, for a file whose layout, a,
 * node rule or fingerprint differs from the handle's, whose size disagrees
 * with its header (a corrupt history length), or that is truncated. */
lrdmc_status lrdmc_save(lrdmc_handle h, const char* path);
lrdmc_status lrdmc_load(lrdmc_handle h, const char* path);

/* Evaluate the lattice-regularised FN Hamiltonian at n <= n_w arbitrary
 * configurations (Appendix D), each from a freshly inverted Slater matrix.
 *   x       device, n x n_e x 3
 *   ratios  device, n x 6 n_e: Psi_G(x_p)/Psi_G(x) for every hop p
 *   ev      device, n x 4: b_bar, V_sf, W, e_L
 *   n_node  device, n: electrons with at least one node-crossing hop
 * Does not touch the walkers.  Asynchronous. */
lrdmc_status lrdmc_eval_configs(lrdmc_handle h, int n, const double* x, double* ratios,
                                double* ev, int32_t* n_node);

/* Reconfiguration indices alone (Sec. II.A, Eqs. for p_alpha and the comb
 * Z_alpha = (xi + alpha - 1)/N_w), handle-free:
 *   q_b = floor(w_b / max w * 2^S), S = 62 - bitlength(n), Q = inclusive prefix
 *   sum, and slot alpha (0-based) copies the first b with
 *   (xi32 + alpha 2^32) Q_total < n 2^32 Q_b   (exact 128-bit integer test).
 *   w          device, n doubles, finite, >= 0, not all 0
 *   src        device, n int32 outputs
 *   scratch    device, >= lrdmc_reconfigure_scratch_bytes(n) bytes, 256-byte aligned
 *   status_out device, 2 int32 (may be NULL): [0] = 0 ok / 1 invalid weights
 *              (src untouched), [1] = number of distinct source walkers
 * 1 <= n <= 2^24.  Asynchronous on stream. */
size_t lrdmc_reconfigure_scratch_bytes(int n);
lrdmc_status lrdmc_reconfigure_indices(int n, const double* w, uint32_t xi32, int32_t* src,
                                       void* scratch, size_t scratch_bytes,
                                       int32_t* status_out, void* stream);

/* Allocation-free variant of lrdmc_reconfigure_indices (the paper has no
 * counterpart; this is a library convenience).  It is meant for callers that
 * cannot call cudaMalloc -- for example a host whose device memory is managed
 * by its own (or an exhausted) allocator, or an embedding runtime that forbids
 * allocation on its hot path.  Instead of a
 * caller-provided scratch buffer it uses one fixed array in the library's
 * device memory, sized for LRDMC_NOALLOC_MAX_WALKERS walkers (about 2 MiB,
 * held on every GPU that loads the library until the process exits).
 *   - Same inputs, outputs and results as lrdmc_reconfigure_indices (w, xi32,
 *     src and status_out with the same meaning); nothing is allocated.
 *   - n must be in [1, LRDMC_NOALLOC_MAX_WALKERS]; a larger n returns
 *     LRDMC_ERR_UNSUPPORTED without launching anything, other bad arguments
 *     LRDMC_ERR_ARG.
 *   - The first call on a device looks up that device's copy of the array
 *     (a one-time set-up with that device current); make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after cudaDeviceReset on a device (which unloads the library's
 *     device code there) it is stale, so do not call this entry point on that
 *     device again.
 *   - All calls share the one array and it keeps the last call's contents;
 *     the kernel overwrites every scratch word before reading it.  Calls that
 *     overlap on the GPU (e.g. on two streams at once) race on the array and
 *     must be serialised by the caller. */
#define LRDMC_NOALLOC_MAX_WALKERS (1 << 18)
lrdmc_status lrdmc_reconfigure_indices_noalloc(int n, const double* w, uint32_t xi32, int32_t* src,
                                               int32_t* status_out, void* stream);

/* Philox4x32-10 block for counter (c0, c1, c2, c3) under key = seed, computed on
 * the host with the library's own implementation (testing aid). */
void lrdmc_philox4x32(uint64_t seed, const uint32_t ctr[4], uint32_t out[4]);

/* Testing aid: the library's reduced-slot FP64 exp, reciprocal and reciprocal
 * square root (table-driven exponential after Tang 1989; hardware approximations
 * refined by one third-order step) applied elementwise to n device doubles.  Any
 * output may be NULL.  Asynchronous on stream.  The first call on a device
 * copies the 2 KB exponential table to it (synchronous, under a lock). */
lrdmc_status lrdmc_fp64math(int n, const double* x, double* exp_out, double* rcp_out, double* rsqrt_out,
                            void* stream);

/* Testing aids for the screened potential -Z erf(r/r_c)/r of Appendix D's
 * local potential.  The library evaluates erf(r/r_c)/r = F(t)/r_c,
 * F(t) = erf(sqrt t)/sqrt t, t = r^2/r_c^2, from a table of one polynomial per
 * interval of width 1/2 in t (centred at k/2, k = 0 .. n_int - 1, powers of
 * t - k/2, lowest first, n_coef per interval), and as 1/r beyond the table.
 * lrdmc_erf_ratio_table writes the n_int x n_coef coefficients to out (host;
 * out may be NULL to query the sizes).  lrdmc_erf_over_r evaluates
 * erf(r/r_c)/r on the device for n device doubles s = r^2 (asynchronous on
 * stream); LRDMC_ERR_ARG for n < 0, NULL arrays or r_c <= 0. */
lrdmc_status lrdmc_erf_ratio_table(double* out, int* n_int, int* n_coef);
lrdmc_status lrdmc_erf_over_r(int n, const double* s, double r_c, double* out, void* stream);

/* Sherman-Morrison drift check (the paper is silent; numerical safeguard).
 * Between the periodic from-scratch inversions (every reinv_period hops) B is
 * kept by rank-1 updates, each adding rounding; near a node A is
 * ill-conditioned and the error grows.  The FP64 propagate kernel, on every
 * fourth hop since the last inversion, forms one row of A B - I (the row of
 * the electron after the moved one in its spin block, which the last update
 * did not touch; A from the cached FP64 orbital values) and re-inverts the
 * walker's Slater matrices at once when the largest |entry| exceeds tol.
 * The mixed-precision kernels (whose hop loop runs at its register limit)
 * check one row per spin block once per interval, before the first hop of a
 * walker that has hopped since its last inversion; on a hit they re-invert
 * before the first hop and evaluate that walker in full after it.
 * Such a walker gets the LRDMC_WALKER_DRIFT status bit.
 * lrdmc_set_drift_tol: tol >= 0 (0 disables the check; default 1e-11, which
 * keeps the hop ratios an order of magnitude inside 1e-10 relative);
 * LRDMC_ERR_ARG for a negative or NaN tol.  Takes effect at the next propagate.
 * lrdmc_drift_reinversions: drift-triggered re-inversions since the handle
 * was created, all walkers (synchronises). */
lrdmc_status lrdmc_set_drift_tol(lrdmc_handle h, double tol);

/* Checked build (library facility; the paper has no counterpart).  The build
 * step also compiles liblrdmc_checked.so with LRDMC_CHECKED defined: there every
 * data-derived index of the walker and branching kernels (hop, electron and
 * walker indices, comb and slot indices, shell / primitive / basis / nucleus
 * indices read from the system image, offsets into the per-hop shared scratch
 * and into the cache-block arrays) is tested against its extent before use.  A
 * failed test records the first violation in a device word -- source line of
 * the check in the high 32 bits, the offending index in the low 32 -- and
 * redirects the access to index 0 instead of faulting or trapping, so the
 * context stays usable.  It replaces a memory checker on small cases.
 *   lrdmc_checked_build: 1 in the checked library, 0 otherwise.
 *   lrdmc_check_word: synchronises the current device, then reads the word
 *     (0 = no violation) into *word and, with clear != 0, resets it.
 *   lrdmc_check_selftest: evaluates the check for index i against extent n on
 *     the device; *result is i when 0 <= i < n, else 0 with the violation
 *     recorded (a testing aid for the mechanism itself).
 * Both return LRDMC_ERR_UNSUPPORTED in the normal library. */
int lrdmc_checked_build(void);
lrdmc_status lrdmc_check_word(uint64_t* word, int clear);
lrdmc_status lrdmc_check_selftest(int i, int n, int* result);
lrdmc_status lrdmc_drift_reinversions(lrdmc_handle h, int64_t* n);

/* Load-imbalance measurement (the in-GPU image of the paper's argument that
 * a synchronised interval waits for its slowest walker).  With timing enabled
 * every propagate records, per walker, its start and stop time and SM;
 * lrdmc_interval_timing then reports for the last interval (synchronises):
 *   out[0] span of the interval (first start to last stop), ms
 *   out[1] mean and out[2] max walker time, ms
 *   out[3] busy fraction: total walker time / (span x resident warps)
 *   out[4] mean hops per walker, out[5] max hops per walker. */
lrdmc_status lrdmc_set_timing(lrdmc_handle h, int enable);
lrdmc_status lrdmc_interval_timing(lrdmc_handle h, double out[6]);

/* Number of kernels this handle has launched so far (all entry points). */
lrdmc_status lrdmc_launch_count(lrdmc_handle h, int64_t* n);

/* The cudaStream_t given at creation (for event timing on that stream). */
lrdmc_status lrdmc_stream(lrdmc_handle h, void** stream);

const char* lrdmc_last_error(lrdmc_handle h);
const char* lrdmc_status_string(lrdmc_status s);

/* ------------------------------------------------------------------ batches
 * Several independent systems (each with its own walkers, E_0 and history, as
 * in Sec. II) propagated by ONE persistent kernel launch per interval and
 * branched by one batched launch of each branching kernel.  Each system k is
 * described exactly as for lrdmc_create (sys[k], wf[k], prm[k] with its own
 * n_w and seed, x0[k] a host array n_w x N_e x 3) and owns an ordinary handle
 * (lrdmc_batch_handle) for readback, energies, history and checkpoints; the
 * batch owns those handles.  All systems must use the same precision and the
 * same CUDA device; the stream is shared.  A system's walkers follow the
 * trajectory they would follow in their own handle (the batch changes only
 * which warp runs which walker): the same hops and positions, with weights and
 * energies equal up to rounding (the batched kernel is compiled separately
 * and may fuse the same operations differently). */
typedef struct lrdmc_batch_s* lrdmc_batch;

/* Create the batch (allocates each system's workspace with cudaMalloc).
 * LRDMC_ERR_ARG for n_sys < 1, NULL arrays or mixed precisions; otherwise the
 * status of the first system that fails to create (its message is kept). */
lrdmc_status lrdmc_batch_create(int n_sys, const lrdmc_system* sys, const lrdmc_trial_wf* wf,
                                const lrdmc_params* prm, const double* const* x0, void* stream, lrdmc_batch* out);
lrdmc_status lrdmc_batch_destroy(lrdmc_batch b);

/* The handle of system k (owned by the batch: do not destroy it; its
 * propagate/branch calls remain valid and act on that system alone). */
lrdmc_status lrdmc_batch_handle(lrdmc_batch b, int k, lrdmc_handle* h);

/* One interval for every walker of every system: a single launch of the
 * persistent batched kernel (sch as for lrdmc_propagate; the randomised
 * lattice is refused with LRDMC_ERR_UNSUPPORTED). */
lrdmc_status lrdmc_batch_propagate(lrdmc_batch b, const lrdmc_schedule* sch);

/* Branch every system: one launch each of the batched reduction, comb and
 * gather kernels and one readback of all systems' statistics; each system's
 * history and E_0 are updated as by lrdmc_branch.  A system whose weights are
 * invalid keeps its population and history and makes the call return
 * LRDMC_ERR_NONFINITE after the other systems are branched. */
lrdmc_status lrdmc_batch_branch(lrdmc_batch b);

/* Order in which the persistent kernel hands out walkers: 0 = system by system
 * in creation order, 1 (default) = systems by decreasing estimated cost per
 * walker (N_e (N_bf + N_nuc + N_e)), the longest jobs first. */
lrdmc_status lrdmc_batch_set_order(lrdmc_batch b, int policy);

/* Autotuner of the launch shape.  The batched kernel runs persistent CTAs; a
 * CTA takes an item (system k, up to c_k consecutive walkers), gives each warp
 * one walker and splits its shared memory into c_k regions of system k's
 * per-walker size, so c_k follows the CTA's shared-memory size.  Candidates:
 * 1, 2, 3 or 4 CTAs per SM (each CTA with 1/1, 1/2, 1/3, 1/4 of the opt-in
 * shared memory; candidates where some system does not fit are skipped).  The
 * tuner times one interval of schedule sch with each candidate, restoring every
 * walker and cache after each trial, and keeps the fastest.  times_ms (may be
 * NULL) receives the 4 timings (0 where the candidate does not fit);
 * *best_ctas (may be NULL) the chosen CTAs per SM. */
lrdmc_status lrdmc_batch_tune(lrdmc_batch b, const lrdmc_schedule* sch, double times_ms[4], int* best_ctas);

/* Timing of the last batched interval over all systems (requires
 * lrdmc_batch_set_timing(b, 1) before it), from every walker's start and stop
 * time and SM: out[0] span ms, out[1] mean and out[2] max walker ms, out[3] SM
 * idle fraction = 1 - (time each SM runs at least one walker, summed over SMs)
 * / (span x SMs), out[4] mean idle tail ms per SM (span end - its last
 * walker's end), out[5] walker-slot busy fraction = total walker time /
 * sum over items of (walkers in the item x item duration) — the warps of a
 * CTA wait at the end of an item for its slowest walker — out[6] walkers,
 * out[7] items. */
lrdmc_status lrdmc_batch_set_timing(lrdmc_batch b, int enable);
lrdmc_status lrdmc_batch_timing(lrdmc_batch b, double out[8]);

/* Kernels launched by the batch's own entry points. */
lrdmc_status lrdmc_batch_launch_count(lrdmc_batch b, int64_t* n);
const char* lrdmc_batch_last_error(lrdmc_batch b);

#ifdef __cplusplus
}
#endif
#endif /* LRDMC_H */
