"""Pins for the oracle's schedules, heat-bath choice, reconfiguration and
estimator: closed forms, invariants, distribution laws and an exact
diagonalisation of a one-electron lattice Hamiltonian."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import stats

import workloads as W
from oracle import estimator as est
from oracle import lrdmc as L
from oracle import philox
from oracle import wavefunction as WF


# ---------------------------------------------------------------- reconfiguration
@pytest.mark.parametrize("n", [1, 2, 7, 100, 4096])
def test_reconfiguration_invariants(n):
    rng = np.random.default_rng(n)
    w = rng.lognormal(0.0, 0.7, n)
    xi = int(rng.integers(0, 2**32))
    src = L.reconfigure_indices(w, xi)
    assert len(src) == n
    assert np.all(np.diff(src) >= 0)                    # comb order is monotone
    counts = np.bincount(src, minlength=n)
    expect = n * w / w.sum()
    # each walker is copied floor or ceil of N w / sum w times (up to 2^-S quantisation)
    assert np.all(counts >= np.floor(expect - 1e-9)) and np.all(counts <= np.ceil(expect + 1e-9))


@pytest.mark.parametrize("n", [1, 2, 7, 100, 4096])
def test_slot_assignment_keeps_survivors_in_place(n):
    """The stored population holds every walker as often as the comb copies it;
    a selected walker stays in its own slot; only unselected slots change, and
    they receive the further copies in comb order; equal weights move nothing."""
    rng = np.random.default_rng(n + 7)
    w = rng.lognormal(0.0, 0.7, n)
    src = L.reconfigure_indices(w, int(rng.integers(0, 2**32)))
    slot = L.slot_assignment(src)
    np.testing.assert_array_equal(np.bincount(slot, minlength=n), np.bincount(src, minlength=n))
    selected = np.bincount(src, minlength=n) > 0
    np.testing.assert_array_equal(slot[selected], np.flatnonzero(selected))
    free = np.flatnonzero(~selected)
    extra = [src[a] for a in range(1, n) if src[a] == src[a - 1]]     # second, third, ... copies
    np.testing.assert_array_equal(slot[free], extra)
    np.testing.assert_array_equal(L.slot_assignment(np.arange(n)), np.arange(n))
    # a hand-worked case: walker 1 copied three times, 0 and 2 not selected, 3 once
    np.testing.assert_array_equal(L.slot_assignment(np.array([1, 1, 1, 3])), [1, 1, 1, 3])
    np.testing.assert_array_equal(L.slot_assignment(np.array([0, 0, 2, 2, 2, 4])), [0, 0, 2, 2, 4, 2])


def test_reconfiguration_equal_weights_is_identity():
    for n in (1, 5, 1000):
        for xi in (0, 1, 2**31, 2**32 - 1):
            np.testing.assert_array_equal(L.reconfigure_indices(np.full(n, 3.7), xi), np.arange(n))


def test_reconfiguration_matches_float_comb():
    """Against the comb of Eq. (correlated random numbers) in exact rational
    arithmetic on the same quantised weights, for random inputs."""
    from fractions import Fraction
    rng = np.random.default_rng(1)
    for n in (3, 17, 64):
        w = rng.random(n) ** 3
        xi = int(rng.integers(0, 2**32))
        S = L.quant_shift(n)
        wmax = w.max()
        q = [int(math.floor((v / wmax) * 2.0**S)) for v in w]
        tot = sum(q)
        cum = np.cumsum(q)
        ref = []
        for alpha in range(n):
            z = (Fraction(xi, 2**32) + alpha) / n
            ref.append(next(b for b in range(n) if z < Fraction(int(cum[b]), tot)))
        np.testing.assert_array_equal(L.reconfigure_indices(w, xi), ref)


def test_reconfiguration_unbiased_copy_counts():
    """E[copies of b] = N w_b / sum w over the comb offset xi."""
    w = np.array([0.1, 2.0, 0.5, 0.5, 1.4, 0.0])
    n = len(w)
    acc = np.zeros(n)
    m = 4000
    for xi in np.linspace(0, 2**32 - 1, m).astype(np.int64):
        acc += np.bincount(L.reconfigure_indices(w, int(xi)), minlength=n)
    np.testing.assert_allclose(acc / m, n * w / w.sum(), atol=2e-3)


# ------------------------------------------------------------------- heat bath
def test_heat_bath_choice_distribution():
    rng = np.random.default_rng(2)
    r = rng.normal(0.5, 0.6, (1, 12))
    n = 200000
    u = rng.random(n)
    hop = L.choose_hop(np.repeat(r, n, axis=0), u)
    kept = np.where(r[0] > 0, r[0], 0.0)
    counts = np.bincount(hop, minlength=12)
    assert np.all(counts[kept == 0] == 0)
    expect = n * kept / kept.sum()
    m = kept > 0
    chi2 = np.sum((counts[m] - expect[m]) ** 2 / expect[m])
    assert stats.chi2.sf(chi2, m.sum() - 1) > 1e-4
    assert np.all(L.choose_hop(-np.abs(r), np.array([0.3])) == -1)


def test_heat_bath_edge_uniforms():
    r = np.array([[0.0, 1.0, -2.0, 3.0, 0.0, 0.0]])
    assert L.choose_hop(r, np.array([0.0]))[0] == 1
    assert L.choose_hop(r, np.array([1.0 - 2.0**-53]))[0] == 3
    assert L.choose_hop(r, np.array([0.2499999]))[0] == 1
    assert L.choose_hop(r, np.array([0.25]))[0] == 3          # strict '>' on the running sum


# --------------------------------------------------------- exact H atom end to end
@pytest.mark.parametrize("schedule", [L.LOAD_BALANCED, L.CONVENTIONAL])
def test_exact_wavefunction_zero_variance_run(schedule):
    s = W.hydrogen_atom_sto(1.0)
    x0 = W.initial_walkers(s, 32, seed=3)
    h, Wk = L.run(s, x0, 0.2, schedule, 8, seed=1, n_proj=10, tau=0.07)
    assert abs(h.energy + 0.5) < 1e-12
    np.testing.assert_allclose(h.ebar, -0.5, atol=1e-12)
    if schedule == L.CONVENTIONAL:
        # w = exp(-tau e_L) exactly for a constant local energy
        np.testing.assert_allclose(h.wbar, math.exp(0.07 * 0.5), rtol=1e-13)
    assert h.status_or == 0


# ------------------------------------------------ conventional persistence times
class _ConstEval:
    """Stand-in Hamiltonian with every hop ratio equal (b_bar constant), local
    energy e: the number of hops in tau is a Poisson(tau b_bar) count."""

    def __init__(self, ratio, a, e=0.0):
        self.ratio, self.a, self.e = ratio, a, e

    def __call__(self, sys, x, a, node_rule=0, versors=None):
        n = x.shape[0]
        ne = x.shape[1]
        bbar = 6 * ne * self.ratio / (2 * a * a)
        return dict(ratios=np.full((n, ne, 6), self.ratio), bbar=np.full(n, bbar),
                    vsf=np.zeros(n), W=np.full(n, bbar + self.e), eL=np.full(n, self.e),
                    n_node=np.zeros(n, np.int64), lap=np.zeros((n, ne)),
                    nu_opt=np.zeros((n, ne)))


def test_conventional_hop_count_is_poisson(monkeypatch):
    a = 0.5
    fake = _ConstEval(1.0 / 3.0, a, e=0.3)
    monkeypatch.setattr(L.ham, "evaluate", fake)
    s = W.hydrogen_atom_sto()
    n = 20000
    Wk = L.init_walkers(s, np.zeros((n, 1, 3)), a)
    bbar = 2.0 * 1.0 / (a * a) * 1.0 / 1.0   # 6 * (1/3) / (2 a^2) = 1/a^2 = 4
    tau = 2.5
    L.propagate_conventional(s, Wk, a, tau, seed=9, interval=4)
    lam = tau * 4.0
    assert abs(Wk.moves.mean() - lam) < 4 * math.sqrt(lam / n)
    assert abs(Wk.moves.var() / lam - 1.0) < 0.05
    ks = np.arange(0, 30)
    obs = np.bincount(Wk.moves, minlength=30)[:30]
    exp_ = n * stats.poisson.pmf(ks, lam)
    m = exp_ > 5
    chi2 = np.sum((obs[m] - exp_[m]) ** 2 / exp_[m])
    assert stats.chi2.sf(chi2, m.sum() - 1) > 1e-4
    np.testing.assert_allclose(Wk.w, math.exp(-tau * 0.3), rtol=1e-12)
    del bbar


def test_conventional_slowest_walker_grows_with_population(monkeypatch):
    """Appendix C's emulation: the mean number of hops to exhaust tau is flat in
    N_w while the maximum (what a synchronised interval waits for) grows."""
    a = 1.0
    monkeypatch.setattr(L.ham, "evaluate", _ConstEval(1.0 / 3.0, a))
    s = W.hydrogen_atom_sto()
    means, maxs = [], []
    for n in (10, 100, 1000, 10000):
        Wk = L.init_walkers(s, np.zeros((n, 1, 3)), a)
        L.propagate_conventional(s, Wk, a, 5.0, seed=3, interval=0)
        means.append(Wk.moves.mean())
        maxs.append(Wk.moves.max())
    assert np.all(np.abs(np.array(means) - 5.0) < 1.5)
    assert maxs[0] < maxs[1] < maxs[3] and maxs[2] <= maxs[3]


def test_load_balanced_every_walker_makes_n_proj_hops():
    s = W.h2_sto3g()
    Wk = L.init_walkers(s, W.initial_walkers(s, 16, seed=2), 0.2)
    L.propagate_lb(s, Wk, 0.2, -1.1, 7, seed=1, interval=0)
    assert np.all(Wk.moves == 7)


# ------------------------------------------------------------- estimator
def test_estimator_worked_example():
    # Gbar_0 = 1, Gbar_1 = 2, Gbar_2 = 2*3 (p = 2): E = (1 + 4 + 24) / 9
    assert abs(est.energy([2.0, 3.0, 5.0], [1.0, 2.0, 4.0], p=2) - 29.0 / 9.0) < 1e-15
    # p = 1: Gbar = 1, 2, 3
    assert abs(est.energy([2.0, 3.0, 5.0], [1.0, 2.0, 4.0], p=1) - (1 + 4 + 12) / 6.0) < 1e-15
    # equilibration cut
    assert abs(est.energy([2.0, 3.0, 5.0], [1.0, 2.0, 4.0], p=2, n_equil=1) - (4 + 24) / 8.0) < 1e-15
    # huge weights do not overflow: Gbar = 1, 1e200, 1e400, 1e600, 1e600
    assert abs(est.energy([1e200] * 5, [1.0, 2.0, 3.0, 4.0, 5.0], p=3) - 4.5) < 1e-12


def test_estimator_error_on_iid_series():
    rng = np.random.default_rng(0)
    n = 4096
    e = rng.normal(-1.0, 0.2, n)
    err = est.energy_error(np.ones(n), e, p=5)
    assert 0.8 * 0.2 / math.sqrt(n) < err < 1.5 * 0.2 / math.sqrt(n)


# ------------------------------------- exact diagonalisation of the lattice problem
def _lattice_ground_energy(psi, lap_over_psi, a, L_side):
    """Lowest eigenvalue of H^a (Appendix D) for one electron and a bare proton
    at the origin, on the sites a (n + 1/2) of an L^3 box (hops that leave the
    box dropped), for a nodeless guiding function psi(r) with continuum
    lap psi / psi given in closed form.  Built directly from the paper's
    definitions: off-diagonal -1/(2a^2) between neighbours; diagonal
    3/a^2 + nu_zv with nu_zv = -1/r + [Delta_a Psi/Psi - Delta Psi/Psi]/2."""
    n1 = np.arange(L_side) - L_side // 2
    c = a * (n1 + 0.5)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    disc = np.zeros_like(r)
    for Q in (X, Y, Z):
        for sgn in (1.0, -1.0):
            rq = np.sqrt(r * r + 2 * sgn * a * Q + a * a)
            disc += psi(rq) / psi(r)
    disc = (disc - 6.0) / (a * a)
    diag = 3.0 / (a * a) - 1.0 / r + 0.5 * (disc - lap_over_psi(r))
    N = L_side ** 3
    idx = np.arange(N).reshape(L_side, L_side, L_side)
    rows, cols = [], []
    for ax in range(3):
        a0 = [slice(None)] * 3
        a1 = [slice(None)] * 3
        a0[ax] = slice(0, L_side - 1)
        a1[ax] = slice(1, L_side)
        rows.append(idx[tuple(a0)].ravel())
        cols.append(idx[tuple(a1)].ravel())
    rr = np.concatenate(rows)
    cc = np.concatenate(cols)
    off = -1.0 / (2 * a * a)
    Hm = sp.coo_matrix((np.full(2 * len(rr), off), (np.concatenate([rr, cc]), np.concatenate([cc, rr]))),
                       shape=(N, N)).tocsr() + sp.diags(diag.ravel())
    vals = spla.eigsh(Hm, k=1, which="SA", tol=1e-10)[0]
    return float(vals[0])


ZETA_ED = 0.8


def lattice_ground_energy_sto(zeta, a, L_side=56):
    return _lattice_ground_energy(lambda r: np.exp(-zeta * r),
                                  lambda r: zeta * zeta - 2.0 * zeta / r, a, L_side)


@pytest.mark.parametrize("schedule", [L.LOAD_BALANCED, L.CONVENTIONAL])
def test_both_schedules_reach_the_lattice_ground_energy(schedule):
    a = 0.4
    e_exact = lattice_ground_energy_sto(ZETA_ED, a)
    s = W.hydrogen_atom_sto(ZETA_ED)
    x0 = W.lattice_walkers(300, a, seed=4, spread=3)
    # conventional: tau chosen for ~15 hops per interval (b_bar ~ 6/(2a^2))
    h, _ = L.run(s, x0, a, schedule, 160, seed=5, n_proj=15, tau=15 / (6 / (2 * a * a)),
                 p_gbar=20, n_equil=30)
    assert h.status_or == 0
    assert h.error < 2e-3
    assert abs(h.energy - e_exact) < 4 * h.error + 1e-4, (h.energy, h.error, e_exact)
    if schedule == L.LOAD_BALANCED:
        # Appendix B: with E_0 at the ground energy, (W - E_0) Psi_G Psi_0 is
        # stationary under the modified Green's function with eigenvalue 1, so
        # the mean weight gained per interval is 1 once equilibrated.
        wb = np.array(h.wbar[30:])
        assert abs(wb.mean() - 1.0) < 5 * wb.std() / math.sqrt(len(wb)) + 2e-3


# ----------------------------------------------------------- randomised lattice
def test_random_versors_are_haar_rotations():
    """Shoemake's construction: orthonormal rows, determinant +1, and each
    rotated axis uniformly distributed on the sphere (its z component is
    uniform on [-1, 1], mean of the matrix 0)."""
    V = L.interval_versors(7, np.arange(40000), 11)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", V, V), np.broadcast_to(np.eye(3), V.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(V), 1.0, atol=1e-14)
    assert np.abs(V.mean(axis=0)).max() < 0.02
    for k in range(3):
        assert stats.kstest(V[:, k, 2], "uniform", args=(-1.0, 2.0)).pvalue > 1e-4
    # different intervals and walkers draw different rotations
    assert not np.allclose(L.interval_versors(7, [0], 11), L.interval_versors(7, [0], 12))


def test_randomised_lattice_keeps_exact_energy_and_hop_length():
    s = W.hydrogen_atom_sto(1.0)
    x0 = W.initial_walkers(s, 24, seed=3)
    for sched in (L.LOAD_BALANCED, L.CONVENTIONAL):
        h, Wk = L.run(s, x0, 0.25, sched, 4, seed=2, n_proj=6, tau=0.05, rotate=True)
        assert abs(h.energy + 0.5) < 1e-12
    # every hop moves an electron by exactly a along one of its interval's versors
    Wk = L.init_walkers(s, x0, 0.25)
    before = Wk.x.copy()
    L.propagate_lb(s, Wk, 0.25, -0.5, 1, seed=2, interval=9, rotate=True)
    step = np.linalg.norm(Wk.x - before, axis=-1)
    np.testing.assert_allclose(step, 0.25, rtol=1e-12)


def test_fixed_lattice_after_randomised_interval_reevaluates_on_the_axes():
    """The evaluation a randomised interval leaves behind belongs to its
    versors; a following fixed-lattice interval starts from the Cartesian
    evaluation (ratios of the six axis hops, checked against the definition
    Psi(x')/Psi(x) from fresh log-amplitudes)."""
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, 6, seed=4)
    Wk = L.init_walkers(s, x0, 0.2)
    L.propagate_lb(s, Wk, 0.2, -1.0, 2, seed=3, interval=0, rotate=True)
    assert Wk.rotated
    L.propagate_lb(s, Wk, 0.2, -1.0, 0, seed=3, interval=1, rotate=False)
    assert not Wk.rotated
    for n in range(2):
        for i in range(s.n_up + s.n_dn):
            for d in range(6):
                xp = Wk.x[n].copy()
                xp[i, d // 2] += 0.2 if d % 2 == 0 else -0.2
                s1, l1 = WF.log_psi(s, xp)
                s0, l0 = WF.log_psi(s, Wk.x[n])
                ref = s1 * s0 * np.exp(l1 - l0)
                assert abs(Wk.ev["ratios"].reshape(6, -1)[n, 6 * i + d] - ref) <= 1e-10 * max(1.0, abs(ref))


def test_zero_weight_walkers_carry_no_statistical_weight():
    """Sec. II.A: the walker-averaged local energy runs over the population
    with weights w; a walker of zero weight (the load-balanced step zeroes the
    weight where W - E_0 <= 0) adds nothing, even with a non-finite e_L or W,
    and the mean weight still counts it in N_w."""
    import numpy as np
    from oracle import lrdmc as L
    ev = {"eL": np.array([-1.0, -2.0, np.nan, -4.0]), "W": np.array([3.0, 4.0, np.nan, 6.0])}
    Wk = L.Walkers(x=np.zeros((4, 1, 3)), w=np.array([1.0, 2.0, 0.0, 1.0]), ev=ev,
                   status=np.zeros(4, np.uint32), moves=np.zeros(4, np.int64))
    wbar, ebar = L.branch_stats(Wk, 1.0, L.CONVENTIONAL)
    assert wbar == 1.0 and ebar == (-1.0 - 4.0 - 4.0) / 4.0
    wbar, ebar = L.branch_stats(Wk, 1.0, L.LOAD_BALANCED)
    f = np.array([1.0 / 2.0, 2.0 / 3.0, 1.0 / 5.0])
    assert abs(ebar - float(np.sum(f * np.array([-1.0, -2.0, -4.0])) / np.sum(f))) < 1e-15


def test_nodal_lattice_hamiltonian_matches_the_oracle_evaluation():
    """Node-crossing pieces of Appendix D pinned against the Hamiltonian built
    from the definitions (tests/lattice_ed.py): for the p_z guiding function
    of the hydrogen atom, at lattice sites on both sides of the nodal plane,
    next to it and next to the nucleus, the oracle's sum of kept ratios
    (2 a^2 b_bar), V_sf and W equal the definitions' values (the cap applied
    exactly where a hop crosses the node); and the lowest eigenvalue of H^a
    has converged in the box size used by the GPU pin."""
    from lattice_ed import pz_lattice_ground_energy, pz_site_terms
    from oracle import hamiltonian as ham
    s = W.hydrogen_atom_pz(0.1)
    a = 0.4
    rng = np.random.default_rng(3)
    n = rng.integers(-12, 12, size=(400, 3)).astype(float)
    n[:20, 2] = rng.choice([-1.0, 0.0], 20)                 # next to the nodal plane
    n[20:40] = rng.integers(-1, 1, size=(20, 3))              # next to the nucleus
    x = a * (n + 0.5)
    kept, vsf, Wd, node = pz_site_terms(0.1, a, x[:, 0], x[:, 1], x[:, 2])
    ev = ham.evaluate(s, x[:, None, :], a, node_rule=0)
    assert node.sum() > 30 and (~node).sum() > 300
    np.testing.assert_allclose(ev["bbar"] * 2 * a * a, kept, rtol=1e-12)
    np.testing.assert_allclose(ev["vsf"], vsf, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ev["W"], Wd, rtol=1e-12)
    assert np.array_equal(ev["n_node"] > 0, node)
    e80, e96 = pz_lattice_ground_energy(0.1, a, 80), pz_lattice_ground_energy(0.1, a, 96)
    assert abs(e80 - e96) < 1e-6
    assert -0.125 < e96 < -0.12       # above the exact 2p energy, by the lattice bias at a = 0.4
