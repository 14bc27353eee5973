"""H2 (the STO-3G hydrogen molecule, 2 electrons, a = 0.2 bohr) at its stated
run size on the GPU against the oracle: 256 walkers, 100 branching intervals
of 20 moves (2000 steps), Philox seed 1, both schedules.

The trial function is nodeless (one doubly occupied orbital with positive
coefficients), so the fixed-node lattice Hamiltonian has no node-crossing
hop.  Its Gaussian orbital has no cusp: near a nucleus nu_zv ~ -1/r is not
bounded below, and in a load-balanced run W(x) - E_0 can come arbitrarily
close to zero, where the estimator weight 1/(W - E_0) (Sec. II.C) dominates
the average.  With node rule 2 (the cap nu^a_ei = -Z/max(r, a) applied to
every electron) W is bounded below and the run is stable; with the paper's
per-electron rule (0) the load-balanced estimate is dominated by such
walkers.  Both are compared: the GPU must reproduce the oracle in either case.

Acceptance: run means within 2 sigma of each other, sigma the
two runs' block-jackknife errors combined in quadrature.  Both programs draw
the same Philox streams and take the same hops, so the per-interval histories
(mean weight and walker-averaged local energy) also agree to floating-point
rounding over the first intervals, which pins far more than the 2 sigma test."""
import numpy as np
import pytest

import workloads as W
from oracle import estimator as OE
from oracle import lrdmc as OL

pytestmark = pytest.mark.gpu

N_W, N_BRANCH, N_PROJ, A, SEED = 256, 100, 20, 0.2, 1


def _tau(s, x0, node_rule):
    """Conventional projection time at the load-balanced move count:
    tau = N_proj / <b_bar>, <b_bar> over the walkers at the end of the first
    five load-balanced oracle intervals (deterministic given the seed)."""
    Wk = OL.init_walkers(s, x0, A, node_rule)
    E0 = float(np.mean(Wk.ev["eL"]))
    wb, eb, bb = [], [], []
    for j in range(5):
        OL.propagate_lb(s, Wk, A, E0, N_PROJ, SEED, j, node_rule)
        bb.append(float(np.mean(Wk.ev["bbar"])))
        w, e = OL.branch_stats(Wk, E0, OL.LOAD_BALANCED)
        wb.append(w)
        eb.append(e)
        OL.reconfigure(Wk, SEED, j)
        E0 = OE.energy(wb, eb, 10, 0)
    return N_PROJ / float(np.mean(bb))


@pytest.mark.parametrize("node_rule", [2, 0])
@pytest.mark.parametrize("schedule", [OL.LOAD_BALANCED, OL.CONVENTIONAL])
def test_h2_full_run_matches_oracle(schedule, node_rule):
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, N_W, seed=11)
    tau = _tau(s, x0, node_rule) if schedule == OL.CONVENTIONAL else None
    ho, _ = OL.run(s, x0, A, schedule, N_BRANCH, SEED, n_proj=N_PROJ, tau=tau, node_rule=node_rule,
                   p_gbar=10, n_equil=10)
    lr = P.Lrdmc(s, x0, A, seed=SEED, p_gbar=10, n_equil=10, node_rule=node_rule)
    for _ in range(N_BRANCH):
        lr.propagate(schedule, n_proj=N_PROJ, tau=tau or 0.0, max_moves=100000)
        lr.branch()
    E, err = lr.energy()
    hg = lr.history()
    assert np.isfinite(E) and np.isfinite(err) and err > 0
    assert abs(E - ho.energy) <= 2.0 * np.hypot(err, ho.error)
    # hop-for-hop: the first 20 intervals' statistics to rounding
    k = 20
    np.testing.assert_allclose(hg["wbar"][:k], ho.wbar[:k], rtol=1e-9)
    np.testing.assert_allclose(hg["ebar"][:k], ho.ebar[:k], rtol=1e-9, atol=1e-9)
    if node_rule == 2:
        # the stable run is near the exact energy at this spacing (the lattice
        # bias at a = 0.2 is about +0.07 Ha for this guiding function)
        assert -1.3 < E < -1.0
        assert hg["status_or"].max() == 0
    lr.close()


def test_h2_lattice_extrapolation_reaches_exact_energy():
    """Whole-path physics pin: the nodeless H2 guiding function makes fixed
    node exact, so the LRDMC energy E(a) tends to the exact non-relativistic
    energy of H2 at R = 1.4 bohr, -1.17447 Ha (Kolos and Wolniewicz; not in the
    paper), as a -> 0, with a bias that is even in a (Sec. II; Appendix D).
    The cusp-less Gaussian orbital makes that bias deviate from a pure a^2 law
    above a ~ 0.1 ((E - E_exact)/a^2 falls from about 2.0 at a = 0.05 to 1.4 at
    a = 0.3), so the scan covers a = 0.05 .. 0.14 and fits E_0 + c_2 a^2 +
    c_4 a^4 (lrdmc_extrapolate_a, weights 1/sigma^2).  Node rule 2 keeps W
    bounded below; the projection per interval is kept constant in imaginary
    time (20 (0.2/a)^2 moves)."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.h2_sto3g()
    spacings, Es, errs = [0.05, 0.07, 0.1, 0.14], [], []
    for a in spacings:
        n_proj = int(round(20 * (0.2 / a) ** 2))
        lr = P.Lrdmc(s, W.initial_walkers(s, 4096, seed=5), a, seed=7, p_gbar=10, n_equil=75, node_rule=2)
        for _ in range(300):
            lr.propagate(P.LOAD_BALANCED, n_proj=n_proj)
            lr.branch()
        E, err = lr.energy()
        assert lr.history()["status_or"].max() == 0
        Es.append(E)
        errs.append(err)
        lr.close()
    # the bias is positive and grows with a
    assert all(E > -1.17447 for E in Es) and np.all(np.diff(Es) > 0)
    coef, cov, _ = P.extrapolate_a(spacings, Es, errs, 2)
    sigma = float(np.sqrt(cov[0, 0]))
    assert sigma < 2e-3
    assert abs(coef[0] - (-1.17447)) <= 2.0 * sigma, (coef[0], sigma)


def test_h2_schedules_sample_the_same_energy():
    """The paper's equivalence of the two algorithms (Sec. II.C and its
    comparison of conventional and load-balanced LRDMC): at the same lattice
    spacing and the same mean number of moves per branching interval, the
    conventional and load-balanced runs of H2 at its stated size estimate the
    same energy, within 2 sigma combined."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, N_W, seed=11)
    tau = _tau(s, x0, 2)
    E, err, moves = {}, {}, {}
    for schedule in (OL.LOAD_BALANCED, OL.CONVENTIONAL):
        lr = P.Lrdmc(s, x0, A, seed=SEED, p_gbar=10, n_equil=10, node_rule=2)
        for _ in range(N_BRANCH):
            lr.propagate(schedule, n_proj=N_PROJ, tau=tau, max_moves=100000)
            lr.branch()
        E[schedule], err[schedule] = lr.energy()
        moves[schedule] = float(np.mean(lr.history()["moves_mean"]))
        lr.close()
    assert abs(moves[OL.CONVENTIONAL] - N_PROJ) < 0.5          # tau gives the same mean move count
    d = abs(E[OL.LOAD_BALANCED] - E[OL.CONVENTIONAL])
    assert d <= 2.0 * np.hypot(err[OL.LOAD_BALANCED], err[OL.CONVENTIONAL]), (E, err)
