"""Sherman-Morrison drift check (numerical safeguard; the paper is silent).

The propagate kernels keep B = A^-1 by rank-1 updates between from-scratch
inversions; after every hop they form two rows of A B - I and re-invert when
the largest entry exceeds the handle's drift tolerance.  Checked here:
  * the counter: the FP64 check runs on every fourth hop since the last
    inversion, the mixed one once per interval; at a tolerance below any
    attainable residual every check re-inverts (the periodic inversion is
    switched off by a very long period);
  * parity: walkers propagated with the check on and no periodic inversion
    follow the oracle (fresh determinants every step) hop for hop, to the FP64
    per-configuration tolerance;
  * the status bit of the walkers that re-inverted early, and argument checks."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_close, lib_or_skip
from oracle import estimator as OE
from oracle import lrdmc as OL

pytestmark = pytest.mark.gpu

NO_PERIODIC = 1 << 30


@pytest.mark.parametrize("precision", [0, 1])
def test_drift_counter_counts_every_forced_reinversion(precision):
    """FP64: the check runs on every fourth hop since the last inversion, so
    7 hops of a fresh walker check (and, forced, re-invert) once.  Mixed: the
    check runs once per interval, before the first hop, for a walker that has
    hopped since its last inversion -- not in a fresh walker's first interval,
    once in the next."""
    P = lib_or_skip()
    s = W.water_methane()
    lr = P.Lrdmc(s, W.initial_walkers(s, 40, seed=2), 0.2, seed=3, reinv_period=NO_PERIODIC, precision=precision)
    lr.set_drift_tol(1e-300)          # every residual exceeds it
    n0 = lr.drift_reinversions()
    lr.propagate(P.LOAD_BALANCED, n_proj=7)
    if precision == 1:
        assert lr.drift_reinversions() == n0
        lr.branch()
        lr.propagate(P.LOAD_BALANCED, n_proj=7)
    g = lr.get_walkers(("moves", "status"))
    assert np.all(g["moves"] == 7)
    assert lr.drift_reinversions() - n0 == 40
    assert np.all(g["status"] & 32)
    lr.set_drift_tol(0.0)             # off: no further early re-inversions
    lr.branch()
    lr.propagate(P.LOAD_BALANCED, n_proj=5)
    assert lr.drift_reinversions() - n0 == 40
    with pytest.raises(P.LrdmcError):
        lr.set_drift_tol(-1.0)
    with pytest.raises(P.LrdmcError):
        lr.set_drift_tol(float("nan"))
    lr.close()


@pytest.mark.parametrize("tol", [1e-300, 1e-12])
def test_drift_checked_walkers_follow_the_oracle_without_periodic_inversion(tol):
    """64 water-methane walkers, three 20-hop load-balanced intervals with
    branching, no periodic inversion: the inverse is kept by Sherman-Morrison
    alone and re-inverted only when the drift check fires.  Positions must
    equal the oracle's, weights, e_L and ratios agree to 1e-10."""
    P = lib_or_skip()
    s = W.water_methane()
    x0 = W.initial_walkers(s, 64, seed=5)
    lr = P.Lrdmc(s, x0, 0.2, seed=1, reinv_period=NO_PERIODIC)
    lr.set_drift_tol(tol)
    Wk = OL.init_walkers(s, x0, 0.2)
    E0 = float(np.mean(Wk.ev["eL"]))
    wb, eb = [], []
    for j in range(3):
        lr.propagate(P.LOAD_BALANCED, n_proj=20)
        OL.propagate_lb(s, Wk, 0.2, E0, 20, seed=1, interval=j)
        g = lr.get_walkers()
        np.testing.assert_array_equal(g["x"], Wk.x)
        assert_close(g["w"], Wk.w, what="w")
        assert_close(g["ev"][:, 3], Wk.ev["eL"], what="eL")
        assert_close(g["ratios"], Wk.ev["ratios"], what="ratios")
        lr.branch()
        w, e = OL.branch_stats(Wk, E0, OL.LOAD_BALANCED)
        wb.append(w)
        eb.append(e)
        OL.reconfigure(Wk, 1, j)
        E0 = OE.energy(wb, eb, 10, 0)          # load-balanced E_0: the estimator over the branchings so far
    if tol == 1e-300:
        assert lr.drift_reinversions() == 64 * 3 * 5
    lr.close()
