"""Failure detection without a GPU fault, and determinism.

Failures are made on the host: walkers are placed at NaN or coincident
positions through lrdmc_set_walkers.  The kernels must not fault (every index
derived from data is masked or clamped: the exponential and erf tables, the
heat-bath choice, the pivot search, the comb), they must flag the walkers
(LRDMC_WALKER_NONFINITE / SINGULAR / STUCK), and the branching must refuse the
population (LRDMC_ERR_NONFINITE) and leave it unchanged.  The checked build
runs this file too (tests/test_gpu_checked_build.py), where any index that
escaped its extent would be recorded.

Determinism: walkers are handed to warps by an atomic work counter, so which
warp runs which walker changes from run to run; every result must not.  Two
runs of the same inputs are compared bit for bit."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib_or_skip

pytestmark = pytest.mark.gpu

ST_NONFINITE, ST_STUCK, ST_SINGULAR = 2, 8, 16


def _bad_walkers(s, x):
    bad = x.copy()
    bad[3, 5, :] = np.nan                 # a NaN electron
    bad[7, 2, :] = bad[7, 9, :]           # two electrons on one point (opposite spins: pair terms blow up)
    bad[11, 1, :] = bad[11, 4, :]         # two electrons on one point (same spin: A singular)
    good = np.ones(len(x), bool)
    good[[3, 7, 11]] = False
    return bad, good


@pytest.mark.parametrize("precision", [0, 1])
def test_broken_walkers_drop_out_of_a_load_balanced_population(precision):
    """Load-balanced schedule: a walker whose W is not finite gets step weight
    0 (the W - E_0 > 0 test fails) and a status bit; it carries no weight in
    the branching averages and the comb never copies it, so after branching
    the population is finite and the statistics and E_0 stay finite."""
    P = lib_or_skip()
    s = W.water_methane()
    x = W.initial_walkers(s, 32, seed=4)
    lr = P.Lrdmc(s, x, 0.2, seed=2, precision=precision)
    bad, good = _bad_walkers(s, x)
    lr.set_walkers(bad)
    lr.propagate(P.LOAD_BALANCED, n_proj=5)
    g = lr.get_walkers()
    assert np.all(g["status"][~good] & (ST_NONFINITE | ST_SINGULAR | ST_STUCK | 1))
    assert np.all(g["w"][~good] == 0.0)
    assert np.all(np.isfinite(g["w"][good])) and np.all(np.isfinite(g["x"][good]))
    lr.branch()
    h = lr.history()
    assert np.isfinite(h["wbar"][-1]) and np.isfinite(h["ebar"][-1]) and np.isfinite(lr.e0)
    after = lr.get_walkers()
    assert np.all(np.isfinite(after["x"])) and np.all(after["w"] == 1.0)
    lr.propagate(P.LOAD_BALANCED, n_proj=5)
    lr.branch()
    assert np.isfinite(lr.history()["ebar"][-1])
    lr.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_weights_make_branching_refuse(precision):
    """Conventional schedule: exp(-tau e_L) of a broken walker is not finite,
    the walker is flagged and the branching refuses the population
    (LRDMC_ERR_NONFINITE) and leaves it unchanged; the handle stays usable."""
    P = lib_or_skip()
    s = W.water_methane()
    x = W.initial_walkers(s, 32, seed=4)
    lr = P.Lrdmc(s, x, 0.2, seed=2, precision=precision)
    bad, good = _bad_walkers(s, x)
    lr.set_walkers(bad)
    lr.propagate(P.CONVENTIONAL, tau=0.005, max_moves=500)
    g = lr.get_walkers()
    assert np.all(g["status"][~good] & (ST_NONFINITE | ST_SINGULAR | ST_STUCK))
    assert not np.all(np.isfinite(g["w"]))
    with pytest.raises(P.LrdmcError) as e:
        lr.branch()
    assert e.value.status == 3                                            # LRDMC_ERR_NONFINITE
    after = lr.get_walkers()
    np.testing.assert_array_equal(after["x"], g["x"])                     # population unchanged
    np.testing.assert_array_equal(after["w"], g["w"])
    # the handle stays usable: clean walkers run and branch again
    lr.set_walkers(x)
    lr.clear_status()
    lr.propagate(P.CONVENTIONAL, tau=0.005, max_moves=500)
    lr.branch()
    assert np.all((lr.get_walkers()["status"] & ~np.uint32(32)) == 0)   # 32: a drift re-inversion, not a failure
    lr.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_reruns_are_bit_identical(precision):
    """Same inputs, two handles: positions, weights, energies, ratios, status,
    move counts and the branching history agree bit for bit after load-balanced
    and conventional intervals with branching (fixed-order reductions, integer
    comb, counter-keyed random numbers; the dynamic walker-to-warp assignment
    changes nothing)."""
    P = lib_or_skip()
    s = W.water_methane()
    x = W.initial_walkers(s, 700, seed=6)
    runs = []
    for _ in range(2):
        lr = P.Lrdmc(s, x, 0.2, seed=9, reinv_period=7, precision=precision)
        for _ in range(3):
            lr.propagate(P.LOAD_BALANCED, n_proj=10)
            lr.branch()
        for _ in range(2):
            lr.propagate(P.CONVENTIONAL, tau=0.008, max_moves=500)
            lr.branch()
        runs.append((lr.get_walkers(), lr.history(), lr.energy()))
        lr.close()
    (ga, ha, ea), (gb, hb, eb) = runs
    for k in ga:
        np.testing.assert_array_equal(ga[k], gb[k])
    for k in ha:
        np.testing.assert_array_equal(ha[k], hb[k])
    assert ea[0] == eb[0]
