"""Batched multi-system propagation: one persistent launch per interval for
several systems of different sizes.  A walker's trajectory does not depend on
which warp or CTA runs it, so every system of a batch must follow the
trajectory of the same system in its own handle (which the single-system
parity tests tie to the oracle): the same hops, positions, hop counts and
status bits, and weights, energies and ratios equal up to the rounding of the
two kernels' compiled arithmetic (the same source, fused differently by the
compiler: 1e-10).  One system is also compared with the oracle directly."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_close, lib_or_skip
from oracle import lrdmc as OL

pytestmark = pytest.mark.gpu

A = 0.2


def _systems():
    return [(W.h2_sto3g(), 40, 3), (W.water_methane(), 24, 5), (W.hydrogen_cluster(16, seed=1), 32, 7),
            (W.hydrogen_cluster(24, seed=2), 20, 9), (W.hydrogen_atom_sto(0.8), 50, 11)]


def _run(obj, P, n_lb=3):
    for _ in range(n_lb):
        obj.propagate(P.LOAD_BALANCED, n_proj=6)
        obj.branch()
    obj.propagate(P.CONVENTIONAL, tau=0.01, max_moves=200)
    obj.branch()


def _same(a, b):
    ga, gb = a.get_walkers(), b.get_walkers()
    for k in ("x", "status", "moves"):
        np.testing.assert_array_equal(ga[k], gb[k], err_msg=k)
    for k in ("w", "ev", "ratios"):
        assert_close(ga[k], gb[k], what=k)
    ha, hb = a.history(), b.history()
    for k in ("moves_mean", "moves_max", "survivors", "status_or"):
        np.testing.assert_array_equal(ha[k], hb[k], err_msg=k)
    for k in ("wbar", "ebar", "e0"):
        assert_close(ha[k], hb[k], what=k)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("policy", [0, 1])
def test_batch_follows_the_single_system_trajectories(precision, policy):
    P = lib_or_skip()
    systems = _systems()
    x0s = [W.initial_walkers(s, n, seed=sd + 20) for s, n, sd in systems]
    batch = P.LrdmcBatch([s for s, _, _ in systems], x0s, A, [sd for _, _, sd in systems], reinv_period=7,
                         precision=precision)
    batch.set_order(policy)
    before = [h.get_walkers() for h in batch.handles]
    best, times = batch.tune(P.LOAD_BALANCED, n_proj=6)
    assert 1 <= best <= 4 and times[best] > 0.0
    # the tuner restores every walker it propagated
    for h, g in zip(batch.handles, before):
        after = h.get_walkers()
        for k in g:
            np.testing.assert_array_equal(after[k], g[k])
    n0 = batch.launch_count()
    _run(batch, P)
    assert batch.launch_count() - n0 == 4 * (1 + 3)   # one propagate and three branching launches per interval
    for (s, n, sd), x0, h in zip(systems, x0s, batch.handles):
        single = P.Lrdmc(s, x0, A, seed=sd, reinv_period=7, precision=precision)
        _run(single, P)
        _same(h, single)


def test_batch_system_matches_oracle():
    P = lib_or_skip()
    s = W.hydrogen_cluster(16, seed=3)
    x0 = W.initial_walkers(s, 12, seed=4)
    h2 = W.h2_sto3g()
    batch = P.LrdmcBatch([h2, s], [W.initial_walkers(h2, 30, seed=1), x0], A, [2, 1], reinv_period=7)
    h = batch.handle(1)
    E0 = h.e0
    Wk = OL.init_walkers(s, x0, A)
    batch.propagate(P.LOAD_BALANCED, n_proj=8)
    OL.propagate_lb(s, Wk, A, E0, 8, seed=1, interval=0)
    g = h.get_walkers()
    np.testing.assert_array_equal(g["moves"], Wk.moves)
    np.testing.assert_array_equal(g["x"], Wk.x)
    assert_close(g["w"], Wk.w, what="w")
    assert_close(g["ev"][:, 3], Wk.ev["eL"], what="eL")
    assert_close(g["ratios"].reshape(len(x0), -1), Wk.ev["ratios"].reshape(len(x0), -1), what="ratios")


def test_batch_timing_and_refusals():
    P = lib_or_skip()
    systems = [W.hydrogen_cluster(n, seed=n) for n in (16, 20, 28)]
    batch = P.LrdmcBatch(systems, [W.initial_walkers(s, 64, seed=1) for s in systems], 0.25, [1, 2, 3])
    batch.set_timing(True)
    batch.propagate(P.LOAD_BALANCED, n_proj=5)
    t = batch.timing()
    assert t["walkers"] == 192 and 0.0 <= t["sm_idle_fraction"] < 1.0
    assert t["walker_ms_max"] <= t["span_ms"] + 1e-9
    assert 0.0 <= t["sm_idle_tail_ms"] <= t["span_ms"] + 1e-9
    assert 0.0 < t["slot_busy_fraction"] <= 1.0 + 1e-9 and t["items"] >= 3
    with pytest.raises(P.LrdmcError) as e:
        batch.propagate(P.CONVENTIONAL, tau=-1.0)
    assert e.value.status == 1
    import ctypes
    s = P.binding._Schedule(1, 5, 0.0, 10, 1)
    assert batch.lib.lrdmc_batch_propagate(batch._b, ctypes.byref(s)) == 7


@pytest.mark.parametrize("precision", [0, 1])
def test_large_system_with_global_working_sets_follows_its_single_trajectory(precision):
    """A 96-electron cluster: its working set (about 70 KB in FP64) leaves fewer
    than four walkers per CTA at every launch shape, so the batched kernel runs
    it with the working sets in global memory, one walker per warp, next to a
    small system that shares CTAs in shared memory."""
    P = lib_or_skip()
    systems = [(W.hydrogen_cluster(96, seed=4), 10, 13), (W.h2_sto3g(), 24, 3)]
    x0s = [W.initial_walkers(s, n, seed=sd + 20) for s, n, sd in systems]
    batch = P.LrdmcBatch([s for s, _, _ in systems], x0s, A, [sd for _, _, sd in systems], reinv_period=7,
                         precision=precision)
    _run(batch, P, n_lb=2)
    for (s, n, sd), x0, h in zip(systems, x0s, batch.handles):
        single = P.Lrdmc(s, x0, A, seed=sd, reinv_period=7, precision=precision)
        _run(single, P, n_lb=2)
        _same(h, single)
