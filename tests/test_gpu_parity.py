"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Per-configuration ratios, b_bar, V_sf, W and e_L agree to 1e-10 (scaled by
max(1, |value|)); node counts, walker positions after hops and reconfiguration
indices agree exactly."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import assert_close, lib_or_skip
from oracle import hamiltonian as H
from oracle import lrdmc as OL
from oracle import philox as OP

pytestmark = pytest.mark.gpu


def _mk(P, sys_, n_w, a=0.2, seed=1, **kw):
    x0 = W.initial_walkers(sys_, n_w, seed=seed + 10)
    return P.Lrdmc(sys_, x0, a, seed=seed, **kw), x0


# h24: a system large enough that its geometry caches live in global memory
CASES = [("h_sto", W.hydrogen_atom_sto, 70), ("h2", W.h2_sto3g, 300), ("wm", W.water_methane, 37),
         ("h6", lambda: W.hydrogen_chain(6, spacing=1.6, mo_seed=3), 45),
         ("h24", lambda: W.hydrogen_cluster(24, seed=5), 16),
         ("h64", lambda: W.hydrogen_cluster(64, seed=6), 3)]


@pytest.mark.parametrize("name,sysf,n", CASES)
@pytest.mark.parametrize("node_rule", [0, 1, 2, -1])
def test_eval_configs_matches_oracle(name, sysf, n, node_rule):
    import torch
    P = lib_or_skip()
    s = sysf()
    lr, _ = _mk(P, s, n, node_rule=node_rule)
    x = W.initial_walkers(s, n, seed=77)
    ratios, ev, nn = lr.eval_configs(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ref = H.evaluate(s, x, 0.2, node_rule=node_rule)
    assert_close(ratios.cpu().numpy(), ref["ratios"], what="ratios")
    assert_close(ev[:, 0].cpu().numpy(), ref["bbar"], what="bbar")
    assert_close(ev[:, 1].cpu().numpy(), ref["vsf"], what="vsf")
    assert_close(ev[:, 2].cpu().numpy(), ref["W"], what="W")
    assert_close(ev[:, 3].cpu().numpy(), ref["eL"], what="eL")
    np.testing.assert_array_equal(nn.cpu().numpy(), ref["n_node"])


def test_initial_walkers_are_evaluated():
    P = lib_or_skip()
    s = W.water_methane()
    lr, x0 = _mk(P, s, 50)
    g = lr.get_walkers()
    np.testing.assert_array_equal(g["x"], x0)
    ref = H.evaluate(s, x0, 0.2)
    assert_close(g["ratios"], ref["ratios"], what="ratios")
    assert_close(g["ev"][:, 3], ref["eL"], what="eL")
    assert abs(lr.e0 - np.mean(ref["eL"])) <= 1e-10 * max(1, abs(lr.e0))
    assert np.all(g["w"] == 1.0) and np.all(g["status"] == 0)


def _oracle_walkers(s, g, a=0.2):
    Wk = OL.init_walkers(s, g["x"], a)
    return Wk


@pytest.mark.parametrize("name,sysf,n_w", [("h2", W.h2_sto3g, 77), ("wm", W.water_methane, 40),
                                           ("h24", lambda: W.hydrogen_cluster(24, seed=5), 12)])
def test_load_balanced_interval_matches_oracle(name, sysf, n_w):
    P = lib_or_skip()
    s = sysf()
    lr, x0 = _mk(P, s, n_w, reinv_period=7)
    E0 = lr.e0
    Wk = OL.init_walkers(s, x0, 0.2)
    n_proj = 9
    lr.propagate(P.LOAD_BALANCED, n_proj=n_proj)
    g = lr.get_walkers()
    OL.propagate_lb(s, Wk, 0.2, E0, n_proj, seed=1, interval=0)
    np.testing.assert_array_equal(g["x"], Wk.x)            # same hops, same float updates
    np.testing.assert_array_equal(g["moves"], Wk.moves)
    assert_close(g["w"], Wk.w, what="w")
    assert_close(g["ev"][:, 3], Wk.ev["eL"], what="eL")
    assert_close(g["ev"][:, 2], Wk.ev["W"], what="W")
    assert_close(g["ratios"], Wk.ev["ratios"], what="ratios")
    # the drift-check bit (32) marks an early re-inversion, an implementation
    # event with no counterpart in the oracle (which inverts afresh every step)
    np.testing.assert_array_equal(g["status"] & ~np.uint32(32), Wk.status)


@pytest.mark.parametrize("name,sysf,n_w,tau", [("h2", W.h2_sto3g, 77, 0.06), ("wm", W.water_methane, 33, 0.006)])
def test_conventional_interval_matches_oracle(name, sysf, n_w, tau):
    P = lib_or_skip()
    s = sysf()
    lr, x0 = _mk(P, s, n_w)
    Wk = OL.init_walkers(s, x0, 0.2)
    lr.propagate(P.CONVENTIONAL, tau=tau, max_moves=1000)
    g = lr.get_walkers()
    OL.propagate_conventional(s, Wk, 0.2, tau, seed=1, interval=0, max_moves=1000)
    assert Wk.moves.max() > 2 and Wk.moves.min() < Wk.moves.max()   # a genuinely uneven interval
    np.testing.assert_array_equal(g["moves"], Wk.moves)
    np.testing.assert_array_equal(g["x"], Wk.x)
    assert_close(g["w"], Wk.w, what="w")
    assert_close(g["ev"][:, 3], Wk.ev["eL"], what="eL")


def test_conventional_step_cap_and_zero_projection():
    P = lib_or_skip()
    s = W.h2_sto3g()
    lr, x0 = _mk(P, s, 20)
    lr.propagate(P.CONVENTIONAL, tau=10.0, max_moves=3)
    g = lr.get_walkers()
    assert np.all(g["moves"] == 3) and np.all(g["status"] & 4)
    Wk = OL.init_walkers(s, x0, 0.2)
    OL.propagate_conventional(s, Wk, 0.2, 10.0, seed=1, interval=0, max_moves=3)
    np.testing.assert_array_equal(g["x"], Wk.x)
    # the drift-check bit (32) marks an early re-inversion, an implementation
    # event with no counterpart in the oracle (which inverts afresh every step)
    np.testing.assert_array_equal(g["status"] & ~np.uint32(32), Wk.status)
    lr.clear_status()
    lr.propagate(P.LOAD_BALANCED, n_proj=0)
    g2 = lr.get_walkers()
    assert np.all(g2["w"] == 1.0) and np.all(g2["moves"] == 0) and np.all(g2["status"] == 0)
    np.testing.assert_array_equal(g2["x"], g["x"])


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1025, 4096, 51200])
def test_reconfigure_indices_bit_exact(n):
    import torch
    P = lib_or_skip()
    rng = np.random.default_rng(n)
    for trial in range(3):
        w = rng.lognormal(0.0, 1.0, n)
        if trial == 1:
            w[rng.random(n) < 0.3] = 0.0
            w[0] = max(w[0], 1e-3)
        if trial == 2:
            w = np.full(n, 0.37)
        xi = int(rng.integers(0, 2**32))
        src, st = P.reconfigure_indices(torch.tensor(w, device="cuda"), xi)
        ref = OL.reconfigure_indices(w, xi)
        np.testing.assert_array_equal(src.cpu().numpy(), ref)
        stc = st.cpu().numpy()
        assert stc[0] == 0 and stc[1] == len(np.unique(ref))


def test_reconfigure_rejects_invalid_weights():
    import torch
    P = lib_or_skip()
    for w in (np.zeros(10), np.array([1.0, np.nan, 2.0]), np.array([1.0, -0.5]), np.array([np.inf, 1.0])):
        src, st = P.reconfigure_indices(torch.tensor(w, device="cuda"), 5)
        assert st.cpu().numpy()[0] == 1


# 1283 walkers: the grid-wide partial sums run in six CTAs, the last one ragged
@pytest.mark.parametrize("n_w", [129, 1283])
@pytest.mark.parametrize("kind", [1, 0])
def test_branch_matches_oracle(kind, n_w):
    P = lib_or_skip()
    s = W.h2_sto3g()
    lr, x0 = _mk(P, s, n_w)
    E0 = lr.e0
    if kind == 1:
        lr.propagate(P.LOAD_BALANCED, n_proj=12)
    else:
        lr.propagate(P.CONVENTIONAL, tau=0.08, max_moves=1000)
    g = lr.get_walkers()
    lr.branch()
    g2 = lr.get_walkers()
    h = lr.history()
    # oracle statistics and comb on the GPU's own pre-branch weights
    Wk = OL.init_walkers(s, g["x"], 0.2)
    Wk.w = g["w"].copy()
    wbar, ebar = OL.branch_stats(Wk, E0, kind)
    assert_close(h["wbar"], [wbar], what="wbar")
    assert_close(h["ebar"], [ebar], what="ebar")
    src = OL.reconfigure_indices(g["w"], OP.branch_offset32(1, 0))
    np.testing.assert_array_equal(g2["x"], g["x"][OL.slot_assignment(src)])
    assert np.all(g2["w"] == 1.0)
    assert h["survivors"][0] == len(np.unique(src))
    if kind == 1:
        assert lr.e0 == pytest.approx(ebar, rel=1e-12)      # E_0 <- estimator over one branching
    else:
        assert lr.e0 == E0


def test_negative_diagonal_is_flagged_and_refused():
    P = lib_or_skip()
    s = W.h2_sto3g()
    lr, _ = _mk(P, s, 16)
    lr.e0 = 1e6                    # W - E_0 < 0 everywhere: every step weight is 0
    lr.propagate(P.LOAD_BALANCED, n_proj=2)
    g = lr.get_walkers()
    assert np.all(g["status"] & 1) and np.all(g["w"] == 0.0)
    with pytest.raises(P.LrdmcError) as e:
        lr.branch()
    assert e.value.status == 3
    np.testing.assert_array_equal(lr.get_walkers()["x"], g["x"])   # population unchanged


def test_sherman_morrison_against_fresh_inversion():
    """After many hops with Sherman-Morrison only, the ratios equal the ones
    from a from-scratch inversion at the same configurations."""
    import torch
    P = lib_or_skip()
    s = W.water_methane()
    lr, _ = _mk(P, s, 24, reinv_period=10**6)
    for _ in range(5):
        lr.propagate(P.LOAD_BALANCED, n_proj=20)
    g = lr.get_walkers()
    ratios, ev, _ = lr.eval_configs(torch.tensor(g["x"], device="cuda"))
    assert_close(g["ratios"], ratios.cpu().numpy(), rtol=1e-9, what="ratios after 100 SM updates")
    assert_close(g["ev"][:, 3], ev[:, 3].cpu().numpy(), rtol=1e-9, what="eL after 100 SM updates")


@pytest.mark.parametrize("kind", [1, 0])
def test_exact_hydrogen_run_on_gpu(kind):
    P = lib_or_skip()
    s = W.hydrogen_atom_sto(1.0)
    lr, _ = _mk(P, s, 64)
    for _ in range(6):
        lr.propagate(kind, n_proj=10, tau=0.07, max_moves=1000)
        lr.branch()
    E, err = lr.energy()
    assert abs(E + 0.5) < 1e-12
    h = lr.history()
    np.testing.assert_allclose(h["ebar"], -0.5, atol=1e-12)


@pytest.mark.parametrize("kind", [1, 0])
def test_short_run_reproduces_oracle_run(kind):
    """Same seeds, same inputs: the GPU run follows the oracle run hop for hop,
    so the branching histories agree to rounding."""
    P = lib_or_skip()
    s = W.h2_sto3g()
    n_w, nb = 64, 6
    lr, x0 = _mk(P, s, n_w, p_gbar=3)
    for _ in range(nb):
        lr.propagate(kind, n_proj=8, tau=0.05, max_moves=1000)
        lr.branch()
    h = lr.history()
    ho, Wk = OL.run(s, x0, 0.2, kind, nb, seed=1, n_proj=8, tau=0.05, p_gbar=3, E0=h["e0"][0])
    assert_close(h["wbar"], ho.wbar, rtol=1e-9, what="wbar")
    assert_close(h["ebar"], ho.ebar, rtol=1e-9, what="ebar")
    np.testing.assert_array_equal(lr.get_walkers()["x"], Wk.x)
    E, _ = lr.energy()
    assert abs(E - ho.energy) <= 1e-9 * max(1, abs(E))


def test_full_size_sampled_walkers():
    """At the benchmark size (water-methane, 4096 walkers, 20-hop interval, the
    launch configuration bench.py times) sampled walkers replayed by the oracle
    with their own Philox slots reproduce the GPU's positions, weights and
    local energies."""
    P = lib_or_skip()
    s = W.water_methane()
    n_w = 4096
    lr, x0 = _mk(P, s, n_w)
    E0 = lr.e0
    lr.propagate(P.LOAD_BALANCED, n_proj=20)
    g = lr.get_walkers()
    ids = np.array([0, 1, 31, 32, 1000, 2047, 3001, 4095])
    Wk = OL.init_walkers(s, x0[ids], 0.2)
    OL.propagate_lb(s, Wk, 0.2, E0, 20, seed=1, interval=0, walker_ids=ids)
    np.testing.assert_array_equal(g["x"][ids], Wk.x)
    assert_close(g["w"][ids], Wk.w, what="w")
    assert_close(g["ev"][ids, 3], Wk.ev["eL"], what="eL")
    # properties that hold for every walker
    assert np.all(g["moves"] == 20)
    hop = np.abs(g["x"] - x0) / 0.2
    assert np.all(np.abs(hop - np.round(hop)) < 1e-9)       # walkers stay on their lattices


def test_largest_size_sampled_walkers():
    """At the largest benchmarked size (water-methane, 51,200 walkers: more than
    twelve waves of resident warps, walkers handed out by the work counter,
    re-inversion every 100 hops as bench.py runs it) sampled walkers of a
    second interval, after a branching, replayed by the oracle from the GPU's
    own post-branching positions reproduce positions, weights and energies."""
    P = lib_or_skip()
    s = W.water_methane()
    n_w = 51200
    lr, x0 = _mk(P, s, n_w, reinv_period=100)
    lr.propagate(P.LOAD_BALANCED, n_proj=20)
    lr.branch()
    g0 = lr.get_walkers()
    E0 = lr.e0
    lr.propagate(P.LOAD_BALANCED, n_proj=20)
    g = lr.get_walkers()
    ids = np.array([0, 4143, 4144, 20000, 25600, 40961, 51198, 51199])
    Wk = OL.init_walkers(s, g0["x"][ids], 0.2)
    OL.propagate_lb(s, Wk, 0.2, E0, 20, seed=1, interval=1, walker_ids=ids)
    np.testing.assert_array_equal(g["x"][ids], Wk.x)
    assert_close(g["w"][ids], Wk.w, what="w")
    assert_close(g["ev"][ids, 3], Wk.ev["eL"], what="eL")
    assert np.all(g["moves"] == 20)
    lr.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bit_identical(tmp_path, precision):
    P = lib_or_skip()
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, 64, seed=5)
    a = P.Lrdmc(s, x0, 0.2, seed=3, precision=precision)
    for _ in range(3):
        a.propagate(P.LOAD_BALANCED, n_proj=6)
        a.branch()
    path = str(tmp_path / "ck.bin")
    a.save(path)
    for _ in range(3):
        a.propagate(P.CONVENTIONAL, tau=0.05, max_moves=500)
        a.branch()
    b = P.Lrdmc(s, W.initial_walkers(s, 64, seed=99), 0.2, seed=3, precision=precision)
    b.load(path)
    for _ in range(3):
        b.propagate(P.CONVENTIONAL, tau=0.05, max_moves=500)
        b.branch()
    ga, gb = a.get_walkers(), b.get_walkers()
    for k in ("x", "w", "ev", "ratios", "status", "moves"):
        np.testing.assert_array_equal(ga[k], gb[k])
    ha, hb = a.history(), b.history()
    for k in ha:
        np.testing.assert_array_equal(ha[k], hb[k])
    assert a.energy() == b.energy() or (np.isnan(a.energy()[1]) and a.energy()[0] == b.energy()[0])
    with pytest.raises(P.LrdmcError):
        c = P.Lrdmc(W.water_methane(), W.initial_walkers(W.water_methane(), 64), 0.2)
        c.load(path)


def test_checkpoint_refuses_another_hamiltonian(tmp_path):
    """A checkpoint's cached ratios, W and e_L belong to one lattice
    Hamiltonian: loading it into a handle of another a, node rule, trial
    function or system of the same shape is refused, as is a file whose
    history length disagrees with its size; the refused handle keeps its own
    walkers."""
    P = lib_or_skip()
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, 64, seed=5)
    a = P.Lrdmc(s, x0, 0.2, seed=3)
    a.propagate(P.LOAD_BALANCED, n_proj=6)
    a.branch()
    path = str(tmp_path / "ck.bin")
    a.save(path)
    x1 = W.initial_walkers(s, 64, seed=99)
    s2 = W.h2_sto3g()
    s2.j2_anti = 0.6                  # another pair Jastrow: same shape, other wavefunction
    s3 = W.h2_sto3g()
    s3.R = s3.R * 1.01                # another geometry
    for kw, sysk in ((dict(a=0.25), s), (dict(node_rule=2), s), ({}, s2), ({}, s3)):
        b = P.Lrdmc(sysk, x1, kw.get("a", 0.2), seed=3, node_rule=kw.get("node_rule", 0))
        before = b.get_walkers()["x"]
        with pytest.raises(P.LrdmcError):
            b.load(path)
        np.testing.assert_array_equal(b.get_walkers()["x"], before)
        b.close()
    # a corrupt history length (header field) is refused before it sizes anything
    raw = bytearray(open(path, "rb").read())
    import struct
    struct.pack_into("<i", raw, 8 + 4 * 4, 2 ** 30)     # n_hist
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    b = P.Lrdmc(s, x1, 0.2, seed=3)
    with pytest.raises(P.LrdmcError):
        b.load(str(bad))
    (tmp_path / "short.bin").write_bytes(bytes(raw[: len(raw) // 2]))
    with pytest.raises(P.LrdmcError):
        b.load(str(tmp_path / "short.bin"))
    b.load(path)                       # the matching file still loads
    np.testing.assert_array_equal(b.get_walkers()["x"], a.get_walkers()["x"])


@pytest.mark.parametrize("name,sysf,n_w,kind", [("h2", W.h2_sto3g, 64, 1), ("wm", W.water_methane, 32, 1),
                                                 ("wm", W.water_methane, 32, 0)])
def test_randomised_lattice_interval_matches_oracle(name, sysf, n_w, kind):
    """Randomised lattice (one rotation of the hop versors per walker and
    interval): the rotation comes from sin/cos/sqrt on both sides, so
    positions agree to rounding (1e-12) rather than bit for bit."""
    P = lib_or_skip()
    s = sysf()
    lr, x0 = _mk(P, s, n_w, reinv_period=7)
    E0 = lr.e0
    Wk = OL.init_walkers(s, x0, 0.2)
    for j in range(2):
        lr.propagate(kind, n_proj=8, tau=0.006, max_moves=1000, rotate=True)
        g = lr.get_walkers()
        # the library's interval counter advances only at branching: both calls use interval 0
        if kind == 1:
            OL.propagate_lb(s, Wk, 0.2, E0, 8, seed=1, interval=0, rotate=True)
        else:
            OL.propagate_conventional(s, Wk, 0.2, 0.006, seed=1, interval=0, max_moves=1000, rotate=True)
        np.testing.assert_array_equal(g["moves"], Wk.moves)
        np.testing.assert_allclose(g["x"], Wk.x, rtol=0, atol=1e-12)
        assert_close(g["w"], Wk.w, what="w")
        assert_close(g["ev"][:, 3], Wk.ev["eL"], rtol=1e-9, what="eL")
        assert_close(g["ratios"], Wk.ev["ratios"], rtol=1e-9, what="ratios")
        # carry the same state into the next interval (no branching in between)
        lr.set_walkers(g["x"])
        Wk = OL.init_walkers(s, g["x"], 0.2)


@pytest.mark.parametrize("kind", [1, 0])
def test_fixed_lattice_after_randomised_interval_matches_oracle(kind):
    """A fixed-lattice interval that follows a randomised one re-evaluates the
    walkers on the Cartesian axes before its first step (both sides)."""
    P = lib_or_skip()
    s = W.water_methane()
    lr, x0 = _mk(P, s, 24, reinv_period=7)
    E0 = lr.e0
    Wk = OL.init_walkers(s, x0, 0.2)
    for rotate in (True, False, False):
        lr.propagate(kind, n_proj=6, tau=0.005, max_moves=1000, rotate=rotate)
        if kind == 1:
            OL.propagate_lb(s, Wk, 0.2, E0, 6, seed=1, interval=0, rotate=rotate)
        else:
            OL.propagate_conventional(s, Wk, 0.2, 0.005, seed=1, interval=0, max_moves=1000, rotate=rotate)
        g = lr.get_walkers()
        np.testing.assert_array_equal(g["moves"], Wk.moves)
        np.testing.assert_allclose(g["x"], Wk.x, rtol=0, atol=1e-12)
        assert_close(g["w"], Wk.w, rtol=1e-9, what="w")
        assert_close(g["ev"][:, 3], Wk.ev["eL"], rtol=1e-9, what="eL")
        assert_close(g["ratios"], Wk.ev["ratios"], rtol=1e-9, what="ratios")


def test_randomised_lattice_exact_hydrogen_and_refusal_in_mixed():
    P = lib_or_skip()
    s = W.hydrogen_atom_sto(1.0)
    lr, _ = _mk(P, s, 64)
    for _ in range(4):
        lr.propagate(P.LOAD_BALANCED, n_proj=10, rotate=True)
        lr.branch()
    assert abs(lr.energy()[0] + 0.5) < 1e-12
    lm, _ = _mk(P, s, 16, precision=1)
    with pytest.raises(P.LrdmcError) as e:
        lm.propagate(P.LOAD_BALANCED, n_proj=2, rotate=True)
    assert e.value.status == 7


def test_energy_error_bar_matches_oracle_on_a_gpu_history():
    """lrdmc_energy's E and error bar against the oracle's estimator
    (oracle.estimator.energy / energy_error, Sec. II.A) fed the branching
    history the GPU run itself recorded: equal to 1e-12 relative."""
    from oracle import estimator as OE
    P = lib_or_skip()
    s = W.h2_sto3g()
    lr = P.Lrdmc(s, W.initial_walkers(s, 128, seed=8), 0.2, seed=4, p_gbar=5, n_equil=4)
    for _ in range(40):
        lr.propagate(P.LOAD_BALANCED, n_proj=10)
        lr.branch()
    h = lr.history()
    E, err = lr.energy()
    Eo = OE.energy(h["wbar"], h["ebar"], 5, 4)
    erro = OE.energy_error(h["wbar"], h["ebar"], 5, 4)
    assert np.isfinite(err) and err > 0
    assert abs(E - Eo) <= 1e-12 * max(1.0, abs(Eo))
    assert abs(err - erro) <= 1e-12 * max(1.0, abs(erro))
    lr.close()
