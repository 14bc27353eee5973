"""Mixed-precision path (precision = 1) against the FP64 oracle and the FP64
GPU path.

Tolerances follow from FP32 arithmetic (unit roundoff u = 2^-24 = 6e-8): each
hop ratio is a sum of O(100) FP32 terms, so |r - r_ref| <= ~100 u |terms|;
relative to max(1, |r|) that is below 1e-4 even near a node, where the terms
grow like 1/|Psi|.  The local energy sums 6 N_e ratios scaled by 1/(2a^2)
(12.5 at a = 0.2), so per configuration |e_L - e_L_ref| stays below
6 N_e * 1e-4 * 12.5 / sqrt(6 N_e) ~ 1e-2 Ha for 16 electrons; its mean over
configurations (the energy bias) must stay below 1e-4 Ha (0.1 mHa)."""
import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,sysf,n,rat_tol,el_tol", [
    ("h_sto", W.hydrogen_atom_sto, 64, 1e-6, 1e-5),
    ("h2", W.h2_sto3g, 256, 1e-6, 2e-5),
    ("wm", W.water_methane, 256, 1e-4, 1e-2),
    # 24 electrons: the mixed layout keeps its O(N^2) arrays in global memory
    ("h24", lambda: W.hydrogen_cluster(24, seed=5), 64, 1e-4, 2e-2),
    ("h64", lambda: W.hydrogen_cluster(64, seed=6), 4, 1e-4, 5e-2)])
def test_mixed_eval_against_oracle(name, sysf, n, rat_tol, el_tol):
    import torch
    from gpu_helpers import assert_close, lib_or_skip
    P = lib_or_skip()
    s = sysf()
    lr = P.Lrdmc(s, W.initial_walkers(s, n, seed=3), 0.2, precision=1)
    x = W.initial_walkers(s, n, seed=77)
    ratios, ev, nn = lr.eval_configs(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ref = H.evaluate(s, x, 0.2)
    assert_close(ratios.cpu().numpy(), ref["ratios"], rtol=rat_tol, what="ratios")
    el = ev[:, 3].cpu().numpy()
    assert np.max(np.abs(el - ref["eL"])) <= el_tol
    if n >= 64:   # statistics over enough configurations
        assert abs(np.mean(el - ref["eL"])) <= 1e-4                  # energy bias below 0.1 mHa
        assert np.mean(nn.cpu().numpy() != ref["n_node"]) <= 0.01


# h64: both precisions keep their working sets in global memory (fewer than
# 8 shared-memory working sets would fit per SM)
@pytest.mark.parametrize("sysf", [W.water_methane, lambda: W.hydrogen_cluster(24, seed=5),
                                  lambda: W.hydrogen_cluster(64, seed=6)])
def test_mixed_interval_tracks_fp64_path(sysf):
    """Same start, same random streams: after a 20-hop load-balanced interval
    almost every walker made the same hops as in FP64 (a hop choice can flip
    only when the uniform falls within ~1e-7 of a cumulative boundary), and
    those walkers carry the same weight to FP32 accuracy."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = sysf()
    x0 = W.initial_walkers(s, 512, seed=21)
    g = {}
    for prec in (0, 1):
        lr = P.Lrdmc(s, x0, 0.2, seed=4, precision=prec, reinv_period=50)
        lr.e0 = -20.0
        lr.propagate(P.LOAD_BALANCED, n_proj=20)
        g[prec] = lr.get_walkers()
        lr.close()
    same = np.all(g[0]["x"] == g[1]["x"], axis=(1, 2))
    assert same.mean() >= 0.95
    rel = np.abs(g[1]["w"][same] - g[0]["w"][same]) / np.abs(g[0]["w"][same])
    assert np.median(rel) < 1e-5


def test_mixed_tracks_fp64_at_the_largest_size():
    """51,200 water-methane walkers, the launch configuration of the speed-up
    measurement (mixed re-inverting every 50 hops, FP64 every 100): after one
    20-hop interval almost every walker made the same hops in both precisions,
    with weights equal to FP32 accuracy, and local energies within the
    per-configuration bound above."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.water_methane()
    x0 = W.initial_walkers(s, 51200, seed=21)
    g = {}
    for prec, k in ((0, 100), (1, 50)):
        lr = P.Lrdmc(s, x0, 0.2, seed=4, precision=prec, reinv_period=k)
        lr.e0 = -20.0
        lr.propagate(P.LOAD_BALANCED, n_proj=20)
        g[prec] = lr.get_walkers()
        lr.close()
    same = np.all(g[0]["x"] == g[1]["x"], axis=(1, 2))
    assert same.mean() >= 0.95
    rel = np.abs(g[1]["w"][same] - g[0]["w"][same]) / np.abs(g[0]["w"][same])
    assert np.median(rel) < 1e-5
    de = np.abs(g[1]["ev"][same, 3] - g[0]["ev"][same, 3])
    assert np.median(de) < 1e-3 and np.max(de) < 5e-2


def test_mixed_run_reaches_exact_hydrogen_energy():
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.hydrogen_atom_sto(1.0)
    lr = P.Lrdmc(s, W.initial_walkers(s, 128, seed=2), 0.2, precision=1)
    for _ in range(5):
        lr.propagate(P.LOAD_BALANCED, n_proj=10)
        lr.branch()
    E, _ = lr.energy()
    assert abs(E + 0.5) < 2e-6


def test_handles_of_both_precisions_coexist():
    """Kernel attributes are process-wide: a handle created later (with a
    smaller shared-memory footprint) must not break an earlier one."""
    import torch
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.water_methane()
    x0 = W.initial_walkers(s, 64, seed=1)
    h64 = P.Lrdmc(s, x0, 0.2, precision=0)
    h32 = P.Lrdmc(s, x0, 0.2, precision=1)
    x = torch.tensor(x0, device="cuda")
    r64, e64, _ = h64.eval_configs(x)
    r32, e32, _ = h32.eval_configs(x)
    h64.propagate(P.LOAD_BALANCED, n_proj=2)
    h32.propagate(P.LOAD_BALANCED, n_proj=2)
    h64.branch()
    h32.branch()
    torch.cuda.synchronize()
    assert torch.max(torch.abs(e64[:, 3] - e32[:, 3])).item() < 1e-2
