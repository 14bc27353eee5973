"""Hand-written adjoint of e_L and log|Psi_G| (nuclear coordinates and Jastrow
parameters) on the GPU: against the oracle's autograd gradients of the same
definitions, against central finite differences (h = 1e-4, one Richardson
step) of the GPU's own energies, and through the torch.autograd entry."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib_or_skip
from oracle import adjoint as AD

pytestmark = pytest.mark.gpu

CASES = [("h_sto", lambda: W.hydrogen_atom_sto(0.8), 6), ("h2", W.h2_sto3g, 6), ("wm", W.water_methane, 2),
         ("h6", lambda: W.hydrogen_cluster(6, seed=2), 3)]


def _rel(g, r):
    return float(np.max(np.abs(g - r) / np.maximum(1.0, np.abs(r))))


@pytest.mark.parametrize("name,sysf,n", CASES)
@pytest.mark.parametrize("node_rule", [0, 2])
def test_gradients_match_oracle_autograd(name, sysf, n, node_rule):
    import torch
    P = lib_or_skip()
    s = sysf()
    x = W.initial_walkers(s, n, seed=31)
    lr = P.Lrdmc(s, W.initial_walkers(s, max(n, 8), seed=1), 0.2, node_rule=node_rule)
    eL, lp, ge, gl = lr.local_energy_grad(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    e_ref, l_ref, ge_ref, gl_ref = AD.gradients(s, x, 0.2, node_rule)
    assert _rel(eL.cpu().numpy(), e_ref) < 1e-10
    assert _rel(lp.cpu().numpy(), l_ref) < 1e-10
    assert _rel(ge.cpu().numpy(), ge_ref) < 1e-8, (ge.cpu().numpy() - ge_ref)
    assert _rel(gl.cpu().numpy(), gl_ref) < 1e-10
    np.testing.assert_array_equal(lr.params(), AD.pack(s))


def test_gradients_match_finite_differences_of_the_gpu_energies():
    import torch
    P = lib_or_skip()
    s = W.water_methane()
    x = torch.tensor(W.initial_walkers(s, 2, seed=8), device="cuda")
    lr = P.Lrdmc(s, W.initial_walkers(s, 8, seed=1), 0.2)
    th0 = lr.params()
    _, _, ge, gl = lr.local_energy_grad(x)
    ge, gl = ge.cpu().numpy(), gl.cpu().numpy()
    nn = s.n_nuc

    def energies(th):
        lr.set_params(th)
        e, l, _, _ = lr.local_energy_grad(x)
        torch.cuda.synchronize()
        return e.cpu().numpy(), l.cpu().numpy()

    for k in (0, 4, 3 * nn - 1, 3 * nn, 3 * nn + 1, 3 * nn + 2, 3 * nn + 3, 4 * nn + 4):
        fd = {}
        for h in (1e-4, 5e-5):
            tp, tm = th0.copy(), th0.copy()
            tp[k] += h
            tm[k] -= h
            ep, lp_ = energies(tp)
            em, lm = energies(tm)
            fd[h] = ((ep - em) / (2 * h), (lp_ - lm) / (2 * h))
        for q, g in ((0, ge[:, k]), (1, gl[:, k])):
            rich = (4 * fd[5e-5][q] - fd[1e-4][q]) / 3
            assert np.all(np.abs(rich - g) <= 1e-6 * np.maximum(1.0, np.abs(g))), (k, q, rich, g)
    lr.set_params(th0)


def test_autograd_entry_accumulates_weighted_gradients():
    import torch
    P = lib_or_skip()
    s = W.h2_sto3g()
    x = torch.tensor(W.initial_walkers(s, 5, seed=2), device="cuda")
    lr = P.Lrdmc(s, W.initial_walkers(s, 8, seed=1), 0.2)
    theta = torch.tensor(lr.params(), dtype=torch.float64, requires_grad=True)
    eL, lp = P.local_energy(lr, theta, x)
    w = torch.linspace(0.5, 1.5, 5, dtype=torch.float64, device="cuda")
    (g,) = torch.autograd.grad((w * eL).sum() + (2.0 * lp).sum(), theta)
    _, _, ge, gl = lr.local_energy_grad(x)
    ref = (w[:, None] * ge).sum(0) + 2.0 * gl.sum(0)
    np.testing.assert_allclose(g.numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-12)
    # moving the parameters through the entry point re-evaluates at the new ones
    th2 = theta.detach().clone()
    th2[2] += 0.05
    e2, _ = P.local_energy(lr, th2, x)
    assert not torch.allclose(e2, eL)
    np.testing.assert_array_equal(lr.params(), th2.numpy())


def test_large_system_and_more_configurations_than_walkers():
    """24 electrons (geometry caches and, for the gradient kernel, the whole
    working set in global memory) against the oracle, with more configurations
    than the handle has walkers."""
    import torch
    P = lib_or_skip()
    s = W.hydrogen_cluster(24, seed=5)
    x = W.initial_walkers(s, 3, seed=12)
    lr = P.Lrdmc(s, W.initial_walkers(s, 2, seed=1), 0.2)
    eL, lp, ge, gl = lr.local_energy_grad(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    e_ref, l_ref, ge_ref, gl_ref = AD.gradients(s, x, 0.2, 0)
    assert _rel(eL.cpu().numpy(), e_ref) < 1e-10
    assert _rel(ge.cpu().numpy(), ge_ref) < 1e-8
    assert _rel(gl.cpu().numpy(), gl_ref) < 1e-10


def test_global_working_set_path_matches_finite_differences():
    """A 64-electron cluster: its shared-memory layout would hold fewer than 8
    working sets per SM, so the gradient kernel keeps them in global memory.
    Gradients against central differences (h = 1e-4, one Richardson step) of
    the GPU's own energies, for nuclear coordinates and Jastrow parameters."""
    import torch
    P = lib_or_skip()
    s = W.hydrogen_cluster(64, seed=6)
    x = torch.tensor(W.initial_walkers(s, 3, seed=9), device="cuda")
    lr = P.Lrdmc(s, W.initial_walkers(s, 2, seed=1), 0.2)
    th0 = lr.params()
    _, _, ge, gl = lr.local_energy_grad(x)
    ge, gl = ge.cpu().numpy(), gl.cpu().numpy()
    nn = s.n_nuc

    def energies(th):
        lr.set_params(th)
        e, l, _, _ = lr.local_energy_grad(x)
        torch.cuda.synchronize()
        return e.cpu().numpy(), l.cpu().numpy()

    for k in (0, 3 * nn - 2, 3 * nn, 3 * nn + 2, 3 * nn + 3 + nn // 2, 4 * nn + 3 + nn - 1):
        fd = {}
        for h in (1e-4, 5e-5):
            tp, tm = th0.copy(), th0.copy()
            tp[k] += h
            tm[k] -= h
            ep, lp_ = energies(tp)
            em, lm = energies(tm)
            fd[h] = ((ep - em) / (2 * h), (lp_ - lm) / (2 * h))
        for q, g in ((0, ge[:, k]), (1, gl[:, k])):
            rich = (4 * fd[5e-5][q] - fd[1e-4][q]) / 3
            assert np.all(np.abs(rich - g) <= 1e-6 * np.maximum(1.0, np.abs(g))), (k, q, rich, g)
    lr.set_params(th0)


def test_h128_chain_gradients_match_finite_differences():
    """The adjoint's own workload: the linear H128 chain (spacing 1.8 bohr,
    64 up / 64 down electrons, s + p Gaussians per atom, seeded MOs, a = 0.25).
    Gradients of e_L and log|Psi_G| at two configurations against central
    differences (h = 1e-4 and 5e-5, one Richardson step) of the GPU's own
    energies, for the first, a middle and the last nuclear coordinate and
    every Jastrow kind (c_anti, c_par, b, one A_I, one B_I)."""
    import torch
    P = lib_or_skip()
    s = W.hydrogen_chain(128)
    x = torch.tensor(W.initial_walkers(s, 2, seed=9), device="cuda")
    lr = P.Lrdmc(s, W.initial_walkers(s, 2, seed=1), 0.25)
    th0 = lr.params()
    _, _, ge, gl = lr.local_energy_grad(x)
    ge, gl = ge.cpu().numpy(), gl.cpu().numpy()
    assert np.all(np.isfinite(ge)) and np.all(np.isfinite(gl))
    nn = s.n_nuc

    def energies(th):
        lr.set_params(th)
        e, l, _, _ = lr.local_energy_grad(x)
        torch.cuda.synchronize()
        return e.cpu().numpy(), l.cpu().numpy()

    for k in (0, 3 * (nn // 2) + 2, 3 * nn - 1, 3 * nn, 3 * nn + 1, 3 * nn + 2, 3 * nn + 3, 4 * nn + 3 + nn - 1):
        fd = {}
        for h in (1e-4, 5e-5):
            tp, tm = th0.copy(), th0.copy()
            tp[k] += h
            tm[k] -= h
            ep, lp_ = energies(tp)
            em, lm = energies(tm)
            fd[h] = ((ep - em) / (2 * h), (lp_ - lm) / (2 * h))
        for q, g in ((0, ge[:, k]), (1, gl[:, k])):
            rich = (4 * fd[5e-5][q] - fd[1e-4][q]) / 3
            assert np.all(np.abs(rich - g) <= 1e-6 * np.maximum(1.0, np.abs(g))), (k, q, rich, g)
    lr.set_params(th0)


def test_h16_chain_gradients_match_oracle_autograd():
    """A 16-atom chain of the same construction (a = 0.25): every gradient
    component against the oracle's autograd gradients of the same definitions
    (fresh determinants for every hop), at two configurations."""
    import torch
    P = lib_or_skip()
    s = W.hydrogen_chain(16)
    x = W.initial_walkers(s, 2, seed=31)
    lr = P.Lrdmc(s, W.initial_walkers(s, 8, seed=1), 0.25)
    eL, lp, ge, gl = lr.local_energy_grad(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    e_ref, l_ref, ge_ref, gl_ref = AD.gradients(s, x, 0.25, 0)
    assert _rel(eL.cpu().numpy(), e_ref) < 1e-10
    assert _rel(lp.cpu().numpy(), l_ref) < 1e-10
    assert _rel(ge.cpu().numpy(), ge_ref) < 1e-8
    assert _rel(gl.cpu().numpy(), gl_ref) < 1e-10
