"""Pins of the oracle's gradients of e_L and log|Psi_G| (nuclear coordinates
and Jastrow parameters): the PyTorch restatement reproduces the numpy oracle's
values; its autograd gradients agree with central finite differences of the
numpy oracle; the exact hydrogen wavefunction gives a local energy independent
of the proton position; translating nuclei and electrons together leaves e_L
unchanged; closed forms for log|Psi_G|."""
import dataclasses

import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as AD
from oracle import hamiltonian as H
from oracle import wavefunction as WF


def _perturbed(sys, theta):
    R, ca, cp, b, A, B = AD.unpack(sys, theta)
    return dataclasses.replace(sys, R=np.array(R).reshape(-1, 3), j2_anti=float(ca), j2_par=float(cp),
                               j2_b=float(b), j1_A=np.array(A), j1_B=np.array(B))


def _wm_small():
    s = W.water_methane()
    return s


@pytest.mark.parametrize("sysf,n", [(W.h2_sto3g, 3), (_wm_small, 2), (lambda: W.hydrogen_cluster(6, seed=2), 2)])
def test_torch_restatement_matches_numpy_oracle(sysf, n):
    s = sysf()
    x = W.initial_walkers(s, n, seed=9)
    th = torch.tensor(AD.pack(s), dtype=torch.float64)
    ref = H.evaluate(s, x, 0.2)
    _, lref = WF.log_psi(s, x)
    for k in range(n):
        xk = torch.tensor(x[k])
        e = float(AD.local_energy(s, th, xk, 0.2))
        _, lp = AD.log_psi(s, th, xk)
        assert abs(e - ref["eL"][k]) <= 1e-10 * max(1.0, abs(e))
        assert abs(float(lp) - lref[k]) <= 1e-12 * max(1.0, abs(lref[k]))


def test_gradients_match_central_differences_of_the_numpy_oracle():
    """h = 1e-4 central differences with one Richardson step (error O(h^4))."""
    s = W.water_methane()
    x = W.initial_walkers(s, 1, seed=4)
    e, lp, ge, gl = AD.gradients(s, x, 0.2)
    th = AD.pack(s)
    rng = np.random.default_rng(1)
    nn = s.n_nuc
    idx = list(rng.choice(3 * nn, 5, replace=False)) + [3 * nn, 3 * nn + 1, 3 * nn + 2,
                                                         3 * nn + 3 + 2, 4 * nn + 3 + 5]

    def fd(f, k, h):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        return (f(_perturbed(s, tp)) - f(_perturbed(s, tm))) / (2 * h)

    fe = lambda sy: H.evaluate(sy, x, 0.2)["eL"][0]
    fl = lambda sy: WF.log_psi(sy, x)[1][0]
    for k in idx:
        for f, g in ((fe, ge[0, k]), (fl, gl[0, k])):
            d1, d2 = fd(f, k, 1e-4), fd(f, k, 5e-5)
            rich = (4 * d2 - d1) / 3
            assert abs(rich - g) <= 1e-6 * max(1.0, abs(g)), (k, rich, g)


def test_exact_hydrogen_energy_does_not_depend_on_the_proton():
    s = W.hydrogen_atom_sto(1.0)
    x = W.initial_walkers(s, 3, seed=2)
    e, lp, ge, gl = AD.gradients(s, x, 0.2)
    np.testing.assert_allclose(e, -0.5, atol=1e-12)
    np.testing.assert_allclose(ge[:, :3], 0.0, atol=1e-10)
    # d log|Psi| / d R = zeta (x - R) / |x - R| for exp(-zeta |x - R|)
    d = x[:, 0, :] - s.R[0]
    np.testing.assert_allclose(gl[:, :3], d / np.linalg.norm(d, axis=1)[:, None], atol=1e-12)


@pytest.mark.parametrize("sysf", [W.h2_sto3g, W.water_methane])
def test_translation_of_nuclei_and_electrons_leaves_e_L_unchanged(sysf):
    s = sysf()
    x = torch.tensor(W.initial_walkers(s, 1, seed=6)[0], requires_grad=True)
    th = torch.tensor(AD.pack(s), dtype=torch.float64, requires_grad=True)
    e = AD.local_energy(s, th, x, 0.2)
    gt, gx = torch.autograd.grad(e, (th, x))
    gR = gt[:3 * s.n_nuc].reshape(-1, 3).sum(0) + gx.sum(0)
    assert float(gR.abs().max()) <= 1e-9 * max(1.0, float(gt.abs().max()))


def test_jastrow_closed_forms_of_log_psi():
    s = W.water_methane()
    x = W.initial_walkers(s, 2, seed=3)
    _, _, _, gl = AD.gradients(s, x, 0.2)
    nn, ne, b = s.n_nuc, s.n_elec, s.j2_b
    for k in range(2):
        da = dp = db = 0.0
        for i in range(ne):
            for j in range(i + 1, ne):
                r = np.linalg.norm(x[k, i] - x[k, j])
                c = s.j2_par if (i < s.n_up) == (j < s.n_up) else s.j2_anti
                if (i < s.n_up) == (j < s.n_up):
                    dp += r / (1 + b * r)
                else:
                    da += r / (1 + b * r)
                db += -c * r * r / (1 + b * r) ** 2
        assert abs(gl[k, 3 * nn] - da) < 1e-12 and abs(gl[k, 3 * nn + 1] - dp) < 1e-12
        assert abs(gl[k, 3 * nn + 2] - db) < 1e-12
        r = np.linalg.norm(x[k][:, None, :] - s.R[None], axis=-1)
        np.testing.assert_allclose(gl[k, 3 * nn + 3:4 * nn + 3], -(r / (1 + s.j1_B * r)).sum(0), atol=1e-12)
