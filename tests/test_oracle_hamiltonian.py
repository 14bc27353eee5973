"""Pins for the oracle's lattice-regularised Hamiltonian (Appendix D)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as H
from oracle import wavefunction as wf


@pytest.mark.parametrize("a", [0.05, 0.2, 0.5])
def test_exact_hydrogen_local_energy_is_constant(a):
    """Psi = exp(-r) is the exact H ground state: -lap Psi/(2 Psi) - 1/r = -1/2 at
    every point, and the lattice local energy equals the continuous one."""
    s = W.hydrogen_atom_sto(1.0)
    x = W.initial_walkers(s, 200, seed=5, sigma=1.0)
    ev = H.evaluate(s, x, a, node_rule=0)
    np.testing.assert_allclose(ev["eL"], -0.5, atol=1e-11)
    assert np.all(ev["vsf"] == 0.0) and np.all(ev["n_node"] == 0)


def test_gaussian_hydrogen_local_energy_closed_form():
    """Psi = exp(-b r^2): e_L = 3b - 2 b^2 r^2 - 1/r (continuum), which the
    lattice form reproduces at any a (Eq. for e_L^a = e_L)."""
    b = 0.37
    s = W.hydrogen_atom_gauss(b)
    x = W.initial_walkers(s, 100, seed=6, sigma=1.0)
    r = np.linalg.norm(x[:, 0], axis=-1)
    ref = 3 * b - 2 * b * b * r * r - 1.0 / r
    for a in (0.1, 0.3):
        ev = H.evaluate(s, x, a)
        np.testing.assert_allclose(ev["eL"], ref, rtol=1e-11, atol=1e-11)
        # W - b_bar = e_L and W contains the kinetic diagonal 3/a^2
        kin_a = -0.5 * (np.sum(ev["ratios"][:, 0, :], axis=-1) - 6.0) / (a * a)
        assert np.all(ev["W"] > 3.0 / (a * a) - 1.0 / r - 10.0)
        np.testing.assert_allclose(ev["W"] - ev["bbar"] - kin_a,
                                   ev["eL"] - kin_a, rtol=1e-12)


def _fd_local_energy(s, x, h=1e-4):
    """Continuum e_L from central differences of Psi (ratios of fresh log|Psi|)."""
    s0, l0 = wf.log_psi(s, x)
    lap = np.zeros(x.shape[0])
    for hh, wgt in ((2 * h, -1.0 / 3.0), (h, 4.0 / 3.0)):
        acc = np.zeros(x.shape[0])
        for i in range(s.n_elec):
            for m in range(3):
                xp, xm = x.copy(), x.copy()
                xp[:, i, m] += hh
                xm[:, i, m] -= hh
                sp, lp = wf.log_psi(s, xp)
                sm, lm = wf.log_psi(s, xm)
                acc += (sp * s0 * np.exp(lp - l0) - 2.0 + sm * s0 * np.exp(lm - l0)) / (hh * hh)
        lap += wgt * acc
    vloc = np.sum(H.nu_ei(s, x), axis=-1) + H.v_ee(x) + H.v_ii(s)
    return -0.5 * lap + vloc


@pytest.mark.parametrize("sysf", [W.h2_sto3g, W.water_methane])
def test_lattice_local_energy_equals_continuum_without_cap(sysf):
    """Eq. (local energy condition): with nu_opt = nu_zv (rule -1) the lattice
    e_L equals the continuum e_L at every configuration, including ones whose
    hops cross the node (this fixes the sign of the spin-flip term)."""
    s = sysf()
    x = W.initial_walkers(s, 6, seed=8)
    ev = H.evaluate(s, x, 0.2, node_rule=-1)
    ref = _fd_local_energy(s, x)
    np.testing.assert_allclose(ev["eL"], ref, rtol=2e-6, atol=2e-5)
    if s.n_elec > 2:
        assert np.any(ev["vsf"] > 0.0)          # the check covered node-crossing hops


def test_node_rules_only_raise_the_potential():
    s = W.water_methane()
    x = W.initial_walkers(s, 20, seed=3)
    e = {r: H.evaluate(s, x, 0.2, node_rule=r) for r in (-1, 0, 1, 2)}
    assert np.all(e[0]["eL"] >= e[-1]["eL"])
    assert np.all(e[1]["eL"] >= e[0]["eL"])
    assert np.all(e[2]["eL"] >= e[1]["eL"])
    nodeless = e[0]["n_node"] == 0
    np.testing.assert_array_equal(e[0]["eL"][nodeless], e[-1]["eL"][nodeless])
    # the bare H2 trial state has no node: V_sf = 0 and nothing is capped
    s2 = W.h2_sto3g()
    e2 = H.evaluate(s2, W.initial_walkers(s2, 30, seed=1), 0.2, node_rule=0)
    assert np.all(e2["vsf"] == 0.0) and np.all(e2["n_node"] == 0)


def test_discrete_laplacian_converges_quadratically():
    """(sum_d r_{i,d} - 6)/a^2 -> lap_i Psi/Psi with an O(a^2) error."""
    s = W.h2_sto3g()
    x = W.initial_walkers(s, 4, seed=2)
    _, lap = wf.local_derivatives(s, x)
    errs = []
    for a in (0.08, 0.04, 0.02):
        r = wf.hop_ratios(s, x, a)
        errs.append(np.abs((np.sum(r, axis=-1) - 6.0) / (a * a) - lap))
    q1 = errs[0] / errs[1]
    q2 = errs[1] / errs[2]
    assert np.all(np.abs(q1 - 4.0) < 0.3) and np.all(np.abs(q2 - 4.0) < 0.3)


def test_potentials_closed_forms():
    s = W.water_methane()
    # screened pseudo-nucleus: finite at the nucleus, -2Z/(sqrt(pi) r_c)
    p = s.R[[0]] + np.array([[1e-9, 0, 0]])
    v = H.nu_ei(s, p)[0]
    others = sum(-s.Z[I] * math.erf(np.linalg.norm(s.R[0] - s.R[I]) / 0.5) /
                 np.linalg.norm(s.R[0] - s.R[I]) for I in range(1, s.n_nuc))
    assert abs(v - (-2 * s.Z[0] / (math.sqrt(math.pi) * 0.5) + others)) < 1e-6
    # all-electron cap
    s2 = W.h2_sto3g()
    p = np.array([[0.0, 0.01, 0.7]])
    a = 0.2
    assert abs(H.nu_ei_capped(s2, p, a)[0] - (-1 / a - 1 / math.hypot(0.01, 1.4))) < 1e-12
    assert abs(H.v_ii(s2) - 1 / 1.4) < 1e-15
