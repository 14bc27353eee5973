"""Pins for the oracle's trial-wavefunction layer (closed forms, brute force,
finite differences, invariances) — none of them re-evaluates the oracle's own
formula."""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import wavefunction as wf


def _fd_grad_lap(f, pts, h=1e-4):
    g = np.zeros(pts.shape + f(pts).shape[pts.ndim - 1:])
    lap = 0.0
    f0 = f(pts)
    grads = []
    for m in range(3):
        e = np.zeros(3)
        e[m] = h
        fp, fm = f(pts + e), f(pts - e)
        grads.append((fp - fm) / (2 * h))
        lap = lap + (fp - 2 * f0 + fm) / (h * h)
    return np.stack(grads, axis=-1), lap


@pytest.mark.parametrize("sysf", [W.hydrogen_atom_sto, W.h2_sto3g, W.water_methane])
def test_basis_derivatives_match_finite_differences(sysf):
    s = sysf()
    rng = np.random.default_rng(1)
    pts = s.R[rng.integers(0, s.n_nuc, 40)] + rng.normal(0, 0.8, (40, 3))
    chi, g, L = wf.basis_derivs(s, pts)
    gfd, Lfd = _fd_grad_lap(lambda p: wf.basis_values(s, p), pts)
    scale = np.maximum(1.0, np.abs(chi).max())
    np.testing.assert_allclose(g, gfd, atol=2e-6 * scale * 30)
    np.testing.assert_allclose(L, Lfd, atol=2e-4 * scale * 30)


def test_gaussian_normalisation():
    """Stored s and p coefficients make unit-norm primitives (radial quadrature)."""
    s = W.water_methane()
    r = np.linspace(0, 30, 200001)
    off = np.concatenate([[0], np.cumsum(s.shell_nprim)])
    for sh in range(s.n_shell):
        a, c = s.exps[off[sh]], s.coefs[off[sh]]
        if s.shell_l[sh] == 0:
            integrand = (c * np.exp(-a * r * r)) ** 2 * 4 * math.pi * r * r
        else:
            integrand = (c * np.exp(-a * r * r)) ** 2 * 4 * math.pi * r ** 4 / 3.0
        assert abs(np.trapezoid(integrand, r) - 1.0) < 1e-6


def _leibniz_det(M):
    n = M.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        sgn = 1
        for i in range(n):
            for j in range(i + 1, n):
                if perm[i] > perm[j]:
                    sgn = -sgn
        prod = 1.0
        for i in range(n):
            prod *= M[i, perm[i]]
        tot += sgn * prod
    return tot


def _psi_bruteforce(s, x):
    phi = wf.orbitals(s, x)
    val = math.exp(float(wf.jastrow(s, x[None])[0]))
    for start, n in wf.spin_blocks(s):
        if n:
            val *= _leibniz_det(phi[start:start + n, :n])
    return val


def test_hop_ratios_match_bruteforce_determinants():
    s = W.hydrogen_chain(6, spacing=1.6, mo_seed=3)      # 3 up + 3 down
    x = W.initial_walkers(s, 3, seed=4)
    a = 0.23
    r = wf.hop_ratios(s, x, a)
    for b in range(3):
        p0 = _psi_bruteforce(s, x[b])
        for i in range(s.n_elec):
            for d in range(6):
                xd = x[b].copy()
                xd[i, wf.HOP_AXIS[d]] += wf.HOP_SIGN[d] * a
                ref = _psi_bruteforce(s, xd) / p0
                assert abs(r[b, i, d] - ref) <= 1e-11 * max(1.0, abs(ref))


def test_ratios_invariant_under_occupied_orbital_mixing():
    s = W.water_methane()
    x = W.initial_walkers(s, 4, seed=9)
    r0 = wf.hop_ratios(s, x, 0.2)
    _, lap0 = wf.local_derivatives(s, x)
    rng = np.random.default_rng(5)
    T = np.eye(8) + 0.3 * rng.standard_normal((8, 8))
    s2 = W.water_methane()
    s2.C = T @ s.C
    r1 = wf.hop_ratios(s2, x, 0.2)
    _, lap1 = wf.local_derivatives(s2, x)
    np.testing.assert_allclose(r1, r0, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(lap1, lap0, rtol=1e-8, atol=1e-8)


def test_log_psi_gradient_and_laplacian_match_finite_differences():
    """grad_i Psi/Psi and lap_i Psi/Psi by central differences of Psi itself
    (as ratios Psi(x +- h e)/Psi(x) of fresh log|Psi|, sign), independent of the
    row-replacement formulas; Richardson-extrapolated to O(h^4)."""
    for s in (W.h2_sto3g(), W.water_methane(), W.hydrogen_chain(6, spacing=1.6, mo_seed=3)):
        x = W.initial_walkers(s, 3, seed=2)
        grad, lap = wf.local_derivatives(s, x)
        s0, l0 = wf.log_psi(s, x)

        def ratio(xx):
            s1, l1 = wf.log_psi(s, xx)
            return s1 * s0 * np.exp(l1 - l0)

        def fd(i, h):
            g_fd = np.zeros((3, 3))
            lap_fd = np.zeros(3)
            for m in range(3):
                xp, xm = x.copy(), x.copy()
                xp[:, i, m] += h
                xm[:, i, m] -= h
                rp, rm = ratio(xp), ratio(xm)
                g_fd[:, m] = (rp - rm) / (2 * h)
                lap_fd += (rp - 2.0 + rm) / (h * h)
            return g_fd, lap_fd

        for i in range(s.n_elec):
            g1, d1 = fd(i, 2e-4)
            g2, d2 = fd(i, 1e-4)
            g_fd = (4 * g2 - g1) / 3
            lap_fd = (4 * d2 - d1) / 3
            np.testing.assert_allclose(grad[:, i, :], g_fd, rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(lap[:, i], lap_fd, rtol=1e-4, atol=1e-3)


def test_hydrogen_sto_closed_forms():
    s = W.hydrogen_atom_sto(1.0)
    x = W.initial_walkers(s, 50, seed=3)
    r = np.linalg.norm(x[:, 0, :], axis=-1)
    sgn, lp = wf.log_psi(s, x)
    np.testing.assert_allclose(lp, -r, rtol=1e-14, atol=1e-14)
    assert np.all(sgn == 1)
    _, lap = wf.local_derivatives(s, x)
    np.testing.assert_allclose(lap[:, 0], 1.0 - 2.0 / r, rtol=1e-12)
    a = 0.15
    rat = wf.hop_ratios(s, x, a)
    for d in range(6):
        xd = x[:, 0, :].copy()
        xd[:, wf.HOP_AXIS[d]] += wf.HOP_SIGN[d] * a
        np.testing.assert_allclose(rat[:, 0, d], np.exp(r - np.linalg.norm(xd, axis=-1)), rtol=1e-13)


def test_jastrow_pair_closed_form_and_cusp():
    """Two electrons, no orbitals' dependence: J = c r/(1 + b r); the
    antiparallel cusp dJ/dr at r=0 equals c = 1/2."""
    s = W.h2_sto3g()
    x = np.array([[[0.1, 0.2, 0.3], [0.1, 0.2, 0.3 + 1e-7]]])
    J = wf.jastrow(s, x)
    assert abs(J[0] / 1e-7 - 0.5) < 1e-6
    x = np.array([[[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]]])
    r = 1.3
    assert abs(wf.jastrow(s, x)[0] - 0.5 * r / (1 + r)) < 1e-15
