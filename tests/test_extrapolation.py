"""Lattice-space extrapolation a -> 0 (Sec. II: O(a^2) bias of the LRDMC energy).

Oracle pins: exact recovery of polynomial data, the reported error equal to
the spread of the fit over resampled data, and the continuum limit -1/2 Ha of
the exactly diagonalised lattice Hamiltonian of the hydrogen atom (Appendix
D) reached from spacings 0.3 to 0.6 bohr.  The library's fit (host code, no
GPU) against the oracle's; on the GPU, an a-scan of LRDMC runs on the same
lattices extrapolated to -1/2 Ha."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import estimator as est
from test_oracle_lrdmc import ZETA_ED, lattice_ground_energy_sto

# spacings and box sizes (about 22 bohr) of the exact-diagonalisation scan
SCAN = [(0.3, 74), (0.4, 56), (0.5, 45), (0.6, 38)]


def test_oracle_recovers_polynomial_data():
    a = np.array([0.1, 0.2, 0.25, 0.3, 0.45])
    for order, c in ((1, [-1.2, 0.07]), (2, [-1.2, 0.07, -0.3]), (3, [0.4, -2.0, 1.5, 0.25])):
        E = sum(cj * a ** (2 * j) for j, cj in enumerate(c))
        coef, cov, chi2 = est.extrapolate_a(a, E, np.full(len(a), 1e-3), order)
        np.testing.assert_allclose(coef, c, rtol=0, atol=1e-10)
        assert chi2 < 1e-16


def test_oracle_error_is_the_sampling_spread():
    """sqrt(cov[0,0]) is the standard deviation of the fitted a -> 0 energy
    over data resampled within their errors; chi2 averages n - (order + 1)."""
    rng = np.random.default_rng(3)
    a = np.array([0.2, 0.3, 0.4, 0.5, 0.6])
    err = np.array([2e-4, 3e-4, 2e-4, 4e-4, 5e-4])
    truth = -1.0 + 0.05 * a ** 2 - 0.02 * a ** 4
    c0, chis = [], []
    for _ in range(4000):
        coef, cov, chi2 = est.extrapolate_a(a, truth + err * rng.standard_normal(len(a)), err, 2)
        c0.append(coef[0])
        chis.append(chi2)
    sd = np.sqrt(cov[0, 0])
    assert abs(np.std(c0) / sd - 1.0) < 0.05
    assert abs(np.mean(c0) + 1.0) < 4 * sd / np.sqrt(4000)
    assert abs(np.mean(chis) / 2.0 - 1.0) < 0.06


def test_oracle_reaches_the_continuum_hydrogen_energy():
    """Lattice ground energies of H^a (exact diagonalisation, Slater guiding
    function exp(-0.8 r)) extrapolate to the continuum ground state -1/2 Ha;
    each spacing alone misses it by 4 to 14 mHa."""
    a = np.array([s for s, _ in SCAN])
    E = np.array([lattice_ground_energy_sto(ZETA_ED, s, n) for s, n in SCAN])
    assert np.all(E + 0.5 > 3e-3)
    coef, cov, chi2 = est.extrapolate_a(a, E, np.full(len(a), 1e-5), 2)
    assert abs(coef[0] + 0.5) < 3e-4, coef


def test_library_fit_matches_oracle():
    from paper_2508_12033_b300 import build
    build.build()
    import paper_2508_12033_b300 as P
    rng = np.random.default_rng(7)
    for order in (1, 2, 3):
        for _ in range(20):
            n = order + 1 + int(rng.integers(0, 6))
            a = np.sort(rng.uniform(0.05, 0.8, n))
            E = rng.normal(-2.0, 0.1, n)
            err = rng.uniform(1e-4, 1e-2, n)
            c_lib, cov_lib, chi_lib = P.extrapolate_a(a, E, err, order)
            c_or, cov_or, chi_or = est.extrapolate_a(a, E, err, order)
            scale = np.sqrt(np.diag(cov_or))
            assert np.all(np.abs(c_lib - c_or) <= 1e-9 * scale), (order, c_lib, c_or)
            np.testing.assert_allclose(cov_lib, cov_or, rtol=1e-7, atol=1e-12 * np.abs(cov_or).max())
            assert abs(chi_lib - chi_or) <= 1e-8 * max(1.0, chi_or)


def test_library_fit_rejects_bad_input():
    from paper_2508_12033_b300 import build
    build.build()
    import paper_2508_12033_b300 as P
    a, E, e = [0.2, 0.3, 0.4], [-1.0, -0.99, -0.98], [1e-3] * 3
    bad = [(a, E, e, 0), (a, E, e, 4), (a, E, e, 3), (a, E, [1e-3, 0.0, 1e-3], 1),
           (a, [-1.0, float("nan"), -0.98], e, 1), ([0.2, -0.3, 0.4], E, e, 1),
           ([0.3, 0.3, 0.3], E, e, 1)]
    for aa, EE, ee, order in bad:
        with pytest.raises(P.LrdmcError) as x:
            P.extrapolate_a(aa, EE, ee, order)
        assert x.value.status == 1
    lib = P.load_library()
    assert lib.lrdmc_extrapolate_a(3, None, None, None, 1, None, None, None) == 1


@pytest.mark.gpu
def test_gpu_a_scan_extrapolates_to_the_continuum_hydrogen_energy():
    """LRDMC on the GPU at each spacing of the scan (walkers on the same lattice
    as the diagonalisation) reproduces the lattice energy, and the extrapolated
    energy is the continuum -1/2 Ha."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.hydrogen_atom_sto(ZETA_ED)
    a_list, E_list, err_list = [], [], []
    for a, n_side in SCAN:
        lr = P.Lrdmc(s, W.lattice_walkers(2048, a, seed=4, spread=3), a, seed=11, p_gbar=20, n_equil=20)
        for _ in range(140):
            lr.propagate(P.LOAD_BALANCED, n_proj=15)
            lr.branch()
        E, err = lr.energy()
        e_lat = lattice_ground_energy_sto(ZETA_ED, a, n_side)
        assert abs(E - e_lat) < 5 * err + 1e-4, (a, E, err, e_lat)
        a_list.append(a)
        E_list.append(E)
        err_list.append(err)
    coef, cov, _ = P.extrapolate_a(a_list, E_list, err_list, 2)
    sd = float(np.sqrt(cov[0, 0]))
    assert abs(coef[0] + 0.5) < 5 * sd + 5e-4, (coef, sd)
