"""Pins for the oracle's Philox generator against independent implementations."""
import ctypes
import ctypes.util
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import philox as P


def test_weyl_constants_closed_form():
    getcontext().prec = 60
    phi_frac = (Decimal(5).sqrt() - 1) / 2            # golden ratio mod 1
    s3_frac = Decimal(3).sqrt() - 1
    for bits, W in ((32, P.W4x32), (64, P.W4x64)):
        assert W[0] == int(phi_frac * (Decimal(2) ** bits))
        assert W[1] == int(s3_frac * (Decimal(2) ** bits))


def test_philox4x64_matches_numpy():
    """numpy's Philox bit generator is an independent Philox4x64-10; its first
    output block is the counter incremented once."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4)]
        key = [int(v) for v in rng.integers(0, 2**63, size=2)]
        bg = np.random.Philox(counter=ctr, key=key)
        got = [int(v) for v in bg.random_raw(8)]
        for blk in range(2):
            c = list(ctr)
            c[0] += blk + 1                                # no carry for these draws
            ref = P.philox_generic(c, key, 64, P.M4x64, P.W4x64)
            assert list(ref) == got[4 * blk:4 * blk + 4]


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2**64 - 1])
def test_philox4x32_matches_curand_host_generator(seed):
    """cuRAND's host-side PHILOX4_32_10 generator (runs on the CPU) emits block b
    from counter (0, 0, b, 0) under key (seed lo, seed hi)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 512
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    k0, k1 = P.seed_key(seed)
    b = np.arange(512)
    r = P.philox4x32(0, 0, b, 0, k0, k1)
    ref = np.stack([v.astype(np.uint32) for v in r], axis=1).reshape(-1)
    np.testing.assert_array_equal(ref, out)


def test_vector_matches_scalar():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2**32, size=(4, 50), dtype=np.uint64)
    k0, k1 = 0xDEADBEEF, 0x01234567
    v = P.philox4x32(c[0], c[1], c[2], c[3], k0, k1)
    for j in range(50):
        s = P.philox_generic([int(c[m, j]) for m in range(4)], (k0, k1), 32, P.M4x32, P.W4x32)
        assert tuple(int(v[m][j]) for m in range(4)) == s


def test_uniform53_range_and_distribution():
    u_tau, u_mv = P.step_uniforms(11, np.arange(20000), 3, 5)
    for u in (u_tau, u_mv):
        assert u.min() >= 0.0 and u.max() < 1.0
        # exact multiples of 2^-53
        assert np.all(np.floor(u * 2.0**53) == u * 2.0**53)
        from scipy.stats import kstest
        assert kstest(u, "uniform").pvalue > 1e-4
    assert P.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0**-53
    assert P.uniform53(0, 0) == 0.0
