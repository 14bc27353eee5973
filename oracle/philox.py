"""Philox counter-based generator, written from Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), Section 3.

Philox-4xW-R applies R rounds of a bijection to a 4-word counter under a
2-word key.  One round multiplies words 0 and 2 by the constants M0, M1
(full 2W-bit products), and outputs
    (hi(M1*X2) ^ X1 ^ K0,  lo(M1*X2),  hi(M0*X0) ^ X3 ^ K1,  lo(M0*X0));
between rounds the key is bumped by the Weyl constants (W0, W1) = the first
W fraction bits of (golden ratio, sqrt(3)) modulo 1.

The generic routine below serves both word sizes; the 4x64 instance exists
only so a test can compare it with numpy's independent Philox implementation.

Stream layout used by the LRDMC runs (both the oracle and the CUDA library
implement it):
    key     = (seed mod 2^32, seed >> 32)
    counter = (walker slot, step index within the interval, interval index, 0)
              -> words (r0, r1) give the persistence-time uniform (conventional
                 schedule), words (r2, r3) the heat-bath move uniform;
    counter = (0, 0, interval index, 1) -> word r0 is the 32-bit comb offset of
              the reconfiguration that ends that interval.
"""
from __future__ import annotations

import numpy as np

# Philox4x32 multipliers (Salmon et al. 2011, Table 2)
M4x32 = (0xD2511F53, 0xCD9E8D57)
# Weyl key increments: floor(2^32 * frac(golden ratio)), floor(2^32 * frac(sqrt 3))
W4x32 = (0x9E3779B9, 0xBB67AE85)
# 64-bit instance (for the cross-check against numpy only)
M4x64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W4x64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox_generic(ctr, key, bits: int, mults, weyl, rounds: int = 10):
    """Scalar Philox on Python ints: ctr = 4 words, key = 2 words."""
    mask = (1 << bits) - 1
    c0, c1, c2, c3 = (int(v) & mask for v in ctr)
    k0, k1 = (int(v) & mask for v in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + weyl[0]) & mask
            k1 = (k1 + weyl[1]) & mask
        p0 = mults[0] * c0
        p1 = mults[1] * c2
        c0, c1, c2, c3 = ((p1 >> bits) ^ c1 ^ k0, p1 & mask,
                          (p0 >> bits) ^ c3 ^ k1, p0 & mask)
    return c0, c1, c2, c3


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Vectorised Philox4x32-R over numpy arrays of 32-bit values (any int dtype).

    Returns four uint64 arrays holding 32-bit outputs."""
    mask = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = (np.asarray(v).astype(np.uint64) & mask for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0, m1 = np.uint64(M4x32[0]), np.uint64(M4x32[1])
    w0, w1 = np.uint64(W4x32[0]), np.uint64(W4x32[1])
    s32 = np.uint64(32)
    for r in range(rounds):
        if r:
            k0 = (k0 + w0) & mask
            k1 = (k1 + w1) & mask
        p0 = m0 * c0                 # < 2^64, exact in uint64
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> s32) ^ c1 ^ k0, p1 & mask,
                          (p0 >> s32) ^ c3 ^ k1, p0 & mask)
    return c0, c1, c2, c3


def seed_key(seed: int):
    seed = int(seed) & ((1 << 64) - 1)
    return seed & 0xFFFFFFFF, seed >> 32


def uniform53(hi, lo):
    """Uniform in [0, 1) from two 32-bit words: the top 32 bits come from ``hi``
    and the next 21 from the top of ``lo``; the 53-bit integer times 2^-53."""
    v = (np.asarray(hi, dtype=np.uint64) << np.uint64(21)) | (np.asarray(lo, dtype=np.uint64) >> np.uint64(11))
    return v.astype(np.float64) * (2.0 ** -53)


def step_uniforms(seed: int, walker, step, interval):
    """(u_tau, u_move) for walker slots ``walker`` at ``step`` of ``interval``."""
    k0, k1 = seed_key(seed)
    walker = np.asarray(walker)
    r0, r1, r2, r3 = philox4x32(walker, step, interval, 0, k0, k1)
    return uniform53(r0, r1), uniform53(r2, r3)


def rotation_uniforms(seed: int, walker, interval):
    """Three uniforms for the lattice rotation of ``walker`` in ``interval``:
    counter (walker, 2^32-1, interval, 2) gives u1 (words 0-1) and u2 (words
    2-3), counter (walker, 2^32-1, interval, 3) gives u3 (words 0-1)."""
    k0, k1 = seed_key(seed)
    walker = np.asarray(walker)
    a0, a1, a2, a3 = philox4x32(walker, 0xFFFFFFFF, interval, 2, k0, k1)
    b0, b1, _, _ = philox4x32(walker, 0xFFFFFFFF, interval, 3, k0, k1)
    return uniform53(a0, a1), uniform53(a2, a3), uniform53(b0, b1)


def branch_offset32(seed: int, interval: int) -> int:
    """32-bit comb offset xi*2^32 for the reconfiguration ending ``interval``."""
    k0, k1 = seed_key(seed)
    r0, _, _, _ = philox4x32(0, 0, interval, 1, k0, k1)
    return int(r0)
