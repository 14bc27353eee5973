"""Seeded initial walker configurations (inputs, no method arithmetic)."""
from __future__ import annotations

import numpy as np

from .systems import System


def _electron_sites(sys: System) -> np.ndarray:
    """Nucleus index for every electron: nuclei take electrons round-robin in
    proportion to their (rounded) charge; spins alternate across the sequence so
    each nucleus receives a balanced mix."""
    remaining = [int(round(z)) for z in sys.Z]
    seq = []
    while sum(remaining) > 0 and len(seq) < sys.n_elec:
        for I in range(sys.n_nuc):
            if remaining[I] > 0 and len(seq) < sys.n_elec:
                seq.append(I)
                remaining[I] -= 1
    while len(seq) < sys.n_elec:          # charged systems: wrap around
        seq.append(len(seq) % sys.n_nuc)
    up = seq[0::2][: sys.n_up]
    dn = seq[1::2][: sys.n_dn]
    # if the alternation left one spin short, top up from the rest
    rest = seq[len(up) + len(dn):]
    while len(up) < sys.n_up:
        up.append(rest.pop(0) if rest else 0)
    while len(dn) < sys.n_dn:
        dn.append(rest.pop(0) if rest else 0)
    return np.array(up + dn, dtype=np.int64)


def initial_walkers(sys: System, n_w: int, seed: int = 1, sigma: float = 0.5) -> np.ndarray:
    """Positions (n_w, n_elec, 3): nucleus + N(0, sigma^2) per component."""
    rng = np.random.default_rng(seed)
    site = _electron_sites(sys)
    base = sys.R[site]                                      # (n_elec, 3)
    x = base[None, :, :] + sigma * rng.standard_normal((n_w, sys.n_elec, 3))
    return np.ascontiguousarray(x)


def lattice_walkers(n_w: int, a: float, seed: int = 1, spread: int = 3,
                    n_elec: int = 1, offset=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Positions on the common lattice a*(Z^3 + offset) near the origin (used when
    every walker must live on the same lattice, e.g. exact-diagonalisation
    comparisons)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(-spread, spread, size=(n_w, n_elec, 3))
    return np.ascontiguousarray(a * (n + np.asarray(offset)[None, None, :]))
