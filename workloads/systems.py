"""Synthetic molecular systems and trial-wavefunction parameters.

Conventions shared by every consumer (they define the *inputs*, not the method):

* Electrons ``0 .. n_up-1`` are spin up, ``n_up .. n_up+n_dn-1`` spin down.
* ``pot_kind[I] == 0``: bare Coulomb nucleus ``-Z/r`` (all-electron);
  ``pot_kind[I] == 1``: local Gaussian-screened pseudo-nucleus
  ``-Z erf(r/r_c)/r`` (valence charge ``Z``).
* Basis shells: ``shell_l == 0`` s-type (1 function), ``1`` p-type (3 functions,
  ordered x, y, z), ``-1`` Slater 1s test type ``exp(-zeta*r)`` (1 function).
  Shell ``s`` uses primitives ``exps[off_s : off_s+nprim_s]`` with coefficients
  ``coefs[...]``; a contracted function is
  ``angular(d) * sum_g coefs_g * exp(-exps_g * |d|^2)`` (Slater type:
  ``sum_g coefs_g * exp(-exps_g * |d|)``) with ``d = r - R_atom``.
  Coefficients are stored *already multiplied* by the primitive normalisation,
  so consumers never normalise.
* Molecular orbitals ``phi_k = sum_mu C[k, mu] chi_mu``; spin-up electrons use
  orbitals ``0..n_up-1`` and spin-down electrons ``0..n_dn-1`` (restricted).
* Jastrow ``J = sum_{i<j} c r_ij/(1 + b r_ij) - sum_{i,I} A_I r_iI/(1 + B_I r_iI)``
  with ``c = j2_anti`` for opposite spins and ``j2_par`` for equal spins.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class System:
    name: str
    R: np.ndarray            # (n_nuc, 3) nuclear positions, bohr
    Z: np.ndarray            # (n_nuc,) charge (valence charge for pseudo-nuclei)
    pot_kind: np.ndarray     # (n_nuc,) int32, 0 bare Coulomb, 1 erf-screened
    r_c: np.ndarray          # (n_nuc,) screening radius (unused for kind 0)
    n_up: int
    n_dn: int
    shell_atom: np.ndarray   # (n_shell,) int32
    shell_l: np.ndarray      # (n_shell,) int32
    shell_nprim: np.ndarray  # (n_shell,) int32
    exps: np.ndarray         # (n_prim_total,)
    coefs: np.ndarray        # (n_prim_total,), normalisation folded in
    C: np.ndarray            # (n_orb, n_bf) MO coefficients
    j2_anti: float
    j2_par: float
    j2_b: float
    j1_A: np.ndarray         # (n_nuc,)
    j1_B: np.ndarray         # (n_nuc,)

    @property
    def n_nuc(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_shell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def n_bf(self) -> int:
        return int(sum(3 if l == 1 else 1 for l in self.shell_l))

    @property
    def n_orb(self) -> int:
        return int(self.C.shape[0])

    @property
    def n_prim_eval(self) -> int:
        """Primitive exponentials evaluated per point."""
        return int(self.exps.shape[0])

    def validate(self) -> None:
        n = self.n_nuc
        assert self.R.shape == (n, 3) and self.Z.shape == (n,)
        assert self.pot_kind.shape == (n,) and self.r_c.shape == (n,)
        assert self.j1_A.shape == (n,) and self.j1_B.shape == (n,)
        assert int(self.shell_nprim.sum()) == self.exps.shape[0] == self.coefs.shape[0]
        assert self.C.shape[1] == self.n_bf
        assert self.n_orb >= max(self.n_up, self.n_dn)
        assert np.all((self.shell_atom >= 0) & (self.shell_atom < n))


def _norm_s(alpha: float) -> float:
    # (2 alpha / pi)^(3/4): unit-norm s Gaussian
    return (2.0 * alpha / math.pi) ** 0.75


def _norm_p(alpha: float) -> float:
    # (2 alpha / pi)^(3/4) * 2 sqrt(alpha): unit-norm Cartesian p Gaussian
    return (2.0 * alpha / math.pi) ** 0.75 * 2.0 * math.sqrt(alpha)


def _arr(x, dt=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dt))


def _build(name, R, Z, pot_kind, r_c, n_up, n_dn, shells, C, j2_anti, j2_par, j2_b,
           j1_A, j1_B) -> System:
    """shells: list of (atom, l, [(exp, raw_coef), ...]); raw_coef multiplies a
    normalised primitive (s/p) or is used as is (Slater type)."""
    atoms, ls, nprims, exps, coefs = [], [], [], [], []
    for atom, l, prims in shells:
        atoms.append(atom)
        ls.append(l)
        nprims.append(len(prims))
        for e, c in prims:
            exps.append(e)
            if l == 0:
                coefs.append(c * _norm_s(e))
            elif l == 1:
                coefs.append(c * _norm_p(e))
            else:
                coefs.append(c)
    n_nuc = len(Z)
    s = System(name=name, R=_arr(R).reshape(n_nuc, 3), Z=_arr(Z),
               pot_kind=_arr(pot_kind, np.int32), r_c=_arr(r_c), n_up=int(n_up),
               n_dn=int(n_dn), shell_atom=_arr(atoms, np.int32), shell_l=_arr(ls, np.int32),
               shell_nprim=_arr(nprims, np.int32), exps=_arr(exps), coefs=_arr(coefs),
               C=_arr(C), j2_anti=float(j2_anti), j2_par=float(j2_par), j2_b=float(j2_b),
               j1_A=_arr(j1_A), j1_B=_arr(j1_B))
    s.validate()
    return s


def hydrogen_atom_sto(zeta: float = 1.0) -> System:
    """One electron, bare proton, Slater 1s trial function exp(-zeta r).

    With zeta = 1 this is the exact ground state, so the local energy is -0.5 Ha
    at every configuration."""
    return _build("H-atom-STO", [[0, 0, 0]], [1.0], [0], [0.0], 1, 0,
                  [(0, -1, [(zeta, 1.0)])], [[1.0]], 0.0, 0.0, 1.0, [0.0], [0.0])


def hydrogen_atom_gauss(beta: float = 8.0 / (9.0 * math.pi)) -> System:
    """One electron, bare proton, nodeless Gaussian trial function exp(-beta r^2)."""
    return _build("H-atom-Gauss", [[0, 0, 0]], [1.0], [0], [0.0], 1, 0,
                  [(0, 0, [(beta, 1.0)])], [[1.0]], 0.0, 0.0, 1.0, [0.0], [0.0])


def hydrogen_atom_pz(beta: float = 0.1) -> System:
    """One electron, bare proton, Gaussian p_z trial function z exp(-beta r^2):
    its nodal plane z = 0 is the node of the exact 2p states."""
    return _build("H-atom-pz", [[0, 0, 0]], [1.0], [0], [0.0], 1, 0,
                  [(0, 1, [(beta, 1.0)])], [[0.0, 0.0, 1.0]], 0.0, 0.0, 1.0, [0.0], [0.0])


STO3G_H_EXPS = (3.42525, 0.62391, 0.16886)
STO3G_H_COEFS = (0.15433, 0.53533, 0.44463)


def h2_sto3g(half_bond: float = 0.7) -> System:
    """All-electron H2 with nuclei at z = +-half_bond; one doubly occupied
    orbital = sum of the two atoms' 3-primitive 1s contractions; Pade e-e
    Jastrow 0.5 r/(1 + r) for the antiparallel pair."""
    prims = list(zip(STO3G_H_EXPS, STO3G_H_COEFS))
    return _build("H2", [[0, 0, -half_bond], [0, 0, half_bond]], [1.0, 1.0], [0, 0],
                  [0.0, 0.0], 1, 1, [(0, 0, prims), (1, 0, prims)], [[1.0, 1.0]],
                  0.5, 0.25, 1.0, [0.0, 0.0], [0.0, 0.0])


def _log_spaced(n: int, lo: float = 0.1, hi: float = 20.0):
    if n == 1:
        return [math.sqrt(lo * hi)]
    return list(np.geomspace(lo, hi, n))


def water_methane(mo_seed: int = 2, r_c: float = 0.5, j1_A: float = 0.1,
                  j1_B: float = 1.0) -> System:
    """Water-methane-shaped complex: C at the origin with four H at 2.06 bohr
    (tetrahedral, even-parity corners), O at +6.5 bohr on z with two H at 1.81
    bohr (HOH 104.5 deg, in the xz-plane, pointing away from C).  Valence charges
    O 6, C 4, H 1 under erf-screened local pseudopotentials; 8 up + 8 down
    electrons.  Basis per heavy atom 4s + 3p, per H 2s + 1p, single-primitive
    shells with exponents log-spaced over [0.1, 20].  MO coefficients are
    standard normal (seeded) with orthonormalised columns."""
    R = [[0.0, 0.0, 0.0]]
    Z = [4.0]
    t = 2.06 / math.sqrt(3.0)
    for sx, sy, sz in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)):
        R.append([sx * t, sy * t, sz * t])
        Z.append(1.0)
    zO = 6.5
    R.append([0.0, 0.0, zO])
    Z.append(6.0)
    half = math.radians(104.5) / 2.0
    for sx in (1.0, -1.0):
        R.append([sx * 1.81 * math.sin(half), 0.0, zO + 1.81 * math.cos(half)])
        Z.append(1.0)
    n_nuc = len(Z)
    shells = []
    for I in range(n_nuc):
        heavy = Z[I] > 1.0
        ns, np_ = (4, 3) if heavy else (2, 1)
        for e in _log_spaced(ns):
            shells.append((I, 0, [(e, 1.0)]))
        for e in _log_spaced(np_):
            shells.append((I, 1, [(e, 1.0)]))
    n_bf = sum(3 if l == 1 else 1 for _, l, _ in shells)
    rng = np.random.default_rng(mo_seed)
    G = rng.standard_normal((n_bf, 8))
    Q, _ = np.linalg.qr(G)
    C = Q.T.copy()
    return _build("water-methane", R, Z, [1] * n_nuc, [r_c] * n_nuc, 8, 8, shells, C,
                  0.5, 0.25, 1.0, [j1_A] * n_nuc, [j1_B] * n_nuc)


def hydrogen_chain(n_atoms: int = 128, spacing: float = 1.8, mo_seed: int = 5,
                   s_exp: float = 1.0, p_exp: float = 0.8) -> System:
    """Linear hydrogen chain along z, all-electron, one s + one p single-primitive
    shell per atom, seeded orthonormalised MOs, spins balanced."""
    R = [[0.0, 0.0, spacing * (I - (n_atoms - 1) / 2.0)] for I in range(n_atoms)]
    shells = []
    for I in range(n_atoms):
        shells.append((I, 0, [(s_exp, 1.0)]))
        shells.append((I, 1, [(p_exp, 1.0)]))
    n_bf = 4 * n_atoms
    n_up = n_atoms // 2
    rng = np.random.default_rng(mo_seed)
    G = rng.standard_normal((n_bf, n_up))
    Q, _ = np.linalg.qr(G)
    return _build(f"H{n_atoms}-chain", R, [1.0] * n_atoms, [0] * n_atoms,
                  [0.0] * n_atoms, n_up, n_atoms - n_up, shells, Q.T.copy(), 0.5,
                  0.25, 1.0, [0.0] * n_atoms, [1.0] * n_atoms)


def hydrogen_cluster(n_atoms: int, seed: int = 0, min_spacing: float = 1.4, density: float = 0.125,
                     mo_seed: int | None = None, s_exp: float = 1.0, p_exp: float = 0.8) -> System:
    """Seeded hydrogen cluster: n_atoms protons at random positions in a sphere
    holding `density` atoms per bohr^3, no two closer than min_spacing (bohr,
    rejection sampling); one s + one p single-primitive shell per atom, seeded
    orthonormalised MOs, spins balanced, bare Coulomb nuclei, e-e Pade Jastrow."""
    rng = np.random.default_rng(seed)
    radius = (3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    R: list = []
    while len(R) < n_atoms:
        p = rng.uniform(-radius, radius, 3)
        if np.dot(p, p) > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= min_spacing for q in R):
            R.append(p)
    shells = []
    for I in range(n_atoms):
        shells.append((I, 0, [(s_exp, 1.0)]))
        shells.append((I, 1, [(p_exp, 1.0)]))
    n_bf = 4 * n_atoms
    n_up = n_atoms // 2
    n_occ = max(n_up, n_atoms - n_up)
    mrng = np.random.default_rng(seed + 1000 if mo_seed is None else mo_seed)
    Q, _ = np.linalg.qr(mrng.standard_normal((n_bf, n_occ)))
    return _build(f"H{n_atoms}-cluster-{seed}", [list(p) for p in R], [1.0] * n_atoms, [0] * n_atoms,
                  [0.0] * n_atoms, n_up, n_atoms - n_up, shells, Q.T.copy(), 0.5, 0.25, 1.0,
                  [0.0] * n_atoms, [1.0] * n_atoms)


def by_name(name: str) -> System:
    table = {"h_sto": hydrogen_atom_sto, "h_gauss": hydrogen_atom_gauss,
             "h2": h2_sto3g, "wm": water_methane}
    return table[name]()
