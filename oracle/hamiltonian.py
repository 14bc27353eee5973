"""Lattice-regularised fixed-node Hamiltonian at one configuration (FP64).

Follows Appendix D of the paper (Eqs. for the discretised Laplacian, the FN
Hamiltonian with the spin-flip term, the regularised local potential and the
per-electron nodal/nuclear regularisation) together with the split
H = H_bar + delta W(x) of the load-balanced algorithm (Sec. II.C):

* kinetic hops: every electron to its 6 lattice neighbours, H_{x',x} = -1/(2a^2),
  diagonal 3 N_e / a^2;
* fixed node: a hop with ratio r < 0 is removed from H_bar and its
  H_{x',x} r = |r|/(2a^2) goes to the spin-flip term V_sf; r = 0 contributes 0;
* b_bar = sum over kept hops of r/(2a^2) (the off-diagonal normalisation);
* nu_zv,i = nu_ei(r_i) + [(sum_d r_{i,d} - 6)/a^2 - lap_i Psi/Psi] / 2;
* nu^a_ei = -sum_I Z_I / max(|r_i - R_I|, a) for bare nuclei, the bare screened
  potential itself for pseudo-nuclei;
* nu_opt,i = max(nu_zv,i, nu^a_ei) where the node rule applies, else nu_zv,i;
* W = 3 N_e/a^2 + sum_i nu_opt,i + sum_{i<j} 1/r_ij + V_ii + V_sf;
* e_L = W - b_bar.

Node rule (the paper's condition "Psi(x) Psi(x_j) < 0 for at least one x_j"):
  0 = per electron (x_j ranges over the hops of electron i),
  1 = per configuration (x_j ranges over all 6 N_e hops),
  2 = always apply the max (a bounded-below variant),
 -1 = never apply it (the unregularised lattice potential; used by tests).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import wavefunction as wf


def nu_ei(sys, r_i):
    """Bare electron-ion potential at electron positions (..., 3)."""
    v = np.zeros(r_i.shape[:-1])
    for I in range(sys.n_nuc):
        r = np.linalg.norm(r_i - sys.R[I], axis=-1)
        if sys.pot_kind[I] == 0:
            v = v - sys.Z[I] / r
        else:
            v = v - sys.Z[I] * erf(r / sys.r_c[I]) / r
    return v


def nu_ei_capped(sys, r_i, a):
    """nu^a_ei: -Z/max(r, a) for bare nuclei, the screened potential for pseudo-nuclei."""
    v = np.zeros(r_i.shape[:-1])
    for I in range(sys.n_nuc):
        r = np.linalg.norm(r_i - sys.R[I], axis=-1)
        if sys.pot_kind[I] == 0:
            v = v - sys.Z[I] / np.maximum(r, a)
        else:
            v = v - sys.Z[I] * erf(r / sys.r_c[I]) / r
    return v


def v_ee(x):
    ne = x.shape[-2]
    v = np.zeros(x.shape[:-2])
    for i in range(ne):
        for j in range(i + 1, ne):
            v = v + 1.0 / np.linalg.norm(x[..., i, :] - x[..., j, :], axis=-1)
    return v


def v_ii(sys):
    v = 0.0
    for I in range(sys.n_nuc):
        for J in range(I + 1, sys.n_nuc):
            v += sys.Z[I] * sys.Z[J] / np.linalg.norm(sys.R[I] - sys.R[J])
    return v


def evaluate(sys, x, a, node_rule=0, versors=None):
    """All per-configuration quantities at x (..., n_e, 3); hops along the
    Cartesian axes or along the rows of ``versors`` (..., 3, 3).

    Returns a dict with
      ratios (..., n_e, 6), bbar, vsf, W, eL (...), n_node (...) = number of
      electrons with at least one node-crossing hop, lap (..., n_e),
      nu_opt (..., n_e)."""
    x = np.asarray(x, dtype=np.float64)
    ne = sys.n_elec
    r = wf.hop_ratios(sys, x, a, versors)                      # (..., ne, 6)
    pos = r > 0.0
    neg = r < 0.0
    inv2a2 = 1.0 / (2.0 * a * a)
    bbar = np.sum(np.where(pos, r, 0.0), axis=(-1, -2)) * inv2a2
    vsf = np.sum(np.where(neg, -r, 0.0), axis=(-1, -2)) * inv2a2
    _, lap = wf.local_derivatives(sys, x)                      # (..., ne)
    nu = nu_ei(sys, x)                                         # (..., ne)
    nu_zv = nu + 0.5 * ((np.sum(r, axis=-1) - 6.0) / (a * a) - lap)
    nu_cap = nu_ei_capped(sys, x, a)
    node_e = np.any(neg, axis=-1)                              # (..., ne)
    if node_rule == 0:
        apply = node_e
    elif node_rule == 1:
        apply = np.broadcast_to(np.any(node_e, axis=-1)[..., None], node_e.shape)
    elif node_rule == 2:
        apply = np.ones_like(node_e)
    elif node_rule == -1:          # never cap: V^a_loc exactly as in the lattice-potential Eq.
        apply = np.zeros_like(node_e)
    else:
        raise ValueError(node_rule)
    nu_opt = np.where(apply, np.maximum(nu_zv, nu_cap), nu_zv)
    W = 3.0 * ne / (a * a) + np.sum(nu_opt, axis=-1) + v_ee(x) + v_ii(sys) + vsf
    return dict(ratios=r, bbar=bbar, vsf=vsf, W=W, eL=W - bbar,
                n_node=np.sum(node_e, axis=-1).astype(np.int64), lap=lap, nu_opt=nu_opt)


def continuum_local_energy(sys, x):
    """e_L of the continuous Hamiltonian, -lap Psi/(2 Psi) + V_loc (no lattice)."""
    _, lap = wf.local_derivatives(sys, x)
    return -0.5 * np.sum(lap, axis=-1) + np.sum(nu_ei(sys, x), axis=-1) + v_ee(x) + v_ii(sys)
