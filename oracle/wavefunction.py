"""Slater-Jastrow trial wavefunction, evaluated from its plain definition (FP64).

Psi_G(x) = det A_up(x) * det A_dn(x) * exp(J(x)),   A_s[i, k] = phi_k(r_i),
phi_k = sum_mu C[k, mu] chi_mu.  Wavefunction ratios Psi_G(x')/Psi_G(x) are
taken as quotients of *freshly computed* determinants (no rank-1 updates), and
per-electron derivatives of the determinant as determinants with one row
replaced by the derivative of the orbitals (linearity of det in a row).
Everything is vectorised over a leading batch of configurations only.
"""
from __future__ import annotations

import numpy as np

# hop order used everywhere: d = 0..5 -> (+x, -x, +y, -y, +z, -z)
HOP_AXIS = np.array([0, 0, 1, 1, 2, 2])
HOP_SIGN = np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0])


def _shell_offsets(sys):
    off = np.concatenate([[0], np.cumsum(sys.shell_nprim)]).astype(int)
    return off


def basis_values(sys, pts):
    """chi_mu at points ``pts`` (..., 3) -> (..., n_bf)."""
    return basis_derivs(sys, pts, order=0)[0]


def basis_derivs(sys, pts, order=2):
    """Basis values, gradients and Laplacians at ``pts`` (..., 3).

    Returns (chi (..., n_bf), grad (..., n_bf, 3) or None, lap (..., n_bf) or None).
    Closed forms per primitive h:
      s   h = exp(-a r^2):        grad = -2a d h,  lap = (4a^2 r^2 - 6a) h
      p_m d_m h:                   grad_n = (delta_mn - 2a d_m d_n) h,
                                   lap = d_m (4a^2 r^2 - 10a) h
      1s  h = exp(-z r):          grad = -z d/r h, lap = (z^2 - 2z/r) h
    """
    pts = np.asarray(pts, dtype=np.float64)
    lead = pts.shape[:-1]
    off = _shell_offsets(sys)
    chi, grad, lap = [], [], []
    for s in range(sys.n_shell):
        d = pts - sys.R[sys.shell_atom[s]]
        r2 = np.sum(d * d, axis=-1)
        l = int(sys.shell_l[s])
        ex = sys.exps[off[s]:off[s + 1]]
        co = sys.coefs[off[s]:off[s + 1]]
        if l == -1:
            r = np.sqrt(r2)
            h = sum(c * np.exp(-z * r) for z, c in zip(ex, co))
            chi.append(h)
            if order:
                g_r = sum(-c * z * np.exp(-z * r) for z, c in zip(ex, co))  # dh/dr
                grad.append(g_r[..., None] * d / r[..., None])
                lap.append(sum(c * (z * z - 2.0 * z / r) * np.exp(-z * r) for z, c in zip(ex, co)))
            continue
        hs = [c * np.exp(-a * r2) for a, c in zip(ex, co)]
        if l == 0:
            chi.append(sum(hs))
            if order:
                grad.append(sum((-2.0 * a) * h[..., None] * d for a, h in zip(ex, hs)))
                lap.append(sum((4.0 * a * a * r2 - 6.0 * a) * h for a, h in zip(ex, hs)))
        elif l == 1:
            for m in range(3):
                chi.append(sum(d[..., m] * h for h in hs))
                if order:
                    g = np.zeros(lead + (3,))
                    for a, h in zip(ex, hs):
                        e_m = np.zeros(3)
                        e_m[m] = 1.0
                        g = g + h[..., None] * (e_m - 2.0 * a * d[..., m:m + 1] * d)
                    grad.append(g)
                    lap.append(sum(d[..., m] * (4.0 * a * a * r2 - 10.0 * a) * h
                                   for a, h in zip(ex, hs)))
        else:
            raise ValueError(f"unsupported shell type {l}")
    chi = np.stack(chi, axis=-1)
    if not order:
        return chi, None, None
    return chi, np.stack(grad, axis=-2), np.stack(lap, axis=-1)


def orbitals(sys, pts):
    """phi_k at points (..., 3) -> (..., n_orb)."""
    return basis_values(sys, pts) @ sys.C.T


def spin_blocks(sys):
    """[(first electron, count)] for the up and down determinants."""
    return [(0, sys.n_up), (sys.n_up, sys.n_dn)]


def slater_matrices(sys, x):
    """A_up, A_dn for configurations x (..., n_e, 3): A[..., i, k] = phi_k(r_i)."""
    phi = orbitals(sys, x)                       # (..., n_e, n_orb)
    out = []
    for start, n in spin_blocks(sys):
        out.append(phi[..., start:start + n, :n])
    return out


def _slogdet(A):
    if A.shape[-1] == 0:
        lead = A.shape[:-2]
        return np.ones(lead), np.zeros(lead)
    return np.linalg.slogdet(A)


def pair_u(sys, r, parallel):
    """Pade electron-electron term c r/(1 + b r)."""
    c = np.where(parallel, sys.j2_par, sys.j2_anti)
    return c * r / (1.0 + sys.j2_b * r)


def jastrow(sys, x):
    """J(x) for configurations (..., n_e, 3)."""
    ne = sys.n_elec
    spin = np.arange(ne) >= sys.n_up
    J = np.zeros(x.shape[:-2])
    for i in range(ne):
        for j in range(i + 1, ne):
            r = np.linalg.norm(x[..., i, :] - x[..., j, :], axis=-1)
            J = J + pair_u(sys, r, spin[i] == spin[j])
        for I in range(sys.n_nuc):
            r = np.linalg.norm(x[..., i, :] - sys.R[I], axis=-1)
            J = J - sys.j1_A[I] * r / (1.0 + sys.j1_B[I] * r)
    return J


def jastrow_grad_lap(sys, x):
    """Per-electron grad_i J (..., n_e, 3) and lap_i J (..., n_e).

    For a radial term f(r): grad = f'(r) d/r, lap = f''(r) + 2 f'(r)/r.
      u = c r/(1+br):  u' = c/(1+br)^2,  u'' = -2bc/(1+br)^3
      v = -A r/(1+Br): v' = -A/(1+Br)^2, v'' = 2AB/(1+Br)^3
    """
    ne = sys.n_elec
    spin = np.arange(ne) >= sys.n_up
    g = np.zeros(x.shape)
    L = np.zeros(x.shape[:-1])
    b = sys.j2_b
    for i in range(ne):
        for j in range(ne):
            if j == i:
                continue
            d = x[..., i, :] - x[..., j, :]
            r = np.linalg.norm(d, axis=-1)
            c = sys.j2_par if spin[i] == spin[j] else sys.j2_anti
            up = c / (1.0 + b * r) ** 2
            upp = -2.0 * b * c / (1.0 + b * r) ** 3
            g[..., i, :] += (up / r)[..., None] * d
            L[..., i] += upp + 2.0 * up / r
        for I in range(sys.n_nuc):
            d = x[..., i, :] - sys.R[I]
            r = np.linalg.norm(d, axis=-1)
            A, B = sys.j1_A[I], sys.j1_B[I]
            vp = -A / (1.0 + B * r) ** 2
            vpp = 2.0 * A * B / (1.0 + B * r) ** 3
            g[..., i, :] += (vp / r)[..., None] * d
            L[..., i] += vpp + 2.0 * vp / r
    return g, L


def log_psi(sys, x):
    """(sign, log|Psi_G|) for configurations (..., n_e, 3)."""
    sign = np.ones(x.shape[:-2])
    logv = jastrow(sys, x)
    for A in slater_matrices(sys, x):
        s, l = _slogdet(A)
        sign = sign * s
        logv = logv + l
    return sign, logv


def hop_vector(a, d, versors=None):
    """Displacement of hop d: HOP_SIGN[d] * a along versor HOP_AXIS[d] (the
    Cartesian axes, or the rows of ``versors`` (..., 3, 3) when given)."""
    if versors is None:
        v = np.zeros(3)
        v[HOP_AXIS[d]] = HOP_SIGN[d] * a
        return v
    return HOP_SIGN[d] * a * versors[..., HOP_AXIS[d], :]


def displaced(x, a, versors=None):
    """All 6 n_e single-electron lattice hops: (..., n_e, 6, n_e, 3), hop (i, d)
    moves electron i by HOP_SIGN[d] * a along versor HOP_AXIS[d]."""
    ne = x.shape[-2]
    xd = np.broadcast_to(x[..., None, None, :, :], x.shape[:-2] + (ne, 6, ne, 3)).copy()
    for i in range(ne):
        for d in range(6):
            if versors is None:
                xd[..., i, d, i, HOP_AXIS[d]] += HOP_SIGN[d] * a
            else:
                xd[..., i, d, i, :] += hop_vector(a, d, versors)
    return xd


def hop_ratios(sys, x, a, versors=None):
    """r_{i,d} = Psi_G(x_{i,d}) / Psi_G(x) for every hop, (..., n_e, 6), each from
    freshly computed determinants and Jastrow factors."""
    s0, l0 = log_psi(sys, x)
    xd = displaced(x, a, versors)
    s1, l1 = log_psi(sys, xd)
    return (s1 * s0[..., None, None]) * np.exp(l1 - l0[..., None, None])


def local_derivatives(sys, x):
    """Per electron: grad_i Psi/Psi (..., n_e, 3) and lap_i Psi/Psi (..., n_e).

    Determinant part by row replacement: d det(A)/det(A) = det(A with row i
    replaced by d phi(r_i)) / det(A); Jastrow part analytic; combined with
    lap(DJ)/(DJ) = lap D/D + 2 grad D/D . grad J + lap J + |grad J|^2."""
    ne = sys.n_elec
    _, gchi, lchi = basis_derivs(sys, x, order=2)          # (..., ne, nbf, 3), (..., ne, nbf)
    chi = basis_values(sys, x)
    phi = chi @ sys.C.T                                      # (..., ne, norb)
    gphi = np.einsum("...ebx,kb->...ekx", gchi, sys.C)       # (..., ne, norb, 3)
    lphi = lchi @ sys.C.T                                    # (..., ne, norb)
    gD = np.zeros(x.shape)
    lD = np.zeros(x.shape[:-1])
    for start, n in spin_blocks(sys):
        if n == 0:
            continue
        A = phi[..., start:start + n, :n]
        detA = np.linalg.det(A)
        for ii in range(n):
            i = start + ii
            for m in range(3):
                Ar = A.copy()
                Ar[..., ii, :] = gphi[..., i, :n, m]
                gD[..., i, m] = np.linalg.det(Ar) / detA
            Ar = A.copy()
            Ar[..., ii, :] = lphi[..., i, :n]
            lD[..., i] = np.linalg.det(Ar) / detA
    gJ, lJ = jastrow_grad_lap(sys, x)
    grad = gD + gJ
    lap = lD + 2.0 * np.sum(gD * gJ, axis=-1) + lJ + np.sum(gJ * gJ, axis=-1)
    return grad, lap
