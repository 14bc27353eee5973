"""Gradients of the local energy and of log|Psi_G| with respect to the nuclear
coordinates and the Jastrow parameters (oracle, test infrastructure).

The lattice-regularised local energy e_L = W - b_bar of Appendix D and
log|Psi_G| are restated here with PyTorch CPU tensors in float64, from the same
definitions as ``oracle.hamiltonian.evaluate`` and ``oracle.wavefunction``:
fresh determinants for every hop ratio, row-replaced determinants for the
per-electron determinant derivatives, closed-form radial derivatives for the
basis functions and the Jastrow factor, and the fixed-node split, regularised
potential and node rules of Appendix D.  The gradients are taken by autograd
(reverse mode) through these definitions; nothing in this module knows how
the GPU path differentiates.

Parameters, in this order (the flat vector ``theta``):
  R (n_nuc x 3), j2_anti, j2_par, j2_b, j1_A (n_nuc), j1_B (n_nuc).
"""
from __future__ import annotations

import numpy as np
import torch

HOP_AXIS = (0, 0, 1, 1, 2, 2)
HOP_SIGN = (1.0, -1.0, 1.0, -1.0, 1.0, -1.0)


def pack(sys):
    """The parameter vector of a system."""
    return np.concatenate([sys.R.reshape(-1), [sys.j2_anti, sys.j2_par, sys.j2_b], sys.j1_A, sys.j1_B])


def unpack(sys, theta):
    nn = sys.n_nuc
    R = theta[:3 * nn].reshape(nn, 3)
    return R, theta[3 * nn], theta[3 * nn + 1], theta[3 * nn + 2], theta[3 * nn + 3:4 * nn + 3], theta[4 * nn + 3:]


def _basis(sys, R, pts, derivs):
    """Basis values (and with derivs: gradients and Laplacians) at pts (..., 3)."""
    off = np.concatenate([[0], np.cumsum(sys.shell_nprim)]).astype(int)
    chi, grad, lap = [], [], []
    for s in range(sys.n_shell):
        d = pts - R[int(sys.shell_atom[s])]
        r2 = (d * d).sum(-1)
        l = int(sys.shell_l[s])
        ex = [float(e) for e in sys.exps[off[s]:off[s + 1]]]
        co = [float(c) for c in sys.coefs[off[s]:off[s + 1]]]
        if l == -1:
            r = torch.sqrt(r2)
            fs = [c * torch.exp(-z * r) for z, c in zip(ex, co)]
            chi.append(sum(fs))
            if derivs:
                fp = sum(-z * f for z, f in zip(ex, fs))
                grad.append((fp / r)[..., None] * d)
                lap.append(sum((z * z - 2.0 * z / r) * f for z, f in zip(ex, fs)))
            continue
        hs = [c * torch.exp(-a * r2) for a, c in zip(ex, co)]
        if l == 0:
            chi.append(sum(hs))
            if derivs:
                grad.append(sum((-2.0 * a) * h[..., None] * d for a, h in zip(ex, hs)))
                lap.append(sum((4.0 * a * a * r2 - 6.0 * a) * h for a, h in zip(ex, hs)))
        else:
            for m in range(3):
                chi.append(d[..., m] * sum(hs))
                if derivs:
                    e_m = torch.zeros(3, dtype=pts.dtype)
                    e_m[m] = 1.0
                    grad.append(sum(h[..., None] * (e_m - 2.0 * a * d[..., m:m + 1] * d) for a, h in zip(ex, hs)))
                    lap.append(sum(d[..., m] * (4.0 * a * a * r2 - 10.0 * a) * h for a, h in zip(ex, hs)))
    chi = torch.stack(chi, -1)
    if not derivs:
        return chi
    return chi, torch.stack(grad, -2), torch.stack(lap, -1)


def _pair_terms(sys, c_anti, c_par, b, x):
    """Pair Jastrow sum J_ee(x) for configurations (..., n_e, 3)."""
    ne = sys.n_up + sys.n_dn
    J = torch.zeros(x.shape[:-2], dtype=x.dtype)
    for i in range(ne):
        for j in range(i + 1, ne):
            r = torch.linalg.norm(x[..., i, :] - x[..., j, :], dim=-1)
            c = c_par if (i < sys.n_up) == (j < sys.n_up) else c_anti
            J = J + c * r / (1.0 + b * r)
    return J


def _one_body(R, A, B, x):
    d = x[..., :, None, :] - R
    r = torch.linalg.norm(d, dim=-1)
    return (-A * r / (1.0 + B * r)).sum((-1, -2))


def log_psi(sys, theta, x):
    """(sign, log|Psi_G|) at configurations x (..., n_e, 3)."""
    R, ca, cp, b, A, B = unpack(sys, theta)
    phi = _basis(sys, R, x, False) @ torch.as_tensor(sys.C, dtype=x.dtype).T
    sign = torch.ones(x.shape[:-2], dtype=x.dtype)
    logv = _pair_terms(sys, ca, cp, b, x) + _one_body(R, A, B, x)
    for start, n in ((0, sys.n_up), (sys.n_up, sys.n_dn)):
        if n == 0:
            continue
        s, l = torch.linalg.slogdet(phi[..., start:start + n, :n])
        sign = sign * s
        logv = logv + l
    return sign, logv


def _local_lap(sys, theta, x):
    """lap_i Psi / Psi per electron (row-replaced determinants + analytic Jastrow)."""
    R, ca, cp, b, A, B = unpack(sys, theta)
    Ct = torch.as_tensor(sys.C, dtype=x.dtype)
    chi, gchi, lchi = _basis(sys, R, x, True)
    phi = chi @ Ct.T
    gphi = torch.einsum("...ebx,kb->...ekx", gchi, Ct)
    lphi = lchi @ Ct.T
    ne = sys.n_up + sys.n_dn
    gD = [None] * ne
    lD = [None] * ne
    for start, n in ((0, sys.n_up), (sys.n_up, sys.n_dn)):
        if n == 0:
            continue
        Am = phi[..., start:start + n, :n]
        det = torch.linalg.det(Am)
        for ii in range(n):
            i = start + ii
            g = []
            for m in range(3):
                rows = [gphi[..., i, :n, m] if q == ii else Am[..., q, :] for q in range(n)]
                g.append(torch.linalg.det(torch.stack(rows, -2)) / det)
            gD[i] = torch.stack(g, -1)
            rows = [lphi[..., i, :n] if q == ii else Am[..., q, :] for q in range(n)]
            lD[i] = torch.linalg.det(torch.stack(rows, -2)) / det
    laps = []
    for i in range(ne):
        gJ = torch.zeros(x.shape[:-2] + (3,), dtype=x.dtype)
        lJ = torch.zeros(x.shape[:-2], dtype=x.dtype)
        for j in range(ne):
            if j == i:
                continue
            d = x[..., i, :] - x[..., j, :]
            r = torch.linalg.norm(d, dim=-1)
            c = cp if (i < sys.n_up) == (j < sys.n_up) else ca
            up = c / (1.0 + b * r) ** 2
            upp = -2.0 * b * c / (1.0 + b * r) ** 3
            gJ = gJ + (up / r)[..., None] * d
            lJ = lJ + upp + 2.0 * up / r
        for I in range(sys.n_nuc):
            d = x[..., i, :] - R[I]
            r = torch.linalg.norm(d, dim=-1)
            vp = -A[I] / (1.0 + B[I] * r) ** 2
            vpp = 2.0 * A[I] * B[I] / (1.0 + B[I] * r) ** 3
            gJ = gJ + (vp / r)[..., None] * d
            lJ = lJ + vpp + 2.0 * vp / r
        laps.append(lD[i] + 2.0 * (gD[i] * gJ).sum(-1) + lJ + (gJ * gJ).sum(-1))
    return torch.stack(laps, -1)


def _potentials(sys, R, x, a):
    """nu_ei and nu^a_ei per electron (Appendix D)."""
    nu = torch.zeros(x.shape[:-1], dtype=x.dtype)
    cap = torch.zeros(x.shape[:-1], dtype=x.dtype)
    for I in range(sys.n_nuc):
        r = torch.linalg.norm(x - R[I], dim=-1)
        Z = float(sys.Z[I])
        if int(sys.pot_kind[I]) == 0:
            nu = nu - Z / r
            cap = cap - Z / torch.clamp(r, min=a)
        else:
            v = -Z * torch.special.erf(r / float(sys.r_c[I])) / r
            nu = nu + v
            cap = cap + v
    return nu, cap


def local_energy(sys, theta, x, a, node_rule=0):
    """e_L = W - b_bar at configurations x (..., n_e, 3) (Appendix D)."""
    R, ca, cp, b, A, B = unpack(sys, theta)
    ne = sys.n_up + sys.n_dn
    s0, l0 = log_psi(sys, theta, x)
    ratios = []
    for i in range(ne):
        row = []
        for d in range(6):
            xd = x.clone()
            xd[..., i, HOP_AXIS[d]] = xd[..., i, HOP_AXIS[d]] + HOP_SIGN[d] * a
            s1, l1 = log_psi(sys, theta, xd)
            row.append(s1 * s0 * torch.exp(l1 - l0))
        ratios.append(torch.stack(row, -1))
    r = torch.stack(ratios, -2)                                   # (..., ne, 6)
    inv2a2 = 1.0 / (2.0 * a * a)
    bbar = torch.where(r > 0, r, torch.zeros_like(r)).sum((-1, -2)) * inv2a2
    vsf = torch.where(r < 0, -r, torch.zeros_like(r)).sum((-1, -2)) * inv2a2
    lap = _local_lap(sys, theta, x)
    nu, cap = _potentials(sys, R, x, a)
    nu_zv = nu + 0.5 * ((r.sum(-1) - 6.0) / (a * a) - lap)
    node = (r < 0).any(-1)
    if node_rule == 0:
        apply = node
    elif node_rule == 1:
        apply = node.any(-1, keepdim=True).expand_as(node)
    elif node_rule == 2:
        apply = torch.ones_like(node)
    else:
        apply = torch.zeros_like(node)
    nu_opt = torch.where(apply, torch.maximum(nu_zv, cap), nu_zv)
    vee = torch.zeros(x.shape[:-2], dtype=x.dtype)
    for i in range(ne):
        for j in range(i + 1, ne):
            vee = vee + 1.0 / torch.linalg.norm(x[..., i, :] - x[..., j, :], dim=-1)
    vii = torch.zeros((), dtype=x.dtype)
    for I in range(sys.n_nuc):
        for J in range(I + 1, sys.n_nuc):
            vii = vii + float(sys.Z[I] * sys.Z[J]) / torch.linalg.norm(R[I] - R[J])
    W = 3.0 * ne / (a * a) + nu_opt.sum(-1) + vee + vii + vsf
    return W - bbar


def gradients(sys, x, a, node_rule=0):
    """Per configuration: e_L, log|Psi|, d e_L / d theta and d log|Psi| / d theta
    (numpy arrays; x (n, n_e, 3))."""
    th = torch.tensor(pack(sys), dtype=torch.float64)
    out_e, out_l, ge, gl = [], [], [], []
    for k in range(x.shape[0]):
        t = th.clone().requires_grad_(True)
        xk = torch.tensor(x[k], dtype=torch.float64)
        e = local_energy(sys, t, xk, a, node_rule)
        (g,) = torch.autograd.grad(e, t)
        t2 = th.clone().requires_grad_(True)
        _, lp = log_psi(sys, t2, xk)
        (h,) = torch.autograd.grad(lp, t2)
        out_e.append(float(e.detach()))
        out_l.append(float(lp.detach()))
        ge.append(g.numpy())
        gl.append(h.numpy())
    return np.array(out_e), np.array(out_l), np.array(ge), np.array(gl)
