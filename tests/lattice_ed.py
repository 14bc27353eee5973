"""Exact diagonalisation of the one-electron fixed-node lattice Hamiltonian
with a nodal guiding function (test infrastructure; built from the paper's
definitions, not from the oracle).

Hydrogen atom (bare proton at the origin), guiding function
Psi(r) = z exp(-beta r^2), whose nodal plane z = 0 is the node of the exact 2p
states.  Sites a (n + 1/2) of an L^3 box (no site on the node).  Appendix D:
kinetic hops to the six neighbours with H_{x',x} = -1/(2a^2); a hop whose ratio
Psi(x')/Psi(x) is negative crosses the node and is removed, its |ratio|/(2a^2)
added to the diagonal as V_sf; the diagonal is
    W(x) = 3/a^2 + nu_opt(x) + V_sf(x),
    nu_zv = -1/r + [ (sum_d Psi(x_d)/Psi(x) - 6)/a^2 - lap Psi/Psi ] / 2,
    nu_opt = max(nu_zv, -1/max(r, a)) where a hop crosses the node, else nu_zv,
with lap Psi / Psi = 4 beta^2 r^2 - 10 beta for this Gaussian p function.  The
six ratios and V_sf are those of the infinite lattice (as a walker sees them);
the box only truncates the hops, with a zero boundary.  Its lowest eigenvalue
is the energy the LRDMC projection converges to on this lattice; as a -> 0 it
tends to the exact 2p energy, -1/8 Ha."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def pz_psi(beta, x, y, z):
    return z * np.exp(-beta * (x * x + y * y + z * z))


def pz_site_terms(beta, a, X, Y, Z):
    """Per-site pieces of H^a at positions (X, Y, Z): (sum of kept ratios,
    V_sf, W, node flag)."""
    r = np.sqrt(X * X + Y * Y + Z * Z)
    p0 = pz_psi(beta, X, Y, Z)
    rs = np.zeros_like(r)
    kept = np.zeros_like(r)
    vsf = np.zeros_like(r)
    node = np.zeros(r.shape, bool)
    for ax in range(3):
        for sg in (1.0, -1.0):
            d = [X.copy(), Y.copy(), Z.copy()]
            d[ax] = d[ax] + sg * a
            rat = pz_psi(beta, *d) / p0
            rs += rat
            kept += np.where(rat > 0, rat, 0.0)
            vsf += np.where(rat < 0, -rat, 0.0) / (2 * a * a)
            node |= rat < 0
    nu_zv = -1.0 / r + 0.5 * ((rs - 6.0) / (a * a) - (4 * beta * beta * r * r - 10 * beta))
    nu_opt = np.where(node, np.maximum(nu_zv, -1.0 / np.maximum(r, a)), nu_zv)
    W = 3.0 / (a * a) + nu_opt + vsf
    return kept, vsf, W, node


def pz_lattice_ground_energy(beta, a, L_side):
    n1 = np.arange(L_side) - L_side // 2
    c = a * (n1 + 0.5)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    _, _, W, _ = pz_site_terms(beta, a, X, Y, Z)
    N = L_side ** 3
    idx = np.arange(N).reshape(L_side, L_side, L_side)
    rows, cols = [], []
    zf = Z.ravel()
    for ax in range(3):
        a0 = [slice(None)] * 3
        a1 = [slice(None)] * 3
        a0[ax] = slice(0, L_side - 1)
        a1[ax] = slice(1, L_side)
        i0, i1 = idx[tuple(a0)].ravel(), idx[tuple(a1)].ravel()
        keep = zf[i0] * zf[i1] > 0            # same side of the node: positive ratio
        rows.append(i0[keep])
        cols.append(i1[keep])
    rr = np.concatenate(rows)
    cc = np.concatenate(cols)
    off = -1.0 / (2 * a * a)
    H = sp.coo_matrix((np.full(2 * len(rr), off), (np.concatenate([rr, cc]), np.concatenate([cc, rr]))),
                      shape=(N, N)).tocsr() + sp.diags(W.ravel())
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-10)[0][0])
