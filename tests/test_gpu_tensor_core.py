"""Tensor-core forms of the mixed path (precision 2: TF32, 3: BF16, 4: split
TF32) against the FP64 oracle, with error bounds derived from the operand
rounding.

The tensor cores take the two FP32 orbital contractions against the MO
coefficients C: the orbital differences of a hop, dphi_k = sum_mu C_k,mu
dchi_mu (dchi = chi(r') - chi(r_i)), and the gradient / Laplacian rows
sum_mu C_k,mu d chi_mu(r_i).  With both operands rounded to a format of unit
roundoff u (TF32: 11 significant bits, u = 2^-11; BF16: 8 bits, u = 2^-8) each
product carries a relative error of at most 2u + u^2, so
    |d dphi_k| <= (2u + u^2) sum_mu |C_k,mu| |dchi_mu|,
and the hop's determinant ratio minus one, D = sum_k dphi_k B_k,i, carries at
most (2u + u^2) S_p with S_p = sum_k |B_k,i| sum_mu |C_k,mu| |dchi_mu|; the
ratio r = (1 + D)(1 + J) carries that times |1 + J| (J the Jastrow factor minus
one).  The split form (hi + lo parts, three products) leaves about 3u^2 per
product.  On top comes the FP32 error of precision 1 (1e-4 max(1, |r|), derived
in test_gpu_mixed.py).  The local energy takes each ratio with a weight of at
most 1/a^2 (b_bar, V_sf and the discrete Laplacian of nu_zv) and the analytic
Laplacian L_i with weight 1/2, whose determinant part carries
(2u + u^2) sum_k |B_k,i| sum_mu |C_k,mu| (|lap chi_mu| + 2 |grad J_i| |grad chi_mu|).
A wrong fragment layout or a dropped k-step gives errors of order S_p itself,
far outside these bounds."""
import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as H
from oracle import wavefunction as WF

pytestmark = pytest.mark.gpu

U = {2: 2.0 ** -11, 3: 2.0 ** -8}


def _product_error(precision):
    if precision == 4:
        u = 2.0 ** -11
        return 3 * u * u + 2.0 ** -22
    u = U[precision]
    return 2 * u + u * u


def _bounds(s, x, a, precision):
    """Per-hop ratio bounds and per-configuration e_L bounds (see the module
    docstring), from the oracle's basis values, orbitals and Jastrow."""
    n, ne = x.shape[0], s.n_elec
    eps = _product_error(precision)
    absC = np.abs(s.C)
    chi, gchi, lchi = WF.basis_derivs(s, x.reshape(-1, 3))
    chi = chi.reshape(n, ne, -1)
    gchi = gchi.reshape(n, ne, 3, -1)
    lchi = np.abs(lchi.reshape(n, ne, -1))
    xd = WF.displaced(x, a)                                   # (n, ne, 6, ne, 3)
    moved = xd[:, np.arange(ne), :, np.arange(ne), :]          # (ne, n, 6, 3)
    chid = WF.basis_values(s, moved.reshape(-1, 3)).reshape(ne, n, 6, -1).transpose(1, 0, 2, 3)
    dchi = np.abs(chid - chi[:, :, None, :])                  # (n, ne, 6, n_bf)
    gJ, _ = WF.jastrow_grad_lap(s, x)                          # (n, ne, 3)
    J0 = WF.jastrow(s, x)
    Jd = WF.jastrow(s, xd.reshape(-1, ne, 3)).reshape(n, ne, 6)
    onepJ = np.exp(Jd - J0[:, None, None])
    rat_b = np.zeros((n, ne, 6))
    lap_b = np.zeros((n, ne))
    for e0, ns in WF.spin_blocks(s):
        if ns == 0:
            continue
        A = WF.orbitals(s, x[:, e0:e0 + ns].reshape(-1, 3)).reshape(n, ns, -1)[:, :, :ns]
        B = np.linalg.inv(A)                                   # B[k, ii]: (A^-1)[k, ii]
        cd = np.einsum("km,neDm->neDk", absC[:ns], dchi[:, e0:e0 + ns])   # sum_mu |C_k,mu| |dchi_mu|
        Bi = np.abs(B)                                         # (n, k, ii)
        S = np.einsum("neDk,nke->neD", cd, Bi)
        rat_b[:, e0:e0 + ns] = eps * S * onepJ[:, e0:e0 + ns]
        gterm = np.einsum("nec,necm->nem", np.abs(gJ[:, e0:e0 + ns]), np.abs(gchi[:, e0:e0 + ns]))
        cl = np.einsum("km,nem->nek", absC[:ns], lchi[:, e0:e0 + ns] + 2 * gterm)
        lap_b[:, e0:e0 + ns] = eps * np.einsum("nek,nke->ne", cl, Bi)
    el_b = np.sum(rat_b, axis=(1, 2)) / a ** 2 + 0.5 * np.sum(lap_b, axis=1)
    return rat_b.reshape(n, 6 * ne), el_b


@pytest.mark.parametrize("precision", [2, 3, 4])
@pytest.mark.parametrize("name,sysf,n,el_fp32", [
    ("h2", W.h2_sto3g, 128, 2e-5),
    ("wm", W.water_methane, 128, 1e-2),
    ("h24", lambda: W.hydrogen_cluster(24, seed=5), 32, 2e-2)])
def test_tensor_core_eval_within_rounding_bounds(precision, name, sysf, n, el_fp32):
    import torch
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = sysf()
    a = 0.2
    x = W.initial_walkers(s, n, seed=77)
    lr = P.Lrdmc(s, W.initial_walkers(s, n, seed=3), a, precision=precision)
    ratios, ev, _ = lr.eval_configs(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ref = H.evaluate(s, x, a)
    rat_b, el_b = _bounds(s, x, a, precision)
    r = ratios.cpu().numpy().reshape(n, -1)
    rref = ref["ratios"].reshape(n, -1)            # hop p = 6 i + d
    err = np.abs(r - rref)
    allowed = 1.5 * rat_b + 1e-4 * np.maximum(1.0, np.abs(rref))
    assert np.all(err <= allowed), (float(np.max(err / allowed)), name, precision)
    de = np.abs(ev[:, 3].cpu().numpy() - ref["eL"])
    assert np.all(de <= 1.5 * el_b + el_fp32), (float(np.max(de / (1.5 * el_b + el_fp32))), name, precision)
    lr.close()


def test_split_tf32_keeps_the_mixed_energy_bias():
    """Split TF32 (precision 4): the local energies of 256 water-methane
    configurations stay within the FP32 bound of precision 1 and their mean
    differs from the oracle's by less than 0.1 mHa."""
    import torch
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.water_methane()
    x = W.initial_walkers(s, 256, seed=78)
    lr = P.Lrdmc(s, W.initial_walkers(s, 256, seed=3), 0.2, precision=4)
    _, ev, _ = lr.eval_configs(torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ref = H.evaluate(s, x, 0.2)
    d = ev[:, 3].cpu().numpy() - ref["eL"]
    assert np.max(np.abs(d)) <= 1e-2
    assert abs(np.mean(d)) <= 1e-4


@pytest.mark.parametrize("precision", [2, 3, 4])
def test_tensor_core_interval_runs_and_tracks_fp64(precision):
    """Same start and random streams as the FP64 path: a 20-hop load-balanced
    interval of 512 water-methane walkers keeps most trajectories (the split
    form as many as precision 1: >= 95 %; TF32 / BF16 ratios are coarser, so
    more hop choices flip) and gives finite weights."""
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    s = W.water_methane()
    x0 = W.initial_walkers(s, 512, seed=21)
    g = {}
    for prec in (0, precision):
        lr = P.Lrdmc(s, x0, 0.2, seed=4, precision=prec, reinv_period=50)
        lr.e0 = -20.0
        lr.propagate(P.LOAD_BALANCED, n_proj=20)
        g[prec] = lr.get_walkers()
        lr.close()
    same = np.all(g[0]["x"] == g[precision]["x"], axis=(1, 2))
    assert np.all(np.isfinite(g[precision]["w"]))
    assert same.mean() >= {2: 0.5, 3: 0.3, 4: 0.95}[precision]
