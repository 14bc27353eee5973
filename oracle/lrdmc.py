"""LRDMC walker propagation and reconfiguration, plain FP64 (oracle).

Load-balanced schedule (Algorithm 2, Eqs. for the modified Green's function
and the lattice update of Sec. II.C): every walker makes exactly N_proj moves;
at each step, with the evaluation at the current configuration x,
    b_x = b_bar(x) / (W(x) - E_0),   w <- w b_x,
then one hop (i, d) is drawn with probability r_{i,d} / sum_{r>0} r over the
kept hops (heat bath) and applied.

Conventional schedule (Algorithm 1, Eqs. for the persistence time and the
continuous-time weight update of Sec. II.B): with tau_left = tau,
    tau_xi = min(-ln(1 - xi) / b_bar(x), tau_left),  w <- w exp(-tau_xi e_L(x)),
    tau_left <- tau_left - tau_xi;
the walker stops when the minimum was tau_left (a flag, not a float test),
otherwise it hops as above.  A walker that reaches ``max_moves`` hops stops
with the STEP_CAP status.

After the interval each walker keeps w and the evaluation at its final
configuration (the local energy stored "after the projection").

Reconfiguration (Eqs. for the selection probability and the correlated comb
Z_alpha = (xi + alpha - 1)/N_w of Sec. II.A), integer form: weights are
quantised q_b = floor(w_b / w_max * 2^S) with S = 62 - bitlength(N_w), Q is
their inclusive prefix sum, xi32 is a 32-bit Philox word, and slot alpha
(0-based) copies the first walker b with
    (xi32 + alpha 2^32) * Q_total  <  N_w 2^32 Q_b
(exact integer comparison); afterwards every weight is 1.

Heat-bath choice: the kept hops are scanned in the order p = 6 i + d; the
first p whose running sum of kept ratios exceeds u * (their total) is taken;
if rounding leaves none, the last kept hop is taken; with no kept hop the
walker does not move (status STUCK).

Random numbers: Philox4x32-10, see ``oracle.philox`` for the stream layout.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import estimator as est
from . import hamiltonian as ham
from . import philox
from .wavefunction import HOP_AXIS, HOP_SIGN

ST_NEG_DIAG = 1      # W - E_0 <= 0 at a load-balanced step (weight set to 0)
ST_NONFINITE = 2     # non-finite weight or local energy
ST_STEP_CAP = 4      # conventional walker hit max_moves
ST_STUCK = 8         # no kept hop (b_bar = 0)

LOAD_BALANCED = 1
CONVENTIONAL = 0


@dataclasses.dataclass
class Walkers:
    x: np.ndarray          # (n_w, n_e, 3)
    w: np.ndarray          # (n_w,)
    ev: dict               # evaluation at x (ratios, bbar, vsf, W, eL, n_node, ...)
    status: np.ndarray     # (n_w,) uint32, sticky
    moves: np.ndarray      # (n_w,) hops made in the last interval
    rotated: bool = False  # ev was taken on a randomised lattice (its versors)


def rotation_matrices(u1, u2, u3):
    """Uniformly distributed rotations from three uniforms (Shoemake, "Uniform
    random rotations", Graphics Gems III, 1992): the unit quaternion
    (x, y, z, w) = (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2,
                    sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3)
    and its rotation matrix.  Returns (..., 3, 3); row k is versor k = R e_k."""
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x, y = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    z, w = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.empty(np.shape(u1) + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return np.swapaxes(R, -1, -2)          # rows = columns of R = rotated axes


def interval_versors(seed, walker_ids, interval):
    """Hop versors of the randomised lattice (Appendix D): one uniformly random
    rotation of the three axes per walker and interval."""
    return rotation_matrices(*philox.rotation_uniforms(seed, walker_ids, interval))


def init_walkers(sys, x0, a, node_rule=0):
    x = np.array(x0, dtype=np.float64, copy=True)
    ev = ham.evaluate(sys, x, a, node_rule)
    n = x.shape[0]
    return Walkers(x=x, w=np.ones(n), ev=ev, status=np.zeros(n, np.uint32),
                   moves=np.zeros(n, np.int64))


def choose_hop(ratios, u):
    """Heat-bath hop index p in 0..6 n_e - 1 per walker (-1 if no kept hop).

    The running sum is the sequential prefix sum over p (numpy's cumsum adds
    left to right), its last entry is the total."""
    n = ratios.shape[0]
    kept = np.where(ratios.reshape(n, -1) > 0.0, ratios.reshape(n, -1), 0.0)
    run = np.cumsum(kept, axis=1)
    total = run[:, -1]
    t = np.asarray(u) * total
    hit = run > t[:, None]
    first = np.argmax(hit, axis=1)
    npos = kept.shape[1]
    last_kept = npos - 1 - np.argmax((kept > 0.0)[:, ::-1], axis=1)
    out = np.where(hit.any(axis=1), first, last_kept)
    return np.where(total > 0.0, out, -1).astype(np.int64)


def _apply_hops(W: Walkers, sel, hop, a, versors=None):
    """Move walkers ``sel`` (indices) by hops ``hop`` (same length)."""
    i = hop // 6
    d = hop % 6
    if versors is None:
        W.x[sel, i, HOP_AXIS[d]] += HOP_SIGN[d] * a
    else:
        for k in range(len(sel)):
            W.x[sel[k], i[k], :] += HOP_SIGN[d[k]] * a * versors[sel[k], HOP_AXIS[d[k]], :]


def _reevaluate(sys, W: Walkers, sel, a, node_rule, versors=None):
    if len(sel) == 0:
        return
    ev = ham.evaluate(sys, W.x[sel], a, node_rule, None if versors is None else versors[sel])
    for k, v in ev.items():
        W.ev[k][sel] = v


def _rotate(sys, W: Walkers, a, node_rule, seed, interval, ids, rotate):
    """With a randomised lattice, draw this interval's versors and re-evaluate
    every walker with them (the stored evaluation used the previous axes).  On
    the fixed lattice, an evaluation left by a randomised interval is redone
    on the Cartesian axes."""
    if not rotate:
        if W.rotated:
            _reevaluate(sys, W, np.arange(W.x.shape[0]), a, node_rule, None)
            W.rotated = False
        return None
    V = interval_versors(seed, ids, interval)
    _reevaluate(sys, W, np.arange(W.x.shape[0]), a, node_rule, V)
    W.rotated = True
    return V


def propagate_lb(sys, W: Walkers, a, E0, n_proj, seed, interval, node_rule=0, walker_ids=None, rotate=False):
    """One load-balanced interval (Algorithm 2, inner loop) for all walkers.
    ``walker_ids``: Philox walker slots of the rows of W (default 0..n-1).
    ``rotate``: randomised lattice, hop versors redrawn for the interval."""
    n = W.x.shape[0]
    ids = np.arange(n) if walker_ids is None else np.asarray(walker_ids)
    V = _rotate(sys, W, a, node_rule, seed, interval, ids, rotate)
    W.w = np.ones(n)
    W.moves = np.zeros(n, np.int64)
    for k in range(n_proj):
        denom = W.ev["W"] - E0
        bad = ~(denom > 0.0)
        b = np.where(bad, 0.0, W.ev["bbar"] / np.where(bad, 1.0, denom))
        W.status |= np.where(bad, ST_NEG_DIAG, 0).astype(np.uint32)
        W.w = W.w * b
        _, u_move = philox.step_uniforms(seed, ids, k, interval)
        hop = choose_hop(W.ev["ratios"], u_move)
        W.status |= np.where(hop < 0, ST_STUCK, 0).astype(np.uint32)
        sel = np.nonzero(hop >= 0)[0]
        _apply_hops(W, sel, hop[sel], a, V)
        W.moves[sel] += 1
        _reevaluate(sys, W, sel, a, node_rule, V)
    W.status |= np.where(~np.isfinite(W.w) | ~np.isfinite(W.ev["eL"]), ST_NONFINITE, 0).astype(np.uint32)


def propagate_conventional(sys, W: Walkers, a, tau, seed, interval, node_rule=0,
                           max_moves=100000, walker_ids=None, rotate=False):
    """One conventional interval (Algorithm 1, inner loop) for all walkers.
    ``walker_ids``: Philox walker slots of the rows of W (default 0..n-1).
    ``rotate``: randomised lattice, hop versors redrawn for the interval."""
    n = W.x.shape[0]
    ids = np.arange(n) if walker_ids is None else np.asarray(walker_ids)
    V = _rotate(sys, W, a, node_rule, seed, interval, ids, rotate)
    W.w = np.ones(n)
    W.moves = np.zeros(n, np.int64)
    tau_left = np.full(n, float(tau))
    active = np.ones(n, dtype=bool)
    k = 0
    while np.any(active):
        act = np.nonzero(active)[0]
        u_tau, u_move = philox.step_uniforms(seed, ids[act], k, interval)
        bbar = W.ev["bbar"][act]
        with np.errstate(divide="ignore"):
            t = -np.log(1.0 - u_tau) / bbar
        clipped = ~(t < tau_left[act])
        t = np.where(clipped, tau_left[act], t)
        W.w[act] = W.w[act] * np.exp(-t * W.ev["eL"][act])
        tau_left[act] = tau_left[act] - t
        done = act[clipped]
        active[done] = False
        go = act[~clipped]
        if len(go):
            hop = choose_hop(W.ev["ratios"][go], u_move[~clipped])
            W.status[go] |= np.where(hop < 0, ST_STUCK, 0).astype(np.uint32)
            ok = hop >= 0
            _apply_hops(W, go[ok], hop[ok], a, V)
            W.moves[go[ok]] += 1
            _reevaluate(sys, W, go[ok], a, node_rule, V)
        k += 1
        if k >= max_moves and np.any(active):
            cap = np.nonzero(active)[0]
            W.status[cap] |= ST_STEP_CAP
            active[cap] = False
    W.status |= np.where(~np.isfinite(W.w) | ~np.isfinite(W.ev["eL"]), ST_NONFINITE, 0).astype(np.uint32)


def quant_shift(n_w: int) -> int:
    return 62 - int(n_w).bit_length()


def reconfigure_indices(w, xi32: int):
    """Source index s(alpha) for every slot alpha (integer comb, exact)."""
    w = np.asarray(w, dtype=np.float64)
    n = len(w)
    if n == 0:
        return np.zeros(0, np.int64)
    wmax = float(np.max(w))
    if not (wmax > 0.0) or not np.all(np.isfinite(w)) or np.any(w < 0.0):
        raise ValueError("weights must be finite, non-negative, not all zero")
    S = quant_shift(n)
    scale = float(2 ** S)
    q = [int(np.floor((wb / wmax) * scale)) for wb in w]
    Q = []
    acc = 0
    for v in q:
        acc += v
        Q.append(acc)
    tot = Q[-1]
    src = np.zeros(n, np.int64)
    b = 0
    for alpha in range(n):
        lhs = (int(xi32) + alpha * (1 << 32)) * tot
        while not (lhs < n * (1 << 32) * Q[b]):
            b += 1
        src[alpha] = b
    return src


def branch_stats(W: Walkers, E0, schedule):
    """(wbar, ebar) before reconfiguration: Eq. for the walker-averaged local
    energy (conventional, weights w) or its load-balanced form (weights
    w / (W(x) - E_0)).  The averages run over the walkers of the population:
    a walker of zero weight (the load-balanced step sets w = 0 where
    W - E_0 <= 0) carries no weight and contributes nothing, also when its
    e_L or W is not finite."""
    w = W.w
    wbar = float(np.sum(w)) / len(w)
    live = w != 0.0
    wl = w[live]
    if schedule == LOAD_BALANCED:
        f = wl / (W.ev["W"][live] - E0)
    else:
        f = wl
    ebar = float(np.sum(f * W.ev["eL"][live]) / np.sum(f))
    return wbar, ebar


def slot_assignment(src):
    """Slot of every copy of the reconfigured population.  The comb of
    Sec. II.A fixes how many copies each walker gets, not where they are
    stored; here each selected walker keeps its own slot for its first copy,
    and its further copies, taken in the comb's order alpha, fill the slots of
    the walkers that were not selected, in increasing slot order.  Returns
    slot -> source walker."""
    src = np.asarray(src, dtype=np.int64)
    n = len(src)
    out = np.arange(n, dtype=np.int64)
    if n == 0:
        return out
    selected = np.zeros(n, bool)
    selected[src] = True
    free = np.flatnonzero(~selected)
    extra = src[1:][src[1:] == src[:-1]]
    assert len(extra) == len(free)
    out[free] = extra
    return out


def reconfigure(W: Walkers, seed, interval):
    """Integer comb, then the copies stored by ``slot_assignment``; returns the
    comb's source indices."""
    xi32 = philox.branch_offset32(seed, interval)
    src = reconfigure_indices(W.w, xi32)
    slot = slot_assignment(src)
    W.x = W.x[slot].copy()
    W.ev = {k: v[slot].copy() for k, v in W.ev.items()}
    W.status = W.status[slot].copy()
    W.moves = W.moves[slot].copy()
    W.w = np.ones(len(src))
    return src


@dataclasses.dataclass
class RunResult:
    wbar: list
    ebar: list
    e0: list
    survivors: list
    moves_mean: list
    moves_max: list
    status_or: int
    energy: float
    error: float


def run(sys, x0, a, schedule, n_branch, seed, n_proj=20, tau=None, node_rule=0,
        p_gbar=10, n_equil=0, E0=None, max_moves=100000, rotate=False):
    """Full oracle run (both algorithms' outer loop)."""
    W = init_walkers(sys, x0, a, node_rule)
    if E0 is None:
        E0 = float(np.mean(W.ev["eL"]))
    hist = RunResult([], [], [], [], [], [], 0, float("nan"), float("nan"))
    for j in range(n_branch):
        if schedule == LOAD_BALANCED:
            propagate_lb(sys, W, a, E0, n_proj, seed, j, node_rule, rotate=rotate)
        else:
            propagate_conventional(sys, W, a, tau, seed, j, node_rule, max_moves, rotate=rotate)
        wbar, ebar = branch_stats(W, E0, schedule)
        hist.wbar.append(wbar)
        hist.ebar.append(ebar)
        hist.e0.append(E0)
        hist.moves_mean.append(float(np.mean(W.moves)))
        hist.moves_max.append(int(np.max(W.moves)))
        hist.status_or |= int(np.bitwise_or.reduce(W.status))
        src = reconfigure(W, seed, j)
        hist.survivors.append(int(len(np.unique(src))))
        if schedule == LOAD_BALANCED:
            E0 = est.energy(hist.wbar, hist.ebar, p_gbar, 0)
    hist.energy = est.energy(hist.wbar, hist.ebar, p_gbar, n_equil)
    hist.error = est.energy_error(hist.wbar, hist.ebar, p_gbar, n_equil)
    return hist, W
