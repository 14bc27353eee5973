"""ctypes binding of liblrdmc.so (argument marshalling only).

Device memory comes from PyTorch's caching allocator (the handle's workspace
and every device buffer passed to the library are torch tensors) and work is
enqueued on a torch CUDA stream; all computation happens in the library's
kernels.  Names follow the C ABI in include/lrdmc.h.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LOAD_BALANCED = 1
CONVENTIONAL = 0

_LIB = None
# LRDMC_CHECKED=1 in the environment selects the checked build (every
# data-derived kernel index tested; see lrdmc_check_word in lrdmc.h)
_LIBPATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "liblrdmc_checked.so" if os.environ.get("LRDMC_CHECKED") == "1" else "liblrdmc.so")

c_double_p = C.POINTER(C.c_double)
c_int_p = C.POINTER(C.c_int)


class _System(C.Structure):
    _fields_ = [("n_nuc", C.c_int), ("R", c_double_p), ("Z", c_double_p), ("pot_kind", c_int_p),
                ("r_c", c_double_p), ("n_up", C.c_int), ("n_dn", C.c_int)]


class _TrialWF(C.Structure):
    _fields_ = [("n_shell", C.c_int), ("shell_atom", c_int_p), ("shell_l", c_int_p),
                ("shell_nprim", c_int_p), ("exps", c_double_p), ("coefs", c_double_p),
                ("n_orb", C.c_int), ("C", c_double_p), ("j2_anti", C.c_double),
                ("j2_par", C.c_double), ("j2_b", C.c_double), ("j1_A", c_double_p),
                ("j1_B", c_double_p)]


class _Schedule(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_proj", C.c_int), ("tau", C.c_double), ("max_moves", C.c_int),
                ("rotate", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("a", C.c_double), ("n_w", C.c_int), ("seed", C.c_uint64), ("node_rule", C.c_int),
                ("reinv_period", C.c_int), ("p_gbar", C.c_int), ("n_equil", C.c_int),
                ("precision", C.c_int)]


class LrdmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lrdmc status {status}: {msg}")
        self.status = status


def load_library():
    """Load liblrdmc.so from the package directory (raises if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_LIBPATH):
        raise RuntimeError(f"{_LIBPATH} is missing: build it with paper_2508_12033_b300.build.build()")
    lib = C.CDLL(_LIBPATH)
    P = C.c_void_p
    sigs = {
        "lrdmc_workspace_bytes": [C.POINTER(_System), C.POINTER(_TrialWF), C.POINTER(_Params), C.POINTER(C.c_size_t)],
        "lrdmc_create": [C.POINTER(_System), C.POINTER(_TrialWF), C.POINTER(_Params), c_double_p, P, C.c_size_t,
                         P, C.POINTER(P)],
        "lrdmc_destroy": [P],
        "lrdmc_propagate": [P, C.POINTER(_Schedule)],
        "lrdmc_branch": [P],
        "lrdmc_energy": [P, c_double_p, c_double_p],
        "lrdmc_history": [P, C.c_int, c_int_p, c_double_p, c_double_p, c_double_p, c_double_p, c_int_p, c_int_p,
                          C.POINTER(C.c_uint32)],
        "lrdmc_get_e0": [P, c_double_p],
        "lrdmc_set_e0": [P, C.c_double],
        "lrdmc_get_walkers": [P, c_double_p, c_double_p, c_double_p, c_double_p, C.POINTER(C.c_uint32),
                              C.POINTER(C.c_int32)],
        "lrdmc_set_walkers": [P, c_double_p, c_double_p],
        "lrdmc_clear_status": [P],
        "lrdmc_eval_configs": [P, C.c_int, P, P, P, P],
        "lrdmc_reconfigure_indices": [C.c_int, P, C.c_uint32, P, P, C.c_size_t, P, P],
        "lrdmc_launch_count": [P, C.POINTER(C.c_int64)],
        "lrdmc_save": [P, C.c_char_p],
        "lrdmc_set_timing": [P, C.c_int],
        "lrdmc_interval_timing": [P, c_double_p],
        "lrdmc_load": [P, C.c_char_p],
        "lrdmc_stream": [P, C.POINTER(P)],
        "lrdmc_checked_build": [],
        "lrdmc_check_word": [C.POINTER(C.c_uint64), C.c_int],
        "lrdmc_check_selftest": [C.c_int, C.c_int, c_int_p],
        "lrdmc_set_drift_tol": [P, C.c_double],
        "lrdmc_drift_reinversions": [P, C.POINTER(C.c_int64)],
        "lrdmc_estimate": [C.c_int, c_double_p, c_double_p, C.c_int, C.c_int, c_double_p, c_double_p],
        "lrdmc_extrapolate_a": [C.c_int, c_double_p, c_double_p, c_double_p, C.c_int, c_double_p, c_double_p,
                                c_double_p],
        "lrdmc_param_count": [P, c_int_p],
        "lrdmc_get_params": [P, c_double_p],
        "lrdmc_set_params": [P, c_double_p],
        "lrdmc_local_energy_grad": [P, C.c_int, P, P, P, P, P],
        "lrdmc_weighted_rows": [P, C.c_int, C.c_int, P, P, P],
        "lrdmc_batch_create": [C.c_int, C.POINTER(_System), C.POINTER(_TrialWF), C.POINTER(_Params),
                               C.POINTER(c_double_p), P, C.POINTER(P)],
        "lrdmc_batch_destroy": [P],
        "lrdmc_batch_handle": [P, C.c_int, C.POINTER(P)],
        "lrdmc_batch_propagate": [P, C.POINTER(_Schedule)],
        "lrdmc_batch_branch": [P],
        "lrdmc_batch_set_order": [P, C.c_int],
        "lrdmc_batch_tune": [P, C.POINTER(_Schedule), c_double_p, c_int_p],
        "lrdmc_batch_set_timing": [P, C.c_int],
        "lrdmc_batch_timing": [P, c_double_p],
        "lrdmc_batch_launch_count": [P, C.POINTER(C.c_int64)],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.lrdmc_reconfigure_scratch_bytes.argtypes = [C.c_int]
    lib.lrdmc_reconfigure_scratch_bytes.restype = C.c_size_t
    lib.lrdmc_philox4x32.argtypes = [C.c_uint64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.lrdmc_philox4x32.restype = None
    lib.lrdmc_last_error.argtypes = [P]
    lib.lrdmc_last_error.restype = C.c_char_p
    lib.lrdmc_batch_last_error.argtypes = [P]
    lib.lrdmc_batch_last_error.restype = C.c_char_p
    _LIB = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(c_double_p)


def _iptr(a):
    return a.ctypes.data_as(c_int_p)


def _tptr(t):
    return C.c_void_p(t.data_ptr())


class Lrdmc:
    """One LRDMC population on one GPU.

    ``system`` is any object with the attributes of ``lrdmc_system`` and
    ``lrdmc_trial_wf`` (R, Z, pot_kind, r_c, n_up, n_dn, shell_atom, shell_l,
    shell_nprim, exps, coefs, C, j2_anti, j2_par, j2_b, j1_A, j1_B)."""

    def __init__(self, system, x0, a, seed=1, node_rule=0, reinv_period=100, p_gbar=10,
                 n_equil=0, device=None, stream=None, precision=0):
        import torch
        self._torch = torch
        lib = load_library()
        self.lib = lib
        self.device = torch.device(device if device is not None else "cuda")
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        self.n_w, self.n_e = int(x0.shape[0]), int(x0.shape[1])
        keep = {}

        def d(v):
            arr = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
            keep[id(arr)] = arr
            return _dptr(arr)

        def i(v):
            arr = np.ascontiguousarray(v, dtype=np.int32).reshape(-1)
            keep[id(arr)] = arr
            return _iptr(arr)

        self._sys = _System(len(system.Z), d(system.R), d(system.Z), i(system.pot_kind), d(system.r_c),
                            int(system.n_up), int(system.n_dn))
        self._wf = _TrialWF(len(system.shell_l), i(system.shell_atom), i(system.shell_l), i(system.shell_nprim),
                            d(system.exps), d(system.coefs), int(system.C.shape[0]), d(system.C),
                            float(system.j2_anti), float(system.j2_par), float(system.j2_b), d(system.j1_A),
                            d(system.j1_B))
        self._prm = _Params(float(a), self.n_w, int(seed) & (2**64 - 1), int(node_rule), int(reinv_period),
                            int(p_gbar), int(n_equil), int(precision))
        nbytes = C.c_size_t(0)
        self._check(lib.lrdmc_workspace_bytes(C.byref(self._sys), C.byref(self._wf), C.byref(self._prm),
                                              C.byref(nbytes)), None)
        with torch.cuda.device(self.device):
            self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = C.c_void_p()
            st = lib.lrdmc_create(C.byref(self._sys), C.byref(self._wf), C.byref(self._prm), _dptr(x0),
                                  C.c_void_p(aligned), C.c_size_t(nbytes.value), C.c_void_p(self.stream.cuda_stream),
                                  C.byref(h))
        self._h = h
        self._keep = keep
        self._check(st)

    # ---------------------------------------------------------------- plumbing
    def _check(self, status, h=0):
        if status != 0:
            hh = self._h if h == 0 else h
            msg = self.lib.lrdmc_last_error(hh).decode() if hh else ""
            raise LrdmcError(status, msg)

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self.lib.lrdmc_destroy(self._h)
            self._h = None

    @classmethod
    def _view(cls, lib, h, n_w, n_e, device, stream, owner):
        """A non-owning view of a handle that belongs to a batch."""
        import torch
        obj = cls.__new__(cls)
        obj._torch = torch
        obj.lib = lib
        obj._h = h
        obj.n_w, obj.n_e = int(n_w), int(n_e)
        obj.device = device
        obj.stream = stream
        obj._owned = False
        obj._owner = owner
        obj._keep = {}
        return obj

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- hot path
    def propagate(self, kind=LOAD_BALANCED, n_proj=20, tau=0.0, max_moves=100000, rotate=False):
        s = _Schedule(int(kind), int(n_proj), float(tau), int(max_moves), 1 if rotate else 0)
        self._check(self.lib.lrdmc_propagate(self._h, C.byref(s)))

    def branch(self):
        self._check(self.lib.lrdmc_branch(self._h))

    def energy(self):
        E, err = C.c_double(), C.c_double()
        self._check(self.lib.lrdmc_energy(self._h, C.byref(E), C.byref(err)))
        return E.value, err.value

    @property
    def e0(self):
        v = C.c_double()
        self._check(self.lib.lrdmc_get_e0(self._h, C.byref(v)))
        return v.value

    @e0.setter
    def e0(self, v):
        self._check(self.lib.lrdmc_set_e0(self._h, float(v)))

    def history(self):
        n = C.c_int()
        self._check(self.lib.lrdmc_history(self._h, 0, C.byref(n), None, None, None, None, None, None, None))
        m = n.value
        out = dict(wbar=np.zeros(m), ebar=np.zeros(m), e0=np.zeros(m), moves_mean=np.zeros(m),
                   moves_max=np.zeros(m, np.int32), survivors=np.zeros(m, np.int32),
                   status_or=np.zeros(m, np.uint32))
        self._check(self.lib.lrdmc_history(self._h, m, C.byref(n), _dptr(out["wbar"]), _dptr(out["ebar"]),
                                           _dptr(out["e0"]), _dptr(out["moves_mean"]), _iptr(out["moves_max"]),
                                           _iptr(out["survivors"]),
                                           out["status_or"].ctypes.data_as(C.POINTER(C.c_uint32))))
        return out

    WALKER_FIELDS = ("x", "w", "ev", "ratios", "status", "moves")

    def get_walkers(self, fields=WALKER_FIELDS, out=None):
        """Walker fields on the host: x (n_w, n_e, 3), w, ev (b_bar, V_sf, W, e_L),
        ratios (n_w, n_e, 6), status, moves.  ``fields`` selects what is copied;
        ``out`` may supply destination arrays (e.g. views of pinned memory) by
        name, which are filled in place."""
        n, ne = self.n_w, self.n_e
        shapes = dict(x=((n, ne, 3), np.float64), w=((n,), np.float64), ev=((n, 4), np.float64),
                      ratios=((n, ne, 6), np.float64), status=((n,), np.uint32), moves=((n,), np.int32))
        res = {}
        for f in fields:
            shp, dt = shapes[f]
            a = (out or {}).get(f)
            if a is None:
                a = np.zeros(shp, dt)
            assert a.shape == shp and a.dtype == dt and a.flags.c_contiguous
            res[f] = a
        ptr = lambda f, t: res[f].ctypes.data_as(C.POINTER(t)) if f in res else None
        self._check(self.lib.lrdmc_get_walkers(self._h, ptr("x", C.c_double), ptr("w", C.c_double),
                                               ptr("ev", C.c_double), ptr("ratios", C.c_double),
                                               ptr("status", C.c_uint32), ptr("moves", C.c_int32)))
        return res

    def set_walkers(self, x, w=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.n_w, self.n_e, 3)
        wp = None
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float64)
            wp = _dptr(w)
        self._check(self.lib.lrdmc_set_walkers(self._h, _dptr(x), wp))

    def clear_status(self):
        self._check(self.lib.lrdmc_clear_status(self._h))

    def eval_configs(self, x):
        """x: CUDA float64 tensor (n, n_e, 3) -> (ratios (n, n_e, 6), ev (n, 4), n_node (n,))."""
        torch = self._torch
        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
        n = int(x.shape[0])
        ratios = torch.empty((n, self.n_e, 6), dtype=torch.float64, device=x.device)
        ev = torch.empty((n, 4), dtype=torch.float64, device=x.device)
        nn = torch.empty((n,), dtype=torch.int32, device=x.device)
        self._check(self.lib.lrdmc_eval_configs(self._h, n, _tptr(x), _tptr(ratios), _tptr(ev), _tptr(nn)))
        return ratios, ev, nn

    # ---------------------------------------------------------------- derivatives
    def param_count(self):
        n = C.c_int()
        self._check(self.lib.lrdmc_param_count(self._h, C.byref(n)))
        return n.value

    def params(self):
        """theta = (R (n_nuc x 3), j2_anti, j2_par, j2_b, j1_A (n_nuc), j1_B (n_nuc))."""
        th = np.zeros(self.param_count())
        self._check(self.lib.lrdmc_get_params(self._h, _dptr(th)))
        return th

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        assert th.shape == (self.param_count(),)
        self._check(self.lib.lrdmc_set_params(self._h, _dptr(th)))

    def local_energy_grad(self, x):
        """x: CUDA float64 tensor (n, n_e, 3) -> (e_L (n,), log|Psi| (n,), d e_L/d theta (n, m),
        d log|Psi|/d theta (n, m))."""
        torch = self._torch
        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
        n, m = int(x.shape[0]), self.param_count()
        eL = torch.empty(n, dtype=torch.float64, device=x.device)
        lp = torch.empty(n, dtype=torch.float64, device=x.device)
        ge = torch.empty((n, m), dtype=torch.float64, device=x.device)
        gl = torch.empty((n, m), dtype=torch.float64, device=x.device)
        self._check(self.lib.lrdmc_local_energy_grad(self._h, n, _tptr(x), _tptr(eL), _tptr(lp), _tptr(ge),
                                                     _tptr(gl)))
        return eL, lp, ge, gl

    def weighted_rows(self, rows, w):
        torch = self._torch
        rows, w = rows.contiguous(), w.contiguous().to(torch.float64)
        out = torch.empty(rows.shape[1], dtype=torch.float64, device=rows.device)
        self._check(self.lib.lrdmc_weighted_rows(self._h, int(rows.shape[0]), int(rows.shape[1]), _tptr(rows),
                                                 _tptr(w), _tptr(out)))
        return out

    def set_timing(self, enable=True):
        self._check(self.lib.lrdmc_set_timing(self._h, 1 if enable else 0))

    def interval_timing(self):
        """Load-imbalance figures of the last interval (see lrdmc_interval_timing)."""
        out = np.zeros(6)
        self._check(self.lib.lrdmc_interval_timing(self._h, _dptr(out)))
        return dict(span_ms=out[0], walker_ms_mean=out[1], walker_ms_max=out[2], busy_fraction=out[3],
                    moves_mean=out[4], moves_max=out[5])

    def save(self, path):
        self._check(self.lib.lrdmc_save(self._h, os.fsencode(path)))

    def load(self, path):
        self._check(self.lib.lrdmc_load(self._h, os.fsencode(path)))

    def set_drift_tol(self, tol):
        """Tolerance of the Sherman-Morrison drift check (0 disables it)."""
        self._check(self.lib.lrdmc_set_drift_tol(self._h, float(tol)))

    def drift_reinversions(self):
        """Drift-triggered re-inversions since creation (all walkers)."""
        n = C.c_int64()
        self._check(self.lib.lrdmc_drift_reinversions(self._h, C.byref(n)))
        return n.value

    def launch_count(self):
        v = C.c_int64()
        self._check(self.lib.lrdmc_launch_count(self._h, C.byref(v)))
        return v.value

    def synchronize(self):
        self.stream.synchronize()


def reconfigure_indices(w, xi32, stream=None):
    """Integer-comb source indices for device weights ``w`` (float64 CUDA tensor).

    Returns (src int32 tensor, status int32 tensor of 2: [ok/invalid, survivors])."""
    import torch
    lib = load_library()
    assert w.is_cuda and w.dtype == torch.float64 and w.is_contiguous() and w.dim() == 1
    n = int(w.shape[0])
    src = torch.empty(n, dtype=torch.int32, device=w.device)
    st = torch.empty(2, dtype=torch.int32, device=w.device)
    nb = lib.lrdmc_reconfigure_scratch_bytes(n)
    scratch = torch.empty(nb + 256, dtype=torch.uint8, device=w.device)
    sp = (scratch.data_ptr() + 255) // 256 * 256
    s = stream if stream is not None else torch.cuda.current_stream(w.device)
    r = lib.lrdmc_reconfigure_indices(n, _tptr(w), int(xi32) & 0xFFFFFFFF, _tptr(src), C.c_void_p(sp),
                                      C.c_size_t(nb), _tptr(st), C.c_void_p(s.cuda_stream))
    if r != 0:
        raise LrdmcError(r, "lrdmc_reconfigure_indices failed")
    s.synchronize()
    del scratch
    return src, st


class LrdmcBatch:
    """Several independent LRDMC populations propagated by one persistent
    kernel launch per interval and branched by batched launches.

    ``systems``: list of system objects (as for ``Lrdmc``); ``x0s``: list of
    initial positions (n_w_k, n_e_k, 3); ``seeds``: one seed per system.
    ``handle(k)`` gives an ``Lrdmc`` view of system k (readback, energy,
    history; owned by the batch)."""

    def __init__(self, systems, x0s, a, seeds, node_rule=0, reinv_period=100, p_gbar=10, n_equil=0,
                 device=None, stream=None, precision=0):
        import torch
        lib = load_library()
        self.lib = lib
        self.device = torch.device(device if device is not None else "cuda")
        n = len(systems)
        assert len(x0s) == n and len(seeds) == n
        keep = []

        def d(v):
            arr = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
            keep.append(arr)
            return _dptr(arr)

        def i(v):
            arr = np.ascontiguousarray(v, dtype=np.int32).reshape(-1)
            keep.append(arr)
            return _iptr(arr)

        sys_arr = (_System * n)()
        wf_arr = (_TrialWF * n)()
        prm_arr = (_Params * n)()
        x_ptrs = (c_double_p * n)()
        self._shapes = []
        for k, (sy, x0) in enumerate(zip(systems, x0s)):
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            keep.append(x0)
            self._shapes.append((int(x0.shape[0]), int(x0.shape[1])))
            sys_arr[k] = _System(len(sy.Z), d(sy.R), d(sy.Z), i(sy.pot_kind), d(sy.r_c), int(sy.n_up), int(sy.n_dn))
            wf_arr[k] = _TrialWF(len(sy.shell_l), i(sy.shell_atom), i(sy.shell_l), i(sy.shell_nprim), d(sy.exps),
                                 d(sy.coefs), int(sy.C.shape[0]), d(sy.C), float(sy.j2_anti), float(sy.j2_par),
                                 float(sy.j2_b), d(sy.j1_A), d(sy.j1_B))
            prm_arr[k] = _Params(float(a), int(x0.shape[0]), int(seeds[k]) & (2**64 - 1), int(node_rule),
                                 int(reinv_period), int(p_gbar), int(n_equil), int(precision))
            x_ptrs[k] = _dptr(x0)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            b = C.c_void_p()
            st = lib.lrdmc_batch_create(n, sys_arr, wf_arr, prm_arr, x_ptrs, C.c_void_p(self.stream.cuda_stream),
                                        C.byref(b))
        self._b = b
        self._keep = keep
        self._check(st)
        self.handles = []
        for k in range(n):
            h = C.c_void_p()
            self._check(lib.lrdmc_batch_handle(self._b, k, C.byref(h)))
            self.handles.append(Lrdmc._view(lib, h, self._shapes[k][0], self._shapes[k][1], self.device,
                                            self.stream, self))

    def _check(self, status):
        if status != 0:
            msg = self.lib.lrdmc_batch_last_error(self._b).decode() if self._b else ""
            raise LrdmcError(status, msg)

    def close(self):
        if getattr(self, "_b", None):
            for v in getattr(self, "handles", []):
                v._h = None
            self.lib.lrdmc_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def handle(self, k):
        return self.handles[k]

    def propagate(self, kind=LOAD_BALANCED, n_proj=20, tau=0.0, max_moves=100000):
        s = _Schedule(int(kind), int(n_proj), float(tau), int(max_moves), 0)
        self._check(self.lib.lrdmc_batch_propagate(self._b, C.byref(s)))

    def branch(self):
        self._check(self.lib.lrdmc_batch_branch(self._b))

    def set_order(self, policy):
        self._check(self.lib.lrdmc_batch_set_order(self._b, int(policy)))

    def tune(self, kind=LOAD_BALANCED, n_proj=20, tau=0.0, max_moves=100000):
        s = _Schedule(int(kind), int(n_proj), float(tau), int(max_moves), 0)
        times = np.zeros(4)
        best = C.c_int()
        self._check(self.lib.lrdmc_batch_tune(self._b, C.byref(s), _dptr(times), C.byref(best)))
        return best.value, dict(zip((1, 2, 3, 4), times))

    def set_timing(self, enable=True):
        self._check(self.lib.lrdmc_batch_set_timing(self._b, 1 if enable else 0))

    def timing(self):
        out = np.zeros(8)
        self._check(self.lib.lrdmc_batch_timing(self._b, _dptr(out)))
        return dict(span_ms=out[0], walker_ms_mean=out[1], walker_ms_max=out[2], sm_idle_fraction=out[3],
                    sm_idle_tail_ms=out[4], slot_busy_fraction=out[5], walkers=int(out[6]), items=int(out[7]))

    def launch_count(self):
        v = C.c_int64()
        self._check(self.lib.lrdmc_batch_launch_count(self._b, C.byref(v)))
        return v.value


def _autograd_function():
    import torch

    class LocalEnergy(torch.autograd.Function):
        """(e_L, log|Psi_G|) at configurations x as functions of theta (the
        handle's nuclear coordinates and Jastrow parameters), with the
        library's hand-written adjoint as the backward pass (no gradient for x)."""

        @staticmethod
        def forward(ctx, theta, x, lr):
            th = theta.detach().cpu().numpy().astype(np.float64)
            if not np.array_equal(th, lr.params()):
                lr.set_params(th)
            eL, lp, ge, gl = lr.local_energy_grad(x.detach().contiguous())
            ctx.save_for_backward(ge, gl)
            ctx.lr = lr
            ctx.theta_device = theta.device
            return eL, lp

        @staticmethod
        def backward(ctx, g_e, g_l):
            ge, gl = ctx.saved_tensors
            lr = ctx.lr
            grad = None
            if g_e is not None:
                grad = lr.weighted_rows(ge, g_e)
            if g_l is not None:
                gg = lr.weighted_rows(gl, g_l)
                grad = gg if grad is None else grad + gg
            return grad.to(ctx.theta_device), None, None

    return LocalEnergy


_LOCAL_ENERGY = None


def local_energy(lr, theta, x):
    """torch.autograd entry: (e_L, log|Psi_G|) at x with gradients to theta
    (a float64 tensor of lr.param_count() values)."""
    global _LOCAL_ENERGY
    if _LOCAL_ENERGY is None:
        _LOCAL_ENERGY = _autograd_function()
    return _LOCAL_ENERGY.apply(theta, x, lr)


def extrapolate_a(a, E, err, order=1):
    """a -> 0 extrapolation of energies at lattice spacings a (standard errors
    err): weighted least squares E(a) = sum_j coef[j] a^(2j), j <= order.
    Returns (coef, cov, chi2); coef[0] is the extrapolated energy, sqrt(cov[0, 0])
    its standard error."""
    lib = load_library()
    a = np.ascontiguousarray(a, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    err = np.ascontiguousarray(err, dtype=np.float64)
    if not (a.shape == E.shape == err.shape and a.ndim == 1):
        raise ValueError("a, E and err must be 1-D arrays of one length")
    coef = np.zeros(order + 1)
    cov = np.zeros((order + 1, order + 1))
    chi2 = C.c_double()
    r = lib.lrdmc_extrapolate_a(len(a), _dptr(a), _dptr(E), _dptr(err), int(order), _dptr(coef), _dptr(cov),
                                C.byref(chi2))
    if r != 0:
        raise LrdmcError(r, "lrdmc_extrapolate_a: invalid points or order")
    return coef, cov, chi2.value


def estimate(wbar, ebar, p_gbar=10, n_equil=0):
    """The library's energy estimator (lrdmc_estimate) over a branching
    history: returns (E, err)."""
    lib = load_library()
    wbar = np.ascontiguousarray(wbar, dtype=np.float64)
    ebar = np.ascontiguousarray(ebar, dtype=np.float64)
    if wbar.shape != ebar.shape or wbar.ndim != 1:
        raise ValueError("wbar and ebar must be 1-D arrays of one length")
    E, err = C.c_double(), C.c_double()
    r = lib.lrdmc_estimate(len(wbar), _dptr(wbar), _dptr(ebar), int(p_gbar), int(n_equil), C.byref(E), C.byref(err))
    if r != 0:
        raise LrdmcError(r, "lrdmc_estimate: invalid history")
    return E.value, err.value


def check_word(clear=True):
    """(violation word, checked) of the checked build: the first out-of-extent
    index recorded by the kernels (0 = none; source line << 32 | index);
    checked is False in the normal library, where the word is always 0."""
    lib = load_library()
    if not lib.lrdmc_checked_build():
        return 0, False
    w = C.c_uint64()
    r = lib.lrdmc_check_word(C.byref(w), int(bool(clear)))
    if r != 0:
        raise LrdmcError(r, "lrdmc_check_word failed")
    return int(w.value), True


def philox4x32(seed, ctr):
    lib = load_library()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    o = (C.c_uint32 * 4)()
    lib.lrdmc_philox4x32(int(seed) & (2**64 - 1), c, o)
    return tuple(int(v) for v in o)


def reconfigure_indices_noalloc(w, xi32, stream=None):
    """Same as ``reconfigure_indices`` through the allocation-free entry point
    (the library's fixed device scratch array; n <= LRDMC_NOALLOC_MAX_WALKERS).

    For callers that cannot allocate device memory at call time.  The output
    tensors here are allocated by PyTorch only because this helper returns new
    tensors; the library call itself allocates nothing."""
    import torch
    lib = load_library()
    f = lib.lrdmc_reconfigure_indices_noalloc
    f.argtypes = [C.c_int, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    assert w.is_cuda and w.dtype == torch.float64 and w.is_contiguous() and w.dim() == 1
    n = int(w.shape[0])
    src = torch.empty(n, dtype=torch.int32, device=w.device)
    st = torch.empty(2, dtype=torch.int32, device=w.device)
    s = stream if stream is not None else torch.cuda.current_stream(w.device)
    r = f(n, _tptr(w), int(xi32) & 0xFFFFFFFF, _tptr(src), _tptr(st), C.c_void_p(s.cuda_stream))
    if r != 0:
        raise LrdmcError(r, "lrdmc_reconfigure_indices_noalloc failed")
    s.synchronize()
    return src, st
