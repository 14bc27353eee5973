"""The library's reduced-slot FP64 functions against CUDA's own exp, 1/x and
rsqrt (computed by PyTorch on the same GPU): a few ulp over wide ranges."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_fp64math_against_cuda():
    import torch
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    lib = P.load_library()
    f = lib.lrdmc_fp64math
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    rng = np.random.default_rng(0)
    n = 1 << 20
    xe = np.concatenate([rng.uniform(-700, 700, n // 2), rng.uniform(-5, 5, n // 2)])
    xp = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), n))
    for x, which in ((xe, "exp"), (xp, "pos")):
        xt = torch.tensor(x, device="cuda")
        e = torch.empty_like(xt)
        r = torch.empty_like(xt)
        q = torch.empty_like(xt)
        s = torch.cuda.current_stream().cuda_stream
        assert f(n, xt.data_ptr(), e.data_ptr(), r.data_ptr(), q.data_ptr(), s) == 0
        torch.cuda.synchronize()
        if which == "exp":
            ref = torch.exp(xt)
            rel = ((e - ref).abs() / ref).max().item()
            assert rel < 8e-16, rel
            edge = torch.tensor([-701.0, -1e4, 0.0, float("nan"), float("inf"), -float("inf"), 701.0, -699.9],
                                dtype=torch.float64, device="cuda")
            assert f(len(edge), edge.data_ptr(), e.data_ptr(), None, None, s) == 0
            torch.cuda.synchronize()
            got = e[:len(edge)].cpu().numpy()
            assert got[0] == 0.0 and got[1] == 0.0 and got[2] == 1.0
            assert np.isnan(got[3]) and got[4] == np.inf and got[5] == 0.0 and got[6] == np.inf
            assert abs(got[7] / np.exp(-699.9) - 1.0) < 8e-16
        else:
            rel_r = ((r - 1.0 / xt).abs() * xt).max().item()
            rel_q = ((q - torch.rsqrt(xt)).abs() / torch.rsqrt(xt)).max().item()
            assert rel_r < 4e-16 and rel_q < 6e-16, (rel_r, rel_q)


def test_screened_potential_against_cuda_erf():
    """erf(r/r_c)/r from the library's table against CUDA's erf on the same GPU,
    over r from 1e-6 to 10 r_c and beyond the table, and at r = 0."""
    import torch
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    lib = P.load_library()
    f = lib.lrdmc_erf_over_r
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    rng = np.random.default_rng(3)
    stream = torch.cuda.current_stream().cuda_stream
    for rc in (0.5, 1.3):
        r = np.concatenate([np.exp(rng.uniform(np.log(1e-6), np.log(10 * rc), 1 << 18)),
                            rng.uniform(0, 7 * rc, 1 << 18)])
        s = torch.tensor(r * r, device="cuda")
        out = torch.empty_like(s)
        assert f(len(r), s.data_ptr(), rc, out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        rr = torch.sqrt(s)
        ref = torch.special.erf(rr / rc) / rr
        assert ((out - ref).abs() / ref).max().item() < 2e-15
        z = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert f(1, z.data_ptr(), rc, out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert abs(out[0].item() * rc * np.sqrt(np.pi) / 2 - 1.0) < 1e-15
    assert f(1, s.data_ptr(), 0.0, out.data_ptr(), stream) == 1
