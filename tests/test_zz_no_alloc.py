"""The allocation-free reconfiguration entry point gives the same indices as
the regular one.

lrdmc_reconfigure_indices_noalloc exists for callers that cannot allocate
device memory when they call the library (device memory held by the host's
own or an exhausted allocator, an embedding runtime that forbids allocation
on its hot path).  It
uses a fixed device array inside the library instead of caller scratch, so
this test calls both entry points through the C ABI on the same weights, twice
in a row with different sizes (the shared array keeps the previous call's
contents), and requires identical source indices and status words.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_12033_b300 import build
    build.build()
    from paper_2508_12033_b300 import load_library
    return load_library()


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    lib = _lib()
    f = lib.lrdmc_reconfigure_indices_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    for n in (5000, 1237):                          # second call smaller than the first
        w = torch.tensor(rng.lognormal(0.0, 0.8, n), device="cuda")
        xi = int(rng.integers(0, 2**32))
        src_a = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        st_a = torch.full((2,), -7, dtype=torch.int32, device="cuda")
        assert f(n, w.data_ptr(), xi, src_a.data_ptr(), st_a.data_ptr(), stream.cuda_stream) == 0
        nb = lib.lrdmc_reconfigure_scratch_bytes(n)
        scratch = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        sp = (scratch.data_ptr() + 255) // 256 * 256
        src_b = torch.full((n,), -9, dtype=torch.int32, device="cuda")
        st_b = torch.full((2,), -9, dtype=torch.int32, device="cuda")
        assert lib.lrdmc_reconfigure_indices(n, ctypes.c_void_p(w.data_ptr()), xi,
                                             ctypes.c_void_p(src_b.data_ptr()), ctypes.c_void_p(sp),
                                             ctypes.c_size_t(nb), ctypes.c_void_p(st_b.data_ptr()),
                                             ctypes.c_void_p(stream.cuda_stream)) == 0
        torch.cuda.synchronize()
        assert torch.equal(src_a, src_b)
        assert torch.equal(st_a, st_b) and int(st_a[0]) == 0


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    lib = _lib()
    f = lib.lrdmc_reconfigure_indices_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    w = torch.ones(4, dtype=torch.float64, device="cuda")
    src = torch.empty(4, dtype=torch.int32, device="cuda")
    assert f((1 << 18) + 1, w.data_ptr(), 0, src.data_ptr(), None, None) == 7    # LRDMC_ERR_UNSUPPORTED
    assert f(0, w.data_ptr(), 0, src.data_ptr(), None, None) == 1                 # LRDMC_ERR_ARG


def test_noalloc_refuses_invalid_weights_like_the_regular_entry_point():
    """A NaN weight: both entry points report status word 0 = 1 (invalid
    weights) and leave the source indices untouched."""
    import torch
    lib = _lib()
    f = lib.lrdmc_reconfigure_indices_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    stream = torch.cuda.current_stream()
    n = 777
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    w[100] = float("nan")
    src_a = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st_a = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    assert f(n, w.data_ptr(), 12345, src_a.data_ptr(), st_a.data_ptr(), stream.cuda_stream) == 0
    nb = lib.lrdmc_reconfigure_scratch_bytes(n)
    scratch = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    sp = (scratch.data_ptr() + 255) // 256 * 256
    src_b = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st_b = torch.full((2,), -9, dtype=torch.int32, device="cuda")
    assert lib.lrdmc_reconfigure_indices(n, ctypes.c_void_p(w.data_ptr()), 12345,
                                         ctypes.c_void_p(src_b.data_ptr()), ctypes.c_void_p(sp),
                                         ctypes.c_size_t(nb), ctypes.c_void_p(st_b.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert int(st_a[0]) == 1 and int(st_b[0]) == 1
    assert torch.equal(st_a, st_b)
    assert bool((src_a == -7).all()) and bool((src_b == -7).all())
