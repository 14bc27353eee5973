"""Shared helpers for the GPU tests (no method arithmetic here)."""
import numpy as np

RTOL = 1e-10      # |gpu - ref| <= RTOL * max(1, |ref|) for FP64 per-configuration values


def assert_close(gpu, ref, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    err = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    worst = float(np.max(err)) if err.size else 0.0
    assert worst <= rtol, f"{what}: max scaled error {worst:.3e} at {np.unravel_index(np.argmax(err), err.shape)}"


def lib_or_skip():
    import pytest
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_12033_b300 import build
    build.build()
    import paper_2508_12033_b300 as P
    return P
