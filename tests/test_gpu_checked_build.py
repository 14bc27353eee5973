"""The checked build (liblrdmc_checked.so, LRDMC_CHECKED): every data-derived
index of the walker and branching kernels is tested against its extent; a
violation is recorded in a device word and the access redirected, so nothing
faults or traps.  This file runs the small per-configuration and per-interval
parity cases, the batched kernels and the host-injected failures (NaN and
coincident walkers) under the checked library in a child process (the library is
chosen when the binding loads, once per process); the autouse fixture of
conftest.py then requires the violation word to be zero after every test, and
the self-test below shows that a violation is recorded and cleared."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_check_selftest_records_a_violation_without_faulting():
    """Runs only inside the checked child process (skipped otherwise)."""
    if os.environ.get("LRDMC_CHECKED") != "1":
        pytest.skip("runs in the checked child process")
    import ctypes
    from gpu_helpers import lib_or_skip
    P = lib_or_skip()
    lib = P.load_library()
    assert lib.lrdmc_checked_build() == 1
    assert P.binding.check_word(clear=True) == (0, True)
    r = ctypes.c_int(-1)
    assert lib.lrdmc_check_selftest(5, 8, ctypes.byref(r)) == 0 and r.value == 5
    assert P.binding.check_word(clear=True) == (0, True)
    assert lib.lrdmc_check_selftest(9, 8, ctypes.byref(r)) == 0 and r.value == 0
    word, _ = P.binding.check_word(clear=True)
    assert word != 0 and (word & 0xffffffff) == 9
    assert P.binding.check_word(clear=True) == (0, True)


def test_small_parity_cases_pass_under_the_checked_build():
    if os.environ.get("LRDMC_CHECKED") == "1":
        pytest.skip("the parent process starts the checked run")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_12033_b300 import build
    build.build()
    env = dict(os.environ, LRDMC_CHECKED="1")
    files = ["tests/test_gpu_checked_build.py", "tests/test_gpu_parity.py", "tests/test_gpu_mixed.py",
             "tests/test_gpu_drift.py", "tests/test_gpu_failures.py", "tests/test_gpu_batch.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", *files,
                        "-k", "not largest_size and not full_size and not energy_error_bar"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
