"""Host-side checks of the C ABI library that need no GPU."""
import ctypes
import subprocess

import pytest

import paper_2203_05632_gb300 as pkg
from paper_2203_05632_gb300 import _binding as B


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return B.load_library()


def test_library_exports_every_declared_entry_point(lib):
    declared = B.header_symbols()
    assert len(declared) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_binding_covers_every_declared_entry_point():
    assert set(B.header_symbols()) <= set(B.SIGNATURES)


def test_workspace_size_is_a_host_computation(lib):
    d = B.Dims(6, 300, 80, 400, 1024, 4)
    f64 = B.workspace_bytes(d, B.MCMP2_FP64)
    mixed = B.workspace_bytes(d, B.MCMP2_MIXED)
    assert f64 > 8 * 1024 * 480 * 16  # phi alone
    assert mixed > 0
    assert B.workspace_bytes(B.Dims(2, 20, 4, 16, 16, 1), B.MCMP2_FP64) < f64


@pytest.mark.parametrize("bad", [
    (0, 20, 4, 16, 16, 1),   # no centres
    (2, 20, 3, 16, 16, 1),   # odd occupied count (Kramers pairs)
    (2, 20, 4, 16, 1, 1),    # a single walker pair has no pair of pairs
    (2, 20, 4, 16, 16, 0),   # no imaginary time
])
def test_invalid_dims_are_rejected(lib, bad):
    n = ctypes.c_size_t(0)
    d = B.Dims(*bad)
    assert lib.mcmp2_workspace_bytes(ctypes.byref(d), 0, ctypes.byref(n)) == -1


def test_create_without_an_sm103_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.mcmp2_create(ctypes.byref(h), 0, None, 0)
    assert rc == -7 and not h.value


def test_null_context_calls_return_einval(lib):
    assert lib.mcmp2_run_steps(None, 1, 0, None) == -1
    assert lib.mcmp2_eval_fixed(None, 1, None, None, None) == -1
    assert lib.mcmp2_last_error(None) == b"null context"
    lib.mcmp2_destroy(None)


@pytest.mark.parametrize("m,n_tau,code", [
    (1 << 20, 1, -1),   # beyond the largest m any entry point accepts (65536)
    (65537, 1, -1),
    (65536, 1, -6),     # 33.6e6 tiles of 8 pairs: far beyond the fixed scratch array
    (1024, 65, -1),     # more times than a context accepts
    (1024, 8, -6),      # 8,256 tiles x 8 times > 65,536 partial sums
    (1, 1, -1),
])
def test_noalloc_size_checks_come_before_any_device_work(lib, m, n_tau, code):
    """The allocation-free call rejects its sizes on the host (64-bit tile counts) before it
    touches a device, so these calls need no GPU; the pointers are never dereferenced."""
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    rc = lib.mcmp2_pair_sum_f64_noalloc(m, 4, 16, n_tau, p, p, p, 1.0, p, None)
    assert rc == code


def test_dims_limits_match_the_header(lib):
    n = ctypes.c_size_t(0)
    ok = B.Dims(2, 20, 4, 16, 65536, 64)
    assert lib.mcmp2_workspace_bytes(ctypes.byref(ok), 0, ctypes.byref(n)) == 0
    for bad in (B.Dims(2, 20, 4, 16, 65537, 1), B.Dims(2, 20, 4, 16, 16, 65)):
        assert lib.mcmp2_workspace_bytes(ctypes.byref(bad), 0, ctypes.byref(n)) == -1
