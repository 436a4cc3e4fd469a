"""The C-ABI library loads and exports every entry point of include/klr.h, and
its host-only logic (configuration enumeration, argument checks that fail
before touching a device) behaves as documented.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "klr.h")


def _lib_or_skip():
    try:
        import paper_1911_02373_gb300 as klr
    except ImportError as e:  # library not built in this checkout
        pytest.skip(str(e))
    return klr


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(
        r"^\s*(?:klr_status|const char\*|int|int64_t|size_t)\s+(klr_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("klr_fit", "klr_eval", "klr_argmin", "klr_enumerate_configs",
              "klr_ctx_create", "klr_ctx_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    klr = _lib_or_skip()
    out = subprocess.run(["nm", "-D", "--defined-only", klr.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(declared_symbols()) == set(klr.ABI_SYMBOLS)
    for s in declared_symbols():
        assert hasattr(klr._lib, s)


def test_enumerate_configs_matches_closed_forms_and_oracle():
    klr = _lib_or_skip()
    from oracle import configs
    for dims, n in ((1, 6), (2, 51), (3, 251)):
        F = klr.enumerate_configs(dims)
        assert F.shape == (n, 3)
        want = [tuple(c) + (1,) * (3 - dims) for c in configs.enumerate_configs(dims)]
        assert [tuple(map(int, r)) for r in F] == want
    # smaller range and the capacity check
    F = klr.enumerate_configs(2, 64, 128)
    assert len(F) == 7 + 8
    n = ctypes.c_int(0)
    buf = np.zeros((3, 3), dtype=np.int32)
    st = klr._lib.klr_enumerate_configs(2, 32, 1024, buf.ctypes.data_as(ctypes.c_void_p), 3,
                                        ctypes.byref(n))
    assert st == klr.EINVAL and n.value == 51
    assert klr._lib.klr_enumerate_configs(4, 32, 1024, None, 0, ctypes.byref(n)) == klr.EINVAL


def test_argument_errors_before_any_device_work():
    klr = _lib_or_skip()
    b = klr.FitBatch()
    assert klr._lib.klr_fit(None, ctypes.byref(b), None, 0, None, None, None) == klr.EINVAL
    assert b"NULL" in klr._lib.klr_last_error()
    assert klr._lib.klr_eval(None, None, None, None, 0, None, None, 0, None) == klr.EINVAL
    assert klr._lib.klr_argmin(None, None, None, None, 0, None, None, None, 0, None, None,
                               None, None) == klr.EINVAL
    assert klr.version() == 1


def test_binding_refuses_host_tensors_for_device_arguments():
    """Every address the binding hands the library comes from a CUDA tensor;
    a host tensor is refused before any call (the GPU could otherwise read
    or write host memory in place)."""
    torch = pytest.importorskip("torch")
    klr = _lib_or_skip()
    with pytest.raises(ValueError):
        klr._dptr(torch.zeros(4))
    with pytest.raises(ValueError):
        klr._ptr(torch.zeros(4, dtype=torch.int32))
    assert klr._ptr(None) is None


def test_probe_peaks_refuses_a_null_context():
    klr = _lib_or_skip()
    pk = klr.Peaks()
    assert klr._lib.klr_probe_peaks(None, ctypes.byref(pk), None) == klr.EINVAL
