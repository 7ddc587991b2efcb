"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(mpw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpw_create", "mpw_create_patch", "mpw_set_fields", "mpw_step", "mpw_get_fields",
                     "mpw_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(mpw_lib):
    lib = ctypes.CDLL(mpw_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding covers the same set, nothing more
    assert sorted(mpw_lib.SIGNATURES) == declared_functions()


def test_binding_refuses_to_run_without_the_library(mpw_lib, tmp_path, monkeypatch):
    """No CPU fallback: a missing libmpw.so is an import error."""
    monkeypatch.setattr(mpw_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mpw_lib._load()


def test_conv_entry_points_validate_shapes_before_any_launch(mpw_lib):
    """Unsupported channel counts and volumes are refused on the host."""
    n_bad = (ctypes.c_int * 3)(24, 8, 4)   # n0 not a multiple of 16
    n_ok = (ctypes.c_int * 3)(16, 8, 4)
    fake = ctypes.c_void_p(256)            # never dereferenced: validation comes first
    L = mpw_lib.lib
    assert L.mpw_conv3_forward(fake, 32, fake, None, 32, 1, n_bad, 0, None, fake, None, None) == 1
    assert L.mpw_conv3_forward(fake, 8, fake, None, 8, 1, n_ok, 0, None, fake, None, None) == 1
    assert L.mpw_conv3_forward(fake, 16, fake, None, 32, 1, n_ok, 0, None, fake, None, None) == 1
    assert L.mpw_conv3_backward_data(fake, 32, fake, 32, 0, n_ok, None, fake, None, None) == 1
    assert L.mpw_conv3_wgrad_scratch_bytes(16, 32) == 0
    assert L.mpw_adam_step(fake, None, fake, fake, fake, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == 1
    assert L.mpw_mse_grad(fake, 8, fake, 9, 10, fake, None, None) == 1


def test_surrogate_entry_points_validate_arguments(mpw_lib):
    """Refused on the host, before any CUDA call."""
    L = mpw_lib.lib
    h = ctypes.c_void_p()
    assert L.mpw_sur_create(0, None, 0.0, 0.1, 1e-4, ctypes.byref(h)) == 1      # dt <= 0
    assert L.mpw_sur_create(0, None, 1e-3, -0.1, 1e-4, ctypes.byref(h)) == 1    # h <= 0
    assert L.mpw_sur_create(0, None, 1e-3, 0.1, 0.0, ctypes.byref(h)) == 1      # sigma <= 0
    assert L.mpw_sur_create(0, None, 1e-3, 0.1, 1e-4, None) == 1                # no output handle
    assert not h.value
    n = (ctypes.c_int * 3)(16, 8, 8)
    assert L.mpw_sur_predict(None, None, None, 1, n, None, None) == 1           # null handle
    assert L.mpw_step_surrogate(None, None, 1e-3, 1, 1e-4, None, None) == 1     # null context
    assert L.mpw_sur_param_count() == sum(co * 27 * ci + co for ci, co in [(8, 32), (32, 32), (32, 32), (32, 8)])


def test_wait_limit_entry_point_validates_its_context(mpw_lib):
    assert mpw_lib.lib.mpw_set_wait_limit(None, 0) == 1


def test_noalloc_refuses_bad_arguments_before_any_launch(mpw_lib):
    """Host-side checks of the allocation-free entry point: sizes beyond the
    fixed work array are refused by the library itself, and the Python
    binding refuses tensors whose shape, dtype, layout or device would make
    the kernels read or write outside them."""
    import torch
    L = mpw_lib.lib
    fake = ctypes.c_void_p(256)            # never dereferenced: validation comes first
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    big = (ctypes.c_int * 3)(mpw_lib.NOALLOC_MAX_N + 1, 8, 8)
    small = (ctypes.c_int * 3)(5, 8, 8)
    assert L.mpw_step_periodic_noalloc(big, lo, hi, 0.005, 1e-3, 1, fake, fake, None) == mpw_lib.ERR_ARG
    assert L.mpw_step_periodic_noalloc(small, lo, hi, 0.005, 1e-3, 1, fake, fake, None) == mpw_lib.ERR_ARG
    n = (16, 8, 4)
    good = torch.zeros((4, 8, 16), dtype=torch.float64)
    cases = [
        (torch.zeros((4, 8, 15), dtype=torch.float64), "shape"),
        (torch.zeros((4, 8, 16), dtype=torch.float32), "float64"),
        (torch.zeros((4, 16, 8), dtype=torch.float64).transpose(1, 2), "contiguous"),
        (good, "CUDA device"),                 # a host tensor: no CUDA device here
    ]
    for bad, what in cases:
        with pytest.raises(ValueError, match=what):
            mpw_lib.check_noalloc_fields(n, bad, good)
        with pytest.raises(ValueError, match=what):
            mpw_lib.step_periodic_noalloc(n, (0, 0, 0), (1, 1, 1), 0.005, 1e-3, 1, good, bad)


def test_conv_kernel_selection_is_validated(mpw_lib):
    L = mpw_lib.lib
    assert L.mpw_conv3_select(2) == mpw_lib.ERR_ARG
    assert L.mpw_conv3_select(1) == 0 and L.mpw_conv3_select(0) == 0
