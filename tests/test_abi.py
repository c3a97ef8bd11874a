"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/fhs.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "fhs.h")).read()
    return sorted(set(re.findall(r"^\s*(?:fhs_status|const char\*|uint64_t)\s+(fhs_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_07358_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_six_hot_path_calls():
    syms = header_symbols()
    for name in ("fhs_measure", "fhs_adjoint", "fhs_prox_l21_sara_facets", "fhs_prox_nuclear_facets",
                 "fhs_proj_l2ball_blocks", "fhs_pdfb_iter"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in header_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2003_07358_gb300 import fhs
    assert sorted(fhs.SYMBOLS) == header_symbols()


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    lib.fhs_create.restype = ctypes.c_int32
    lib.fhs_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    lib.fhs_last_error.restype = ctypes.c_char_p
    lib.fhs_last_error.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.fhs_create(None, 0, None, ctypes.byref(out)) == 1      # FHS_ERR_INVALID_ARG
    assert out.value is None
    assert b"cube" in lib.fhs_last_error(None)
    assert lib.fhs_create(None, 1, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2003_07358_gb300 import fhs
    with pytest.raises(fhs.FhsError):
        fhs._lib = None
        fhs.load(str(tmp_path / "missing.so"))
    fhs._lib = None


def test_noalloc_wrapper_rejects_bad_arguments_before_the_call():
    """The allocation-free entry point has no length arguments, so its binding checks
    the offsets, radii, dtypes and sizes on the host (ValueError, no device work)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2003_07358_gb300 import fhs
    z = torch.zeros(10, dtype=torch.complex64)
    v = torch.empty_like(z)
    off = np.array([0, 4, 10])
    with pytest.raises(ValueError, match="eps"):
        fhs.fhs_proj_l2ball_noalloc(z, z, off, np.ones(3), v)
    with pytest.raises(ValueError, match="non-decreasing"):
        fhs.fhs_proj_l2ball_noalloc(z, z, np.array([0, 6, 4]), np.ones(2), v)
    with pytest.raises(ValueError, match="complex64"):
        fhs.fhs_proj_l2ball_noalloc(z.to(torch.complex128), z, off, np.ones(2), v)
    with pytest.raises(ValueError, match="elements"):
        fhs.fhs_proj_l2ball_noalloc(z, z, np.array([0, 4, 11]), np.ones(2), v)
    with pytest.raises(ValueError, match="CUDA"):
        fhs.fhs_proj_l2ball_noalloc(z, z, off, np.ones(2), v)
