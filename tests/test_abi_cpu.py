"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/sp2.h; calls fail cleanly without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sp2.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp2_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_06385_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sp2_init", "sp2_finalize", "sp2_density_matrix", "sp2_density_matrix_batched",
                     "sp2_network_forward", "sp2_network_backward", "sp2_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_calls_before_init_report_not_initialized(lib):
    lib.sp2_density_matrix.restype = ctypes.c_int
    lib.sp2_last_error.restype = ctypes.c_char_p
    st = lib.sp2_density_matrix(None, 4, 2, ctypes.c_double(0.0), 10, None, None)
    assert st == -2  # SP2_ERR_NOT_INITIALIZED
    assert b"sp2_init" in lib.sp2_last_error()


def test_python_binding_fails_loudly_without_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2101_06385_gb300 as sp2

    with pytest.raises(Exception):
        sp2.density_matrix(torch.zeros(4, 4), 2)
