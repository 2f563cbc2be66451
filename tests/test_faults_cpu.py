"""Host side of the fault injection (failure detection without a GPU fault):
the fault specification is parsed by the library without a GPU, bad
specifications are refused before anything changes, and SP2_FAULT in the
environment is applied by sp2_init before it touches a device."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_06385_gb300 import _build

    l = ctypes.CDLL(_build.build())
    l.sp2_set_fault.restype = ctypes.c_int
    l.sp2_set_fault.argtypes = [ctypes.c_char_p]
    l.sp2_last_error.restype = ctypes.c_char_p
    return l


@pytest.mark.parametrize("spec", [b"", b"none", b"alloc_fail", b"nan_input", b"timeout", b"wait_ms=50",
                                  b"timeout,wait_ms=100", b"alloc_fail,nan_input,timeout,wait_ms=60000"])
def test_valid_specifications_are_accepted(lib, spec):
    assert lib.sp2_set_fault(spec) == 0, lib.sp2_last_error()
    assert lib.sp2_set_fault(None) == 0


@pytest.mark.parametrize("spec", [b"bogus", b"timeout,bogus", b"wait_ms=", b"wait_ms=0", b"wait_ms=60001",
                                  b"wait_ms=12x", b"alloc_fail;nan_input"])
def test_invalid_specifications_are_refused(lib, spec):
    assert lib.sp2_set_fault(spec) == -1  # SP2_ERR_INVALID_ARG
    assert b"sp2_set_fault" in lib.sp2_last_error()


def _init_in_child(env_value):
    code = (
        "import ctypes, paper_2101_06385_gb300 as m\n"
        "l = ctypes.CDLL(m.library_path()); l.sp2_last_error.restype = ctypes.c_char_p\n"
        "print(l.sp2_init(None), l.sp2_last_error().decode())\n")
    env = dict(os.environ, SP2_FAULT=env_value, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    status, _, msg = r.stdout.strip().partition(" ")
    return int(status), msg


def test_environment_fault_is_parsed_by_init(lib):
    # a malformed SP2_FAULT stops sp2_init before any device call
    status, msg = _init_in_child("nonsense")
    assert status == -1 and "unknown item" in msg
    # a valid one passes the parser; with no visible device the CUDA query fails next
    status, msg = _init_in_child("timeout,wait_ms=100")
    assert status == -5, msg  # SP2_ERR_CUDA
