"""The allocation-free entry point (for callers that cannot allocate device
memory when they need D: a fixed memory budget, a real-time loop that an
allocation would stall, a host that manages all device memory itself) gives
the same density matrix as sp2_density_matrix, call after call, through the
C ABI."""
import ctypes

import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as sp2

    sp2.init(0)
    lib = ctypes.CDLL(sp2.library_path())
    fn = lib.sp2_density_matrix_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    lib.sp2_last_error.restype = ctypes.c_char_p
    return sp2, lib, fn


def test_noalloc_matches_density_matrix_on_consecutive_calls(libs):
    sp2, lib, fn = libs
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row; the second one finds the first one's data in the scratch
    for N, n_occ, seed in [(1000, 400, 21), (512, 256, 22), (1000, 400, 21)]:
        h = si.gapped_hamiltonian(N, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=seed)
        H = torch.from_numpy(h.h32()).cuda()
        D_ref, st_ref = sp2.density_matrix(H, n_occ, precision="split")
        D = torch.full_like(H, float("nan"))
        st = sp2._Stats()
        status = fn(H.data_ptr(), N, n_occ, 0.0, 100, D.data_ptr(), ctypes.byref(st), stream)
        assert status == 0, lib.sp2_last_error()
        Dn = D.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(Dn - D_ref.cpu().numpy())) <= 5e-5
        m = o.error_metrics(Dn, o.density_matrix_closed_form(h.Q, n_occ), n_occ)
        assert m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4, m
        assert st.iterations > 0 and st.converged_by in (1, 2, 3)


def _call(fn, H, N, n_occ, D, st, stream):
    return fn(H.data_ptr(), N, n_occ, 0.0, 100, D.data_ptr(), ctypes.byref(st) if st is not None else None, stream)


@pytest.mark.parametrize("N", [1, 2, 33, 1024])
def test_noalloc_edge_sizes_against_the_closed_form(libs, N):
    """One row, a 2 x 2 problem, a size below one 128-row tile, and the
    documented maximum SP2_NOALLOC_MAX_N."""
    sp2, lib, fn = libs
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n_occ = N // 2
    h = si.gapped_hamiltonian(N, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=30 + N)
    H = torch.from_numpy(h.h32()).cuda()
    D = torch.full_like(H, float("nan"))
    st = sp2._Stats()
    status = _call(fn, H, N, n_occ, D, st, stream)
    assert status == 0, lib.sp2_last_error()
    m = o.error_metrics(D.cpu().numpy(), o.density_matrix_closed_form(h.Q, n_occ), n_occ)
    print(f"noalloc N={N}: layers={st.iterations} max_abs={m['max_abs']:.2e} trace_err={m['trace_err']:.2e}")
    assert m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4, m


def test_noalloc_leaves_free_device_memory_unchanged(libs):
    """After one warm call, a further call changes neither the device's free
    memory (cudaMemGetInfo) nor the memory torch's allocator holds."""
    sp2, lib, fn = libs
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = si.gapped_hamiltonian(700, 350, (-1.0, -0.1), (0.1, 1.0), seed=41)
    H = torch.from_numpy(h.h32()).cuda()
    D = torch.empty_like(H)
    st = sp2._Stats()
    assert _call(fn, H, 700, 350, D, st, stream) == 0, lib.sp2_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for _ in range(2):
        assert _call(fn, H, 700, 350, D, None, stream) == 0
        assert _call(fn, H, 700, 350, D, st, stream) == 0, lib.sp2_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == res0


def test_noalloc_rejects_sizes_beyond_its_maximum(libs):
    sp2, lib, fn = libs
    H = torch.zeros(1025, 1025, device="cuda")
    D = torch.empty_like(H)
    status = fn(H.data_ptr(), 1025, 10, 0.0, 100, D.data_ptr(), None, None)
    assert status == -1
    assert b"SP2_NOALLOC_MAX_N" in lib.sp2_last_error()
