"""Failure detection on the GPU without a GPU fault: each injected fault
(sp2_set_fault) takes its error path, reports its status, and leaves the
library usable; the next call returns the correct density matrix.  The
time-out case makes a bounded device wait run out (a barrier that nothing
arrives on) under a 100 ms bound, so the whole call ends within a second or
so; no trap, no invalid access, no unbounded wait."""
import time

import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as m

    m.init(0)
    m.set_precision("split")
    yield m
    m.set_fault(None)


@pytest.fixture(scope="module")
def case():
    h = si.gapped_hamiltonian(512, 200, (-1.0, -0.1), (0.1, 1.0), seed=91)
    return h, torch.from_numpy(h.h32()).cuda()


def _good_solve(sp2, h, H):
    D, st = sp2.density_matrix(H, h.n_occ)
    m = o.error_metrics(D.cpu().numpy(), o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
    assert st.status == 0 and m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4, m


@pytest.mark.parametrize("kernel", ["pairs", "single"])
def test_device_wait_runs_out(sp2, case, kernel, monkeypatch):
    h, H = case
    if kernel == "single":
        # the single-CTA squaring kernel is selected at sp2_init
        monkeypatch.setenv("SP2_SQUARE_KERNEL", "single")
        sp2.init(0)
    try:
        sp2.set_fault("timeout,wait_ms=100")
        D = torch.empty_like(H)
        t0 = time.perf_counter()
        with pytest.raises(sp2.SP2Error) as e:
            sp2.density_matrix(H, h.n_occ, out=D)
        dt = time.perf_counter() - t0
        assert e.value.status == -7  # SP2_ERR_DEVICE_TIMEOUT
        assert dt < 30.0
        sp2.set_fault(None)  # back to the 4 s bound
        # every CTA freed its tensor memory and left: the next solve (one
        # 512-column allocation per SM again) runs and is correct
        _good_solve(sp2, h, H)
    finally:
        sp2.set_fault(None)
        if kernel == "single":
            monkeypatch.delenv("SP2_SQUARE_KERNEL")
            sp2.init(0)


def test_injected_allocation_failure(sp2, case):
    h, H = case
    D = torch.full_like(H, 7.0)
    sp2.set_fault("alloc_fail")
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix(H, h.n_occ, out=D)
    assert e.value.status == -6  # SP2_ERR_OOM
    torch.cuda.synchronize()
    assert bool((D == 7.0).all())  # refused before any work was enqueued
    _good_solve(sp2, h, H)


def test_injected_nan_input(sp2, case):
    h, H = case
    sp2.set_fault("nan_input")
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix(H, h.n_occ)
    assert e.value.status == -4  # SP2_ERR_NONFINITE
    _good_solve(sp2, h, H)
