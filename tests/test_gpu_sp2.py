"""GPU parity of the whole SP2 solve (Alg. 1 + Eq. 15) against the FP64 oracle.

Tolerances (split-FP16 path): max-abs <= 5e-5 and |tr D - N_occ| <= 1e-4;
plain FP16: max-abs <= 2e-3.  The exact D is the closed form Q_occ Q_occ^T
of the generated spectrum (Eq. 6).
"""
import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split": 5e-5, "fp32": 5e-5, "fp16": 2e-3}


@pytest.fixture(scope="module")
def sp2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as m

    m.init(0)
    return m


def _solve(sp2, h, prec, tol=0.0, max_iter=100):
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix(H, h.n_occ, tol=tol, max_iter=max_iter, precision=prec)
    return D.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("prec", ["split", "fp16", "fp32"])
def test_n128_config(sp2, prec):
    c = si.CONFIGS["n128_fp64"]
    h = si.gapped_hamiltonian(c["N"], c["n_occ"], c["occ"], c["virt"], c["seed"])
    D, st = _solve(sp2, h, prec)
    m = o.error_metrics(D, o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
    assert st.status == 0
    assert m["max_abs"] <= TOL[prec], m
    if prec != "fp16":
        assert m["trace_err"] <= 1e-4, m
    # branch sequence against the FP64 oracle, up to the last few (noise-decided) layers
    r = o.sp2(h.H.astype(np.float32).astype(np.float64), h.n_occ)
    k = min(len(r.sigmas), st.iterations) - 6
    assert st.sigmas[:k] == r.sigmas[:k]


@pytest.mark.parametrize("N,n_occ", [(257, 100), (1000, 500), (1536, 1)])
def test_ragged_sizes(sp2, N, n_occ):
    h = si.gapped_hamiltonian(N, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=N)
    D, st = _solve(sp2, h, "split")
    m = o.error_metrics(D, o.density_matrix_closed_form(h.Q, n_occ), n_occ)
    assert st.status == 0 and m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4, (m, st.iterations)


@pytest.mark.parametrize("prec", ["split", "fp16", "fp32"])
def test_n4096_config(sp2, prec):
    c = si.CONFIGS["n4096_split"]
    h = si.gapped_hamiltonian(c["N"], c["n_occ"], c["occ"], c["virt"], c["seed"])
    D, st = _solve(sp2, h, prec)
    m = o.error_metrics(D, o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
    print(prec, st.iterations, st.converged_by, m, st.time_ms)
    assert st.status == 0
    assert m["max_abs"] <= TOL[prec], m
    if prec != "fp16":
        assert m["trace_err"] <= 1e-4, m
    assert 30 <= st.iterations <= 50


def test_occupation_extremes(sp2):
    for n_occ in (0, 200):
        h = si.gapped_hamiltonian(200, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=9)
        D, st = _solve(sp2, h, "split")
        want = np.zeros((200, 200)) if n_occ == 0 else np.eye(200)
        assert np.max(np.abs(D - want)) <= 5e-5


def test_tiny_and_2x2(sp2):
    for a, b, d in [(0.3, -0.2, -0.5), (1.0, 0.5, 0.25)]:
        H = np.array([[a, b], [b, d]])
        t = 0.5 * (a + d)
        r = np.sqrt((0.5 * (a - d)) ** 2 + b * b)
        D_exact = 0.5 * (np.eye(2) - (H - t * np.eye(2)) / r)
        Dg, st = sp2.density_matrix(torch.tensor(H, dtype=torch.float32).cuda(), 1)
        assert np.max(np.abs(Dg.cpu().numpy() - D_exact)) <= 5e-5
    for n_occ in (0, 1):
        Dg, st = sp2.density_matrix(torch.tensor([[0.7]], dtype=torch.float32).cuda(), n_occ)
        assert abs(float(Dg.cpu()[0, 0]) - n_occ) <= 1e-6


def test_errors(sp2):
    H = torch.eye(64, device="cuda") * 0.5
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix(H, 10)
    assert e.value.status == -3  # degenerate
    Hn = torch.randn(64, 64, device="cuda")
    Hn[3, 5] = float("nan")
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix(Hn, 10)
    assert e.value.status == -4  # non-finite
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix(torch.zeros(8, 8, device="cuda"), 9)
    assert e.value.status == -1
    # a cI Hamiltonian with N_occ in {0, N} is well posed
    D, st = sp2.density_matrix(H, 64)
    assert torch.allclose(D, torch.eye(64, device="cuda"), atol=1e-6)


def test_max_iter_reports_not_converged(sp2):
    """A solve cut off at max_iter still returns f_final of its last iterate
    (Eq. 15), written whole although the iterate is kept as its upper
    triangle between the layers: it matches the oracle's five-layer result
    and is symmetric."""
    h = si.gapped_hamiltonian(300, 150, seed=2)
    D, st = _solve(sp2, h, "split", max_iter=5)
    assert st.status == 1 and st.iterations == 5 and st.converged_by == "max_iter"
    want = o.sp2(h.h32().astype(np.float64), h.n_occ, max_iter=5).D
    assert np.max(np.abs(D - want)) <= 5e-5
    assert np.max(np.abs(D - D.T)) <= 1e-6


@pytest.mark.parametrize("N", [257, 1000])
def test_fused_energy(sp2, N):
    """Tr[D H] (Alg. 1, last line) accumulated by the launch that writes D
    equals the observable of the returned D and the exact band energy."""
    h = si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=50 + N)
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix(H, h.n_occ, precision="split")
    e_obs = sp2.observable(D, H)
    e_exact = float(np.sum(np.sort(h.eps)[: h.n_occ]))
    print(f"N={N}: fused {st.energy:.9f} observable {e_obs:.9f} exact {e_exact:.9f}")
    assert abs(st.energy - e_obs) <= 1e-6 * np.sum(np.abs(h.eps))
    assert abs(st.energy - e_exact) <= 1e-5 * np.sum(np.abs(h.eps))
    Da, sa = sp2.density_matrix_accelerated(H, h.n_occ, float(np.max(h.eps[: h.n_occ])),
                                            float(np.min(h.eps[h.n_occ:])))
    assert abs(sa.energy - sp2.observable(Da, H)) <= 1e-6 * np.sum(np.abs(h.eps))
