"""Accelerated Deep-NN SP2 on the GPU (Sec. "Accelerated Deep-NN SP2") against
the closed-form projector and the FP64 oracle's layer sequence."""
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
    return m


def _homo_lumo(h):
    return float(h.eps[: h.n_occ].max()), float(h.eps[h.n_occ:].min())


TOL = {"split": 5e-5, "fp16": 2e-3, "fp32": 5e-5}


@pytest.mark.parametrize("prec", ["split", "fp16", "fp32"])
@pytest.mark.parametrize("N", [300, 1000])
def test_matches_closed_form_and_oracle_layers(sp2, N, prec):
    h = si.gapped_hamiltonian(N, N // 2 - 3, (-1.0, -0.05), (0.05, 1.0), seed=31 + N)
    homo, lumo = _homo_lumo(h)
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix_accelerated(H, h.n_occ, homo, lumo, precision=prec)
    m = o.error_metrics(D.cpu().numpy().astype(np.float64), o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
    print(f"N={N} {prec}: {st.iterations} layers, max-abs {m['max_abs']:.2e}, trace err {m['trace_err']:.2e}")
    assert st.status == 0 and st.converged_by == "bounds"
    assert m["max_abs"] <= TOL[prec] and m["trace_err"] <= (1e-4 if prec != "fp16" else 1e-2)
    # same layer sequence as the FP64 oracle on the FP32 matrix
    r = o.sp2_accelerated(h.h32().astype(np.float64), h.n_occ, homo, lumo, tol=1e-9)
    assert st.sigmas == r.sigmas
    # and fewer layers than the trace-driven solve
    _, s2 = sp2.density_matrix(H, h.n_occ, precision=prec)
    assert st.iterations < s2.iterations + 2


def test_n4096_split(sp2):
    c = si.CONFIGS["n4096_split"]
    h = si.gapped_hamiltonian(c["N"], c["n_occ"], c["occ"], c["virt"], c["seed"], device="cuda")
    homo, lumo = _homo_lumo(h)
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix_accelerated(H, h.n_occ, homo, lumo)
    Dh = D.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2)
    ii, jj = rng.integers(0, c["N"], 4096), rng.integers(0, c["N"], 4096)
    want = np.einsum("ik,ik->i", h.Q[ii, : h.n_occ], h.Q[jj, : h.n_occ])
    err = np.max(np.abs(Dh[ii, jj] - want))
    print(f"N=4096 accelerated: {st.iterations} layers, sampled max-abs {err:.2e}")
    assert err <= 5e-5 and abs(np.trace(Dh) - h.n_occ) <= 1e-4


def test_conservative_estimates(sp2):
    h = si.gapped_hamiltonian(500, 200, (-1.0, -0.1), (0.1, 1.0), seed=41)
    homo, lumo = _homo_lumo(h)
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix_accelerated(H, h.n_occ, homo + 0.06, lumo - 0.06)
    m = o.error_metrics(D.cpu().numpy().astype(np.float64), o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
    assert m["max_abs"] <= 5e-5


def test_unsafe_and_invalid_estimates(sp2):
    h = si.gapped_hamiltonian(256, 128, (-1.0, -0.1), (0.1, 1.0), seed=43)
    H = torch.from_numpy(h.h32()).cuda()
    occ = np.sort(h.eps[: h.n_occ])
    # a gap reaching into the occupied band: eigenvalues cross, Tr D != N_occ
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix_accelerated(H, h.n_occ, float(occ[-20]), 0.9)
    assert e.value.status == -9
    # no gap
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix_accelerated(H, h.n_occ, 0.2, 0.1)
    assert e.value.status == -1
    # both estimates above the spectral bounds: no gap left after clamping (device check)
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix_accelerated(H, h.n_occ, 50.0, 60.0)
    assert e.value.status == -1
    # the library still works afterwards
    D, st = sp2.density_matrix(H, h.n_occ)
    assert st.status == 0


@pytest.mark.parametrize("N,n_occ", [(7, 3), (65, 1), (130, 129)])
def test_ragged_and_extreme_occupations(sp2, N, n_occ):
    h = si.gapped_hamiltonian(N, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=70 + N)
    homo, lumo = _homo_lumo(h)
    D, st = sp2.density_matrix_accelerated(torch.from_numpy(h.h32()).cuda(), n_occ, homo, lumo)
    m = o.error_metrics(D.cpu().numpy().astype(np.float64), o.density_matrix_closed_form(h.Q, n_occ), n_occ)
    assert st.status == 0 and m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4


def test_batched_accelerated(sp2):
    sizes = [300, 64, 777, 5, 1000]
    hs = [si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=810 + i) for i, N in enumerate(sizes)]
    Hs = [torch.from_numpy(h.h32()).cuda() for h in hs]
    hl = [_homo_lumo(h) for h in hs]
    Ds, stats = sp2.density_matrix_batched_accelerated(Hs, [h.n_occ for h in hs], [x[0] for x in hl],
                                                       [x[1] for x in hl])
    for h, D, st, (homo, lumo) in zip(hs, Ds, stats, hl):
        m = o.error_metrics(D.cpu().numpy().astype(np.float64), o.density_matrix_closed_form(h.Q, h.n_occ), h.n_occ)
        assert st.status == 0 and st.converged_by == "bounds"
        assert m["max_abs"] <= 5e-5 and m["trace_err"] <= 1e-4
        # the same layer sequence as solving the instance alone
        _, s1 = sp2.density_matrix_accelerated(torch.from_numpy(h.h32()).cuda(), h.n_occ, homo, lumo)
        assert s1.sigmas == st.sigmas
        assert abs(st.energy - float(np.sum(np.sort(h.eps)[: h.n_occ]))) <= 1e-5 * np.sum(np.abs(h.eps))
    # an unsafe estimate in one instance is reported
    bad = [x[1] for x in hl]
    occ1 = np.sort(hs[1].eps[: hs[1].n_occ])
    homo_bad = [x[0] for x in hl]
    homo_bad[1] = float(occ1[-8])
    bad[1] = 0.9
    with pytest.raises(sp2.SP2Error) as e:
        sp2.density_matrix_batched_accelerated(Hs, [h.n_occ for h in hs], homo_bad, bad)
    assert e.value.status == -9
