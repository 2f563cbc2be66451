"""Full-size parity: the N = 16384 workload in the launch configuration the
benchmark times (split-FP16, default max_iter), checked on sampled entries
of D against the closed form Q_occ Q_occ^T (Eq. 6) and on the trace."""
import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as sp2

    c = si.CONFIGS["n16384_split"]
    h = si.gapped_hamiltonian(c["N"], c["n_occ"], c["occ"], c["virt"], c["seed"], device="cuda")
    sp2.init(0)
    return sp2, h


def test_n16384_sampled_parity_and_determinism(big):
    sp2, h = big
    N, n_occ = h.N, h.n_occ
    H = torch.from_numpy(h.h32()).cuda()
    D1, st1 = sp2.density_matrix(H, n_occ, precision="split")
    D2, st2 = sp2.density_matrix(H, n_occ, precision="split")
    assert st1.status == 0
    # deterministic: fixed-order FP64 reductions, static tile schedule
    assert st1.sigmas == st2.sigmas and torch.equal(D1, D2)
    rng = np.random.default_rng(7)
    rows = rng.integers(0, N, 64)
    cols = rng.integers(0, N, 64)
    want = o.density_matrix_closed_form(h.Q, n_occ, rows, cols)
    got = D1[torch.as_tensor(rows).cuda()][:, torch.as_tensor(cols).cuda()].cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - want))
    diag = torch.diagonal(D1).double().sum().item()
    print(f"N={N} layers={st1.iterations} stop={st1.converged_by} max_abs(sampled 64x64)={err:.3e} "
          f"|trD-Nocc|={abs(diag - n_occ):.3e} time={st1.time_ms:.1f} ms")
    assert err <= 5e-5
    assert abs(diag - n_occ) <= 1e-4
    # symmetry of the mirrored stores
    blk = D1[:512, -512:].cpu().numpy()
    blkT = D1[-512:, :512].cpu().numpy().T
    assert np.max(np.abs(blk - blkT)) <= 1e-6


def test_n16384_whole_super_rows(big):
    """Three complete 256-row blocks of D (the first, middle and last super
    rows, all 16384 columns) against Q_occ Q_occ^T element by element.  Every
    K block of these rows' products was read both ways (K-major right of the
    diagonal, transposed from the stored upper block left of it), so a wrong
    transposed read in any super-tile column shows up here."""
    sp2, h = big
    N, n_occ = h.N, h.n_occ
    H = torch.from_numpy(h.h32()).cuda()
    D, st = sp2.density_matrix(H, n_occ, precision="split")
    assert st.status == 0
    T = (N + 255) // 256
    worst = 0.0
    for I in (0, T // 2, T - 1):
        rows = np.arange(I * 256, min(N, (I + 1) * 256))
        want = o.density_matrix_closed_form(h.Q, n_occ, rows, None)
        got = D[int(rows[0]): int(rows[-1]) + 1].cpu().numpy().astype(np.float64)
        err = float(np.max(np.abs(got - want)))
        worst = max(worst, err)
        print(f"super row {I}: max_abs over {got.size} entries = {err:.3e}")
        assert err <= 5e-5
    print(f"N={N}: whole super rows worst max_abs = {worst:.3e}")


@pytest.mark.parametrize("N,precision", [(1000, "split"), (4096, "split"), (1000, "fp16"), (2053, "fp16")])
def test_wide_units_match_single_super_tiles(N, precision):
    """The CTA-pair kernel's wide units (two super tiles of a row per pass,
    the A panel loaded once; chosen automatically at N = 16384) give the same
    bits as one super tile per pass: each tile's products and epilogue are
    unchanged, only the order of the FP64 tile partials differs, and no
    branch decision moves.  Both sizes have rows with an odd last tile (a
    unit with a null second tile)."""
    import os

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as sp2

    h = si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=60 + N % 89)
    H = torch.from_numpy(h.h32()).cuda()
    out = {}
    try:
        for mode in ("0", "1"):
            os.environ["SP2_WIDE"] = mode
            sp2.finalize()
            sp2.init(0)
            D, st = sp2.density_matrix(H, N // 2, precision=precision)
            assert st.status == 0, st
            out[mode] = (D.clone(), st.iterations, st.sigmas)
    finally:
        os.environ.pop("SP2_WIDE", None)
        sp2.finalize()
        sp2.init(0)
    assert torch.equal(out["0"][0], out["1"][0])
    assert out["0"][1:] == out["1"][1:]
    m = o.error_metrics(out["1"][0].cpu().numpy().astype(np.float64), o.density_matrix_closed_form(h.Q, N // 2),
                        N // 2)
    tol = 5e-5 if precision == "split" else 2e-3
    assert m["max_abs"] <= tol and m["trace_err"] <= 1e-4 * (1 if precision == "split" else 20), m
