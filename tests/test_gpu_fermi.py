"""Finite-temperature expansion on the GPU (Sec. "Optimized SP2 Finite
Temperature Fermi-Operator Expansion") against the FP64 oracle's matrix form
and the Fermi-Dirac matrix, with the oracle-fitted beta = 40, 11-layer
coefficients."""
import json
import os

import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def sp2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as m

    m.init(0)
    return m


def _fit():
    with open(os.path.join(HERE, "golden", "fermi_fit_beta40_L11.json")) as f:
        d = json.load(f)
    return np.array(d["theta"]), np.array(d["c"])


@pytest.mark.parametrize("prec,tol", [("split", 1e-4), ("fp16", 3e-3)])
@pytest.mark.parametrize("B,N", [(3, 300), (1, 1000)])
def test_matches_oracle_matrix_form(sp2, B, N, prec, tol):
    theta, c = _fit()
    hs = [si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=600 + i) for i in range(B)]
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    sp2.set_precision(prec)
    try:
        D, bounds = sp2.fermi_expansion(H, theta, c)
    finally:
        sp2.set_precision("split")
    Dh = D.cpu().numpy().astype(np.float64)
    bh = bounds.cpu().numpy()
    for b, h in enumerate(hs):
        H64 = h.h32().astype(np.float64)
        lo, hi = o.gershgorin_bounds(H64)
        assert abs(bh[b, 0] - lo) <= 1e-6 * abs(lo) and abs(bh[b, 1] - hi) <= 1e-6 * abs(hi)
        # the oracle maps the spectrum with its own bounds
        want = o.fermi_expansion_matrix(H64, theta, c, (lo, hi))
        err = np.max(np.abs(Dh[b] - want))
        eps = (h.eps - lo) / (hi - lo)
        fd = (h.Q * o.fermi_dirac_scaled(eps, 40.0)) @ h.Q.T
        efd = np.max(np.abs(Dh[b] - fd))
        print(f"{prec} B={B} N={N} inst {b}: vs oracle {err:.2e}, vs Fermi-Dirac {efd:.2e}")
        assert err <= tol
        assert np.max(np.abs(Dh[b] - Dh[b].T)) <= 1e-6


def test_fixed_window(sp2):
    """An explicit energy window maps [e_lo, e_hi] to [0, 1] for every instance."""
    theta, c = _fit()
    h = si.gapped_hamiltonian(400, 200, (-1.0, -0.1), (0.1, 1.0), seed=77)
    H = torch.from_numpy(h.h32()).cuda()
    D, bounds = sp2.fermi_expansion(H, theta, c, window=(-1.5, 1.5))
    assert np.allclose(bounds.cpu().numpy(), [[-1.5, 1.5]])
    want = o.fermi_expansion_matrix(h.h32().astype(np.float64), theta, c, (-1.5, 1.5))
    assert np.max(np.abs(D.cpu().numpy() - want)) <= 1e-4
    # trace against the scalar expansion on the exact spectrum
    eps = (h.eps + 1.5) / 3.0
    assert abs(float(torch.trace(D.double())) - np.sum(o.fermi_expansion_scalar(theta, c, eps))) <= 1e-3


def test_invalid_arguments(sp2):
    theta, c = _fit()
    H = torch.zeros(64, 64, device="cuda")
    with pytest.raises(sp2.SP2Error):
        sp2.fermi_expansion(H, theta, c, window=(1.0, -1.0))
    with pytest.raises(ValueError):
        sp2.fermi_expansion(H, theta, c[:-1])
    sp2.set_precision("fp32")
    try:
        with pytest.raises(sp2.SP2Error) as e:
            sp2.fermi_expansion(H + torch.eye(64, device="cuda"), theta, c)
        assert e.value.status == -8
    finally:
        sp2.set_precision("split")


@pytest.mark.parametrize("N", [1, 5, 130])
def test_ragged_and_tiny_sizes(sp2, N):
    """Sizes below one tile and not a multiple of 4 (scalar paths)."""
    theta, c = _fit()
    rng = np.random.default_rng(N)
    A = rng.uniform(-1.0, 1.0, (N, N))
    H64 = ((A + A.T) / 2).astype(np.float32).astype(np.float64)
    H = torch.from_numpy(H64.astype(np.float32)).cuda()
    D, bounds = sp2.fermi_expansion(H, theta, c)
    lo, hi = bounds.cpu().numpy()[0]
    want = o.fermi_expansion_matrix(H64, theta, c, (lo, hi))
    assert np.max(np.abs(D.cpu().numpy() - want)) <= 1e-4
