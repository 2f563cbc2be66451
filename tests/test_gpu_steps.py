"""GPU parity of the single steps of the path against the FP64 oracle.

Every call goes through the C ABI (via the ctypes binding).  Sizes span
several tiles and a ragged tail.
"""
import math

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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# ------------------------------------------------------------------ a1 bounds
@pytest.mark.parametrize("N", [1, 7, 300, 1000, 2053])
def test_gershgorin_matches_oracle(sp2, N):
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N)).astype(np.float32)
    A = ((A + A.T) / 2).astype(np.float32)
    A[np.diag_indices(N)] += np.float32(3.0)
    lo, hi = sp2.gershgorin(_cuda(A))
    wlo, whi = o.gershgorin_bounds(A.astype(np.float64))
    # float4 groups are pre-summed in FP32 (two roundings of 2^-24): relative 1e-6
    assert abs(lo - wlo) <= 1e-6 * max(1.0, abs(wlo))
    assert abs(hi - whi) <= 1e-6 * max(1.0, abs(whi))


# ------------------------------------------------------------------ Eq. 12 split
@pytest.mark.parametrize("s", [0, 11])
def test_split_is_bit_exact(sp2, s):
    rng = np.random.default_rng(s)
    N = 333
    X = (rng.uniform(-1, 1, (N, N)) * 10.0 ** rng.uniform(-9, 0, (N, N))).astype(np.float32)
    hi, lo = sp2.split(_cuda(X), s)
    ohi, olo = o.split_fp16(X, s)
    assert np.array_equal(hi.cpu().numpy().view(np.uint16), ohi.view(np.uint16))
    assert np.array_equal(lo.cpu().numpy().view(np.uint16), olo.view(np.uint16))


# ------------------------------------------------------------------ a4 layer
def _sym(rng, N, scale=1.0):
    A = rng.uniform(-1, 1, (N, N))
    return ((A + A.T) / 2 * scale).astype(np.float32)


def _fp32_bound(absA, absB, K, extra=0.0):
    # FP32 accumulation of K exact products: |err| <= K 2^-24 sum|a||b| (+ rounding of the result)
    return (K + 2) * 2.0 ** -24 * (absA @ absB) + extra


@pytest.mark.parametrize("N,B", [(300, 1), (512, 2), (1000, 1), (64, 3)])
@pytest.mark.parametrize("prec", ["split", "fp16", "fp32"])
def test_layer_matches_oracle(sp2, N, B, prec):
    rng = np.random.default_rng(N + B)
    X = np.stack([_sym(rng, N, 1.0 / math.sqrt(N)) for _ in range(B)])
    a, b, c = -1.0, 2.0, 0.25
    out, tr = sp2.layer(_cuda(X), a, b, c, precision=prec)
    out = out.cpu().numpy().astype(np.float64)
    for i in range(B):
        Xi = X[i]
        if prec == "fp32":
            P = Xi.astype(np.float64) @ Xi.astype(np.float64)
            absX = np.abs(Xi.astype(np.float64))
            bound = _fp32_bound(absX, absX, N)
        else:
            hi, lo = o.split_fp16(Xi, 11)
            P = o.split_square(hi, lo, 11, plain=(prec == "fp16"))
            ah, al = np.abs(hi.astype(np.float64)), np.abs(lo.astype(np.float64)) * 2.0 ** -11
            bound = _fp32_bound(ah, ah, N) + (0 if prec == "fp16" else 2 * _fp32_bound(ah, al, N))
        # the kernels take the diagonal of X^2 from FP64 row norms of the FP32 X
        P[np.diag_indices(N)] = np.sum(Xi.astype(np.float64) ** 2, axis=1)
        want = a * P + b * Xi.astype(np.float64) + c * np.eye(N)
        err = np.abs(out[i] - want)
        tol = abs(a) * bound + 2.0 ** -23 * np.abs(want) + 1e-30
        assert np.all(err <= tol), (prec, N, float(np.max(err)), float(np.max(err / tol)))
        # traces: tr X_out sums the FP64 diagonal before its rounding to FP32
        # (N roundings of at most 2^-24 |x_ii|), ||X_out||_F^2 the stored values
        d = np.abs(np.diag(out[i]))
        assert abs(tr[i][0] - np.trace(out[i])) <= 2.0 ** -24 * d.sum() + 1e-12
        assert abs(tr[i][1] - np.sum(out[i] ** 2)) <= 1e-6 * np.sum(out[i] ** 2)


def test_layer_is_symmetric_and_mirrored(sp2):
    rng = np.random.default_rng(5)
    N = 700
    X = _sym(rng, N, 0.05)
    out, _ = sp2.layer(_cuda(X), 1.0, 0.0, 0.0, precision="split")
    out = out.cpu().numpy()
    assert np.max(np.abs(out - out.T)) <= 1e-6 * np.max(np.abs(out))


def test_accumulation_bias(sp2):
    """All-positive square: the tensor-core off-diagonal sums come out biased
    low (truncating accumulation), the FFMA path does not; the diagonal, taken
    from FP64 row norms, is unbiased in every precision."""
    N = 2048
    rng = np.random.default_rng(0)
    X = (rng.uniform(0.5, 1.0, (N, N)) / N).astype(np.float32)
    X = ((X + X.T) / 2).astype(np.float32)
    exact = X.astype(np.float64) @ X.astype(np.float64)
    off = ~np.eye(N, dtype=bool)
    for prec in ("split", "fp32"):
        out, _ = sp2.layer(_cuda(X), 1.0, 0.0, 0.0, precision=prec)
        rel = (out.cpu().numpy().astype(np.float64) - exact) / exact
        print(f"{prec}: mean rel err off-diagonal {rel[off].mean():.3e}, diagonal {np.diag(rel).mean():.3e}")
        assert abs(np.diag(rel).mean()) < 1e-7
        if prec == "fp32":
            assert abs(rel[off].mean()) < 1e-7


# ------------------------------------------------------------------ observable
def test_observable(sp2):
    rng = np.random.default_rng(8)
    N = 1001
    D, A = _sym(rng, N), _sym(rng, N)
    v = sp2.observable(_cuda(D), _cuda(A))
    assert abs(v - np.sum(D.astype(np.float64) * A.astype(np.float64))) <= 1e-9 * N * N
