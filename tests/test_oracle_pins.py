"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types an oracle formula: each compares the oracle to
an independent quantity (the generator's exact spectrum, a closed form, an
invariant, brute force, finite differences, or a number the paper prints).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _paper():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------- bounds, S_0
def test_gershgorin_hand_example():
    H = np.array([[2.0, -1.0, 0.5], [-1.0, 3.0, 0.0], [0.5, 0.0, -1.0]])
    # discs: [0.5, 3.5], [2, 4], [-1.5, -0.5]
    assert o.gershgorin_bounds(H) == (-1.5, 4.0)


@pytest.mark.parametrize("N,seed", [(64, 0), (200, 3)])
def test_gershgorin_encloses_exact_spectrum(N, seed):
    h = si.gapped_hamiltonian(N, N // 2, seed=seed)
    lo, hi = o.gershgorin_bounds(h.H)
    assert lo <= h.eps.min() and hi >= h.eps.max()


def test_input_layer_reverses_spectrum_into_unit_interval():
    h = si.gapped_hamiltonian(96, 40, seed=5)
    lo, hi = o.gershgorin_bounds(h.H)
    S0 = o.input_layer(h.H, lo, hi)
    got = np.linalg.eigvalsh(S0)
    want = np.sort((hi - h.eps) / (hi - lo))
    assert np.max(np.abs(got - want)) < 1e-13
    assert got.min() >= 0.0 and got.max() <= 1.0


# ------------------------------------------------------------- SP2 vs exact D
def test_sp2_n128_matches_closed_form():
    c = si.CONFIGS["n128_fp64"]
    h = si.gapped_hamiltonian(c["N"], c["n_occ"], c["occ"], c["virt"], c["seed"])
    r = o.sp2(h.H, h.n_occ, tol=1e-12, max_iter=100)
    D = o.density_matrix_closed_form(h.Q, h.n_occ)
    m = o.error_metrics(r.D, D, h.n_occ)
    assert m["max_abs"] <= 1e-12
    assert m["trace_err"] <= 1e-10
    assert 25 <= r.n_layers <= 36


def test_sp2_2x2_analytic():
    rng = np.random.default_rng(11)
    for _ in range(20):
        a, b, d = rng.uniform(-1, 1, 3)
        if abs(b) < 1e-3:
            continue
        H = np.array([[a, b], [b, d]])
        t = 0.5 * (a + d)
        r = math.sqrt((0.5 * (a - d)) ** 2 + b * b)
        D_exact = 0.5 * (np.eye(2) - (H - t * np.eye(2)) / r)
        res = o.sp2(H, 1)
        assert np.max(np.abs(res.D - D_exact)) < 1e-10
        assert np.max(np.abs(o.sp2(H, 0).D)) < 1e-10
        assert np.max(np.abs(o.sp2(H, 2).D - np.eye(2))) < 1e-10


@pytest.mark.parametrize("n_occ", [0, 37, 96])
def test_sp2_invariants(n_occ):
    h = si.gapped_hamiltonian(96, n_occ, (-1.0, -0.1), (0.1, 1.0), seed=7)
    D = o.sp2(h.H, n_occ).D
    assert np.max(np.abs(D @ D - D)) < 1e-12
    assert abs(np.trace(D) - n_occ) < 1e-10
    assert np.max(np.abs(D @ h.H - h.H @ D)) < 1e-12
    w = np.linalg.eigvalsh(D)
    assert np.all((np.abs(w) < 1e-10) | (np.abs(w - 1) < 1e-10))
    assert np.max(np.abs(D - o.density_matrix_closed_form(h.Q, n_occ))) < 1e-11


def _scalar_sp2(lam, n_occ, max_iter=100):
    """SP2 acting on eigenvalues (written independently of the oracle)."""
    lam = np.array(lam, dtype=np.float64)
    sig_prev, sig_prev2 = 0, 0
    errs = {}
    sigmas = []
    for n in range(1, max_iter + 1):
        ns, nx = lam.sum(), (lam * lam).sum()
        err = ns - nx
        keep_square = abs(nx - n_occ) <= abs(2 * ns - nx - n_occ)
        s = 1 if keep_square else -1
        lam = lam * lam if s == 1 else 2 * lam - lam * lam
        sigmas.append(s)
        errs[n] = err
        stop = err <= 0 or (n > 2 and sig_prev != sig_prev2 and err > 4.5 * errs[n - 2] ** 2)
        sig_prev2, sig_prev = sig_prev, s
        if stop:
            break
    return sigmas


def test_sp2_branch_sequence_equals_eigenvalue_recurrence():
    h = si.gapped_hamiltonian(128, 64, (-1.0, -0.1), (0.1, 1.0), seed=0)
    r = o.sp2(h.H, 64)
    lam0 = (r.e_max - h.eps) / (r.e_max - r.e_min)
    sig = _scalar_sp2(lam0, 64)
    # the last few layers are decided by rounding noise; the rest must agree
    k = len(sig) - 4
    assert r.sigmas[:k] == sig[:k]
    assert abs(len(sig) - r.n_layers) <= 2


# ----------------------------------------------------------------- refinement
def test_f_final_is_alternating_composition():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    lam = rng.uniform(0, 1, 24)
    S = (Q * lam) @ Q.T
    for s, f in [(1, lambda x: 2 * x * x - x ** 4), (-1, lambda x: (2 * x - x * x) ** 2)]:
        got = o.f_final(S, s)
        want = (Q * f(lam)) @ Q.T
        assert np.max(np.abs(got - want)) < 1e-13


def test_theorem_constant_matches_paper():
    p = _paper()["theorem_constant"]
    closed = (71.0 + 17.0 * math.sqrt(17.0)) / 32.0
    C = o.theorem_constant()
    assert abs(C - closed) < 1e-10
    assert abs(C - p["approx"]) < 0.005
    assert C < _paper()["convergence_threshold"]["value"]


def test_theorem_inequality_holds_for_refinement():
    C = (71.0 + 17.0 * math.sqrt(17.0)) / 32.0
    rng = np.random.default_rng(4)
    for trial in range(10):
        Q, _ = np.linalg.qr(rng.standard_normal((32, 32)))
        lam = rng.uniform(0, 1, 32) ** rng.uniform(0.2, 5)
        S = (Q * lam) @ Q.T
        e0 = np.trace(S - S @ S)
        for s in (1, -1):
            T = o.f_final(S, s)
            e2 = np.trace(T - T @ T)
            assert e2 <= C * e0 * e0 * (1 + 1e-9) + 1e-12


def test_idempotency_trace_bracket():
    rng = np.random.default_rng(9)
    for _ in range(10):
        N = 20
        Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
        X = (Q * rng.uniform(0, 1, N)) @ Q.T
        E = X - X @ X
        two = np.linalg.norm(E, 2)
        tr = np.trace(E)
        assert two <= tr + 1e-12 and tr <= N * two + 1e-12


# ------------------------------------------------------- Fig. 5 and Fig. 2
def test_fig5_plain_layer_count_band():
    p = _paper()["fig5_plain_layers"]
    counts = []
    for seed in range(5):
        h = si.uniform_random_symmetric(p["N"], p["n_occ"], seed)
        w = np.linalg.eigvalsh(h.H)
        counts.append(o.sp2(h.H, p["n_occ"], bounds=(w[0], w[-1])).n_layers)
    assert all(25 <= c <= 36 for c in counts), counts
    assert abs(np.mean(counts) - p["value"]) <= 4


def test_fig2_refinement_gains_orders():
    """Fig. 2: once the iterate is close to idempotent, the refinement layer
    (two alternating layers at once) improves idempotency by orders of
    magnitude (quadratic in the error)."""
    p = _paper()["fig2_example"]
    h = si.uniform_random_symmetric(p["N"], p["n_occ"], 0)
    for m in range(5, 60):
        r = o.sp2(h.H, p["n_occ"], max_iter=m, refine=True)
        S = r.S_last
        before = np.linalg.norm(S @ S - S, 2)
        if before < 1e-3:
            break
    after = np.linalg.norm(r.D @ r.D - r.D, 2)
    assert 1e-9 < before < 1e-3
    assert after < before * 1e-2


# -------------------------------------------------------------- eigen-solver
@pytest.mark.parametrize("N", [33, 64])
def test_jacobi_against_generator(N):
    h = si.gapped_hamiltonian(N, N // 2, (-1.0, -0.1), (0.1, 1.0), seed=N)
    w, V = o.jacobi_eigh(h.H)
    assert np.max(np.abs(w - h.eps)) < 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(N))) < 1e-13
    assert np.max(np.abs(h.H @ V - V * w)) < 1e-13
    D = o.density_matrix_jacobi(h.H, N // 2)
    assert np.max(np.abs(D - o.density_matrix_closed_form(h.Q, N // 2))) < 1e-12


def test_closed_form_subblock_entries():
    h = si.gapped_hamiltonian(50, 20, seed=1)
    D = o.density_matrix_closed_form(h.Q, 20)
    rows, cols = np.array([3, 7, 49]), np.array([0, 7, 11])
    assert np.allclose(o.density_matrix_closed_form(h.Q, 20, rows, cols), D[np.ix_(rows, cols)], atol=1e-15)


# ------------------------------------------------------------------- Fermi
def test_fermi_dirac_limits():
    h = si.gapped_hamiltonian(40, 20, (-1.0, -0.1), (0.1, 1.0), seed=2)
    cold = o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 1e-4)
    assert np.max(np.abs(cold - o.density_matrix_closed_form(h.Q, 20))) < 1e-12
    warm = o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05)
    f = 1.0 / (1.0 + np.exp(h.eps / 0.05))
    assert abs(np.trace(warm) - f.sum()) < 1e-12
    w = np.linalg.eigvalsh(warm)
    assert w.min() > 0 and w.max() < 1


# ------------------------------------------------------------------- split
def _nearest_fp16_bruteforce(x):
    """Nearest FP16 to x, ties to the even significand, by enumerating all
    finite FP16 bit patterns."""
    allh = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    allh = np.concatenate([-allh[::-1], allh])
    bits = np.concatenate([np.arange(0x7C00 - 1, -1, -1, dtype=np.uint16) | 0x8000,
                           np.arange(0, 0x7C00, dtype=np.uint16)])
    i = np.searchsorted(allh, x)
    best = None
    for j in (i - 1, i):
        if 0 <= j < len(allh):
            d = abs(allh[j] - x)
            if best is None or d < best[0] or (d == best[0] and bits[j] % 2 == 0):
                best = (d, allh[j])
    return best[1]


def test_split_fp16_rounds_to_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-1, 1, 300) * 10.0 ** rng.integers(-7, 1, 300),
                        [2049.0 / 2048 / 1024, 2051.0 / 2048 / 1024, 1e-7, -3e-8]]).astype(np.float32)
    for s in (0, 11):
        hi, lo = o.split_fp16(x, s)
        for xv, hv in zip(x.astype(np.float64), hi.astype(np.float64)):
            assert hv == _nearest_fp16_bruteforce(xv)
        r = (x.astype(np.float64) - hi.astype(np.float64)) * 2.0 ** s
        for rv, lv in zip(r, lo.astype(np.float64)):
            assert lv == _nearest_fp16_bruteforce(rv)


def test_split_fp16_scaled_low_part_is_accurate():
    rng = np.random.default_rng(1)
    x = (rng.uniform(-1, 1, 5000) * 10.0 ** rng.uniform(-4, 0, 5000)).astype(np.float32)
    hi, lo = o.split_fp16(x, 11)
    rec = hi.astype(np.float64) + lo.astype(np.float64) * 2.0 ** -11
    err = np.abs(rec - x.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(x) + 2.0 ** -36)


def test_split_square_exact_small():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (4, 4)).astype(np.float32)
    X = (X + X.T) / 2
    hi, lo = o.split_fp16(X, 11)
    got = o.split_square(hi, lo, 11)
    H = [[Fraction(float(v)) for v in row] for row in hi.astype(np.float64)]
    L = [[Fraction(float(v)) / 2048 for v in row] for row in lo.astype(np.float64)]
    for i in range(4):
        for j in range(4):
            e = sum(H[i][k] * H[k][j] + H[i][k] * L[k][j] + L[i][k] * H[k][j] for k in range(4))
            assert abs(float(e) - got[i, j]) <= 1e-15 * max(1.0, abs(float(e)))


# ----------------------------------------------------------------- network
def test_network_forward_is_polynomial_of_eigenvalues():
    rng = np.random.default_rng(5)
    N, L = 20, 7
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = rng.uniform(0, 1, N)
    coef = rng.uniform(-1, 1, (L, 3))
    XL = o.network_forward((Q * lam) @ Q.T, coef)
    x = lam.copy()
    for a, b, c in coef:
        x = a * x * x + b * x + c
    assert np.max(np.abs(XL - (Q * x) @ Q.T)) < 1e-12


def test_network_with_branch_coefficients_reproduces_sp2_layers():
    h = si.gapped_hamiltonian(64, 32, (-1.0, -0.1), (0.1, 1.0), seed=1)
    r = o.sp2(h.H, 32, refine=False)
    coef = o.sp2_branch_coefficients(r.sigmas, r.n_layers)
    S0 = o.input_layer(h.H, r.e_min, r.e_max)
    assert np.max(np.abs(o.network_forward(S0, coef) - r.S_last)) < 1e-12


def test_network_adjoint_against_central_differences():
    rng = np.random.default_rng(6)
    B, N, L = 2, 8, 5
    X0 = np.stack([(lambda A: (A + A.T) / 2)(rng.uniform(0, 1, (N, N)) / N) + 0.5 * np.eye(N) for _ in range(B)])
    coef = np.array([[1, 0, 0], [-1, 2, 0]] * 3)[:L].astype(np.float64) + rng.uniform(-0.05, 0.05, (L, 3))
    T = np.stack([np.eye(N) * 0.3] * B)

    def loss(c, x0):
        return o.network_loss(o.network_forward(x0, c), T)

    XL = o.network_forward(X0, coef)
    G_L = 2.0 * (XL - T) / B
    dcoef, G0 = o.network_adjoint(X0, coef, G_L)
    h = 1e-4
    for n in range(L):
        for k in range(3):
            cp, cm = coef.copy(), coef.copy()
            cp[n, k] += h
            cm[n, k] -= h
            fd = (loss(cp, X0) - loss(cm, X0)) / (2 * h)
            assert abs(fd - dcoef[n, k]) <= 1e-6 * max(1.0, abs(fd))
    for (b, i, j) in [(0, 0, 0), (1, 2, 5), (0, 7, 3)]:
        E = np.zeros_like(X0)
        E[b, i, j] += 1
        E[b, j, i] += 1
        fd = (loss(coef, X0 + h * E) - loss(coef, X0 - h * E)) / (2 * h)
        assert abs(fd - np.sum(G0 * E)) <= 1e-6 * max(1.0, abs(fd))
