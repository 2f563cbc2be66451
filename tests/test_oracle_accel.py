"""Pins of the accelerated Deep-NN SP2 oracle (Sec. "Accelerated Deep-NN
SP2", readings C19-C21), checked against the generator's exact spectrum,
the definition of the projector and the paper's layer-count example."""
import json
import os

import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

HERE = os.path.dirname(__file__)


def _paper():
    with open(os.path.join(HERE, "golden", "paper_values.json")) as f:
        return json.load(f)


def _homo_lumo(h):
    return float(h.eps[: h.n_occ].max()), float(h.eps[h.n_occ:].min())


@pytest.mark.parametrize("N,occ,virt", [(128, (-1.0, -0.1), (0.1, 1.0)), (200, (-1.0, -0.02), (0.02, 1.0))])
def test_closed_form_projector(N, occ, virt):
    h = si.gapped_hamiltonian(N, N // 2, occ, virt, seed=3)
    homo, lumo = _homo_lumo(h)
    r = o.sp2_accelerated(h.H, h.n_occ, homo, lumo, tol=1e-13)
    P = o.density_matrix_closed_form(h.Q, h.n_occ)
    assert np.max(np.abs(r.D - P)) <= 1e-11
    # and fewer layers than the plain scheme with the same spectral bounds
    plain = o.sp2(h.H, h.n_occ)
    print(f"N={N}: accelerated {r.n_layers} layers, plain {plain.n_layers}")
    assert r.n_layers < plain.n_layers


def test_conservative_estimates_are_safe():
    """A narrower gap than the true one (C21) still gives the projector."""
    h = si.gapped_hamiltonian(160, 50, (-1.0, -0.1), (0.1, 1.0), seed=4)
    homo, lumo = _homo_lumo(h)
    r = o.sp2_accelerated(h.H, h.n_occ, homo + 0.05, lumo - 0.05, tol=1e-13)
    assert np.max(np.abs(r.D - o.density_matrix_closed_form(h.Q, h.n_occ))) <= 1e-11


def test_too_wide_estimates_swap_eigenvalues():
    """An estimated gap reaching into the occupied band folds occupied
    eigenvalues onto unoccupied ones: the result is not the projector."""
    h = si.gapped_hamiltonian(120, 60, (-1.0, -0.1), (0.1, 1.0), seed=5)
    occ = np.sort(h.eps[: h.n_occ])
    r = o.sp2_accelerated(h.H, h.n_occ, occ[-10], 0.9, tol=1e-13)
    assert abs(np.trace(r.D) - h.n_occ) > 0.5


def test_bounds_enclose_true_eigenvalue_images():
    """The bounds the scheme carries enclose the images of the true scaled
    eigenvalues under the layer polynomials at every layer."""
    h = si.gapped_hamiltonian(96, 40, (-1.0, -0.05), (0.05, 1.0), seed=6)
    homo, lumo = _homo_lumo(h)
    r = o.sp2_accelerated(h.H, h.n_occ, homo, lumo, tol=1e-13)
    x = (r.e_max - h.eps) / (r.e_max - r.e_min)   # spectrum of S_0 (occupied first)
    occ, virt = x[: h.n_occ], x[h.n_occ:]
    for (a, b, c), (l, hh) in zip(r.coefficients, r.bounds[1:]):
        occ = a * occ * occ + b * occ + c
        virt = a * virt * virt + b * virt + c
        assert virt.max() <= l * (1 + 1e-12) + 1e-15
        assert occ.min() >= hh * (1 - 1e-12) - 1e-15
        assert virt.min() >= -1e-15 and occ.max() <= 1 + 1e-12


@pytest.mark.parametrize("l,h", [(0.49, 0.51), (0.3, 0.9), (0.05, 0.2), (0.8, 0.95), (0.0, 0.5), (0.5, 1.0)])
def test_layer_polynomials(l, h):
    a, b, c, s, l2, h2 = o.accelerated_layer(l, h)
    p = lambda x: a * x * x + b * x + c  # noqa: E731
    if s > 0:
        assert s == 1 and 1.0 - h <= l
        assert abs(p(1.0) - 1.0) <= 1e-15                    # 1 stays fixed
        assert abs(p(0.5 * l)) <= 1e-15                      # minimum at the fold centre
        assert abs(p(0.0) - p(l)) <= 1e-15 and abs(p(l) - l2) <= 1e-15
    else:
        assert abs(p(0.0)) <= 1e-15                          # 0 stays fixed
        assert abs(p(1.0 - 0.5 * (1.0 - h)) - 1.0) <= 1e-15  # maximum at the mirrored fold centre
        assert abs(p(1.0) - p(h)) <= 1e-15 and abs(p(h) - h2) <= 1e-15
    # the occupied and unoccupied sets stay apart and inside [0, 1]
    xs_v = np.linspace(0.0, l, 201)
    xs_o = np.linspace(h, 1.0, 201)
    assert p(xs_v).max() <= l2 + 1e-15
    assert p(xs_o).min() >= h2 - 1e-15
    assert l2 < h2
    assert p(xs_v).min() >= -1e-15 and p(xs_o).max() <= 1.0 + 1e-15


def test_accelerated_layer_count_trend():
    """Sec. "Accelerated Deep-NN SP2": 17 layers instead of 28 for a 100 x
    100 test Hamiltonian with N_occ = 10.  The paper's matrix and its exact
    scheme are not given (C19); with the Fig. 2 recipe and exact bounds the
    ratio of the two counts lands in a band around 17/28."""
    p = _paper()["fig5_plain_layers"]
    ratios = []
    for seed in range(5):
        h = si.uniform_random_symmetric(p["N"], p["n_occ"], seed)
        w = np.linalg.eigvalsh(h.H)
        bounds = (w[0], w[-1])
        plain = o.sp2(h.H, p["n_occ"], bounds=bounds).n_layers
        acc = o.sp2_accelerated(h.H, p["n_occ"], w[p["n_occ"] - 1], w[p["n_occ"]], tol=1e-12, bounds=bounds)
        ratios.append(acc.n_layers / plain)
        # the iterate reaches the projector of the lowest N_occ states
        V = np.linalg.eigh(h.H)[1][:, : p["n_occ"]]
        assert np.max(np.abs(acc.D - V @ V.T)) <= 1e-9
    print("accelerated / plain layers:", [round(r, 2) for r in ratios], "paper:", p["accelerated_value"] / p["value"])
    assert 0.4 <= np.mean(ratios) <= 0.75


def test_rejects_gapless_estimates():
    h = si.gapped_hamiltonian(40, 20, seed=1)
    with pytest.raises(ValueError):
        o.sp2_accelerated(h.H, 20, 0.5, 0.4)
