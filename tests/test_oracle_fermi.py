"""Pins of the finite-temperature expansion oracle (Sec. "Optimized SP2 Finite
Temperature Fermi-Operator Expansion", Eq. 19, Fig. 6; readings C22, C23)."""
import json
import os

import numpy as np

import oracle as o
import sp2_inputs as si

HERE = os.path.dirname(__file__)


def _fit():
    with open(os.path.join(HERE, "golden", "fermi_fit_beta40_L11.json")) as f:
        return json.load(f)


def _paper():
    with open(os.path.join(HERE, "golden", "paper_values.json")) as f:
        return json.load(f)


def test_identity_layers_give_one_minus_eps():
    L = 4
    theta = np.tile([0.0, 1.0, 0.0], (L, 1))
    c = np.zeros(L + 1)
    c[0] = 1.0
    e = np.linspace(0, 1, 11)
    assert np.array_equal(o.fermi_expansion_scalar(theta, c, e), 1.0 - e)
    # readout spread over the layers: the same, since every eps_i = eps
    c = np.full(L + 1, 1.0 / (L + 1))
    assert np.allclose(o.fermi_expansion_scalar(theta, c, e), 1.0 - e, atol=1e-15)


def test_sp2_branch_layers_reproduce_the_scalar_map():
    """x^2 / 2x - x^2 layers with the readout on the last layer: F~ = 1 - p(eps)
    for the composed SP2 polynomial, evaluated independently."""
    sig = [1, -1, -1, 1, -1]
    theta = np.array([[1.0, 0.0, 0.0] if s > 0 else [-1.0, 2.0, 0.0] for s in sig])
    c = np.zeros(len(sig) + 1)
    c[-1] = 1.0
    e = np.linspace(0, 1, 101)
    x = e.copy()
    for s in sig:
        x = x * x if s > 0 else x * (2.0 - x)
    assert np.allclose(o.fermi_expansion_scalar(theta, c, e), 1.0 - x, atol=1e-15)


def test_matrix_form_is_the_scalar_map_on_the_spectrum():
    h = si.gapped_hamiltonian(120, 60, (-1.0, -0.05), (0.05, 1.0), seed=11)
    d = _fit()
    theta, c = np.array(d["theta"]), np.array(d["c"])
    lo, hi = o.gershgorin_bounds(h.H)
    D = o.fermi_expansion_matrix(h.H, theta, c, (lo, hi))
    eps = (h.eps - lo) / (hi - lo)
    want = (h.Q * o.fermi_expansion_scalar(theta, c, eps)) @ h.Q.T
    assert np.max(np.abs(D - want)) <= 1e-12
    # and close to the Fermi-Dirac matrix with beta = 40 on the scaled axis
    fd = (h.Q * o.fermi_dirac_scaled(eps, 40.0)) @ h.Q.T
    assert np.max(np.abs(D - fd)) <= 2e-4


def test_fit_matches_fermi_dirac_with_eleven_layers():
    """Fig. 6: the Fermi function with beta = 40 learned with 11 layers.  The
    stored fit (written by tests/golden/make_fermi_fit.py from the oracle)
    stays within 1e-4 of F on a grid 50x finer than the fit grid."""
    p = _paper()["fig6_fermi"]
    d = _fit()
    assert d["beta"] == p["beta"] and d["layers"] == p["layers"]
    theta, c = np.array(d["theta"]), np.array(d["c"])
    fine = np.linspace(0.0, 1.0, 100001)
    err = np.max(np.abs(o.fermi_expansion_scalar(theta, c, fine) - o.fermi_dirac_scaled(fine, p["beta"])))
    print(f"max |F~ - F| on [0, 1]: {err:.2e}")
    assert err <= 1e-4
    # intermediate layer values stay bounded (|x| < 16 keeps the FP16 split exact)
    e = fine
    for a, b, cc in theta:
        e = a * e * e + b * e + cc
        assert np.max(np.abs(e)) < 4.0


# --- pins of the target function itself, F(eps) = 1/(exp(beta (eps - 1/2)) + 1)
# (Eq. 19).  Each one is a property of the logistic step that a dropped beta,
# a flipped sign of (eps - 1/2) or a wrong centre fails.

def test_fermi_scaled_is_one_half_at_the_centre():
    for beta in (1.0, 40.0, 880.0):
        assert o.fermi_dirac_scaled(0.5, beta) == 0.5


def test_fermi_scaled_value_where_the_exponential_is_three():
    # at eps = 1/2 + ln(3)/beta the exponential equals 3, so F = 1/4; the
    # mirrored point gets 3/4 (a sign error swaps them, a missing beta gives ~0.49)
    beta = 40.0
    x = 0.5 + np.log(3.0) / beta
    assert abs(o.fermi_dirac_scaled(x, beta) - 0.25) <= 1e-15
    assert abs(o.fermi_dirac_scaled(1.0 - x, beta) - 0.75) <= 1e-15


def test_fermi_scaled_particle_hole_symmetry_and_monotone():
    e = np.linspace(0.0, 1.0, 1001)
    f = o.fermi_dirac_scaled(e, 40.0)
    assert np.max(np.abs(f + o.fermi_dirac_scaled(1.0 - e, 40.0) - 1.0)) <= 1e-15
    assert np.all(np.diff(f) < 0.0)             # occupied below the centre, empty above
    assert f[0] > 1.0 - 1e-8 and f[-1] < 1e-8  # e^(-20) ~ 2e-9 from the integers


def test_fermi_scaled_slope_at_the_centre():
    # dF/deps at 1/2 is -beta/4 (derivative of the logistic at its midpoint)
    beta, h = 40.0, 1e-6
    d = (o.fermi_dirac_scaled(0.5 + h, beta) - o.fermi_dirac_scaled(0.5 - h, beta)) / (2 * h)
    assert abs(d + beta / 4.0) <= 1e-6 * beta


def test_fermi_scaled_is_fermi_dirac_on_the_mapped_axis():
    """Q diag(F((E - e_lo)/(e_hi - e_lo))) Q^T equals the Fermi-Dirac matrix
    (Eqs. 1, 5) with kT = (e_hi - e_lo)/beta and mu = (e_lo + e_hi)/2."""
    h = si.gapped_hamiltonian(48, 24, (-1.0, -0.1), (0.1, 1.0), seed=5)
    e_lo, e_hi, beta = -1.3, 1.1, 40.0
    scaled = (h.eps - e_lo) / (e_hi - e_lo)
    D1 = (h.Q * o.fermi_dirac_scaled(scaled, beta)) @ h.Q.T
    D2 = o.fermi_dirac_closed_form(h.Q, h.eps, 0.5 * (e_lo + e_hi), (e_hi - e_lo) / beta)
    assert np.max(np.abs(D1 - D2)) <= 1e-13
