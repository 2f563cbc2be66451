"""Writes fermi_fit_beta40_L11.json: the finite-temperature expansion
coefficients fitted by the FP64 oracle (Sec. "Optimized SP2 Finite Temperature
Fermi-Operator Expansion", Fig. 6 set-up: beta = 40, 11 layers).  Calls only
``oracle``.  Run from the repository root:  python tests/golden/make_fermi_fit.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

theta, c, err = oracle.fit_fermi_expansion(beta=40.0, layers=11, n_grid=2001)
out = {
    "cite": "Sec. 'Optimized SP2 Finite Temperature Fermi-Operator Expansion', Eq. 19 and Fig. 6: "
            "beta = 40, 11 layers; fitted by oracle.fit_fermi_expansion (readings C22, C23)",
    "beta": 40.0,
    "layers": 11,
    "grid_points": 2001,
    "max_abs_error_on_grid": err,
    "theta": [[float(v) for v in row] for row in theta],
    "c": [float(v) for v in c],
}
with open(os.path.join(HERE, "fermi_fit_beta40_L11.json"), "w") as f:
    json.dump(out, f, indent=1)
print("max error on the fit grid", err)
