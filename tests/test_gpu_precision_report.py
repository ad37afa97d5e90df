"""Measured error of each precision against the FP64 oracle (FP64, MD_MIXED, MD_FP32).

For every precision the same seeded inputs are run through the library and the oracle, and the
errors are measured and asserted against the bars of the parity tests: step-0 forces (relative
L2), the 100-step trajectory (largest minimum-image position error, relative L2 of velocities),
and the per-atom differences of E, U, K, the virial W and the pressure P at steps 0 and 100.
The values are written to precision_errors.json in the directory named by GBMD_REPORT_DIR (if
set), so that a run on the GPU leaves the table behind.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2003_14061_gb300 import inputs
from paper_2003_14061_gb300.system import WCA_RC, MDSystem

pytestmark = pytest.mark.gpu

CASES = {
    # name: (fcc cells, density, cutoff, skin, T, perturbation, seed)
    "wca2048": (8, 0.8, WCA_RC, 0.4, 1.0, 0.15, 1),
    "lj1372": (7, 0.8442, 2.5, 0.3, 0.72, 0.08, 3),
}
_REPORT = {}


def _min_image(d, box):
    return d - box * np.round(d / box)


def _props_diff(pr, op, n, V):
    U, K, W, P = op[0], op[1], op[2], op[3]
    return {"E_per_atom": abs(pr["E_per_atom"] - (U + K) / n), "U_per_atom": abs(pr["U"] - U) / n,
            "K_per_atom": abs(pr["K"] - K) / n, "W_per_atom": abs(pr["virial"] - W) / n,
            "P": abs(pr["pressure"] - P), "P_rel": abs(pr["pressure"] - P) / max(abs(P), 1e-300)}


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_precision_errors(name, prec):
    ncell, rho, rc, skin, T, amp, seed = CASES[name]
    x, box = inputs.fcc_lattice(ncell, rho)
    x = inputs.perturb(x, box, amp, seed)
    n = x.shape[0]
    v = inputs.maxwell(n, T, seed=5)
    V = float(np.prod(box))
    p = oracle.pot(rc=rc)
    s = MDSystem(x, v, box, rc=rc, skin=skin, precision=prec)
    _, _, f = s.state(x=False, v=False, f=True)
    of, _, _, _ = oracle.forces(x, box, p)
    pr0 = s.props()[0]
    op0 = oracle.props(x, v, box, p)
    s.integrate(100)
    xg, vg, _ = s.state()
    pr1 = s.props()[0]
    s.close()
    xo, vo, po, _ = oracle.run(x, v, box, p, dt=0.005, nsteps=100)
    rec = {
        "atoms": n,
        "force_rel_l2_step0": float(np.linalg.norm(f - of) / np.linalg.norm(of)),
        "max_abs_dx_step100": float(np.abs(_min_image(xg - xo, box)).max()),
        "v_rel_l2_step100": float(np.linalg.norm(vg - vo) / np.linalg.norm(vo)),
        "step0": _props_diff(pr0, op0, n, V),
        "step100": _props_diff(pr1, po[-1], n, V),
    }
    _REPORT.setdefault(name, {})[prec] = rec
    out = os.environ.get("GBMD_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_errors.json"), "w") as fh:
            json.dump(_REPORT, fh, indent=1, sort_keys=True)
    # the parity bars
    assert rec["force_rel_l2_step0"] <= (1e-12 if prec == "fp64" else 1e-5)
    assert rec["max_abs_dx_step100"] <= 1e-4 and rec["v_rel_l2_step100"] <= 1e-4
    assert rec["step0"]["E_per_atom"] <= 1e-6 and rec["step100"]["E_per_atom"] <= 1e-6
    if prec == "fp64":
        # FP64 everywhere: differences are summation-order rounding only
        assert rec["force_rel_l2_step0"] <= 1e-13 and rec["max_abs_dx_step100"] <= 1e-9
