"""The warm bubble over the Gaussian hill at its configured size and length: 256 x 256 x 128 cells,
500 RK3 steps (125 s), FP64, the launch configuration the benchmark times.  The GPU's state is
compared with the oracle's 500-step state at 10^6 elements per field, stored in
tests/golden/hill_bubble_256x256x128_500steps.npz by tests/golden/make_hill_bubble_500.py (which
calls only the oracle and the seeded input generator).

Bar, per field on the sampled elements: relative L2 <= max(1e-11, 3 x the run's round-off floor),
the rule the short full-size runs use.  The floor is the oracle's own sensitivity: the same 500
steps from an initial rho theta perturbed by a random relative 1.1e-16 (about one ulp), stored by
the same script (--ulp-floor) in hill_bubble_256x256x128_500steps_ulp.json.  Also the whole-field
L2 norm of every field within 1e-11 of the oracle's, and the domain mass drift within 1e-12 of the
oracle's.  The measured gaps are printed against both 1e-11 and the floor.
"""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "hill_bubble_256x256x128_500steps.npz")
FLOOR = os.path.join(HERE, "golden", "hill_bubble_256x256x128_500steps_ulp.json")
TOL = 1e-11
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def test_hill_bubble_500_steps_full_size():
    if not (os.path.exists(GOLDEN) and os.path.exists(FLOOR)):
        pytest.fail("stored oracle values missing: run tests/golden/make_hill_bubble_500.py (and --ulp-floor)")
    import json
    floor = json.load(open(FLOOR))["rel_l2_on_samples"]
    import __graft_entry__ as ge
    ge.build()
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_hill_bubble_500 import sample_indices
    from paper_2412_04395_gb300 import workloads as W
    from paper_2412_04395_gb300.erf import Dycore
    g = np.load(GOLDEN)
    steps = int(g["steps"])
    wl = W.hill_bubble()
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    m0 = d.erf_diagnostics()["mass"]
    d.erf_rk3_step(steps)
    diag = d.erf_diagnostics()
    assert diag["status"] == 0, diag
    out = {}
    for f in FIELDS:
        a = d.erf_get_state(f).ravel()
        idx = sample_indices(a.size, int(g["samples"]), int(g["stride"]))
        ref = g[f]
        out[f] = float(np.linalg.norm(a[idx] - ref) / np.linalg.norm(ref))
        out[f + "_norm"] = abs(float(np.linalg.norm(a)) - float(g[f + "_l2"])) / float(g[f + "_l2"])
    print("hill bubble 256x256x128, 500 steps, GPU vs oracle:", {k: "%.1e" % v for k, v in out.items()},
          "oracle one-ulp floor:", {k: "%.1e" % v for k, v in floor.items()})
    bad = {f: (out[f], floor[f]) for f in FIELDS if not out[f] <= max(TOL, 3.0 * floor[f])}
    bad.update({k: v for k, v in out.items() if k.endswith("_norm") and not v <= TOL})
    assert not bad, (bad, out, floor)
    drift_gpu = (diag["mass"] - m0) / m0
    drift_orc = (float(g["mass"]) - float(g["mass0"])) / float(g["mass0"])
    assert abs(drift_gpu - drift_orc) <= 1e-12, (drift_gpu, drift_orc)
    assert abs(m0 - float(g["mass0"])) <= 1e-13 * abs(m0)
    d.close()
