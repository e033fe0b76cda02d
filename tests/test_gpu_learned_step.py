"""The learned-closure step end to end (features, BF16 tensor-core network, Smagorinsky fallback,
backscatter limit, edge/face interpolation and the stress divergence inside each RK3 stage) on the
mixed-precision GPU path against the FP64 oracle step with the same closure (closure 3 of
oracle/erf_oracle.c, the model of oracle/mlp_oracle.py with BF16 operands).

Two measures: the states themselves (mixed-precision bounds as for the other mixed cases), and the
closure's own effect, learned minus no closure on each side, which isolates the SGS terms from the
rest of the step: its relative L2 gap is the network's BF16 inference error (2e-5 .. 2e-4 of the
outputs) plus FP32 rounding of a small increment."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle
from test_gpu_closure import _params, _turbulent_like

pytestmark = pytest.mark.gpu
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def _gpu(wl, blob=None):
    from paper_2412_04395_gb300.erf import Dycore
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if blob is not None:
        d.erf_set_closure_weights(blob)
    return d


def _learned_oracle(wl, blob):
    o = make_oracle(wl.with_(closure=W.CLOSURE_LEARNED))
    th0 = o.get("base_theta")[:, 0, 0]
    m = M.LearnedClosure(blob, wl.zeta, wl.dx, wl.dy, th0, wl.Cs, wl.Pr_t, wl.gravity)
    o.set_sgs_model(m)
    return o, m


@pytest.mark.parametrize("case", ["network", "fallback"])
def test_learned_step_against_the_oracle_step(case):
    """network: inputs standardised with three times the state's own spread, so every cell stays
    inside |z| <= 6 and takes the network (no decision near the threshold); fallback: a spread so
    small that every cell leaves it and takes the cell-centre Smagorinsky-Lilly fallback."""
    steps = 5
    wl = _turbulent_like().with_(precision=W.PREC_MIXED32)
    o0 = make_oracle(wl)
    st = o0.state()
    th0 = o0.get("base_theta")[:, 0, 0]
    fo = M.features(st["rho"], st["rhotheta"], st["rhou"], st["rhov"], st["rhow"], wl.zeta, wl.dx, wl.dy, th0)
    mu, sd = M.standardise_stats(fo.reshape(-1, 12))
    in_sd, scale = (3.0 * sd, 10.0) if case == "network" else (np.full(12, 1e-9), 1.0)
    blob = M.pack_blob(_params(31), mu, in_sd, scale * np.linspace(-0.01, 0.01, 9), scale * np.linspace(0.02, 0.06, 9))
    with np.errstate(over="ignore", invalid="ignore"):   # the fallback case's unused network outputs
        oL, m = _learned_oracle(wl, blob)
        oL.step(steps)
    oN = make_oracle(wl.with_(closure=W.CLOSURE_NONE))
    oN.step(steps)
    gL = _gpu(wl.with_(closure=W.CLOSURE_LEARNED), blob)
    gN = _gpu(wl.with_(closure=W.CLOSURE_NONE))
    gL.erf_rk3_step(steps)
    gN.erf_rk3_step(steps)
    # every fallback decision far from the threshold, so FP32 and FP64 inputs take it alike
    assert m.margin > 1.0, m.margin
    ncell = wl.nx * wl.ny * wl.nz
    assert m.fallbacks == ([0] if case == "network" else [ncell]) * (3 * steps), m.fallbacks
    sL, sN, rL, rN = gL.state(), gN.state(), oL.state(), oN.state()
    mom = np.sqrt(sum(np.linalg.norm(rL[f]) ** 2 for f in ("rhou", "rhov", "rhow")))
    state, effect = {}, {}
    for f in FIELDS:
        den = np.linalg.norm(rL[f]) if f in ("rho", "rhotheta") else mom
        state[f] = float(np.linalg.norm(sL[f] - rL[f]) / den)
        dO = rL[f] - rN[f]
        effect[f] = float(np.linalg.norm((sL[f] - sN[f]) - dO) / np.linalg.norm(dO))
    print(case, "learned step vs oracle, state:", state)
    print(case, "closure effect (learned - none) vs oracle:", effect,
          "effect / momentum norm:", {f: float(np.linalg.norm(rL[f] - rN[f]) / mom) for f in FIELDS[2:]})
    assert state["rho"] < 1e-8 and state["rhotheta"] < 1e-8
    for f in ("rhou", "rhov", "rhow"):
        assert state[f] < 1e-6, f
    for f in ("rhotheta", "rhou", "rhov", "rhow"):
        assert effect[f] < 1e-2, f
