#!/usr/bin/env python3
"""Writes the stored expected values of the full-size hill-bubble run: the FP64 oracle's state
after the configured 500 RK3 steps of the 3D warm bubble over a Gaussian hill (256 x 256 x 128,
dx = dy = 50 m, stretched dz from 20 m, WENO5 scalars, upwind-5 momenta, dt 0.25 s, 6 acoustic
substeps), sampled at SAMPLES elements per prognostic field.

Only the oracle (oracle/) and the seeded input generator (workloads.py, which holds none of the
method's arithmetic) are called.  The sampled indices are not stored: element m of a field of n
values is index (m * STRIDE) mod n, with STRIDE a prime that divides no field size, so the
SAMPLES indices are distinct and spread over the whole field.  Run (about an hour on 8 cores):

    python tests/golden/make_hill_bubble_500.py [--threads N]

With --ulp-floor it instead measures the run's round-off floor: the oracle from the same initial
state with rho theta perturbed by a seeded random relative 1.1e-16 (about one ulp), 500 steps, and
the relative L2 of its difference from the stored values on the same samples, written (five
numbers, one per field) to hill_bubble_256x256x128_500steps_ulp.json.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "hill_bubble_256x256x128_500steps.npz")
SAMPLES = 1_000_000
STRIDE = 2_654_435_761          # prime; coprime with every field size of this grid
STEPS = 500
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def sample_indices(n, samples=SAMPLES, stride=STRIDE):
    """The stored elements of a field of n values: (m * stride) mod n, m = 0 .. samples-1."""
    m = np.arange(samples, dtype=np.uint64)
    return ((m * np.uint64(stride)) % np.uint64(n)).astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--ulp-floor", action="store_true")
    args = ap.parse_args()
    import oracle
    from oracle import Oracle, OracleConfig
    from paper_2412_04395_gb300 import workloads as W
    wl = W.hill_bubble()
    oracle.build_oracle()
    used = oracle.set_threads(args.threads)
    cfg = OracleConfig(nx=wl.nx, ny=wl.ny, nz=wl.nz, dx=wl.dx, dy=wl.dy, terrain_beta=wl.terrain_beta,
                       dt=wl.dt, n_substeps=wl.n_substeps, beta_s=wl.beta_s, beta_d=wl.beta_d,
                       mom_adv=wl.mom_adv, scal_adv=wl.scal_adv, closure=wl.closure, Cs=wl.Cs,
                       Pr_t=wl.Pr_t, nu=wl.nu, gravity=wl.gravity, theta_s=wl.theta_s,
                       brunt_N=wl.brunt_N, p_s=wl.p_s)
    o = Oracle(cfg, wl.zeta, wl.terrain, wl.knots)
    o.set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if args.ulp_floor:
        r = o.get("rhotheta")
        o.set("rhotheta", r * (1 + 1.1e-16 * np.random.default_rng(1).standard_normal(r.shape)))
    mass0 = o.mass()
    t0 = time.time()
    for s in range(STEPS):
        o.step(1)
        if (s + 1) % 25 == 0:
            print(f"step {s + 1}/{STEPS}  {time.time() - t0:.0f} s", flush=True)
    if args.ulp_floor:
        import json
        g = np.load(args.out)
        floor = {}
        for f in FIELDS:
            a = o.get(f).ravel()[sample_indices(o.get(f).size)]
            floor[f] = float(np.linalg.norm(a - g[f]) / np.linalg.norm(g[f]))
        path = os.path.join(HERE, "hill_bubble_256x256x128_500steps_ulp.json")
        json.dump({"steps": STEPS, "perturbation": "rho theta x (1 + 1.1e-16 N(0,1)), seed 1",
                   "rel_l2_on_samples": floor}, open(path, "w"), indent=1)
        print(f"wrote {path}: {floor}")
        return
    out = {"steps": np.int64(STEPS), "samples": np.int64(SAMPLES), "stride": np.int64(STRIDE),
           "mass0": np.float64(mass0), "mass": np.float64(o.mass()), "threads": np.int64(used)}
    for f in FIELDS:
        a = o.get(f).ravel()
        idx = sample_indices(a.size)
        assert np.unique(idx).size == SAMPLES
        out[f] = a[idx]
        out[f + "_l2"] = np.float64(np.linalg.norm(a))
    tmp = args.out + ".tmp.npz"
    np.savez_compressed(tmp, **out)
    os.replace(tmp, args.out)
    print(f"wrote {args.out} ({os.path.getsize(args.out) / 1e6:.1f} MB) in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
