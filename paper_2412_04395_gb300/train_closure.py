"""Training pipeline of the learned subgrid closure (runs every step in the CUDA library).

  1. fine run of this solver (mixed precision) from seeded initial noise, spun up;
  2. snapshots Favre-filtered r x r x r into coarse C-grid states + SGS targets (erf_filter_state);
  3. features of each coarse state (erf_closure_features on a coarse handle);
  4. standardisation statistics and mini-batch Adam on the GPU (erf_column_stats,
     erf_standardise, erf_train_closure);
  5. a closure blob (erf_set_closure_weights format) and an a-priori comparison on held-out
     snapshots: learned closure vs Smagorinsky vs no model;
  6. an a-posteriori comparison: coarse runs (learned, Smagorinsky, no model) started from the
     filtered fine state and compared, at several horizons, with the filtered fine run.

    python -m paper_2412_04395_gb300.train_closure --out closure.bin [--grid 256 256 128] ...
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W


def coarse_workload(fine: W.Workload, r: int) -> W.Workload:
    """The r-times coarser grid of the same case (same physics, sounding and spacing ratio)."""
    zeta = fine.zeta[::r]
    return fine.with_(name=fine.name + f"_coarse{r}", nx=fine.nx // r, ny=fine.ny // r, nz=fine.nz // r,
                      dx=fine.dx * r, dy=fine.dy * r, zeta=zeta, dtheta=None, u=None, v=None, w=None,
                      closure=W.CLOSURE_LEARNED)


def init_params(seed: int):
    """He-style random initial parameters (FP32 vector of 9737), drawn on the host as inputs."""
    rng = np.random.default_rng(seed)
    layers = (12, 64, 64, 64, 9)
    out = []
    for a, b in zip(layers[:-1], layers[1:]):
        out.append((rng.normal(size=(b, a)) * np.sqrt(2.0 / a)).ravel())
        out.append(np.zeros(b))
    return np.concatenate(out).astype(np.float32)


def smagorinsky_prediction(F, rho_unused, delta, Cs=0.17, Pr_t=1.0 / 3.0, g=9.81, theta0=None):
    """Kinematic Smagorinsky stresses/fluxes from coarse features (for the a-priori comparison)."""
    s11, s22, s33 = F[:, 0], F[:, 4], F[:, 8]
    s12, s13, s23 = 0.5 * (F[:, 1] + F[:, 3]), 0.5 * (F[:, 2] + F[:, 6]), 0.5 * (F[:, 5] + F[:, 7])
    SS = s11 ** 2 + s22 ** 2 + s33 ** 2 + 2 * (s12 ** 2 + s13 ** 2 + s23 ** 2)
    nu = (Cs * delta) ** 2 * np.sqrt(2 * SS)
    tr = (s11 + s22 + s33) / 3
    dthdz = F[:, 11] * theta0 / g
    out = np.stack([-2 * nu * (s11 - tr), -2 * nu * (s22 - tr), -2 * nu * (s33 - tr), -2 * nu * s12,
                    -2 * nu * s13, -2 * nu * s23, -nu / Pr_t * F[:, 9], -nu / Pr_t * F[:, 10],
                    -nu / Pr_t * dthdz], axis=1)
    return out


def collect(fine: W.Workload, r: int, spinup: int, n_snap: int, every: int, log=print, keep_fine=False):
    """Fine run + filtered snapshots.  Returns (features per snapshot [Nc,12], targets per
    snapshot [Nc,9], coarse states per snapshot, coarse workload[, the fine Dycore])."""
    import torch
    from .erf import Dycore
    d = Dycore(fine.with_(precision=W.PREC_MIXED32))
    d.erf_set_initial(fine.dtheta, fine.u, fine.v, fine.w)
    t0 = time.time()
    d.erf_rk3_step(spinup)
    torch.cuda.synchronize()
    log(f"spin-up {spinup} steps of {fine.nx}x{fine.ny}x{fine.nz}: {time.time() - t0:.1f} s")
    cw = coarse_workload(fine, r)
    c = Dycore(cw)
    Xs, Ts, states = [], [], []
    for s in range(n_snap):
        d.erf_rk3_step(every)
        f, T = d.erf_filter_state(r)
        for k in ("rho", "rhotheta", "rhou", "rhov", "rhow"):
            c.erf_set_state(k, f[k].contiguous())
        Xs.append(c.erf_closure_features())
        Ts.append(T)
        states.append(f)
    torch.cuda.synchronize()
    if keep_fine:
        return Xs, Ts, states, cw, d
    d.close()
    return Xs, Ts, states, cw


def train(Xs, Ts, train_idx, epochs, batch, lr, seed, log=print):
    """Statistics over the training snapshots, standardisation and Adam on the GPU."""
    import torch
    from . import erf
    X = torch.cat([Xs[i] for i in train_idx])
    T = torch.cat([Ts[i] for i in train_idx])
    # one seeded shuffle (the trainer visits samples in the given order)
    perm = torch.as_tensor(np.random.default_rng(seed).permutation(X.shape[0]), device=X.device)
    X, T = X[perm].contiguous(), T[perm].contiguous()
    xm, xs = erf.erf_column_stats(X)
    tm, ts = erf.erf_column_stats(T)
    Xz = erf.erf_standardise(X, xm, xs)
    Tz = erf.erf_standardise(T, tm, ts)
    params = torch.as_tensor(init_params(seed), device=X.device)
    t0 = time.time()
    losses = erf.erf_train_closure(Xz, Tz, params, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    log(f"training: {X.shape[0]} samples x {epochs} epochs in {time.time() - t0:.1f} s, "
        f"loss {losses[0].item():.4f} -> {losses[-1].item():.4f}")
    return params, (xm, xs, tm, ts), losses


def blob_from(params, stats) -> bytes:
    xm, xs, tm, ts = (t.detach().cpu().numpy().astype(np.float32) for t in stats)
    body = np.concatenate([xm, xs, tm, ts, params.detach().cpu().numpy().astype(np.float32)])
    return np.array([0x4D465245, 1], dtype=np.uint32).tobytes() + body.astype(np.float32).tobytes()


def apriori(blob, Xs, Ts, states, cw, test_idx, stats):
    """Held-out snapshots: mean squared error on standardised targets (all 9 outputs) of the
    learned closure (tensor-core inference on the coarse state), of Smagorinsky (Cs = 0.17, from
    the same coarse gradients) and of no model (zero SGS terms)."""
    from .erf import Dycore
    xm, xs, tm, ts = (t.detach().cpu().numpy().astype(np.float64) for t in stats)
    c = Dycore(cw)
    c.erf_set_closure_weights(blob)
    dz = float(np.diff(cw.zeta)[0])
    delta = (cw.dx * cw.dy * dz) ** (1.0 / 3.0)
    res = {"learned": [], "smagorinsky": [], "none": [], "fallback_cells": []}
    z = lambda A: (A - tm) / ts
    for X, T, f in ((Xs[i], Ts[i], states[i]) for i in test_idx):
        for k in ("rho", "rhotheta", "rhou", "rhov", "rhow"):
            c.erf_set_state(k, f[k].contiguous())
        tau, nfb = c.erf_closure_fields()
        rho = f["rho"].cpu().numpy().reshape(-1)
        learned = (tau.cpu().numpy().reshape(9, -1) / rho).T
        F = X.cpu().numpy().astype(np.float64)
        Tt = T.cpu().numpy().astype(np.float64)
        sm = smagorinsky_prediction(F, None, delta, theta0=float(np.mean(cw.knots[1][:1])) if cw.knots else 300.0)
        res["learned"].append(float(np.mean((z(learned) - z(Tt)) ** 2)))
        res["smagorinsky"].append(float(np.mean((z(sm) - z(Tt)) ** 2)))
        res["none"].append(float(np.mean((z(np.zeros_like(Tt)) - z(Tt)) ** 2)))
        res["fallback_cells"].append(int(nfb))
    return {k: (float(np.mean(v)) if k != "fallback_cells" else int(np.sum(v))) for k, v in res.items()}


def primitives(st):
    """theta at cells and u, v, w at their faces of a flat periodic C-grid state (numpy dict)."""
    rho = st["rho"]
    th = st["rhotheta"] / rho
    u = st["rhou"] / (0.5 * (np.roll(rho, 1, axis=2) + rho))
    v = st["rhov"] / (0.5 * (np.roll(rho, 1, axis=1) + rho))
    rz = np.concatenate([rho[:1], 0.5 * (rho[:-1] + rho[1:]), rho[-1:]])
    w = st["rhow"] / rz
    return th, u, v, w


def field_errors(coarse, ref, th_mean0, u_g, v_g):
    """Relative L2 errors of a coarse state against the filtered fine state (reading of the
    2% criterion): theta - <theta>_0(z) (planar mean of the filtered field at the start) and the
    velocity departure from the geostrophic wind, pointwise; the same on the raw fields; and the
    planar-mean theta profile against its change since the start."""
    tc, uc, vc, wc = primitives(coarse)
    tf, uf, vf, wf = primitives(ref)
    m = th_mean0[:, None, None]
    dv = np.sqrt(np.sum((uc - uf) ** 2) + np.sum((vc - vf) ** 2) + np.sum((wc - wf) ** 2))
    pc, pf = tc.mean(axis=(1, 2)), tf.mean(axis=(1, 2))
    return {
        "theta_dev": float(np.linalg.norm(tc - tf) / np.linalg.norm(tf - m)),
        "vel_dev": float(dv / np.sqrt(np.sum((uf - u_g) ** 2) + np.sum((vf - v_g) ** 2) + np.sum(wf ** 2))),
        "theta_raw": float(np.linalg.norm(tc - tf) / np.linalg.norm(tf)),
        "vel_raw": float(dv / np.sqrt(np.sum(uf ** 2) + np.sum(vf ** 2) + np.sum(wf ** 2))),
        "theta_mean_profile": float(np.linalg.norm(pc - pf) / max(np.linalg.norm(pf - th_mean0), 1e-300)),
    }


def aposteriori(fine_d, fine: W.Workload, cw: W.Workload, blob: bytes, r: int, horizons, log=print):
    """Coarse runs from the filtered fine state at t0 with the learned closure, Smagorinsky and no
    model (coarse dt = r x fine dt, so one coarse step spans r fine steps), compared with the
    filtered fine run after each horizon (in fine steps, multiples of r)."""
    from .erf import Dycore
    f0, _ = fine_d.erf_filter_state(r)
    s0 = {k: v.cpu().numpy() for k, v in f0.items()}
    th_mean0 = (s0["rhotheta"] / s0["rho"]).mean(axis=(1, 2))
    runs = {}
    for name, clo in (("learned", W.CLOSURE_LEARNED), ("smagorinsky", W.CLOSURE_SMAGORINSKY),
                      ("none", W.CLOSURE_NONE)):
        c = Dycore(cw.with_(closure=clo, dt=fine.dt * r, precision=W.PREC_MIXED32))
        for k in ("rho", "rhotheta", "rhou", "rhov", "rhow"):
            c.erf_set_state(k, f0[k].contiguous())
        if clo == W.CLOSURE_LEARNED:
            c.erf_set_closure_weights(blob)
        runs[name] = c
    out = []
    done = 0
    for h in horizons:
        assert h % r == 0 and h > done
        fine_d.erf_rk3_step(h - done)
        for c in runs.values():
            c.erf_rk3_step((h - done) // r)
        done = h
        fh, _ = fine_d.erf_filter_state(r)
        ref = {k: v.cpu().numpy() for k, v in fh.items()}
        row = {"seconds": h * fine.dt}
        for name, c in runs.items():
            row[name] = field_errors(c.state(), ref, th_mean0, cw.u_g, cw.v_g)
        out.append(row)
        log(f"a-posteriori after {h * fine.dt:.0f} s: " + ", ".join(
            f"{n}: theta_dev {row[n]['theta_dev']:.3f} vel_dev {row[n]['vel_dev']:.3f} "
            f"theta_raw {row[n]['theta_raw']:.2e} vel_raw {row[n]['vel_raw']:.3f}" for n in runs))
    for c in runs.values():
        c.close()
    return out


def run(grid=(256, 256, 128), dx=10.0, dt=0.1, spinup=6000, snapshots=10, every=300, test_every=5,
        epochs=20, batch=8192, lr=1e-3, seed=7, horizons=(), log=print, holdout_last=0):
    """Every test_every-th snapshot is held out (interleaved, so train and test see the same
    stage of the boundary layer's development), or, with holdout_last > 0, the last holdout_last
    snapshots (the test set then lies later in time than anything trained on).  With horizons
    (fine steps), the fine run goes on after the last snapshot for the a-posteriori comparison."""
    nx, ny, nz = grid
    r = 4
    fine = W.convective_abl(nx=nx, ny=ny, nz=nz, dx=dx).with_(dt=dt)
    res = collect(fine, r, spinup, snapshots, every, log, keep_fine=bool(horizons))
    Xs, Ts, states, cw = res[:4]
    if holdout_last > 0:
        assert holdout_last < snapshots
        test_idx = list(range(snapshots - holdout_last, snapshots))
    else:
        test_idx = [i for i in range(snapshots) if i % test_every == test_every - 1]
    train_idx = [i for i in range(snapshots) if i not in test_idx]
    params, stats, losses = train(Xs, Ts, train_idx, epochs, batch, lr, seed, log)
    blob = blob_from(params, stats)
    ap = apriori(blob, Xs, Ts, states, cw, test_idx, stats)
    log(f"a-priori MSE (standardised, held-out): {ap}")
    post = None
    if horizons:
        post = aposteriori(res[4], fine, cw, blob, r, horizons, log)
        res[4].close()
    return blob, ap, losses, cw, post


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="closure.bin")
    ap.add_argument("--grid", type=int, nargs=3, default=[256, 256, 128])
    ap.add_argument("--dx", type=float, default=10.0)
    ap.add_argument("--dt", type=float, default=0.1)
    ap.add_argument("--spinup", type=int, default=6000)
    ap.add_argument("--snapshots", type=int, default=10)
    ap.add_argument("--every", type=int, default=300)
    ap.add_argument("--test-every", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--horizons", type=int, nargs="*", default=[],
                    help="a-posteriori comparison after these numbers of fine steps (multiples of 4)")
    ap.add_argument("--holdout-last", type=int, default=0,
                    help="hold out the last N snapshots instead of every test-every-th")
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    blob, ap, losses, cw, post = run(tuple(args.grid), args.dx, args.dt, args.spinup, args.snapshots, args.every,
                                     args.test_every, args.epochs, args.batch, args.lr, args.seed,
                                     tuple(args.horizons), holdout_last=args.holdout_last)
    open(args.out, "wb").write(blob)
    print(f"wrote {args.out} ({len(blob)} bytes)")
    if args.report:
        json.dump({"apriori_mse": ap, "aposteriori": post, "loss_first": float(losses[0]),
                   "loss_last": float(losses[-1]), "args": vars(args)}, open(args.report, "w"), indent=1)


if __name__ == "__main__":
    main()
