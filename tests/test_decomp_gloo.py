"""x-y pencil decomposition with deep halos (paper_2412_04395_gb300/decomp.py), on CPU ranks.

Each rank advances the oracle on its pencil widened by the halo, and the halo is refreshed from
the neighbours once per RK3 step.  The interiors, assembled, must equal the undivided oracle run
bit for bit, and the domain mass summed over ranks in rank order must equal the undivided mass to
round-off.  The transport is exercised twice: a single-process router (every rank's engine in one
list) and real torch.distributed gloo ranks (world size 2 and 4).
"""
import os
import tempfile

import numpy as np
import pytest
import torch

from paper_2412_04395_gb300 import decomp as D
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def test_shard_grid_is_the_squarest_factorisation():
    assert [D.shard_grid(n) for n in (1, 2, 3, 4, 6, 8, 12, 16)] == \
        [(1, 1), (2, 1), (3, 1), (2, 2), (3, 2), (4, 2), (4, 3), (4, 4)]


class OracleEngine:
    """One rank's oracle on its window; pack/unpack copy column blocks of every field."""

    def __init__(self, o):
        self.o = o
        self.nz = o.cfg.nz

    def _levels(self, f):
        return self.nz + 1 if f == "rhow" else self.nz

    def empty(self, ni, nj):
        n = sum(self._levels(f) for f in FIELDS) * ni * nj
        return torch.empty(n, dtype=torch.float64)

    def pack(self, i0, ni, j0, nj):
        return torch.from_numpy(np.concatenate(
            [self.o.get(f)[:, j0:j0 + nj, i0:i0 + ni].ravel() for f in FIELDS]))

    def unpack(self, i0, ni, j0, nj, buf):
        b = np.asarray(buf, dtype=np.float64)
        off = 0
        for f in FIELDS:
            a = self.o.get(f)
            n = self._levels(f) * ni * nj
            a[:, j0:j0 + nj, i0:i0 + ni] = b[off:off + n].reshape(self._levels(f), nj, ni)
            off += n
            self.o.set(f, a)


def cases():
    hill = W.hill_bubble(nx=64, ny=64, nz=20, dx=50.0)
    abl = W.abl_window(W.neutral_abl, 1024, 1024, 100, 200, 64, 64, nz=16)
    return {"hill": hill, "abl": abl}


def halo_of(wl):
    return D.step_reach(wl.n_substeps, wl.terrain is not None)


def undivided(wl, steps):
    o = make_oracle(wl)
    for _ in range(steps):
        o.step(1)
    return o.state(), o.mass()


def interior_mass(o, p, wl):
    Hc = D.interior_view(p, o.geom("Hc"))
    return float(np.sum(D.interior_view(p, o.get("rho")) * Hc) * wl.dx * wl.dy)


def test_plan_pairs_every_send_with_a_receive():
    for px, py in ((2, 1), (1, 3), (2, 2), (3, 2), (4, 4)):
        dec = D.PencilDecomp(128, 96, px, py, 20)
        sends = {}
        for r in range(dec.size):
            s, rv = dec.messages(r)
            for ph, peer, tag, box in s:
                sends[(r, peer, tag)] = box
        for r in range(dec.size):
            p = dec.pencil(r)
            _, rv = dec.messages(r)
            for ph, peer, tag, box in rv:
                sb = sends[(peer, r, tag)]
                assert (sb[1], sb[3]) == (box[1], box[3])          # same strip shape
                i0, ni, j0, nj = box
                assert 0 <= i0 and i0 + ni <= p.nxw and 0 <= j0 and j0 + nj <= p.nyw
                # received strips land in the halo, sent strips come from the interior
                in_halo_x = i0 + ni <= p.hx or i0 >= p.hx + p.nxl
                in_halo_y = j0 + nj <= p.hy or j0 >= p.hy + p.nyl
                assert in_halo_x or in_halo_y
    with pytest.raises(ValueError):
        D.PencilDecomp(60, 16, 4, 1, 20)          # interior 15 < halo 20


def test_step_reach_is_within_the_measured_window_margin():
    # one step of the ABL cases reaches at most 24 columns (tests/test_oracle_windows.py)
    assert D.step_reach(10, False) >= 24
    assert D.step_reach(6, True) >= D.step_reach(6, False)


@pytest.mark.parametrize("name,px,py", [("hill", 2, 1), ("hill", 1, 3), ("abl", 2, 2)])
def test_local_router_matches_the_undivided_run(name, px, py):
    wl = cases()[name]
    if py == 3:
        wl = W.hill_bubble(nx=32, ny=96, nz=20, dx=50.0)
    steps = 3
    ref, mass_ref = undivided(wl, steps)
    dec = D.PencilDecomp(wl.nx, wl.ny, px, py, halo_of(wl))
    orcs = [make_oracle(D.window_workload(wl, dec, r)) for r in range(dec.size)]
    router = D.LocalRouter(dec, [OracleEngine(o) for o in orcs])
    for _ in range(steps):
        for o in orcs:
            o.step(1)
        router.exchange()
    shapes = {f: ref[f].shape for f in FIELDS}
    got = D.gather_interior(dec, lambda r: orcs[r].state(), shapes)
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), (name, f, np.abs(got[f] - ref[f]).max())
    mass = D.fixed_order_sum([interior_mass(orcs[r], dec.pencil(r), wl) for r in range(dec.size)])
    assert abs(mass - mass_ref) <= 1e-14 * abs(mass_ref)
    # after the exchange the halos hold the neighbours' interiors too: every window equals the
    # undivided state restricted to it
    for r in range(dec.size):
        st = orcs[r].state()
        for f in FIELDS:
            assert np.array_equal(st[f], dec.window_slices(r, ref[f])), (r, f)


def _gloo_rank(rank, world, px, py, name, steps, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    oracle.set_threads(1)
    wl = cases()[name]
    dec = D.PencilDecomp(wl.nx, wl.ny, px, py, halo_of(wl))
    o = make_oracle(D.window_workload(wl, dec, rank))
    eng = OracleEngine(o)
    for _ in range(steps):
        o.step(1)
        D.exchange(dec, rank, eng, dist)
    part = torch.tensor([interior_mass(o, dec.pencil(rank), wl)], dtype=torch.float64)
    parts = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, part)
    mass = D.fixed_order_sum([float(t.item()) for t in parts])
    np.savez(os.path.join(outdir, f"r{rank}.npz"), mass=mass, **o.state())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,px,py,name", [(2, 2, 1, "hill"), (4, 2, 2, "abl")])
def test_gloo_ranks_match_the_undivided_run(world, px, py, name):
    import torch.multiprocessing as mp
    steps = 2
    wl = cases()[name]
    ref, mass_ref = undivided(wl, steps)
    port = 29500 + (os.getpid() % 1000) + world
    with tempfile.TemporaryDirectory() as td:
        mp.start_processes(_gloo_rank, args=(world, px, py, name, steps, port, td), nprocs=world,
                           join=True, start_method="spawn")
        res = [dict(np.load(os.path.join(td, f"r{r}.npz"))) for r in range(world)]
    dec = D.PencilDecomp(wl.nx, wl.ny, px, py, halo_of(wl))
    got = D.gather_interior(dec, lambda r: res[r], {f: ref[f].shape for f in FIELDS})
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), (f, np.abs(got[f] - ref[f]).max())
    for r in range(world):
        assert float(res[r]["mass"]) == float(res[0]["mass"])      # every rank holds the same sum
        assert abs(float(res[r]["mass"]) - mass_ref) <= 1e-14 * abs(mass_ref)
