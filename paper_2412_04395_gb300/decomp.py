"""x-y pencil decomposition of the dycore with deep halos (one exchange per RK3 step).

The paper distributes AMReX boxes over MPI ranks and refreshes their ghost cells with
FillBoundary (GPU-aware MPI, Sec. 5.1 and 5.2): every stage and every acoustic substep exchanges a
few cells.  The path shards naturally in x-y pencils with whole columns per rank (the vertical
tridiagonal never crosses ranks), and this module keeps that partition but exchanges differently:
each rank advances the unchanged periodic step on its pencil widened by a halo of H columns on
each sharded side, where H is at least the number of columns one RK3 step reaches sideways.  After
a step the interior columns are exactly those of the undivided run (the periodic wrap of the
widened window corrupts only columns within H of its edges); the halo is then refreshed from the
neighbours' interiors, once per step.  One exchange round per step replaces 3 stage rounds and
1 + ns/2 + ns substep rounds, the step stays one CUDA graph, and the price is the redundant update
of the halo columns (2H / interior width per sharded direction).

Reach of one step (columns, per direction): each stage's slow tendencies reach 4 (the 6-point
upwind/WENO stencils of a face flux, the divergence, and the face-averaged density of the
advected velocity); each acoustic substep reaches 1 (the Theta~ gradient of the horizontal
momenta, then their divergence), 2 over terrain (the 4-point averages of the metric shift).  So
H = 3 * 4 + S * r_sub with S = 1 + ns/2 + ns substep passes; the tests check the interior against
the undivided run bit for bit.

Exchange (two phases, so corners need no diagonal messages): phase x sends the H interior columns
next to each x-edge, over the interior rows, to the x-neighbours' halos; phase y then sends the H
interior rows next to each y-edge, over the whole widened x range (its x-halos fresh from phase
x), to the y-neighbours.  A rank's interior must be at least H wide in every sharded direction.
A direction with one rank has no halo: the periodic wrap of the window is the domain's.

Engines: anything with ``pack(i0, ni, j0, nj) -> 1-D tensor`` and ``unpack(i0, ni, j0, nj, buf)``
over its window's local column indices (every prognostic field, all levels, field-major).  The
transport is ``torch.distributed`` point-to-point (gloo for CPU tensors, NCCL for device tensors)
or, for several engines in one process, ``LocalRouter``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Dict, List, Sequence

import numpy as np


def split_range(n: int, parts: int, r: int):
    """Interior [a, b) of part r when n items are split into `parts` near-equal parts."""
    return (r * n) // parts, ((r + 1) * n) // parts


def step_reach(n_substeps: int, terrain: bool, substep_mode: int = 0) -> int:
    """Columns one RK3 step reaches sideways (see the module docstring)."""
    passes = 3 if substep_mode == 1 else 1 + n_substeps // 2 + n_substeps
    r_sub = 0 if substep_mode == 1 else (2 if terrain else 1)
    return 3 * 4 + passes * r_sub


@dataclass(frozen=True)
class Pencil:
    rank: int
    rx: int
    ry: int
    x0: int          # interior, global column indices [x0, x1) x [y0, y1)
    x1: int
    y0: int
    y1: int
    hx: int          # halo widths (0 in a direction with one rank)
    hy: int

    @property
    def nxl(self) -> int:
        return self.x1 - self.x0

    @property
    def nyl(self) -> int:
        return self.y1 - self.y0

    @property
    def nxw(self) -> int:
        return self.nxl + 2 * self.hx

    @property
    def nyw(self) -> int:
        return self.nyl + 2 * self.hy

    def window_columns(self, nx: int, ny: int):
        """Global x and y indices (periodic) of the window's columns."""
        return (np.arange(self.x0 - self.hx, self.x1 + self.hx) % nx,
                np.arange(self.y0 - self.hy, self.y1 + self.hy) % ny)


class PencilDecomp:
    """px x py ranks over an nx x ny periodic domain, rank = ry * px + rx."""

    def __init__(self, nx: int, ny: int, px: int, py: int, halo: int):
        if px < 1 or py < 1:
            raise ValueError("px, py must be >= 1")
        self.nx, self.ny, self.px, self.py, self.halo = nx, ny, px, py, halo
        self.hx = halo if px > 1 else 0
        self.hy = halo if py > 1 else 0
        for r in range(px):
            a, b = split_range(nx, px, r)
            if px > 1 and b - a < self.hx:
                raise ValueError(f"x interior of {b - a} columns is narrower than the halo {self.hx}")
        for r in range(py):
            a, b = split_range(ny, py, r)
            if py > 1 and b - a < self.hy:
                raise ValueError(f"y interior of {b - a} rows is narrower than the halo {self.hy}")

    @property
    def size(self) -> int:
        return self.px * self.py

    def rank_of(self, rx: int, ry: int) -> int:
        return (ry % self.py) * self.px + (rx % self.px)

    def pencil(self, rank: int) -> Pencil:
        rx, ry = rank % self.px, rank // self.px
        x0, x1 = split_range(self.nx, self.px, rx)
        y0, y1 = split_range(self.ny, self.py, ry)
        return Pencil(rank, rx, ry, x0, x1, y0, y1, self.hx, self.hy)

    def window_slices(self, rank: int, arr: np.ndarray) -> np.ndarray:
        """A global [k][j][i] array restricted to the rank's window (periodic wrap)."""
        p = self.pencil(rank)
        ii, jj = p.window_columns(self.nx, self.ny)
        return np.ascontiguousarray(np.asarray(arr)[..., jj, :][..., ii])

    def window_nodes(self, rank: int, nodes: np.ndarray) -> np.ndarray:
        """Nodal terrain [ny][nx] (nodes at (i dx, j dy)) restricted to the window: node i of the
        window is global node (x0 - hx + i) mod nx."""
        p = self.pencil(rank)
        ii, jj = p.window_columns(self.nx, self.ny)
        return np.ascontiguousarray(np.asarray(nodes)[jj][:, ii])

    # ----------------------------------------------------------------- exchange plan
    def messages(self, rank: int):
        """The strips rank `rank` sends and receives, in order: lists of
        (phase, peer, tag, (i0, ni, j0, nj)) in the window's local indices."""
        p = self.pencil(rank)
        sends, recvs = [], []
        if self.px > 1:
            h = self.hx
            left, right = self.rank_of(p.rx - 1, p.ry), self.rank_of(p.rx + 1, p.ry)
            rows = (p.hy, p.nyl)
            # my first h interior columns -> the left neighbour's right halo (tag 0); my last h
            # interior columns -> the right neighbour's left halo (tag 1)
            sends.append(("x", left, 0, (h, h) + rows))
            sends.append(("x", right, 1, (p.nxl, h) + rows))
            recvs.append(("x", right, 0, (h + p.nxl, h) + rows))
            recvs.append(("x", left, 1, (0, h) + rows))
        if self.py > 1:
            h = self.hy
            down, up = self.rank_of(p.rx, p.ry - 1), self.rank_of(p.rx, p.ry + 1)
            cols = (0, p.nxw)
            sends.append(("y", down, 2, cols + (h, h)))
            sends.append(("y", up, 3, cols + (p.nyl, h)))
            recvs.append(("y", up, 2, cols + (h + p.nyl, h)))
            recvs.append(("y", down, 3, cols + (0, h)))
        return sends, recvs


def shard_grid(n: int):
    """(px, py) for n ranks: the factorisation n = px * py closest to square, px >= py."""
    py = int(np.floor(np.sqrt(n)))
    while n % py:
        py -= 1
    return n // py, py


def window_workload(wl, decomp: PencilDecomp, rank: int):
    """The workload of rank `rank`: its window of every initial field and of the nodal terrain,
    on the window's grid (the spacing, levels and physics of `wl`)."""
    p = decomp.pencil(rank)
    kw = dict(nx=p.nxw, ny=p.nyw)
    for name in ("dtheta", "u", "v", "w", "phi"):
        a = getattr(wl, name)
        kw[name] = None if a is None else decomp.window_slices(rank, a)
    kw["terrain"] = None if wl.terrain is None else decomp.window_nodes(rank, wl.terrain)
    return wl.with_(**kw)


def exchange(decomp: PencilDecomp, rank: int, engine, dist) -> None:
    """Refreshes one rank's halo from its neighbours (collective over all ranks).  `dist` is
    torch.distributed (initialised); the engine's buffers must live where the backend expects
    them (CPU tensors for gloo, device tensors for NCCL)."""
    sends, recvs = decomp.messages(rank)
    for phase in ("x", "y"):
        ops = []
        bufs = []
        for ph, peer, tag, box in recvs:
            if ph != phase:
                continue
            b = engine.empty(box[1], box[3])
            bufs.append((box, b))
            ops.append(dist.P2POp(dist.irecv, b, peer, tag=tag))
        for ph, peer, tag, box in sends:
            if ph != phase:
                continue
            ops.append(dist.P2POp(dist.isend, engine.pack(*box), peer, tag=tag))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for box, b in bufs:
            engine.unpack(*box, b)


class LocalRouter:
    """Exchange between several engines held by one process (every rank's engine in a list):
    the same messages as `exchange`, delivered by direct copies.  No kernel waits on another;
    each copy is an ordinary pack / unpack between steps."""

    def __init__(self, decomp: PencilDecomp, engines: Sequence):
        assert len(engines) == decomp.size
        self.d, self.e = decomp, list(engines)

    def exchange(self) -> None:
        for phase in ("x", "y"):
            inbox: Dict[tuple, object] = {}
            for r in range(self.d.size):
                sends, _ = self.d.messages(r)
                for ph, peer, tag, box in sends:
                    if ph == phase:
                        inbox[(peer, r, tag)] = self.e[r].pack(*box)
            for r in range(self.d.size):
                _, recvs = self.d.messages(r)
                for ph, peer, tag, box in recvs:
                    if ph == phase:
                        self.e[r].unpack(*box, inbox[(r, peer, tag)])


def gather_interior(decomp: PencilDecomp, fields_of_rank: Callable[[int], Dict[str, np.ndarray]],
                    shapes: Dict[str, tuple]) -> Dict[str, np.ndarray]:
    """Assembles the global fields from every rank's window (its interior columns only)."""
    out = {k: np.empty(s) for k, s in shapes.items()}
    for r in range(decomp.size):
        p = decomp.pencil(r)
        f = fields_of_rank(r)
        for k in out:
            out[k][..., p.y0:p.y1, p.x0:p.x1] = f[k][..., p.hy:p.hy + p.nyl, p.hx:p.hx + p.nxl]
    return out


def interior_view(p: Pencil, arr):
    """The interior columns of a window field [.., nyw, nxw]."""
    return arr[..., p.hy:p.hy + p.nyl, p.hx:p.hx + p.nxl]


def fixed_order_sum(parts: List[float]) -> float:
    """Sum of per-rank partial sums in rank order (the same on every rank)."""
    s = 0.0
    for v in parts:
        s += v
    return s
