"""Spatial domain decomposition of one scattered-field PIC simulation along x (the
propagation axis) over several ranks: the method's one real exchange step when a single
simulation spans several GPUs (the paper's own runs used Smilei's MPI patches on 5120
cores, Conclusion).  Host logic only: the decomposition, the ghost regions and the three
exchanges of a step, written against a small per-rank stepper interface and
torch.distributed point-to-point messages (gloo for host arrays; the same messages carry
device tensors over NCCL).

Rank r owns the cells [x0, x1) of the global x axis and the field points whose global x
index lies in [x0, x1) (the last rank also owns node n_x).  Its local box is the owned
slab widened by GHOST cells on each side that has a neighbour; a local array holds the
global x indices l0 .. l1.  One step, in the order of the Sec. 2 cycle:

  1. the stepper's particle phase (gather, incident field, push, move, Esirkepov
     deposit) on the rank's electrons, all in owned cells: their stencils reach at most
     three nodes past the cut, inside the ghost region;
  2. current ghost sum: over the region two neighbours' boxes share, each adds the other's
     J, so every owned point and the ghost points next to the cut hold the whole J^{n+1/2};
  3. the stepper's field phase (the Yee update) on the local box.  An owned point needs
     its neighbours within one point, correct at the start of the phase; the ghost points
     near the box's outer face go wrong (nothing beyond it, the face's absorbing
     condition) and are never used before the refresh;
  4. field ghost refresh: every ghost point of E and B is overwritten by its owner's value;
  5. migration: electrons that moved into a neighbour's cells (at most one cell per step at
     CFL < 1) are handed over.

The incident field needs no exchange: it is evaluated locally at every electron.  With
GHOST = 4 the particle stencils (three nodes past a cell), the field update (one point)
and the removal margin at the local box's face (three cells, so that an electron which
just crossed the cut is not taken for one leaving the box) all stay inside the local box.

Stepper interface (duck-typed), in the rank's local coordinates (x from the local box's
first node):  step_particles(), step_fields(), fields() -> float64 (9, ext_z, ext_y,
ext_x) of Ex Ey Ez Bx By Bz Jx Jy Jz, set_fields(F), particles() -> dict(x, u, w, id),
set_particles(x, u, w, id).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GHOST = 4


@dataclass(frozen=True)
class Slab:
    """One rank's part of the global x axis (cells)."""
    rank: int
    world: int
    n_x: int        # global cells along x
    x0: int         # owned cells [x0, x1)
    x1: int
    l0: int         # local box cells [l0, l1): its arrays hold x indices l0 .. l1
    l1: int

    @property
    def lower(self):
        return self.rank - 1 if self.rank > 0 else None

    @property
    def upper(self):
        return self.rank + 1 if self.rank < self.world - 1 else None

    @property
    def n_local(self) -> int:
        return self.l1 - self.l0

    def owned_points(self) -> tuple:
        """Global x indices [a, b) of the points this rank owns (every component; the last
        rank's b includes node n_x, which only the components not staggered along x use)."""
        return self.x0, self.x1 + (1 if self.upper is None else 0)


def decompose(n_x: int, world: int, ghost: int = GHOST) -> list:
    """Equal slabs of the x axis (the remainder on the first ranks).  Every slab is wider
    than twice the ghost region (plus two), so a rank's ghost points are all owned by its
    neighbours and the regions shared across different cuts do not meet."""
    if world < 1 or n_x < world * (2 * ghost + 2):
        raise ValueError(f"{n_x} cells cannot be split over {world} ranks with {ghost} ghost cells")
    base, extra = divmod(n_x, world)
    out, x = [], 0
    for r in range(world):
        w = base + (1 if r < extra else 0)
        x0, x1 = x, x + w
        out.append(Slab(r, world, n_x, x0, x1, x0 - ghost if r > 0 else 0, x1 + ghost if r < world - 1 else n_x))
        x = x1
    return out


def owner_of_cell(slabs, cell) -> np.ndarray:
    """Rank owning each global x cell index."""
    return np.searchsorted(np.array([s.x1 for s in slabs]), np.asarray(cell), side="right")


def shift_of(slab: Slab, dx: float) -> float:
    """Global coordinate of the local box's first node: local x = global x - shift, and the
    beam's focus / reference plane moves by the same amount in the local configuration."""
    return slab.l0 * dx


def ghost_on_side(slab: Slab, peer: Slab) -> tuple:
    """Global x indices [a, b) of `slab`'s ghost points that `peer` (a neighbour) owns."""
    if peer.rank == slab.rank - 1:
        return slab.l0, slab.x0
    return slab.x1, slab.l1 + 1


def _loc(slab: Slab, a: int, b: int) -> slice:
    return slice(a - slab.l0, b - slab.l0)


# ---- point-to-point messages ----------------------------------------------------------
def _exchange(dist, sends: dict, recv_shapes: dict) -> dict:
    """Send float64 arrays sends[peer] and receive arrays of shape recv_shapes[peer] from
    every peer at once (non-blocking pairs: no order of the ranks can deadlock)."""
    import torch

    reqs, bufs = [], {}
    for peer, shape in recv_shapes.items():
        bufs[peer] = torch.empty(tuple(int(v) for v in shape), dtype=torch.float64)
        reqs.append(dist.irecv(bufs[peer], src=peer))
    keep = []
    for peer, arr in sends.items():
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64))
        keep.append(t)
        reqs.append(dist.isend(t, dst=peer))
    for r in reqs:
        r.wait()
    return {p: b.numpy() for p, b in bufs.items()}


def _neighbours(slabs, slab):
    return [slabs[p] for p in (slab.lower, slab.upper) if p is not None]


def overlap(a: Slab, b: Slab) -> tuple:
    """Global x indices [lo, hi) held by both neighbours' local boxes: the ghost region on
    each side of their cut and the owned points it mirrors."""
    return max(a.l0, b.l0), min(a.l1, b.l1) + 1


def sum_current_ghosts(dist, slabs, rank: int, F: np.ndarray) -> None:
    """Step 2 (in place on the local array F): over the region two neighbours' boxes share,
    each holds the J of its own electrons only; each sends its J there to the other and adds
    what it receives, so both hold the whole J on every point of the region.  The owned
    points need it, and so does the first ghost point past the cut, whose E the owned B
    next to the cut reads within the same Yee update.  Regions of different cuts are
    disjoint (slabs wider than twice the ghost region)."""
    me = slabs[rank]
    sends, shapes, where = {}, {}, {}
    for nb in _neighbours(slabs, me):
        a, b = overlap(me, nb)
        sends[nb.rank] = F[6:9, :, :, _loc(me, a, b)]
        where[nb.rank] = (a, b)
        shapes[nb.rank] = (3,) + F.shape[1:3] + (b - a,)
    for peer, arr in _exchange(dist, sends, shapes).items():
        a, b = where[peer]
        F[6:9, :, :, _loc(me, a, b)] += arr


def refresh_field_ghosts(dist, slabs, rank: int, F: np.ndarray) -> None:
    """Step 4 (in place on F): E and B at every ghost point become the owner's values."""
    me = slabs[rank]
    sends, shapes, where = {}, {}, {}
    for nb in _neighbours(slabs, me):
        a2, b2 = ghost_on_side(nb, me)          # points I own that the neighbour mirrors
        sends[nb.rank] = F[0:6, :, :, _loc(me, a2, b2)]
        a, b = ghost_on_side(me, nb)
        where[nb.rank] = (a, b)
        shapes[nb.rank] = (6,) + F.shape[1:3] + (b - a,)
    for peer, arr in _exchange(dist, sends, shapes).items():
        a, b = where[peer]
        F[0:6, :, :, _loc(me, a, b)] = arr


def migrate(dist, slabs, rank: int, parts: dict, dx: float) -> tuple:
    """Step 5: electrons whose x cell a neighbour owns are sent there (global coordinates on
    the wire); returns the rank's new particle set (kept, then received) and the number
    handed over."""
    me = slabs[rank]
    sh = shift_of(me, dx)
    cell = np.floor(parts["x"][:, 0] / dx).astype(np.int64) + me.l0
    own = owner_of_cell(slabs, cell)
    rec = np.concatenate([parts["x"] + np.array([sh, 0.0, 0.0]), parts["u"], parts["w"][:, None],
                          parts["id"][:, None].astype(np.float64)], axis=1) if len(cell) else np.zeros((0, 8))
    nbrs = _neighbours(slabs, me)
    if np.any((own != rank) & ~np.isin(own, [nb.rank for nb in nbrs])):
        raise RuntimeError("an electron moved past a neighbour's slab in one step")
    out = {nb.rank: rec[own == nb.rank] for nb in nbrs}
    counts = _exchange(dist, {p: np.array([float(len(v))]) for p, v in out.items()},
                       {nb.rank: (1,) for nb in nbrs})
    got = _exchange(dist, out, {p: (int(c[0]), 8) for p, c in counts.items()})
    keep = rec[own == rank]
    allr = np.concatenate([keep] + [got[p] for p in sorted(got)], axis=0)
    new = {"x": allr[:, 0:3] - np.array([sh, 0.0, 0.0]), "u": allr[:, 3:6].copy(), "w": allr[:, 6].copy(),
           "id": allr[:, 7].astype(np.int64)}
    return new, int(len(rec) - len(keep))


class DomainRun:
    """One rank of a simulation split along x: drives the rank's stepper through the five
    parts of a step above."""

    def __init__(self, dist, slabs, rank: int, stepper, dx: float):
        self.dist, self.slabs, self.rank, self.sim, self.dx = dist, slabs, rank, stepper, dx
        self.migrated = 0

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            self.sim.step_particles()
            F = self.sim.fields()
            sum_current_ghosts(self.dist, self.slabs, self.rank, F)
            self.sim.set_fields(F)
            self.sim.step_fields()
            F = self.sim.fields()
            refresh_field_ghosts(self.dist, self.slabs, self.rank, F)
            self.sim.set_fields(F)
            p, moved = migrate(self.dist, self.slabs, self.rank, self.sim.particles(), self.dx)
            self.sim.set_particles(p["x"], p["u"], p["w"], p["id"])
            self.migrated += moved

    def owned_fields(self) -> tuple:
        """(global x index of the first owned point, F restricted to the owned points)."""
        me = self.slabs[self.rank]
        a, b = me.owned_points()
        return a, self.sim.fields()[:, :, :, _loc(me, a, b)]

    def particles_global(self) -> dict:
        p = self.sim.particles()
        x = p["x"] + np.array([shift_of(self.slabs[self.rank], self.dx), 0.0, 0.0])
        return {"x": x, "u": p["u"], "w": p["w"], "id": p["id"]}
