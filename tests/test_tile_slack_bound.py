"""The bound behind the particle buffers' tile slack (host-side model, no GPU).

The push writes every particle into its destination tile's slots of the other buffer set,
so each tile must be given, before the push, at least as many slots as particles can end up
in it.  A move is under one cell per axis (CFL), so the particles that can enter a tile are
those within one cell outside it: its frame.  The library gives tile t  count(t) + frame(t)
slots, frame(t) counted per particle as the neighbour tiles whose one-cell frame holds the
particle's cell (first cell of its tile along an axis: the neighbour below; last cell: the
neighbour above; and their combinations), and sizes each buffer set for 2^dim slots per
particle.  This model checks both claims on random and adversarial particle sets."""
import itertools

import numpy as np
import pytest


def tiles_of(c, pt, npt):
    q = c // pt
    t = np.zeros(len(c), np.int64)
    m = 1
    for d in range(c.shape[1]):
        t += q[:, d] * m
        m *= npt[d]
    return t


def frame_counts(c, pt, npt):
    """Per tile, the particles whose cell lies in its one-cell frame (the kernel's rule)."""
    dim = c.shape[1]
    q = c // pt
    loc = c - q * pt
    f = np.zeros(int(np.prod(npt)), np.int64)
    for off in itertools.product((-1, 0, 1), repeat=dim):
        if not any(off):
            continue
        ok = np.ones(len(c), bool)
        t = np.zeros(len(c), np.int64)
        m = 1
        for d, o in enumerate(off):
            if o < 0:
                ok &= loc[:, d] == 0
            elif o > 0:
                ok &= loc[:, d] == pt[d] - 1
            nq = q[:, d] + o
            ok &= (nq >= 0) & (nq < npt[d])
            t += nq * m
            m *= npt[d]
        np.add.at(f, t[ok], 1)
    return f


@pytest.mark.parametrize("dim,n,pt", [(1, (64,), (4,)), (2, (48, 40), (8, 4)), (2, (40, 40), (2, 2)),
                                      (3, (24, 16, 16), (4, 4, 2)), (3, (16, 16, 16), (2, 2, 2))])
def test_arrivals_never_exceed_count_plus_frame(dim, n, pt):
    rng = np.random.default_rng(dim * 100 + pt[0])
    n, pt = np.array(n), np.array(pt)
    npt = -(-n // pt)
    for trial in range(20):
        N = 4000
        x = rng.uniform(3, n - 3, size=(N, dim))
        c = np.floor(x).astype(np.int64)
        # moves under one cell per axis, some of them just under
        mv = rng.uniform(-0.999, 0.999, size=(N, dim))
        if trial % 2:
            mv = np.sign(mv) * 0.999
        c1 = np.floor(x + mv).astype(np.int64)
        cnt = np.bincount(tiles_of(c, pt, npt), minlength=int(np.prod(npt)))
        after = np.bincount(tiles_of(c1, pt, npt), minlength=int(np.prod(npt)))
        slots = cnt + frame_counts(c, pt, npt)
        assert np.all(after <= slots)
        assert slots.sum() <= (2 ** dim) * N


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_slots_reach_two_to_the_dim_per_particle_only_in_the_worst_case(dim):
    """Every particle in a tile corner cell (away from the box faces): each lies in the
    frames of 2^dim - 1 other tiles, and the slots add up to exactly 2^dim per particle."""
    pt = np.full(dim, 4)
    npt = np.full(dim, 6)
    cells = []
    for q in itertools.product(range(1, 5), repeat=dim):
        for corner in itertools.product((0, 3), repeat=dim):
            cells.append(np.array(q) * 4 + np.array(corner))
    c = np.array(cells)
    cnt = np.bincount(tiles_of(c, pt, npt), minlength=int(np.prod(npt)))
    slots = cnt + frame_counts(c, pt, npt)
    assert slots.sum() == (2 ** dim) * len(c)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_a_tile_whose_frame_all_moves_in_is_filled_exactly(dim):
    """Electrons at rest in tile (1, ...) and one in every cell of its frame moving straight
    in (diagonally from the edges and corners): the tile ends with exactly its slots."""
    pt = np.full(dim, 4)
    npt = np.full(dim, 4)
    lo = pt.copy()                       # tile (1, 1, ...) covers [4, 8) per axis
    c0, c1 = [], []
    for cell in itertools.product(*[range(3, 9)] * dim):
        cell = np.array(cell)
        step = np.where(cell < lo, 1, np.where(cell >= lo + pt, -1, 0))
        c0.append(cell)
        c1.append(cell + step)
    c0, c1 = np.array(c0), np.array(c1)
    t = int(np.sum(np.array([4 ** d for d in range(dim)])))   # index of tile (1, 1, ...)
    cnt = np.bincount(tiles_of(c0, pt, npt), minlength=int(np.prod(npt)))
    after = np.bincount(tiles_of(c1, pt, npt), minlength=int(np.prod(npt)))
    slots = cnt + frame_counts(c0, pt, npt)
    assert after[t] == slots[t] == 6 ** dim
    assert np.all(after <= slots)
