"""Placement of the pushed particles into their destination tiles (a layout choice of this
implementation; the paper has no counterpart).  Each tile of a particle buffer set keeps
slack for exactly the particles within one cell outside it, the only ones a step can bring
in; these cases fill that slack to the last slot and check that every particle arrives,
with the physics of the oracle."""
import math

import numpy as np
import pytest

import synth
from _support import match_by_id, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    pic.load()
    return pic


def crowd(w, tile, per_cell, speed):
    """Electrons at rest filling tile (2, 2) of the grid, and electrons in its one-cell frame
    moving straight into it (diagonally from the corners), each at the offset nearest the
    tile so that all of them enter in the first step."""
    t0 = (2 * tile[0], 2 * tile[1])
    x, u = [], []
    rng = np.random.default_rng(5)
    for cy in range(t0[1] - 1, t0[1] + tile[1] + 1):
        for cx in range(t0[0] - 1, t0[0] + tile[0] + 1):
            sx = 1.0 if cx < t0[0] else (-1.0 if cx >= t0[0] + tile[0] else 0.0)
            sy = 1.0 if cy < t0[1] else (-1.0 if cy >= t0[1] + tile[1] else 0.0)
            for _ in range(per_cell):
                ox = 0.95 if sx > 0 else (0.05 if sx < 0 else rng.uniform(0.2, 0.8))
                oy = 0.95 if sy > 0 else (0.05 if sy < 0 else rng.uniform(0.2, 0.8))
                x.append([(cx + ox) * w.dx, (cy + oy) * w.dx, 0.0])
                u.append([speed * sx, speed * sy, 0.0])
    x, u = np.array(x), np.array(u)
    return x, u, np.full(len(x), 1e-4), np.arange(len(x))


@pytest.mark.parametrize("prec", [synth.FP64, synth.FP32])
def test_a_tile_filled_to_its_slack_keeps_every_particle(P, orc, prec):
    w = small_2d(precision=prec).with_(beam=synth.BEAM_NONE, ppc=0, a0=0.0)
    tile = (16, 16)
    x, u, wt, ids = crowd(w, tile, per_cell=4, speed=4.0)
    sim = P.Simulation(P.config_from(w, tile=tile, max_particles=len(ids)))
    sim.set_particles(x, u, wt, ids)
    ref = orc.Sim(orc.config_from(w))
    ref.set_particles(x, u, wt, ids)
    for step in range(1, 4):
        sim.step(1)
        ref.step(1)
        pg, pr = sim.particles(), ref.particles()      # raises if a particle found no slot
        assert sim.info().n_alive == len(pr["id"]) == len(ids), step
        assert np.array_equal(np.sort(pg["id"]), np.sort(pr["id"])), step
        common, ia, ib = match_by_id(pg, pr)
        tol = 1e-9 if prec == synth.FP64 else 1e-5
        assert np.abs(pg["x"][ia] - pr["x"][ib]).max() < tol * 100 * w.dx, step
        assert np.abs(pg["u"][ia] - pr["u"][ib]).max() < tol * 10, step
        if step == 1:
            # every frame electron has entered tile (2, 2), which now holds its own 16 x 16
            # x 4 plus the frame's 68 x 4: the slots it was given, to the last one
            c = np.floor(pg["x"][:, :2] / w.dx).astype(int)
            in_tile = np.all((c >= [32, 32]) & (c < [48, 48]), axis=1)
            assert in_tile.sum() == (16 * 16 + 68) * 4
    sim.close()


def test_particles_leave_in_every_direction_each_step(P, orc):
    """A hot slab (|u| ~ 3 in random directions, FP64): a large share of the electrons change
    tile every step; the run keeps matching the oracle particle by particle."""
    w = small_2d(precision=synth.FP64).with_(beam=synth.BEAM_NONE, ppc=0, a0=0.0)
    rng = np.random.default_rng(9)
    n = 6000
    x = np.column_stack([rng.uniform(20, 76, n) * w.dx, rng.uniform(12, 68, n) * w.dx, np.zeros(n)])
    ang = rng.uniform(0, 2 * math.pi, n)
    u = np.column_stack([3 * np.cos(ang), 3 * np.sin(ang), rng.normal(0, 0.5, n)])
    wt, ids = np.full(n, 1e-4), np.arange(n)
    sim = P.Simulation(P.config_from(w, tile=(8, 8), max_particles=n))
    sim.set_particles(x, u, wt, ids)
    ref = orc.Sim(orc.config_from(w))
    ref.set_particles(x, u, wt, ids)
    sim.step(12)
    ref.step(12)
    pg, pr = sim.particles(), ref.particles()
    assert np.array_equal(np.sort(pg["id"]), np.sort(pr["id"]))
    common, ia, ib = match_by_id(pg, pr)
    assert np.abs(pg["x"][ia] - pr["x"][ib]).max() < 1e-9 * 100 * w.dx
    assert np.abs(pg["u"][ia] - pr["u"][ib]).max() < 1e-8
    sim.close()


def test_set_particles_rejects_the_first_invalid_particle(P):
    """A large upload (converted on several host threads): an out-of-range position or id
    is rejected with the index of the first offending particle, and nothing is changed."""
    w = synth.c2_2d_lp()
    x, u, wt, ids = synth.slab_particles(w)
    n = len(ids)
    sim = P.Simulation(P.config_from(w, tile=(32, 16), chunk=1024))
    before = sim.info().n_alive
    bad_x = x.copy()
    bad_x[n - 5, 1] = 1.0 * w.dx          # inside the removal margin on axis 1
    bad_x[n // 2, 0] = -3.0                # outside the box on axis 0: the first offender
    with pytest.raises(P.PicError) as e:
        sim.set_particles(bad_x, u, wt, ids)
    assert e.value.status == P.PIC_EINVAL and f"particle {n // 2} " in str(e.value) and "axis 0" in str(e.value)
    bad_id = ids.copy()
    bad_id[n - 3] = -1
    with pytest.raises(P.PicError) as e:
        sim.set_particles(x, u, wt, bad_id)
    assert "id out of range" in str(e.value)
    with pytest.raises(P.PicError) as e:
        sim.set_particles(np.vstack([x, x[:1]]), np.vstack([u, u[:1]]), np.append(wt, wt[:1]), np.append(ids, n))
    assert e.value.status == P.PIC_ECAPACITY
    assert sim.info().n_alive == before
    # a valid upload of the same records round-trips through the tile slots
    sim.set_particles(x, u, wt, ids)
    p = sim.particles()
    order = np.argsort(p["id"])
    assert np.array_equal(p["id"][order], ids)
    assert np.abs(p["x"][order] - x).max() < 1e-6 * w.dx * 1024
    sim.close()
