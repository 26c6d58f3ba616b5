"""Autotuner of the particle tile and work-item size, and the physics under every tile and
work-item size it may pick: the same results against the oracle (the tile only regroups the
particles and the order of the current sums)."""
import time

import numpy as np
import pytest

import synth
from _support import momentum_error, field_errors, small_2d, small_3d

pytestmark = pytest.mark.gpu

TILES = {2: [(16, 16), (32, 16), (16, 8), (32, 32), (8, 8), (64, 8), (64, 16)],
         3: [(8, 8, 8), (16, 8, 8), (8, 8, 4), (16, 8, 4), (8, 4, 4), (32, 4, 4), (32, 4, 2), (32, 8, 2)]}


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    pic.load()
    return pic


@pytest.mark.parametrize("dim", [2, 3])
def test_every_candidate_tile_matches_the_oracle(P, orc, dim):
    w = small_2d() if dim == 2 else small_3d()
    steps = 20
    ref = orc.Sim(orc.config_from(w))
    ref.step(steps)
    pr, fr = ref.particles(), ref.fields()
    for tile in TILES[dim]:
        for chunk in (256, 1024, 4096):
            sim = P.Simulation(P.config_from(w, tile=tile, chunk=chunk))
            assert list(sim.info().params.tile)[:dim] == list(tile)
            sim.step(steps)
            err, n = momentum_error(sim.particles(), pr, w.a0)
            assert n == len(pr["id"]), (tile, chunk)
            assert err < 1e-5, (tile, chunk, err)
            assert field_errors(sim.fields(), fr)[:6].max() < 1e-5, (tile, chunk)
            sim.close()


def test_autotune_picks_a_candidate_and_caches_it(P):
    w = small_2d()
    c = P.config_from(w)
    t0 = time.perf_counter()
    ms = P.pic_autotune(c, 3)
    t1 = time.perf_counter()
    assert ms > 0
    assert tuple(c.tile)[:2] in TILES[2]
    assert c.chunk in (256, 512, 1024, 2048, 4096)
    c2 = P.config_from(w)
    ms2 = P.pic_autotune(c2, 3)
    t2 = time.perf_counter()
    assert (tuple(c2.tile), c2.chunk, ms2) == (tuple(c.tile), c.chunk, ms)
    assert t2 - t1 < 0.25 * (t1 - t0)          # cached: nothing measured


def test_init_with_autotune_runs_the_tuned_layout(P, orc):
    w = small_2d()
    sim = P.Simulation(P.config_from(w, autotune_steps=2))
    prm = sim.info().params
    assert tuple(prm.tile)[:2] in TILES[2] and prm.chunk in (256, 512, 1024, 2048, 4096)
    sim.step(10)
    ref = orc.Sim(orc.config_from(w))
    ref.step(10)
    err, n = momentum_error(sim.particles(), ref.particles(), w.a0)
    assert err < 1e-5
