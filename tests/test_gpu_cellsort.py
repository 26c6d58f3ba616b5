"""Cell sort within the particle tiles (a layout choice of this implementation; the paper
has no counterpart): every sort_every-th step the re-sort leaves each tile's particles in
cell order.  Checked: the order itself (tile-major, then the cell's rank in its tile, x
fastest), that the particle set is unchanged, and that the physics matches a run without
the sort and the oracle (only the order of the current sums differs)."""
import numpy as np
import pytest

from _support import field_errors, momentum_error, small_2d, small_3d

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


def order_keys(sim, w):
    """(tile index, rank of the cell in its tile) of every particle in buffer order."""
    prm = sim.info().params
    pt = [int(v) for v in prm.tile][: w.dim]
    c = np.floor(sim.particles()["x"][:, : w.dim] / w.dx).astype(np.int64)
    npt = [-(-int(w.n[d]) // pt[d]) for d in range(w.dim)]
    tile = np.zeros(len(c), np.int64)
    rank = np.zeros(len(c), np.int64)
    mt, mr = 1, 1
    for d in range(w.dim):
        tile += mt * (c[:, d] // pt[d])
        rank += mr * (c[:, d] % pt[d])
        mt *= npt[d]
        mr *= pt[d]
    return tile, rank


def is_sorted(tile, rank):
    key = tile * (1 << 20) + rank
    return bool(np.all(np.diff(key) >= 0))


@pytest.mark.parametrize("dim,tile", [(2, (16, 16)), (2, (32, 8)), (3, (8, 8, 4))])
def test_sort_step_leaves_every_tile_in_cell_order(P, dim, tile):
    w = small_2d() if dim == 2 else small_3d()
    sim = P.Simulation(P.config_from(w, tile=tile, sort_every=3))
    ids0 = np.sort(sim.particles()["id"])
    # step 25-ish: the pulse is on the plasma and the electrons move between cells
    for k in range(1, 31):
        sim.step(1)
        t, r = order_keys(sim, w)
        assert np.all(np.diff(t) >= 0), k             # every step: ordered by tile
        if k % 3 == 0:
            assert is_sorted(t, r), k                 # cell-sort steps: by cell within the tile
    p = sim.particles()
    # nothing created or lost but the box leavers
    ex = sim.exits()
    assert np.array_equal(np.sort(np.concatenate([p["id"], ex["id"]])), ids0)
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_sort_changes_only_the_rounding(P, orc, dim):
    w = small_2d() if dim == 2 else small_3d()
    steps = 40 if dim == 2 else 30
    ref = orc.Sim(orc.config_from(w))
    ref.step(steps)
    pr, fr = ref.particles(), ref.fields()
    out = {}
    for k in (1, 4, -1):
        sim = P.Simulation(P.config_from(w, sort_every=k))
        sim.step(steps)
        p, F = sim.particles(), sim.fields()
        err, n = momentum_error(p, pr, w.a0)
        assert n == len(pr["id"]), k
        assert err < 1e-5, (k, err)
        assert field_errors(F, fr)[:6].max() < 1e-5, k
        out[k] = (p, F, sim.energies())
        sim.close()
    # sorted and unsorted runs agree to FP32 rounding of the sums
    for k in (1, 4):
        assert field_errors(out[k][1], out[-1][1])[:6].max() < 1e-5
        np.testing.assert_allclose(out[k][2][:3], out[-1][2][:3], rtol=1e-5, atol=1e-12)


def test_batch_sorts_the_members_that_have_a_cell_sort(P):
    w = small_2d()
    a = P.Simulation(P.config_from(w, tile=(16, 16), sort_every=2))
    b = P.Simulation(P.config_from(w.with_(seed=22), tile=(16, 16), sort_every=-1))
    for k in range(1, 31):
        P.pic_batch_step([a.h, b.h], 1, 0)
        ta, ra = order_keys(a, w)
        tb, rb = order_keys(b, w)
        assert np.all(np.diff(ta) >= 0) and np.all(np.diff(tb) >= 0), k
        if k % 2 == 0:
            assert is_sorted(ta, ra), k
    a.close()
    b.close()
