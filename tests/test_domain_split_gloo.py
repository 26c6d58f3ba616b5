"""The spatial domain split of one simulation along x (paper_2310_11393_gb300.domain) on
two and three gloo ranks on the CPU, each rank stepping its slab with the oracle's two
step phases, against the unsplit oracle run element by element: every electron's position
and momentum by id, the exits, and all nine field components (E, B and the last step's J)
at every grid point.  The runs are chosen so that electrons cross the cuts and their
currents straddle them (a tightly focused LP pulse at a0 = 10 through a 2D slab, an RP pulse
at a0 = 10 through a 3D slab, the cuts running through both).  Only the summation order of J at points next to a cut differs from the unsplit
run (contributions from both sides), so the bar is FP64 round-off."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(dim=2):
    import synth

    if dim == 3:
        # a tightly focused RP pulse through a 3D slab the cuts run through
        n = (48, 14, 14)
        dx = 2 * math.pi / 16
        dt = 0.95 * dx / math.sqrt(3)
        return synth.Workload(name="3d_rp_split", dim=3, n=n, dx=dx, steps=30, beam=synth.BEAM_RP, a0=10.0,
                              duration=synth.fs(5.0), w0=2 * math.pi * 0.7, slab_lo=(8, 3, 3), slab_hi=(40, 11, 11),
                              n_e=0.05, ppc=1, seed=43, focus=(24 * dx, 7 * dx, 7 * dx), t_focus=15 * dt,
                              precision=synth.FP64)
    n = (96, 40, 1)
    dx = 2 * math.pi / 32
    dt = 0.95 * dx / math.sqrt(2)
    return synth.Workload(name="2d_lp_split", dim=2, n=n, dx=dx, steps=40, beam=synth.BEAM_LP, a0=10.0,
                          duration=synth.fs(5.0), w0=2 * math.pi * 0.5, slab_lo=(20, 6, 0), slab_hi=(76, 34, 1),
                          n_e=0.05, ppc=2, seed=41, focus=(48 * dx, 20 * dx, 0.0), t_focus=20 * dt,
                          precision=synth.FP64)


class OracleSlab:
    """The stepper interface of the domain module on an oracle simulation of one slab."""

    def __init__(self, sim):
        self.s = sim

    def step_particles(self):
        self.s.step_particles()

    def step_fields(self):
        self.s.step_fields()

    def fields(self):
        return self.s.fields()

    def set_fields(self, F):
        self.s.set_fields(F)

    def particles(self):
        return self.s.particles()

    def set_particles(self, x, u, w, ids):
        self.s.set_particles(x, u, w, ids)


def _rank(rank, world, port, steps, q, dim):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2310_11393_gb300 import domain

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _workload(dim)
    slabs = domain.decompose(w.n[0], world)
    me = slabs[rank]
    sh = domain.shift_of(me, w.dx)
    # the slab's own box: the global workload moved by -shift along x, electrons set explicitly
    lw = w.with_(n=(me.n_local, w.n[1], w.n[2]), focus=(w.focus[0] - sh, w.focus[1], w.focus[2]), ppc=0)
    cfg = oracle.config_from(lw)
    gcfg = oracle.config_from(w)
    cfg.a, cfg.s, cfg.psi0 = gcfg.a, gcfg.s, gcfg.psi0          # the global pulse parameters
    sim = oracle.Sim(cfg)
    x, u, wt, ids = synth.slab_particles(w)
    cell = np.floor(x[:, 0] / w.dx).astype(np.int64)
    mine = domain.owner_of_cell(slabs, cell) == rank
    sim.set_particles(x[mine] - np.array([sh, 0.0, 0.0]), u[mine], wt[mine], ids[mine])
    run = domain.DomainRun(dist, slabs, rank, OracleSlab(sim), w.dx)
    run.step(steps)
    a, F = run.owned_fields()
    q.put((rank, run.particles_global(), sim.exits(), a, F, run.migrated))
    dist.barrier()
    dist.destroy_process_group()


def _split_run(world, steps, dim=2):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, q, dim)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=600) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("dim,world", [(2, 2), (2, 3), (3, 2)])
def test_split_run_equals_the_unsplit_run(orc, dim, world):
    import synth
    from paper_2310_11393_gb300 import domain

    w = _workload(dim)
    steps = w.steps
    ref = orc.Sim(orc.config_from(w))
    ref.step(steps)
    out = _split_run(world, steps, dim)
    # electrons: the union over the ranks is the unsplit set, value by value
    parts = {k: np.concatenate([o[1][k] for o in out]) for k in ("x", "u", "w", "id")}
    pr = ref.particles()
    assert len(parts["id"]) == len(np.unique(parts["id"]))
    np.testing.assert_array_equal(np.sort(parts["id"]), np.sort(pr["id"]))
    ia, ib = np.argsort(parts["id"]), np.argsort(pr["id"])
    assert np.abs(parts["x"][ia] - pr["x"][ib]).max() < 1e-11 * w.n[0] * w.dx
    assert np.abs(parts["u"][ia] - pr["u"][ib]).max() < 1e-10 * max(1.0, np.abs(pr["u"]).max())
    assert np.abs(pr["u"]).max() > 1.0                      # relativistic electrons
    # exits
    ex = {k: np.concatenate([o[2][k] for o in out]) for k in ("u", "id", "step")}
    er = ref.exits()
    np.testing.assert_array_equal(np.sort(ex["id"]), np.sort(er["id"]))
    ja, jb = np.argsort(ex["id"]), np.argsort(er["id"])
    np.testing.assert_array_equal(ex["step"][ja], er["step"][jb])
    if len(er["id"]):
        assert np.abs(ex["u"][ja] - er["u"][jb]).max() < 1e-10 * max(1.0, np.abs(er["u"]).max())
    # fields: the owned points of the ranks tile the global grid
    Fr = ref.fields()
    G = np.zeros_like(Fr)
    covered = np.zeros(Fr.shape[-1], dtype=int)
    for o in out:
        a, F = o[3], o[4]
        G[..., a:a + F.shape[-1]] = F
        covered[a:a + F.shape[-1]] += 1
    assert np.all(covered == 1)
    nonzero = 0
    for c in range(9):
        scale = np.abs(Fr[c]).max()
        nonzero += scale > 0            # the in-plane components (Ex, Ey, Bz, Jx, Jy, Jz)
        assert np.abs(G[c] - Fr[c]).max() <= 1e-10 * scale, (c, np.abs(G[c] - Fr[c]).max() / max(scale, 1e-300))
    assert nonzero >= 5
    # the cuts were exercised: electrons crossed them and currents straddle them
    assert sum(o[5] for o in out) > 0
    slabs = domain.decompose(w.n[0], world)
    for s in slabs[1:]:
        assert np.abs(Fr[6:9, ..., s.x0 - 2:s.x0 + 3]).max() > 0


def test_decomposition_tiles_the_axis():
    from paper_2310_11393_gb300 import domain

    for n, world in ((96, 2), (97, 3), (80, 8)):
        slabs = domain.decompose(n, world)
        assert slabs[0].x0 == 0 and slabs[-1].x1 == n
        for a, b in zip(slabs, slabs[1:]):
            assert a.x1 == b.x0
            assert domain.ghost_on_side(a, b) == (a.x1, a.l1 + 1)
            assert domain.ghost_on_side(b, a) == (b.l0, b.x0)
            # every ghost point is owned by the neighbour on that side
            assert b.x0 <= a.x1 and a.l1 + 1 <= b.x1 + (1 if b.upper is None else 0)
            assert a.x0 <= b.l0
        cells = np.arange(n)
        own = domain.owner_of_cell(slabs, cells)
        for s in slabs:
            assert np.all(own[s.x0:s.x1] == s.rank)
        for a, b in zip(slabs, slabs[1:]):
            lo, hi = domain.overlap(a, b)
            assert (lo, hi) == (b.l0, a.l1 + 1)
        for a, b, c in zip(slabs, slabs[1:], slabs[2:]):
            assert domain.overlap(a, b)[1] <= domain.overlap(b, c)[0]     # disjoint regions
    with pytest.raises(ValueError):
        domain.decompose(70, 8)
