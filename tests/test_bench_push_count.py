"""The benchmark's host logic (CPU).  Its push count: every electron alive at the end of the
timed steps counts each of them, one that left the box counts the timed steps up to the one
in which it left (its exit record holds that step's index); checked on a fake simulation and
on the oracle, whose per-step particle count gives the same sum step by step.  Its timed
window: centred on the pulse's crossing of the focus."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakeSim:
    def __init__(self, steps):
        self._steps = np.asarray(steps, dtype=np.int64)

    def exits(self):
        return {"step": self._steps}


def test_pushes_of_counts_the_steps_up_to_each_exit():
    import bench

    # window of 10 steps from step 100; exits before the window are ignored, one in its
    # first step counts 1 push, one in its last counts 10
    sim = _FakeSim([5, 99, 100, 104, 109])
    assert bench.pushes_of(sim, 100, 10, n_end=7) == 7 * 10 + 1 + 5 + 10
    assert bench.pushes_of(_FakeSim([]), 0, 3, n_end=4) == 12


def test_exit_record_count_matches_the_stepwise_sum_on_the_oracle(orc):
    import synth

    # a small 2D box; a few electrons sit next to the +x face moving out at 0.9 c, others
    # inside at rest, so that exits fall in different steps of the window
    n = (48, 32, 1)
    dx = 2 * math.pi / 16
    w = synth.Workload(name="2d_exits", dim=2, n=n, dx=dx, steps=12, beam=synth.BEAM_LP, a0=0.0,
                       duration=synth.fs(5.0), w0=2 * math.pi, slab_lo=(8, 8, 0), slab_hi=(40, 24, 1),
                       n_e=0.01, ppc=0, seed=3, focus=(24 * dx, 16 * dx, 0.0), t_focus=0.0,
                       precision=synth.FP64)
    sim = orc.Sim(orc.config_from(w))
    k = 12
    xs = [(n[0] - 4.0 - 0.3 * j) * dx for j in range(k)] + [20.5 * dx] * 4
    x = np.array([[xv, 16.5 * dx, 0.0] for xv in xs])
    u = np.zeros((len(xs), 3))
    u[:k, 0] = 2.0                                   # gamma v = 2: v = 0.89 c outwards
    wt = np.full(len(xs), 1e-3)
    ids = np.arange(len(xs), dtype=np.int64)
    sim.set_particles(x, u, wt, ids)
    s0, steps = 2, 8
    sim.step(s0)
    stepwise = 0
    for _ in range(steps):
        stepwise += sim.num_particles()              # every electron alive now is pushed
        sim.step(1)
    ex = sim.exits()["step"]
    inside = ex[(ex >= s0) & (ex < s0 + steps)]
    assert len(inside) > 2 and len(np.unique(inside)) > 1   # exits spread over the window
    counted = float(sim.num_particles()) * steps + float(np.sum(inside - s0 + 1))
    assert counted == stepwise


def test_focus_window_of_the_benchmark_workloads():
    """The timed window is centred on the step at which the pulse peak crosses the focus
    and kept inside the run: 3D RP steps 457-477, 2D LP 752-772 (the windows the profiles
    and the measurements name)."""
    import bench
    import synth

    w3, w2 = synth.c3_3d_rp(), synth.c2_2d_lp()
    assert bench.window_start(w3, 20, "focus") == 457
    assert bench.window_start(w2, 20, "focus") == 752
    assert bench.window_start(w3, 20, "start") == 0
    assert bench.window_start(w3, w3.steps, "focus") == 0          # K covers the run
    k = w3.steps - 10                                                # kept inside the run
    assert bench.window_start(w3, k, "focus") + k <= w3.steps
