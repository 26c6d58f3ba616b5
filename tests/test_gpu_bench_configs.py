"""The CUDA path against the FP64 oracle at the particle densities, tiles and work-item
sizes the benchmark runs (the 2D LP and 3D RP workloads of Secs. 4.2-4.3's kind, boxes
shrunk eightfold per axis with the cell size, pulse, density and particles per cell kept):

  * 2D LP, 128 x 128 cells, 8 electrons per cell (32 768; the push's lane stride is 8),
    tiles of 32 x 16 cells, work items of 1024 particles;
  * 3D RP, 64 x 32 x 32 cells, 4 electrons per cell (32 768; lane stride 4), tiles of
    16 x 8 x 4 cells (the 16-cell-row bank layout of the push), work items of 1024.

First 50 steps (the Sec. 2 cycle from t = 0, the pulse entering the slab), checked every
10 steps in FP32 and FP64, element by element: every electron's momentum and position by
id, every grid point of all nine components (E, B and the current J of the last step),
the energies.  Bars (tests/_support.py): FP32 |p_gpu - p_ref| / max(|p_ref|, a0) <= 1e-5, or
the accumulated impulse error of the FP32 incident field once that is larger; per particle
against max(|p_ref|, 1e-2 a0) within 1e-5 plus that impulse error; per component
max |F_gpu - F_ref| <= 1e-5 max |F_ref| (3D: 1e-4, the fields following the electrons' FP32
trajectories in the a0 = 20 focus); FP64 1e-9 for all, the momenta against
max(|p_ref|, 1e-3 a0).  The tightest reading of the momentum metric (floor 1e-3 a0) is
printed beside them.

Whole runs at the same configurations (1500 and 1200 steps, the workloads' own lengths):
energies every 50 steps to 1e-3 and the Kolmogorov-Smirnov distance of the electron energy
and angle distributions to 1e-3 (FP32), 1e-9 / one electron's weight (FP64).
"""
import numpy as np
import pytest

import synth
from _support import (POSITION_BAR_FP32, field_bar, field_errors, momentum_bar, momentum_error, momentum_report,
                      position_error, tight_bar)
from test_gpu_longrun import energy_angle, ks_distance

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


def bench_2d(precision):
    return synth.scaled(synth.c2_2d_lp(), 8).with_(precision=precision)


def bench_3d(precision):
    return synth.scaled(synth.c3_3d_rp(), 8).with_(precision=precision)


CASES = {"2d_lp_div8": (bench_2d, (32, 16)), "3d_rp_div8": (bench_3d, (16, 8, 4))}
CHUNK = 1024


def _sim(P, w, tile):
    return P.Simulation(P.config_from(w, tile=tile, chunk=CHUNK))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_first_50_steps_at_the_benchmark_configuration(P, orc, case, prec):
    make, tile = CASES[case]
    w = make(synth.FP32 if prec == "fp32" else synth.FP64)
    assert w.n_particles == 32768
    tol = 1e-5 if prec == "fp32" else 1e-9
    sim = _sim(P, w, tile)
    prm = sim.info().params
    assert tuple(prm.tile[: w.dim]) == tile and prm.chunk == CHUNK
    ref = orc.Sim(orc.config_from(w))
    worst = {"p": np.zeros(3), "x": 0.0, "F": np.zeros(9)}
    for done in range(10, 51, 10):
        sim.step(10)
        ref.step(10)
        pg, pr = sim.particles(), ref.particles()
        np.testing.assert_array_equal(np.sort(pg["id"]), np.sort(pr["id"]))   # same electrons left
        rep = momentum_report(pg, pr, w.a0)
        err, n = momentum_error(pg, pr, w.a0, floor=1.0 if prec == "fp32" else 1e-3)
        assert n == len(pr["id"])
        worst["p"] = np.maximum(worst["p"], [rep[1.0], rep[1e-2], rep[1e-3]])
        worst["x"] = max(worst["x"], position_error(pg, pr, w.dx))
        fe = field_errors(sim.fields(), ref.fields())
        worst["F"] = np.maximum(worst["F"], fe)
        assert err < (momentum_bar(done, w.dt) if prec == "fp32" else tol), (done, err)
        if prec == "fp32":
            assert rep[1e-2] < tight_bar(done, w.dt), (done, rep[1e-2], tight_bar(done, w.dt))
        assert worst["x"] < (POSITION_BAR_FP32 if prec == "fp32" else tol), (done, worst["x"])
        assert fe.max() < field_bar(w.dim, done, prec), (done, fe)
    assert max(np.abs(pr["u"]).max() for pr in [ref.particles()]) > 1.0      # relativistic by step 50
    assert np.abs(ref.fields()[6:]).max() > 0                                # current deposited
    eg, er = sim.energies(), ref.energies()
    for k in (0, 1, 2):
        assert abs(eg[k] / er[k] - 1) < field_bar(w.dim, 50, prec), (k, eg[k], er[k])
    print(f"{case} {prec}: momentum floor a0 {worst['p'][0]:.2e}, floor 1e-2 a0 {worst['p'][1]:.2e} "
          f"(bar {tight_bar(50, w.dt):.1e}), floor 1e-3 a0 {worst['p'][2]:.2e}; "
          f"position {worst['x']:.2e} cells, fields E,B {worst['F'][:6].max():.2e}, J {worst['F'][6:].max():.2e}")


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_whole_run_at_the_benchmark_configuration(P, orc, case, prec):
    make, tile = CASES[case]
    w = make(synth.FP32 if prec == "fp32" else synth.FP64)
    tol = 1e-3 if prec == "fp32" else 1e-9
    sim = _sim(P, w, tile)
    ref = orc.Sim(orc.config_from(w))
    worst = {"em": 0.0, "kin": 0.0}
    for done in range(50, w.steps + 1, 50):
        sim.step(done - sim.info().step)
        ref.step(done - ref.step_index)
        eg, er = sim.energies(), ref.energies()
        for name, g, r in (("em", eg[0], er[0]), ("kin", eg[2] + eg[3], er[2] + er[3])):
            assert r > 0
            worst[name] = max(worst[name], abs(g - r) / r)
    rest = w.steps - sim.info().step
    if rest:
        sim.step(rest)
        ref.step(rest)
    assert sim.info().step == w.steps
    eg_, ag, wg, ig = energy_angle(sim.particles(), sim.exits())
    er_, ar, wr, ir = energy_angle(ref.particles(), ref.exits())
    assert len(eg_) == len(er_) == w.n_particles
    np.testing.assert_array_equal(ig, ir)
    assert er_.max() > 1.0
    d_e = ks_distance(eg_, wg, er_, wr)
    d_a = ks_distance(ag, wg, ar, wr)
    print(f"{case} {prec} {w.steps} steps: energy {worst}, KS energy {d_e:.2e}, KS angle {d_a:.2e}")
    assert worst["em"] < tol and worst["kin"] < tol, worst
    assert d_e < 1e-3 and d_a < 1e-3, (d_e, d_a)
    if prec == "fp64":
        de = float(np.abs(eg_ - er_).max() / er_.max())
        print(f"  per-electron energy difference {de:.2e} of the largest")
        assert de < 1e-9
