"""Vay and Higuera-Cary momentum updates on the GPU (Sec. 2 cites them beside Boris): the
2D LP run against the oracle with each scheme, and the force-free E x B drift of a
relativistic electron, which both schemes keep and Boris does not."""
import math

import numpy as np
import pytest

import synth
from _support import field_errors, momentum_error, small_2d

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


@pytest.mark.parametrize("pusher", [1, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_2d_lp_parity_with_each_pusher(P, orc, pusher, prec):
    w = small_2d(precision=synth.FP32 if prec == "fp32" else synth.FP64).with_(pusher=pusher)
    tol = 1e-5 if prec == "fp32" else 1e-9
    sim = P.Simulation(P.config_from(w))
    ref = orc.Sim(orc.config_from(w))
    for _ in range(3):
        sim.step(10)
        ref.step(10)
        err, n = momentum_error(sim.particles(), ref.particles(), w.a0)
        assert n == len(ref.particles()["id"])
        assert err < tol, err
    assert field_errors(sim.fields(), ref.fields())[:6].max() < tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_force_free_drift_on_the_gpu(P, prec):
    vd = np.array([0.9, 0.0, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    E = -np.cross(vd, B)
    u0 = vd / math.sqrt(1 - vd @ vd)
    dx = 0.2
    w = synth.Workload(name="exb", dim=1, n=(4096, 1, 1), dx=dx, steps=200, beam=synth.BEAM_UNIFORM, a0=0.0,
                       duration=0.0, slab_lo=(0, 0, 0), slab_hi=(0, 1, 1), n_e=0.0, ppc=0, seed=1,
                       e_unif=tuple(E), b_unif=tuple(B), cfl=0.5,
                       precision=synth.FP32 if prec == "fp32" else synth.FP64)
    err = []
    for pusher in (0, 1, 2):
        sim = P.Simulation(P.config_from(w.with_(pusher=pusher), max_particles=1))
        sim.set_particles([[100 * dx, 0, 0]], [u0], [0.0], [0])
        sim.step(200)
        err.append(np.abs(sim.particles()["u"][0] - u0).max() / np.abs(u0).max())
        sim.close()
    tol = 2e-6 if prec == "fp32" else 1e-13
    assert err[1] < tol and err[2] < tol, err
    assert err[0] > 1e-3, err
