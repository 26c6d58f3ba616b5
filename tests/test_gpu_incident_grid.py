"""Incident field evaluated on the Yee nodes and gathered (the prescribed-field route of
Smilei that the paper's runs used, Sec. 2 last paragraph) on the GPU: parity with the
oracle's run in the same mode (1D/2D/3D), and the accuracy of the route against the
per-particle evaluation of Sec. 2 (an O((k dx)^2) interpolation error)."""
import numpy as np
import pytest

import synth
from _support import field_errors, momentum_error, small_1d, small_2d, small_3d

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


CASES = {"1d": (small_1d, 300, 100), "2d": (small_2d, 30, 10), "3d": (small_3d, 20, 10)}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_parity_with_the_oracle_on_the_grid_route(P, orc, case, prec):
    make, steps, every = CASES[case]
    w = make().with_(incident_grid=1, precision=synth.FP32 if prec == "fp32" else synth.FP64)
    tol = 1e-5 if prec == "fp32" else 1e-9
    sim = P.Simulation(P.config_from(w))
    ref = orc.Sim(orc.config_from(w))
    for _ in range(steps // every):
        sim.step(every)
        ref.step(every)
        err, n = momentum_error(sim.particles(), ref.particles(), w.a0)
        assert n == len(ref.particles()["id"])
        assert err < tol, err
    assert field_errors(sim.fields(), ref.fields())[:6].max() < tol


def test_grid_route_against_the_particle_route(P):
    """Same 2D LP run both ways (FP64): the momenta differ by the interpolation error of the
    incident field, a fraction of a percent of a0 at lambda/32."""
    w = small_2d(precision=synth.FP64)
    a = P.Simulation(P.config_from(w))
    b = P.Simulation(P.config_from(w.with_(incident_grid=1)))
    a.step(40)
    b.step(40)
    err, n = momentum_error(b.particles(), a.particles(), w.a0, floor=1.0)   # |du| / max(|u|, a0)
    print(f"grid vs particle route, 2D LP at lambda/32, 40 steps: max |du| / a0 = {err:.2e}")
    assert 1e-6 < err < 3e-2
