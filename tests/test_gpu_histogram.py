"""The energy-angle histogram diagnostic (Sec. 4's weighted spectra) against a numpy
histogram of the same run's electrons (in the box and at exit), and against the oracle's
electrons for an FP64 run."""
import math

import numpy as np
import pytest

import synth
from _support import small_2d

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


def numpy_hist(parts, exits, n_e, e_max, n_a):
    u = np.concatenate([parts["u"], exits["u"]])
    w = np.concatenate([parts["w"], exits["w"]])
    e = np.sqrt(1.0 + (u * u).sum(axis=1)) - 1.0
    ang = np.arctan2(np.hypot(u[:, 1], u[:, 2]), u[:, 0])
    h, _, _ = np.histogram2d(e, ang, bins=[n_e, n_a], range=[[0.0, e_max], [0.0, math.pi]], weights=w)
    return h


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_histogram_matches_the_electrons(P, orc, prec):
    w = small_2d(precision=synth.FP32 if prec == "fp32" else synth.FP64, steps=120)
    sim = P.Simulation(P.config_from(w))
    sim.step(120)
    n_e, e_max, n_a = 40, 40.0, 18
    got = sim.histogram(n_e, e_max, n_a)
    want = numpy_hist(sim.particles(), sim.exits(), n_e, e_max, n_a)
    total = want.sum()
    assert total > 0 and (want > 0).sum() > 20
    # bin edges: an electron exactly on an edge may fall either side in the two codes
    assert np.abs(got - want).sum() <= 2 * w.n_e / w.ppc + 1e-12 * total
    if prec == "fp64":
        ref = orc.Sim(orc.config_from(w))
        ref.step(120)
        want_ref = numpy_hist(ref.particles(), ref.exits(), n_e, e_max, n_a)
        assert np.abs(got - want_ref).sum() <= 2 * w.n_e / w.ppc + 1e-9 * total
