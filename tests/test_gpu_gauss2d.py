"""The 2D paraxial Gaussian beam (Sec. 3.2) and the super-Gaussian slab profile (Sec. 3.1)
on the GPU against the oracle: the incident field point by point, the seeded weights, and
a short run with both."""
import math

import numpy as np
import pytest

import synth
from _support import field_errors, momentum_error, small_2d

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    pic.load()
    return pic


def gauss_small(prec):
    """The Sec. 3.2 set-up shrunk to 96 x 80 cells at lambda/32: Gaussian beam (w0 = lambda,
    E0 = 4.86, FWHM_T = 2 pi) focused at the box centre into a super-Gaussian slab (p = 12)
    of peak density 0.31 n_c."""
    w = small_2d(precision=prec)
    dx = w.dx
    return w.with_(name="2d_gauss_small", beam=synth.BEAM_GAUSS2D, w0=TWO_PI, a0=4.86, duration=TWO_PI,
                   n_e=0.31, ppc=4, profile=synth.PROFILE_SUPERGAUSS, prof_order=12, prof_x0=48 * dx,
                   prof_fwhm=40 * dx, prof_cut=20 * dx, phi0=0.4)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gaussian_beam_point_parity(P, orc, prec):
    w = gauss_small(synth.FP32 if prec == "fp32" else synth.FP64)
    sim = P.Simulation(P.config_from(w))
    cfg = orc.config_from(w)
    rng = np.random.default_rng(8)
    pts = np.array([[rng.uniform(4, 92) * w.dx, rng.uniform(4, 76) * w.dx, 0.0,
                     w.t_focus + rng.uniform(-25, 25)] for _ in range(1500)])
    got = sim.eval_incident(pts)
    want = np.array([np.concatenate(orc.incident(cfg, p[:3], p[3])) for p in pts])
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < (5e-6 if prec == "fp32" else 1e-11), err


def test_profile_weights_match_the_oracle(P, orc):
    w = gauss_small(synth.FP64)
    pg = P.Simulation(P.config_from(w)).particles()
    pr = orc.Sim(orc.config_from(w)).particles()
    ia, ib = np.argsort(pg["id"]), np.argsort(pr["id"])
    np.testing.assert_array_equal(pg["id"][ia], pr["id"][ib])
    assert np.abs(pg["w"][ia] - pr["w"][ib]).max() <= 1e-15 * pr["w"].max()
    assert (pr["w"] == 0).any() and pr["w"].max() > 0.99 * w.n_e / w.ppc


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gaussian_beam_in_super_gaussian_slab(P, orc, prec):
    w = gauss_small(synth.FP32 if prec == "fp32" else synth.FP64)
    tol = 1e-5 if prec == "fp32" else 1e-9
    sim = P.Simulation(P.config_from(w))
    ref = orc.Sim(orc.config_from(w))
    for _ in range(4):
        sim.step(10)
        ref.step(10)
        err, n = momentum_error(sim.particles(), ref.particles(), w.a0)
        assert n == len(ref.particles()["id"])
        assert err < tol, err
    assert np.abs(ref.particles()["u"]).max() > 0.5
    assert field_errors(sim.fields(), ref.fields())[:6].max() < tol
