"""Pins of the oracle's 2D paraxial Gaussian beam (Sec. 3.2, Eq. gauss2D) and of the
super-Gaussian slab profile (Sec. 3.1) against what the mathematics fixes:

* the complex amplitude A(X, Z) of E_y = Re[A e^{i(Z - t)}] solves the paraxial wave
  equation 2i dA/dZ + d2A/dX2 = 0 (the 2D beam is an exact solution of it): this fixes the
  amplitude law sqrt(w0/w), the waist w(Z), the curvature 1/R(Z) and the Gouy phase eta(Z);
* the cycle-averaged flux int |A|^2 dX is the same through every plane Z (2D energy flux);
* div E = d E_x/dx + d E_y/dy vanishes to first order in 1/(k w0) at the focus and away from
  it: the residual falls 4-fold when w0 doubles (with the printed factor X/w instead of
  X/w^2, or without the curvature term of E_z away from the focus, it would not fall);
* the wide-beam limit is the Gaussian-envelope plane wave of Sec. 3.1;
* slab weights follow n0 f(x): their sum matches n0 times the closed-form integral
  F Gamma(1 + 1/p) / (ln 2)^(1/p) of the super-Gaussian.
"""
import math

import numpy as np
import pytest


def cfg(orc, **kw):
    base = dict(dim=2, n=(64, 64, 1), dx=0.2, dt=0.1, beam=orc.BEAM_GAUSS2D, a0=1.3, duration=1e9,
                t_focus=0.0, focus=(0.0, 0.0, 0.0), w0=20.0, phi0=0.3)
    base.update(kw)
    return orc.make_config(**base)


def Ey(orc, c, X, Z, t):
    return orc.incident(c, [Z, X, 0.0], t)[0][1]


def amplitude(orc, c, X, Z, t=7.0):
    """A with E_y = Re[A e^{i(Z - t)}]: E_y(t) + i E_y(t + pi/2) = A e^{i(Z - t)}."""
    z = Ey(orc, c, X, Z, t) + 1j * Ey(orc, c, X, Z, t + math.pi / 2)
    return z * np.exp(-1j * (Z - t))


@pytest.mark.parametrize("Z", [0.0, 37.0, 200.0, 700.0])
def test_amplitude_solves_the_paraxial_wave_equation(orc, Z):
    c = cfg(orc, w0=20.0)
    h = 0.02
    for X in (0.0, 5.0, 13.0, 24.0):
        A = lambda x, z: amplitude(orc, c, x, z)
        dZ = (A(X, Z + h) - A(X, Z - h)) / (2 * h)
        dXX = (A(X + h, Z) - 2 * A(X, Z) + A(X - h, Z)) / (h * h)
        scale = abs(dXX) + abs(A(X, Z)) / c.w0 ** 2
        assert abs(2j * dZ + dXX) < 1e-4 * scale, (X, Z)


def test_flux_is_the_same_through_every_plane(orc):
    c = cfg(orc, w0=15.0)
    zR = 0.5 * c.w0 ** 2
    X = np.linspace(-8 * c.w0, 8 * c.w0, 4001)
    want = c.a0 ** 2 * c.w0 * math.sqrt(math.pi / 2)
    for Z in (0.0, 0.5 * zR, zR, 3 * zR):
        f = np.array([abs(amplitude(orc, c, x, Z)) ** 2 for x in X])
        assert abs(np.trapezoid(f, X) / want - 1) < 1e-6, Z


def test_divergence_vanishes_to_first_order_in_the_waist(orc):
    res = []
    for w0 in (10.0, 20.0, 40.0):
        c = cfg(orc, w0=w0, duration=1e9)
        h = 1e-3
        worst = scale = 0.0
        for X in np.linspace(-1.5 * w0, 1.5 * w0, 13):
            for Z in (0.0, 0.3 * w0 ** 2):
                f = lambda x, z: orc.incident(c, [z, x, 0.0], 3.0)[0]
                div = (f(X, Z + h)[0] - f(X, Z - h)[0]) / (2 * h) + (f(X + h, Z)[1] - f(X - h, Z)[1]) / (2 * h)
                worst = max(worst, abs(div))
                scale = max(scale, abs((f(X + h, Z)[1] - f(X - h, Z)[1]) / (2 * h)))
        res.append(worst / scale)
    assert res[2] < 2e-3
    assert 3.0 < res[0] / res[1] < 5.0 and 3.0 < res[1] / res[2] < 5.0


def test_wide_beam_is_the_gaussian_plane_wave(orc):
    t0, T = 3.0, 6.0
    g = cfg(orc, w0=1e4, duration=T, t_focus=t0, phi0=math.pi / 2 + t0, focus=(0.0, 0.0, 0.0))
    p = orc.make_config(dim=2, n=(64, 64, 1), dx=0.2, dt=0.1, beam=orc.BEAM_PLANE, envelope=orc.ENV_GAUSS,
                        a0=g.a0, duration=T, t_focus=t0, phi0=0.0, focus=(0.0, 0.0, 0.0))
    rng = np.random.default_rng(3)
    for _ in range(200):
        Z, X, t = rng.uniform(-10, 10), rng.uniform(-10, 10), rng.uniform(-5, 12)
        Eg, Bg = orc.incident(g, [Z, X, 0.0], t)
        Ep, Bp = orc.incident(p, [Z, X, 0.0], t)
        assert np.abs(Eg - Ep).max() < 1e-5 * g.a0 and np.abs(Bg - Bp).max() < 1e-5 * g.a0


def test_super_gaussian_slab_weights(orc):
    n, dx, ppc, n0, p = 4096, 0.1, 64, 0.31, 12
    x0, F, cut = 200.0, 160.0, 60.0
    c = orc.make_config(dim=1, n=(n, 1, 1), dx=dx, dt=0.09, beam=orc.BEAM_NONE, slab_lo=(10, 0, 0),
                        slab_hi=(n - 10, 1, 1), n_e=n0, ppc=ppc, seed=5, profile=orc.PROFILE_SUPERGAUSS,
                        prof_order=p, prof_x0=x0, prof_fwhm=F, prof_cut=cut)
    sim = orc.Sim(c)
    parts = sim.particles()
    w, x = parts["w"], parts["x"][:, 0]
    assert np.all(w[x <= cut] == 0.0)
    integral = F * math.gamma(1 + 1 / p) / math.log(2) ** (1 / p)
    assert abs(w.sum() * dx / (n0 * integral) - 1) < 2e-3
