"""Pins of the oracle's incident fields (Sec. 4.1, Eqs. components, phasor, poisson,
poisson_dstr) against quantities computed independently of it:

* mpmath (40 digits) numerical second derivatives of Psi (Eq. phasor) pushed through the
  component rules of Eq. (components) for LP and through the Hertz-vector rules for RP;
  this also covers the axis (the paper's x/r form is 0/0 there) and points next to the
  ring R~ = 0 where the printed terms cancel (the oracle switches to its series there);
* the vacuum Maxwell equations by central differences;
* propagation toward +z and a paraxial focal spot of 1/e^2 radius w0;
* the on-axis focal envelope FWHM and peak re-measured from mpmath Psi.
"""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

A, S, PSI0, PHI0 = 20.715, 27.13, 1.0, 0.3


def _psi(a, s, psi0, phi0):
    def f(t):
        return mp.exp(1j * phi0) * (1 - 1j * t / s) ** (-(s + 1))

    def Psi(x, y, z, t):
        R = mp.sqrt(x * x + y * y + (z + 1j * a) ** 2)
        return psi0 / R * (f(t + R + 1j * a) - f(t - R + 1j * a))

    return Psi


def _mp_fields(beam, a, s, psi0, phi0, p):
    mp.mp.dps = 40
    Psi = _psi(a, s, psi0, phi0)
    cache = {}

    def d2(i, j):
        key = tuple(sorted((i, j)))
        if key not in cache:
            o = [0, 0, 0, 0]
            o[i] += 1
            o[j] += 1
            cache[key] = mp.diff(Psi, p, tuple(o))
        return cache[key]

    X, Y, Z, T = 0, 1, 2, 3
    if beam == "lp":   # Eq. (components), c = 1
        v = [d2(X, X) - d2(T, T) + d2(T, Z), d2(X, Y), d2(Z, X) - d2(T, X),
             d2(X, Y), d2(Y, Y) - d2(T, T) + d2(T, Z), d2(Z, Y) - d2(T, Y)]
    else:              # electric Hertz vector Psi z^
        v = [d2(X, Z), d2(Y, Z), d2(Z, Z) - d2(T, T), d2(T, Y), -d2(T, X), mp.mpf(0)]
    return np.array([float(mp.re(x)) for x in v])


def _orc_fields(orc, beam, a, s, psi0, phi0, p, branch=0):
    b = orc.BEAM_LP if beam == "lp" else orc.BEAM_RP
    E, B = orc.beam_field(b, a, s, psi0, phi0, *p, branch=branch)
    return np.concatenate([E, B])


# (X, Y, Z, tau) in the beam frame; R = |R~|/a noted where relevant
POINTS = [
    (3.1, -2.2, 5.3, 4.0),            # generic, near focus
    (0.0, 0.0, 1.5, 0.5),             # on the axis
    (1e-3, 0.0, -4.0, -3.5),          # next to the axis
    (A * (1 + 1e-4), 0.0, 2e-3, 1.0), # |R| ~ 1e-2: series branch
    (A * 0.99, 0.5, 0.3, 0.2),        # |R| ~ 0.14: series branch
    (A * 1.03, 1.0, 2.0, -1.0),       # |R| ~ 0.3: closed form near the ring
    (7.0, 4.0, -30.0, -29.0),         # behind focus, on the pulse
    (5.0, -6.0, 60.0, 61.0),          # ahead of focus, on the pulse
    (2.0, 1.0, 3.0, 45.0),            # far from the pulse in time
]


@pytest.mark.parametrize("beam", ["lp", "rp"])
@pytest.mark.parametrize("p", POINTS)
def test_beam_matches_mpmath_derivatives_of_psi(orc, beam, p):
    got = _orc_fields(orc, beam, A, S, PSI0, PHI0, p)
    want = _mp_fields(beam, A, S, PSI0, PHI0, p)
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() <= 1e-11 * scale, (got, want)


@pytest.mark.parametrize("beam", ["lp", "rp"])
def test_tight_focus_other_parameters(orc, beam):
    # w0 = 0.5 lambda (a = 5.85), short pulse, nonzero phase, three points
    a, s, psi0, phi0 = 5.85, 12.0, 3.0, -1.1
    for p in [(1.0, 2.0, -0.5, 0.7), (a * 1.01, 0.0, 0.05, 0.0), (0.0, 0.0, -10.0, -9.0)]:
        got = _orc_fields(orc, beam, a, s, psi0, phi0, p)
        want = _mp_fields(beam, a, s, psi0, phi0, p)
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("beam", ["lp", "rp"])
def test_series_and_closed_form_agree_where_both_hold(orc, beam):
    rng = np.random.default_rng(7)
    for _ in range(40):
        # |R| in [0.2, 0.6] around the ring rho = 1, zeta = 0
        rad = rng.uniform(0.2, 0.6) ** 2 / 2
        ang = rng.uniform(0, 2 * math.pi)
        rho = math.sqrt(max(1 + rad * math.cos(ang), 0.0))
        zeta = rad * math.sin(ang)
        phi = rng.uniform(0, 2 * math.pi)
        p = (A * rho * math.cos(phi), A * rho * math.sin(phi), A * zeta, rng.uniform(-20, 20))
        c = _orc_fields(orc, beam, A, S, PSI0, PHI0, p, branch=1)
        s = _orc_fields(orc, beam, A, S, PSI0, PHI0, p, branch=2)
        assert np.abs(c - s).max() <= 1e-11 * max(np.abs(c).max(), 1e-300)


@pytest.mark.parametrize("beam", ["lp", "rp"])
def test_vacuum_maxwell_residual(orc, beam):
    """div E = div B = 0, d_t B = -curl E, d_t E = curl B (normalised units, c = 1)."""
    h = 1e-3
    rng = np.random.default_rng(3)
    b = orc.BEAM_LP if beam == "lp" else orc.BEAM_RP

    def F(q):
        E, B = orc.beam_field(b, 10.6, 27.0, 1.0, 0.2, *q)
        return np.concatenate([E, B])

    for _ in range(6):
        p = np.array([rng.uniform(-8, 8), rng.uniform(-8, 8), rng.uniform(-8, 8), 0.0])
        p[3] = p[2] + rng.uniform(-4, 4)
        d = []
        for k in range(4):
            e = np.zeros(4)
            e[k] = h
            d.append((F(p + e) - F(p - e)) / (2 * h))
        dx, dy, dz, dt = d
        scale = np.abs(F(p)).max()
        Ex, Ey, Ez, Bx, By, Bz = range(6)
        res = [
            dx[Ex] + dy[Ey] + dz[Ez],
            dx[Bx] + dy[By] + dz[Bz],
            dt[Bx] + (dy[Ez] - dz[Ey]), dt[By] + (dz[Ex] - dx[Ez]), dt[Bz] + (dx[Ey] - dy[Ex]),
            dt[Ex] - (dy[Bz] - dz[By]), dt[Ey] - (dz[Bx] - dx[Bz]), dt[Ez] - (dx[By] - dy[Bx]),
        ]
        assert max(abs(r) for r in res) <= 2e-5 * scale


@pytest.mark.parametrize("beam", ["lp", "rp"])
def test_pulse_travels_toward_plus_z(orc, beam):
    b = orc.BEAM_LP if beam == "lp" else orc.BEAM_RP
    a = 10.6
    # Poynting flux S_z = Ex By - Ey Bx, time-averaged over a cycle at a point off focus
    for z in (-40.0, 40.0):
        x = 2.0 if beam == "rp" else 0.0
        sz = 0.0
        for t in np.linspace(z - 3.0, z + 3.0, 200):
            E, B = orc.beam_field(b, a, 27.0, 1.0, 0.0, x, 0.5, z, t)
            sz += E[0] * B[1] - E[1] * B[0]
        assert sz > 0


def test_lp_focal_spot_has_waist_w0(orc):
    """k^2 w0^2 = 2(sqrt(1+(ka)^2)-1): in the quasi-monochromatic limit (s large; the
    isodiffracting pulse focuses each frequency to a different spot) and the paraxial
    regime (w0 = 6 lambda), the focal-plane |E_x^c|^2 falls to e^-2 at r = w0."""
    w0 = 6 * 2 * math.pi
    a = orc.a_from_w0(w0)
    E0, _ = orc.beam_complex(orc.BEAM_LP, a, 5000.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    for X, Y in ((w0, 0.0), (0.0, w0)):
        Ew, _ = orc.beam_complex(orc.BEAM_LP, a, 5000.0, 1.0, 0.0, X, Y, 0.0, 0.0)
        ratio = abs(Ew[0]) ** 2 / abs(E0[0]) ** 2
        assert abs(ratio / math.exp(-2.0) - 1.0) < 0.02


@pytest.mark.parametrize("beam", ["lp", "rp"])
def test_pulse_parameters_remeasured_with_mpmath(orc, beam):
    """s from a field FWHM and Psi0 from a peak field, re-measured on mpmath's Psi."""
    b = orc.BEAM_LP if beam == "lp" else orc.BEAM_RP
    w0, dur, a0 = 2 * math.pi * 1.0, 11.781, 10.0
    a, s, psi0 = orc.derive_pulse(b, w0, dur, a0)
    assert abs(a - 20.715) < 1e-3                       # k^2 w0^2 = 2(sqrt(1+(ka)^2)-1) at w0 = lambda
    comp = 0 if beam == "lp" else 2

    def env(t):
        return abs(complex(_mp_complex_onaxis(beam, a, s, psi0, t)[comp]))

    tpk = 0.0
    for _ in range(3):  # refine the peak locally
        ts = np.linspace(tpk - 0.5, tpk + 0.5, 21)
        tpk = ts[int(np.argmax([env(t) for t in ts]))]
    peak = env(tpk)
    assert abs(peak / a0 - 1.0) < 2e-4
    half = 0.5 * peak

    def cross(direction):
        lo, hi = tpk, tpk + direction * 3 * dur
        for _ in range(40):
            m = 0.5 * (lo + hi)
            if env(m) > half:
                lo = m
            else:
                hi = m
        return 0.5 * (lo + hi)

    fwhm = cross(+1) - cross(-1)
    assert abs(fwhm / dur - 1.0) < 1e-6


def _mp_complex_onaxis(beam, a, s, psi0, t):
    mp.mp.dps = 30
    Psi = _psi(a, s, psi0, 0.0)
    p = (0, 0, 0, t)

    def d2(i, j):
        o = [0, 0, 0, 0]
        o[i] += 1
        o[j] += 1
        return mp.diff(Psi, p, tuple(o))

    X, Y, Z, T = 0, 1, 2, 3
    if beam == "lp":
        return [d2(X, X) - d2(T, T) + d2(T, Z), 0, 0]
    return [0, 0, d2(Z, Z) - d2(T, T)]
