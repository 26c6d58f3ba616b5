"""Pins of the oracle's PIC step against what the physics and the mathematics fix:

* no plasma -> the scattered field stays exactly zero (Sec. 2: the incident field is a
  vacuum solution; only currents source the scattered field);
* one electron in the plane wave of Sec. 3.1 follows the closed-form trajectory
  p_y = A(xi), gamma - p_x = 1, with error O(dt^2);
* Boris rotation in a uniform B: exact angle 2 atan(Omega dt/2) per step;
* the Vay and Higuera-Cary pushers (Sec. 2 cites both besides Boris): exact in a pure E
  field, |u| kept in a pure B field, the force-free E x B drift of a relativistic
  electron kept to round-off (where Boris is off at O(dt^2) -- the property both were
  built for), gyration phase and plane-wave trajectory converging at second order;
* the incident field evaluated on the Yee nodes and gathered (the prescribed-field route):
  exact for a uniform field (the shapes sum to one), and the single-electron plane-wave
  trajectory converging at second order as the cell and the step shrink together;
* Gauss law div E - rho = 0 to round-off under Esirkepov deposition (2D and 3D, open
  and periodic);
* the Yee vacuum dispersion relation sin^2(w dt/2)/dt^2 = sum_d sin^2(k_d dx/2)/dx^2
  (order 2, Sec. 3.1) -- exact discrete solution;
* the cold-plasma Langmuir frequency w_p = sqrt(n_e) (Table tab:units);
* first-order Mur faces absorb a 1D pulse;
* the energy diagnostic: the EM energy of a sampled sin^2 pulse (scattered, and total with
  the incident field on the grid) equals its closed-form integral, the kinetic energy of a
  drifting plasma its integral, and a Langmuir oscillation trades one for the other at a
  constant sum;
* 1D total-field (boundary injection, case (i)) and scattered-field (case (ii)) runs
  agree and converge together (Sec. 3.1, Eqs. L2_t, L2_t_cross, Table tab:delta_E).
"""
import math

import numpy as np
import pytest

import synth


def cfg(orc, **kw):
    base = dict(dim=1, n=(64, 1, 1), dx=0.2, dt=0.19, field_bc=orc.BC_MUR, beam=orc.BEAM_NONE, ppc=0,
                remove_margin=3)
    base.update(kw)
    return orc.make_config(**base)


def test_splitmix64_reference_outputs(orc):
    # published first outputs of SplitMix64 seeded with 0 (Vigna's reference splitmix64.c)
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    k = np.arange(1000, dtype=np.uint64)
    ref = [orc.splitmix64(12345, int(i)) for i in k]
    assert [int(v) for v in synth.splitmix64(12345, k)] == ref


def test_seeded_slab_matches_generator(orc):
    w = synth.scaled(synth.c2_2d_lp(), 16, steps=1)
    sim = orc.Sim(orc.config_from(w))
    p = sim.particles()
    x, u, wt, ids = synth.slab_particles(w)
    assert len(ids) == w.n_particles == len(p["id"])
    np.testing.assert_array_equal(p["id"], ids)
    np.testing.assert_array_equal(p["x"], x)
    np.testing.assert_array_equal(p["w"], wt)


def test_no_plasma_scattered_field_stays_zero(orc):
    w = synth.scaled(synth.c2_2d_lp(), 16, steps=1).with_(ppc=0)
    sim = orc.Sim(orc.config_from(w))
    sim.step(30)
    assert np.all(sim.fields() == 0.0)


def _A_plane(xi, a0, T):
    """A(xi) = -int_0^xi E_y, E_y = a0 sin(xi - T) sin^2(pi xi/(2T)) on [0, 2T]."""
    xi = np.clip(xi, 0.0, 2 * T)
    k = math.pi / T
    c = math.cos(T)
    i1 = c - np.cos(xi - T)
    i2 = 0.5 * ((c - np.cos((1 + k) * xi - T)) / (1 + k) + (c - np.cos((1 - k) * xi - T)) / (1 - k))
    return -a0 * (0.5 * i1 - 0.5 * i2)


def _single_electron_error(orc, dt, a0=1.5, T=4 * math.pi, pusher=0):
    dx = 0.25
    n = 2400
    c = cfg(orc, n=(n, 1, 1), dx=dx, dt=dt, beam=orc.BEAM_PLANE, envelope=orc.ENV_SIN2, a0=a0, duration=T,
            focus=(0.0, 0.0, 0.0), pusher=pusher)
    sim = orc.Sim(c)
    x0 = 40.0
    sim.set_particles([[x0, 0, 0]], [[0, 0, 0]], [0.0], [0])
    nsteps = int((2 * T + 60.0) / dt)
    err = dev = 0.0
    for it in range(nsteps):
        x_old = sim.particles()["x"][0, 0]
        sim.step(1)
        p = sim.particles()
        x_new = p["x"][0, 0]
        u = p["u"][0]
        # u^{n+1/2} belongs to t^{n+1/2} and the midpoint of the move
        xi = (it + 0.5) * dt - 0.5 * (x_old + x_new)
        err = max(err, abs(u[1] - _A_plane(xi, a0, T)))
        dev = max(dev, abs(np.sqrt(1 + u @ u) - u[0] - 1.0))   # gamma - p_x = 1
    return err, u, dev


@pytest.mark.parametrize("pusher", [0, 1, 2])
def test_single_electron_in_plane_wave(orc, pusher):
    e1, u1, d1 = _single_electron_error(orc, 0.2, pusher=pusher)
    e2, u2, d2 = _single_electron_error(orc, 0.1, pusher=pusher)
    assert e2 < 2e-3
    assert 3.0 < e1 / e2 < 5.0            # second order in dt
    assert d2 < 1e-3 and 3.0 < d1 / d2 < 5.0   # the light-front invariant, to the same order
    assert abs(u2[1]) < 2e-3               # zero net A after the pulse: electron back at rest


def test_boris_rotation_in_uniform_B(orc):
    B0, dt = 0.7, 0.1
    c = cfg(orc, n=(64, 1, 1), dx=0.2, dt=dt, field_bc=orc.BC_PERIODIC, beam=orc.BEAM_UNIFORM,
            b_unif=(0.0, 0.0, B0))
    sim = orc.Sim(c)
    u0 = np.array([0.5, 0.2, 0.1])
    sim.set_particles([[6.0, 0, 0]], [u0], [0.0], [0])
    g = math.sqrt(1 + u0 @ u0)
    nst = 300
    sim.step(nst)
    u = sim.particles()["u"][0]
    phi = nst * 2 * math.atan(B0 * dt / (2 * g))   # electron: counter-clockwise about +z
    want = np.array([u0[0] * math.cos(phi) - u0[1] * math.sin(phi),
                     u0[0] * math.sin(phi) + u0[1] * math.cos(phi), u0[2]])
    assert np.abs(u - want).max() < 1e-12


def _one_electron(orc, pusher, u0, steps, dt=0.1, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0)):
    c = cfg(orc, n=(64, 1, 1), dx=0.2, dt=dt, field_bc=orc.BC_PERIODIC, beam=orc.BEAM_UNIFORM,
            e_unif=tuple(E), b_unif=tuple(B), pusher=pusher)
    sim = orc.Sim(c)
    sim.set_particles([[6.0, 0, 0]], [list(u0)], [0.0], [0])
    sim.step(steps)
    return sim.particles()["u"][0]


def test_incident_on_the_grid_is_exact_for_a_uniform_field(orc):
    E, B = (0.3, -0.2, 0.5), (0.1, 0.4, -0.7)
    u0 = [0.5, 0.2, 0.1]
    out = []
    for grid in (0, 1):
        c = cfg(orc, n=(64, 1, 1), dx=0.2, dt=0.1, field_bc=orc.BC_PERIODIC, beam=orc.BEAM_UNIFORM,
                e_unif=E, b_unif=B, incident_grid=grid)
        sim = orc.Sim(c)
        sim.set_particles([[6.3, 0, 0]], [u0], [0.0], [0])
        sim.step(50)
        out.append(sim.particles()["u"][0])
    assert np.abs(out[0] - out[1]).max() < 1e-13


def test_incident_on_the_grid_converges_at_second_order(orc):
    """Single electron in the sin^2 plane wave with the incident field on the nodes: the
    closed-form trajectory error falls 4-fold when dx and dt halve together."""
    a0, T = 1.5, 4 * math.pi
    errs = []
    for dx in (0.2, 0.1, 0.05):
        dt = 0.95 * dx
        n = int(round(600 / dx))
        c = cfg(orc, n=(n, 1, 1), dx=dx, dt=dt, beam=orc.BEAM_PLANE, envelope=orc.ENV_SIN2, a0=a0, duration=T,
                focus=(0.0, 0.0, 0.0), incident_grid=1)
        sim = orc.Sim(c)
        sim.set_particles([[40.0, 0, 0]], [[0, 0, 0]], [0.0], [0])
        err = 0.0
        for it in range(int((2 * T + 60.0) / dt)):
            x_old = sim.particles()["x"][0, 0]
            sim.step(1)
            p = sim.particles()
            xi = (it + 0.5) * dt - 0.5 * (x_old + p["x"][0, 0])
            err = max(err, abs(p["u"][0][1] - _A_plane(xi, a0, T)))
        errs.append(err)
    assert errs[2] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


@pytest.mark.parametrize("pusher", [0, 1, 2])
def test_pushers_pure_electric_kick_is_exact(orc, pusher):
    E = np.array([0.3, -0.2, 0.5])
    u0 = np.array([0.5, 0.2, 0.1])
    u = _one_electron(orc, pusher, u0, 1, dt=0.1, E=E)
    assert np.abs(u - (u0 - 0.1 * E)).max() < 1e-15          # q = -1: du = -dt E


@pytest.mark.parametrize("pusher", [0, 1, 2])
def test_pushers_keep_the_momentum_magnitude_in_pure_B(orc, pusher):
    u0 = np.array([0.5, 0.2, 0.1])
    u = _one_electron(orc, pusher, u0, 300, B=(0.0, 0.0, 0.7))
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-13
    assert abs(u[2] - u0[2]) < 1e-14                        # no change along B


def test_force_free_drift_is_kept_by_vay_and_higuera_cary(orc):
    """E = -v_d x B with |v_d| = 0.9: an electron moving at v_d feels no force.  Vay's and
    Higuera-Cary's schemes keep it (their design property); Boris turns it."""
    vd = np.array([0.9, 0.0, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    E = -np.cross(vd, B)
    u0 = vd / math.sqrt(1 - vd @ vd)
    err = [np.abs(_one_electron(orc, p, u0, 200, E=E, B=B) - u0).max() for p in (0, 1, 2)]
    assert err[1] < 1e-13 and err[2] < 1e-13
    assert err[0] > 1e-3


@pytest.mark.parametrize("pusher", [0, 1, 2])
def test_gyration_phase_converges_at_second_order(orc, pusher):
    """Electron in a uniform B: after time T the momentum has turned by Omega T, Omega = B/gamma
    (counter-clockwise about +B); the phase error falls 4-fold per halving of dt."""
    B0, T = 0.7, 30.0
    u0 = np.array([0.8, 0.0, 0.3])
    g = math.sqrt(1 + u0 @ u0)
    phi = B0 / g * T
    want = np.array([u0[0] * math.cos(phi), u0[0] * math.sin(phi), u0[2]])
    errs = []
    for dt in (0.2, 0.1, 0.05):
        u = _one_electron(orc, pusher, u0, int(round(T / dt)), dt=dt, B=(0.0, 0.0, B0))
        errs.append(np.abs(u - want).max())
    assert errs[2] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("dim,bc", [(2, "mur"), (2, "periodic"), (3, "mur"), (1, "mur")])
def test_gauss_law_holds_to_roundoff(orc, dim, bc):
    dx = 2 * math.pi / 16
    if dim == 1:
        n, lo, hi, steps = (96, 1, 1), (30, 0, 0), (66, 1, 1), 60
    elif dim == 2:
        n, lo, hi, steps = (48, 40, 1), (14, 12, 0), (34, 28, 1), 40
    else:
        n, lo, hi, steps = (24, 20, 20), (7, 6, 6), (17, 14, 14), 12
    focus = tuple(n[d] * dx / 2 if d < dim else 0.0 for d in range(3))
    beam = orc.BEAM_LP if dim >= 2 else orc.BEAM_PLANE
    a = orc.a_from_w0(0.7 * 2 * math.pi)
    c = orc.make_config(dim=dim, n=n, dx=dx, dt=0.95 * dx / math.sqrt(dim),
                        field_bc=orc.BC_PERIODIC if bc == "periodic" else orc.BC_MUR,
                        beam=beam, a0=8.0, duration=8.0, envelope=orc.ENV_GAUSS, t_focus=2.0,
                        focus=focus if dim >= 2 else (-10.0, 0, 0),
                        a=a, s=20.0, psi0=1.0, slab_lo=lo, slab_hi=hi, n_e=0.2, ppc=3, seed=11,
                        remove_margin=3)
    sim = orc.Sim(c)
    sim.step(steps)
    p = sim.particles()
    assert len(p["id"]) == c.ppc * np.prod([hi[d] - lo[d] for d in range(dim)])    # nobody left
    assert np.abs(p["u"]).max() > 1e-2                                               # fields did work
    rho_scale = 0.2
    assert sim.gauss_residual() < 1e-12 * rho_scale * 1e3


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_yee_vacuum_dispersion_exact(orc, dim):
    dx, dt = 0.3, 0.3 * 0.9 / math.sqrt(dim)
    n = {1: (40, 1, 1), 2: (20, 16, 1), 3: (12, 10, 8)}[dim]
    c = cfg(orc, dim=dim, n=n, dx=dx, dt=dt, field_bc=orc.BC_PERIODIC)
    sim = orc.Sim(c)
    ext = sim.ext
    F = np.zeros((9, ext[2], ext[1], ext[0]))
    L = [n[d] * dx for d in range(3)]
    kv = [2 * math.pi / L[0] * 3, (2 * math.pi / L[1] * 2) if dim >= 2 else 0.0,
          (2 * math.pi / L[2]) if dim >= 3 else 0.0]
    # E_z mode varying in x, y (E_z is not staggered along x, y); divergence free
    ii, jj = np.meshgrid(np.arange(ext[0]), np.arange(ext[1]), indexing="xy")
    mode = np.cos(kv[0] * ii * dx + kv[1] * jj * dx)
    F[2] = mode[None, :, :]
    if dim == 3:
        # plus an E_x mode varying in y, z (staggered only along x)
        kk = np.arange(ext[2])[:, None, None]
        F[0] = np.cos(kv[1] * jj[None] * dx + kv[2] * kk * dx)
    sim.set_fields(F)
    lam_z = sum(math.sin(k * dx / 2) ** 2 for k in kv[:2]) / dx ** 2
    th_z = 2 * math.asin(dt * math.sqrt(lam_z))
    lam_x = sum(math.sin(k * dx / 2) ** 2 for k in kv[1:]) / dx ** 2
    th_x = 2 * math.asin(dt * math.sqrt(lam_x))
    for m in (1, 7, 100, 333):
        sim.step(m - sim.step_index)
        G = sim.fields()
        nx, ny, nz = n[0], (n[1] if dim >= 2 else 1), (n[2] if dim >= 3 else 1)   # periodic: n points per axis
        got = G[2][:nz, :ny, :nx]
        want = math.cos(m * th_z) * F[2][:nz, :ny, :nx]
        assert np.abs(got - want).max() < 1e-11
        if dim == 3:
            got = G[0][:nz, :ny, :nx]
            want = math.cos(m * th_x) * F[0][:nz, :ny, :nx]
            assert np.abs(got - want).max() < 1e-11


def test_langmuir_frequency(orc):
    """Cold 1D plasma with a small velocity perturbation oscillates at w_p = sqrt(n_e)."""
    N, dx, dt, ne, ppc = 256, 0.1, 0.095, 0.01, 8
    c = cfg(orc, n=(N, 1, 1), dx=dx, dt=dt, field_bc=orc.BC_PERIODIC)
    sim = orc.Sim(c)
    npart = N * ppc
    x = (np.arange(npart) + 0.5) * (dx / ppc)
    k = 2 * math.pi / (N * dx)
    X = np.zeros((npart, 3)); X[:, 0] = x
    U = np.zeros((npart, 3)); U[:, 0] = 1e-4 * np.sin(k * x)
    sim.set_particles(X, U, np.full(npart, ne / ppc), np.arange(npart))
    i_probe = int(round((N * dx / 4) / dx))     # E_x ~ cos(k x) sin(w t): probe near x = 0
    i_probe = 0
    sig = []
    for _ in range(1400):
        sim.step(1)
        sig.append(sim.fields()[0, 0, 0, i_probe])
    sig = np.array(sig)
    t = (np.arange(len(sig)) + 1) * dt
    zc = []
    for m in range(1, len(sig)):
        if sig[m - 1] == 0.0:
            continue
        if np.sign(sig[m - 1]) != np.sign(sig[m]):
            zc.append(t[m - 1] + dt * sig[m - 1] / (sig[m - 1] - sig[m]))
    half_periods = np.diff(zc)
    w = math.pi / half_periods.mean()
    assert len(zc) >= 3
    assert abs(w / math.sqrt(ne) - 1.0) < 1e-3


def test_mur_faces_absorb_1d_pulses(orc):
    N, dx = 400, 2 * math.pi / 32
    c = cfg(orc, n=(N, 1, 1), dx=dx, dt=0.95 * dx)
    for sign in (+1, -1):   # right-moving (E_y = B_z) and left-moving (E_y = -B_z)
        sim = orc.Sim(c)
        ext = sim.ext
        F = np.zeros((9, 1, 1, ext[0]))
        x0, sig = N * dx / 2, 6.0
        xp = np.arange(ext[0]) * dx              # E_y at primal nodes
        xd = (np.arange(ext[0]) + 0.5) * dx      # B_z at dual nodes
        f = lambda x: np.exp(-((x - x0) / sig) ** 2) * np.sin(x - x0)
        F[1, 0, 0] = f(xp)
        F[5, 0, 0, :N] = sign * f(xd[:N])
        sim.set_fields(F)
        e0 = sim.energies()[0]
        sim.step(int(1.2 * (N * dx / 2 + 4 * sig) / c.dt))
        assert sim.energies()[0] < 1e-4 * e0


def _tf_sf_history(orc, dxc, tf):
    """1D run of Sec. 3.1's kind: Gaussian plane wave (t0 = 4 FWHM) into a 0.1 n_c slab;
    total-field (laser creator at x = 0) or scattered-field (analytic incident field)."""
    L, fwhm = 2 * math.pi * 14, 2 * math.pi
    n = int(round(L / dxc))
    dt = 0.95 * dxc
    slab = (int(round(2 * math.pi * 7 / dxc)), int(round(2 * math.pi * 10 / dxc)))
    c = orc.make_config(dim=1, n=(n, 1, 1), dx=dxc, dt=dt, field_bc=orc.BC_MUR, tf_mode=1 if tf else 0,
                        beam=orc.BEAM_PLANE, envelope=orc.ENV_GAUSS, a0=2.0, duration=fwhm,
                        t_focus=4 * fwhm, focus=(0.0, 0, 0), slab_lo=(slab[0], 0, 0), slab_hi=(slab[1], 1, 1),
                        n_e=0.1, ppc=16, seed=9, remove_margin=3)
    sim = orc.Sim(c)
    T = 2 * math.pi * 16
    nst = int(T / dt)
    hist = []
    for k in range(1, 9):
        sim.step(int(k * nst / 8) - sim.step_index)
        e = sim.energies()
        hist.append(((e[0] if tf else e[1]), e[2] + e[3]))
    return np.array(hist)


@pytest.mark.slow
def test_total_field_and_scattered_field_runs_agree(orc):
    crosses = []
    for dxc in (2 * math.pi / 32, 2 * math.pi / 64):
        h_tf = _tf_sf_history(orc, dxc, True)
        h_sf = _tf_sf_history(orc, dxc, False)
        norm = (h_sf[:, 0] + h_sf[:, 1]).max()
        d_em = np.mean(np.abs(h_tf[:, 0] - h_sf[:, 0])) / norm     # Eq. (L2_t_cross)
        d_kin = np.mean(np.abs(h_tf[:, 1] - h_sf[:, 1])) / norm
        crosses.append((d_em, d_kin))
        assert h_sf[:, 1].max() > 1e-3 * norm                      # the plasma took up energy
    (em1, k1), (em2, k2) = crosses
    assert em2 < 0.01 and k2 < 0.01            # within 1 % at dx = lambda/64
    assert em2 < em1 / 2.5                      # and converging with the cell size


# ---- the energy diagnostic (Sec. 3.1: total energies E_EM = int (E^2 + B^2)/2 dV and
# E_kin = int n (gamma - 1) dV in the units of Table tab:units, whose curves Eqs. L2_t and
# L2_t_cross compare) pinned against closed forms --------------------------------------
def _sin2_pulse_energy(a0, T):
    """int (E_y^2 + B_z^2)/2 dx of the sin^2 plane-wave pulse E_y = B_z = a0 sin(xi - T)
    sin^2(pi xi/(2T)) on [0, 2T], in closed form: with eta = xi - T the envelope is
    cos^4(pi eta/(2T)) = 3/8 + cos(pi eta/T)/2 + cos(2 pi eta/T)/8 and sin^2 = (1 - cos 2eta)/2."""
    def cc(a):   # int_{-T}^{T} cos(a eta) cos(2 eta) d eta
        return math.sin(2 * T) if a == 0 else (math.sin((a - 2) * T) / (a - 2) + math.sin((a + 2) * T) / (a + 2))
    env4 = 0.75 * T                                   # int cos^4
    cross = 0.375 * cc(0.0) + 0.5 * cc(math.pi / T) + 0.125 * cc(2 * math.pi / T)
    return a0 * a0 * 0.5 * (env4 - cross)


@pytest.mark.parametrize("dim", [1, 2])
def test_field_energy_of_a_sampled_pulse_is_its_integral(orc, dim):
    """A plane-wave pulse written onto the grid (E_y at its nodes, B_z half a cell further
    along x, both at the same time): the EM energy is the closed-form integral times the
    transverse length (a dropped 1/2, cell volume or component would fail), and the Yee
    update in vacuum keeps it."""
    a0, T, dxc = 1.7, 23.546, 2 * math.pi / 64
    N = int(round(2 * math.pi * 16 / dxc))
    ny = 8 if dim == 2 else 1
    c = cfg(orc, dim=dim, n=(N, ny, 1), dx=dxc, dt=0.95 * dxc / math.sqrt(dim), field_bc=orc.BC_PERIODIC)
    sim = orc.Sim(c)
    ext = sim.ext
    xs = 10.0
    f = lambda x: np.where((x > xs) & (x < xs + 2 * T), a0 * np.sin(x - xs - T) * np.sin(np.pi * (x - xs) / (2 * T)) ** 2, 0.0)
    F = np.zeros((9, ext[2], ext[1], ext[0]))
    F[1, :, :, :] = f(np.arange(ext[0]) * dxc)[None, None, :]
    F[5, :, :, :] = f((np.arange(ext[0]) + 0.5) * dxc)[None, None, :]
    sim.set_fields(F)
    exact = _sin2_pulse_energy(a0, T) * (ny * dxc if dim == 2 else 1.0)
    e = sim.energies()
    assert abs(e[0] / exact - 1) < 1e-10, (e[0], exact)
    assert e[2] == 0.0 and e[3] == 0.0
    sim.step(200)
    assert abs(sim.energies()[0] / exact - 1) < 1e-5


def test_incident_pulse_energy_on_the_grid(orc):
    """Scattered-field run without plasma: the scattered energy stays 0 and the total-field
    energy (scattered + incident at the grid points) is the incident pulse's closed-form
    energy once the whole pulse is inside the box (pins the incident term's stagger and
    time)."""
    a0, T, dxc = 1.3, 23.546, 2 * math.pi / 64
    N = 900
    dt = 0.95 * dxc
    c = cfg(orc, n=(N, 1, 1), dx=dxc, dt=dt, beam=orc.BEAM_PLANE, envelope=orc.ENV_SIN2, a0=a0, duration=T,
            focus=(0.0, 0, 0))
    sim = orc.Sim(c)
    sim.step(int(round((2 * T + 8.0) / dt)))      # pulse in [~8, 2T + 8]
    e = sim.energies()
    assert e[0] == 0.0
    assert abs(e[1] / _sin2_pulse_energy(a0, T) - 1) < 1e-10, e


def test_kinetic_energy_of_a_drifting_plasma(orc):
    """Electrons evenly spread over a periodic 2D box with u_x = u0 sin(k x): the kinetic
    energy is n_e int (gamma - 1) dA, i.e. n_e L_y int_0^L (sqrt(1 + u0^2 sin^2 kx) - 1) dx
    (pins the macro-weight, gamma - 1 and the cell area)."""
    from scipy.integrate import quad

    N, ny, dx, ne, ppc, u0 = 64, 4, 0.1, 0.03, 8, 0.8
    c = cfg(orc, dim=2, n=(N, ny, 1), dx=dx, dt=0.06, field_bc=orc.BC_PERIODIC)
    sim = orc.Sim(c)
    L, Ly = N * dx, ny * dx
    npx = N * ppc
    xs = (np.arange(npx) + 0.5) * (L / npx)
    X = np.zeros((npx * ny, 3)); U = np.zeros((npx * ny, 3))
    for j in range(ny):
        X[j * npx:(j + 1) * npx, 0] = xs
        X[j * npx:(j + 1) * npx, 1] = (j + 0.5) * dx
        U[j * npx:(j + 1) * npx, 0] = u0 * np.sin(2 * math.pi * xs / L)
    # each particle stands for the density n_e over a cell area: ppc per cell (N*ny cells)
    sim.set_particles(X, U, np.full(npx * ny, ne / ppc), np.arange(npx * ny))
    k = 2 * math.pi / L
    want = ne * Ly * quad(lambda x: math.sqrt(1 + (u0 * math.sin(k * x)) ** 2) - 1, 0, L, limit=200)[0]
    assert abs(sim.energies()[2] / want - 1) < 1e-10


def test_langmuir_energy_exchange(orc):
    """Cold periodic plasma with a velocity perturbation: kinetic energy turns into field
    energy and back (a Langmuir oscillation) while their sum stays within 1e-3 of itself,
    the deviation shrinking with dt: fixes the relative normalisation of the two energies
    (u lives at half steps: the kinetic energy at step n is the mean of its values at
    n -/+ 1/2)."""
    N, dx, ne, ppc = 128, 0.1, 0.04, 8
    var = []
    for dt in (0.095, 0.0475):
        c = cfg(orc, n=(N, 1, 1), dx=dx, dt=dt, field_bc=orc.BC_PERIODIC)
        sim = orc.Sim(c)
        npart = N * ppc
        x = (np.arange(npart) + 0.5) * (dx / ppc)
        X = np.zeros((npart, 3)); X[:, 0] = x
        U = np.zeros((npart, 3)); U[:, 0] = 1e-2 * np.sin(2 * math.pi * x / (N * dx))
        sim.set_particles(X, U, np.full(npart, ne / ppc), np.arange(npart))
        em, kin = [], []
        for _ in range(int(round(300 * 0.095 / dt))):   # about 1.4 plasma periods
            sim.step(1)
            e = sim.energies()
            em.append(e[0]); kin.append(e[2])
        em, kin = np.array(em), np.array(kin)
        tot = em[:-1] + 0.5 * (kin[1:] + kin[:-1])
        scale = tot.mean()
        assert em.max() > 0.99 * scale and em.min() < 1e-3 * scale        # full exchange
        assert kin.max() > 0.99 * scale and kin.min() < 1e-3 * scale
        var.append((tot.max() - tot.min()) / scale)
    assert var[0] < 1e-3
    assert var[1] < 0.7 * var[0]            # shrinks with dt (measured: first order)
