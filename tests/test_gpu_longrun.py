"""Whole runs against the oracle, checked statistically: a PIC run is chaotic, so single
trajectories of the single-precision path part ways with the double-precision oracle after
some hundred steps, while the distributions do not.

  * scattered-field energy and kinetic energy (electrons in the box and those that left it)
    at every 50th step: relative difference <= 1e-3
    (FP32) and <= 1e-9 (FP64, where only the order of the deposit sums differs);
  * at the end of the run, the weighted cumulative distributions of electron kinetic energy
    and of the angle to the propagation axis, over the electrons in the box and those that
    left it (momentum at exit): sup-distance (Kolmogorov-Smirnov) <= 1e-3.  In FP64 the
    distance can still be one particle's weight, where two electrons have energies equal to
    round-off (a CDF step is then taken in either order); there the electrons' energies are
    compared one by one as well, to 1e-9 of the largest.
"""
import numpy as np
import pytest

import synth
from _support import small_2d, small_3d

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


def energy_angle(parts, exits):
    """kinetic energy, angle to the propagation axis, weight and id of every electron (in the
    box, or at its exit), ordered by id"""
    u = np.concatenate([parts["u"], exits["u"]])
    w = np.concatenate([parts["w"], exits["w"]])
    ids = np.concatenate([parts["id"], exits["id"]])
    o = np.argsort(ids)
    u, w, ids = u[o], w[o], ids[o]
    e = np.sqrt(1.0 + (u * u).sum(axis=1)) - 1.0
    ang = np.arctan2(np.hypot(u[:, 1], u[:, 2]), u[:, 0])
    return e, ang, w, ids


def ks_distance(a, wa, b, wb):
    """sup over x of |F_a(x) - F_b(x)|, F the weight fraction of samples <= x."""
    xs = np.union1d(a, b)
    def cdf(v, w):
        o = np.argsort(v, kind="stable")
        cw = np.concatenate([[0.0], np.cumsum(w[o])]) / w.sum()
        return cw[np.searchsorted(v[o], xs, side="right")]
    return float(np.abs(cdf(a, wa) - cdf(b, wb)).max())


CASES = {"2d_lp": (small_2d, 250), "3d_rp": (small_3d, 120)}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_run_statistics(P, orc, case, prec):
    make, steps = CASES[case]
    w = make(precision=synth.FP32 if prec == "fp32" else synth.FP64, steps=steps)
    tol = 1e-3 if prec == "fp32" else 1e-9
    sim = P.Simulation(P.config_from(w))
    ref = orc.Sim(orc.config_from(w))
    worst = {"em": 0.0, "kin": 0.0}
    for done in range(50, steps + 1, 50):
        k = done - sim.info().step
        sim.step(k)
        ref.step(k)
        eg, er = sim.energies(), ref.energies()
        # scattered EM energy; kinetic energy of the electrons in the box plus that carried out
        for name, g, r in (("em", eg[0], er[0]), ("kin", eg[2] + eg[3], er[2] + er[3])):
            assert r > 0
            worst[name] = max(worst[name], abs(g - r) / r)
    rest = steps - sim.info().step
    if rest:
        sim.step(rest)
        ref.step(rest)
    eg_, ag, wg, ig = energy_angle(sim.particles(), sim.exits())
    er_, ar, wr, ir = energy_angle(ref.particles(), ref.exits())
    assert len(eg_) == len(er_) == w.n_particles
    np.testing.assert_array_equal(ig, ir)
    assert er_.max() > 1.0                      # the run is relativistic
    d_e = ks_distance(eg_, wg, er_, wr)
    d_a = ks_distance(ag, wg, ar, wr)
    print(f"{case} {prec}: energy {worst}, KS energy {d_e:.2e}, KS angle {d_a:.2e}")
    assert worst["em"] < tol and worst["kin"] < tol, worst
    assert d_e < 1e-3 and d_a < 1e-3, (d_e, d_a)
    if prec == "fp64":
        de = float(np.abs(eg_ - er_).max() / er_.max())
        print(f"  per-electron energy difference {de:.2e} of the largest")
        assert de < 1e-9
