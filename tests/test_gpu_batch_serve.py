"""Batched stepping and the continuous-batching server against standalone runs: every
simulation gives the same result alone and in the mix (up to the summation order of the
current deposit in single precision)."""
import math
import time

import numpy as np
import pytest

import synth
from _support import field_errors, match_by_id, momentum_error

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


def mix():
    """Four uneven 2D runs: LP and RP, different sizes, densities, waists and amplitudes."""
    out = []
    dx = 2 * math.pi / 32
    for i, (N, beam, w0, a0, ne, ppc) in enumerate([(96, synth.BEAM_LP, 0.5, 10.0, 0.05, 4),
                                                    (128, synth.BEAM_RP, 0.7, 20.0, 0.02, 2),
                                                    (80, synth.BEAM_LP, 1.0, 5.0, 0.08, 6),
                                                    (112, synth.BEAM_RP, 0.5, 30.0, 0.01, 3)]):
        dt = 0.95 * dx / math.sqrt(2)
        out.append(synth.Workload(name=f"mix{i}", dim=2, n=(N, N, 1), dx=dx, steps=40, beam=beam, a0=a0,
                                  duration=synth.fs(5.0), w0=2 * math.pi * w0, slab_lo=(N // 4, N // 4, 0),
                                  slab_hi=(3 * N // 4, 3 * N // 4, 1), n_e=ne, ppc=ppc, seed=100 + i,
                                  focus=(N * dx / 2, N * dx / 2, 0.0), t_focus=20 * dt))
    return out


def test_batch_equals_alone(P):
    ws = mix()
    alone = []
    for w in ws:
        s = P.Simulation(P.config_from(w))
        s.step(40)
        alone.append((s.particles(), s.fields(), s.energies()))
        s.close()
    sims = [P.Simulation(P.config_from(w)) for w in ws]
    P.pic_batch_step([s.h for s in sims], 25)
    P.pic_batch_step([s.h for s in sims], 15)
    for w, s, (pa, fa, ea) in zip(ws, sims, alone):
        pb = s.particles()
        assert s.info().step == 40
        assert set(pb["id"].tolist()) == set(pa["id"].tolist())
        err, n = momentum_error(pb, pa, w.a0)
        assert err < 1e-5, (w.name, err)      # FP32: deposit summation order differs
        assert field_errors(s.fields(), fa)[:6].max() < 1e-5


def test_batch_against_the_oracle(P, orc):
    ws = mix()[:2]
    sims = [P.Simulation(P.config_from(w)) for w in ws]
    P.pic_batch_step([s.h for s in sims], 30)
    for w, s in zip(ws, sims):
        ref = orc.Sim(orc.config_from(w))
        ref.step(30)
        err, n = momentum_error(s.particles(), ref.particles(), w.a0)
        assert err < 1e-5, (w.name, err)


@pytest.mark.parametrize("fill", [0, 1])
def test_server_results_equal_alone(P, fill):
    """fill = 1: each quantum advances only the request with the least remaining work, so
    the others wait; the results are the same either way."""
    ws = mix()
    steps = [40, 25, 60, 33]
    alone = []
    for w, k in zip(ws, steps):
        s = P.Simulation(P.config_from(w))
        s.step(k)
        alone.append(s.energies())
        s.close()
    srv = P.pic_serve_open(quantum=10, fill_particles=fill)
    tickets = []
    for w, k in zip(ws, steps):
        tickets.append(P.pic_serve_submit(srv, P.config_from(w), k))
        time.sleep(0.01)
    results = {}
    deadline = time.time() + 120
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t in results:
                continue
            st, r = P.pic_serve_poll(srv, t)
            if st == P.PIC_OK:
                results[t] = r
            else:
                assert st == P.PIC_EBUSY, st
        time.sleep(0.01)
    P.pic_serve_close(srv)
    assert len(results) == len(tickets)
    for t, k, ea in zip(tickets, steps, alone):
        r = results[t]
        assert r.steps_done == k
        assert r.energies[6] == k
        assert r.submit_time <= r.start_time <= r.finish_time
        for j in (0, 2):
            rel = abs(r.energies[j] - ea[j]) / abs(ea[j])
            print(f"served vs alone, {k} steps, energy {j}: {rel:.2e}")
            assert rel <= 1e-5, (k, j, r.energies[j], ea[j])


def test_alone_batch_and_profiled_steps_interleave(P):
    """One simulation advanced alone, in two different batches, one kernel at a time and
    after a particle reload, in turns: each kind of step numbers its work items for its own
    launch group, and a step after another group's (or after a new particle layout) first
    renumbers them.  The result equals the same number of plain steps."""
    ws = mix()
    ref = P.Simulation(P.config_from(ws[0]))
    ref.step(40)
    pr, fr = ref.particles(), ref.fields()
    ref.close()
    a = P.Simulation(P.config_from(ws[0]))
    b = P.Simulation(P.config_from(ws[1]))
    c = P.Simulation(P.config_from(ws[2]))
    a.step(5)
    P.pic_batch_step([a.h, b.h], 5)
    a.step(3)
    P.pic_batch_step([c.h, a.h], 4)
    P.pic_batch_step([a.h, b.h], 3)
    P.pic_profile_step(a.h, 4)
    a.step(2)
    # a reload of the particles as they are (a new layout, same state)
    p = a.particles()
    a.set_particles(p["x"], p["u"], p["w"], p["id"])
    P.pic_batch_step([a.h, b.h], 6)
    a.step(8)
    assert a.info().step == 40
    pa = a.particles()
    assert set(pa["id"].tolist()) == set(pr["id"].tolist())
    err, n = momentum_error(pa, pr, ws[0].a0)
    assert err < 1e-5, err
    assert field_errors(a.fields(), fr)[:6].max() < 1e-5
    for s in (a, b, c):
        s.close()


def test_batch_profile_equals_batched_steps(P):
    """The phase-by-phase batched step (pic_batch_profile_step) advances the list exactly as the
    batched graph does (FP64: the same kernels in the same order), and reports every phase."""
    ws = [w.with_(precision=synth.FP64) for w in mix()[:3]]
    a = [P.Simulation(P.config_from(w)) for w in ws]
    b = [P.Simulation(P.config_from(w)) for w in ws]
    P.pic_batch_step([s.h for s in a], 12)
    P.pic_batch_step([s.h for s in b], 5)
    ph = P.pic_batch_profile_step([s.h for s in b], 7)
    assert ph[0] > 0 and ph[1] > 0 and ph[3] > 0 and ph[4] > 0
    assert ph[2] < 0.1 * ph[0]          # no cell sort here: the events around an empty phase
    for sa, sb in zip(a, b):
        assert sb.info().step == 12
        pa, pb = sa.particles(), sb.particles()
        assert set(pa["id"].tolist()) == set(pb["id"].tolist())
        common, ia, ib = match_by_id(pa, pb)
        assert np.abs(pa["u"][ia] - pb["u"][ib]).max() < 1e-12 * max(1.0, np.abs(pa["u"]).max())
        assert field_errors(sa.fields(), sb.fields()).max() < 1e-12
    for s in a + b:
        s.close()
