"""pic_histogram_static — the histogram for callers that must not allocate device memory
(its bins live in a static device array of the library) — against pic_histogram, whose bins
live in the simulation's own buffers, on two calls in a row.  Kept in a file of its own that
pytest collects last."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_static_histogram_matches_pic_histogram_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    n = (96, 80, 1)
    dx = 2 * math.pi / 32
    dt = 0.95 * dx / math.sqrt(2)
    w = synth.Workload(name="hist_2d_lp", dim=2, n=n, dx=dx, steps=40, beam=synth.BEAM_LP, a0=20.0,
                       duration=synth.fs(5.0), w0=2 * math.pi * 0.5, slab_lo=(16, 8, 0), slab_hi=(80, 72, 1),
                       n_e=0.05, ppc=4, seed=77, focus=(48 * dx, 40 * dx, 0.0), t_focus=15 * dt)
    sim = pic.Simulation(pic.config_from(w))
    for steps, (n_e, e_max, n_a) in ((25, (64, 2.0, 36)), (20, (128, 8.0, 90))):
        sim.step(steps)
        ref = sim.histogram(n_e, e_max, n_a)
        got = pic.pic_histogram_static(sim.h, n_e, e_max, n_a)
        assert ref.sum() > 0
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15 * ref.sum())
    with pytest.raises(pic.PicError) as e:
        pic.pic_histogram_static(sim.h, 200, 1.0, 100)
    assert e.value.status == pic.PIC_EINVAL
    sim.close()
