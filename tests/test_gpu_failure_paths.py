"""Failure detection on the GPU without a fault, a trap or a hang:

  * a non-finite momentum given through pic_set_particles spreads through the deposit and
    the field solve and the energy diagnostic reports PIC_ENAN;
  * a bounded device wait that runs out: one block of the multi-block tile scan is held
    (pic_test_hold_scan) so that the look-back of the blocks after it polls a flag that
    nothing sets, gives up after its bound, flags PIC_FLAG_TIMEOUT, and the next synchronous
    call returns PIC_ETIMEOUT; the CUDA context stays usable (a new simulation runs and its
    results are finite).  No TMA copy is pending during that wait.
"""
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


@pytest.mark.parametrize("prec", [synth.FP32, synth.FP64])
def test_non_finite_momentum_is_reported(P, prec):
    w = small_2d(precision=prec)
    sim = P.Simulation(P.config_from(w))
    p = sim.particles()
    u = p["u"].copy()
    u[len(u) // 2, 0] = float("nan")
    sim.set_particles(p["x"], u, p["w"], p["id"])
    sim.step(5)
    with pytest.raises(P.PicError) as e:
        sim.energies()
    assert e.value.status == P.PIC_ENAN
    sim.close()
    fresh = P.Simulation(P.config_from(w))
    fresh.step(5)
    assert np.all(np.isfinite(fresh.energies()))


def _many_tiles():
    """2D box of 512 x 512 cells in 4 x 4-cell particle tiles: 16 384 tiles, scanned by four
    look-back blocks."""
    dx = 2 * math.pi / 32
    n = (512, 512, 1)
    return synth.Workload(name="2d_many_tiles", dim=2, n=n, dx=dx, steps=10, beam=synth.BEAM_LP, a0=5.0,
                          duration=synth.fs(5.0), w0=2 * math.pi, slab_lo=(192, 192, 0), slab_hi=(320, 320, 1),
                          n_e=0.01, ppc=1, seed=12, focus=(256 * dx, 256 * dx, 0.0), t_focus=256 * dx)


def test_lookback_wait_that_runs_out_is_reported(P):
    w = _many_tiles()
    sim = P.Simulation(P.config_from(w, tile=(4, 4), chunk=256))
    assert sim.info().params.tile[0] == 4
    sim.step(2)
    assert sim.info().status == 0
    P.pic_test_hold_scan(sim.h, 1, 1 << 12)      # block 1 publishes nothing; 4096 polls each
    sim.step(1)
    st = sim.info().status
    assert st & P.PIC_FLAG_TIMEOUT, st
    with pytest.raises(P.PicError) as e:
        sim.energies()
    assert e.value.status == P.PIC_ETIMEOUT
    for hist in (P.pic_histogram, P.pic_histogram_static):   # read the same status word
        with pytest.raises(P.PicError) as e:
            hist(sim.h, 8, 1.0, 4)
        assert e.value.status == P.PIC_ETIMEOUT
    sim.close()
    # the context is still usable
    fresh = P.Simulation(P.config_from(w, tile=(4, 4), chunk=256))
    fresh.step(3)
    info = fresh.info()
    assert info.status == 0 and info.n_alive == w.n_particles
    assert np.all(np.isfinite(fresh.energies()))


def test_pipe_rate_probe(P):
    import torch

    pk = P.pic_probe_peaks(torch.cuda.current_stream().cuda_stream)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    print(f"sms {pk.sms}, FP32 {pk.fp32_tflops:.1f} TFLOP/s ({pk.fp32_flop_per_clk_sm:.0f} per clock and SM), "
          f"FP64 {pk.fp64_tflops:.2f} TFLOP/s, SFU {pk.sfu_gops:.0f} G/s, SM clock {pk.sm_clock_mhz:.0f} MHz")
    assert pk.sms == props.multi_processor_count
    assert 100.0 < pk.sm_clock_mhz < 3000.0
    assert 128.0 < pk.fp32_flop_per_clk_sm < 260.0      # 128 FP32 lanes per SM, an FMA = 2
    assert 0.0 < pk.fp64_tflops < pk.fp32_tflops
    assert pk.sfu_gops > 0
