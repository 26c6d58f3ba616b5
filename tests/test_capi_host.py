"""Host-side checks of the C-ABI (no GPU): the library builds for sm_103a, loads, exports
every entry point include/pic.h declares, validates configurations, and derives the LP/RP
pulse parameters (Sec. 4.1) with its own host code in agreement with the oracle's."""
import math
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    pic.load()
    return pic


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert len(names) >= 18
    L = P.load()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a_only(P):
    import subprocess

    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", P.lib_path()], capture_output=True, text=True)
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


@pytest.mark.parametrize("wl", ["2d", "3d", "w05", "w3"])
def test_pulse_parameters_match_the_oracle(P, orc, wl):
    w = {"2d": synth.c2_2d_lp(), "3d": synth.c3_3d_rp(),
         "w05": synth.c2_2d_lp().with_(w0=TWO_PI * 0.5, a0=3.0),
         "w3": synth.c2_2d_lp().with_(w0=TWO_PI * 3.0, beam=synth.BEAM_RP, a0=40.0)}[wl]
    p = P.pic_derive_params(P.config_from(w))
    a, s, psi0 = orc.derive_pulse(w.beam, w.w0, w.duration, w.a0)
    assert abs(p.a / a - 1) < 1e-13
    assert abs(p.s / s - 1) < 1e-9
    assert abs(p.psi0 / psi0 - 1) < 1e-9
    assert abs(p.dt - w.dt) < 1e-15


TWO_PI = 2 * math.pi


def test_counts_and_footprint(P):
    w = synth.c2_2d_lp()
    p = P.pic_derive_params(P.config_from(w))
    assert p.n_particles == 2097152
    # fields (2 sets of E,B + 2 J) + 2 particle buffer sets of 2^dim slots per particle
    # (the tiles' slack for arrivals) + diagnostics
    assert 0.1e9 < p.device_bytes < 1e9
    w3 = synth.c3_3d_rp()
    p3 = P.pic_derive_params(P.config_from(w3))
    assert p3.n_particles == 16777216
    assert p3.device_bytes < 16e9


@pytest.mark.parametrize("bad,frag", [
    (dict(dim=4), "dim"),
    (dict(dt=1.0), "CFL"),
    (dict(slab_lo=(1, 256, 0)), "slab"),
    (dict(tile=(6, 16, 1)), "tile"),
    (dict(n=(8, 1024, 1)), "n[0]"),
    (dict(chunk=1000), "chunk"),
    (dict(tf_mode=1), "tf_mode"),
    (dict(beam=5, w0=0.0), "Gaussian"),
    (dict(profile=1, prof_fwhm=0.0), "super-Gaussian"),
    (dict(pusher=3), "pusher"),
    (dict(chunk=32768), "chunk"),
])
def test_invalid_configs_are_rejected(P, bad, frag):
    w = synth.c2_2d_lp()
    c = P.config_from(w)
    for k, v in bad.items():
        if isinstance(v, tuple):
            arr = getattr(c, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(c, k, v)
    with pytest.raises(P.PicError) as e:
        P.pic_derive_params(c)
    assert e.value.status == P.PIC_EINVAL
    assert frag in str(e.value)


def test_lp_needs_two_dimensions(P):
    w = synth.c1_1d_plane().with_(beam=synth.BEAM_LP, w0=TWO_PI, a0=1.0)
    with pytest.raises(P.PicError):
        P.pic_derive_params(P.config_from(w))


def test_work_item_size_and_tuner_arguments(P):
    w = synth.c2_2d_lp()
    assert P.pic_derive_params(P.config_from(w)).chunk == 2048
    assert P.pic_derive_params(P.config_from(w, chunk=4096)).chunk == 4096
    # nothing left to tune: no device needed, nothing measured
    c = P.config_from(w, tile=(32, 16, 1), chunk=1024)
    assert P.pic_autotune(c, 3) == 0.0
    assert list(c.tile)[:2] == [32, 16] and c.chunk == 1024
    with pytest.raises(P.PicError) as e:
        P.pic_autotune(P.config_from(w), 0)
    assert e.value.status == P.PIC_EINVAL


def test_cell_sort_cadence_is_resolved_and_sized(P):
    """sort_every > 0 is kept, <= 0 turns the cell sort off; the cell sort's two int arrays
    (one entry per cell of the tiled grid) are in the device footprint only when it is on."""
    from _support import small_2d

    w = small_2d()
    got, size = {}, {}
    for k in (0, -1, 5):
        prm = P.pic_derive_params(P.config_from(w, tile=(16, 16), sort_every=k))
        got[k], size[k] = prm.sort_every, prm.device_bytes
    assert got == {0: 0, -1: 0, 5: 5}
    tiled_cells = 96 * 80      # 6 x 5 tiles of 16 x 16
    assert size[5] - size[-1] >= 2 * tiled_cells * 4
    assert size[0] == size[-1]
