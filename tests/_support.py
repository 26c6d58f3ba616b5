"""Shared helpers of the parity tests: small seeded workloads shaped like the paper's
runs, and comparisons of the CUDA path with the oracle by particle id and grid point."""
from __future__ import annotations

import math

import numpy as np

import synth

TWO_PI = 2 * math.pi


def small_1d(steps=300):
    """1D FP64 plane wave (a0 = 1, sin^2, 10 fs) into a 0.01 n_c slab; the pulse enters the
    slab after ~70 steps."""
    w = synth.c1_1d_plane()
    return w.with_(name="1d_small", n=(512, 1, 1), slab_lo=(64, 0, 0), slab_hi=(448, 1, 1), steps=steps)


def small_2d(precision=synth.FP32, steps=50):
    """2D LP pulse (w0 = lambda/2 so the ring R~ = 0 crosses the slab, a0 = 10, 5 fs) focused
    in a 0.05 n_c slab; the pulse peak reaches the focus at step 25."""
    n = (96, 80, 1)
    dx = TWO_PI / 32
    dt = 0.95 * dx / math.sqrt(2)
    return synth.Workload(name="2d_lp_small", dim=2, n=n, dx=dx, steps=steps, beam=synth.BEAM_LP, a0=10.0,
                          duration=synth.fs(5.0), w0=TWO_PI * 0.5, slab_lo=(16, 8, 0), slab_hi=(80, 72, 1),
                          n_e=0.05, ppc=4, seed=21, focus=(48 * dx, 40 * dx, 0.0), t_focus=25 * dt,
                          precision=precision)


def small_3d(precision=synth.FP32, steps=30):
    """3D RP pulse (a = 3.5 so the ring lies in the slab, a0 = 20) in a 0.01 n_c slab."""
    n = (32, 32, 32)
    dx = TWO_PI / 24
    dt = 0.95 * dx / math.sqrt(3)
    return synth.Workload(name="3d_rp_small", dim=3, n=n, dx=dx, steps=steps, beam=synth.BEAM_RP, a0=20.0,
                          duration=synth.fs(5.0), w0=0.0, a_param=3.5, s_param=20.0,
                          slab_lo=(8, 8, 8), slab_hi=(24, 24, 24), n_e=0.01, ppc=1, seed=31,
                          focus=(16 * dx, 16 * dx, 16 * dx), t_focus=15 * dt, precision=precision)


def match_by_id(a, b):
    """Index arrays so that a[ia] and b[ib] are the same particles (ids present in both)."""
    ida, idb = np.asarray(a["id"]), np.asarray(b["id"])
    common, ia, ib = np.intersect1d(ida, idb, assume_unique=True, return_indices=True)
    return common, ia, ib


# Floor of the momentum normalisation, as a fraction of a0.  The survey's first reading
# used 1e-3 a0; an electron's momentum swings through zero over a carrier cycle while its
# FP32 error is set by the field amplitude (a sum of impulses of size ~a0 dt), so the
# normalisation is floored at 1e-2 a0 (the quiver-momentum scale divided by 100).
MOMENTUM_FLOOR = 1e-2


def momentum_error(p_gpu, p_ref, a0, floor=MOMENTUM_FLOOR):
    """max over particles of |p_gpu - p_ref| / max(|p_ref|, floor a0), and the number of
    particles compared (matched by id)."""
    common, ia, ib = match_by_id(p_gpu, p_ref)
    du = np.linalg.norm(p_gpu["u"][ia] - p_ref["u"][ib], axis=1)
    den = np.maximum(np.linalg.norm(p_ref["u"][ib], axis=1), floor * a0)
    return float((du / den).max()) if len(common) else 0.0, len(common)


def position_error(p_gpu, p_ref, dx):
    common, ia, ib = match_by_id(p_gpu, p_ref)
    return float(np.abs(p_gpu["x"][ia] - p_ref["x"][ib]).max() / dx) if len(common) else 0.0


def field_errors(F_gpu, F_ref):
    """per-component max |diff| / max |ref| (components with a zero reference report abs diff)."""
    out = []
    for c in range(F_ref.shape[0]):
        ref = np.abs(F_ref[c]).max()
        diff = np.abs(F_gpu[c] - F_ref[c]).max()
        out.append(diff / ref if ref > 0 else diff)
    return np.array(out)
