"""Seeded synthetic workloads shaped like the paper's runs (arXiv 2310.11393).

This module holds no part of the PIC method's arithmetic.  It defines the named
workload presets (box, resolution, slab, beam and pulse request) in the paper's
dimensionless units (c = 1, omega = 1, lengths in lambda/2pi, densities in n_c)
and a numpy SplitMix64 so tests can build explicit particle sets.  Both the
oracle and the CUDA library receive the same preset; each side derives its own
pulse parameters and places its own seeded particles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

LAMBDA_UM = 0.8                                  # central wavelength of the presets
T_R_FS = LAMBDA_UM * 1e-6 / (2 * math.pi * 299792458.0) * 1e15   # 1/omega in fs
TWO_PI = 2.0 * math.pi

BEAM_NONE, BEAM_PLANE, BEAM_LP, BEAM_RP, BEAM_UNIFORM, BEAM_GAUSS2D = 0, 1, 2, 3, 4, 5
PROFILE_UNIFORM, PROFILE_SUPERGAUSS = 0, 1
ENV_SIN2, ENV_GAUSS = 0, 1
FP64, FP32 = 0, 1


def fs(t_fs: float) -> float:
    """Femtoseconds to code time units (1/omega)."""
    return t_fs / T_R_FS


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    dx: float
    steps: int
    beam: int
    a0: float
    duration: float                      # field-amplitude FWHM, code units
    slab_lo: tuple
    slab_hi: tuple
    n_e: float
    ppc: int
    seed: int
    cfl: float = 0.95
    precision: int = FP32
    w0: float = 0.0                      # LP/RP waist, code units
    envelope: int = ENV_SIN2
    phi0: float = 0.0
    focus: tuple = (0.0, 0.0, 0.0)
    t_focus: float = 0.0
    a_param: float = 0.0                 # explicit LP/RP parameters (0: derive from w0, duration, a0)
    s_param: float = 0.0
    psi0: float = 0.0
    e_unif: tuple = (0.0, 0.0, 0.0)
    b_unif: tuple = (0.0, 0.0, 0.0)
    remove_margin: int = 3
    pusher: int = 0                      # 0 Boris, 1 Vay, 2 Higuera-Cary
    profile: int = PROFILE_UNIFORM       # slab density along x: uniform or super-Gaussian (Sec. 3.1)
    prof_order: int = 12
    prof_x0: float = 0.0
    prof_fwhm: float = 1.0
    prof_cut: float = 0.0
    tf_mode: int = 0                     # 1: total-field run, plane wave through x = 0 (1D)
    incident_grid: int = 0               # 1: incident field on the Yee nodes, gathered (prescribed-field route)

    @property
    def dt(self) -> float:
        return self.cfl * self.dx / math.sqrt(self.dim)

    @property
    def n_particles(self) -> int:
        if self.ppc <= 0:
            return 0
        k = self.ppc
        for d in range(self.dim):
            k *= max(0, self.slab_hi[d] - self.slab_lo[d])
        return k

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _centred(dim, n, dx):
    return tuple((n[d] * dx / 2.0) if d < dim else 0.0 for d in range(3))


def c1_1d_plane() -> Workload:
    """1D FP64: Nx = 4096, dx = lambda/64, plane wave a0 = 1, sin^2 envelope of 10 fs FWHM,
    slab cells [1024, 3072) at 0.01 n_c, 16 ppc, 2000 steps."""
    return Workload(name="1d_plane_fp64_4096", dim=1, n=(4096, 1, 1), dx=TWO_PI / 64, steps=2000,
                    beam=BEAM_PLANE, a0=1.0, duration=fs(10.0), slab_lo=(1024, 0, 0), slab_hi=(3072, 1, 1),
                    n_e=0.01, ppc=16, seed=1, precision=FP64, envelope=ENV_SIN2, focus=(0.0, 0.0, 0.0))


def c2_2d_lp() -> Workload:
    """2D: 1024 x 1024, dx = lambda/32, LP beam w0 = lambda, a0 = 10, 5 fs, focus at the slab
    centre, slab 512 x 512 cells at 0.05 n_c with 8 ppc (2 097 152 electrons), 1500 steps."""
    n = (1024, 1024, 1)
    dx = TWO_PI / 32
    return Workload(name="2d_lp_1024sq", dim=2, n=n, dx=dx, steps=1500, beam=BEAM_LP, a0=10.0,
                    duration=fs(5.0), w0=TWO_PI * 1.0, slab_lo=(256, 256, 0), slab_hi=(768, 768, 1),
                    n_e=0.05, ppc=8, seed=2, focus=_centred(2, n, dx), t_focus=n[0] * dx / 2.0)


def c3_3d_rp() -> Workload:
    """3D: 512 x 256 x 256, dx = lambda/24, RP beam w0 = 0.7 lambda, a0 = 20, 5 fs, slab
    256 x 128 x 128 cells at 0.01 n_c with 4 ppc (16 777 216 electrons), 1200 steps."""
    n = (512, 256, 256)
    dx = TWO_PI / 24
    return Workload(name="3d_rp_512x256x256", dim=3, n=n, dx=dx, steps=1200, beam=BEAM_RP, a0=20.0,
                    duration=fs(5.0), w0=TWO_PI * 0.7, slab_lo=(128, 64, 64), slab_hi=(384, 192, 192),
                    n_e=0.01, ppc=4, seed=3, focus=_centred(3, n, dx), t_focus=n[0] * dx / 2.0)


def c6_2d_gauss(dx_div: int = 32) -> Workload:
    """Sec. 3.2's 2D set-up at a cell of lambda/dx_div (the paper runs lambda/16 .. lambda/256):
    window 2 pi [64, 32] (propagation x, transverse y), paraxial Gaussian beam w0 = 16 lambda,
    E0 = 4.86, FWHM_T = 2 pi, the envelope peak crossing the focus at t_f = 133 with the focus
    at x = 133 on the axis y = 32 pi; plasma: the 1D super-Gaussian profile (p = 12) shrunk
    twofold along x (centre 140.75, FWHM 167.55, nothing before 10 pi), uniform in y, peak
    0.31 n_c, 4 ppc; CFL 0.95; T_sim = 64 pi."""
    dx = TWO_PI / dx_div
    n = (64 * dx_div, 32 * dx_div, 1)
    x0, F, cut = 281.5 / 2, 335.1 / 2, 10 * math.pi
    lo = int(math.floor(cut / dx))
    hi = min(n[0] - 4, int(math.ceil((x0 + 0.65 * F) / dx)))
    w = Workload(name=f"2d_gauss_sec32_dx{dx_div}", dim=2, n=n, dx=dx, steps=0, beam=BEAM_GAUSS2D, a0=4.86,
                 duration=TWO_PI, w0=16 * TWO_PI, slab_lo=(lo, 4, 0), slab_hi=(hi, n[1] - 4, 1), n_e=0.31, ppc=4,
                 seed=6, focus=(133.0, 32 * math.pi, 0.0), t_focus=133.0, profile=PROFILE_SUPERGAUSS,
                 prof_order=12, prof_x0=x0, prof_fwhm=F, prof_cut=cut)
    return w.with_(steps=int(round(64 * math.pi / w.dt)))


def scaled(w: Workload, factor: int, steps: Optional[int] = None, name: Optional[str] = None) -> Workload:
    """Same physics on a box `factor` times smaller per axis (cell size unchanged):
    slab and focus shrink with the box, the focal time follows the new box."""
    n = tuple((w.n[d] // factor) if d < w.dim else 1 for d in range(3))
    lo = tuple((w.slab_lo[d] // factor) if d < w.dim else 0 for d in range(3))
    hi = tuple((w.slab_hi[d] // factor) if d < w.dim else 1 for d in range(3))
    focus = _centred(w.dim, n, w.dx)
    t_focus = n[0] * w.dx / 2.0 if w.beam in (BEAM_LP, BEAM_RP) else w.t_focus
    return replace(w, name=name or f"{w.name}_div{factor}", n=n, slab_lo=lo, slab_hi=hi, focus=focus,
                   t_focus=t_focus, steps=steps if steps is not None else w.steps)


# ------------------------------------------------------------------------------------
# batched and served workloads
# ------------------------------------------------------------------------------------
def c4_batch(count: int = 256, seed: int = 4) -> list:
    """Independent 2D runs of uneven size: N uniform in [128, 768] (multiple of 16) per axis,
    ppc uniform in 4..16, w0 log-uniform in [0.5, 3] lambda, a0 log-uniform in [1, 50],
    n_e log-uniform in [0.001, 0.1] n_c, LP/RP half and half; slab = central half per axis;
    500 steps each."""
    rng = np.random.default_rng(seed)
    out = []
    dx = TWO_PI / 32
    for i in range(count):
        N = int(rng.integers(8, 49)) * 16
        ppc = int(rng.integers(4, 17))
        w0 = TWO_PI * float(np.exp(rng.uniform(np.log(0.5), np.log(3.0))))
        a0 = float(np.exp(rng.uniform(np.log(1.0), np.log(50.0))))
        ne = float(np.exp(rng.uniform(np.log(0.001), np.log(0.1))))
        beam = BEAM_LP if i % 2 == 0 else BEAM_RP
        n = (N, N, 1)
        out.append(Workload(name=f"batch2d_{i}", dim=2, n=n, dx=dx, steps=500, beam=beam, a0=a0,
                            duration=fs(5.0), w0=w0, slab_lo=(N // 4, N // 4, 0), slab_hi=(3 * N // 4, 3 * N // 4, 1),
                            n_e=ne, ppc=ppc, seed=1000 + i, focus=_centred(2, n, dx), t_focus=N * dx / 2.0))
    return out


def c5_requests(count: int, rate_hz: float = 20.0, seed: int = 5, max_2d: int = 1024, max_3d: int = 256,
                steps_range=(500, 2000)) -> list:
    """Poisson request stream: (arrival time in s, Workload).  2D N in [256, max_2d] or 3D N in
    [128, max_3d] per axis from a clipped log-normal, RP beam as the 3D preset, steps uniform."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        is3d = rng.random() < 0.5
        if is3d:
            N = int(np.clip(np.exp(rng.normal(np.log(160), 0.25)), 128, max_3d)) // 16 * 16
            n = (N, N, N); dim = 3; dx = TWO_PI / 24
        else:
            N = int(np.clip(np.exp(rng.normal(np.log(512), 0.35)), 256, max_2d)) // 16 * 16
            n = (N, N, 1); dim = 2; dx = TWO_PI / 32
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        lo = tuple((n[d] // 4) if d < dim else 0 for d in range(3))
        hi = tuple((3 * n[d] // 4) if d < dim else 1 for d in range(3))
        w = Workload(name=f"req{i}", dim=dim, n=n, dx=dx, steps=steps, beam=BEAM_RP, a0=20.0, duration=fs(5.0),
                     w0=TWO_PI * 0.7, slab_lo=lo, slab_hi=hi, n_e=0.01, ppc=4, seed=5000 + i,
                     focus=_centred(dim, n, dx), t_focus=n[0] * dx / 2.0)
        out.append((t, w))
    return out


# ------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014) and explicit particle sets
# ------------------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """k-th outputs of the SplitMix64 stream seeded with `seed` (vectorised)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def slab_particles(w: Workload):
    """The seeded slab both sides generate: slab cells x-fastest, `ppc` per cell, particle p
    takes outputs 3p+d of SplitMix64(seed); in-cell offset = top 24 bits / 2^24.
    Returns (x[n,3] grid coordinates, u[n,3], weight[n], id[n])."""
    ns = [max(0, w.slab_hi[d] - w.slab_lo[d]) if d < w.dim else 1 for d in range(3)]
    n = w.n_particles
    p = np.arange(n, dtype=np.uint64)
    cell_lin = p // np.uint64(w.ppc)
    cx = cell_lin % np.uint64(ns[0])
    cy = (cell_lin // np.uint64(ns[0])) % np.uint64(ns[1])
    cz = cell_lin // np.uint64(ns[0] * ns[1])
    cells = [cx, cy, cz]
    x = np.zeros((n, 3))
    for d in range(w.dim):
        r = splitmix64(w.seed, np.uint64(3) * p + np.uint64(d))
        off = (r >> np.uint64(40)).astype(np.float64) / 16777216.0
        x[:, d] = ((w.slab_lo[d] + cells[d].astype(np.float64)) + off) * w.dx
    u = np.zeros((n, 3))
    wt = np.full(n, w.n_e / max(w.ppc, 1))
    return x, u, wt, p.astype(np.int64)


PRESETS = {"1d": c1_1d_plane, "2d": c2_2d_lp, "3d": c3_3d_rp}
