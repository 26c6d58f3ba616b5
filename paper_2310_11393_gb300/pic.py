"""Thin ctypes binding of include/pic.h (argument marshalling only).

Every function keeps the C name and argument order; every step of the PIC cycle
runs in the CUDA library libsffpic.so.  There is no CPU fallback: loading fails
loudly when the library has not been built.  PyTorch is used only to hand device
memory (its caching allocator) and streams to the library.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t,
                    c_uint32, c_uint64, c_void_p)

import numpy as np

from . import _build

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ETIMEOUT = 0, -1, -2, -3, -4
PIC_ENAN, PIC_EBUSY, PIC_ECAPACITY, PIC_ENODEV, PIC_ENOTFOUND = -5, -6, -7, -8, -9
PIC_BEAM_NONE, PIC_BEAM_PLANE, PIC_BEAM_LP, PIC_BEAM_RP, PIC_BEAM_UNIFORM = 0, 1, 2, 3, 4
PIC_ENV_SIN2, PIC_ENV_GAUSS = 0, 1
PIC_FP64, PIC_FP32 = 0, 1
PIC_DIAG_ENERGIES, PIC_DIAG_GAUSS, PIC_DIAG_PARTICLES, PIC_DIAG_EXITS, PIC_DIAG_FIELDS = 0, 1, 2, 3, 4
PIC_FLAG_TIMEOUT, PIC_FLAG_CFL, PIC_FLAG_EXIT_OVERFLOW, PIC_FLAG_CAPACITY = 1, 2, 4, 8


class pic_config(Structure):
    _fields_ = [
        ("dim", c_int32), ("n", c_int32 * 3), ("dx", c_double), ("dt", c_double), ("cfl", c_double),
        ("precision", c_int32), ("beam", c_int32), ("envelope", c_int32), ("remove_margin", c_int32),
        ("a0", c_double), ("duration", c_double), ("w0", c_double), ("phi0", c_double), ("t_focus", c_double),
        ("focus", c_double * 3), ("a_param", c_double), ("s_param", c_double), ("psi0", c_double),
        ("e_unif", c_double * 3), ("b_unif", c_double * 3), ("slab_lo", c_int32 * 3), ("slab_hi", c_int32 * 3),
        ("n_e", c_double), ("ppc", c_int32), ("tile", c_int32 * 3), ("seed", c_uint64),
        ("max_particles", c_int64), ("max_exits", c_int64), ("chunk", c_int32), ("pusher", c_int32), ("profile", c_int32), ("prof_order", c_int32),
        ("prof_x0", c_double), ("prof_fwhm", c_double), ("prof_cut", c_double), ("tf_mode", c_int32),
        ("incident_grid", c_int32), ("autotune_steps", c_int32), ("sort_every", c_int32),
    ]


class pic_params(Structure):
    _fields_ = [("a", c_double), ("s", c_double), ("psi0", c_double), ("dt", c_double),
                ("n_particles", c_int64), ("device_bytes", c_int64), ("tile", c_int32 * 3),
                ("yee_tile", c_int32 * 3), ("chunk", c_int32), ("sort_every", c_int32)]


class pic_info(Structure):
    _fields_ = [("step", c_int64), ("time", c_double), ("n_alive", c_int64), ("n_exits", c_int64),
                ("status", c_uint32), ("params", pic_params)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class pic_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class pic_serve_config(Structure):
    _fields_ = [("memory_budget", c_int64), ("max_resident", c_int32), ("quantum", c_int32),
                ("fill_particles", c_int64)]


class pic_result(Structure):
    _fields_ = [("state", c_int32), ("error", c_int32), ("steps_done", c_int64), ("submit_time", c_double),
                ("start_time", c_double), ("finish_time", c_double), ("energies", c_double * 8),
                ("pushes", c_int64)]


class pic_peaks(Structure):
    _fields_ = [("sms", c_int32), ("fp32_tflops", c_double), ("fp64_tflops", c_double), ("sfu_gops", c_double),
                ("sm_clock_mhz", c_double), ("fp32_flop_per_clk_sm", c_double)]


_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load():
    """Load libsffpic.so (build it first with __graft_entry__.build() or _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P = c_void_p
    DP = POINTER(c_double)
    L.pic_derive_params.restype = c_int
    L.pic_derive_params.argtypes = [POINTER(pic_config), POINTER(pic_params)]
    L.pic_init.restype = c_int
    L.pic_init.argtypes = [POINTER(pic_config), POINTER(pic_allocator), P, POINTER(P)]
    L.pic_step.restype = c_int
    L.pic_step.argtypes = [P, c_int, P]
    L.pic_profile_step.restype = c_int
    L.pic_profile_step.argtypes = [P, c_int, P, POINTER(c_double)]
    L.pic_destroy.restype = c_int
    L.pic_destroy.argtypes = [P]
    L.pic_last_error.restype = c_char_p
    L.pic_last_error.argtypes = [P]
    L.pic_info_get.restype = c_int
    L.pic_info_get.argtypes = [P, POINTER(pic_info), P]
    L.pic_set_particles.restype = c_int
    L.pic_set_particles.argtypes = [P, c_int64, DP, DP, DP, POINTER(c_int64), P]
    L.pic_set_fields.restype = c_int
    L.pic_set_fields.argtypes = [P, DP, P]
    L.pic_set_step.restype = c_int
    L.pic_set_step.argtypes = [P, c_int64, P]
    L.pic_diag.restype = c_int
    L.pic_diag.argtypes = [P, c_int, P, c_size_t, P]
    L.pic_histogram.restype = c_int
    L.pic_histogram.argtypes = [P, c_int, c_double, c_int, DP, P]
    L.pic_histogram_static.restype = c_int
    L.pic_histogram_static.argtypes = [P, c_int, c_double, c_int, DP, P]
    L.pic_eval_incident.restype = c_int
    L.pic_eval_incident.argtypes = [P, c_int64, DP, DP, P]
    L.pic_autotune.restype = c_int
    L.pic_autotune.argtypes = [POINTER(pic_config), c_int, P, POINTER(c_double)]
    L.pic_batch_profile_step.restype = c_int
    L.pic_batch_profile_step.argtypes = [POINTER(P), c_int, c_int, P, POINTER(c_double)]
    L.pic_batch_step.restype = c_int
    L.pic_batch_step.argtypes = [POINTER(P), c_int, c_int, P]
    L.pic_serve_open.restype = c_int
    L.pic_serve_open.argtypes = [POINTER(pic_serve_config), POINTER(P)]
    L.pic_serve_submit.restype = c_int
    L.pic_serve_submit.argtypes = [P, POINTER(pic_config), c_int64, POINTER(c_uint64)]
    L.pic_serve_poll.restype = c_int
    L.pic_serve_poll.argtypes = [P, c_uint64, POINTER(pic_result)]
    L.pic_serve_clock.restype = c_double
    L.pic_serve_clock.argtypes = [P]
    L.pic_serve_close.restype = c_int
    L.pic_serve_close.argtypes = [P]
    L.pic_test_hold_scan.restype = c_int
    L.pic_test_hold_scan.argtypes = [P, c_int, c_int]
    L.pic_probe_peaks.restype = c_int
    L.pic_probe_peaks.argtypes = [POINTER(pic_peaks), P]
    _lib = L
    return L


PIC_PUSHER_BORIS, PIC_PUSHER_VAY, PIC_PUSHER_HC = 0, 1, 2
PIC_BEAM_GAUSS2D = 5
PIC_PROFILE_UNIFORM, PIC_PROFILE_SUPERGAUSS = 0, 1


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def check(status: int, sim=None):
    if status != PIC_OK:
        msg = load().pic_last_error(sim)
        raise PicError(status, msg.decode() if msg else "")
    return status


# ---- the C entry points, same names ---------------------------------------------------
def pic_derive_params(cfg: pic_config) -> pic_params:
    out = pic_params()
    check(load().pic_derive_params(byref(cfg), byref(out)))
    return out


def pic_init(cfg: pic_config, allocator=None, stream=0):
    h = c_void_p()
    check(load().pic_init(byref(cfg), byref(allocator) if allocator is not None else None, c_void_p(stream),
                          byref(h)))
    return h


def pic_step(sim, n_steps: int, stream=0):
    return check(load().pic_step(sim, int(n_steps), c_void_p(stream)), sim)


def pic_profile_step(sim, n_steps: int, stream=0) -> np.ndarray:
    out = np.zeros(5)
    check(load().pic_profile_step(sim, int(n_steps), c_void_p(stream), _dp(out)), sim)
    return out


def pic_destroy(sim):
    return load().pic_destroy(sim)


def pic_last_error(sim=None) -> str:
    m = load().pic_last_error(sim)
    return m.decode() if m else ""


def pic_info_get(sim, stream=0) -> pic_info:
    out = pic_info()
    check(load().pic_info_get(sim, byref(out), c_void_p(stream)), sim)
    return out


def _dp(a):
    return a.ctypes.data_as(POINTER(c_double))


def pic_set_particles(sim, x, u, w, ids, stream=0):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    return check(load().pic_set_particles(sim, len(w), _dp(x), _dp(u), _dp(w), ids.ctypes.data_as(POINTER(c_int64)),
                                          c_void_p(stream)), sim)


def pic_set_fields(sim, fields, stream=0):
    f = np.ascontiguousarray(fields, dtype=np.float64)
    return check(load().pic_set_fields(sim, _dp(f), c_void_p(stream)), sim)


def pic_set_step(sim, step: int, stream=0):
    return check(load().pic_set_step(sim, int(step), c_void_p(stream)), sim)


def pic_diag(sim, kind: int, out: np.ndarray, stream=0):
    return check(load().pic_diag(sim, int(kind), out.ctypes.data_as(c_void_p), out.nbytes, c_void_p(stream)), sim)


def pic_histogram(sim, n_e: int, e_max: float, n_a: int, stream=0) -> np.ndarray:
    out = np.zeros((n_e, n_a))
    check(load().pic_histogram(sim, n_e, e_max, n_a, _dp(out), c_void_p(stream)), sim)
    return out


PIC_HIST_STATIC_MAX_BINS = 16384


def pic_histogram_static(sim, n_e: int, e_max: float, n_a: int, stream=0) -> np.ndarray:
    out = np.zeros((n_e, n_a))
    check(load().pic_histogram_static(sim, n_e, e_max, n_a, _dp(out), c_void_p(stream)), sim)
    return out


def pic_eval_incident(sim, pts, stream=0) -> np.ndarray:
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 4)
    out = np.zeros((len(pts), 6))
    check(load().pic_eval_incident(sim, len(pts), _dp(pts), _dp(out), c_void_p(stream)), sim)
    return out


def pic_autotune(cfg: pic_config, trial_steps: int = 4, stream=0) -> float:
    """Fills cfg.tile / cfg.chunk (entries left at 0) with the fastest measured choice;
    returns its time per step in ms (0 when nothing was left to tune)."""
    ms = c_double()
    check(load().pic_autotune(byref(cfg), int(trial_steps), c_void_p(stream), byref(ms)))
    return ms.value


def pic_test_hold_scan(sim, block: int, spins: int):
    """Test aid: one tile-scan block stops publishing, so the look-back waits after it time out."""
    return check(load().pic_test_hold_scan(sim, int(block), int(spins)), sim)


def pic_probe_peaks(stream=0) -> pic_peaks:
    """Measured FP32 / FP64 / special-function issue rates and SM clock of the current device."""
    out = pic_peaks()
    check(load().pic_probe_peaks(byref(out), c_void_p(stream)))
    return out


def pic_batch_step(sims, n_steps: int, stream=0):
    arr = (c_void_p * len(sims))(*[s.value if isinstance(s, c_void_p) else s for s in sims])
    st = load().pic_batch_step(arr, len(sims), int(n_steps), c_void_p(stream))
    return check(st, sims[0])


def pic_batch_profile_step(sims, n_steps: int, stream=0) -> np.ndarray:
    """Phase times (push, tile scan, cell sort, field solve, step end; seconds) of n_steps
    batched steps, each phase launched on its own."""
    arr = (c_void_p * len(sims))(*[s.value if isinstance(s, c_void_p) else s for s in sims])
    out = np.zeros(5)
    check(load().pic_batch_profile_step(arr, len(sims), int(n_steps), c_void_p(stream),
                                        out.ctypes.data_as(POINTER(c_double))))
    return out


def pic_serve_open(memory_budget=0, max_resident=0, quantum=0, fill_particles=0):
    cfg = pic_serve_config(memory_budget, max_resident, quantum, fill_particles)
    h = c_void_p()
    check(load().pic_serve_open(byref(cfg), byref(h)))
    return h


def pic_serve_submit(srv, cfg: pic_config, n_steps: int) -> int:
    t = c_uint64()
    check(load().pic_serve_submit(srv, byref(cfg), int(n_steps), byref(t)))
    return t.value


def pic_serve_poll(srv, ticket: int):
    r = pic_result()
    st = load().pic_serve_poll(srv, c_uint64(ticket), byref(r))
    return st, r


def pic_serve_clock(srv) -> float:
    return load().pic_serve_clock(srv)


def pic_serve_close(srv):
    return load().pic_serve_close(srv)


# ---- helpers for callers -----------------------------------------------------------------
_torch_alloc_keep = []


def torch_allocator(device=None):
    """pic_allocator drawing device memory from PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = pic_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _torch_alloc_keep.append(a)
    return a


def config_from(w, precision=None, tile=None, max_particles=0, max_exits=0, chunk=0, autotune_steps=0,
                sort_every=0) -> pic_config:
    """pic_config for a workload description (attributes as synth.Workload)."""
    c = pic_config()
    c.dim = w.dim
    for d in range(3):
        c.n[d] = int(w.n[d]) if d < w.dim else 1
        c.focus[d] = float(w.focus[d])
        c.e_unif[d] = float(w.e_unif[d])
        c.b_unif[d] = float(w.b_unif[d])
        c.slab_lo[d] = int(w.slab_lo[d]) if d < w.dim else 0
        c.slab_hi[d] = int(w.slab_hi[d]) if d < w.dim else 1
        c.tile[d] = int(tile[d]) if tile is not None and d < len(tile) else 0
    c.dx = w.dx
    c.dt = w.dt
    c.cfl = w.cfl
    c.precision = w.precision if precision is None else precision
    c.beam = w.beam
    c.envelope = w.envelope
    c.remove_margin = w.remove_margin
    c.a0 = w.a0
    c.duration = w.duration
    c.w0 = w.w0
    c.phi0 = w.phi0
    c.t_focus = w.t_focus
    c.a_param = w.a_param
    c.s_param = w.s_param
    c.psi0 = w.psi0
    c.n_e = w.n_e
    c.ppc = w.ppc
    c.seed = w.seed
    c.max_particles = max_particles
    c.max_exits = max_exits
    c.chunk = chunk
    c.autotune_steps = autotune_steps
    c.sort_every = sort_every
    c.pusher = getattr(w, "pusher", 0)
    c.profile = getattr(w, "profile", 0)
    c.prof_order = getattr(w, "prof_order", 12)
    c.prof_x0 = getattr(w, "prof_x0", 0.0)
    c.prof_fwhm = getattr(w, "prof_fwhm", 1.0)
    c.prof_cut = getattr(w, "prof_cut", 0.0)
    c.tf_mode = getattr(w, "tf_mode", 0)
    c.incident_grid = getattr(w, "incident_grid", 0)
    return c


class Simulation:
    """Owning handle with numpy-returning diagnostics (the calls underneath are the C-ABI)."""

    def __init__(self, cfg: pic_config, allocator=None, stream=0):
        self.cfg = cfg
        self.stream = stream
        self.h = pic_init(cfg, allocator, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, stream=None):
        pic_step(self.h, n, self.stream if stream is None else stream)

    def info(self) -> pic_info:
        return pic_info_get(self.h, self.stream)

    def energies(self) -> np.ndarray:
        out = np.zeros(8)
        pic_diag(self.h, PIC_DIAG_ENERGIES, out, self.stream)
        return out

    def gauss_residual(self) -> float:
        out = np.zeros(1)
        pic_diag(self.h, PIC_DIAG_GAUSS, out, self.stream)
        return float(out[0])

    def particles(self):
        n = self.info().n_alive
        out = np.empty((n, 8))          # every entry is written
        pic_diag(self.h, PIC_DIAG_PARTICLES, out, self.stream)
        return {"x": out[:, 0:3], "u": out[:, 3:6], "w": out[:, 6], "id": out[:, 7].astype(np.int64)}

    def exits(self):
        n = self.info().n_exits
        out = np.empty((n, 6))          # every entry is written
        pic_diag(self.h, PIC_DIAG_EXITS, out, self.stream)
        return {"u": out[:, 0:3], "w": out[:, 3], "id": out[:, 4].astype(np.int64), "step": out[:, 5].astype(np.int64)}

    def ext(self):
        d = self.cfg.dim
        return (self.cfg.n[0] + 1, self.cfg.n[1] + 1 if d > 1 else 1, self.cfg.n[2] + 1 if d > 2 else 1)

    def fields(self) -> np.ndarray:
        e = self.ext()
        out = np.zeros((9, e[2], e[1], e[0]))
        pic_diag(self.h, PIC_DIAG_FIELDS, out, self.stream)
        return out

    def set_fields(self, F):
        pic_set_fields(self.h, F, self.stream)

    def set_particles(self, x, u, w, ids):
        pic_set_particles(self.h, x, u, w, ids, self.stream)

    def histogram(self, n_e, e_max, n_a):
        return pic_histogram(self.h, n_e, e_max, n_a, self.stream)

    def eval_incident(self, pts):
        return pic_eval_incident(self.h, pts, self.stream)
