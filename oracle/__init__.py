"""FP64 CPU oracle for the scattered-field PIC step (arXiv 2310.11393).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` use it.  The CUDA library never
imports, links or calls it, and it shares no code with the CUDA path.

The arithmetic lives in ``orc.c`` (plain C, double precision); this module only
compiles it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

BEAM_NONE, BEAM_PLANE, BEAM_LP, BEAM_RP, BEAM_UNIFORM, BEAM_GAUSS2D = 0, 1, 2, 3, 4, 5
PUSHER_BORIS, PUSHER_VAY, PUSHER_HC = 0, 1, 2
PROFILE_UNIFORM, PROFILE_SUPERGAUSS = 0, 1
ENV_SIN2, ENV_GAUSS = 0, 1
BC_MUR, BC_PERIODIC = 0, 1


def build(force: bool = False) -> str:
    """Compile orc.c into oracle/_build/liborc.so (portable flags: x86 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "orc.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("field_bc", ctypes.c_int),
        ("tf_mode", ctypes.c_int),
        ("beam", ctypes.c_int),
        ("envelope", ctypes.c_int),
        ("a0", ctypes.c_double),
        ("duration", ctypes.c_double),
        ("phi0", ctypes.c_double),
        ("t_focus", ctypes.c_double),
        ("focus", ctypes.c_double * 3),
        ("a", ctypes.c_double),
        ("s", ctypes.c_double),
        ("psi0", ctypes.c_double),
        ("e_unif", ctypes.c_double * 3),
        ("b_unif", ctypes.c_double * 3),
        ("slab_lo", ctypes.c_int * 3),
        ("slab_hi", ctypes.c_int * 3),
        ("n_e", ctypes.c_double),
        ("ppc", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("remove_margin", ctypes.c_int),
        ("pusher", ctypes.c_int),
        ("w0", ctypes.c_double),
        ("profile", ctypes.c_int),
        ("prof_order", ctypes.c_int),
        ("prof_x0", ctypes.c_double),
        ("prof_fwhm", ctypes.c_double),
        ("prof_cut", ctypes.c_double),
        ("incident_grid", ctypes.c_int),
    ]


_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcConfig)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_step_particles.argtypes = [ctypes.c_void_p]
            L.orc_step_fields.argtypes = [ctypes.c_void_p]
            for f in ("orc_num_particles", "orc_num_exits", "orc_step_index"):
                getattr(L, f).restype = ctypes.c_int64
                getattr(L, f).argtypes = [ctypes.c_void_p]
            L.orc_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_int64, _DP, _DP, _DP, _I64P]
            L.orc_get_particles.argtypes = [ctypes.c_void_p, _DP, _DP, _DP, _I64P]
            L.orc_get_exits.argtypes = [ctypes.c_void_p, _DP, _DP, _I64P, _I64P]
            L.orc_extents.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
            L.orc_get_fields.argtypes = [ctypes.c_void_p, _DP]
            L.orc_set_fields.argtypes = [ctypes.c_void_p, _DP]
            L.orc_energies.argtypes = [ctypes.c_void_p, _DP]
            L.orc_gauss_residual.restype = _D
            L.orc_gauss_residual.argtypes = [ctypes.c_void_p]
            L.orc_charge_density.argtypes = [ctypes.c_void_p, _DP]
            L.orc_incident.argtypes = [ctypes.POINTER(OrcConfig), _DP, _D, _DP, _DP]
            for f in ("orc_lp_field", "orc_rp_field"):
                getattr(L, f).argtypes = [_D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int, _DP, _DP]
            L.orc_beam_complex.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int,
                                           _DP, _DP, _DP, _DP]
            L.orc_a_from_w0.restype = _D
            L.orc_a_from_w0.argtypes = [_D]
            L.orc_focal_fwhm.restype = _D
            L.orc_focal_fwhm.argtypes = [ctypes.c_int, _D, _D]
            L.orc_s_from_duration.restype = _D
            L.orc_s_from_duration.argtypes = [ctypes.c_int, _D, _D]
            L.orc_psi0_from_a0.restype = _D
            L.orc_psi0_from_a0.argtypes = [ctypes.c_int, _D, _D, _D]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def make_config(**kw) -> OrcConfig:
    """Build an OrcConfig from keyword arguments (names as in orc.h)."""
    c = OrcConfig()
    c.remove_margin = 3
    for k, v in kw.items():
        if k in ("n", "focus", "e_unif", "b_unif", "slab_lo", "slab_hi"):
            arr = getattr(c, k)
            vals = list(v) + [0] * (3 - len(v))
            for i in range(3):
                arr[i] = vals[i]
        else:
            setattr(c, k, v)
    return c


class Sim:
    """Owning handle on an oracle simulation."""

    def __init__(self, cfg: OrcConfig):
        self.cfg = cfg
        self._L = lib()
        self.h = self._L.orc_create(ctypes.byref(cfg))
        ext = (ctypes.c_int * 3)()
        self._L.orc_extents(self.h, ext)
        self.ext = tuple(ext)

    def __del__(self):
        if getattr(self, "h", None):
            self._L.orc_destroy(self.h)
            self.h = None

    def step(self, n: int = 1):
        self._L.orc_step(self.h, int(n))

    def step_particles(self):
        """First part of one step: gather, incident field, push, move, deposit, exits."""
        self._L.orc_step_particles(self.h)

    def step_fields(self):
        """Second part of one step: Yee update driven by the deposited J, step counter."""
        self._L.orc_step_fields(self.h)

    @property
    def step_index(self) -> int:
        return self._L.orc_step_index(self.h)

    def num_particles(self) -> int:
        return self._L.orc_num_particles(self.h)

    def particles(self):
        n = self.num_particles()
        x = np.zeros((n, 3)); u = np.zeros((n, 3)); w = np.zeros(n); i = np.zeros(n, dtype=np.int64)
        self._L.orc_get_particles(self.h, _dp(x), _dp(u), _dp(w), i.ctypes.data_as(_I64P))
        return {"x": x, "u": u, "w": w, "id": i}

    def set_particles(self, x, u, w, ids):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        self._L.orc_set_particles(self.h, len(w), _dp(x), _dp(u), _dp(w), ids.ctypes.data_as(_I64P))

    def exits(self):
        n = self._L.orc_num_exits(self.h)
        u = np.zeros((n, 3)); w = np.zeros(n); i = np.zeros(n, dtype=np.int64); st = np.zeros(n, dtype=np.int64)
        self._L.orc_get_exits(self.h, _dp(u), _dp(w), i.ctypes.data_as(_I64P), st.ctypes.data_as(_I64P))
        return {"u": u, "w": w, "id": i, "step": st}

    def fields(self) -> np.ndarray:
        """(9, ext_z, ext_y, ext_x): Ex Ey Ez Bx By Bz Jx Jy Jz."""
        out = np.zeros((9, self.ext[2], self.ext[1], self.ext[0]))
        self._L.orc_get_fields(self.h, _dp(out))
        return out

    def set_fields(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == (9, self.ext[2], self.ext[1], self.ext[0])
        self._L.orc_set_fields(self.h, _dp(F))

    def energies(self) -> np.ndarray:
        out = np.zeros(4)
        self._L.orc_energies(self.h, _dp(out))
        return out

    def gauss_residual(self) -> float:
        return self._L.orc_gauss_residual(self.h)

    def charge_density(self) -> np.ndarray:
        out = np.zeros((self.ext[2], self.ext[1], self.ext[0]))
        self._L.orc_charge_density(self.h, _dp(out))
        return out


def incident(cfg: OrcConfig, x, t):
    E = np.zeros(3); B = np.zeros(3)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    lib().orc_incident(ctypes.byref(cfg), _dp(xx), float(t), _dp(E), _dp(B))
    return E, B


def beam_field(beam: int, a, s, psi0, phi0, X, Y, Z, tau, branch: int = 0):
    E = np.zeros(3); B = np.zeros(3)
    f = lib().orc_lp_field if beam == BEAM_LP else lib().orc_rp_field
    f(a, s, psi0, phi0, X, Y, Z, tau, branch, _dp(E), _dp(B))
    return E, B


def beam_complex(beam: int, a, s, psi0, phi0, X, Y, Z, tau, branch: int = 0):
    Er = np.zeros(3); Ei = np.zeros(3); Br = np.zeros(3); Bi = np.zeros(3)
    lib().orc_beam_complex(beam, a, s, psi0, phi0, X, Y, Z, tau, branch, _dp(Er), _dp(Ei), _dp(Br), _dp(Bi))
    return Er + 1j * Ei, Br + 1j * Bi


def a_from_w0(w0: float) -> float:
    return lib().orc_a_from_w0(w0)


def focal_fwhm(beam: int, a: float, s: float) -> float:
    return lib().orc_focal_fwhm(beam, a, s)


def s_from_duration(beam: int, a: float, duration: float) -> float:
    return lib().orc_s_from_duration(beam, a, duration)


def psi0_from_a0(beam: int, a: float, s: float, a0: float) -> float:
    return lib().orc_psi0_from_a0(beam, a, s, a0)


def splitmix64(seed: int, k: int) -> int:
    return lib().orc_splitmix64(seed, k)


def derive_pulse(beam: int, w0: float, duration: float, a0: float):
    """(a, s, Psi0) of the LP/RP pulse from waist, on-axis focal field FWHM and peak field."""
    a = a_from_w0(w0)
    s = s_from_duration(beam, a, duration)
    return a, s, psi0_from_a0(beam, a, s, a0)


def config_from(w, field_bc: int = BC_MUR, tf_mode: int = None) -> OrcConfig:
    """OrcConfig for a workload description (any object with the attributes of
    synth.Workload); LP/RP parameters not given explicitly are derived here."""
    if tf_mode is None:
        tf_mode = getattr(w, "tf_mode", 0)
    a, s, psi0 = w.a_param, w.s_param, w.psi0
    if w.beam in (BEAM_LP, BEAM_RP) and (a <= 0 or s <= 0 or psi0 <= 0):
        da, ds, dp = derive_pulse(w.beam, w.w0, w.duration, w.a0)
        a = a if a > 0 else da
        s = s if s > 0 else ds
        psi0 = psi0 if psi0 > 0 else psi0_from_a0(w.beam, a, s, w.a0)
    return make_config(dim=w.dim, n=w.n, dx=w.dx, dt=w.dt, field_bc=field_bc, tf_mode=tf_mode, beam=w.beam,
                       envelope=w.envelope, a0=w.a0, duration=w.duration, phi0=w.phi0, t_focus=w.t_focus,
                       focus=w.focus, a=a, s=s, psi0=psi0, e_unif=w.e_unif, b_unif=w.b_unif,
                       slab_lo=w.slab_lo, slab_hi=w.slab_hi, n_e=w.n_e, ppc=w.ppc, seed=w.seed,
                       remove_margin=w.remove_margin, pusher=w.pusher, w0=w.w0, profile=w.profile,
                       prof_order=w.prof_order, prof_x0=w.prof_x0, prof_fwhm=w.prof_fwhm, prof_cut=w.prof_cut,
                       incident_grid=w.incident_grid)
