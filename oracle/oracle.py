"""Python handle on the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The product path never imports
this module.  It shares nothing with the CUDA library but the seeded inputs.

The library is compiled on first use (gcc, ``-ffp-contract=off`` so that
results are the same on x86-64 and aarch64 hosts) and cached next to the
source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ncomp", C.c_int),
        ("bx", C.c_int), ("by", C.c_int), ("bz", C.c_int),
        ("periodic", C.c_int * 3),
        ("progressive", C.c_int),
        ("tau", C.c_double), ("beta", C.c_double),
        ("pr_a", C.c_double), ("pr_b", C.c_double), ("pr_R", C.c_double),
        ("pr_omega", C.c_double), ("T_over_Tc", C.c_double),
        ("g_self", C.c_double), ("g_cross", C.c_double),
        ("g_ads", C.c_double * 2),
        ("grav", C.c_double * 3),
        ("rho_ref", C.c_double * 2),
        ("S", C.c_double),
    ]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    ub = C.POINTER(C.c_ubyte)
    P = C.POINTER(Params)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [P, ub, dp, dp, dp]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int]
    lib.orc_macro.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp]
    lib.orc_forces.argtypes = [C.c_void_p, C.c_int, dp]
    lib.orc_active_blocks.restype = C.c_long
    lib.orc_active_blocks.argtypes = [C.c_void_p, ip]
    lib.orc_mass.argtypes = [C.c_void_p, dp]
    lib.orc_crit.argtypes = [C.c_void_p, dp]
    lib.orc_get_f.argtypes = [C.c_void_p, C.c_int, dp]
    lib.orc_set_f.argtypes = [C.c_void_p, C.c_int, dp]
    lib.orc_set_active.argtypes = [C.c_void_p, ub]
    lib.orc_set_time.argtypes = [C.c_void_p, C.c_long]
    lib.orc_time.restype = C.c_long
    lib.orc_time.argtypes = [C.c_void_p]
    lib.orc_lattice.argtypes = [ip, dp, ip]
    lib.orc_feq.argtypes = [C.c_double, dp, dp]
    lib.orc_collide.argtypes = [C.c_double, C.c_double, dp, dp, dp, dp]
    lib.orc_eos_constants.argtypes = [P, dp]
    lib.orc_pressure.restype = C.c_double
    lib.orc_pressure.argtypes = [P, C.c_double]
    lib.orc_psi.restype = C.c_double
    lib.orc_psi.argtypes = [P, C.c_double]
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(**kw) -> Params:
    """Oracle parameters from the same keyword set the CUDA binding takes."""
    p = Params()
    p.nx, p.ny, p.nz = kw["nx"], kw["ny"], kw["nz"]
    p.ncomp = kw.get("ncomp", 2)
    p.bx, p.by, p.bz = kw.get("block", (8, 8, 8))
    per = kw.get("periodic", (1, 1, 0))
    for a in range(3):
        p.periodic[a] = int(per[a])
    p.progressive = int(kw.get("progressive", 1))
    p.tau = kw.get("tau", 1.0)
    p.beta = kw.get("beta", 1.16)
    p.pr_a = kw.get("pr_a", 2.0 / 49.0)
    p.pr_b = kw.get("pr_b", 2.0 / 21.0)
    p.pr_R = kw.get("pr_R", 1.0)
    p.pr_omega = kw.get("pr_omega", 0.344)
    p.T_over_Tc = kw.get("T_over_Tc", 0.85)
    p.g_self = kw.get("g_self", -1.0)
    p.g_cross = kw.get("g_cross", 0.0)
    ga = kw.get("g_ads", (0.0, 0.0))
    p.g_ads[0], p.g_ads[1] = ga[0], ga[1]
    g = kw.get("grav", (0.0, 0.0, 0.0))
    for d in range(3):
        p.grav[d] = g[d]
    rr = kw.get("rho_ref", None)
    if rr is None:
        rr = kw.get("rho_amb", (0.0, 0.0))
    p.rho_ref[0] = rr[0]
    p.rho_ref[1] = rr[1] if len(rr) > 1 else 0.0
    p.S = kw.get("S", 0.0)
    return p


def lattice():
    lib = _load()
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    opp = np.zeros(Q, dtype=np.int32)
    lib.orc_lattice(e.ctypes.data_as(C.POINTER(C.c_int)), _dp(w),
                    opp.ctypes.data_as(C.POINTER(C.c_int)))
    return e, w, opp


def feq(rho: float, u) -> np.ndarray:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib.orc_feq(float(rho), _dp(uu), _dp(out))
    return out


def collide(tau, rho, u, F, fin) -> np.ndarray:
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    out = np.zeros(Q)
    lib.orc_collide(float(tau), float(rho), _dp(u), _dp(F), _dp(fin), _dp(out))
    return out


def eos_constants(**kw):
    lib = _load()
    p = make_params(nx=8, ny=8, nz=8, **kw)
    out = np.zeros(4)
    lib.orc_eos_constants(C.byref(p), _dp(out))
    return dict(Tc=out[0], T=out[1], kappa=out[2], theta=out[3])


def pressure(rho, **kw) -> float:
    lib = _load()
    p = make_params(nx=8, ny=8, nz=8, **kw)
    return lib.orc_pressure(C.byref(p), float(rho))


def psi(rho, **kw) -> float:
    lib = _load()
    p = make_params(nx=8, ny=8, nz=8, **kw)
    return lib.orc_psi(C.byref(p), float(rho))


class OracleSim:
    """One oracle simulation.

    ``cell_type``: uint8 [nz, ny, nx] (0 fluid, 1 solid, 2 held);
    ``rho_init``: [ncomp, nz, ny, nx]; ``u_init``: [ncomp, 3, nz, ny, nx] or
    None; ``rho_amb``: [ncomp].  Keyword parameters as in ``make_params``.
    """

    def __init__(self, cell_type, rho_init, u_init, rho_amb, **kw):
        self.lib = _load()
        self.kw = dict(kw)
        nz, ny, nx = cell_type.shape
        self.shape = (nz, ny, nx)
        kw = {k: v for k, v in kw.items() if k not in ("nx", "ny", "nz")}
        kw.setdefault("rho_amb", tuple(float(r) for r in rho_amb))
        self.params = make_params(nx=nx, ny=ny, nz=nz, **kw)
        self.ncomp = self.params.ncomp
        self.ncell = nx * ny * nz
        ct = np.ascontiguousarray(cell_type, dtype=np.uint8)
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).reshape(self.ncomp, -1)
        ra = np.zeros(2)
        ra[: self.ncomp] = np.asarray(rho_amb, dtype=np.float64)[: self.ncomp]
        uptr = None
        if u_init is not None:
            ui = np.ascontiguousarray(u_init, dtype=np.float64).reshape(self.ncomp, 3, -1)
            self._ui = ui
            uptr = _dp(ui)
        self._keep = (ct, ri, ra)
        self.h = self.lib.orc_create(C.byref(self.params), ct.ctypes.data_as(C.POINTER(C.c_ubyte)),
                                     _dp(ri), uptr, _dp(ra))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        bx, by, bz = kw.get("block", (8, 8, 8))
        self.nblock = (nx // bx) * (ny // by) * (nz // bz)

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    @property
    def t(self) -> int:
        return int(self.lib.orc_time(self.h))

    def macro(self, comp: int):
        out = [np.zeros(self.ncell) for _ in range(4)]
        self.lib.orc_macro(self.h, int(comp), *[_dp(a) for a in out])
        return tuple(a.reshape(self.shape) for a in out)

    def forces(self, comp: int):
        F = np.zeros((self.ncell, 3))
        self.lib.orc_forces(self.h, int(comp), _dp(F))
        return F.reshape(self.shape + (3,))

    def active_blocks(self) -> np.ndarray:
        n = self.lib.orc_active_blocks(self.h, None)
        ids = np.zeros(max(n, 1), dtype=np.int32)
        self.lib.orc_active_blocks(self.h, ids.ctypes.data_as(C.POINTER(C.c_int)))
        return ids[:n].copy()

    def mass(self) -> np.ndarray:
        m = np.zeros(2)
        self.lib.orc_mass(self.h, _dp(m))
        return m[: self.ncomp].copy()

    def crit(self) -> np.ndarray:
        out = np.zeros(self.nblock)
        self.lib.orc_crit(self.h, _dp(out))
        return out

    def get_f(self, comp: int) -> np.ndarray:
        out = np.zeros((self.ncell, Q))
        self.lib.orc_get_f(self.h, int(comp), _dp(out))
        return out.reshape(self.shape + (Q,))

    def set_f(self, comp: int, f: np.ndarray):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncell, Q)
        self.lib.orc_set_f(self.h, int(comp), _dp(a))

    def set_active(self, act: np.ndarray):
        a = np.ascontiguousarray(act, dtype=np.uint8)
        self.lib.orc_set_active(self.h, a.ctypes.data_as(C.POINTER(C.c_ubyte)))

    def set_time(self, t: int):
        self.lib.orc_set_time(self.h, int(t))


def threads() -> int:
    """OpenMP threads the oracle will use."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)
