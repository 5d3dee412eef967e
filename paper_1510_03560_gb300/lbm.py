"""ctypes binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch
provides the device memory (its caching allocator, through the library's
allocator callbacks) and the CUDA stream.  There is no fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_CHECKED=1 selects the bounds-checked debug build (build(checked=True))
LIB_PATH = os.path.join(_PKG, "liblbm_checked.so" if os.environ.get("LBM_CHECKED") == "1"
                        else "liblbm.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT = 0, 1, 2, 3, 4, 5
EXEC = {"stream": 0, "graph": 1, "persistent": 2, "staged": 3}  # LBM_EXEC_*
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}  # LBM_STORAGE_*
STREAMING = {"ab": 0, "aa": 1}  # LBM_STREAM_*
Q = 19
EDGE = 8
SHAPES = ((8, 8, 8), (16, 8, 4), (16, 4, 8), (32, 4, 4))  # block shapes of the library

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ncomp", C.c_int),
        ("periodic", C.c_int * 3),
        ("progressive", C.c_int),
        ("storage", C.c_int),
        ("streaming", C.c_int),
        ("block", C.c_int * 3),
        ("tau", C.c_double), ("beta", C.c_double),
        ("pr_a", C.c_double), ("pr_b", C.c_double), ("pr_R", C.c_double), ("pr_omega", C.c_double),
        ("T_over_Tc", C.c_double),
        ("g_self", C.c_double), ("g_cross", C.c_double),
        ("g_ads", C.c_double * 2),
        ("grav", C.c_double * 3),
        ("rho_ref", C.c_double * 2),
        ("S", C.c_double),
        ("max_blocks", C.c_longlong),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", C.c_void_p),
        ("stream", C.c_void_p),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_longlong), ("active_blocks", C.c_longlong), ("capacity", C.c_longlong),
        ("total_blocks", C.c_longlong), ("nonsolid_blocks", C.c_longlong),
        ("cell_updates", C.c_longlong), ("fluid_updates", C.c_longlong),
        ("launches", C.c_longlong), ("device_bytes", C.c_longlong),
        ("kernel_ms", C.c_double * 4), ("kernel_launches", C.c_longlong * 4),
        ("created_blocks", C.c_longlong), ("prepared_blocks", C.c_longlong),
        ("prepared_hits", C.c_longlong), ("slot_sorts", C.c_longlong),
        ("fused_deferred", C.c_longlong), ("fused_waited", C.c_longlong),
        ("fused_lag_distance", C.c_longlong),
    ]


EXPORTS = ["lbm_create", "lbm_destroy", "lbm_set_geometry", "lbm_step", "lbm_step_async",
           "lbm_sync", "lbm_get_macro", "lbm_active_blocks", "lbm_mass",
           "lbm_get_block_populations", "lbm_velocities", "lbm_set_profiling", "lbm_get_stats",
           "lbm_last_error", "lbm_mass_noalloc", "lbm_frontier_features", "lbm_activation_steps",
           "lbm_mlp_create", "lbm_mlp_destroy", "lbm_mlp_set_params", "lbm_mlp_get_params",
           "lbm_mlp_set_scaling", "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_adam",
           "lbm_set_proposer", "lbm_set_exec", "lbm_barrier_selftest", "lbm_set_slot_order",
           "lbm_set_slot_strip", "lbm_set_fusion", "lbm_set_density_partials"]
NOALLOC_MAX_BLOCKS = 65536
MLP_IN, MLP_HIDDEN = 34, 64
MLP_NPARAM = MLP_IN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + 2 * MLP_HIDDEN + 1

_lib = None


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


def load():
    """Load liblbm.so (built by paper_1510_03560_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1510_03560_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, ip, fp, dp, u8p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float), \
        C.POINTER(C.c_double), C.POINTER(C.c_uint8)
    lib.lbm_create.argtypes = [C.POINTER(Params), C.POINTER(vp)]
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_set_geometry.argtypes = [vp, u8p, fp, fp, fp]
    lib.lbm_step.argtypes = [vp, C.c_int]
    lib.lbm_step_async.argtypes = [vp, C.c_int]
    lib.lbm_sync.argtypes = [vp]
    lib.lbm_get_macro.argtypes = [vp, C.c_int, fp, fp, fp, fp]
    lib.lbm_active_blocks.argtypes = [vp, ip, C.c_longlong, C.POINTER(C.c_longlong)]
    lib.lbm_mass.argtypes = [vp, dp]
    lib.lbm_get_block_populations.argtypes = [vp, C.c_int32, fp]
    lib.lbm_velocities.argtypes = [ip]
    lib.lbm_set_profiling.argtypes = [vp, C.c_int]
    lib.lbm_get_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = C.c_char_p
    lib.lbm_mass_noalloc.argtypes = [vp, vp, C.c_longlong, C.c_int, dp, vp]
    lib.lbm_frontier_features.argtypes = [vp, ip, fp, C.c_longlong, C.POINTER(C.c_longlong)]
    lib.lbm_activation_steps.argtypes = [vp, ip]
    lib.lbm_mlp_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
    lib.lbm_mlp_destroy.argtypes = [vp]
    lib.lbm_mlp_set_params.argtypes = [vp, fp]
    lib.lbm_mlp_get_params.argtypes = [vp, fp]
    lib.lbm_mlp_set_scaling.argtypes = [vp, fp, fp]
    lib.lbm_mlp_forward.argtypes = [vp, vp, C.c_int, C.c_int, vp]
    lib.lbm_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, dp, fp]
    lib.lbm_mlp_adam.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int]
    lib.lbm_set_proposer.argtypes = [vp, vp, C.c_int, C.c_float]
    lib.lbm_set_exec.argtypes = [vp, C.c_int]
    lib.lbm_barrier_selftest.argtypes = [C.c_int, C.c_longlong]
    lib.lbm_set_slot_order.argtypes = [vp, C.c_int]
    lib.lbm_set_slot_strip.argtypes = [vp, C.c_int]
    lib.lbm_set_fusion.argtypes = [vp, C.c_int, C.c_int]
    lib.lbm_set_density_partials.argtypes = [vp, C.c_int]
    for name in EXPORTS:
        if name != "lbm_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def mass_noalloc(f_ptr: int, solid_ptr, nblocks: int, ncomp: int, stream_ptr=None) -> np.ndarray:
    """lbm_mass_noalloc on a caller-held device population pool (device
    pointers as ints); allocates nothing on the device."""
    lib = load()
    m = np.zeros(2)
    rc = lib.lbm_mass_noalloc(C.c_void_p(f_ptr), C.c_void_p(solid_ptr) if solid_ptr else None,
                              int(nblocks), int(ncomp), m.ctypes.data_as(C.POINTER(C.c_double)),
                              C.c_void_p(stream_ptr) if stream_ptr else None)
    if rc != OK:
        raise LBMError(rc, lib.lbm_last_error(None).decode())
    return m[:ncomp].copy()


def velocities() -> np.ndarray:
    e = np.zeros((Q, 3), dtype=np.int32)
    load().lbm_velocities(e.ctypes.data_as(C.POINTER(C.c_int32)))
    return e


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


class _TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, torch, device, stream):
        self.torch = torch
        self.device = device
        self.stream = stream

        def alloc(nbytes, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def free(ptr, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class LBM:
    """One simulation context (lbm_ctx).

    Keyword parameters mirror lbm_params: nx, ny, nz, ncomp, periodic,
    progressive, storage ("fp32", "fp16", "bf16" or the LBM_STORAGE_* code),
    streaming ("ab" or "aa", the LBM_STREAM_* pattern), block (cells per
    block along x, y, z: one of SHAPES),
    tau, beta, pr_a, pr_b, pr_R, pr_omega, T_over_Tc, g_self, g_cross, g_ads,
    grav, rho_ref, S, max_blocks.  ``stream``: a
    torch.cuda.Stream (default: the current stream).  ``torch_alloc``:
    allocate through torch's caching allocator (default) or let the library
    use cudaMallocAsync.  ``slot_strip`` (lbm_set_slot_strip, before the
    geometry), ``fusion`` = (on, max_lag) (lbm_set_fusion) and ``partials``
    (lbm_set_density_partials) are applied right after the context is
    created when given.
    """

    def __init__(self, stream=None, torch_alloc=True, **kw):
        import torch
        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA GPU")
        self.device = torch.cuda.current_device()
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        p = Params()
        p.nx, p.ny, p.nz = int(kw["nx"]), int(kw["ny"]), int(kw["nz"])
        self.shape = (p.nz, p.ny, p.nx)
        blk = tuple(int(v) for v in kw.get("block", (8, 8, 8)))
        for a in range(3):
            p.block[a] = blk[a]
        self.block = blk
        self.nblocks = (p.nx // blk[0]) * (p.ny // blk[1]) * (p.nz // blk[2])
        p.ncomp = int(kw.get("ncomp", 2))
        self.ncomp = p.ncomp
        per = kw.get("periodic", (1, 1, 0))
        for a in range(3):
            p.periodic[a] = int(per[a])
        p.progressive = int(kw.get("progressive", 1))
        st = kw.get("storage", 0)
        p.storage = STORAGE[st] if isinstance(st, str) else int(st)
        self.storage = p.storage
        sp = kw.get("streaming", 0)
        p.streaming = STREAMING[sp] if isinstance(sp, str) else int(sp)
        self.streaming = p.streaming
        p.tau = float(kw.get("tau", 1.0))
        p.beta = float(kw.get("beta", 1.16))
        p.pr_a = float(kw.get("pr_a", 2.0 / 49.0))
        p.pr_b = float(kw.get("pr_b", 2.0 / 21.0))
        p.pr_R = float(kw.get("pr_R", 1.0))
        p.pr_omega = float(kw.get("pr_omega", 0.344))
        p.T_over_Tc = float(kw.get("T_over_Tc", 0.85))
        p.g_self = float(kw.get("g_self", -1.0))
        p.g_cross = float(kw.get("g_cross", 0.0))
        ga = kw.get("g_ads", (0.0, 0.0))
        p.g_ads[0], p.g_ads[1] = float(ga[0]), float(ga[1])
        g = kw.get("grav", (0.0, 0.0, 0.0))
        for d in range(3):
            p.grav[d] = float(g[d])
        rr = kw.get("rho_ref", (0.0, 0.0))
        p.rho_ref[0] = float(rr[0])
        p.rho_ref[1] = float(rr[1]) if len(rr) > 1 else 0.0
        p.S = float(kw.get("S", 0.0))
        p.max_blocks = int(kw.get("max_blocks", 0))
        strip = kw.get("slot_strip", None)
        fusion = kw.get("fusion", None)
        partials = kw.get("partials", None)
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(torch, self.device, self.torch_stream.cuda_stream)
            p.dev_alloc = self._alloc.alloc
            p.dev_free = self._alloc.free
        p.stream = self.torch_stream.cuda_stream
        self.params = p
        h = C.c_void_p()
        rc = self.lib.lbm_create(C.byref(p), C.byref(h))
        if rc != OK:
            raise LBMError(rc, self.lib.lbm_last_error(None).decode())
        self.h = h
        if strip is not None:
            self.set_slot_strip(strip)
        if fusion is not None:
            self.set_fusion(*fusion)
        if partials is not None:
            self.set_density_partials(partials)

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != OK:
            raise LBMError(rc, self.lib.lbm_last_error(self.h).decode())

    # -- API
    def set_geometry(self, cell_type, rho_init, u_init, rho_amb):
        ct = np.ascontiguousarray(cell_type, dtype=np.uint8)
        assert ct.shape == self.shape
        self._keep = (ct, _f32(rho_init), None if u_init is None else _f32(u_init), _f32(rho_amb))
        ct, ri, ui, ra = self._keep
        self._check(self.lib.lbm_set_geometry(self.h, ct.ctypes.data_as(C.POINTER(C.c_uint8)),
                                              _fptr(ri), _fptr(ui), _fptr(ra)))

    def step(self, n: int = 1):
        self._check(self.lib.lbm_step(self.h, int(n)))

    def step_async(self, n: int = 1):
        self._check(self.lib.lbm_step_async(self.h, int(n)))

    def sync(self):
        self._check(self.lib.lbm_sync(self.h))

    def macro(self, comp: int):
        out = [np.zeros(self.shape, dtype=np.float32) for _ in range(4)]
        self._check(self.lib.lbm_get_macro(self.h, int(comp), *[_fptr(a) for a in out]))
        return tuple(out)

    def active_blocks(self) -> np.ndarray:
        n = C.c_longlong()
        self._check(self.lib.lbm_active_blocks(self.h, None, 0, C.byref(n)))
        ids = np.zeros(max(n.value, 1), dtype=np.int32)
        self._check(self.lib.lbm_active_blocks(self.h, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                               n.value, C.byref(n)))
        return ids[: n.value].copy()

    def mass(self) -> np.ndarray:
        m = np.zeros(2)
        self._check(self.lib.lbm_mass(self.h, m.ctypes.data_as(C.POINTER(C.c_double))))
        return m[: self.ncomp].copy()

    def block_populations(self, block_id: int) -> np.ndarray:
        out = np.zeros((self.ncomp, Q, 512), dtype=np.float32)
        self._check(self.lib.lbm_get_block_populations(self.h, int(block_id), _fptr(out)))
        return out

    def set_profiling(self, on: bool):
        self._check(self.lib.lbm_set_profiling(self.h, 1 if on else 0))

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.lbm_get_stats(self.h, C.byref(s)))
        d = {k: getattr(s, k) for k, _ in Stats._fields_ if k not in ("kernel_ms", "kernel_launches")}
        d["kernel_ms"] = list(s.kernel_ms)
        d["kernel_launches"] = list(s.kernel_launches)
        return d


def _lbm_frontier_features(self):
    """Frontier blocks (ascending) and their LBM_MLP_IN features."""
    n = C.c_longlong(0)
    self._check(self.lib.lbm_frontier_features(self.h, None, None, 0, C.byref(n)))
    cap = n.value
    ids = np.zeros(max(cap, 1), dtype=np.int32)
    feat = np.zeros((max(cap, 1), MLP_IN), dtype=np.float32)
    self._check(self.lib.lbm_frontier_features(self.h, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                               _fptr(feat), cap, C.byref(n)))
    m = min(cap, n.value)
    return ids[:m].copy(), feat[:m].copy()


def _lbm_activation_steps(self):
    """Per block: 0 initial, t + 1 when created in step t, -1 unmeshed."""
    out = np.zeros(self.nblocks, dtype=np.int32)
    self._check(self.lib.lbm_activation_steps(self.h, out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out


def _lbm_set_proposer(self, mlp, period=16, threshold=0.5):
    """Use an MLP (or None to turn the proposer off)."""
    self._proposer = mlp
    self._check(self.lib.lbm_set_proposer(self.h, None if mlp is None else mlp.h, int(period),
                                          float(threshold)))


def _lbm_set_exec(self, mode):
    """"stream", "graph", "persistent" or "staged" (or the LBM_EXEC_* code)."""
    self._check(self.lib.lbm_set_exec(self.h, EXEC[mode] if isinstance(mode, str) else int(mode)))


def barrier_selftest(missing: int, spins: int) -> int:
    """Status of one bounded grid barrier that expects `missing` extra CTAs."""
    return load().lbm_barrier_selftest(int(missing), int(spins))


LBM.set_exec = _lbm_set_exec


def _lbm_set_slot_order(self, period: int):
    """Check for renumbering the meshed slots in block order every `period`
    steps (0 = never; lbm_set_slot_order)."""
    self._check(self.lib.lbm_set_slot_order(self.h, int(period)))


LBM.set_slot_order = _lbm_set_slot_order


def _lbm_set_slot_strip(self, rows: int):
    """Slot order: strips of `rows` block rows (0 block order, -1 automatic;
    lbm_set_slot_strip; applies at the next set_geometry and renumbering)."""
    self._check(self.lib.lbm_set_slot_strip(self.h, int(rows)))


def _lbm_set_fusion(self, on: bool = True, max_lag: int = 0):
    """Collision of a step and pass 1 of the next in one launch (lbm_set_fusion)."""
    self._check(self.lib.lbm_set_fusion(self.h, 1 if on else 0, int(max_lag)))


def _lbm_set_density_partials(self, on: bool = True):
    """Pass 1 sums the densities the collision prepared instead of pulling
    (lbm_set_density_partials)."""
    self._check(self.lib.lbm_set_density_partials(self.h, 1 if on else 0))


LBM.set_slot_strip = _lbm_set_slot_strip
LBM.set_fusion = _lbm_set_fusion
LBM.set_density_partials = _lbm_set_density_partials
LBM.frontier_features = _lbm_frontier_features
LBM.activation_steps = _lbm_activation_steps
LBM.set_proposer = _lbm_set_proposer


class MLP:
    """lbm_mlp: the activation proposer's network, trained and run by the
    library's kernels.  Data arrays are torch CUDA tensors (float32)."""

    def __init__(self, max_batch: int, stream=None):
        import torch
        self.lib = load()
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = self.lib.lbm_mlp_create(int(max_batch), C.c_void_p(self.torch_stream.cuda_stream),
                                     C.byref(h))
        if rc != OK:
            raise LBMError(rc, self.lib.lbm_last_error(None).decode())
        self.h = h
        self.max_batch = int(max_batch)

    def _check(self, rc):
        if rc != OK:
            raise LBMError(rc, self.lib.lbm_last_error(None).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.shape == (MLP_NPARAM,)
        self._check(self.lib.lbm_mlp_set_params(self.h, _fptr(p)))

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(self.lib.lbm_mlp_get_params(self.h, _fptr(p)))
        return p

    def set_scaling(self, mean, scale):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        assert m.shape == (MLP_IN,) and sc.shape == (MLP_IN,)
        self._check(self.lib.lbm_mlp_set_scaling(self.h, _fptr(m), _fptr(sc)))

    def forward(self, x, bf16: bool = False):
        import torch
        x = x.contiguous()
        n = x.shape[0]
        prob = torch.empty(n, dtype=torch.float32, device=x.device)
        self._check(self.lib.lbm_mlp_forward(self.h, C.c_void_p(x.data_ptr()), n, 1 if bf16 else 0,
                                             C.c_void_p(prob.data_ptr())))
        return prob

    def loss_grad(self, x, y, want_grad: bool = False):
        x, y = x.contiguous(), y.contiguous()
        loss = C.c_double(0.0)
        g = np.zeros(MLP_NPARAM, dtype=np.float32) if want_grad else None
        self._check(self.lib.lbm_mlp_loss_grad(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                               int(x.shape[0]), C.byref(loss),
                                               _fptr(g) if g is not None else None))
        return loss.value, g

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.lbm_mlp_adam(self.h, float(lr), float(beta1), float(beta2), float(eps), int(t)))


def from_case(case, **over):
    """Context + geometry from a workloads case dict.  The case's block
    shape is used when the library has it (SHAPES), else 8^3."""
    p = dict(case["params"])
    blk = p.pop("block", None)
    if blk is not None and tuple(blk) in SHAPES:
        p["block"] = tuple(blk)
    p.update(over)
    sim = LBM(**p)
    sim.set_geometry(case["cell_type"], case["rho_init"], case["u_init"], case["rho_amb"])
    return sim
