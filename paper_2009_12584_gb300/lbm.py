"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: PyTorch provides the device memory (the workspace
and the caller's arrays) and the CUDA stream; every step of the computation
runs in the CUDA library ``liblbm_gb300.so``. There is no CPU fallback: if
the library has not been built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_SPACE, ERR_TIMEOUT = range(6)
WET_MARTYS_CHEN, WET_LLKC, WET_VIRTUAL_AVG, WET_CONSTANT = range(4)
PAIR_CROSS, PAIR_SELF = 0, 1
STORAGE = {"fp32": 0, "fp64": 1, "fp16": 2, "bf16": 3}
KERNEL = {"auto": 0, "two_pass": 1, "fused": 2, "tiled": 3, "halo": 4, "tma": 5}
WETTING = {"martys_chen": 0, "mc": 0, "llkc": 1, "virtual_avg": 2, "improved": 2, "constant": 3}


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("tau", ctypes.c_double * 2), ("G_AB", ctypes.c_double),
        ("storage", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("rho_ref", ctypes.c_double * 2), ("max_interface", ctypes.c_int64),
        ("velocity_refs", ctypes.c_int32),
    ]


class LbmWetting(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("pairing", ctypes.c_int32),
        ("avg_stencil", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("G_s", ctypes.c_double * 2), ("chi", ctypes.c_double * 2),
        ("rho_s", ctypes.c_double * 2),
    ]


class LbmDiagParams(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("tangent", ctypes.c_double * 2), ("wall_point", ctypes.c_double * 2),
        ("wall_angle_deg", ctypes.c_double), ("exclude", ctypes.c_double),
        ("box", ctypes.c_double * 4), ("bridge_x", ctypes.c_int32), ("bridge_y0", ctypes.c_int32),
    ]


class LbmDiag(ctypes.Structure):
    _fields_ = [
        ("weight", ctypes.c_double), ("com", ctypes.c_double * 2),
        ("com_velocity", ctypes.c_double * 2), ("sliding_velocity", ctypes.c_double),
        ("max_u", ctypes.c_double), ("contour_points", ctypes.c_int64),
        ("circle", ctypes.c_double * 3), ("contact_angle_deg", ctypes.c_double),
        ("bridge_radius", ctypes.c_double), ("nonfinite_nodes", ctypes.c_int64),
    ]


EXPORTS = [
    "lbm_workspace_bytes", "lbm_create", "lbm_set_stream", "lbm_set_geometry", "lbm_set_wetting",
    "lbm_init_fields", "lbm_step", "lbm_step_profiled", "lbm_moments", "lbm_forces", "lbm_get_populations",
    "lbm_set_populations", "lbm_mass", "lbm_diagnostics", "lbm_set_l2_fetch_granularity", "lbm_interface_count",
    "lbm_sync", "lbm_run_host", "lbm_run_host_f32", "lbm_debug_tma_expect_extra",
    "lbm_destroy", "lbm_status_str", "lbm_last_error", "lbm_launch_count",
    "lbm_batch_workspace_bytes", "lbm_batch_create", "lbm_batch_set_graph_steps", "lbm_batch_step",
    "lbm_batch_autotune", "lbm_batch_set_schedule", "lbm_batch_config", "lbm_batch_launch_count",
    "lbm_batch_last_error", "lbm_batch_destroy",
]

_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_str(status)}) {detail}".strip())


def _status_str(s):
    try:
        return load().lbm_status_str(s).decode()
    except Exception:  # pragma: no cover - only while reporting another error
        return "?"


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Open the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2009_12584_gb300.build` "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        P = ctypes.POINTER(LbmParams)
        W = ctypes.POINTER(LbmWetting)
        sig = {
            "lbm_workspace_bytes": [P, ctypes.POINTER(ctypes.c_size_t)],
            "lbm_create": [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
            "lbm_set_stream": [vp, vp],
            "lbm_set_geometry": [vp, vp],
            "lbm_set_wetting": [vp, W],
            "lbm_init_fields": [vp, dp, dp, dp, dp],
            "lbm_step": [vp, i32],
            "lbm_step_profiled": [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)],
            "lbm_moments": [vp, dp, dp, dp, dp],
            "lbm_forces": [vp, dp],
            "lbm_get_populations": [vp, dp],
            "lbm_set_populations": [vp, dp],
            "lbm_mass": [vp, ctypes.POINTER(ctypes.c_double)],
            "lbm_diagnostics": [vp, ctypes.POINTER(LbmDiagParams), ctypes.POINTER(LbmDiag)],
            "lbm_set_l2_fetch_granularity": [i32, ctypes.POINTER(i32)],
            "lbm_interface_count": [vp, ctypes.POINTER(i64)],
            "lbm_sync": [vp],
            "lbm_debug_tma_expect_extra": [vp, i32],
            "lbm_run_host": [vp, W, vp, vp, vp, i32, vp, vp, vp, vp],
            "lbm_run_host_f32": [vp, W, vp, vp, vp, i32, vp, vp, vp, vp],
            "lbm_destroy": [vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.lbm_status_str.argtypes = [ctypes.c_int]
        lib.lbm_status_str.restype = ctypes.c_char_p
        lib.lbm_last_error.argtypes = [vp]
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_launch_count.argtypes = [vp]
        lib.lbm_launch_count.restype = ctypes.c_int64
        ctxs = ctypes.POINTER(vp)
        for name, args in {
            "lbm_batch_workspace_bytes": [i32, ctxs, ctypes.POINTER(ctypes.c_size_t)],
            "lbm_batch_create": [i32, ctxs, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
            "lbm_batch_set_graph_steps": [vp, i32],
            "lbm_batch_step": [vp, i32],
            "lbm_batch_autotune": [vp, i32, ctypes.POINTER(i32)],
            "lbm_batch_set_schedule": [vp, i32],
            "lbm_batch_config": [vp, ctypes.POINTER(i32)],
            "lbm_batch_destroy": [vp],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.lbm_batch_launch_count.argtypes = [vp]
        lib.lbm_batch_launch_count.restype = ctypes.c_int64
        lib.lbm_batch_last_error.argtypes = [vp]
        lib.lbm_batch_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def set_l2_fetch_granularity(nbytes: int) -> int:
    """Set the L2 fetch granularity hint of the current CUDA device's context
    (32, 64 or 128 bytes; lbm_set_l2_fetch_granularity) and return the
    previous value. It applies to every kernel of this process on that
    device; the library never sets it by itself. On porous geometries 128
    bytes is fastest for the tiled schedule (the default for FP32/FP64) and
    the batched one, 32 bytes for the two-pass schedule."""
    lib = load()
    prev = ctypes.c_int32()
    st = lib.lbm_set_l2_fetch_granularity(int(nbytes), ctypes.byref(prev))
    if st != OK:
        raise LbmError(st, "lbm_set_l2_fetch_granularity")
    return prev.value


def make_params(nx, ny, *, tau=(1.0, 1.0), G_AB=3.0, periodic_x=False, periodic_y=False,
                storage="fp32", kernel="auto", rho_ref=(1.0, 1.0), max_interface=0,
                velocity_refs=False) -> LbmParams:
    """lbm_params of the C ABI. kernel: "auto" (tiled for fp32/fp64, two-pass
    for fp16/bf16), "two_pass", "fused" (marching single pass, fp32/fp64) or
    "tiled"; every schedule gives the same results bit for bit."""
    p = LbmParams()
    p.nx, p.ny = int(nx), int(ny)
    p.periodic_x, p.periodic_y = int(bool(periodic_x)), int(bool(periodic_y))
    p.tau[0], p.tau[1] = tau
    p.G_AB = G_AB
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    p.rho_ref[0], p.rho_ref[1] = rho_ref
    p.max_interface = int(max_interface)
    p.velocity_refs = int(bool(velocity_refs))
    return p


def make_wetting(kind="martys_chen", *, G_s=(0.0, 0.0), chi=(1.0, 1.0), rho_s=(0.0, 0.0),
                 pairing=PAIR_CROSS, avg_stencil=25) -> LbmWetting:
    w = LbmWetting()
    w.kind = WETTING[kind] if isinstance(kind, str) else int(kind)
    w.pairing = int(pairing)
    w.avg_stencil = int(avg_stencil)
    w.G_s[0], w.G_s[1] = G_s
    w.chi[0], w.chi[1] = chi
    w.rho_s[0], w.rho_s[1] = rho_s
    return w


def workspace_bytes(params: LbmParams) -> int:
    n = ctypes.c_size_t()
    st = load().lbm_workspace_bytes(ctypes.byref(params), ctypes.byref(n))
    if st:
        raise LbmError(st, "lbm_workspace_bytes")
    return n.value


class Simulation:
    """One simulation context on the current CUDA device and stream."""

    def __init__(self, nx, ny, *, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2009_12584_gb300 needs a CUDA GPU (there is no CPU fallback)")
        self.torch = torch
        self.lib = load()
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(nx, ny, **kw)
        self.storage = kw.get("storage", "fp32")
        nbytes = workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        self._check(self.lib.lbm_create(ctypes.byref(self.params), self.workspace.data_ptr(), nbytes,
                                        self.stream.cuda_stream, ctypes.byref(h)), "lbm_create", ctx=False)
        self.h = h
        self.mask = None

    # -- helpers -----------------------------------------------------------------
    def _check(self, st, where, ctx=True):
        if st != OK:
            detail = ""
            if ctx and getattr(self, "h", None):
                detail = self.lib.lbm_last_error(self.h).decode()
            raise LbmError(st, where, detail)

    def _dev(self, a, dtype):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        return a.to(device="cuda", dtype=dtype).contiguous()

    # -- API -----------------------------------------------------------------------
    def set_geometry(self, mask):
        self.mask = self._dev(mask, self.torch.uint8).reshape(self.ny, self.nx)
        self._check(self.lib.lbm_set_geometry(self.h, self.mask.data_ptr()), "lbm_set_geometry")
        return self

    def set_wetting(self, kind="martys_chen", **kw):
        self.wetting = make_wetting(kind, **kw)
        self._check(self.lib.lbm_set_wetting(self.h, ctypes.byref(self.wetting)), "lbm_set_wetting")
        return self

    def init_fields(self, rhoA, rhoB, ux=None, uy=None):
        f64 = self.torch.float64
        self._init = [self._dev(a, f64) if a is not None else None for a in (rhoA, rhoB, ux, uy)]
        ptr = [a.data_ptr() if a is not None else None for a in self._init]
        self._check(self.lib.lbm_init_fields(self.h, *ptr), "lbm_init_fields")
        return self

    def step(self, n=1):
        self._check(self.lib.lbm_step(self.h, int(n)), "lbm_step")
        return self

    def step_profiled(self, n):
        """Advance n steps timing every kernel; returns (ms, launches) dicts
        keyed by kernel class (density, virtual, collide, fused)."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        self._check(self.lib.lbm_step_profiled(self.h, int(n), ms, cnt), "lbm_step_profiled")
        names = ("density", "virtual", "collide", "fused")
        return dict(zip(names, list(ms))), dict(zip(names, list(cnt)))

    def moments(self):
        t = self.torch
        out = t.empty((4, self.ny, self.nx), dtype=t.float64, device="cuda")
        ptrs = [out[i].data_ptr() for i in range(4)]
        self._check(self.lib.lbm_moments(self.h, *ptrs), "lbm_moments")
        return out[0], out[1], out[2:4]

    def forces(self):
        t = self.torch
        out = t.empty((2, 2, self.ny, self.nx), dtype=t.float64, device="cuda")
        self._check(self.lib.lbm_forces(self.h, out.data_ptr()), "lbm_forces")
        return out

    def populations(self):
        t = self.torch
        out = t.empty((2, 9, self.ny, self.nx), dtype=t.float64, device="cuda")
        self._check(self.lib.lbm_get_populations(self.h, out.data_ptr()), "lbm_get_populations")
        return out

    def set_populations(self, f):
        self._setf = self._dev(f, self.torch.float64).reshape(2, 9, self.ny, self.nx)
        self._check(self.lib.lbm_set_populations(self.h, self._setf.data_ptr()), "lbm_set_populations")
        return self

    def mass(self):
        out = (ctypes.c_double * 2)()
        self._check(self.lib.lbm_mass(self.h, out), "lbm_mass")
        return np.array([out[0], out[1]])

    def diagnostics(self, *, level=0.5, rho_out=0.055, tangent=(1.0, 0.0), wall_point=(0.0, 0.5),
                    wall_angle_deg=0.0, exclude=3.0, box=None, bridge=None) -> dict:
        """Device-side measurements of the current state (lbm_diagnostics):
        weighted centre of mass and its velocity, sliding velocity along
        ``tangent``, max |u|, circle fit of the rho^A = ``level`` contour and
        the contact angle on the wall line through ``wall_point`` at
        ``wall_angle_deg``, and the bridge radius on column ``bridge[0]``
        above the first fluid row ``bridge[1]``. ``box`` = (x0, x1, y0, y1)
        keeps only contour points inside it."""
        p = LbmDiagParams()
        p.level, p.rho_out = level, rho_out
        p.tangent[0], p.tangent[1] = tangent
        p.wall_point[0], p.wall_point[1] = wall_point
        p.wall_angle_deg, p.exclude = wall_angle_deg, exclude
        b = box if box is not None else (1.0, 0.0, 0.0, 0.0)
        for i in range(4):
            p.box[i] = b[i]
        p.bridge_x, p.bridge_y0 = bridge if bridge is not None else (-1, 0)
        o = LbmDiag()
        self._check(self.lib.lbm_diagnostics(self.h, ctypes.byref(p), ctypes.byref(o)), "lbm_diagnostics")
        return {
            "weight": o.weight, "com": (o.com[0], o.com[1]),
            "com_velocity": (o.com_velocity[0], o.com_velocity[1]),
            "sliding_velocity": o.sliding_velocity, "max_u": o.max_u,
            "contour_points": o.contour_points, "circle": (o.circle[0], o.circle[1], o.circle[2]),
            "contact_angle_deg": o.contact_angle_deg, "bridge_radius": o.bridge_radius,
            "nonfinite_nodes": o.nonfinite_nodes,
        }

    def interface_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.lbm_interface_count(self.h, ctypes.byref(n)), "lbm_interface_count")
        return n.value

    def sync(self):
        self._check(self.lib.lbm_sync(self.h), "lbm_sync")

    def debug_tma_expect_extra(self, nbytes):
        """Test hook of the TMA schedule's bounded wait (see lbm.h)."""
        self._check(self.lib.lbm_debug_tma_expect_extra(self.h, int(nbytes)), "lbm_debug_tma_expect_extra")
        return self

    @property
    def launch_count(self):
        return self.lib.lbm_launch_count(self.h)

    def run_host(self, wetting: LbmWetting, mask, rhoA, rhoB, nsteps, outputs=None):
        """End-to-end call on host arrays (pinned torch CPU tensors or numpy)."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                return a.ctypes.data
            return a.data_ptr()
        outs = outputs if outputs is not None else [None] * 4
        self._check(self.lib.lbm_run_host(self.h, ctypes.byref(wetting), hp(mask), hp(rhoA), hp(rhoB),
                                          int(nsteps), *[hp(o) for o in outs]), "lbm_run_host")

    def run_host_f32(self, wetting: LbmWetting, mask, rhoA, rhoB, nsteps, outputs=None):
        """run_host with FP32 host arrays (densities in; rho^A, rho^B, u_x,
        u_y out): half the transfer bytes (lbm_run_host_f32)."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                assert a.dtype in (np.float32, np.uint8)
                return a.ctypes.data
            return a.data_ptr()
        outs = outputs if outputs is not None else [None] * 4
        self._check(self.lib.lbm_run_host_f32(self.h, ctypes.byref(wetting), hp(mask), hp(rhoA), hp(rhoB),
                                              int(nsteps), *[hp(o) for o in outs]), "lbm_run_host_f32")

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent simulations advanced together: one launch per kernel
    class per step for all of them, replayed from a CUDA graph."""

    def __init__(self, sims, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.sims = list(sims)
        n = len(self.sims)
        self._arr = (ctypes.c_void_p * n)(*[s.h.value for s in self.sims])
        nbytes = ctypes.c_size_t()
        st = self.lib.lbm_batch_workspace_bytes(n, self._arr, ctypes.byref(nbytes))
        if st:
            raise LbmError(st, "lbm_batch_workspace_bytes")
        self.workspace = torch.empty(max(256, nbytes.value), dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.lbm_batch_create(n, self._arr, self.workspace.data_ptr(), self.workspace.numel(),
                                       self.stream.cuda_stream, ctypes.byref(h))
        if st:
            raise LbmError(st, "lbm_batch_create")
        self.h = h

    def _check(self, st, where):
        if st != OK:
            raise LbmError(st, where, self.lib.lbm_batch_last_error(self.h).decode())

    def set_graph_steps(self, steps):
        self._check(self.lib.lbm_batch_set_graph_steps(self.h, int(steps)), "lbm_batch_set_graph_steps")
        return self

    def step(self, n=1):
        self._check(self.lib.lbm_batch_step(self.h, int(n)), "lbm_batch_step")
        return self

    def autotune(self, trial_steps=32):
        """Pick threads per block and steps per graph replay by timing; the
        members advance by the timed steps. Returns (threads, steps)."""
        ch = (ctypes.c_int32 * 2)()
        self._check(self.lib.lbm_batch_autotune(self.h, int(trial_steps), ch), "lbm_batch_autotune")
        return int(ch[0]), int(ch[1])

    def set_schedule(self, kernel):
        """"two_pass" (default) or "tiled" (4-/8-byte storage)."""
        self._check(self.lib.lbm_batch_set_schedule(self.h, KERNEL[kernel] if isinstance(kernel, str) else int(kernel)),
                    "lbm_batch_set_schedule")
        return self

    def config(self):
        """(schedule name, threads per block, steps per graph replay)."""
        c = (ctypes.c_int32 * 3)()
        self._check(self.lib.lbm_batch_config(self.h, c), "lbm_batch_config")
        names = {v: k for k, v in KERNEL.items()}
        return names[c[0]], int(c[1]), int(c[2])

    @property
    def launch_count(self):
        return self.lib.lbm_batch_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
