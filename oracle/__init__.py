"""FP64 CPU oracle of the two-component Shan-Chen D2Q9 step with wetting
boundary conditions (arXiv:2009.12584, Sec. 2), wrapped for numpy.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library
and its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``lbm_oracle.c`` (plain loops in double precision);
this module compiles it with the host C compiler on first use and marshals
numpy arrays. Array conventions are those of ``lbm_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

BC_MARTYS_CHEN = 0
BC_LLKC = 1
BC_VIRTUAL_AVG = 2
BC_CONSTANT = 3
PAIR_CROSS = 0
PAIR_SELF = 1


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int),
        ("periodic_y", ctypes.c_int),
        ("tau", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double),
        ("bc", ctypes.c_int),
        ("pairing", ctypes.c_int),
        ("G_s", ctypes.c_double * 2),
        ("chi", ctypes.c_double * 2),
        ("rho_s", ctypes.c_double * 2),
        ("avg_stencil", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math"]
        # OpenMP over nodes (bit-identical to a serial build); a compiler
        # without it gets the serial build
        r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            # idle OpenMP threads sleep instead of spinning, so that several
            # processes sharing the cores (parallel test ranks) do not starve
            # one another; read once, when the OpenMP runtime starts
            os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
            _lib = load_library(_LIB_PATH)
    return _lib


def load_library(path):
    """Open an oracle shared library at ``path`` (the tests also load copies
    compiled with a planted mistake, to show that the pins catch it)."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(OracleParams)
    d = ctypes.POINTER(ctypes.c_double)
    u8 = ctypes.POINTER(ctypes.c_ubyte)
    i32 = ctypes.POINTER(ctypes.c_int)
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_lattice.argtypes = [i32, i32, d, i32]
    lib.oracle_d2q25.argtypes = [i32, i32, d]
    lib.oracle_d2q25.restype = ctypes.c_int
    lib.oracle_check.argtypes = [P, u8]
    lib.oracle_check.restype = ctypes.c_int
    lib.oracle_equilibrium.argtypes = [ctypes.c_double] * 3 + [d]
    lib.oracle_source.argtypes = [ctypes.c_double] * 5 + [d]
    lib.oracle_densities.argtypes = [P, u8, d, d]
    lib.oracle_interface_solid.argtypes = [P, u8, u8]
    lib.oracle_virtual_density.argtypes = [P, u8, d, d]
    lib.oracle_forces.argtypes = [P, u8, d, d, d]
    lib.oracle_velocity.argtypes = [P, u8, d, d, d, d]
    lib.oracle_fields.argtypes = [P, u8, d, d, d, d, d]
    lib.oracle_collide.argtypes = [P, u8, d, d, d, d, d]
    lib.oracle_stream.argtypes = [P, u8, d, d]
    lib.oracle_init.argtypes = [P, u8, d, d, d, d, d]
    lib.oracle_init.restype = ctypes.c_int
    lib.oracle_step.argtypes = [P, u8, d, ctypes.c_int]
    lib.oracle_step.restype = ctypes.c_int
    lib.oracle_mass.argtypes = [P, u8, d, d]
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _mp(m: np.ndarray):
    assert m.dtype == np.uint8 and m.flags.c_contiguous
    return m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def set_threads(n: int = 0, lib=None) -> int:
    """Threads of the oracle's parallel node loops (0: one per core); the
    results do not depend on it. Returns the count in effect."""
    return (lib or _load()).oracle_set_threads(int(n))


def max_threads(lib=None) -> int:
    return (lib or _load()).oracle_max_threads()


def lattice(lib=None):
    """D2Q9 tables: (cx, cy, w, opp)."""
    lib = lib or _load()
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9)
    opp = np.zeros(9, np.int32)
    i32 = ctypes.POINTER(ctypes.c_int)
    lib.oracle_lattice(cx.ctypes.data_as(i32), cy.ctypes.data_as(i32), _dp(w),
                       opp.ctypes.data_as(i32))
    return cx, cy, w, opp


def d2q25(lib=None):
    """The 24 averaging vectors and weights of Eq. 8: (ex, ey, W)."""
    lib = lib or _load()
    ex = np.zeros(24, np.int32)
    ey = np.zeros(24, np.int32)
    W = np.zeros(24)
    i32 = ctypes.POINTER(ctypes.c_int)
    k = lib.oracle_d2q25(ex.ctypes.data_as(i32), ey.ctypes.data_as(i32), _dp(W))
    assert k == 24
    return ex, ey, W


def equilibrium(rho: float, ux: float, uy: float, lib=None) -> np.ndarray:
    """Eq. 2 for one component at one node."""
    out = np.zeros(9)
    (lib or _load()).oracle_equilibrium(rho, ux, uy, _dp(out))
    return out


def source(tau: float, ux: float, uy: float, Fx: float, Fy: float, lib=None) -> np.ndarray:
    """Eq. 4 for one component at one node."""
    out = np.zeros(9)
    (lib or _load()).oracle_source(tau, ux, uy, Fx, Fy, _dp(out))
    return out


class Oracle:
    """A simulation state (post-streaming populations, FP64) plus its
    parameters. ``mask`` is [ny, nx] uint8, 1 = solid."""

    def __init__(self, nx, ny, mask, *, tau=(1.0, 1.0), G_AB=3.0,
                 bc=BC_MARTYS_CHEN, G_s=(0.0, 0.0), chi=(1.0, 1.0),
                 rho_s=(0.0, 0.0), pairing=PAIR_CROSS, avg_stencil=25,
                 periodic_x=False, periodic_y=False, lib=None):
        self.lib = lib or _load()
        self.p = OracleParams()
        self.p.nx, self.p.ny = nx, ny
        self.p.periodic_x, self.p.periodic_y = int(periodic_x), int(periodic_y)
        self.p.tau[0], self.p.tau[1] = tau
        self.p.G_AB = G_AB
        self.p.bc = bc
        self.p.pairing = pairing
        self.p.G_s[0], self.p.G_s[1] = G_s
        self.p.chi[0], self.p.chi[1] = chi
        self.p.rho_s[0], self.p.rho_s[1] = rho_s
        self.p.avg_stencil = avg_stencil
        self.nx, self.ny = nx, ny
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(ny, nx)
        rc = self.lib.oracle_check(ctypes.byref(self.p), _mp(self.mask))
        if rc:
            raise ValueError(f"oracle_check rejected the parameters/mask (code {rc})")
        self.f = np.zeros((2, 9, ny, nx))

    def init(self, rhoA, rhoB, ux=None, uy=None):
        rA = np.ascontiguousarray(rhoA, dtype=np.float64).reshape(self.ny, self.nx)
        rB = np.ascontiguousarray(rhoB, dtype=np.float64).reshape(self.ny, self.nx)
        null = ctypes.POINTER(ctypes.c_double)()
        pux, puy = null, null
        if ux is not None:
            self._ux = np.ascontiguousarray(ux, dtype=np.float64)
            pux = _dp(self._ux)
        if uy is not None:
            self._uy = np.ascontiguousarray(uy, dtype=np.float64)
            puy = _dp(self._uy)
        rc = self.lib.oracle_init(ctypes.byref(self.p), _mp(self.mask), _dp(rA),
                                  _dp(rB), pux, puy, _dp(self.f))
        if rc:
            raise ValueError("oracle_init failed")
        return self

    def step(self, n: int = 1):
        rc = self.lib.oracle_step(ctypes.byref(self.p), _mp(self.mask), _dp(self.f), n)
        if rc:
            raise RuntimeError(f"oracle_step failed ({rc})")
        return self

    def fields(self):
        """(rho[2], rho_tilde[2], F[2][2], u[2]) of the current state."""
        ny, nx = self.ny, self.nx
        rho = np.zeros((2, ny, nx))
        rt = np.zeros((2, ny, nx))
        F = np.zeros((2, 2, ny, nx))
        u = np.zeros((2, ny, nx))
        self.lib.oracle_fields(ctypes.byref(self.p), _mp(self.mask), _dp(self.f),
                               _dp(rho), _dp(rt), _dp(F), _dp(u))
        return rho, rt, F, u

    def interface_solid(self):
        flag = np.zeros((self.ny, self.nx), np.uint8)
        self.lib.oracle_interface_solid(ctypes.byref(self.p), _mp(self.mask), _mp(flag))
        return flag

    def collide(self, rho, u, F):
        out = np.zeros_like(self.f)
        self.lib.oracle_collide(ctypes.byref(self.p), _mp(self.mask), _dp(self.f),
                                _dp(np.ascontiguousarray(rho)), _dp(np.ascontiguousarray(u)),
                                _dp(np.ascontiguousarray(F)), _dp(out))
        return out

    def stream(self, fpost):
        out = np.zeros_like(self.f)
        self.lib.oracle_stream(ctypes.byref(self.p), _mp(self.mask),
                               _dp(np.ascontiguousarray(fpost)), _dp(out))
        return out

    def mass(self):
        out = np.zeros(2)
        self.lib.oracle_mass(ctypes.byref(self.p), _mp(self.mask), _dp(self.f), _dp(out))
        return out
