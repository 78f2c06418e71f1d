"""The C-ABI library loads without a GPU, exports every function that
include/lbm.h declares, and the ctypes mirrors of its structs have the
C layout (checked against a C program compiled from the header)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2009_12584_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(lbm.EXPORTS) <= set(names)


def test_status_strings_without_gpu(lib):
    lib.lbm_status_str.restype = ctypes.c_char_p
    assert lib.lbm_status_str(0) == b"ok"
    assert lib.lbm_status_str(2) == b"call out of order"


def test_workspace_bytes_and_argument_checks_without_gpu():
    lbm.load()
    p = lbm.make_params(8192, 8192, periodic_x=True, periodic_y=True)
    n = lbm.workspace_bytes(p)
    # two population buffers of 18 FP32 planes dominate
    assert n > 2 * 18 * 8192 * 8192 * 4
    with pytest.raises(lbm.LbmError):
        lbm.workspace_bytes(lbm.make_params(3, 8))
    with pytest.raises(lbm.LbmError):
        lbm.workspace_bytes(lbm.make_params(8, 8, tau=(0.5, 1.0)))
    with pytest.raises(lbm.LbmError):
        lbm.workspace_bytes(lbm.make_params(8, 8, storage=7))
    n64 = lbm.workspace_bytes(lbm.make_params(64, 64, storage="fp64"))
    n16 = lbm.workspace_bytes(lbm.make_params(64, 64, storage="fp16"))
    assert n64 > n16


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(lbm_params), offsetof(lbm_params, tau),
         offsetof(lbm_params, storage), offsetof(lbm_params, rho_ref), offsetof(lbm_params, max_interface));
  printf("%zu %zu %zu %zu\n", sizeof(lbm_wetting_params), offsetof(lbm_wetting_params, G_s),
         offsetof(lbm_wetting_params, chi), offsetof(lbm_wetting_params, rho_s));
  printf("%zu %zu %zu %zu %zu\n", sizeof(lbm_diag_params), offsetof(lbm_diag_params, tangent),
         offsetof(lbm_diag_params, box), offsetof(lbm_diag_params, bridge_x), offsetof(lbm_diag_params, bridge_y0));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(lbm_diag), offsetof(lbm_diag, com_velocity),
         offsetof(lbm_diag, max_u), offsetof(lbm_diag, contour_points), offsetof(lbm_diag, circle),
         offsetof(lbm_diag, bridge_radius));
  printf("%zu\n", offsetof(lbm_diag, nonfinite_nodes));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    a = [int(v) for v in out[0].split()]
    b = [int(v) for v in out[1].split()]
    P, W = lbm.LbmParams, lbm.LbmWetting
    assert a == [ctypes.sizeof(P), P.tau.offset, P.storage.offset, P.rho_ref.offset, P.max_interface.offset]
    assert b == [ctypes.sizeof(W), W.G_s.offset, W.chi.offset, W.rho_s.offset]
    c = [int(v) for v in out[2].split()]
    d = [int(v) for v in out[3].split()]
    DP, D = lbm.LbmDiagParams, lbm.LbmDiag
    assert c == [ctypes.sizeof(DP), DP.tangent.offset, DP.box.offset, DP.bridge_x.offset, DP.bridge_y0.offset]
    assert d == [ctypes.sizeof(D), D.com_velocity.offset, D.max_u.offset, D.contour_points.offset,
                 D.circle.offset, D.bridge_radius.offset]
    assert int(out[4]) == D.nonfinite_nodes.offset


def test_argument_checks_before_any_cuda_call(lib):
    lib.lbm_set_l2_fetch_granularity.argtypes = [ctypes.c_int32, ctypes.c_void_p]
    lib.lbm_set_l2_fetch_granularity.restype = ctypes.c_int
    for bad in (0, 16, 48, 256):
        assert lib.lbm_set_l2_fetch_granularity(bad, None) == lbm.ERR_ARG
    lib.lbm_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.lbm_diagnostics.restype = ctypes.c_int
    assert lib.lbm_diagnostics(None, None, None) == lbm.ERR_ARG
    lib.lbm_debug_tma_expect_extra.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.lbm_debug_tma_expect_extra.restype = ctypes.c_int
    assert lib.lbm_debug_tma_expect_extra(None, 16) == lbm.ERR_ARG


def test_tiled_schedule_workspace_without_gpu():
    """The tiled schedule adds its per-tile lists (2 bytes per region slot of
    each 32 x 14 tile plus per-tile offsets and (owned, listed) count pairs,
    each array 256-byte aligned), and for 16-bit storage a third density
    plane pair; the TMA schedule (FP32 only) adds a 16-byte work item per
    tile; AUTO keeps the tiled lists (and the halo lists) for 4- and 8-byte
    storage only; an unknown schedule is rejected."""
    lbm.load()
    align = lambda n: (n + 255) // 256 * 256
    for nx, ny in ((8192, 8192), (100, 70), (4, 4)):
        nt = -(-nx // 32) * -(-ny // 14)
        extra = align(nt * 34 * 16 * 2) + align((nt + 1) * 4) + align(nt * 8)
        for st in ("fp32", "fp64"):
            base = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="two_pass"))
            tiled = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="tiled"))
            assert tiled - base == extra, (nx, ny, st)
            if st == "fp32":
                tma = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="tma"))
                assert tma - tiled == align(nt * 16), (nx, ny)
            # AUTO keeps the tiled lists and room for the halo lists (4- and
            # 8-byte storage: tiled under the improved scheme, halo under the
            # one-node-reach schemes)
            nh = -(-nx // 32) * -(-ny // 14)
            halo_extra = align(nh * 38 * 20 * 2) + align((nh + 1) * 4) + align(nh * 16) + align(nh * 24 * 4)
            assert lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="auto")) == tiled + halo_extra
        px = -(-(32 + nx + 4) // 32) * 32  # padded pitch and rows
        plane = px * (ny + 8)
        for st in ("fp16", "bf16"):
            base = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="two_pass"))
            # AUTO runs the two-pass schedule for 16-bit storage
            assert lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="auto")) == base
            # TILED adds the tile lists and a third density plane pair (FP32)
            tiled = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="tiled"))
            assert tiled - base == extra + 2 * plane * 4, (nx, ny, st)
    with pytest.raises(lbm.LbmError):
        lbm.workspace_bytes(lbm.make_params(8, 8, kernel=6))


def test_halo_schedule_workspace_without_gpu():
    """The halo schedule adds its per-tile lists: 2 bytes per slot of each
    tile's (32 + 6) x (14 + 6) region, per-tile offsets, four cumulative ring
    counts and a fluid bitmask of the region (24 words), each array 256-byte
    aligned; 16-bit storage runs the two-pass schedule and keeps none."""
    lbm.load()
    align = lambda n: (n + 255) // 256 * 256
    for nx, ny in ((8192, 8192), (100, 70), (4, 4)):
        nt = -(-nx // 32) * -(-ny // 14)
        extra = align(nt * 38 * 20 * 2) + align((nt + 1) * 4) + align(nt * 16) + align(nt * 24 * 4)
        for st in ("fp32", "fp64"):
            base = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="two_pass"))
            halo = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="halo"))
            assert halo - base == extra, (nx, ny, st)
        for st in ("fp16", "bf16"):
            base = lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="two_pass"))
            assert lbm.workspace_bytes(lbm.make_params(nx, ny, storage=st, kernel="halo")) == base


def test_binding_enums_match_header():
    """The binding's names for status codes, storage types, schedules,
    wetting schemes and pairings carry the values include/lbm.h declares."""
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "lbm.h")).read()
    decl = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    assert [decl[f"LBM_{n}"] for n in ("OK", "ERR_ARG", "ERR_STATE", "ERR_CUDA", "ERR_SPACE", "ERR_TIMEOUT")] == \
        [lbm.OK, lbm.ERR_ARG, lbm.ERR_STATE, lbm.ERR_CUDA, lbm.ERR_SPACE, lbm.ERR_TIMEOUT]
    assert {k: decl[f"LBM_STORE_{k.upper()}"] for k in lbm.STORAGE} == lbm.STORAGE
    assert {k: decl[f"LBM_KERNEL_{k.upper()}"] for k in lbm.KERNEL} == lbm.KERNEL
    assert len(lbm.KERNEL) == len([n for n in decl if n.startswith("LBM_KERNEL_")])
    for name, hname in (("martys_chen", "MARTYS_CHEN"), ("llkc", "LLKC"), ("virtual_avg", "VIRTUAL_AVG"),
                        ("constant", "CONSTANT")):
        assert lbm.WETTING[name] == decl[f"LBM_WET_{hname}"]
    assert (lbm.PAIR_CROSS, lbm.PAIR_SELF) == (decl["LBM_PAIR_CROSS"], decl["LBM_PAIR_SELF"])


def test_size_limit_without_gpu():
    """Padded node indices stay below 2^30 (list entries keep two tag bits
    above them): the largest square grid under the limit is accepted (its
    workspace holds two population buffers of 18 FP32 planes), one just
    above it and a thin grid of 2^28 rows are rejected."""
    lbm.load()
    n_ok, n_bad = 32700, 32760
    px_ok = -(-(32 + n_ok + 4) // 32) * 32
    px_bad = -(-(32 + n_bad + 4) // 32) * 32
    assert px_ok * (n_ok + 8) < 1 << 30 <= px_bad * (n_bad + 8)
    assert lbm.workspace_bytes(lbm.make_params(n_ok, n_ok)) > 2 * 18 * px_ok * (n_ok + 8) * 4
    for nx, ny in ((n_bad, n_bad), (4, 1 << 28)):
        with pytest.raises(lbm.LbmError):
            lbm.workspace_bytes(lbm.make_params(nx, ny))
