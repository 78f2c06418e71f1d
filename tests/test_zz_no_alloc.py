"""The allocation-free mass reduction (lbm_field_mass_noalloc) agrees with
the workspace-based lbm_mass on two calls in a row.

lbm_field_mass_noalloc serves callers that cannot allocate device memory
when they need the reduction (a memory-capped or pre-allocated pool, or a
host thread that must not call cudaMalloc because it would synchronise the
device): its scratch is a fixed 256 KiB __device__ array inside the library,
so the caller passes only the density fields, the mask and the output.
The test calls the entry point through the C ABI with ctypes."""
import ctypes

import numpy as np
import pytest

from paper_2009_12584_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import lbm  # noqa: E402


def _entry():
    fn = lbm.load().lbm_field_mass_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_mass_matches_lbm_mass_twice():
    nx, ny = 301, 157  # several 4096-node blocks and a ragged last block
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 20)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 20)
    sim = lbm.Simulation(nx, ny, storage="fp64")
    sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=(1.2, 0.8)).init_fields(rA, rB)
    fn = _entry()
    stream = torch.cuda.current_stream()
    d_mask = torch.from_numpy(mask).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for steps in (7, 23):  # two calls in a row, on different states
        sim.step(steps)
        expect = sim.mass()  # the workspace-based reduction over the populations
        rhoA, rhoB, _ = sim.moments()
        out.fill_(-1.0)
        st = fn(rhoA.data_ptr(), rhoB.data_ptr(), d_mask.data_ptr(), nx, ny, out.data_ptr(),
                stream.cuda_stream)
        assert st == lbm.OK
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, expect, rtol=1e-13)


def test_noalloc_mass_without_mask_and_size_limit():
    fn = _entry()
    stream = torch.cuda.current_stream()
    nx, ny = 64, 33
    g = torch.Generator().manual_seed(0)
    a = torch.rand((ny, nx), generator=g, dtype=torch.float64)
    b = torch.rand((ny, nx), generator=g, dtype=torch.float64)
    da, db = a.cuda(), b.cuda()  # keep the device copies alive while the kernels run
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        st = fn(da.data_ptr(), db.data_ptr(), None, nx, ny, out.data_ptr(), stream.cuda_stream)
        assert st == lbm.OK
        np.testing.assert_allclose(out.cpu().numpy(), [a.sum().item(), b.sum().item()], rtol=1e-13)
    # beyond the static scratch: rejected before any launch
    assert fn(da.data_ptr(), db.data_ptr(), None, 8193, 8192, out.data_ptr(), stream.cuda_stream) == lbm.ERR_ARG
