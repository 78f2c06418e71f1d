"""Parity at the full size of the throughput workload: the 8192 x 8192
porous medium of the benchmark (same recipe, seeds, wetting and launch
configuration), checked on sampled outputs that the oracle computes one by
one.

After a few steps on the GPU, windows of the post-streaming populations are
cut out with a margin of M = 5 nodes around a W x W interior and a solid
frame around that; the oracle takes one step on each window and its
interior must match the GPU's next state. One step at a node reads the
populations within 1 node, the densities within 2 (force) and the virtual
densities of Eq. 8 within 4, so the frame and the cut do not reach the
interior.

Tolerances. FP32: the GPU's step rounds each result a few times in FP32 on
values below 0.5 (one FP32 unit at 0.5 is 6e-8): 1e-6 (also for the
single-pass schedules). FP16: the stored deviation from w_i rho_ref is
rounded to 11 significant bits, at most 2^-11 x 0.5 = 2.4e-4 for |f| < 0.5,
plus the FP32 term: 2.5e-4. BF16: 8 significant bits, 2^-8 x 0.5 = 2.0e-3:
2.5e-3."""
import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import lbm  # noqa: E402

N = 8192
STEPS = 20
W = 32          # interior width of a window
M = 5           # margin between the interior and the frame
SPAN = W + 2 * M + 2
CHI = (1.2, 0.8)  # xi = -0.2 under the chi = (1 - xi, 1 + xi) reading, as the benchmark


@pytest.fixture(scope="module")
def workload():
    mask = inputs.porous_disks(N, N, solid_fraction=0.40, rmin=8, rmax=40, seed=1)
    rA, rB = inputs.pore_droplets(mask, a_fraction=0.30, rmin=8, rmax=32, seed=2)
    return mask, rA, rB


def _windows(mask, rA, count=4, seed=7):
    """Window origins whose interior holds walls and both phases."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(5000):
        x0, y0 = (int(v) for v in rng.integers(0, N - SPAN, 2))
        inner = (slice(y0 + M + 1, y0 + M + 1 + W), slice(x0 + M + 1, x0 + M + 1 + W))
        m = mask[inner]
        a = rA[inner][m == 0]
        if 0.15 < m.mean() < 0.6 and (a > 0.5).any() and (a < 0.5).any():
            out.append((x0, y0))
            if len(out) == count:
                break
    return out


@pytest.mark.parametrize("storage,kernel,tol", [("fp32", "two_pass", 1e-6), ("fp16", "auto", 2.5e-4),
                                                ("bf16", "auto", 2.5e-3), ("fp32", "fused", 1e-6),
                                                ("fp32", "tiled", 1e-6), ("fp16", "tiled", 2.5e-4),
                                                ("fp32", "halo", 1e-6), ("fp32", "tma", 1e-6)])
def test_full_size_step_matches_oracle_on_windows(workload, storage, kernel, tol):
    mask, rA, rB = workload
    wins = _windows(mask, rA)
    assert len(wins) == 4
    sim = lbm.Simulation(N, N, periodic_x=True, periodic_y=True, storage=storage, kernel=kernel)
    sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=CHI).init_fields(rA, rB).step(STEPS)

    def cut():
        f = sim.populations()
        w = [f[:, :, y0:y0 + SPAN, x0:x0 + SPAN].cpu().numpy() for x0, y0 in wins]
        del f
        torch.cuda.empty_cache()
        return w

    before = cut()
    sim.step(1)
    after = cut()
    sim.close()
    inner = (slice(None), slice(None), slice(M + 1, M + 1 + W), slice(M + 1, M + 1 + W))
    for (x0, y0), fb, fa in zip(wins, before, after):
        pm = np.ascontiguousarray(mask[y0:y0 + SPAN, x0:x0 + SPAN]).copy()
        pm[0, :] = pm[-1, :] = 1
        pm[:, 0] = pm[:, -1] = 1
        o = oracle.Oracle(SPAN, SPAN, pm, tau=(1.0, 1.0), G_AB=3.0, bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0),
                          chi=CHI)
        o.f[...] = fb * (pm == 0)[None, None]
        o.step(1)
        fluid = pm[M + 1:M + 1 + W, M + 1:M + 1 + W] == 0
        d = np.abs(o.f[inner] - fa[inner])[:, :, fluid]
        assert d.max() < tol, (storage, (x0, y0), d.max())
        # the windows do hold wall and interface nodes: the step there is not trivial
        assert np.abs(fa[inner] - fb[inner])[:, :, fluid].max() > 1e-4
