"""The TMA schedule's bounded wait, made to run out without any fault: the
test hook makes every tile's copy barrier expect more bytes than the copies
deliver, so that no wait can complete. Each CTA must give up after about a
second, wait (bounded) for the copies it has in flight and stop; the next
lbm_sync must report LBM_ERR_TIMEOUT, and the context must stay usable: a
re-initialised state then steps bit for bit like the tiled schedule."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import inputs, lbm  # noqa: E402


def _sim(kernel, mask, rA, rB):
    nx, ny = mask.shape[1], mask.shape[0]
    sim = lbm.Simulation(nx, ny, storage="fp32", kernel=kernel)
    sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=(1.2, 0.8)).init_fields(rA, rB)
    return sim


def test_tma_wait_runs_out_and_context_recovers():
    nx, ny, R0 = 96, 64, 12
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, R0)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
    sim = _sim("tma", mask, rA, rB)
    sim.step(2).sync()
    sim.debug_tma_expect_extra(16)
    t0 = time.time()
    sim.step(1)
    with pytest.raises(lbm.LbmError) as e:
        sim.sync()
    took = time.time() - t0
    assert e.value.status == lbm.ERR_TIMEOUT
    assert 0.5 < took < 30.0, took  # each CTA gave up after its bounded waits
    # the error is reported once; the context is usable again
    sim.debug_tma_expect_extra(0)
    sim.sync()
    sim.init_fields(rA, rB).step(7)
    ref = _sim("tiled", mask, rA, rB).step(7)
    for a, b in zip(sim.moments(), ref.moments()):
        assert torch.equal(a, b)
    assert np.array_equal(np.asarray(sim.mass()), np.asarray(ref.mass()))
    sim.close()
    ref.close()
