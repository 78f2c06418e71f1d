"""The batched arm in the configuration the benchmark times: 512
inclined-wall simulations (seed 0, sizes 64x64 ... 512x256, the three
wetting schemes mixed), autotuned schedule, block size and graph length,
FP32 and FP16. Sampled members must end bit-identical to the same
simulations stepped alone (whose parity with the oracle the other tests
check)."""
import numpy as np
import pytest

from paper_2009_12584_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import lbm  # noqa: E402


def _make(w, storage):
    s = lbm.Simulation(w["nx"], w["ny"], storage=storage)
    s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
    return s


def autotune_steps(trial, candidates, graph_lengths=(2, 8, 32)):
    """Steps lbm_batch_autotune advances every member by: per candidate
    (schedule and block size) and graph length S, S warm-up steps and
    ceil(trial / S) * S timed ones."""
    return candidates * sum(S + -(-trial // S) * S for S in graph_lengths)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_full_batch_members_match_solo_runs(storage):
    work = inputs.batched_workload(512, seed=0)
    sims = [_make(w, storage) for w in work]
    b = lbm.Batch(sims)
    b.autotune(16)  # as the benchmark: tuned on the batch itself, which it advances
    b.step(48)
    # two-pass at 128 and 256 threads, and the tiled schedule for FP32 (its
    # members keep tile lists); FP16 members run the two-pass one only
    total = autotune_steps(16, 3 if storage == "fp32" else 2) + 48
    picks = [int(i) for i in np.random.default_rng(11).choice(512, 6, replace=False)]
    for i in picks:
        solo = _make(work[i], storage)
        solo.step(total)
        assert torch.equal(solo.populations(), sims[i].populations()), (storage, i)
        solo.close()
    b.close()
    for s_ in sims:
        s_.close()
