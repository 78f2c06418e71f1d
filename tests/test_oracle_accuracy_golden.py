"""tests/golden/oracle_accuracy.json holds what the FP64 oracle gives on the
400 x 200 inclined-plane set-up (see make_oracle_accuracy.py, which calls
only the oracle); the reduced-storage GPU tests and the benchmark's accuracy
arm compare against it. This re-derives the first sliding-velocity sample of
one case (1,000 oracle steps) and checks the stored value, so that the file
cannot drift from the oracle."""
import importlib.util
import json
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_first_sample_matches_oracle():
    spec = importlib.util.spec_from_file_location("make_oracle_accuracy",
                                                  os.path.join(GOLDEN, "make_oracle_accuracy.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    gold = json.load(open(os.path.join(GOLDEN, "oracle_accuracy.json")))
    stored = next(c for c in gold["cases"] if c["scheme"] == "mc" and c["beta"] == 20.0)
    fresh = gen.case("mc", 20.0, stored["every"], stored["every"])
    assert abs(fresh["sliding_velocity"][0] - stored["sliding_velocity"][0]) <= 1e-12
    assert (gold["nx"], gold["ny"], gold["R0"]) == (gen.NX, gen.NY, gen.R0)
