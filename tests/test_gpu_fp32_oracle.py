"""FP32 mode against the FP64 oracle on an eight-coil volume drawn by the full workload's
recipe (64 x 64 x 32, 8 coils, echoes 0/2/10 ms, +-250 Hz + a 40 Hz step, SNR 15 dB,
beta 2^-3), 100 NCG-MLS-IC(0) iterations from the Eq. 6 start.

Targets: the FP32 solve's final cost within 1e-6 relative of the oracle's, and its field
map within RMSE 0.05 Hz and max 0.5 Hz of the oracle's over the mask.  The FP64 GPU solve
matches the oracle's per-iteration cost to 1e-10.  The oracle runs here on every host core
(its results do not depend on the thread count); its cost history must reproduce the stored
one (tests/golden/full8_oracle_cost.json, written by tests/golden/make_golden.py)."""
import json
import math
import os

import numpy as np
import pytest

from gpu_util import open_fm, to_np
from oracle import Oracle, set_threads
from synth import full8_small_config

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full8_oracle_cost.json")


@pytest.fixture(scope="module")
def case():
    vol = full8_small_config()
    gold = json.load(open(GOLDEN))
    set_threads(os.cpu_count() or 1)
    try:
        ref = Oracle.from_volume(vol).solve(niter=gold["niter"], nls=5)
    finally:
        set_threads(1)
    np.testing.assert_allclose(ref["cost"], gold["cost"], rtol=1e-12, atol=0)
    return vol, ref


def test_fp32_solve_reaches_the_oracle_cost_and_map(case):
    vol, ref = case
    fm = open_fm(vol, "fp32")
    w, cost = fm.solve(niter=len(ref["cost"]) - 1)
    fm.close()
    rel = abs(cost[-1] - ref["cost"][-1]) / abs(ref["cost"][-1])
    assert rel < 1e-6, rel
    m = vol.mask.astype(bool)
    dhz = (to_np(w) - ref["w"])[m] * 1000.0 / (2.0 * math.pi)
    assert math.sqrt(float(np.mean(dhz ** 2))) < 0.05
    assert float(np.abs(dhz).max()) < 0.5


def test_fp64_solve_matches_the_oracle_per_iteration(case):
    vol, ref = case
    fm = open_fm(vol, "fp64")
    w, cost = fm.solve(niter=len(ref["cost"]) - 1)
    fm.close()
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-8)
