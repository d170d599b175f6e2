"""The stored expected values are the oracle's: regenerating them with the committed FP64
oracle (as tests/golden/make_golden.py does) reproduces the files."""
import json
import os

import numpy as np

from oracle import Oracle
from synth import small_config

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_small_workload_cost_history_is_the_oracles():
    """The time-to-oracle-cost target: 50 NCG-MLS-IC(0) iterations on the 64x64x16 workload."""
    g = json.load(open(os.path.join(GOLDEN, "small_oracle_cost.json")))
    r = Oracle.from_volume(small_config()).solve(niter=g["niter"], nls=5)
    np.testing.assert_allclose(r["cost"], g["cost"], rtol=1e-12, atol=0)
    assert abs(r["cost"][-1] - g["final_cost"]) <= 1e-12 * abs(g["final_cost"])
    assert np.all(np.diff(r["cost"]) <= 0)  # monotone, as the line search guarantees
