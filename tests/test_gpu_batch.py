"""Batched form: independent volumes of uneven size and coil count, solved together with one
CUDA graph launch per two outer iterations, each held to the FP64 oracle's solve of that
volume alone (per-iteration cost to 1e-10 in FP64 mode)."""
import numpy as np
import pytest

from gpu_util import dev_inputs, to_np
from oracle import Oracle
from synth import make_volume

pytestmark = pytest.mark.gpu

SHAPES = [(40, 34, 9, 1), (21, 35, 17, 3), (64, 16, 8, 2), (8, 8, 8, 8), (37, 21, 11, 1)]


def _vols():
    return [make_volume(nx, ny, nz, ncoil=nc, snr_db=12.0 + 3 * k, seed=500 + k, fmax_hz=120.0, nblobs=3)
            for k, (nx, ny, nz, nc) in enumerate(SHAPES)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fraction", [1.0, 0.25])
def test_batch_solve_matches_oracle_per_volume(prec, fraction):
    from paper_2005_08661_gb300 import FieldMapBatch
    vols = _vols()
    refs = [Oracle.from_volume(v).solve(niter=7, nls=5) for v in vols]
    b = FieldMapBatch([(v.nx, v.ny, v.nz, v.ncoil, v.necho) for v in vols], precision=prec)
    b.set_fraction(fraction)
    keep = []
    for k, v in enumerate(vols):
        y, s, m = dev_inputs(v, prec)
        keep.append((y, s, m))
        b.set_data(k, y, s, v.te, m, v.beta)
    for rep in range(2):  # the second solve replays the captured batch graph
        ws, costs = b.solve(niter=7)
        for k, v in enumerate(vols):
            if prec == "fp64":
                np.testing.assert_allclose(costs[k], refs[k]["cost"], rtol=1e-10)
                np.testing.assert_allclose(to_np(ws[k]), refs[k]["w"], rtol=0, atol=1e-9)
            else:
                assert abs(costs[k][-1] - refs[k]["cost"][-1]) <= 2e-5 * abs(refs[k]["cost"][-1])
    b.close()


def test_batch_autotune_picks_a_candidate_and_results_stay_correct():
    from paper_2005_08661_gb300 import FieldMapBatch
    vols = _vols()
    b = FieldMapBatch([(v.nx, v.ny, v.nz, v.ncoil, v.necho) for v in vols], precision="fp64")
    keep = []
    for k, v in enumerate(vols):
        y, s, m = dev_inputs(v, "fp64")
        keep.append((y, s, m))
        b.set_data(k, y, s, v.te, m, v.beta)
    f, ms = b.autotune(niter_probe=2)
    assert f in (1.0, 0.5, 0.25, 0.125) and ms > 0
    frac, weights = b.schedule()
    assert frac == f and weights in ((2, 1), (1, 1), (3, 2))
    assert b.bwd_blocks_per_sm() in (1, 2, 3)
    ws, costs = b.solve(niter=4)
    for k, v in enumerate(vols):
        r = Oracle.from_volume(v).solve(niter=4, nls=5)
        np.testing.assert_allclose(costs[k], r["cost"], rtol=1e-10)
    b.close()
