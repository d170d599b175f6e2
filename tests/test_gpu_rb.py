"""Red-black IC(0) on the GPU (FM_PC_RB, the labelled multicolour variant): its factor and
apply against the oracle's generic IC(0) of the red-black permuted H, and the solve's
per-iteration cost against the oracle's solve with the same preconditioner."""
import numpy as np
import pytest

from gpu_util import open_fm, to_dev, to_np
from oracle import Oracle
from synth import make_volume

pytestmark = pytest.mark.gpu

CASES = [(70, 37, 19, 1), (45, 33, 17, 2), (13, 9, 10, 3), (1, 40, 9, 2), (1, 1, 1, 1)]


def _vol(nx, ny, nz, nc):
    v = make_volume(nx, ny, nz, ncoil=nc, snr_db=15.0, seed=300 + nx + nc, fmax_hz=150.0, nblobs=3)
    if v.mask.size > 8:
        rng = np.random.default_rng(nx)
        v.mask = (v.mask & (rng.uniform(size=v.mask.shape) > 0.08)).astype(np.uint8)
    if v.mask.sum() == 0:
        v.mask[:] = 1
    return v


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_red_black_factor_and_apply_match_oracle(prec, case):
    from paper_2005_08661_gb300 import FmError, FM_ERR_NOT_PD
    vol = _vol(*case)
    o = Oracle.from_volume(vol)
    rng = np.random.default_rng(2)
    w = (o.init() + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask
    g = rng.standard_normal(vol.mask.shape) * vol.mask
    fm = open_fm(vol, prec, precond="rb")
    try:
        p_ref = o.precondition(o.curv(w), g, order=1)
    except RuntimeError:  # a non-positive pivot: the GPU must report it too
        fm.ic_factor(to_dev(w, prec))
        with pytest.raises(FmError) as e:
            fm.cost_grad(to_dev(w, prec))  # the next synchronising call reports it
        assert e.value.status == FM_ERR_NOT_PD
        fm.close()
        return
    fm.ic_factor(to_dev(w, prec))
    p = to_np(fm.ic_apply(to_dev(g, prec)))
    tol = 1e-10 if prec == "fp64" else 2e-4
    assert np.max(np.abs(p - p_ref)) <= tol * np.max(np.abs(p_ref))
    assert np.all(p[vol.mask == 0] == 0)
    fm.close()


@pytest.mark.parametrize("case", CASES[:3])
def test_fp64_red_black_solve_matches_oracle_per_iteration(case):
    vol = _vol(*case)
    ref = Oracle.from_volume(vol).solve(niter=15, nls=5, precond=3)
    fm = open_fm(vol, "fp64", precond="rb")
    w, cost = fm.solve(niter=15)
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-9)
    fm.close()


def test_fp32_red_black_solve_decreases_the_cost():
    vol = _vol(45, 33, 17, 2)
    fm = open_fm(vol, "fp32", precond="rb")
    _, cost = fm.solve(niter=30)
    assert np.all(np.diff(cost) <= 2e-6 * np.abs(cost[:-1])) and cost[-1] < cost[0]
    fm.close()
