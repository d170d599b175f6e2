"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances.  FP64 mode differs from the oracle only in summation order and in the
exact pair factorisation of Eq. 3 (k_setup.cu), so values agree to ~1e-13 relative;
the tests allow 1e-10.  FP32 mode rounds every voxel quantity to float: the phase
theta = angle R + w dt carries an absolute error of about |w dt| * 2^-24 <= 1e-6 rad, so
gradients agree to about 1e-6 of their maximum and curvatures (a sum of sinc terms,
Taylor-truncated at 7e-9) to about 1e-6 relative; the tests allow 3e-5 and 1e-5.
Global sums are FP64 in both modes.
"""
import math

import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from oracle import Oracle, ic0_factor, ic0_solve
from synth import make_volume, small_config

pytestmark = pytest.mark.gpu

TOL = {
    "fp64": dict(cost=1e-11, g=1e-10, d=1e-11, w0=1e-12, ip=1e-11, p=1e-10),
    "fp32": dict(cost=2e-6, g=3e-5, d=1e-5, w0=2e-6, ip=3e-5, p=2e-4),
}

CASES = [
    # nx, ny, nz, ncoil: several 32x32x8 tiles with ragged tails, all coil-count code paths
    (70, 37, 19, 1),
    (45, 33, 17, 2),
    (13, 9, 10, 3),
    (40, 34, 9, 8),
    (1, 1, 1, 1),
    (33, 1, 1, 1),
    (1, 40, 9, 2),
]


def _vol(nx, ny, nz, nc, seed=0, holes=True):
    v = make_volume(nx, ny, nz, ncoil=nc, snr_db=15.0, seed=100 + seed + nx + 3 * nc, fmax_hz=150.0,
                    nblobs=3)
    if holes and v.mask.size > 8:
        rng = np.random.default_rng(seed + 7)
        v.mask = (v.mask & (rng.uniform(size=v.mask.shape) > 0.08)).astype(np.uint8)
    if v.mask.sum() == 0:
        v.mask[:] = 1
    return v


def _fp32_cost_atol(vol, w):
    """Bound on |Psi_fp32 - Psi_fp64|: each pair term 4|R| sin^2(theta/2) moves by at most
    2|R| |dtheta|, and rounding theta's inputs (angle R, w, w dt) to float gives
    |dtheta| <= 2^-23 (pi + 2 |w dt|); sincosf adds about one ulp.  R_mn = conj(Z_m) Z_n with
    Z_m = sum_c conj(s_c) y_cm / sqrt(L S) is formed here only to scale this bound."""
    y = vol.y.astype(np.complex128)
    s = vol.smap.astype(np.complex128) if vol.smap is not None else np.ones((1,) + vol.mask.shape)
    S = np.sum(np.abs(s) ** 2, axis=0)
    Z = np.sum(np.conj(s)[None] * y, axis=1) / np.sqrt(vol.necho * np.maximum(S, 1e-300))[None]
    tot = 0.0
    m = vol.mask.astype(bool)
    for a in range(vol.necho):
        for b in range(a + 1, vol.necho):
            dt = abs(vol.te[a] - vol.te[b])
            tot += np.sum((np.abs(Z[a]) * np.abs(Z[b]) * (math.pi + 2 * np.abs(w) * dt + 2.0))[m])
    return 2.0 ** -21 * tot


def _omega(o, vol, seed=0):
    rng = np.random.default_rng(seed)
    return (o.init() + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_cost_gradient_curvature_and_init(prec, case):
    vol = _vol(*case)
    o = Oracle.from_volume(vol)
    w = _omega(o, vol)
    fm = open_fm(vol, prec)
    cost, g, d = fm.cost_grad(to_dev(w, prec))
    tol = TOL[prec]
    c_ref = o.cost(w)
    atol = _fp32_cost_atol(vol, w) if prec == "fp32" else 1e-12
    assert cost == pytest.approx(c_ref, rel=tol["cost"], abs=atol)
    g_ref, d_ref = o.grad(w), o.curv(w)
    g, d = to_np(g), to_np(d)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol["g"] * max(np.abs(g_ref).max(), 1e-30))
    np.testing.assert_allclose(d, d_ref, rtol=tol["d"], atol=tol["d"] * max(np.abs(d_ref).max(), 1e-30))
    w0 = to_np(fm.init_omega())
    w0_ref = o.init()
    np.testing.assert_allclose(w0, w0_ref, rtol=0, atol=tol["w0"] * max(np.abs(w0_ref).max(), 1.0))
    fm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("te", [(0.0, 2.5), (0.0, 1.5, 4.0, 9.5)])
@pytest.mark.parametrize("nc", [2, 3, 8])
def test_cost_gradient_curvature_other_echo_counts(prec, te, nc):
    """Two and four echoes: the evaluators for any echo count (compile-time coil counts 2
    and 8, the runtime coil count for 3), whose curvature reads the coil angles in FP32 as
    fixed-point turns (the runtime one wraps them in fixed point), against the oracle."""
    vol = make_volume(19, 13, 7, ncoil=nc, te=te, snr_db=15.0, seed=300 + nc + 7 * len(te), fmax_hz=150.0,
                      nblobs=3)
    o = Oracle.from_volume(vol)
    w = _omega(o, vol, seed=2)
    fm = open_fm(vol, prec)
    cost, g, d = fm.cost_grad(to_dev(w, prec))
    tol = TOL[prec]
    atol = _fp32_cost_atol(vol, w) if prec == "fp32" else 1e-12
    assert cost == pytest.approx(o.cost(w), rel=tol["cost"], abs=atol)
    g_ref, d_ref = o.grad(w), o.curv(w)
    g, d = to_np(g), to_np(d)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol["g"] * max(np.abs(g_ref).max(), 1e-30))
    np.testing.assert_allclose(d, d_ref, rtol=tol["d"], atol=tol["d"] * max(np.abs(d_ref).max(), 1e-30))
    fm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_ic0_pivots_and_apply(prec, case):
    vol = _vol(*case, seed=1)
    o = Oracle.from_volume(vol)
    w = _omega(o, vol, seed=1)
    fm = open_fm(vol, prec)
    ip = to_np(fm.ic_factor(to_dev(w, prec)))
    colptr, rowidx, val, umap = ic0_factor(vol.mask.shape, vol.mask, o.curv(w), vol.beta)
    ip_ref = np.zeros(vol.mask.size)
    ip_ref[umap] = 1.0 / val[colptr[:-1]] ** 2  # 1 / pi_j with pi_j = L_jj^2
    tol = TOL[prec]
    np.testing.assert_allclose(ip.reshape(-1), ip_ref, rtol=tol["ip"], atol=0)
    rng = np.random.default_rng(3)
    gvec = rng.standard_normal(vol.mask.shape) * vol.mask
    p = to_np(fm.ic_apply(to_dev(gvec, prec)))
    p_ref = np.zeros(vol.mask.size)
    p_ref[umap] = ic0_solve(colptr, rowidx, val, gvec.reshape(-1)[umap])
    np.testing.assert_allclose(p.reshape(-1), p_ref, rtol=0, atol=tol["p"] * np.abs(p_ref).max())
    fm.close()


@pytest.fixture(scope="module")
def small_ref():
    vol = small_config()
    o = Oracle.from_volume(vol)
    r = o.solve(niter=50, nls=5)
    return vol, r


def test_fp64_solve_matches_oracle_every_iteration(small_ref):
    """64x64x16, one coil, 50 iterations, FP64: per-iteration cost to 1e-10 relative."""
    vol, r = small_ref
    fm = open_fm(vol, "fp64")
    w, cost = fm.solve(niter=50)
    np.testing.assert_allclose(cost, r["cost"], rtol=1e-10, atol=0)
    alpha, mu = fm.history(50)
    np.testing.assert_allclose(alpha, r["alpha"], rtol=1e-6)
    np.testing.assert_allclose(mu, r["mu"], rtol=1e-6, atol=1e-12)
    m = vol.mask.astype(bool)
    hz = 1000.0 / (2 * math.pi)
    assert np.max(np.abs(to_np(w) - r["w"])[m]) * hz < 1e-6
    fm.close()


def test_fp32_solve_reaches_the_oracle_cost(small_ref):
    """FP32 voxel arithmetic with FP64 sums: final cost within 1e-6 relative of the FP64
    oracle's, field-map RMSE below 0.05 Hz and max error below 0.5 Hz inside the mask."""
    vol, r = small_ref
    fm = open_fm(vol, "fp32")
    w, cost = fm.solve(niter=50)
    assert abs(cost[-1] - r["cost"][-1]) <= 1e-6 * abs(r["cost"][-1])
    m = vol.mask.astype(bool)
    err_hz = (to_np(w) - r["w"])[m] * 1000.0 / (2 * math.pi)
    assert math.sqrt(np.mean(err_hz ** 2)) < 0.05
    assert np.max(np.abs(err_hz)) < 0.5
    fm.close()


@pytest.mark.parametrize("precond", ["diag", "none"])
def test_labelled_preconditioner_variants_match_oracle(precond):
    vol = _vol(40, 34, 9, 2, seed=5)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=8, nls=3, precond={"diag": 1, "none": 2}[precond])
    fm = open_fm(vol, "fp64", precond=precond, nls=3)
    w, cost = fm.solve(niter=8)
    np.testing.assert_allclose(cost, r["cost"], rtol=1e-10)
    fm.close()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("niter", [0, 1, 2, 5])
def test_graph_replay_and_odd_iteration_counts(use_graph, niter):
    vol = _vol(45, 33, 17, 2, seed=9)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=niter, nls=4)
    fm = open_fm(vol, "fp64", nls=4, use_graph=use_graph)
    for _ in range(2):  # second solve replays the captured graph
        w, cost = fm.solve(niter=niter)
        np.testing.assert_allclose(cost, r["cost"], rtol=1e-10)
        np.testing.assert_allclose(to_np(w), r["w"], rtol=0, atol=1e-9)
    fm.close()


def test_solve_from_a_given_start_and_single_step_line_search():
    vol = _vol(37, 21, 11, 1, seed=11)
    o = Oracle.from_volume(vol)
    w0 = _omega(o, vol, seed=4)
    r = o.solve(w0=w0, niter=6, nls=1)
    fm = open_fm(vol, "fp64", nls=1)
    w, cost = fm.solve(to_dev(w0, "fp64"), niter=6)
    np.testing.assert_allclose(cost, r["cost"], rtol=1e-10)
    fm.close()


def test_empty_mask_gives_zero_map_and_zero_cost():
    vol = _vol(20, 20, 9, 1, holes=False)
    vol.mask[:] = 0
    fm = open_fm(vol, "fp32")
    w, cost = fm.solve(niter=3)
    assert np.all(to_np(w) == 0.0)
    assert np.all(cost == 0.0)
    fm.close()


def test_zero_data_and_zero_beta_reports_a_nonpositive_pivot():
    from paper_2005_08661_gb300 import FmError, FM_ERR_NOT_PD
    vol = _vol(20, 20, 9, 1, holes=False)
    vol.y[:] = 0
    vol.beta = 0.0
    fm = open_fm(vol, "fp32")
    with pytest.raises(FmError) as e:
        fm.solve(niter=2)
    assert e.value.status == FM_ERR_NOT_PD
    fm.close()


def test_wavefront_wait_limit_reports_timeout_and_the_device_stays_usable():
    """spin_limit = 1 makes a tile that must wait for its neighbour give up at once: the
    kernel records FM_ERR_TIMEOUT and returns; nothing hangs and later work runs."""
    from paper_2005_08661_gb300 import FmError, FM_ERR_TIMEOUT
    vol = _vol(128, 128, 32, 1, seed=13, holes=False)
    fm = open_fm(vol, "fp32", spin_limit=1)
    with pytest.raises(FmError) as e:
        fm.solve(niter=2)
    assert e.value.status == FM_ERR_TIMEOUT
    fm.close()
    o = Oracle.from_volume(vol)
    r = o.solve(niter=2)
    fm = open_fm(vol, "fp64")
    w, cost = fm.solve(niter=2)
    np.testing.assert_allclose(cost, r["cost"], rtol=1e-10)
    fm.close()


@pytest.mark.parametrize("precond,pc", [("ic0", 0), ("ict", 4)])
def test_a_timed_out_solve_leaves_the_same_context_usable(precond, pc):
    """A wait that gives up (spin_limit = 1: the IC tile flags, the line search's and the
    drop-tolerance sweeps' grid barriers) leaves its barrier arrival counted; the next call
    on the same context must start from a clean barrier, so a solve with the normal limit
    then matches the oracle per iteration."""
    from paper_2005_08661_gb300 import FmError, FM_ERR_TIMEOUT
    vol = _vol(128, 96, 24, 1, seed=14, holes=False)
    fm = open_fm(vol, "fp64", precond=precond)
    fm.set_spin_limit(1)
    with pytest.raises(FmError) as e:
        fm.solve(niter=3)
    assert e.value.status == FM_ERR_TIMEOUT
    fm.set_spin_limit(1 << 21)
    ref = Oracle.from_volume(vol).solve(niter=4, nls=5, precond=pc)
    w, cost = fm.solve(niter=4)
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-9)
    fm.close()


def test_binding_rejects_wrong_dtypes():
    import torch
    vol = _vol(8, 8, 8, 1, holes=False)
    fm = open_fm(vol, "fp32")
    with pytest.raises(TypeError):
        fm.cost_grad(torch.zeros(vol.mask.shape, dtype=torch.float64, device="cuda"))
    y, s, m = dev_inputs(vol, "fp64")
    with pytest.raises(TypeError):
        fm.set_data(y, s, vol.te, m, vol.beta)
    fm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_combined_curvature_variant_matches_oracle(prec):
    """FM_CURV_COMBINED (labelled variant): the same solve with the coil-combined curvature."""
    vol = _vol(40, 34, 9, 3, seed=17)
    o = Oracle.from_volume(vol)
    o.set_curvature("combined")
    w = _omega(o, vol, seed=2)
    fm = open_fm(vol, prec, curvature="combined")
    _, g, d = fm.cost_grad(to_dev(w, prec))
    d_ref = o.curv(w)
    tol = TOL[prec]
    np.testing.assert_allclose(to_np(d), d_ref, rtol=tol["d"], atol=tol["d"] * np.abs(d_ref).max())
    if prec == "fp64":
        r = o.solve(niter=6, nls=5)
        _, cost = fm.solve(niter=6)
        np.testing.assert_allclose(cost, r["cost"], rtol=1e-10)
    fm.close()


def test_non_finite_input_inside_the_mask_is_reported_and_outside_is_ignored():
    """A NaN image value at a mask voxel makes the cost constant non-finite: the next
    synchronising call reports FM_ERR_NONFINITE.  Outside the mask the images are never read."""
    from paper_2005_08661_gb300 import FmError, FM_ERR_NONFINITE
    vol = make_volume(12, 10, 6, ncoil=2, snr_db=20.0, seed=77, fmax_hz=100.0, nblobs=2)
    out = np.argwhere(vol.mask == 0)[0]
    vol.y[0, 0, out[0], out[1], out[2]] = np.nan
    fm = open_fm(vol, "fp64")
    w = fm.init_omega()
    cost, _, _ = fm.cost_grad(w)
    assert np.isfinite(cost)
    fm.close()
    inside = np.argwhere(vol.mask > 0)[0]
    vol.y[1, 1, inside[0], inside[1], inside[2]] = np.nan
    fm = open_fm(vol, "fp64")
    with pytest.raises(FmError) as e:
        fm.cost_grad(fm.init_omega())
    assert e.value.status == FM_ERR_NONFINITE
    fm.close()


def test_voxels_without_coil_sensitivity_carry_no_data_term():
    """S_j = 0 (every coil sensitivity zero at a mask voxel): r = 0 there (reading of Eq. 3),
    so only the regulariser acts; the FP64 solve still matches the oracle per iteration."""
    vol = make_volume(14, 12, 7, ncoil=2, snr_db=20.0, seed=78, fmax_hz=100.0, nblobs=2)
    inside = np.argwhere(vol.mask > 0)
    for z, y, x in inside[len(inside) // 2: len(inside) // 2 + 5]:
        vol.smap[:, z, y, x] = 0.0
    ref = Oracle.from_volume(vol).solve(niter=10, nls=5)
    fm = open_fm(vol, "fp64")
    w, cost = fm.solve(niter=10)
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-9)
    fm.close()
