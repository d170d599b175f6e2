"""Parity at the full 256x256x128, 8-coil workload, in the launch configuration bench.py
times (FP32, IC(0), N_ls = 5, captured graph).

The FP64 oracle cannot run a whole solve at this size, so the check uses sampled outputs:
after a few NCG iterations on the GPU, the gradient and Huber curvature at sampled mask
voxels (interior and mask-boundary) are compared with the oracle evaluated on each
voxel's 3x3x3 neighbourhood, which holds every input the voxel's gradient needs (its
data and its six stencil neighbours).  The cost history must be finite and, up to FP32
rounding of the cost, non-increasing (monotonic line search, Sec. III-C).
"""
import os

import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from oracle import Oracle, curv_raw, ic0_factor, ic0_solve, set_threads
from synth import full_config

pytestmark = pytest.mark.gpu

TOL = {"fp32": dict(g=3e-5, d=1e-5), "fp64": dict(g=1e-10, d=1e-11)}


@pytest.fixture(scope="module")
def full():
    return full_config()


def _sample_voxels(mask, n, seed):
    rng = np.random.default_rng(seed)
    idx = np.argwhere(mask > 0)
    inner = idx[rng.choice(len(idx), n // 2, replace=False)]
    # mask-boundary voxels: fewer than six in-mask neighbours
    m = mask.astype(bool)
    nb = np.zeros(m.shape, np.int8)
    for ax in range(3):
        for sh in (-1, 1):
            r = np.roll(m, sh, axis=ax)
            sl = [slice(None)] * 3
            sl[ax] = slice(0, 1) if sh == 1 else slice(-1, None)
            r[tuple(sl)] = False
            nb += r
    edge = np.argwhere(m & (nb < 6))
    edge = edge[rng.choice(len(edge), n - n // 2, replace=False)]
    return np.concatenate([inner, edge])


def _oracle_at(vol, w, z, y, x):
    nz, ny, nx = vol.mask.shape
    z0, z1 = max(z - 1, 0), min(z + 2, nz)
    y0, y1 = max(y - 1, 0), min(y + 2, ny)
    x0, x1 = max(x - 1, 0), min(x + 2, nx)
    sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
    o = Oracle(vol.y[(slice(None), slice(None)) + sl], vol.smap[(slice(None),) + sl], vol.te,
               vol.mask[sl], vol.beta)
    ws = np.ascontiguousarray(w[sl])
    c = (z - z0, y - y0, x - x0)
    g, d = o.grad(ws)[c], o.curv(ws)[c]
    o.close()
    return g, d


def test_full_size_fp32_solve_sampled_parity(full):
    vol = full
    fm = open_fm(vol, "fp32")  # defaults: IC(0), N_ls = 5, graph replay
    w, cost = fm.solve(niter=6)
    assert np.all(np.isfinite(cost))
    assert np.all(np.diff(cost) <= 2e-6 * np.abs(cost[:-1]))
    assert cost[-1] < cost[0]
    _, g, d = fm.cost_grad(w)
    w_np, g_np, d_np = to_np(w), to_np(g), to_np(d)
    assert np.all(w_np[vol.mask == 0] == 0.0)
    gmax = np.abs(g_np).max()
    for (z, y, x) in _sample_voxels(vol.mask, 48, seed=7):
        g_ref, d_ref = _oracle_at(vol, w_np, z, y, x)
        assert abs(g_np[z, y, x] - g_ref) <= TOL["fp32"]["g"] * gmax, (z, y, x, g_np[z, y, x], g_ref)
        assert abs(d_np[z, y, x] - d_ref) <= TOL["fp32"]["d"] * max(abs(d_ref), 1e-3 * d_np.max()), (z, y, x)
    fm.close()


def _full_w(vol, seed=3):
    """A seeded field map near the truth (inputs of both sides come from synth)."""
    rng = np.random.default_rng(seed)
    return (vol.omega_true + 0.02 * rng.standard_normal(vol.mask.shape)) * vol.mask


def test_full_size_fp64_cost_grad_sampled_parity(full):
    vol = full
    w = _full_w(vol)
    fm = open_fm(vol, "fp64")
    _, g, d = fm.cost_grad(to_dev(w, "fp64"))
    g_np, d_np = to_np(g), to_np(d)
    gmax = np.abs(g_np).max()
    for (z, y, x) in _sample_voxels(vol.mask, 24, seed=11):
        g_ref, d_ref = _oracle_at(vol, w, z, y, x)
        assert abs(g_np[z, y, x] - g_ref) <= TOL["fp64"]["g"] * gmax, (z, y, x)
        assert abs(d_np[z, y, x] - d_ref) <= TOL["fp64"]["d"] * max(abs(d_ref), 1e-3 * d_np.max()), (z, y, x)
    fm.close()


@pytest.fixture(scope="module")
def full_ic_ref(full):
    """The oracle's generic IC(0) of H = diag(d(w)) + beta C'C on every mask voxel of the full
    grid (2.1 M unknowns), with d of Eq. 10 formed voxel by voxel from the raw data."""
    vol = full
    w = _full_w(vol)
    set_threads(os.cpu_count() or 1)
    try:
        d = curv_raw(vol.y, vol.smap, vol.te, vol.mask, w)
    finally:
        set_threads(1)
    colptr, rowidx, val, umap = ic0_factor(vol.mask.shape, vol.mask, d, vol.beta)
    inv_piv = np.zeros(vol.mask.size)
    inv_piv[umap] = 1.0 / val[colptr[:-1]] ** 2  # pi_j = L_jj^2
    rng = np.random.default_rng(17)
    g = rng.standard_normal(vol.mask.shape) * vol.mask
    p = np.zeros(vol.mask.size)
    p[umap] = ic0_solve(colptr, rowidx, val, g.reshape(-1)[umap])
    return w, inv_piv.reshape(vol.mask.shape), g, p.reshape(vol.mask.shape)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_ic0_factor_and_apply_match_the_oracle(full, full_ic_ref, prec):
    """The bench's IC(0) path at full size -- 2.1 M unknowns, 8 x 8 x 16 tiles (30 tile
    levels), the forward sweep on one block per SM with streamed faces and the back
    substitution on two blocks per SM -- against the oracle's generic factor and triangular
    solves, element by element on every grid voxel."""
    vol = full
    w, ip_ref, g, p_ref = full_ic_ref
    fm = open_fm(vol, prec)
    ip = to_np(fm.ic_factor(to_dev(w, prec)))
    p = to_np(fm.ic_apply(to_dev(g, prec)))
    fm.close()
    tol_ip, tol_p = (1e-10, 1e-10) if prec == "fp64" else (3e-5, 2e-4)
    np.testing.assert_allclose(ip, ip_ref, rtol=tol_ip, atol=0)
    np.testing.assert_allclose(p, p_ref, rtol=0, atol=tol_p * np.abs(p_ref).max())


def test_full_size_fp32_pivot_pair_carries_the_recurrence_to_double_accuracy(full):
    """FP32 mode keeps each inverse pivot as a float pair hi + lo.  On the float curvature the
    factor actually used (fm_cost_grad's d at the same w, the same kernel and inputs), the
    pivots from fm_ic_factor64 must satisfy the IC(0) recurrence of Eq. 12,
    pi_j = d_j + beta n_j - beta^2 sum_{k lower in-mask neighbour} 1/pi_k, to about 1e-12
    relative at every voxel -- a float-only recurrence leaves residuals near 1e-7."""
    vol = full
    w = to_dev(_full_w(vol), "fp32")
    fm = open_fm(vol, "fp32")
    _, _, d = fm.cost_grad(w, want_cost=False, want_grad=False)
    ip64 = fm.ic_factor64(w).cpu().numpy()
    ip_hi = to_np(fm.ic_factor(w))
    fm.close()
    d = to_np(d)
    m = vol.mask.astype(bool)
    inv = np.where(m, ip64, 0.0)
    n = np.zeros(m.shape)
    lower = np.zeros(m.shape)
    for ax in range(3):
        lo_nb = np.zeros(m.shape, bool)
        sl_dst = [slice(None)] * 3
        sl_src = [slice(None)] * 3
        sl_dst[ax] = slice(1, None)
        sl_src[ax] = slice(None, -1)
        lo_nb[tuple(sl_dst)] = m[tuple(sl_src)]
        hi_nb = np.zeros(m.shape, bool)
        hi_nb[tuple(sl_src)] = m[tuple(sl_dst)]
        n += lo_nb & m
        n += hi_nb & m
        sh = np.zeros(m.shape)
        sh[tuple(sl_dst)] = inv[tuple(sl_src)]
        lower += np.where(lo_nb & m, sh, 0.0)
    pi = 1.0 / ip64[m]
    rhs = (d + vol.beta * n - vol.beta ** 2 * lower)[m]
    rel = np.abs(pi - rhs) / np.abs(pi)
    assert rel.max() < 1e-12, rel.max()
    # and the float hi alone is the float-rounded pair
    np.testing.assert_allclose(ip_hi[m], ip64[m], rtol=1e-6, atol=0)
