"""Parity at the full 256x256x128, 8-coil workload, in the launch configuration bench.py
times (FP32, IC(0), N_ls = 5, captured graph).

The FP64 oracle cannot run a whole solve at this size, so the check uses sampled outputs:
after a few NCG iterations on the GPU, the gradient and Huber curvature at sampled mask
voxels (interior and mask-boundary) are compared with the oracle evaluated on each
voxel's 3x3x3 neighbourhood, which holds every input the voxel's gradient needs (its
data and its six stencil neighbours).  The cost history must be finite and, up to FP32
rounding of the cost, non-increasing (monotonic line search, Sec. III-C).
"""
import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from oracle import Oracle
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


def test_full_size_fp64_cost_grad_sampled_parity(full):
    vol = full
    fm32 = open_fm(vol, "fp32")
    w0 = to_np(fm32.init_omega())
    fm32.close()
    rng = np.random.default_rng(3)
    w = (w0 + 0.02 * rng.standard_normal(w0.shape)) * vol.mask
    fm = open_fm(vol, "fp64")
    _, g, d = fm.cost_grad(to_dev(w, "fp64"))
    g_np, d_np = to_np(g), to_np(d)
    gmax = np.abs(g_np).max()
    for (z, y, x) in _sample_voxels(vol.mask, 24, seed=11):
        g_ref, d_ref = _oracle_at(vol, w, z, y, x)
        assert abs(g_np[z, y, x] - g_ref) <= TOL["fp64"]["g"] * gmax, (z, y, x)
        assert abs(d_np[z, y, x] - d_ref) <= TOL["fp64"]["d"] * max(abs(d_ref), 1e-3 * d_np.max()), (z, y, x)
    fm.close()
