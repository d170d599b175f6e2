"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against an independent fact, never against a retyped copy
of its own formula: the profiled-likelihood identity of Eq. 2 (min over x of Eq. 1's
least-squares cost), central finite differences, the majoriser inequality of Sec. III-C,
the IC(0) defining property (L L' = H on H's pattern), the printed counts of the toy
example (Table 1), closed forms for noise-free data and for beta = 0, and brute force.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import Oracle, ic0_factor, ic0_solve, voxel_terms
from synth import make_volume

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _grid_H(shape, mask, d, beta):
    """H = diag(d) + beta C'C over the mask voxels, built with scipy from the grid graph."""
    import scipy.sparse as sp
    nz, ny, nx = shape

    def lap1(n):
        if n == 1:
            return sp.csr_matrix((1, 1))
        e = sp.diags([np.ones(n - 1)], [1], shape=(n, n))
        a = sp.diags([np.ones(n)], [0]) * 0
        return (e + e.T + a).tocsr()

    ix, iy, iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    A = (sp.kron(iz, sp.kron(iy, lap1(nx))) + sp.kron(iz, sp.kron(lap1(ny), ix))
         + sp.kron(lap1(nz), sp.kron(iy, ix))).tocsr()  # adjacency, x fastest
    m = np.ones(nx * ny * nz, bool) if mask is None else mask.reshape(-1).astype(bool)
    A = A[m][:, m]
    deg = np.asarray(A.sum(axis=1)).ravel()
    return (sp.diags(d.reshape(-1)[m] + beta * deg) - beta * A).tocsc()


def _L_sparse(colptr, rowidx, val):
    import scipy.sparse as sp
    n = colptr.size - 1
    return sp.csc_matrix((val, rowidx, colptr), shape=(n, n))


# ---------------------------------------------------------------- Eq. 1 -> Eq. 2 (profiling)

def test_profiled_cost_equals_min_over_image_plus_constant():
    """Phi(w) (Eq. 2, with r of Eq. 3) = min_x Phi~(w, x) (Eq. 1) + an w-independent constant."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        nc, L = [(1, 2), (1, 3), (3, 3), (2, 4), (4, 3), (2, 6)][trial]
        te = np.sort(rng.uniform(0.0, 12.0, L))
        y = _rand_c(rng, L, nc)
        s = _rand_c(rng, nc) if nc > 1 else None
        sv = s if s is not None else np.ones(1)
        diffs = []
        for w in rng.uniform(-3.0, 3.0, 7):
            phi = voxel_terms(te, y, s, w)[0]
            # min over the complex image m of sum_{l,c} |y_cl - e^{i w t_l} s_c m|^2
            a = (np.exp(1j * w * te)[:, None] * sv[None, :]).reshape(-1, 1)
            m_hat, *_ = np.linalg.lstsq(a, y.reshape(-1), rcond=None)
            resid = float(np.sum(np.abs(y.reshape(-1) - a[:, 0] * m_hat[0]) ** 2))
            diffs.append(phi - resid)
        scale = float(np.sum(np.abs(y) ** 2) * max(1.0, np.sum(np.abs(sv) ** 2)))
        assert np.ptp(diffs) <= 1e-12 * scale, (trial, diffs)


# ---------------------------------------------------------------- Eq. 8 by finite differences

def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    nz, ny, nx, nc, L = 3, 4, 5, 2, 3
    te = np.array([0.0, 2.0, 10.0])
    y = _rand_c(rng, L, nc, nz, ny, nx)
    s = _rand_c(rng, nc, nz, ny, nx)
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.25).astype(np.uint8)
    o = Oracle(y, s, te, mask, beta=0.37)
    w = rng.uniform(-1.0, 1.0, (nz, ny, nx))
    g = o.grad(w)
    h = 1e-6
    fd = np.zeros_like(w)
    for j in range(w.size):
        e = np.zeros(w.size)
        e[j] = h
        fd.flat[j] = (o.cost(w.reshape(-1) + e) - o.cost(w.reshape(-1) - e)) / (2 * h)
    m = mask.astype(bool)
    np.testing.assert_allclose(g[m], fd[m], rtol=1e-6, atol=1e-6 * np.abs(g).max())
    assert np.all(g[~m] == 0.0)
    assert np.all(fd[~m] == 0.0)  # voxels outside the mask are not unknowns


# ---------------------------------------------------------------- Sec. III-C majoriser

def _one_voxel(te, y, s, beta=0.0):
    L, nc = y.shape
    return Oracle(y.reshape(L, nc, 1, 1, 1), None if s is None else s.reshape(nc, 1, 1, 1), te,
                  None, beta)


@pytest.mark.parametrize("curv", ["literal", "combined"])
@pytest.mark.parametrize("nc,L", [(1, 2), (1, 3), (2, 3), (3, 4)])
def test_huber_curvature_gives_a_majoriser(nc, L, curv):
    """q(w) = Phi(w0) + Phi'(w0)(w - w0) + d(w0)/2 (w - w0)^2 >= Phi(w) for all w, for the
    literal curvature of Eq. 10 and for the coil-combined variant."""
    rng = np.random.default_rng(100 + 10 * nc + L)
    te = np.concatenate([[0.0], np.sort(rng.uniform(0.5, 4.0, L - 1))])
    grid = np.linspace(-25.0, 25.0, 20001)
    for _ in range(12):
        y = _rand_c(rng, L, nc)
        s = _rand_c(rng, nc) if nc > 1 else None
        o = _one_voxel(te, y, s)
        o.set_curvature(curv)
        w0 = rng.uniform(-8.0, 8.0)
        f0, g0, d0 = o.phi([w0]), o.grad_phi([w0])[0, 0, 0], o.curv([w0])[0, 0, 0]
        ws = w0 + grid
        f = np.array([o.phi([w]) for w in ws[::20]])
        q = f0 + g0 * (ws[::20] - w0) + 0.5 * d0 * (ws[::20] - w0) ** 2
        assert np.all(q >= f - 1e-10 * (1 + abs(f0))), (w0, np.min(q - f))


def test_huber_curvature_is_the_smallest_majorising_curvature():
    """For one 1-cos term the sinc curvature touches the cost at the reflected angle, so any
    smaller curvature fails to majorise (this rejects wrap readings other than [-pi, pi])."""
    te = np.array([0.0, 1.0])
    rng = np.random.default_rng(3)
    for _ in range(20):
        y = _rand_c(rng, 2, 1)
        o = _one_voxel(te, y, None)
        w0 = rng.uniform(-9.0, 9.0)
        f0, g0, d0 = o.phi([w0]), o.grad_phi([w0])[0, 0, 0], o.curv([w0])[0, 0, 0]
        ang = np.angle(np.conj(y[0, 0]) * y[1, 0])  # angle of r_{1,1,1,2}
        th = ang + w0 * (te[0] - te[1])
        u = th - 2 * math.pi * np.round(th / (2 * math.pi))
        if abs(u) < 0.3:
            continue
        ws = w0 + np.linspace(-7.0, 7.0, 14001)
        f = np.array([o.phi([w]) for w in ws])
        q = f0 + g0 * (ws - w0) + 0.5 * 0.97 * d0 * (ws - w0) ** 2
        assert np.min(q - f) < -1e-9 * (1 + f0), (w0, u)


def test_line_search_majoriser_on_a_volume():
    """f(a) = Psi(w + a z) <= q_k(a) of Sec. III-C with d^(k) = sum_j z_j^2 d_j(w + a_k z)."""
    rng = np.random.default_rng(9)
    nz, ny, nx, nc = 3, 4, 5, 2
    te = np.array([0.0, 2.0, 10.0])
    y = _rand_c(rng, 3, nc, nz, ny, nx)
    s = _rand_c(rng, nc, nz, ny, nx)
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.2).astype(np.uint8)
    o = Oracle(y, s, te, mask, beta=0.5)
    w = rng.uniform(-1, 1, (nz, ny, nx)) * mask
    z = rng.uniform(-1, 1, (nz, ny, nx)) * mask
    for ak in (-0.7, 0.0, 0.4):
        wk = w + ak * z
        phik = o.phi(wk)
        gk = float(np.sum(z * o.grad_phi(wk)))
        dk = float(np.sum(z * z * o.curv(wk)))
        for a in np.linspace(ak - 6, ak + 6, 601):
            f = o.cost(w + a * z)
            q = phik + gk * (a - ak) + 0.5 * dk * (a - ak) ** 2 + o.reg(w + a * z)
            assert q >= f - 1e-10 * abs(f)


# ---------------------------------------------------------------- IC(0), Eq. 12, Table 1

def _e1_case():
    gold = json.load(open(os.path.join(GOLDEN, "e1_toy_ichol.json")))
    nx, ny, nz = gold["grid"]
    rng = np.random.default_rng(2005)
    d = rng.uniform(*gold["d_range"], size=(nz, ny, nx))
    return gold, (nz, ny, nx), d, gold["beta"]


def test_toy_example_nonzero_counts():
    """Table 1: nnz(H) = 1.67e4 and nnz(L_0) = 0.96e4 for the 20x16x8 toy problem."""
    gold, shape, d, beta = _e1_case()
    colptr, rowidx, val, umap = ic0_factor(shape, None, d, beta)
    nnz_L0 = int(np.count_nonzero(val))
    H = _grid_H(shape, None, d, beta)
    assert round(nnz_L0 / 1e4, 2) == gold["nnz_x1e4"]["L_0"]
    assert round(H.nnz / 1e4, 2) == gold["nnz_x1e4"]["H"]
    nv = d.size
    assert nnz_L0 <= 4 * nv
    assert H.nnz == 2 * nnz_L0 - nv  # same pattern, lower triangle plus diagonal


def test_toy_example_complete_cholesky():
    """Table 1 / Sec. III-B: L_c has >= (N_v - NxNy) NxNy nonzeros (72.5e4 printed), its
    inverse error is at round-off (3e-16 printed), and H^-1 is full (655e4)."""
    gold, shape, d, beta = _e1_case()
    nz, ny, nx = shape
    H = _grid_H(shape, None, d, beta).toarray()
    Lc = np.linalg.cholesky(H)
    nv = H.shape[0]
    nnz_c = int(np.count_nonzero(Lc))
    assert nnz_c >= (nv - nx * ny) * nx * ny
    assert round(nnz_c / 1e4, 1) == gold["nnz_x1e4"]["L_c"]
    assert round(np.count_nonzero(np.linalg.inv(H)) / 1e4) == gold["nnz_x1e4"]["Hinv"]
    Li = np.linalg.inv(Lc)
    nrmse = np.linalg.norm(np.eye(nv) - Li @ H @ Li.T) / math.sqrt(nv)
    assert nrmse < 10 * gold["nrmse"]["L_c"] * 10


def test_ic0_matches_H_on_its_pattern():
    """IC(0) 'matches H on its nonzero set' (Sec. III-B): (L L')_jk = H_jk on the pattern."""
    _, shape, d, beta = _e1_case()
    colptr, rowidx, val, umap = ic0_factor(shape, None, d, beta)
    L = _L_sparse(colptr, rowidx, val)
    H = _grid_H(shape, None, d, beta)
    LLt = (L @ L.T).tocsc()
    Hc = H.tocoo()
    diff = np.array([LLt[i, j] - v for i, j, v in zip(Hc.row, Hc.col, Hc.data)])
    assert np.max(np.abs(diff)) <= 1e-14 * np.max(np.abs(Hc.data))
    # and L is lower triangular with H's lower pattern
    assert np.all(rowidx >= np.repeat(np.arange(colptr.size - 1), np.diff(colptr)))


def test_ic0_on_a_masked_grid_with_holes():
    rng = np.random.default_rng(77)
    shape = (5, 6, 7)
    mask = (rng.uniform(size=shape) > 0.3).astype(np.uint8)
    d = rng.uniform(0.0, 3.0, shape)
    colptr, rowidx, val, umap = ic0_factor(shape, mask, d, 0.8)
    assert np.array_equal(umap, np.flatnonzero(mask.reshape(-1)))
    L = _L_sparse(colptr, rowidx, val)
    H = _grid_H(shape, mask, d, 0.8)
    LLt = (L @ L.T).tocsc()
    Hc = H.tocoo()
    diff = np.array([LLt[i, j] - v for i, j, v in zip(Hc.row, Hc.col, Hc.data)])
    assert np.max(np.abs(diff)) <= 1e-13 * np.max(np.abs(Hc.data))


def test_toy_example_ic0_inverse_error_band():
    """Table 1 prints NRMSE(L_0) = 3e-2; the stated formula gives about 0.1 here for every
    seed, so this entry is unpinned and only an order-of-magnitude band is checked."""
    _, shape, d, beta = _e1_case()
    colptr, rowidx, val, umap = ic0_factor(shape, None, d, beta)
    L = _L_sparse(colptr, rowidx, val).toarray()
    H = _grid_H(shape, None, d, beta).toarray()
    Li = np.linalg.inv(L)
    nrmse = np.linalg.norm(np.eye(H.shape[0]) - Li @ H @ Li.T) / math.sqrt(H.shape[0])
    assert 1e-2 < nrmse < 0.5


def test_ic0_is_exact_cholesky_on_a_line():
    """On an Nx x 1 x 1 line H is tridiagonal, IC(0) has no dropped fill, so it is the
    exact Cholesky factor and (L L')^-1 H g = g."""
    rng = np.random.default_rng(1)
    nx = 37
    d = rng.uniform(0.01, 2.0, (1, 1, nx))
    colptr, rowidx, val, umap = ic0_factor((1, 1, nx), None, d, 0.7)
    H = _grid_H((1, 1, nx), None, d, 0.7).toarray()
    np.testing.assert_allclose(_L_sparse(colptr, rowidx, val).toarray(), np.linalg.cholesky(H),
                               rtol=1e-13, atol=1e-14)
    g = rng.standard_normal(nx)
    np.testing.assert_allclose(ic0_solve(colptr, rowidx, val, H @ g), g, rtol=1e-11, atol=1e-12)


def test_ic0_with_zero_beta_is_sqrt_of_diagonal():
    rng = np.random.default_rng(2)
    d = rng.uniform(0.5, 2.0, (3, 4, 5))
    colptr, rowidx, val, umap = ic0_factor(d.shape, None, d, 0.0)
    L = _L_sparse(colptr, rowidx, val).toarray()
    np.testing.assert_allclose(np.diag(L), np.sqrt(d.reshape(-1)), rtol=1e-15)
    assert np.count_nonzero(L - np.diag(np.diag(L))) == 0


def test_ic0_reports_a_nonpositive_pivot():
    d = np.zeros((2, 3, 4))
    with pytest.raises(RuntimeError, match="-4"):
        ic0_factor(d.shape, None, d, 0.0)


# ---------------------------------------------------------------- closed forms

def test_noise_free_data_truth_is_a_zero_cost_stationary_point():
    """Noise-free y = e^{i w t} s x: Phi(w_true) = 0 (its minimum, Phi >= 0) with zero
    gradient, for any number of coils; Eq. 6 returns w_true when |w (t2 - t1)| < pi."""
    vol = make_volume(12, 10, 6, ncoil=3, snr_db=200.0, seed=4, fmax_hz=40.0,
                      dtype=np.complex128)
    o = Oracle.from_volume(vol)
    w = vol.omega_true * vol.mask
    scale = float(np.sum(np.abs(vol.y) ** 2))
    assert o.phi(w) <= 1e-9 * scale
    g = o.grad_phi(w)
    assert np.max(np.abs(g)) <= 1e-7 * np.sqrt(scale)
    w0 = o.init()
    m = vol.mask.astype(bool)
    np.testing.assert_allclose(w0[m], vol.omega_true[m], atol=1e-6)
    assert np.all(w0[~m] == 0.0)


def test_two_echo_init_is_the_per_voxel_minimiser_at_zero_beta():
    """With L = 2 and beta = 0, Eq. 6 zeroes the gradient and minimises Phi per voxel."""
    rng = np.random.default_rng(8)
    nz, ny, nx, nc = 2, 3, 4, 3
    te = np.array([0.0, 1.5])
    y = _rand_c(rng, 2, nc, nz, ny, nx)
    s = _rand_c(rng, nc, nz, ny, nx)
    o = Oracle(y, s, te, None, 0.0)
    w0 = o.init()
    g = o.grad_phi(w0)
    assert np.max(np.abs(g)) <= 1e-10 * np.max(np.abs(y)) ** 2 * 10
    assert np.all(o.curv(w0) > 0)
    for dw in (-0.3, 0.2, 1.0):
        assert o.phi(w0 + dw) >= o.phi(w0)


# ---------------------------------------------------------------- Algorithm box + MLS

def test_solve_is_monotone_at_every_inner_and_outer_step():
    vol = make_volume(16, 14, 6, ncoil=2, snr_db=12.0, seed=21, fmax_hz=150.0)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=8, nls=5, inner=True)
    seq = [r["cost"][0]]
    for i in range(8):
        seq.extend(r["inner"][i])
        assert r["cost"][i + 1] == pytest.approx(r["inner"][i][-1], rel=1e-14)
    seq = np.array(seq)
    assert np.all(np.diff(seq) <= 1e-13 * np.abs(seq[:-1]))
    assert r["cost"][-1] < r["cost"][0]
    assert r["mu"][0] == 0.0


def test_first_direction_is_a_descent_direction():
    vol = make_volume(12, 12, 5, ncoil=1, snr_db=20.0, seed=22)
    o = Oracle.from_volume(vol)
    w0 = o.init()
    g, d = o.grad(w0), o.curv(w0)
    p = o.precondition(d, g)
    assert float(np.sum(g * (-p))) < 0
    r = o.solve(niter=1, nls=5)
    assert r["alpha"][0] > 0  # z = -p, so the accepted step is positive


def test_many_line_search_steps_reach_the_line_minimum():
    """The MLS recursion converges to a stationary point of f(a) = Psi(w + a z) that is the
    minimum of a brute-force grid over the same basin."""
    vol = make_volume(10, 9, 4, ncoil=2, snr_db=20.0, seed=23, fmax_hz=100.0)
    o = Oracle.from_volume(vol)
    w0 = o.init()
    z = -o.precondition(o.curv(w0), o.grad(w0))
    r = o.solve(niter=1, nls=80)
    a = r["alpha"][0]
    grid = np.linspace(0.5 * a, 1.5 * a, 4001)
    f = np.array([o.cost(w0 + t * z) for t in grid])
    k = int(np.argmin(f))
    assert abs(grid[k] - a) <= 2 * (grid[1] - grid[0])
    assert o.cost(w0 + a * z) <= f[k] + 1e-12 * abs(f[k])
    assert r["cost"][1] == pytest.approx(o.cost(w0 + a * z), rel=1e-14)


def test_zero_beta_solve_reaches_the_brute_force_per_voxel_minimiser():
    """beta = 0 makes Psi separable; each voxel's minimiser is found by brute force on the
    profiled least-squares cost of Eq. 1 (period 2 pi / gcd(dt) = pi rad/ms for 0/2/10 ms)."""
    vol = make_volume(6, 5, 3, ncoil=2, snr_db=25.0, seed=24, fmax_hz=60.0, beta=0.0,
                      dtype=np.complex128)
    te = vol.te
    m = vol.mask.astype(bool)
    period = math.pi
    grid = np.linspace(-period / 2, period / 2, 100001)
    ybest = np.zeros(vol.mask.shape)
    for idx in zip(*np.nonzero(m)):
        yv = vol.y[(slice(None), slice(None)) + idx]            # [L][Nc]
        sv = vol.smap[(slice(None),) + idx]                      # [Nc]
        S = float(np.sum(np.abs(sv) ** 2))
        # profiled Eq. 1: sum|y|^2 - |sum conj(s) y e^{-i w t}|^2 / (L S)
        q = np.exp(-1j * np.outer(grid, te)) @ (np.conj(sv)[None, :] * yv).sum(axis=1)
        cost = -np.abs(q) ** 2
        k = int(np.argmin(cost))
        wb = grid[k]
        for _ in range(30):  # Newton polish on the same closed form
            e = np.exp(-1j * wb * te)
            b = (np.conj(sv)[None, :] * yv).sum(axis=1)
            qv = np.sum(e * b)
            dq = np.sum(-1j * te * e * b)
            d2q = np.sum(-(te ** 2) * e * b)
            f1 = -2 * np.real(np.conj(qv) * dq)
            f2 = -2 * (np.abs(dq) ** 2 + np.real(np.conj(qv) * d2q))
            wb -= f1 / f2
        ybest[idx] = wb
    o = Oracle.from_volume(vol)
    r = o.solve(w0=ybest + 0.02 * m, niter=40, nls=5)
    np.testing.assert_allclose(r["w"][m], ybest[m], atol=1e-7)


def test_combined_curvature_is_tighter_and_equal_for_one_coil():
    """The coil-combined curvature never exceeds the literal one (|sum| <= sum of moduli,
    sinc <= 1 on the wrapped angle) and equals it for one coil."""
    rng = np.random.default_rng(31)
    for nc in (1, 3):
        vol = make_volume(8, 7, 5, ncoil=nc, snr_db=10.0, seed=40 + nc)
        o = Oracle.from_volume(vol)
        w = o.init() + 0.1 * rng.standard_normal(vol.mask.shape) * vol.mask
        lit = o.curv(w)
        o.set_curvature("combined")
        comb = o.curv(w)
        if nc == 1:
            np.testing.assert_allclose(comb, lit, rtol=1e-12, atol=1e-14)
        else:
            assert np.all(comb <= lit * (1 + 1e-12) + 1e-14)
            assert np.any(comb < lit * (1 - 1e-6))


def test_noise_free_minimisers_repeat_with_the_gcd_of_the_echo_spacings():
    """Noise-free data: Phi_j vanishes exactly on w_true + k 2 pi / gcd(t_m - t_n) and only
    there (echoes 0/2/10 ms: spacings 2, 10, 8, gcd 2, period pi rad/ms)."""
    rng = np.random.default_rng(17)
    te = np.array([0.0, 2.0, 10.0])
    for nc in (1, 3):
        s = _rand_c(rng, nc) if nc > 1 else None
        sv = s if s is not None else np.ones(1)
        x = complex(rng.standard_normal(), rng.standard_normal())
        w_true = float(rng.uniform(-1.0, 1.0))
        y = (np.exp(1j * w_true * te)[:, None] * sv[None, :] * x).astype(np.complex128)
        period = 2 * np.pi / 2.0
        for k in (-3, -1, 0, 1, 2):
            assert abs(voxel_terms(te, y, s, w_true + k * period)[0]) <= 1e-11 * abs(x) ** 2
        grid = w_true + np.linspace(-period, period, 401)[1:-1]
        off = np.abs(((grid - w_true) / period) - np.rint((grid - w_true) / period)) > 1e-3
        vals = np.array([voxel_terms(te, y, s, w)[0] for w in grid[off]])
        assert vals.min() > 1e-9 * abs(x) ** 2
