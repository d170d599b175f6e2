"""Pins of the oracle's red-black IC(0) (the labelled multicolour variant of Sec. III-B's
preconditioner): the factor reproduces P H P' on its pattern for the red-black permutation P,
and on the bipartite 6-neighbour grid every red column is the exact Cholesky column of H."""
import numpy as np

from oracle import Oracle, ic0_factor
from synth import make_volume
from test_oracle_pins import _grid_H, _L_sparse


def _rb_perm(shape, mask):
    """Mask voxels with x + y + z even (voxel order), then the odd ones: unknown indices into
    the natural-order numbering."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    par = ((x + y + z) % 2).reshape(-1)
    m = mask.reshape(-1).astype(bool)
    nat = np.flatnonzero(m)  # natural unknown u -> voxel
    order = np.concatenate([nat[par[nat] == 0], nat[par[nat] == 1]])
    pos = {v: i for i, v in enumerate(nat)}
    return np.array([pos[v] for v in order]), order


def _case(seed=5, shape=(5, 6, 7)):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=shape) > 0.25).astype(np.uint8)
    d = rng.uniform(0.0, 2.0, shape)
    return shape, mask, d, 0.7


def test_red_black_ic0_matches_the_permuted_H_on_its_pattern():
    shape, mask, d, beta = _case()
    colptr, rowidx, val, umap = ic0_factor(shape, mask, d, beta, order=1)
    perm, order = _rb_perm(shape, mask)
    np.testing.assert_array_equal(umap, order)
    L = _L_sparse(colptr, rowidx, val)
    H = _grid_H(shape, mask, d, beta)[perm][:, perm].tocoo()
    LLt = (L @ L.T).tocsc()
    diff = np.array([LLt[i, j] - v for i, j, v in zip(H.row, H.col, H.data)])
    assert np.max(np.abs(diff)) <= 1e-13 * np.max(np.abs(H.data))
    assert np.all(rowidx >= np.repeat(np.arange(colptr.size - 1), np.diff(colptr)))


def test_red_columns_are_exact_cholesky_columns():
    """Reds have no earlier neighbour in the red-black order, so each red column of L is
    H's column scaled by 1/sqrt(H_rr) with nothing subtracted, and the factor differs from
    the exact Cholesky factor of P H P' only in the black block."""
    shape, mask, d, beta = _case(seed=6)
    colptr, rowidx, val, umap = ic0_factor(shape, mask, d, beta, order=1)
    perm, order = _rb_perm(shape, mask)
    H = _grid_H(shape, mask, d, beta)[perm][:, perm].toarray()
    Lc = np.linalg.cholesky(H)
    L = _L_sparse(colptr, rowidx, val).toarray()
    nz, ny, nx = shape
    vox = order
    red = ((vox % nx + (vox // nx) % ny + vox // (nx * ny)) % 2) == 0
    nred = int(red.sum())
    assert np.all(red[:nred]) and not np.any(red[nred:])
    np.testing.assert_allclose(L[:, :nred], Lc[:, :nred], rtol=0, atol=1e-14 * np.abs(Lc).max())


def test_red_black_preconditioned_solve_decreases_the_cost():
    vol = make_volume(12, 10, 6, ncoil=2, snr_db=20.0, seed=8, fmax_hz=100.0, nblobs=2, dtype=np.complex128)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=12, nls=5, precond=3)
    c = r["cost"]
    assert np.all(np.diff(c) <= 1e-12 * np.abs(c[:-1]))
    assert c[-1] < c[0]
    g = o.grad(o.init())
    p = o.precondition(o.curv(o.init()), g, order=1)
    assert float(np.sum(g * p)) > 0  # (L L')^{-1} is positive definite
