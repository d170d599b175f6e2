"""Pins of the oracle's IC with a drop tolerance (Sec. III-B, the paper's L_t and the
preconditioner of NCG-MLS-IC) against what the definition fixes:

* tolerance 0 drops nothing, so the factor is the complete Cholesky factor (numpy);
* a tolerance above every entry drops every off-diagonal, leaving diag(sqrt(H_jj));
* for any tolerance, the left-looking factor is characterised column by column by three
  facts -- L L' = H on L's own pattern (diagonal included), every kept off-diagonal has
  magnitude >= tau, and every position left out holds a would-be entry
  (H - L L')_ij / L_jj of magnitude < tau -- which determine L uniquely by induction over
  the columns, so checking all three on a case that keeps fill-in and drops entries of H
  pins the whole routine;
* with a huge tolerance the NCG-MLS-IC solve is exactly the diagonally preconditioned
  solve (NCG-MLS-D).
"""
import numpy as np

from oracle import Oracle, ict_factor
from synth import make_volume
from test_oracle_pins import _grid_H, _L_sparse


def _case(seed=31, shape=(5, 6, 7), lo=0.1, hi=100.0, beta=0.7, hole=0.25):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=shape) > hole).astype(np.uint8)
    d = np.exp(rng.uniform(np.log(lo), np.log(hi), shape))  # spans heavy and light voxels
    return shape, mask, d, beta


def _dense_L(shape, mask, d, beta, tau):
    colptr, rowidx, val, umap = ict_factor(shape, mask, d, beta, tau)
    return _L_sparse(colptr, rowidx, val).toarray(), colptr, rowidx, umap


def test_zero_tolerance_gives_the_complete_cholesky_factor():
    shape, mask, d, beta = _case(seed=32, shape=(4, 5, 6))
    H = _grid_H(shape, mask, d, beta).toarray()
    L, colptr, rowidx, umap = _dense_L(shape, mask, d, beta, 0.0)
    Lc = np.linalg.cholesky(H)
    np.testing.assert_allclose(L, Lc, rtol=0, atol=1e-13 * np.abs(Lc).max())
    np.testing.assert_array_equal(umap, np.flatnonzero(mask.reshape(-1)))


def test_tolerance_above_every_entry_leaves_the_diagonal():
    shape, mask, d, beta = _case(seed=33)
    H = _grid_H(shape, mask, d, beta).toarray()
    L, colptr, rowidx, _ = _dense_L(shape, mask, d, beta, 1e30)
    assert colptr[-1] == H.shape[0]
    np.testing.assert_allclose(L, np.diag(np.sqrt(np.diag(H))), rtol=1e-15, atol=0)


def test_factor_obeys_the_drop_rule_and_reproduces_H_on_its_pattern():
    shape, mask, d, beta = _case(seed=34, shape=(6, 7, 8), hi=300.0)
    tau = 0.05
    H = _grid_H(shape, mask, d, beta).toarray()
    L, colptr, rowidx, _ = _dense_L(shape, mask, d, beta, tau)
    n = H.shape[0]
    pat = L != 0.0
    low = np.tril(np.ones((n, n), bool), -1)
    # the case exercises both halves of the rule: fill-in kept and entries of H dropped
    fill = pat & low & (H == 0.0)
    dropped_h = (~pat) & low & (H != 0.0)
    assert fill.sum() > 20 and dropped_h.sum() > 20, (fill.sum(), dropped_h.sum())
    R = H - L @ L.T
    scale = np.abs(H).max()
    assert np.abs(R[pat]).max() <= 1e-13 * scale  # L L' = H on L's pattern (lower, incl. diagonal)
    assert np.all(np.abs(L[pat & low]) >= tau)
    would_be = R / np.diag(L)[None, :]  # (H - L L')_ij / L_jj at the positions left out
    assert np.abs(would_be[(~pat) & low]).max() < tau
    # columns are stored diagonal first, rows ascending
    for j in range(n):
        rows = rowidx[colptr[j]:colptr[j + 1]]
        assert rows[0] == j and np.all(np.diff(rows) > 0)


def test_without_surviving_fill_the_factor_is_ic0_with_whole_columns_dropped():
    """When every would-be fill entry is below tau (the data-dominated regime of the field-map
    workloads), the generic factor keeps a subset of H's pattern.  Each column k of IC(0)
    holds the single value -beta / sqrt(pi_k) in all its off-diagonal rows, so the column
    is kept or dropped as a whole, and the pivots follow
    pi_j = H_jj - beta^2 sum_{earlier nbr k, beta / sqrt(pi_k) >= tau} 1 / pi_k."""
    shape, mask, d, beta = _case(seed=35, shape=(6, 7, 8), lo=20.0, hi=150.0, beta=0.5, hole=0.15)
    H = _grid_H(shape, mask, d, beta)
    tau = 0.07  # between beta / sqrt(H_jj) of light and heavy voxels, above every fill entry
    colptr, rowidx, val, umap = ict_factor(shape, mask, d, beta, tau)
    L = _L_sparse(colptr, rowidx, val).toarray()
    Hd = H.toarray()
    low = np.tril(np.ones(Hd.shape, bool), -1)
    assert not np.any((L != 0.0) & low & (Hd == 0.0))  # no fill survived
    kept = np.array([np.any(L[j + 1:, j] != 0.0) for j in range(L.shape[0])])
    later = np.array([np.any(Hd[j + 1:, j] != 0.0) for j in range(L.shape[0])])
    assert kept.sum() > 20 and (later & ~kept).sum() > 20
    # closed-form pivots in natural order over the grid
    nz, ny, nx = shape
    m = mask.reshape(-1).astype(bool)
    pi = np.zeros(m.size)
    for j in np.flatnonzero(m):
        x, y, z = j % nx, (j // nx) % ny, j // (nx * ny)
        nb = [k for k, ok in ((j - 1, x > 0), (j + 1, x < nx - 1), (j - nx, y > 0), (j + nx, y < ny - 1),
                              (j - nx * ny, z > 0), (j + nx * ny, z < nz - 1)) if ok and m[k]]
        s = sum(1.0 / pi[k] for k in nb if k < j and beta / np.sqrt(pi[k]) >= tau)
        pi[j] = d.reshape(-1)[j] + beta * len(nb) - beta * beta * s
    np.testing.assert_allclose(np.diag(L) ** 2, pi[umap], rtol=1e-14, atol=0)
    # and the kept columns are exactly those with beta / sqrt(pi_k) >= tau that have a later neighbour
    np.testing.assert_array_equal(kept, later & (beta / np.sqrt(pi[umap]) >= tau))


def test_preconditioner_applies_the_factor_inverse():
    vol = make_volume(9, 8, 5, ncoil=2, seed=36, snr_db=20.0, beta=2.0 ** -3)
    o = Oracle.from_volume(vol)
    w = o.init()
    d = o.curv(w)
    g = o.grad(w)
    tau = 1e-3 * o.hmax(d) * 0.05
    p = o.precondition_ict(d, g, tau)
    colptr, rowidx, val, umap = ict_factor(o.shape, vol.mask, d, vol.beta, tau)
    L = _L_sparse(colptr, rowidx, val)
    r = (L @ (L.T @ p.reshape(-1)[umap])) - g.reshape(-1)[umap]
    assert np.abs(r).max() <= 1e-12 * np.abs(g).max()
    assert np.all(p[vol.mask == 0] == 0.0)


def test_hmax_is_the_largest_entry_of_H():
    shape, mask, d, beta = _case(seed=37)
    vol_like = np.zeros((3, 1) + shape, np.complex128)
    vol_like[:] = 1.0
    o = Oracle(vol_like, None, np.array([0.0, 1.0, 2.0]), mask, beta)
    H = _grid_H(shape, mask, d, beta)
    assert o.hmax(d) == np.abs(H.toarray()).max()


def test_solve_with_a_tolerance_above_every_entry_is_the_diagonal_solve():
    vol = make_volume(10, 9, 6, ncoil=1, seed=38, snr_db=20.0, beta=2.0 ** -3)
    o = Oracle.from_volume(vol)
    o.set_droptol(1e30)
    a = o.solve(niter=6, precond=4)
    b = o.solve(niter=6, precond=1)
    np.testing.assert_allclose(a["cost"], b["cost"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(a["w"], b["w"], rtol=0, atol=1e-13 * np.abs(b["w"]).max())


def test_solve_with_the_papers_tolerance_is_monotone_and_beats_the_start():
    vol = make_volume(12, 10, 6, ncoil=2, seed=39, snr_db=20.0, beta=2.0 ** -3)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=12, precond=4, inner=True)
    c = r["cost"]
    assert np.all(np.diff(c) <= 1e-12 * abs(c[0]))
    assert c[-1] < c[0]
    ic0 = o.solve(niter=12, precond=0)["cost"]
    assert abs(c[-1] - ic0[-1]) <= 1e-3 * abs(ic0[0] - ic0[-1])  # same minimiser reached


def test_tolerance_between_fill_and_ic0_entries_gives_the_ic0_factor():
    """With the data dominating H, every would-be fill entry is far smaller than every entry of
    IC(0)'s factor; a tolerance between the two drops all fill and nothing else, so the
    threshold factor equals the generic IC(0) factor (a separate routine of the oracle)."""
    from oracle import ic0_factor
    shape, mask, d, beta = _case(seed=40, shape=(6, 5, 7), lo=50.0, hi=100.0, beta=0.3, hole=0.2)
    colptr0, rowidx0, val0, umap0 = ic0_factor(shape, mask, d, beta)
    L0 = _L_sparse(colptr0, rowidx0, val0).toarray()
    off = np.abs(L0[np.tril(np.ones(L0.shape, bool), -1) & (L0 != 0.0)])
    # largest would-be fill entry: beta^2 / (pi_k sqrt(pi_j)) < beta^2 / min(H)^1.5
    fill_bound = beta ** 2 / d[mask > 0].min() ** 1.5
    assert fill_bound < 0.5 * off.min()
    tau = 0.5 * (fill_bound + off.min())
    colptr, rowidx, val, umap = ict_factor(shape, mask, d, beta, tau)
    np.testing.assert_array_equal(umap, umap0)
    np.testing.assert_array_equal(colptr, colptr0)
    np.testing.assert_array_equal(rowidx, rowidx0)
    np.testing.assert_allclose(val, val0, rtol=1e-14, atol=0)
