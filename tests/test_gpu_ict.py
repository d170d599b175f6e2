"""IC with a drop tolerance on the GPU (FM_PC_ICT; Sec. III-B's L_t and the paper's
NCG-MLS-IC).  The factor is held on a set of grid offsets -- IC(0)'s plus the level-1 fill
offsets at first -- and grows, inside the calls that factor, until the drop tolerance keeps
nothing outside it; FM_ERR_FILL remains only beyond 64 offsets.  Checked here against the
oracle's generic left-looking threshold IC:

* Table 1's toy problem (20 x 16 x 8, d ~ U(0, 0.1), beta = 0.1, tolerance 1e-3 H_max),
  whose factor keeps fill at dozens of offsets: every entry, the pivots and the apply;
* volumes whose factor keeps fill beyond level 1 (previously reported as FM_ERR_FILL): the
  factor entry by entry, and the FP64 solve per iteration;
* the factor's inverse pivots and the apply, on volumes whose factor keeps level-1 fill
  (echoes 0/1/2.3 ms, tolerance 1e-2 H_max) and on volumes that keep none (echoes 0/2/10 ms,
  the paper's 1e-3 H_max), with grids spanning several columns' worth of levels and ragged
  edges;
* FM_ERR_FILL only where the kept fill needs more than 64 offsets (complete Cholesky);
* the solve's per-iteration cost against the oracle's solve with the same preconditioner,
  alone and inside a batch;
* the implicit-differentiation CG with this preconditioner reaches IC(0)'s solution;
* at full size (256x256x128, 8 coils, FP32), the pivots' recurrence at sampled voxels."""
import numpy as np
import pytest

from gpu_util import open_fm, to_dev, to_np
from oracle import Oracle, ict_factor
from synth import make_volume

pytestmark = pytest.mark.gpu

PHANTOM_TE = (0.0, 1.0, 2.3)
HELD = {(-1, 0, 0), (0, -1, 0), (0, 0, -1), (1, -1, 0), (1, 0, -1), (0, 1, -1)}
LEVEL1 = {(1, -1, 0), (1, 0, -1), (0, 1, -1)}

# (nx, ny, nz, ncoil, echo times, drop tolerance relative to H_max)
KEEPS_LEVEL1 = [(45, 33, 9, 4, PHANTOM_TE, 1e-2), (70, 37, 19, 2, PHANTOM_TE, 1e-2),
                (13, 9, 10, 3, PHANTOM_TE, 1e-2), (33, 1, 17, 2, PHANTOM_TE, 1e-2)]
KEEPS_NONE = [(70, 37, 19, 1, (0.0, 2.0, 10.0), 1e-3), (1, 1, 1, 1, (0.0, 2.0, 10.0), 1e-3)]
KEEPS_MORE = [(45, 33, 9, 4, PHANTOM_TE, 1e-3), (1, 40, 9, 2, PHANTOM_TE, 1e-2)]


def _vol(nx, ny, nz, nc, te):
    seed = {(45, 33, 9): 11, (70, 37, 19): 12 if te == PHANTOM_TE else 16, (13, 9, 10): 13, (1, 40, 9): 14,
            (33, 1, 17): 15}.get((nx, ny, nz), 17)
    return make_volume(nx, ny, nz, ncoil=nc, te=te, snr_db=20.0, seed=seed, fmax_hz=150.0, nblobs=3,
                       beta=2.0 ** -3)


def _offsets(shape, mask, d, beta, tau):
    """Offsets (column voxel - row voxel) of the oracle factor's off-diagonal entries."""
    colptr, rowidx, _, umap = ict_factor(shape, mask, d, beta, tau)
    nz, ny, nx = shape
    cols = np.repeat(np.arange(colptr.size - 1), np.diff(colptr))
    vi, vj = umap[rowidx], umap[cols]
    off = vi != vj

    def vec(a):
        return np.stack([a % nx, (a // nx) % ny, a // (nx * ny)], 1)
    return [tuple(int(t) for t in v) for v in vec(vj[off]) - vec(vi[off])]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", KEEPS_LEVEL1 + KEEPS_NONE)
def test_ict_factor_and_apply_match_oracle(prec, case):
    *dims, te, droptol = case
    vol = _vol(*dims, te)
    o = Oracle.from_volume(vol)
    rng = np.random.default_rng(5)
    w = o.init()
    g = rng.standard_normal(vol.mask.shape) * vol.mask
    d = o.curv(w)
    tau = droptol * o.hmax(d)
    offs = _offsets(o.shape, vol.mask, d, vol.beta, tau)
    assert all(v in HELD for v in offs)
    if case in KEEPS_LEVEL1:
        assert sum(v in LEVEL1 for v in offs) > 50  # the case exercises the fill entries
    colptr, rowidx, val, umap = ict_factor(o.shape, vol.mask, d, vol.beta, tau)
    ip_ref = np.zeros(vol.mask.size)
    ip_ref[umap] = 1.0 / val[colptr[:-1]] ** 2
    p_ref = o.precondition_ict(d, g, tau)
    fm = open_fm(vol, prec, precond="ict", droptol=droptol)
    wd = to_dev(w, prec)
    ip = to_np(fm.ic_factor(wd)).reshape(-1)
    p = to_np(fm.ic_apply(to_dev(g, prec)))
    fm.cost_grad(wd)  # synchronises: no FM_ERR_FILL, no FM_ERR_NOT_PD
    tol = 1e-11 if prec == "fp64" else 2e-4
    assert np.max(np.abs(ip - ip_ref)) <= tol * np.max(np.abs(ip_ref))
    assert np.max(np.abs(p - p_ref)) <= tol * np.max(np.abs(p_ref))
    assert np.all(p[vol.mask == 0] == 0)
    fm.close()


def _entries_match(fm, shape, colptr, rowidx, val, umap, tol):
    """The GPU factor as held (fm_ict_pattern) against the oracle's compressed columns, entry by
    entry: every oracle entry L_ij at its offset's plane, the diagonal as 1 / L_ii, and no
    other nonzero on the GPU side."""
    nz, ny, nx = shape
    off, planes = fm.ict_pattern()
    where = {tuple(int(t) for t in o): h for h, o in enumerate(off)}
    vec = lambda a: np.stack([a % nx, (a // nx) % ny, a // (nx * ny)], 1)
    cols = np.repeat(np.arange(colptr.size - 1), np.diff(colptr))
    vi, vj = umap[rowidx], umap[cols]
    diag = vi == vj
    scale = np.abs(val).max()
    np.testing.assert_allclose(planes[0].reshape(-1)[vi[diag]], 1.0 / val[diag], rtol=tol, atol=0)
    o = vec(vj[~diag]) - vec(vi[~diag])
    h = np.array([where[tuple(int(t) for t in v)] for v in o])  # KeyError: an entry outside the held pattern
    got = planes[1:].reshape(len(off), -1)[h, vi[~diag]]
    assert np.max(np.abs(got - val[~diag])) <= tol * scale
    assert int(np.count_nonzero(planes[1:])) == int((~diag).sum())
    return len(off)


def test_table1_toy_problem_factors_entry_by_entry():
    """Table 1's example: 20 x 16 x 8 grid, every voxel an unknown, d uniform on (0, 0.1), beta =
    0.1, drop tolerance 1e-3 H_max (reading 21).  Its factor keeps fill at dozens of offsets
    (far beyond level 1); the GPU's grown pattern must give the oracle's factor exactly."""
    from paper_2005_08661_gb300 import FieldMap
    import torch
    shape = (8, 16, 20)
    d = np.random.default_rng(2020).uniform(0.0, 0.1, shape)
    beta = 0.1
    te = (0.0, 2.0, 10.0)
    y0 = np.zeros((3, 1) + shape, np.complex128)
    o = Oracle(y0, None, te, None, beta)
    tau = 1e-3 * o.hmax(d)
    colptr, rowidx, val, umap = ict_factor(shape, None, d, beta, tau)
    g = np.random.default_rng(3).standard_normal(shape)
    p_ref = o.precondition_ict(d, g, tau)
    fm = FieldMap(20, 16, 8, ncoil=1, necho=3, precision="fp64", precond="ict", droptol=1e-3)
    fm.set_data(torch.zeros((3, 1) + shape, dtype=torch.complex128, device="cuda"), None, te,
                torch.ones(shape, dtype=torch.uint8, device="cuda"), beta)
    fm.ic_factor_curv(to_dev(d, "fp64"))
    nh = _entries_match(fm, shape, colptr, rowidx, val, umap, 1e-11)
    assert nh > 30  # the toy keeps fill at many offsets
    p = to_np(fm.ic_apply(to_dev(g, "fp64")))
    assert np.max(np.abs(p - p_ref)) <= 1e-11 * np.max(np.abs(p_ref))
    fm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", KEEPS_MORE)
def test_deeper_fill_factor_matches_the_oracle(prec, case):
    """Volumes whose factor keeps fill beyond level 1 (few coils, echoes 0/1/2.3 ms): the
    pattern grows to hold it and the factor, the pivots and the apply match the oracle."""
    *dims, te, droptol = case
    vol = _vol(*dims, te)
    o = Oracle.from_volume(vol)
    w = o.init()
    d = o.curv(w)
    tau = droptol * o.hmax(d)
    offs = _offsets(o.shape, vol.mask, d, vol.beta, tau)
    assert any(v not in HELD for v in offs)
    colptr, rowidx, val, umap = ict_factor(o.shape, vol.mask, d, vol.beta, tau)
    g = np.random.default_rng(5).standard_normal(vol.mask.shape) * vol.mask
    p_ref = o.precondition_ict(d, g, tau)
    fm = open_fm(vol, prec, precond="ict", droptol=droptol)
    wd = to_dev(w, prec)
    fm.ic_factor(wd)
    p = to_np(fm.ic_apply(to_dev(g, prec)))
    if prec == "fp64":
        _entries_match(fm, o.shape, colptr, rowidx, val, umap, 1e-11)
    tol = 1e-11 if prec == "fp64" else 2e-4
    assert np.max(np.abs(p - p_ref)) <= tol * np.max(np.abs(p_ref))
    fm.close()


def test_fp64_deeper_fill_solve_matches_oracle_per_iteration():
    """The solve grows the pattern as its iterates need and reruns from the same start: the
    per-iteration cost is the oracle's drop-tolerance solve's."""
    *dims, te, droptol = KEEPS_MORE[0]
    vol = _vol(*dims, te)
    o = Oracle.from_volume(vol)
    o.set_droptol(droptol)
    ref = o.solve(niter=12, nls=5, precond=4)
    fm = open_fm(vol, "fp64", precond="ict", droptol=droptol)
    w, cost = fm.solve(niter=12)
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-9)
    fm.close()


@pytest.mark.parametrize("droptol", [0.0, 1e-9])
def test_fill_beyond_the_largest_pattern_is_reported(droptol):
    """A tolerance of 0 is the complete Cholesky factor, whose fill spans the whole band: more
    offsets than the factor holds, so FM_ERR_FILL; the context stays usable."""
    from paper_2005_08661_gb300 import FmError, FM_ERR_FILL
    vol = _vol(45, 33, 17, 2, (0.0, 2.0, 10.0))
    o = Oracle.from_volume(vol)
    w = o.init()
    fm = open_fm(vol, "fp64", precond="ict", droptol=droptol)
    wd = to_dev(w, "fp64")
    with pytest.raises(FmError) as e:
        fm.ic_factor(wd)
    assert e.value.status == FM_ERR_FILL
    fm.cost_grad(wd)
    fm.close()


@pytest.mark.parametrize("case", [KEEPS_LEVEL1[0], KEEPS_LEVEL1[2], KEEPS_NONE[0]])
def test_fp64_ict_solve_matches_oracle_per_iteration(case):
    """A fill outside the held pattern at any iterate would raise FM_ERR_FILL here."""
    *dims, te, droptol = case
    vol = _vol(*dims, te)
    o = Oracle.from_volume(vol)
    o.set_droptol(droptol)
    ref = o.solve(niter=15, nls=5, precond=4)
    fm = open_fm(vol, "fp64", precond="ict", droptol=droptol)
    w, cost = fm.solve(niter=15)
    np.testing.assert_allclose(cost, ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(to_np(w), ref["w"], rtol=0, atol=1e-9)
    fm.close()


def test_fp32_ict_solve_decreases_the_cost():
    *dims, te, droptol = KEEPS_LEVEL1[1]
    vol = _vol(*dims, te)
    fm = open_fm(vol, "fp32", precond="ict", droptol=droptol)
    _, cost = fm.solve(niter=30)
    assert np.all(np.diff(cost) <= 2e-6 * np.abs(cost[:-1])) and cost[-1] < cost[0]
    fm.close()


def _nbr_count(mask):
    m = mask.astype(bool)
    n = np.zeros(m.shape, int)
    for ax in range(3):
        a = np.swapaxes(m, 0, ax)
        c = np.zeros(a.shape, int)
        c[1:] += a[:-1]
        c[:-1] += a[1:]
        n += np.swapaxes(c, 0, ax)
    return n * m


def test_full_size_pivots_follow_the_recurrence():
    """256x256x128, 8 coils, FP32, the paper's tolerance 1e-3 H_max: the data dominate H, so
    no fill survives and each column of IC(0) is kept or dropped whole: at sampled voxels the
    stored pivots obey pi_j = H_jj - beta^2 sum over the earlier in-mask neighbours k with
    beta / sqrt(pi_k) >= tau of 1/pi_k, with H_jj from the GPU's own curvature."""
    import torch
    from synth import full_config
    vol = full_config()
    fm = open_fm(vol, "fp32", precond="ict")
    w = fm.init_omega()
    _, _, d = fm.cost_grad(w, want_cost=False, want_grad=False, want_curv=True)
    ip = fm.ic_factor(w)
    fm.cost_grad(w)  # synchronising: FM_ERR_FILL / FM_ERR_NOT_PD would raise here
    torch.cuda.synchronize()
    ip = to_np(ip)
    d = to_np(d)
    mask = vol.mask > 0
    beta = vol.beta
    h = d + beta * _nbr_count(vol.mask)
    tau = 1e-3 * float(h[mask].max())
    kept = beta * np.sqrt(ip) >= tau
    zz, yy, xx = np.nonzero(mask)
    pick = np.random.default_rng(7).choice(zz.size, 20000, replace=False)
    s = np.zeros(pick.size)
    for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
        z, y, x = zz[pick] - dz, yy[pick] - dy, xx[pick] - dx
        ok = (z >= 0) & (y >= 0) & (x >= 0)
        z, y, x = np.where(ok, z, 0), np.where(ok, y, 0), np.where(ok, x, 0)
        ok &= mask[z, y, x] & kept[z, y, x]
        s += np.where(ok, ip[z, y, x], 0.0)
    pi = h[zz[pick], yy[pick], xx[pick]] - beta * beta * s
    rel = np.abs(1.0 / ip[zz[pick], yy[pick], xx[pick]] - pi) / pi
    assert rel.max() <= 2e-6
    frac = kept[mask].mean()
    assert 0.0 < frac < 0.5  # only the weakly weighted voxels' columns reach the tolerance
    fm.close()


def test_adjoint_solution_does_not_depend_on_the_preconditioner():
    """The implicit-differentiation CG (fm_adjoint_solve) with the drop-tolerance factor as its
    preconditioner reaches the same lambda = H_true^{-1} b as with IC(0): the preconditioner
    only changes the iteration count."""
    *dims, te, droptol = KEEPS_LEVEL1[2]
    vol = _vol(*dims, te)
    ref = open_fm(vol, "fp64")
    w, _ = ref.solve(niter=60)
    b = to_dev(np.random.default_rng(9).standard_normal(vol.mask.shape) * vol.mask, "fp64")
    lam0, it0, rr0 = ref.adjoint_solve(w, b, tol=1e-13, maxiter=3000)
    ref.close()
    fm = open_fm(vol, "fp64", precond="ict", droptol=droptol)
    lam1, it1, rr1 = fm.adjoint_solve(w, b, tol=1e-13, maxiter=3000)
    fm.close()
    assert rr0 <= 1e-13 and rr1 <= 1e-13
    l0, l1 = to_np(lam0), to_np(lam1)
    assert np.max(np.abs(l1 - l0)) <= 1e-9 * np.max(np.abs(l0))


def test_batched_drop_tolerance_solves_match_the_oracle_per_volume():
    """FieldMapBatch with the drop-tolerance preconditioner: each volume's per-iteration cost
    equals the oracle's solve of that volume alone (FP64)."""
    from paper_2005_08661_gb300 import FieldMapBatch
    from gpu_util import dev_inputs
    droptol = 1e-2
    cases = [KEEPS_LEVEL1[0], KEEPS_LEVEL1[2], KEEPS_NONE[0]]
    vols = [_vol(*c[:4], c[4]) for c in cases]
    refs = []
    for v in vols:
        o = Oracle.from_volume(v)
        o.set_droptol(droptol)
        refs.append(o.solve(niter=7, nls=5, precond=4))
    b = FieldMapBatch([(v.nx, v.ny, v.nz, v.ncoil, v.necho) for v in vols], precision="fp64", precond="ict",
                      droptol=droptol)
    keep = []
    for k, v in enumerate(vols):
        y, s, m = dev_inputs(v, "fp64")
        keep.append((y, s, m))
        b.set_data(k, y, s, v.te, m, v.beta)
    ws, costs = b.solve(niter=7)
    for k in range(len(vols)):
        np.testing.assert_allclose(costs[k], refs[k]["cost"], rtol=1e-10)
        np.testing.assert_allclose(to_np(ws[k]), refs[k]["w"], rtol=0, atol=1e-9)
    b.close()
