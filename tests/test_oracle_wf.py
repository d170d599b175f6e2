"""Pins of the oracle's water-fat pieces (Eq. gamma, Eq. 3 with complex Gamma, the voxel-wise
sweep and PWLS initialisation, and the amplitude recovery of Eq. wf) against facts the model
fixes: the projector identities, the profiled-likelihood identity against an independent
least-squares fit, exact recovery from noise-free data, and a direct sparse solve."""
import numpy as np

from oracle import Oracle, wf_gamma
from synth import fat_spectrum, make_wf_volume


def _wf(nx=7, ny=6, nz=4, ncoil=1, seed=21, noise=True, snr_db=25.0):
    return make_wf_volume(nx, ny, nz, ncoil=ncoil, seed=seed, snr_db=snr_db, noise=noise, dtype=np.complex128,
                          fmax_hz=150.0, nblobs=2)


def _oracle(vol):
    o = Oracle.from_volume(vol)
    g, G = wf_gamma(vol.te, vol.meta["fat_amps"], vol.meta["fat_freqs_khz"])
    o.set_gamma(G)
    return o, g, G


def test_gamma_is_the_orthogonal_projector_onto_the_water_fat_basis():
    amps, freqs, _ = fat_spectrum()
    te = np.array([1.2, 2.2, 3.2, 4.2, 5.2, 6.2])
    g, G = wf_gamma(te, amps, freqs)
    assert g.shape == (6, 2)
    np.testing.assert_allclose(G @ G, G, atol=1e-13)
    np.testing.assert_allclose(G, G.conj().T, atol=1e-14)
    np.testing.assert_allclose(G @ g, g, atol=1e-13)
    assert abs(np.trace(G) - 2.0) < 1e-13
    assert abs(amps.sum() - 1.0) < 1e-14
    # the one-column basis gamma = 1 gives the field-map weights 1/L
    one = np.ones((6, 1))
    np.testing.assert_allclose(one @ np.linalg.inv(one.T @ one) @ one.T, np.full((6, 6), 1 / 6), atol=1e-15)


def test_field_map_gamma_through_set_gamma_reproduces_the_default_weights():
    vol = _wf(ncoil=2, seed=22)
    o_def = Oracle.from_volume(vol)
    o_g = Oracle.from_volume(vol)
    o_g.set_gamma(np.full((vol.necho, vol.necho), 1.0 / vol.necho, np.complex128))
    rng = np.random.default_rng(1)
    w = rng.standard_normal(vol.mask.shape) * vol.mask
    assert abs(o_def.cost(w) - o_g.cost(w)) <= 1e-13 * abs(o_def.cost(w))
    np.testing.assert_allclose(o_g.grad(w), o_def.grad(w), rtol=0, atol=1e-12 * np.abs(o_def.grad(w)).max())


def _ls_residual(vol, g, w):
    """min over (m_w, m_f) of the Eq. 1 residual at field map w, per voxel, by an
    independent least-squares fit of the water-fat model."""
    L, nc = vol.necho, vol.ncoil
    out = np.zeros(vol.mask.shape)
    s = vol.smap if vol.smap is not None else np.ones((1,) + vol.mask.shape)
    for z, yy, x in np.argwhere(vol.mask > 0):
        B = np.zeros((L * nc, 2), np.complex128)
        b = np.zeros(L * nc, np.complex128)
        for l in range(L):
            for c in range(nc):
                B[l * nc + c] = np.exp(1j * w[z, yy, x] * vol.te[l]) * g[l] * s[c, z, yy, x]
                b[l * nc + c] = vol.y[l, c, z, yy, x]
        u, *_ = np.linalg.lstsq(B, b, rcond=None)
        out[z, yy, x] = np.sum(np.abs(B @ u - b) ** 2)
    return out


def test_profiled_likelihood_identity_with_the_water_fat_model():
    """Eq. 2 with the water-fat Gamma equals the minimum over water and fat of Eq. 1's
    residual up to a constant that does not depend on w (Sec. II)."""
    vol = _wf(ncoil=2, seed=23)
    o, g, _ = _oracle(vol)
    rng = np.random.default_rng(2)
    diffs = []
    for k in range(3):
        w = (vol.omega_true + 0.7 * rng.standard_normal(vol.mask.shape)) * vol.mask
        diffs.append(float(_ls_residual(vol, g, w).sum()) - o.phi(w))
    assert max(diffs) - min(diffs) <= 1e-10 * abs(np.mean(diffs)) + 1e-12


def test_noise_free_data_is_a_stationary_point_and_amplitudes_are_exact():
    vol = _wf(ncoil=2, seed=24, noise=False)
    o, g, _ = _oracle(vol)
    w = vol.omega_true * vol.mask
    gp = o.grad_phi(w)
    rng = np.random.default_rng(3)
    assert np.abs(gp).max() <= 1e-10 * np.abs(o.grad_phi(w + 0.3 * rng.standard_normal(w.shape) * vol.mask)).max()
    mw, mf = o.wf_amplitudes(w, g)
    m = vol.mask > 0
    np.testing.assert_allclose(mw[m], vol.meta["water"][m], atol=1e-12)
    np.testing.assert_allclose(mf[m], vol.meta["fat"][m], atol=1e-12)


def test_sweep_recovers_grid_field_values_from_noise_free_data():
    """With the true field map on the sweep grid, the voxel-wise sweep returns it exactly."""
    amps, freqs, _ = fat_spectrum()
    half = abs(freqs[np.argmax(amps)]) * np.pi  # |Delta_f / 2| in rad/ms
    grid = np.linspace(-half, half, 100)
    vol = _wf(ncoil=1, seed=25, noise=False)
    rng = np.random.default_rng(4)
    # rebuild the images with a field map drawn from the grid
    k_true = rng.integers(10, 90, size=vol.mask.shape)
    w_true = grid[k_true]
    x = vol.meta["water"][None] + vol.meta["fat"][None] * (
        np.exp(2j * np.pi * np.outer(vol.te, freqs)) @ amps)[:, None, None, None]
    y = (np.exp(1j * w_true[None] * vol.te[:, None, None, None]) * x)[:, None]
    o = Oracle(y, None, vol.te, vol.mask, vol.beta)
    o.set_gamma(wf_gamma(vol.te, amps, freqs)[1])
    ws = o.wf_sweep(100, -half, half)
    m = vol.mask > 0
    k = np.rint((ws + half) / (2 * half / 99)).astype(int)  # grid index of each chosen value
    np.testing.assert_array_equal(k[m], k_true[m])
    np.testing.assert_allclose(ws[m], w_true[m], rtol=0, atol=1e-14)
    assert np.all(ws[~m] == 0)


def _pwls_matrix(o, rho):
    import scipy.sparse as sp
    return (sp.diags(2.0 * rho.reshape(-1)) + o.beta * o.laplacian()).tocsr()


def test_pwls_cg_reaches_the_direct_solution_and_decreases_its_objective():
    import scipy.sparse.linalg as spla
    vol = _wf(nx=9, ny=8, nz=5, ncoil=1, seed=26)
    o, _, _ = _oracle(vol)
    half = 1.4
    wt = o.wf_sweep(100, -half, half)
    rho = o.rho()
    A = _pwls_matrix(o, rho)
    m = vol.mask.reshape(-1) > 0
    b = 2.0 * rho.reshape(-1) * wt.reshape(-1)
    direct = np.zeros(m.size)
    direct[m] = spla.spsolve(A[m][:, m].tocsc(), b[m])
    w_cg = o.pwls(wt, 400)
    np.testing.assert_allclose(w_cg.reshape(-1), direct, rtol=0, atol=1e-9 * np.abs(direct).max())

    def objective(w):
        w = w.reshape(-1)
        return float(np.sum(rho.reshape(-1) * (w - wt.reshape(-1)) ** 2)) + 0.5 * o.beta * float(
            w @ (o.laplacian() @ w))
    vals = [objective(o.pwls(wt, k)) for k in range(11)]
    assert all(vals[k + 1] <= vals[k] * (1 + 1e-14) for k in range(10))
    assert vals[10] < vals[0]


def test_rho_is_the_sum_of_pair_weight_moduli():
    """Single coil: |r_mn| = |Gamma_mn| |y_m| |y_n|, so rho = sum_mn |Gamma_mn| |y_m| |y_n|."""
    vol = _wf(ncoil=1, seed=27)
    o, _, G = _oracle(vol)
    a = np.abs(vol.y[:, 0])  # [L][z][y][x]
    ref = np.einsum("mn,mzyx,nzyx->zyx", np.abs(G), a, a) * vol.mask
    np.testing.assert_allclose(o.rho(), ref, rtol=1e-13, atol=0)
