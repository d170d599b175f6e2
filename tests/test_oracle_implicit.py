"""Pins of the oracle pieces used for differentiating the converged field map: the true
Hessian diagonal and the image derivative of the gradient against central differences, and
the whole implicit gradient with respect to beta against differences of converged solves."""
import numpy as np

from oracle import Oracle
from synth import make_volume


def _vol(seed=3, nc=2):
    return make_volume(10, 9, 5, ncoil=nc, snr_db=20.0, seed=seed, fmax_hz=80.0, nblobs=2,
                       dtype=np.complex128)


def test_hessian_diagonal_matches_differences_of_the_gradient():
    vol = _vol()
    o = Oracle.from_volume(vol)
    w = o.init()
    h = o.hess_diag(w)
    eps = 1e-5
    fd = (o.grad_phi(w + eps) - o.grad_phi(w - eps)) / (2 * eps)  # voxelwise: grad_phi is separable
    m = vol.mask.astype(bool)
    np.testing.assert_allclose(h[m], fd[m], rtol=1e-6, atol=1e-6 * np.abs(h).max())


def test_image_derivative_of_the_gradient_matches_differences():
    vol = _vol(seed=5, nc=3)
    o = Oracle.from_volume(vol)
    w = o.init()
    rng = np.random.default_rng(2)
    dy = rng.standard_normal(vol.y.shape) + 1j * rng.standard_normal(vol.y.shape)
    an = o.dgrad_dy(w, dy)
    eps = 1e-6
    op = Oracle(vol.y + eps * dy, vol.smap, vol.te, vol.mask, vol.beta)
    om = Oracle(vol.y - eps * dy, vol.smap, vol.te, vol.mask, vol.beta)
    fd = (op.grad_phi(w) - om.grad_phi(w)) / (2 * eps)
    m = vol.mask.astype(bool)
    np.testing.assert_allclose(an[m], fd[m], rtol=1e-6, atol=1e-7 * np.abs(an).max())


def test_implicit_beta_gradient_matches_differences_of_converged_solves():
    vol = _vol(seed=7, nc=2)
    o = Oracle.from_volume(vol)
    r = o.solve(niter=120, nls=8)
    w_hat = r["w"]
    g = o.grad(w_hat)
    assert np.max(np.abs(g)) < 1e-9 * np.max(np.abs(o.grad(o.init())))  # converged
    target = vol.omega_true * vol.mask
    dl_dw = 2.0 * (w_hat - target) * vol.mask
    lam, dl_dbeta, _ = o.implicit_gradient(w_hat, dl_dw)
    eps = 1e-4 * vol.beta
    ls = []
    for sgn in (1, -1):
        ob = Oracle(vol.y, vol.smap, vol.te, vol.mask, vol.beta + sgn * eps)
        wb = ob.solve(w0=w_hat, niter=80, nls=8)["w"]
        ls.append(float(np.sum((wb - target) ** 2 * vol.mask)))
    fd = (ls[0] - ls[1]) / (2 * eps)
    assert abs(dl_dbeta - fd) <= 1e-5 * max(abs(fd), 1e-12) + 1e-9


def test_image_adjoint_is_the_transpose_of_the_directional_derivative():
    vol = _vol(seed=9, nc=3)
    o = Oracle.from_volume(vol)
    w = o.init()
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(w.shape) * vol.mask
    dy = rng.standard_normal(vol.y.shape) + 1j * rng.standard_normal(vol.y.shape)
    adj = o.dgrad_dy_adj(w, lam)
    lhs = float(np.sum(adj.real * dy.real + adj.imag * dy.imag))
    rhs = float(np.sum(lam * o.dgrad_dy(w, dy)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(rhs), 1.0) * 1e3
    # nothing flows to voxels outside the mask
    assert np.all(adj[:, :, vol.mask == 0] == 0)


def test_implicit_image_gradient_matches_differences_of_converged_solves():
    vol = _vol(seed=11, nc=2)
    o = Oracle.from_volume(vol)
    w_hat = o.solve(niter=120, nls=8)["w"]
    target = vol.omega_true * vol.mask
    lam, _, dl_dy = o.implicit_gradient(w_hat, 2.0 * (w_hat - target) * vol.mask)
    rng = np.random.default_rng(6)

    def loss_at(yp):
        ob = Oracle(yp, vol.smap, vol.te, vol.mask, vol.beta)
        wb = ob.solve(w0=w_hat, niter=80, nls=8)["w"]
        return float(np.sum((wb - target) ** 2 * vol.mask))

    for _ in range(2):
        v = rng.standard_normal(vol.y.shape) + 1j * rng.standard_normal(vol.y.shape)
        # central differences at h and h/2, Richardson-combined to cancel the h^2 error term
        d = []
        for h in (1e-4, 5e-5):
            d.append((loss_at(vol.y + h * v) - loss_at(vol.y - h * v)) / (2 * h))
        fd = (4.0 * d[1] - d[0]) / 3.0
        an = float(np.sum(dl_dy.real * v.real + dl_dy.imag * v.imag))
        assert abs(an - fd) <= 1e-7 * abs(fd) + 1e-10, (an, fd, d)
