"""Differentiation of the converged field map on the GPU (fm_true_curv, fm_adjoint_solve,
fm_implicit_grad and the torch.autograd wrappers), held to the FP64 oracle's implicit
gradient (a direct sparse solve with the true Hessian) and to finite differences of
converged solves."""
import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from oracle import Oracle
from synth import diff_config, make_volume

pytestmark = pytest.mark.gpu

CASES = {
    "c1": dict(nx=40, ny=34, nz=9, ncoil=1, seed=41),
    "c4": dict(nx=33, ny=29, nz=11, ncoil=4, seed=42),
}


def _vol(name):
    c = CASES[name]
    return make_volume(c["nx"], c["ny"], c["nz"], ncoil=c["ncoil"], snr_db=20.0, seed=c["seed"], fmax_hz=120.0,
                       nblobs=3)


@pytest.fixture(scope="module")
def converged():
    """Each case with the oracle's converged map and implicit gradient of
    l = ||w^ - w_true||^2 over the mask."""
    out = {}
    for name in CASES:
        vol = _vol(name)
        o = Oracle.from_volume(vol)
        w_hat = o.solve(niter=150, nls=8)["w"]
        target = vol.omega_true * vol.mask
        b = 2.0 * (w_hat - target) * vol.mask
        lam, dbeta, dy = o.implicit_gradient(w_hat, b)
        out[name] = dict(vol=vol, o=o, w_hat=w_hat, b=b, lam=lam, dbeta=dbeta, dy=dy)
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_true_curvature_matches_oracle(converged, name, prec):
    c = converged[name]
    vol = c["vol"]
    fm = open_fm(vol, prec)
    h = to_np(fm.true_curv(to_dev(c["w_hat"], prec)))
    ref = c["o"].hess_diag(c["w_hat"])
    tol = 1e-10 if prec == "fp64" else 1e-5  # FP32: phase rounding of w (t_m - t_n) up to 1e-6 rad
    assert np.max(np.abs(h - ref)) <= tol * np.max(np.abs(ref))
    assert np.all(h[vol.mask == 0] == 0)
    fm.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_adjoint_and_implicit_gradients_match_oracle(converged, name):
    c = converged[name]
    vol = c["vol"]
    fm = open_fm(vol, "fp64")
    w = to_dev(c["w_hat"], "fp64")
    lam, it, rr = fm.adjoint_solve(w, to_dev(c["b"], "fp64"), tol=1e-13, maxiter=3000)
    assert rr <= 1e-13 and 0 < it < 3000
    lam_np = to_np(lam)
    assert np.max(np.abs(lam_np - c["lam"])) <= 1e-9 * np.max(np.abs(c["lam"]))
    assert np.all(lam_np[vol.mask == 0] == 0)
    y, s, _ = dev_inputs(vol, "fp64")
    dy, dbeta = fm.implicit_grad(w, lam, y, s)
    assert abs(dbeta - c["dbeta"]) <= 1e-9 * abs(c["dbeta"])
    dy_np = dy.cpu().numpy()
    assert np.max(np.abs(dy_np - c["dy"])) <= 1e-9 * np.max(np.abs(c["dy"]))
    assert np.all(dy_np[:, :, vol.mask == 0] == 0)
    fm.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_adjoint_error_against_oracle(converged, name):
    """FP32 vectors, FP64 dot products: CG to a 1e-6 relative residual leaves lambda within
    1e-4 of the oracle's (the error is bounded by cond(H_true) times the residual and the
    FP32 rounding of h); dl/dbeta and dl/dy likewise."""
    c = converged[name]
    vol = c["vol"]
    fm = open_fm(vol, "fp32")
    w = to_dev(c["w_hat"], "fp32")
    lam, it, rr = fm.adjoint_solve(w, to_dev(c["b"], "fp32"), tol=1e-6, maxiter=1000)
    assert rr <= 1e-6
    lam_np = to_np(lam)
    assert np.linalg.norm(lam_np - c["lam"]) <= 1e-4 * np.linalg.norm(c["lam"])
    y, s, _ = dev_inputs(vol, "fp32")
    dy, dbeta = fm.implicit_grad(w, lam, y, s)
    assert abs(dbeta - c["dbeta"]) <= 1e-4 * abs(c["dbeta"])
    dy_np = dy.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(dy_np - c["dy"]) <= 1e-4 * np.linalg.norm(c["dy"])
    fm.close()


def test_adjoint_graph_replay_and_direct_launches_agree(converged):
    c = converged["c4"]
    vol = c["vol"]
    res = []
    for graph in (True, False):
        fm = open_fm(vol, "fp64", use_graph=graph)
        w = to_dev(c["w_hat"], "fp64")
        for _ in range(2):  # the second call replays the cached CG graph
            lam, it, rr = fm.adjoint_solve(w, to_dev(c["b"], "fp64"), tol=1e-10, maxiter=500)
            res.append((to_np(lam), it, rr))
        fm.close()
    for lam, it, rr in res[1:]:
        assert it == res[0][1] and rr == res[0][2]
        np.testing.assert_array_equal(lam, res[0][0])


def test_adjoint_edge_cases(converged):
    from paper_2005_08661_gb300 import FmError, FM_ERR_ARG, FM_ERR_NOT_PD
    c = converged["c1"]
    vol = c["vol"]
    fm = open_fm(vol, "fp64")
    w = to_dev(c["w_hat"], "fp64")
    zero = to_dev(np.zeros_like(c["b"]), "fp64")
    lam, it, rr = fm.adjoint_solve(w, zero)
    assert it == 0 and rr == 0.0 and float(lam.abs().max()) == 0.0
    b = to_dev(c["b"], "fp64")
    lam, it, rr = fm.adjoint_solve(w, b, tol=1e-14, maxiter=0)
    assert it == 0 and rr == 1.0 and float(lam.abs().max()) == 0.0
    lam, it, rr = fm.adjoint_solve(w, b, tol=1e-14, maxiter=3)  # limit reached: not an error
    assert it == 3 and rr > 1e-14
    for kw in (dict(tol=-1.0), dict(maxiter=-1)):
        with pytest.raises(FmError) as e:
            fm.adjoint_solve(w, b, **kw)
        assert e.value.status == FM_ERR_ARG
    fm.close()
    # beta = 0 and every phase residual moved by pi: H_true = diag(h) with h < 0 on the mask
    vol0 = make_volume(24, 20, 6, ncoil=1, snr_db=40.0, seed=43, fmax_hz=60.0, nblobs=2, beta=0.0)
    fm = open_fm(vol0, "fp64")
    dt = vol0.te[1] - vol0.te[0]
    w0 = to_dev((vol0.omega_true + np.pi / dt) * vol0.mask, "fp64")
    h = to_np(fm.true_curv(w0))
    assert np.mean(h[vol0.mask > 0] < 0) > 0.9
    with pytest.raises(FmError) as e:
        fm.adjoint_solve(w0, to_dev(np.ones(vol0.mask.shape) * vol0.mask, "fp64"))
    assert e.value.status == FM_ERR_NOT_PD
    fm.close()


def test_adjoint_empty_mask():
    vol = make_volume(16, 12, 5, ncoil=1, seed=44)
    empty = np.zeros_like(vol.mask)
    from paper_2005_08661_gb300 import FieldMap
    import torch
    fm = FieldMap(vol.nx, vol.ny, vol.nz, precision="fp64")
    y, s, _ = dev_inputs(vol, "fp64")
    fm.set_data(y, s, vol.te, torch.from_numpy(empty).cuda(), vol.beta)
    w = torch.zeros(vol.mask.shape, dtype=torch.float64, device="cuda")
    lam, it, rr = fm.adjoint_solve(w, torch.ones_like(w))
    assert it == 0 and float(lam.abs().max()) == 0.0
    dy, db = fm.implicit_grad(w, lam)
    assert db == 0.0 and float(dy.abs().max()) == 0.0
    fm.close()


def test_cost_autograd_gives_the_gradient_kernel_and_matches_differences(converged):
    import torch
    from paper_2005_08661_gb300 import field_map_cost
    c = converged["c4"]
    vol = c["vol"]
    fm = open_fm(vol, "fp64")
    rng = np.random.default_rng(5)
    w_np = (c["w_hat"] + 0.05 * rng.standard_normal(c["w_hat"].shape)) * vol.mask
    w = to_dev(w_np, "fp64").requires_grad_(True)
    psi = field_map_cost(w, fm)
    (g,) = torch.autograd.grad(2.0 * psi, w)
    _, g_ref, _ = fm.cost_grad(w.detach())
    np.testing.assert_array_equal(to_np(g), 2.0 * to_np(g_ref))
    assert abs(psi.item() - c["o"].cost(w_np)) <= 1e-10 * abs(c["o"].cost(w_np))
    for k in range(3):
        v = rng.standard_normal(w_np.shape) * vol.mask
        h = 1e-6
        fd = (c["o"].cost(w_np + h * v) - c["o"].cost(w_np - h * v)) / (2 * h)
        an = float(np.sum(to_np(g_ref) * v))
        assert abs(an - fd) <= 1e-6 * abs(fd)
    fm.close()


def _loss(w, target, mask):
    return float(((w - target) ** 2 * mask).sum())


def test_autograd_implicit_gradient_against_central_differences_full_size():
    """128x128x64, 8 coils, FP64: dl/dbeta and dl/dy along 16 random directions from one
    backward pass, against central differences of converged solves with step 1e-4
    (Richardson-combined with step 5e-5 to cancel the h^2 truncation term) to 1e-5
    relative.  The solves use the coil-combined curvature: the converged map, and with it
    every derivative checked here, does not depend on the majoriser, and the combined one
    makes the 68 FP64 solves several times cheaper."""
    import torch
    from paper_2005_08661_gb300 import FieldMap, field_map_solve
    vol = diff_config()
    y, s, m = dev_inputs(vol, "fp64")
    fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision="fp64",
                  curvature="combined")
    target = to_dev(vol.omega_true * vol.mask, "fp64")
    mask = m.double()
    yv = y.clone().requires_grad_(True)
    beta = torch.tensor(vol.beta, dtype=torch.float64, requires_grad=True)
    w_hat = field_map_solve(yv, beta, fm, s, vol.te, m, niter=400)
    _, g, _ = fm.cost_grad(w_hat.detach())
    _, g0, _ = fm.cost_grad(fm.init_omega())
    assert float(g.abs().max()) <= 1e-9 * float(g0.abs().max())  # converged
    loss = ((w_hat - target) ** 2 * mask).sum()
    dy, db = torch.autograd.grad(loss, (yv, beta))
    assert fm.last_adjoint["relres"] <= 1e-12
    w0 = w_hat.detach()

    def solve_loss(yp, bp):
        fm.set_data(yp, s, vol.te, m, bp)
        w, _ = fm.solve(w0, niter=150, want_history=False)
        return _loss(w, target, mask)

    def fd(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    fb = fd(lambda t: solve_loss(y, vol.beta * (1 + t)), 1e-4) / vol.beta
    assert abs(float(db) - fb) <= 1e-5 * abs(fb), (float(db), fb)
    gen = torch.Generator(device="cuda").manual_seed(7)
    scale = float(y.abs().pow(2).mean().sqrt())
    for k in range(16):
        v = torch.complex(torch.randn(y.shape, generator=gen, device="cuda", dtype=torch.float64),
                          torch.randn(y.shape, generator=gen, device="cuda", dtype=torch.float64)) * scale
        fv = fd(lambda t: solve_loss((y + t * v).contiguous(), vol.beta), 1e-4)
        an = float((dy.real * v.real + dy.imag * v.imag).sum())
        assert abs(an - fv) <= 1e-5 * abs(fv), (k, an, fv)
    fm.close()
