"""Pin of the oracle's Polak-Ribiere factor mu (Algorithm box; Sec. III-C).

The line search keeps the cost monotone whatever mu is, so the monotone-cost and descent
pins cannot see a wrong mu.  What the mathematics fixes instead: on a quadratic, nonlinear
CG with an exact line search and a fixed preconditioner M is preconditioned linear CG,
whose successive search directions are conjugate under the Hessian A,
    s_i' A s_{i-1} = 0,
and whose gradient collapses within about n iterations.  Near a noise-free minimiser the
cost is quadratic up to O(theta^2) (theta the phase residuals), the majoriser curvature of
Eq. 10-11 agrees with the true curvature to the same order, and so does the preconditioner
built from it; with many monotonic line-search steps the search is exact to rounding.  So
the oracle's steps s_i = w_{i+1} - w_i must be A-conjugate to within ~1e-6, with A the true
Hessian diag(h) + beta C'C at the minimiser.

The test also plants the plausible mistakes in copies of the oracle (mu = 0, mu with the
wrong sign, and the denominator g_i'p_i in place of g_{i-1}'p_{i-1}) and checks that each
of them fails the same property.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle.oracle import compile_oracle, load_oracle_variant, source_path

MU_LINE = "if (i > 0 && gp_prev != 0.0) mu = (gp - gprevp) / gp_prev;"
PLANTED = {
    "mu = 0": "mu = 0.0;",
    "sign of mu flipped": "if (i > 0 && gp_prev != 0.0) mu = -(gp - gprevp) / gp_prev;",
    "denominator g_i'p_i": "if (i > 0 && gp != 0.0) mu = (gp - gprevp) / gp;",
}
W_TRUE = 0.3  # rad/ms, constant: C w_true = 0, so w_true is the exact minimiser of Psi
TE = np.array([0.0, 2.0, 10.0])

# (grid, beta, preconditioner): IC(0) on a grid with cycles and a strong regulariser, so the
# incomplete factor is far from A; the diagonal and the identity on a smaller grid.
SETTINGS = [((3, 4, 5), 200.0, 0), ((2, 3, 4), 20.0, 1), ((2, 3, 4), 20.0, 2)]


def _steps_and_hessian(orc, shape, beta, precond, n=8, nls=40):
    """Iterates w_0..w_n of the oracle's solve from a start 0.002 rad/ms off the minimiser
    (every prefix is the same deterministic run), their steps, and A at the minimiser."""
    rng = np.random.default_rng(5)
    w0 = W_TRUE + 0.002 * rng.uniform(-1.0, 1.0, shape)
    ws = [w0.reshape(-1)]
    for k in range(1, n + 1):
        ws.append(orc.solve(w0=w0, niter=k, nls=nls, precond=precond)["w"].reshape(-1))
    A = np.diag(orc.hess_diag(np.full(shape, W_TRUE)).reshape(-1)) + beta * orc.laplacian().toarray()
    return np.diff(np.array(ws), axis=0), A, np.array([np.linalg.norm(orc.grad(w.reshape(shape))) for w in ws])


def _worst_conjugacy(steps, A):
    out = 0.0
    for i in range(1, steps.shape[0]):
        a, b = steps[i], steps[i - 1]
        na, nb = np.sqrt(a @ A @ a), np.sqrt(b @ A @ b)
        if na == 0.0 or nb == 0.0:
            break
        out = max(out, abs(a @ A @ b) / (na * nb))
    return out


def _oracle(shape, beta, lib=None):
    y = np.exp(1j * W_TRUE * TE)[:, None, None, None, None] * np.ones((TE.size, 1) + shape)
    return Oracle(y, None, TE, None, beta, lib=lib)


@pytest.mark.parametrize("shape,beta,precond", SETTINGS)
def test_successive_ncg_steps_are_conjugate_near_the_minimiser(shape, beta, precond):
    steps, A, g = _steps_and_hessian(_oracle(shape, beta), shape, beta, precond)
    assert _worst_conjugacy(steps[:7], A) < 1e-5
    # and linear CG's fast collapse of the gradient
    assert g[-1] < 1e-4 * g[0]


@pytest.fixture(scope="module")
def planted(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("planted"))
    src = open(source_path()).read()
    assert src.count(MU_LINE) == 1, "the oracle's mu line moved: update this pin"
    libs = {}
    for k, (name, line) in enumerate(PLANTED.items()):
        c = os.path.join(d, f"v{k}.c")
        open(c, "w").write(src.replace(MU_LINE, line))
        libs[name] = load_oracle_variant(compile_oracle(c, os.path.join(d, f"v{k}.so")))
    return libs


@pytest.mark.parametrize("name", list(PLANTED))
@pytest.mark.parametrize("shape,beta,precond", SETTINGS)
def test_each_planted_mistake_in_mu_fails_the_conjugacy_pin(planted, name, shape, beta, precond):
    steps, A, _ = _steps_and_hessian(_oracle(shape, beta, lib=planted[name]), shape, beta, precond)
    assert _worst_conjugacy(steps[:7], A) > 1e-2
