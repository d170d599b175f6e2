"""ctypes binding of the FP64 C oracle (test infrastructure only; see fm_oracle.c)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

ORC_OK, ORC_ERR_ARG, ORC_ERR_NOT_PD, ORC_ERR_OOM = 0, -1, -4, -7

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib_path():
    return os.path.join(_BUILD, "liboracle.so")


def source_path():
    return _SRC


def compile_oracle(src, out):
    """Compile a C source of the oracle (fm_oracle.c or a test's modified copy) into the shared
    library out, with plain IEEE double semantics (no fused contractions) and OpenMP when the
    compiler has it (the results do not depend on it: see orc_set_threads)."""
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, src, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.check_call(base + ["-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def set_threads(n):
    """Host threads the oracle uses (1 = serial); returns the count in effect (1 without
    OpenMP).  Results are bitwise the same for every count."""
    return int(_lib().orc_set_threads(int(n)))


def get_threads():
    return int(_lib().orc_get_threads())


def build_oracle(force=False):
    """Compile fm_oracle.c into oracle/_build/liboracle.so unless it is up to date."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    return compile_oracle(_SRC, out)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _declare(C.CDLL(build_oracle()))
        return _LIB


def load_oracle_variant(path):
    """Load another build of fm_oracle.c (e.g. a copy with a planted mistake, compiled by a
    test) with the same signatures; pass it to Oracle(..., lib=...)."""
    return _declare(C.CDLL(path))


def _declare(lib):
    vp = C.c_void_p
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_set_threads.restype = C.c_int
    lib.orc_get_threads.argtypes = []
    lib.orc_get_threads.restype = C.c_int
    lib.orc_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               _dp, vp, _dp, vp, C.c_double]
    lib.orc_create.restype = C.c_int
    lib.orc_destroy.argtypes = [vp]
    for name in ("orc_phi", "orc_reg", "orc_cost"):
        getattr(lib, name).argtypes = [vp, _dp]
        getattr(lib, name).restype = C.c_double
    for name in ("orc_grad", "orc_grad_phi", "orc_curv"):
        getattr(lib, name).argtypes = [vp, _dp, _dp]
        getattr(lib, name).restype = None
    lib.orc_init.argtypes = [vp, _dp]
    lib.orc_hess_diag.argtypes = [vp, _dp, _dp]
    lib.orc_hess_diag.restype = None
    lib.orc_dgrad_dy.argtypes = [vp, _dp, _dp, _dp]
    lib.orc_dgrad_dy.restype = None
    lib.orc_dgrad_dy_adj.argtypes = [vp, _dp, _dp, _dp]
    lib.orc_dgrad_dy_adj.restype = None
    lib.orc_set_gamma.argtypes = [vp, _dp]
    lib.orc_set_gamma.restype = C.c_int
    lib.orc_phi_vox.argtypes = [vp, _dp, _dp]
    lib.orc_phi_vox.restype = None
    lib.orc_rho.argtypes = [vp, _dp]
    lib.orc_rho.restype = None
    lib.orc_wf_sweep.argtypes = [vp, C.c_int, C.c_double, C.c_double, _dp]
    lib.orc_wf_sweep.restype = None
    lib.orc_pwls.argtypes = [vp, _dp, C.c_int, _dp]
    lib.orc_pwls.restype = C.c_int
    lib.orc_set_curvature.argtypes = [vp, C.c_int]
    lib.orc_set_curvature.restype = None
    lib.orc_num_unknowns.argtypes = [vp]
    lib.orc_num_unknowns.restype = C.c_long
    lib.orc_precondition.argtypes = [vp, _dp, _dp, _dp]
    lib.orc_precondition.restype = C.c_int
    lib.orc_solve.argtypes = [vp, _dp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
    lib.orc_solve.restype = C.c_int
    lib.orc_ic0.argtypes = [C.c_int, C.c_int, C.c_int, vp, _dp, C.c_double, _lp, _lp, _dp,
                            _lp, C.POINTER(C.c_long), C.POINTER(C.c_long)]
    lib.orc_ic0.restype = C.c_int
    lib.orc_ic0_solve.argtypes = [C.c_long, _lp, _lp, _dp, _dp, _dp]
    lib.orc_ic0_ordered.argtypes = [C.c_int, C.c_int, C.c_int, vp, _dp, C.c_double, C.c_int, _lp, _lp, _dp,
                                    _lp, C.POINTER(C.c_long), C.POINTER(C.c_long)]
    lib.orc_ic0_ordered.restype = C.c_int
    lib.orc_precondition_ordered.argtypes = [vp, _dp, _dp, _dp, C.c_int]
    lib.orc_precondition_ordered.restype = C.c_int
    lpp = C.POINTER(C.POINTER(C.c_long))
    dpp = C.POINTER(C.POINTER(C.c_double))
    lib.orc_ict.argtypes = [C.c_int, C.c_int, C.c_int, vp, _dp, C.c_double, C.c_double, lpp, lpp, dpp, lpp,
                            C.POINTER(C.c_long), C.POINTER(C.c_long)]
    lib.orc_ict.restype = C.c_int
    lib.orc_free.argtypes = [vp]
    lib.orc_free.restype = None
    lib.orc_hmax.argtypes = [vp, _dp]
    lib.orc_hmax.restype = C.c_double
    lib.orc_set_droptol.argtypes = [vp, C.c_double]
    lib.orc_set_droptol.restype = None
    lib.orc_precondition_ict.argtypes = [vp, _dp, _dp, _dp, C.c_double]
    lib.orc_precondition_ict.restype = C.c_int
    lib.orc_voxel.argtypes = [C.c_int, C.c_int, _dp, _dp, vp, C.c_double, _dp]
    lib.orc_voxel.restype = C.c_int
    lib.orc_voxel_r.argtypes = [C.c_int, C.c_int, _dp, vp, _dp, _dp]
    lib.orc_voxel_r.restype = C.c_int
    lib.orc_curv_raw.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, vp, _dp, vp, _dp, _dp]
    lib.orc_curv_raw.restype = C.c_int
    return lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """FP64 oracle bound to one volume.

    y: complex [L][N_c][nz][ny][nx]; smap: complex [N_c][nz][ny][nx] or None (s = 1);
    te: [L]; mask: uint8 [nz][ny][nx] or None; beta: Eq. 5 weight.  Field maps are
    float64 arrays of the grid's shape.
    """

    def __init__(self, y, smap, te, mask, beta, lib=None):
        lib = lib or _lib()
        y = np.asarray(y)
        L, nc, nz, ny, nx = y.shape
        self.shape = (nz, ny, nx)
        self.nc, self.L = nc, L
        self.beta = float(beta)
        self.te = np.ascontiguousarray(te, dtype=np.float64)
        self._y = _c128(y)
        self._yshape = y.shape
        self._s = _c128(smap) if smap is not None else None
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self.mask = (np.ones(self.shape, np.uint8) if mask is None else self._mask.reshape(self.shape))
        h = C.c_void_p()
        st = lib.orc_create(C.byref(h), nx, ny, nz, nc, L, self._y.reshape(-1), _ptr(self._s),
                            self.te, _ptr(self._mask), self.beta)
        if st != ORC_OK:
            raise RuntimeError(f"orc_create failed: {st}")
        self._h = h
        self._lib = lib

    @classmethod
    def from_volume(cls, vol):
        return cls(vol.y, vol.smap, vol.te, vol.mask, vol.beta)

    def set_gamma(self, G):
        """Water-fat model (Eq. gamma): use the complex L x L matrix G in place of 1/L in
        Eq. 3 (see wf_gamma)."""
        G = np.ascontiguousarray(G, dtype=np.complex128)
        assert G.shape == (self.L, self.L)
        st = self._lib.orc_set_gamma(self._h, G.view(np.float64).reshape(-1))
        if st != ORC_OK:
            raise RuntimeError(f"orc_set_gamma failed: {st}")
        self.gamma = G

    def phi_vox(self, w):
        """Phi_j(w_j) of Eq. 2 per voxel."""
        return self._vec("orc_phi_vox", w)

    def rho(self):
        """PWLS weights rho_j = sum |r_cdmnj| (Eq. w0_wf)."""
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        self._lib.orc_rho(self._h, out)
        return out.reshape(self.shape)

    def wf_sweep(self, nsweep, wlo, whi):
        """Voxel-wise minimiser of Phi_j over nsweep equally spaced values in [wlo, whi]."""
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        self._lib.orc_wf_sweep(self._h, int(nsweep), float(wlo), float(whi), out)
        return out.reshape(self.shape)

    def pwls(self, wt, niter):
        """niter CG iterations on the PWLS initialisation (Eq. w0_wf) from wt."""
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        st = self._lib.orc_pwls(self._h, self._w(wt), int(niter), out)
        if st != ORC_OK:
            raise RuntimeError(f"orc_pwls failed: {st}")
        return out.reshape(self.shape)

    def wf_amplitudes(self, w, gamma_cols):
        """Water and fat components by the closed form of Eq. wf: per mask voxel, the least-
        squares solution u of ((gamma diag(e^{i w t})) kron s_j) u = y_j, with the matrix
        formed literally and solved by numpy's pseudo-inverse.  Returns (m_w, m_f)."""
        gcols = np.asarray(gamma_cols, dtype=np.complex128)
        L, nc = self.L, self.nc
        w = np.asarray(w, dtype=np.float64).reshape(-1)
        m = self.mask.reshape(-1).astype(bool)
        idx = np.nonzero(m)[0]
        y = self._y.view(np.complex128).reshape(L, nc, -1)[:, :, idx]  # [L][nc][nm]
        s = (self._s.view(np.complex128).reshape(nc, -1)[:, idx] if self._s is not None
             else np.ones((nc, idx.size), np.complex128))
        ph = np.exp(1j * w[idx][None, :] * self.te[:, None])  # [L][nm]
        # B[j, (l, c), k] = e^{i w_j t_l} gamma_lk s_cj
        B = (ph[:, None, None, :] * gcols[:, None, :, None] * s[None, :, None, :])  # [L][nc][2][nm]
        B = np.moveaxis(B, 3, 0).reshape(idx.size, L * nc, gcols.shape[1])
        yv = np.moveaxis(y, 2, 0).reshape(idx.size, L * nc)
        u = np.einsum("jkq,jq->jk", np.linalg.pinv(B), yv)
        out_w = np.zeros(m.size, np.complex128)
        out_f = np.zeros(m.size, np.complex128)
        out_w[idx] = u[:, 0]
        out_f[idx] = u[:, 1]
        return out_w.reshape(self.shape), out_f.reshape(self.shape)

    def set_curvature(self, mode):
        """'literal' (Eq. 10, default) or 'combined' (the labelled coil-combined variant)."""
        self._lib.orc_set_curvature(self._h, {"literal": 0, "combined": 1}[mode])

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _w(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.size == int(np.prod(self.shape))
        return w.reshape(-1)

    def phi(self, w):
        return self._lib.orc_phi(self._h, self._w(w))

    def reg(self, w):
        return self._lib.orc_reg(self._h, self._w(w))

    def cost(self, w):
        return self._lib.orc_cost(self._h, self._w(w))

    def _vec(self, fn, w):
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        getattr(self._lib, fn)(self._h, self._w(w), out)
        return out.reshape(self.shape)

    def grad(self, w):
        return self._vec("orc_grad", w)

    def grad_phi(self, w):
        return self._vec("orc_grad_phi", w)

    def curv(self, w):
        return self._vec("orc_curv", w)

    def hess_diag(self, w):
        """Diagonal of the data term's true Hessian (second derivative of Eq. 2)."""
        return self._vec("orc_hess_diag", w)

    def dgrad_dy(self, w, dy):
        """Directional derivative of grad Phi (Eq. 8) with respect to the images, direction dy."""
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        d = _c128(dy).reshape(-1)
        assert d.size == self._y.size
        self._lib.orc_dgrad_dy(self._h, self._w(w), d, out)
        return out.reshape(self.shape)

    def dgrad_dy_adj(self, w, lam):
        """sum_j lam_j grad_y (grad Phi)_j, complex [L][Nc][z][y][x] (d/dRe y + i d/dIm y)."""
        out = np.zeros(self._y.size, np.float64)
        self._lib.orc_dgrad_dy_adj(self._h, self._w(w), self._w(lam), out)
        return out.view(np.complex128).reshape(self._yshape)

    def laplacian(self):
        """C'C over the mask voxels as a scipy sparse matrix on the grid (identity rows outside)."""
        import scipy.sparse as sp
        nz, ny, nx = self.shape
        m = self.mask.reshape(-1).astype(bool)
        idx = np.arange(m.size).reshape(self.shape)
        rows, cols = [], []
        for ax, n in ((2, nx), (1, ny), (0, nz)):
            a = np.take(idx, np.arange(n - 1), axis=ax).reshape(-1)
            b = np.take(idx, np.arange(1, n), axis=ax).reshape(-1)
            keep = m[a] & m[b]
            rows.append(a[keep])
            cols.append(b[keep])
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        A = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(m.size, m.size)).tocsr()
        A = A + A.T
        deg = np.asarray(A.sum(axis=1)).ravel()
        return (sp.diags(deg) - A).tocsr()

    def implicit_gradient(self, w_hat, dl_dw):
        """Implicit differentiation of the converged map: solve H lam = dl/dw with the true
        Hessian H = diag(hess_diag) + beta C'C on the mask voxels (scipy direct solve);
        returns (lam, dl/dbeta = -lam' C'C w_hat, dl/dy = -sum_j lam_j grad_y (grad Phi)_j)."""
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        m = self.mask.reshape(-1).astype(bool)
        Lap = self.laplacian()
        H = (sp.diags(self.hess_diag(w_hat).reshape(-1)) + self.beta * Lap).tocsr()
        Hm = H[m][:, m].tocsc()
        v = np.ascontiguousarray(dl_dw, dtype=np.float64).reshape(-1)
        lam = np.zeros(m.size)
        lam[m] = spla.spsolve(Hm, v[m])
        dl_dbeta = -float(lam @ (Lap @ np.ascontiguousarray(w_hat, np.float64).reshape(-1)))
        lam = lam.reshape(self.shape)
        return lam, dl_dbeta, -self.dgrad_dy_adj(w_hat, lam)

    def init(self):
        out = np.zeros(int(np.prod(self.shape)), np.float64)
        self._lib.orc_init(self._h, out)
        return out.reshape(self.shape)

    def precondition(self, d, g, order=0):
        """(L L')^{-1} g with the IC(0) factor of diag(d) + beta C'C; order 0 natural, 1 red-black."""
        p = np.zeros(int(np.prod(self.shape)), np.float64)
        st = self._lib.orc_precondition_ordered(self._h, self._w(d), self._w(g), p, int(order))
        if st != ORC_OK:
            raise RuntimeError(f"orc_precondition failed: {st}")
        return p.reshape(self.shape)

    def precondition_ict(self, d, g, tau):
        """(L L')^{-1} g with the drop-tolerance IC factor (absolute tolerance tau) of
        diag(d) + beta C'C (Sec. III-B, L_t)."""
        p = np.zeros(int(np.prod(self.shape)), np.float64)
        st = self._lib.orc_precondition_ict(self._h, self._w(d), self._w(g), p, float(tau))
        if st != ORC_OK:
            raise RuntimeError(f"orc_precondition_ict failed: {st}")
        return p.reshape(self.shape)

    def hmax(self, d):
        """H_max of Sec. III-B: the largest |H_jk| of diag(d) + beta C'C on the mask."""
        return float(self._lib.orc_hmax(self._h, self._w(d)))

    def set_droptol(self, droptol):
        """Drop tolerance of solve(precond=4), relative to each iteration's H_max."""
        self._lib.orc_set_droptol(self._h, float(droptol))

    def solve(self, w0=None, niter=10, nls=5, precond=0, inner=False):
        """Run the NCG-MLS solve; returns dict(w, cost, alpha, mu[, inner])."""
        w = np.zeros(int(np.prod(self.shape)), np.float64) if w0 is None else self._w(w0).copy()
        cost = np.zeros(niter + 1)
        alpha = np.zeros(max(niter, 1))
        mu = np.zeros(max(niter, 1))
        inn = np.zeros(max(niter * nls, 1)) if inner else None
        st = self._lib.orc_solve(self._h, w, 1 if w0 is None else 0, niter, nls, precond,
                                 _ptr(cost), _ptr(alpha), _ptr(mu), _ptr(inn))
        if st != ORC_OK:
            raise RuntimeError(f"orc_solve failed: {st}")
        out = dict(w=w.reshape(self.shape), cost=cost, alpha=alpha[:niter], mu=mu[:niter])
        if inner:
            out["inner"] = inn[: niter * nls].reshape(niter, nls)
        return out


def wf_gamma(te, amps, freqs):
    """The water-fat basis of Eq. gamma and its projector: gamma = [1, sum_p a_p
    e^{i 2 pi f_p t}] (L x 2; freqs in cycles per unit of te) and
    Gamma = gamma (gamma^H gamma)^{-1} gamma^H.  Returns (gamma, Gamma)."""
    t = np.asarray(te, dtype=np.float64)
    fat = np.exp(2j * np.pi * np.outer(t, np.asarray(freqs, np.float64))) @ np.asarray(amps, np.float64)
    g = np.stack([np.ones_like(fat), fat], axis=1)
    G = g @ np.linalg.inv(g.conj().T @ g) @ g.conj().T
    return g, G


def ic0_factor(shape, mask, d, beta, order=0):
    """Generic IC(0) of H = diag(d) + beta C'C on the mask voxels (order 0: natural; 1:
    red-black, even x + y + z first).

    Returns (colptr, rowidx, val, umap): the factor L in compressed-column form over the
    n unknowns (diagonal first in each column) and the voxel index of each unknown.
    """
    lib = _lib()
    nz, ny, nx = shape
    nv = nx * ny * nz
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    colptr = np.zeros(nv + 1, np.int64)
    rowidx = np.zeros(4 * nv, np.int64)
    val = np.zeros(4 * nv, np.float64)
    umap = np.zeros(nv, np.int64)
    n, nnz = C.c_long(), C.c_long()
    st = lib.orc_ic0_ordered(nx, ny, nz, _ptr(m), d, float(beta), int(order), colptr, rowidx, val, umap,
                             C.byref(n), C.byref(nnz))
    if st != ORC_OK:
        raise RuntimeError(f"orc_ic0 failed: {st}")
    n, nnz = n.value, nnz.value
    return colptr[: n + 1].copy(), rowidx[:nnz].copy(), val[:nnz].copy(), umap[:n].copy()


def ict_factor(shape, mask, d, beta, tau):
    """Generic drop-tolerance IC of H = diag(d) + beta C'C on the mask voxels, natural
    order, absolute tolerance tau (Sec. III-B, L_t).  Same return form as ic0_factor."""
    lib = _lib()
    nz, ny, nx = shape
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    cp, ri, um = C.POINTER(C.c_long)(), C.POINTER(C.c_long)(), C.POINTER(C.c_long)()
    va = C.POINTER(C.c_double)()
    n, nnz = C.c_long(), C.c_long()
    st = lib.orc_ict(nx, ny, nz, _ptr(m), d, float(beta), float(tau), C.byref(cp), C.byref(ri), C.byref(va),
                     C.byref(um), C.byref(n), C.byref(nnz))
    if st != ORC_OK:
        raise RuntimeError(f"orc_ict failed: {st}")
    n, nnz = n.value, nnz.value
    try:
        out = (np.ctypeslib.as_array(cp, shape=(n + 1,)).astype(np.int64).copy(),
               np.ctypeslib.as_array(ri, shape=(max(nnz, 1),))[:nnz].astype(np.int64).copy(),
               np.ctypeslib.as_array(va, shape=(max(nnz, 1),))[:nnz].copy(),
               np.ctypeslib.as_array(um, shape=(max(n, 1),))[:n].astype(np.int64).copy())
    finally:
        for ptr in (cp, ri, va, um):
            lib.orc_free(C.cast(ptr, C.c_void_p))
    return out


def ic0_solve(colptr, rowidx, val, b):
    lib = _lib()
    n = colptr.size - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, np.float64)
    lib.orc_ic0_solve(n, np.ascontiguousarray(colptr), np.ascontiguousarray(rowidx),
                      np.ascontiguousarray(val), b, x)
    return x


def voxel_terms(te, y_vox, s_vox, w):
    """(phi_j, dphi_j, d_j) of one voxel from raw data y_vox [L][N_c], s_vox [N_c] or None."""
    lib = _lib()
    y_vox = np.asarray(y_vox)
    L, nc = y_vox.shape
    out = np.zeros(3, np.float64)
    sv = _c128(s_vox) if s_vox is not None else None
    st = lib.orc_voxel(nc, L, np.ascontiguousarray(te, np.float64), _c128(y_vox).reshape(-1),
                       _ptr(sv), float(w), out)
    if st != ORC_OK:
        raise RuntimeError(f"orc_voxel failed: {st}")
    return out


def curv_raw(y, smap, te, mask, w):
    """Curvature d_j (Eq. 10) at w of every voxel of a volume, from the raw images y
    [L][N_c][z][y][x], coil maps smap [N_c][z][y][x] (or None) and mask, without the
    precomputed r that Oracle keeps (for volumes too large for it)."""
    lib = _lib()
    y = np.asarray(y)
    L, nc, nz, ny, nx = y.shape
    yc = _c128(y).reshape(-1)
    sc = _c128(smap).reshape(-1) if smap is not None else None
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    out = np.zeros(nx * ny * nz, np.float64)
    st = lib.orc_curv_raw(nx, ny, nz, nc, L, yc, _ptr(sc), np.ascontiguousarray(te, np.float64), _ptr(m),
                          np.ascontiguousarray(w, np.float64).reshape(-1), out)
    if st != ORC_OK:
        raise RuntimeError(f"orc_curv_raw failed: {st}")
    return out.reshape(nz, ny, nx)


def voxel_r(y_vox, s_vox):
    """|r| and angle(r) of Eq. 3 for one voxel, shaped [N_c][N_c][L][L] (c, d, m, n)."""
    lib = _lib()
    y_vox = np.asarray(y_vox)
    L, nc = y_vox.shape
    T = nc * nc * L * L
    ra, rg = np.zeros(T), np.zeros(T)
    sv = _c128(s_vox) if s_vox is not None else None
    lib.orc_voxel_r(nc, L, _c128(y_vox).reshape(-1), _ptr(sv), ra, rg)
    return ra.reshape(nc, nc, L, L), rg.reshape(nc, nc, L, L)
