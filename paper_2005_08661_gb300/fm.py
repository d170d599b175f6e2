"""Thin ctypes binding of libfm.so (include/fm.h).

Argument marshalling only: every step of the estimator runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  The library must have been
built (``paper_2005_08661_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import functools
import os
import threading

import numpy as np

from . import build as _build

FM_OK, FM_ERR_ARG, FM_ERR_STATE, FM_ERR_CUDA = 0, -1, -2, -3
FM_ERR_NOT_PD, FM_ERR_TIMEOUT, FM_ERR_NONFINITE, FM_ERR_OOM = -4, -5, -6, -7
FM_ERR_SIZE, FM_ERR_FILL = -8, -9
FM_FP64, FM_FP32 = 0, 1
FM_PC_IC0, FM_PC_DIAG, FM_PC_NONE, FM_PC_RB, FM_PC_ICT = 0, 1, 2, 3, 4
FM_CURV_LITERAL, FM_CURV_COMBINED = 0, 1

_PREC = {"fp32": FM_FP32, "fp64": FM_FP64}
_PC = {"ic0": FM_PC_IC0, "diag": FM_PC_DIAG, "none": FM_PC_NONE, "rb": FM_PC_RB, "ict": FM_PC_ICT}
_CURV = {"literal": FM_CURV_LITERAL, "combined": FM_CURV_COMBINED}


class FmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class FmOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("nls", C.c_int), ("precond", C.c_int), ("curvature", C.c_int),
                ("spin_limit", C.c_longlong), ("use_graph", C.c_int), ("droptol", C.c_double)]


_LIB = None
_LOCK = threading.Lock()

EXPORTS = ["fm_default_opts", "fm_create", "fm_set_data", "fm_init_omega", "fm_cost_grad", "fm_ic_factor",
           "fm_ic_apply", "fm_solve", "fm_get_history", "fm_set_profiling", "fm_kernel_times", "fm_destroy",
           "fm_strerror", "fm_last_error", "fm_cost_grad_noalloc", "fm_batch_create", "fm_batch_set_data",
           "fm_batch_solve", "fm_batch_autotune", "fm_batch_set_fraction", "fm_batch_ctx", "fm_batch_destroy",
           "fm_batch_schedule",
           "fm_true_curv", "fm_adjoint_solve", "fm_implicit_grad", "fm_set_fat_model", "fm_wf_sweep",
           "fm_pwls_init", "fm_wf_amplitudes", "fm_wf_sweep_range", "fm_set_spin_limit", "fm_set_data_host",
           "fm_solve_host", "fm_synchronize", "fm_ic_factor64", "fm_ic_factor_curv", "fm_ict_pattern",
           "fm_batch_bwd_blocks"]
KERNELS = ["grad", "ic_fwd", "ic_bwd", "dir", "ls", "h2d", "d2h"]


def lib_path():
    return _build.lib_path()


def load_library(path=None):
    """Load libfm.so and declare its signatures.  Raises if the library is missing."""
    global _LIB
    with _LOCK:
        if _LIB is not None and path is None:
            return _LIB
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build() "
                               "or python -m paper_2005_08661_gb300.build)")
        lib = C.CDLL(p)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        lib.fm_default_opts.argtypes = [C.POINTER(FmOpts)]
        lib.fm_default_opts.restype = None
        lib.fm_create.argtypes = [C.POINTER(vp), i, i, i, i, i, C.POINTER(FmOpts), i, vp]
        lib.fm_set_data.argtypes = [vp, vp, vp, C.POINTER(d), vp, d]
        lib.fm_init_omega.argtypes = [vp, vp]
        lib.fm_cost_grad.argtypes = [vp, vp, C.POINTER(d), vp, vp]
        lib.fm_ic_factor.argtypes = [vp, vp, vp]
        lib.fm_ic_apply.argtypes = [vp, vp, vp]
        lib.fm_solve.argtypes = [vp, vp, i, i, C.POINTER(d)]
        lib.fm_get_history.argtypes = [vp, C.POINTER(d), C.POINTER(d), i]
        lib.fm_set_profiling.argtypes = [vp, i]
        lib.fm_kernel_times.argtypes = [vp, C.POINTER(d), C.POINTER(i)]
        lib.fm_destroy.argtypes = [vp]
        for fn in ("fm_create", "fm_set_data", "fm_init_omega", "fm_cost_grad", "fm_ic_factor", "fm_ic_apply",
                   "fm_solve", "fm_get_history", "fm_set_profiling", "fm_kernel_times", "fm_destroy"):
            getattr(lib, fn).restype = C.c_int
        lib.fm_cost_grad_noalloc.argtypes = [i, i, i, i, i, C.POINTER(FmOpts), vp, vp, C.POINTER(d), vp, d, vp,
                                             C.POINTER(d), vp, vp, i, vp]
        lib.fm_cost_grad_noalloc.restype = C.c_int
        lib.fm_true_curv.argtypes = [vp, vp, vp]
        lib.fm_adjoint_solve.argtypes = [vp, vp, vp, vp, d, i, C.POINTER(i), C.POINTER(d)]
        lib.fm_implicit_grad.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(d)]
        lib.fm_set_fat_model.argtypes = [vp, i, C.POINTER(d), C.POINTER(d)]
        lib.fm_wf_sweep.argtypes = [vp, i, d, d, vp]
        lib.fm_pwls_init.argtypes = [vp, vp, i, vp]
        lib.fm_wf_amplitudes.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.fm_ic_factor64.argtypes = [vp, vp, vp]
        lib.fm_ic_factor64.restype = C.c_int
        lib.fm_ic_factor_curv.argtypes = [vp, vp, vp]
        lib.fm_ic_factor_curv.restype = C.c_int
        lib.fm_ict_pattern.argtypes = [vp, C.POINTER(i), vp, vp]
        lib.fm_ict_pattern.restype = C.c_int
        lib.fm_set_data_host.argtypes = [vp, vp, vp, C.POINTER(d), vp, d]
        lib.fm_solve_host.argtypes = [vp, vp, i, i, C.POINTER(d)]
        lib.fm_synchronize.argtypes = [vp]
        for fn in ("fm_set_data_host", "fm_solve_host", "fm_synchronize"):
            getattr(lib, fn).restype = C.c_int
        lib.fm_wf_sweep_range.argtypes = [vp, C.POINTER(d), C.POINTER(d)]
        lib.fm_set_spin_limit.argtypes = [vp, C.c_longlong]
        for fn in ("fm_true_curv", "fm_adjoint_solve", "fm_implicit_grad", "fm_set_fat_model", "fm_wf_sweep",
                   "fm_pwls_init", "fm_wf_amplitudes", "fm_wf_sweep_range", "fm_set_spin_limit"):
            getattr(lib, fn).restype = C.c_int
        lib.fm_batch_create.argtypes = [C.POINTER(vp), i, C.POINTER(i), C.POINTER(FmOpts), i, vp]
        lib.fm_batch_set_data.argtypes = [vp, i, vp, vp, C.POINTER(d), vp, d]
        lib.fm_batch_solve.argtypes = [vp, C.POINTER(vp), i, i, C.POINTER(C.POINTER(d))]
        lib.fm_batch_autotune.argtypes = [vp, i, C.POINTER(d), C.POINTER(d)]
        lib.fm_batch_set_fraction.argtypes = [vp, d]
        lib.fm_batch_schedule.argtypes = [vp, C.POINTER(d), C.POINTER(i), C.POINTER(i)]
        lib.fm_batch_bwd_blocks.argtypes = [vp, C.POINTER(i)]
        lib.fm_batch_bwd_blocks.restype = C.c_int
        lib.fm_batch_ctx.argtypes = [vp, i]
        lib.fm_batch_ctx.restype = vp
        lib.fm_batch_destroy.argtypes = [vp]
        for fn in ("fm_batch_create", "fm_batch_set_data", "fm_batch_solve", "fm_batch_autotune",
                   "fm_batch_set_fraction", "fm_batch_destroy", "fm_batch_schedule"):
            getattr(lib, fn).restype = C.c_int
        lib.fm_strerror.argtypes = [i]
        lib.fm_strerror.restype = C.c_char_p
        lib.fm_last_error.argtypes = [vp]
        lib.fm_last_error.restype = C.c_char_p
        if path is None:
            _LIB = lib
        return lib


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _ordered(fn):
    """Orders a call that runs on the handle's stream with torch's current stream: the
    handle's stream first waits for the work already queued on the current stream (which
    made the input tensors), and the current stream then waits for the call's kernels, so
    a returned tensor may be used (or freed) on the current stream at once.  Nothing is
    added when the two streams are the same."""
    @functools.wraps(fn)
    def wrapper(self, *args, **kwargs):
        cur = self._torch.cuda.current_stream(self.device)
        same = cur == self.stream
        if not same:
            self.stream.wait_stream(cur)
        try:
            return fn(self, *args, **kwargs)
        finally:
            if not same:
                cur.wait_stream(self.stream)
    return wrapper


class FieldMap:
    """One volume's field-map estimator on one GPU (a handle on an fm_ctx)."""

    def __init__(self, nx, ny, nz, ncoil=1, necho=3, precision="fp32", nls=5, precond="ic0",
                 curvature="literal", spin_limit=1 << 21, use_graph=True, device=None, stream=None, droptol=1e-3):
        """precond: "ic0" (the paper's IC(0)), "ict" (IC with the drop tolerance droptol * H_max,
        Sec. III-B's L_t), "rb" (red-black IC(0)), "diag" or "none"."""
        import torch
        self._torch = torch
        self.lib = load_library()
        self.shape = (nz, ny, nx)
        self.ncoil, self.necho = ncoil, necho
        self.precision = precision
        self.rdtype = torch.float32 if precision == "fp32" else torch.float64
        self.cdtype = torch.complex64 if precision == "fp32" else torch.complex128
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        o = FmOpts()
        self.lib.fm_default_opts(C.byref(o))
        o.precision = _PREC[precision]
        o.nls = int(nls)
        o.precond = _PC[precond]
        o.curvature = _CURV[curvature]
        o.spin_limit = int(spin_limit)
        o.use_graph = 1 if use_graph else 0
        o.droptol = float(droptol)
        self.opts = o
        h = C.c_void_p()
        sp = stream.cuda_stream if stream is not None else 0
        st = self.lib.fm_create(C.byref(h), nx, ny, nz, ncoil, necho, C.byref(o), dev.index,
                                C.c_void_p(sp) if sp else None)
        if st != FM_OK:
            raise FmError(st, f"fm_create: {self.lib.fm_strerror(st).decode()}")
        self._h = h
        self.fat_model = None
        self.data = None

    # ---------------------------------------------------------------- helpers
    def _check(self, st, what):
        if st != FM_OK:
            msg = self.lib.fm_last_error(self._h).decode() if self._h else ""
            raise FmError(st, f"{what}: {self.lib.fm_strerror(st).decode()}: {msg}")

    def _vec(self, x, name):
        t = self._torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.rdtype and x.is_contiguous()
                and x.numel() == int(np.prod(self.shape))):
            raise TypeError(f"{name} must be a contiguous {self.rdtype} CUDA tensor with {int(np.prod(self.shape))} "
                            "elements")
        return x

    def empty(self):
        return self._torch.empty(self.shape, dtype=self.rdtype, device=self.device)

    # ---------------------------------------------------------------- API
    @_ordered
    def set_data(self, y, smap, te, mask=None, beta=2.0 ** -3):
        t = self._torch
        nz, ny, nx = self.shape
        if not (y.is_cuda and y.dtype == self.cdtype and y.is_contiguous()
                and tuple(y.shape) == (self.necho, self.ncoil, nz, ny, nx)):
            raise TypeError(f"y must be a contiguous {self.cdtype} CUDA tensor of shape "
                            f"{(self.necho, self.ncoil, nz, ny, nx)}")
        if smap is not None and not (smap.is_cuda and smap.dtype == self.cdtype and smap.is_contiguous()
                                     and tuple(smap.shape) == (self.ncoil, nz, ny, nx)):
            raise TypeError("smap must match y's dtype with shape (ncoil, nz, ny, nx)")
        if mask is not None and not (mask.is_cuda and mask.dtype == t.uint8 and mask.is_contiguous()
                                     and tuple(mask.shape) == self.shape):
            raise TypeError("mask must be a contiguous uint8 CUDA tensor of the volume's shape")
        te_arr = (C.c_double * self.necho)(*[float(v) for v in te])
        self._check(self.lib.fm_set_data(self._h, _dptr(y), _dptr(smap), te_arr, _dptr(mask), float(beta)),
                    "fm_set_data")
        self.data = (y, smap, tuple(float(v) for v in te), mask, float(beta))

    def set_data_host(self, y, smap, te, mask=None, beta=2.0 ** -3):
        """fm_set_data_host: y, smap and mask are CPU tensors (page-locked for an upload that
        overlaps earlier work); they must stay unchanged until the next synchronize()."""
        t = self._torch
        nz, ny, nx = self.shape
        if not (not y.is_cuda and y.dtype == self.cdtype and y.is_contiguous()
                and tuple(y.shape) == (self.necho, self.ncoil, nz, ny, nx)):
            raise TypeError(f"y must be a contiguous {self.cdtype} CPU tensor of shape "
                            f"{(self.necho, self.ncoil, nz, ny, nx)}")
        if smap is not None and not (not smap.is_cuda and smap.dtype == self.cdtype and smap.is_contiguous()
                                     and tuple(smap.shape) == (self.ncoil, nz, ny, nx)):
            raise TypeError("smap must be a contiguous CPU tensor of y's dtype with shape (ncoil, nz, ny, nx)")
        if mask is not None and not (not mask.is_cuda and mask.dtype == t.uint8 and mask.is_contiguous()
                                     and tuple(mask.shape) == self.shape):
            raise TypeError("mask must be a contiguous uint8 CPU tensor of the volume's shape")
        te_arr = (C.c_double * self.necho)(*[float(v) for v in te])
        self._check(self.lib.fm_set_data_host(self._h, _dptr(y), _dptr(smap), te_arr, _dptr(mask), float(beta)),
                    "fm_set_data_host")
        self.data = None  # the device arrays of fm_set_data are not kept for host input

    def solve_host(self, omega, init=True, niter=50, hist=None):
        """fm_solve_host into the CPU tensor omega (read as the start when init is False);
        hist: a ctypes double array of niter + 1 entries or None (then asynchronous)."""
        if not (not omega.is_cuda and omega.dtype == self.rdtype and omega.is_contiguous()
                and omega.numel() == int(np.prod(self.shape))):
            raise TypeError(f"omega must be a contiguous {self.rdtype} CPU tensor of the volume's size")
        self._check(self.lib.fm_solve_host(self._h, _dptr(omega), 0 if not init else 1, int(niter), hist),
                    "fm_solve_host")
        return omega

    def synchronize(self):
        self._check(self.lib.fm_synchronize(self._h), "fm_synchronize")

    @_ordered
    def init_omega(self):
        out = self.empty()
        self._check(self.lib.fm_init_omega(self._h, _dptr(out)), "fm_init_omega")
        return out

    @_ordered
    def cost_grad(self, omega, want_cost=True, want_grad=True, want_curv=True):
        self._vec(omega, "omega")
        g = self.empty() if want_grad else None
        d = self.empty() if want_curv else None
        cost = C.c_double(0.0)
        self._check(self.lib.fm_cost_grad(self._h, _dptr(omega), C.byref(cost) if want_cost else None,
                                          _dptr(g), _dptr(d)), "fm_cost_grad")
        return (cost.value if want_cost else None), g, d

    @_ordered
    def ic_factor(self, omega, want_pivots=True):
        self._vec(omega, "omega")
        ip = self.empty() if want_pivots else None
        self._check(self.lib.fm_ic_factor(self._h, _dptr(omega), _dptr(ip)), "fm_ic_factor")
        return ip

    @_ordered
    def ic_factor_curv(self, curv, want_pivots=True):
        """fm_ic_factor_curv: the preconditioner factor of diag(curv) + beta C'C."""
        self._vec(curv, "curv")
        ip = self.empty() if want_pivots else None
        self._check(self.lib.fm_ic_factor_curv(self._h, _dptr(curv), _dptr(ip)), "fm_ic_factor_curv")
        return ip

    def ict_pattern(self, planes=True):
        """The drop-tolerance factor as held: (offsets [nh][3] of (dx, dy, dz), planes
        [nh + 1][nz][ny][nx] float64 (1/L_ii, then L_{i,i+o} per offset) or None)."""
        n = C.c_int(0)
        self._check(self.lib.fm_ict_pattern(self._h, C.byref(n), None, None), "fm_ict_pattern")
        off = np.zeros((n.value, 3), np.int32)
        pl = np.zeros((n.value + 1,) + self.shape, np.float64) if planes else None
        self._check(self.lib.fm_ict_pattern(self._h, C.byref(n), off.ctypes.data_as(C.c_void_p),
                                            pl.ctypes.data_as(C.c_void_p) if pl is not None else None),
                    "fm_ict_pattern")
        return off, pl

    @_ordered
    def ic_factor64(self, omega):
        """fm_ic_factor64: IC(0) factor at omega; returns the inverse pivots as a float64 tensor
        (FP32 mode: the hi + lo pair the forward sweep carries)."""
        self._vec(omega, "omega")
        ip = self._torch.empty(self.shape, dtype=self._torch.float64, device=self.device)
        self._check(self.lib.fm_ic_factor64(self._h, _dptr(omega), _dptr(ip)), "fm_ic_factor64")
        return ip

    @_ordered
    def ic_apply(self, g, out=None):
        self._vec(g, "g")
        p = self.empty() if out is None else self._vec(out, "out")
        self._check(self.lib.fm_ic_apply(self._h, _dptr(g), _dptr(p)), "fm_ic_apply")
        return p

    # ---------------------------------------------------------------- water-fat model
    def set_fat_model(self, amps, freqs):
        """Water-fat model for the next set_data: relative peak amplitudes and frequency
        offsets in cycles per unit of the echo times (kHz for ms).  Empty -> field map."""
        amps = [float(v) for v in amps]
        freqs = [float(v) for v in freqs]
        if len(amps) != len(freqs):
            raise ValueError("amps and freqs must have the same length")
        n = len(amps)
        a = (C.c_double * max(n, 1))(*amps)
        f = (C.c_double * max(n, 1))(*freqs)
        self._check(self.lib.fm_set_fat_model(self._h, n, a, f), "fm_set_fat_model")
        self.fat_model = (tuple(amps), tuple(freqs)) if n else None

    def wf_sweep_range(self):
        """The library's default sweep range (fm_wf_sweep_range) for the current fat model."""
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.fm_wf_sweep_range(self._h, C.byref(lo), C.byref(hi)), "fm_wf_sweep_range")
        return lo.value, hi.value

    @_ordered
    def wf_sweep(self, nsweep=100, w_lo=None, w_hi=None, out=None):
        """Voxel-wise sweep initialisation; the default range is the library's
        (fm_wf_sweep_range)."""
        if w_lo is None or w_hi is None:
            w_lo, w_hi = self.wf_sweep_range()
        out = self.empty() if out is None else self._vec(out, "out")
        self._check(self.lib.fm_wf_sweep(self._h, int(nsweep), float(w_lo), float(w_hi), _dptr(out)), "fm_wf_sweep")
        return out

    @_ordered
    def pwls_init(self, omega_tilde, niter=10, out=None):
        """PWLS initialisation (niter CG iterations) from the sweep's map."""
        self._vec(omega_tilde, "omega_tilde")
        out = self.empty() if out is None else self._vec(out, "out")
        self._check(self.lib.fm_pwls_init(self._h, _dptr(omega_tilde), int(niter), _dptr(out)), "fm_pwls_init")
        return out

    def wf_init(self, nsweep=100, niter=10):
        """Sweep then PWLS: the water-fat initial map."""
        return self.pwls_init(self.wf_sweep(nsweep), niter)

    @_ordered
    def wf_amplitudes(self, omega, y=None, smap=None, out=None):
        """(water, fat) complex maps at omega by the closed form of the water-fat model."""
        self._vec(omega, "omega")
        if y is None:
            y, smap = self.data[0], self.data[1]
        if out is None:
            w = self._torch.empty(self.shape, dtype=self.cdtype, device=self.device)
            f = self._torch.empty(self.shape, dtype=self.cdtype, device=self.device)
        else:
            w, f = out
            for t in out:
                if not (t.is_cuda and t.dtype == self.cdtype and t.is_contiguous() and tuple(t.shape) == self.shape):
                    raise TypeError(f"out tensors must be contiguous {self.cdtype} CUDA tensors of shape {self.shape}")
        self._check(self.lib.fm_wf_amplitudes(self._h, _dptr(y), _dptr(smap), _dptr(omega), _dptr(w), _dptr(f)),
                    "fm_wf_amplitudes")
        return w, f

    @_ordered
    def true_curv(self, omega):
        """Exact second derivative of the data term at omega (0 outside the mask)."""
        self._vec(omega, "omega")
        h = self.empty()
        self._check(self.lib.fm_true_curv(self._h, _dptr(omega), _dptr(h)), "fm_true_curv")
        return h

    @_ordered
    def adjoint_solve(self, omega_hat, rhs, tol=None, maxiter=1000):
        """lambda = H_true^{-1} rhs by IC(0)-preconditioned CG.  Returns (lambda, iterations,
        relative residual).  tol defaults to 1e-6 (fp32) or 1e-12 (fp64)."""
        self._vec(omega_hat, "omega_hat")
        self._vec(rhs, "rhs")
        if tol is None:
            tol = 1e-6 if self.precision == "fp32" else 1e-12
        lam = self.empty()
        it, rr = C.c_int(0), C.c_double(0.0)
        self._check(self.lib.fm_adjoint_solve(self._h, _dptr(omega_hat), _dptr(rhs), _dptr(lam), float(tol),
                                              int(maxiter), C.byref(it), C.byref(rr)), "fm_adjoint_solve")
        return lam, it.value, rr.value

    @_ordered
    def implicit_grad(self, omega_hat, lam, y=None, smap=None, want_dy=True, want_dbeta=True):
        """(dl/dy, dl/dbeta) of a loss whose adjoint is lam; y and smap default to the
        arrays of the last set_data."""
        self._vec(omega_hat, "omega_hat")
        self._vec(lam, "lam")
        if y is None:
            y, smap = self.data[0], self.data[1]
        dy = self._torch.empty(tuple(y.shape), dtype=self.cdtype, device=self.device) if want_dy else None
        db = C.c_double(0.0)
        self._check(self.lib.fm_implicit_grad(self._h, _dptr(y), _dptr(smap), _dptr(omega_hat), _dptr(lam),
                                              _dptr(dy), C.byref(db) if want_dbeta else None), "fm_implicit_grad")
        return dy, (db.value if want_dbeta else None)

    @_ordered
    def solve(self, omega=None, niter=50, want_history=True):
        """Run niter NCG-MLS iterations; omega=None starts from Eq. 6.  Returns (omega, costs)."""
        init = omega is None
        w = self.empty() if init else self._vec(omega, "omega").clone()
        hist = (C.c_double * (niter + 1))() if want_history else None
        self._check(self.lib.fm_solve(self._h, _dptr(w), 1 if init else 0, int(niter), hist), "fm_solve")
        return w, (np.array(hist[:], dtype=np.float64) if want_history else None)

    def solve_into(self, omega, init, niter, hist=None):
        """Lowest-overhead form: omega is updated in place; hist is a ctypes double array or None."""
        self._check(self.lib.fm_solve(self._h, _dptr(omega), 1 if init else 0, int(niter), hist), "fm_solve")
        return omega

    def history(self, n):
        a = (C.c_double * max(n, 1))()
        m = (C.c_double * max(n, 1))()
        self._check(self.lib.fm_get_history(self._h, a, m, int(n)), "fm_get_history")
        return np.array(a[:n]), np.array(m[:n])

    def set_spin_limit(self, n):
        """Bound on device-side waits (polls) for the following calls."""
        self._check(self.lib.fm_set_spin_limit(self._h, int(n)), "fm_set_spin_limit")

    def set_profiling(self, on=True):
        self._check(self.lib.fm_set_profiling(self._h, 1 if on else 0), "fm_set_profiling")

    def kernel_times(self):
        """{kernel: (average ms, launches averaged)} of the last profiled iterations."""
        ms = (C.c_double * len(KERNELS))()
        cnt = (C.c_int * len(KERNELS))()
        self._check(self.lib.fm_kernel_times(self._h, ms, cnt), "fm_kernel_times")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNELS)}

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FieldMapBatch:
    """Many independent volumes solved together (fm_batch_*): one CUDA graph launch
    advances every volume's outer iteration."""

    def __init__(self, shapes, precision="fp32", nls=5, precond="ic0", curvature="literal", spin_limit=1 << 21,
                 device=None, stream=None, droptol=1e-3):
        """shapes: list of (nx, ny, nz, ncoil, necho)."""
        import torch
        self._torch = torch
        self.lib = load_library()
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.precision = precision
        self.rdtype = torch.float32 if precision == "fp32" else torch.float64
        self.cdtype = torch.complex64 if precision == "fp32" else torch.complex128
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        o = FmOpts()
        self.lib.fm_default_opts(C.byref(o))
        o.precision = _PREC[precision]
        o.nls = int(nls)
        o.precond = _PC[precond]
        o.curvature = _CURV[curvature]
        o.spin_limit = int(spin_limit)
        o.droptol = float(droptol)
        dims = (C.c_int * (5 * len(shapes)))(*[v for sh in self.shapes for v in sh])
        h = C.c_void_p()
        sp = stream.cuda_stream if stream is not None else 0
        st = self.lib.fm_batch_create(C.byref(h), len(shapes), dims, C.byref(o), dev.index,
                                      C.c_void_p(sp) if sp else None)
        if st != FM_OK:
            raise FmError(st, f"fm_batch_create: {self.lib.fm_strerror(st).decode()}")
        self._h = h

    def _check(self, st, what):
        if st != FM_OK:
            raise FmError(st, f"{what}: {self.lib.fm_strerror(st).decode()}")

    @_ordered
    def set_data(self, k, y, smap, te, mask=None, beta=2.0 ** -3):
        nx, ny, nz, nc, L = self.shapes[k]
        if not (y.is_cuda and y.dtype == self.cdtype and y.is_contiguous() and tuple(y.shape) == (L, nc, nz, ny, nx)):
            raise TypeError(f"y[{k}] must be a contiguous {self.cdtype} CUDA tensor of shape {(L, nc, nz, ny, nx)}")
        te_arr = (C.c_double * L)(*[float(v) for v in te])
        self._check(self.lib.fm_batch_set_data(self._h, k, _dptr(y), _dptr(smap), te_arr, _dptr(mask), float(beta)),
                    "fm_batch_set_data")

    def empty(self, k):
        nx, ny, nz, _, _ = self.shapes[k]
        return self._torch.empty((nz, ny, nx), dtype=self.rdtype, device=self.device)

    @_ordered
    def solve(self, omegas=None, niter=50, want_history=True):
        """Returns (list of field maps, list of cost histories or None)."""
        n = len(self.shapes)
        init = omegas is None
        ws = [self.empty(k) for k in range(n)] if init else [w.clone() for w in omegas]
        ptrs = (C.c_void_p * n)(*[w.data_ptr() for w in ws])
        hists = [(C.c_double * (niter + 1))() for _ in range(n)] if want_history else None
        hp = (C.POINTER(C.c_double) * n)(*[C.cast(hh, C.POINTER(C.c_double)) for hh in hists]) if hists else None
        self._check(self.lib.fm_batch_solve(self._h, ptrs, 1 if init else 0, int(niter), hp), "fm_batch_solve")
        return ws, ([np.array(hh[:]) for hh in hists] if hists else None)

    def solve_into(self, ptrs, init, niter):
        """Lowest-overhead form: ptrs is a ctypes array of device pointers updated in place."""
        self._check(self.lib.fm_batch_solve(self._h, ptrs, 1 if init else 0, int(niter), None), "fm_batch_solve")

    def autotune(self, niter_probe=4):
        f, ms = C.c_double(), C.c_double()
        self._check(self.lib.fm_batch_autotune(self._h, int(niter_probe), C.byref(f), C.byref(ms)), "fm_batch_autotune")
        return f.value, ms.value

    def set_fraction(self, f):
        self._check(self.lib.fm_batch_set_fraction(self._h, float(f)), "fm_batch_set_fraction")

    def schedule(self):
        """(grid fraction, (X + Y weight, Z weight) of the forward tile order) in effect."""
        f, wxy, wz = C.c_double(), C.c_int(), C.c_int()
        self._check(self.lib.fm_batch_schedule(self._h, C.byref(f), C.byref(wxy), C.byref(wz)), "fm_batch_schedule")
        return f.value, (wxy.value, wz.value)

    def bwd_blocks_per_sm(self):
        """Back-substitution blocks per SM in effect (chosen by autotune)."""
        n = C.c_int()
        self._check(self.lib.fm_batch_bwd_blocks(self._h, C.byref(n)), "fm_batch_bwd_blocks")
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
