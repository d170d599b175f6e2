"""fm_cost_grad_noalloc: the context-free, allocation-free cost/gradient call.

It serves callers that cannot call cudaMalloc (code running while a CUDA graph is being
captured on the device, real-time pipelines that must not allocate after start-up,
plug-ins whose runtime owns all device buffers).  The test calls it through the C ABI
twice in a row -- the second call must not see the first call's leftover scratch -- and
checks each result against the context entry point fm_cost_grad with the tolerances of
the parity tests, and (FP64) against the oracle.  The file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import copy
import ctypes as C

import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from synth import make_volume

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(cost=1e-11, g=1e-10, d=1e-11), "fp32": dict(cost=2e-6, g=3e-5, d=1e-5)}


def _call_noalloc(lib, vol, prec, y, s, m, w, curvature=0, expect=0):
    import torch
    from paper_2005_08661_gb300 import FmOpts
    o = FmOpts()
    lib.fm_default_opts(C.byref(o))
    o.precision = 1 if prec == "fp32" else 0
    o.curvature = curvature
    dt = torch.float32 if prec == "fp32" else torch.float64
    g = torch.full(vol.mask.shape, float("nan"), dtype=dt, device="cuda")
    d = torch.full(vol.mask.shape, float("nan"), dtype=dt, device="cuda")
    cost = C.c_double(float("nan"))
    te = (C.c_double * vol.necho)(*vol.te)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.fm_cost_grad_noalloc(vol.nx, vol.ny, vol.nz, vol.ncoil, vol.necho, C.byref(o),
                                  C.c_void_p(y.data_ptr()), C.c_void_p(s.data_ptr()) if s is not None else None,
                                  te, C.c_void_p(m.data_ptr()), vol.beta, C.c_void_p(w.data_ptr()),
                                  C.byref(cost), C.c_void_p(g.data_ptr()), C.c_void_p(d.data_ptr()),
                                  torch.cuda.current_device(), C.c_void_p(stream) if stream else None)
    assert st == expect, st
    torch.cuda.synchronize()
    return cost.value, to_np(g), to_np(d)


CASES = [(45, 33, 17, 2, "literal"), (45, 33, 17, 2, "combined"), (70, 37, 19, 1, "literal"),
         (40, 34, 9, 8, "literal"), (40, 34, 9, 8, "combined")]
CURV = {"literal": 0, "combined": 1}


def _volume(case):
    nx, ny, nz, nc, _ = case
    vol = make_volume(nx, ny, nz, ncoil=nc, snr_db=15.0, seed=300 + nx + nc, fmax_hz=150.0, nblobs=3)
    rng = np.random.default_rng(nx)
    vol.mask = (vol.mask & (rng.uniform(size=vol.mask.shape) > 0.08)).astype(np.uint8)
    return vol, rng


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_the_context_entry_point_on_two_calls(prec, case):
    from paper_2005_08661_gb300 import load_library
    lib = load_library()
    curv = case[4]
    vol, rng = _volume(case)
    y, s, m = dev_inputs(vol, prec)
    fm = open_fm(vol, prec, curvature=curv)
    tol = TOL[prec]
    for call in range(2):  # a second call must not depend on the first call's scratch contents
        w_np = (to_np(fm.init_omega()) + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask
        w = to_dev(w_np, prec)
        c_ref, g_ref, d_ref = fm.cost_grad(w)
        g_ref, d_ref = to_np(g_ref), to_np(d_ref)
        c, g, d = _call_noalloc(lib, vol, prec, y, s, m, w, curvature=CURV[curv])
        assert c == pytest.approx(c_ref, rel=tol["cost"]), call
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol["g"] * np.abs(g_ref).max())
        np.testing.assert_allclose(d, d_ref, rtol=tol["d"], atol=tol["d"] * np.abs(d_ref).max())
    fm.close()


@pytest.mark.parametrize("case", CASES)
def test_noalloc_fp64_matches_the_oracle_on_two_calls(case):
    """The call carries its own copy of the set-up and data-term arithmetic, so it is held to
    the FP64 oracle directly as well: cost (Eq. 5), gradient (Eq. 8), curvature (Eq. 10, or
    the coil-combined variant)."""
    from oracle import Oracle
    from paper_2005_08661_gb300 import load_library
    lib = load_library()
    curv = case[4]
    vol, rng = _volume(case)
    orc = Oracle.from_volume(vol)
    orc.set_curvature(curv)
    y, s, m = dev_inputs(vol, "fp64")
    w0 = orc.init()
    for call in range(2):
        w_np = (w0 + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask
        c, g, d = _call_noalloc(lib, vol, "fp64", y, s, m, to_dev(w_np, "fp64"), curvature=CURV[curv])
        c_ref, g_ref, d_ref = orc.cost(w_np), orc.grad(w_np), orc.curv(w_np)
        assert c == pytest.approx(c_ref, rel=1e-11), call
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-10 * np.abs(g_ref).max())
        np.testing.assert_allclose(d, d_ref, rtol=1e-11, atol=1e-11 * np.abs(d_ref).max())


def test_noalloc_reports_a_nonfinite_image_inside_the_mask():
    """A NaN image value inside the mask is FM_ERR_NONFINITE, as for fm_cost_grad; the same
    value outside the mask is ignored."""
    from paper_2005_08661_gb300 import load_library, FM_ERR_NONFINITE
    lib = load_library()
    vol, _ = _volume((40, 34, 9, 2, "literal"))
    inside = tuple(int(v[0]) for v in np.nonzero(vol.mask))
    outside = tuple(int(v[0]) for v in np.nonzero(vol.mask == 0))
    for where, expect in ((outside, 0), (inside, FM_ERR_NONFINITE)):
        vb = copy.copy(vol)
        vb.y = vol.y.copy()
        vb.y[(1, 0) + where] = np.nan
        y, s, m = dev_inputs(vb, "fp32")
        w = to_dev(np.zeros(vol.mask.shape), "fp32")
        c, _, _ = _call_noalloc(lib, vb, "fp32", y, s, m, w, expect=expect)
        assert np.isfinite(c) == (expect == 0)


def test_noalloc_rejects_volumes_beyond_its_fixed_scratch():
    from paper_2005_08661_gb300 import load_library, FM_ERR_SIZE
    lib = load_library()
    te = (C.c_double * 3)(0.0, 2.0, 10.0)
    one = C.c_void_p(1)  # never dereferenced: the size check comes first
    st = lib.fm_cost_grad_noalloc(1024, 1024, 65, 1, 3, None, one, None, te, None, 0.1, one, None, None, None,
                                  0, None)
    assert st == FM_ERR_SIZE
