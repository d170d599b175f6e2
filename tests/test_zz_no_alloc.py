"""fm_cost_grad_noalloc: the context-free, allocation-free cost/gradient call.

It serves callers that cannot call cudaMalloc (code running while a CUDA graph is being
captured on the device, real-time pipelines that must not allocate after start-up,
plug-ins whose runtime owns all device buffers).  The test calls it through the C ABI
twice in a row -- the second call must not see the first call's leftover scratch -- and
checks each result against the context entry point fm_cost_grad with the tolerances of
the parity tests.  The file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_dev, to_np
from synth import make_volume

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(cost=1e-11, g=1e-10, d=1e-11), "fp32": dict(cost=2e-6, g=3e-5, d=1e-5)}


def _call_noalloc(lib, vol, prec, y, s, m, w, curvature=0):
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
    assert st == 0, st
    torch.cuda.synchronize()
    return cost.value, to_np(g), to_np(d)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", [(45, 33, 17, 2), (70, 37, 19, 1), (40, 34, 9, 8)])
def test_noalloc_matches_the_context_entry_point_on_two_calls(prec, case):
    from paper_2005_08661_gb300 import load_library
    lib = load_library()
    nx, ny, nz, nc = case
    vol = make_volume(nx, ny, nz, ncoil=nc, snr_db=15.0, seed=300 + nx + nc, fmax_hz=150.0, nblobs=3)
    rng = np.random.default_rng(nx)
    vol.mask = (vol.mask & (rng.uniform(size=vol.mask.shape) > 0.08)).astype(np.uint8)
    y, s, m = dev_inputs(vol, prec)
    fm = open_fm(vol, prec)
    tol = TOL[prec]
    for call in range(2):  # a second call must not depend on the first call's scratch contents
        w_np = (to_np(fm.init_omega()) + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask
        w = to_dev(w_np, prec)
        c_ref, g_ref, d_ref = fm.cost_grad(w)
        g_ref, d_ref = to_np(g_ref), to_np(d_ref)
        c, g, d = _call_noalloc(lib, vol, prec, y, s, m, w)
        assert c == pytest.approx(c_ref, rel=tol["cost"]), call
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol["g"] * np.abs(g_ref).max())
        np.testing.assert_allclose(d, d_ref, rtol=tol["d"], atol=tol["d"] * np.abs(d_ref).max())
    fm.close()


def test_noalloc_rejects_volumes_beyond_its_fixed_scratch():
    from paper_2005_08661_gb300 import load_library, FM_ERR_SIZE
    lib = load_library()
    te = (C.c_double * 3)(0.0, 2.0, 10.0)
    one = C.c_void_p(1)  # never dereferenced: the size check comes first
    st = lib.fm_cost_grad_noalloc(1024, 1024, 65, 1, 3, None, one, None, te, None, 0.1, one, None, None, None,
                                  0, None)
    assert st == FM_ERR_SIZE
