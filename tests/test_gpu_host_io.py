"""The host-buffer form of the boundary (fm_set_data_host, fm_solve_host, fm_synchronize):
images, coil maps and mask in host memory, field map back in host memory.  It must give
exactly what the device-pointer calls give on the same inputs, with the uploads of several
acquisitions queued behind one another on the library's copy stream, and report device
errors of its asynchronous solve at the next synchronisation."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import dev_inputs, open_fm, to_np
from oracle import Oracle
from synth import make_volume

pytestmark = pytest.mark.gpu


def _host(vol, prec, pinned):
    import torch
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    y = torch.from_numpy(np.ascontiguousarray(vol.y)).to(cd).contiguous()
    s = torch.from_numpy(np.ascontiguousarray(vol.smap)).to(cd).contiguous() if vol.smap is not None else None
    m = torch.from_numpy(np.ascontiguousarray(vol.mask, dtype=np.uint8)).contiguous()
    if pinned:
        y, m = y.pin_memory(), m.pin_memory()
        s = s.pin_memory() if s is not None else None
    return y, s, m


@pytest.mark.parametrize("prec,pinned", [("fp64", True), ("fp32", True), ("fp32", False)])
def test_host_buffers_give_the_device_path_results(prec, pinned):
    import torch
    from paper_2005_08661_gb300 import FieldMap
    vols = [make_volume(45, 33, 17, ncoil=c, snr_db=15.0, seed=60 + c, fmax_hz=150.0, nblobs=3) for c in (2, 2, 2)]
    fm_dev = open_fm(vols[0], prec)
    ref = []
    for v in vols:
        y, s, m = dev_inputs(v, prec)
        fm_dev.set_data(y, s, v.te, m, v.beta)
        w, cost = fm_dev.solve(niter=6)
        ref.append((to_np(w), cost))
    fm_dev.close()
    v0 = vols[0]
    fm = FieldMap(v0.nx, v0.ny, v0.nz, ncoil=2, necho=3, precision=prec)
    rd = torch.float32 if prec == "fp32" else torch.float64
    outs = [torch.zeros(v0.mask.shape, dtype=rd) for _ in vols]
    if pinned:
        outs = [o.pin_memory() for o in outs]
    hosts = [_host(v, prec, pinned) for v in vols]
    for (y, s, m), v, o in zip(hosts, vols, outs):  # three acquisitions queued without a host wait
        fm.set_data_host(y, s, v.te, m, v.beta)
        fm.solve_host(o, init=True, niter=6)
    fm.synchronize()
    for o, (w_ref, _) in zip(outs, ref):
        assert np.array_equal(o.double().numpy(), w_ref)
    # with a cost history the call synchronises and returns the same history
    hist = (C.c_double * 7)()
    fm.set_data_host(*hosts[1][:2], vols[1].te, hosts[1][2], vols[1].beta)
    fm.solve_host(outs[0], init=True, niter=6, hist=hist)
    assert np.array_equal(np.array(hist[:]), ref[1][1])
    assert np.array_equal(outs[0].double().numpy(), ref[1][0])
    fm.close()


def test_host_solve_from_a_host_start_matches_the_oracle():
    """init = False reads the start map from host memory (FP64, per-iteration cost 1e-10)."""
    import torch
    from paper_2005_08661_gb300 import FieldMap
    vol = make_volume(30, 28, 9, ncoil=3, snr_db=15.0, seed=64, fmax_hz=120.0, nblobs=3)
    o = Oracle.from_volume(vol)
    rng = np.random.default_rng(2)
    w0 = (vol.omega_true + 0.05 * rng.standard_normal(vol.mask.shape)) * vol.mask
    ref = o.solve(w0=w0, niter=5, nls=5)
    fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=3, necho=3, precision="fp64")
    y, s, m = _host(vol, "fp64", True)
    fm.set_data_host(y, s, vol.te, m, vol.beta)
    w = torch.from_numpy(w0.copy()).contiguous()
    hist = (C.c_double * 6)()
    fm.solve_host(w, init=False, niter=5, hist=hist)
    np.testing.assert_allclose(np.array(hist[:]), ref["cost"], rtol=1e-10)
    np.testing.assert_allclose(w.numpy(), ref["w"], rtol=0, atol=1e-9)
    fm.close()


def test_asynchronous_solve_reports_its_error_at_the_next_synchronisation():
    """A solve without a cost history returns once enqueued; a non-positive pivot it meets is
    reported by fm_synchronize."""
    import torch
    from paper_2005_08661_gb300 import FieldMap, FmError, FM_ERR_NOT_PD
    vol = make_volume(20, 20, 9, ncoil=1, snr_db=20.0, seed=65, fmax_hz=100.0, nblobs=2)
    vol.y[:] = 0
    fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=1, necho=3, precision="fp32")
    y, s, m = _host(vol, "fp32", True)
    fm.set_data_host(y, s, vol.te, m, 0.0)
    w = torch.zeros(vol.mask.shape, dtype=torch.float32).pin_memory()
    fm.solve_host(w, init=True, niter=2)
    with pytest.raises(FmError) as e:
        fm.synchronize()
    assert e.value.status == FM_ERR_NOT_PD
    fm.synchronize()  # the error was reported once and cleared
    fm.close()


@pytest.mark.parametrize("precond", ["ic0", "none"])
def test_handle_on_a_side_stream_is_ordered_with_the_current_stream(precond):
    """A FieldMap created on a stream other than torch's current one: the tensors its calls
    return must be complete when read on the current stream right after the call, although
    fm_solve returns without waiting when no cost history is asked for."""
    import torch
    from synth import full8_small_config
    vol = full8_small_config()
    fm_cur = open_fm(vol, "fp32", precond=precond)
    w_ref, _ = fm_cur.solve(niter=40, want_history=False)
    w_ref = w_ref.clone()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    fm_side = open_fm(vol, "fp32", precond=precond, stream=side)
    for niter in (40, 1, 40):
        w, _ = fm_side.solve(niter=niter, want_history=False)
        got = w.clone()  # on the current stream, with no explicit synchronisation
        if niter == 40:
            assert torch.equal(got, w_ref)
        else:
            assert not torch.equal(got, w_ref)
    _, g, _ = fm_side.cost_grad(w_ref)
    _, g_ref, _ = fm_cur.cost_grad(w_ref)
    assert torch.equal(g.clone(), g_ref)
    fm_side.close()
    fm_cur.close()
