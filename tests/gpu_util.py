"""Helpers shared by the GPU tests: move a synthetic volume to the device in the
precision under test and open a FieldMap on it."""
import numpy as np


def dev_inputs(vol, precision):
    import torch
    cd = torch.complex64 if precision == "fp32" else torch.complex128
    y = torch.from_numpy(np.ascontiguousarray(vol.y)).to("cuda").to(cd).contiguous()
    s = None
    if vol.smap is not None:
        s = torch.from_numpy(np.ascontiguousarray(vol.smap)).to("cuda").to(cd).contiguous()
    m = torch.from_numpy(np.ascontiguousarray(vol.mask, dtype=np.uint8)).to("cuda")
    return y, s, m


def open_fm(vol, precision="fp32", **kw):
    from paper_2005_08661_gb300 import FieldMap
    fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision=precision, **kw)
    y, s, m = dev_inputs(vol, precision)
    fm.set_data(y, s, vol.te, m, vol.beta)
    return fm


def to_dev(a, precision):
    import torch
    dt = torch.float32 if precision == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dt).contiguous()


def to_np(t):
    return t.detach().double().cpu().numpy()
