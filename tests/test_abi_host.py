"""Host-side checks of the C ABI: the library builds, loads and exports every symbol that
include/fm.h declares, and argument validation happens before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_08661_gb300 import build as b
    b.build()
    from paper_2005_08661_gb300 import load_library
    return load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fm_create", "fm_set_data", "fm_ic_factor", "fm_ic_apply", "fm_cost_grad", "fm_solve",
              "fm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_2005_08661_gb300 import EXPORTS
    assert sorted(EXPORTS) == _declared()


def test_library_exports_nothing_else():
    from paper_2005_08661_gb300 import build as b
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", b.build()], capture_output=True, text=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    fm_syms = {s for s in syms if s.startswith("fm_")}
    assert fm_syms == set(_declared())


def test_argument_errors_need_no_device(lib):
    from paper_2005_08661_gb300 import FmOpts, FM_ERR_ARG, FM_OK
    h = C.c_void_p()
    assert lib.fm_create(None, 4, 4, 4, 1, 3, None, 0, None) == FM_ERR_ARG
    assert lib.fm_create(C.byref(h), 0, 4, 4, 1, 3, None, 0, None) == FM_ERR_ARG
    assert lib.fm_create(C.byref(h), 4, 4, 4, 0, 3, None, 0, None) == FM_ERR_ARG
    assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 1, None, 0, None) == FM_ERR_ARG   # L >= 2 (Sec. II)
    assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 9, None, 0, None) == FM_ERR_ARG
    assert lib.fm_create(C.byref(h), 4, 4, 4, 33, 3, None, 0, None) == FM_ERR_ARG
    o = FmOpts()
    lib.fm_default_opts(C.byref(o))
    assert (o.precision, o.nls, o.precond, o.curvature, o.use_graph) == (1, 5, 0, 0, 1)
    assert o.spin_limit == 1 << 21
    bad = FmOpts()
    lib.fm_default_opts(C.byref(bad))
    bad.nls = 0
    assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 3, C.byref(bad), 0, None) == FM_ERR_ARG
    bad.nls, bad.precision = 5, 7
    assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 3, C.byref(bad), 0, None) == FM_ERR_ARG
    assert h.value is None
    assert lib.fm_destroy(None) == FM_OK
    for fn, args in (("fm_set_data", (None, None, None, None, None, 0.1)),
                     ("fm_cost_grad", (None, None, None, None, None)),
                     ("fm_ic_factor", (None, None, None)), ("fm_ic_apply", (None, None, None)),
                     ("fm_solve", (None, None, 0, 1, None)), ("fm_init_omega", (None, None)),
                     ("fm_get_history", (None, None, None, 0))):
        assert getattr(lib, fn)(*args) == FM_ERR_ARG, fn
    assert lib.fm_strerror(-4) == b"IC(0) pivot not positive"
    assert lib.fm_last_error(None) == b""


def test_binding_refuses_to_run_without_the_library(tmp_path):
    from paper_2005_08661_gb300 import load_library
    with pytest.raises(RuntimeError, match="not built"):
        load_library(str(tmp_path / "libfm.so"))
