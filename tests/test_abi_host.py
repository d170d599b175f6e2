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
    return sorted(set(re.findall(r"\b(fm_[a-z_0-9]+)\s*\(", src)))


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


def test_opts_struct_layout_matches_the_header(lib):
    """The ctypes mirror of fm_opts has the C struct's size and field offsets (compiled from
    include/fm.h by the host C compiler), and a bad drop tolerance is refused up front."""
    import subprocess
    from paper_2005_08661_gb300 import FmOpts, FM_ERR_ARG
    fields = [f for f, _ in FmOpts._fields_]
    out_dir = os.path.join(ROOT, "paper_2005_08661_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "opts_layout.c"), os.path.join(out_dir, "opts_layout")
    body = "".join(f'    printf(" %zu", offsetof(fm_opts, {f}));\n' for f in fields)
    with open(src, "w") as fh:
        fh.write("#include <stddef.h>\n#include <stdio.h>\n#include \"fm.h\"\n"
                 "int main(void) {\n    printf(\"%zu\", sizeof(fm_opts));\n" + body + "    return 0;\n}\n")
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(FmOpts)
    assert vals[1:] == [getattr(FmOpts, f).offset for f in fields]
    o = FmOpts()
    lib.fm_default_opts(C.byref(o))
    assert o.droptol == 1e-3
    h = C.c_void_p()
    for bad in (-1e-3, float("nan"), float("inf")):
        o.precond, o.droptol = 4, bad
        assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 3, C.byref(o), 0, None) == FM_ERR_ARG
    assert h.value is None


def test_drop_tolerance_is_only_checked_where_it_applies(lib):
    """fm_opts.droptol is read by FM_PC_ICT only: another preconditioner ignores its value."""
    from paper_2005_08661_gb300 import FmOpts, FM_ERR_ARG
    o = FmOpts()
    lib.fm_default_opts(C.byref(o))
    o.precond, o.droptol = 0, float("nan")
    h = C.c_void_p()
    # argument checks pass; creation then needs a GPU, so only "not an argument error" is checked
    assert lib.fm_create(C.byref(h), 4, 4, 4, 1, 3, C.byref(o), 0, None) != FM_ERR_ARG
    if h.value:
        lib.fm_destroy(h)
