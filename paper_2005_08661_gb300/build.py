"""Build the CUDA library libfm.so in-tree for sm_103a (GB300).

Translation units are compiled in parallel with nvcc and linked into one shared
library with the CUDA runtime linked statically, so the library depends only on the
driver.  The result lands in paper_2005_08661_gb300/_build/libfm.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["fm_api.cu", "k_setup.cu", "k_data.cu", "k_ic.cu", "k_adj.cu", "k_wf.cu", "k_rb.cu", "k_ict.cu", "fm_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


PROBE = os.path.join(HERE, "probe", "fp32_rate.cu")


def lib_path():
    return os.path.join(BUILD, "libfm.so")


def probe_path():
    return os.path.join(BUILD, "libfmprobe.so")


def _nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fm.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date():
    out = lib_path()
    if not os.path.exists(out) or not os.path.exists(probe_path()):
        return False
    t = min(os.path.getmtime(out), os.path.getmtime(probe_path()))
    return all(os.path.getmtime(f) <= t for f in _deps() + [PROBE])


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link libfm.so unless it is up to date; returns its path."""
    if not force and up_to_date():
        return lib_path()
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    def build_probe():
        tmp = probe_path() + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, *FLAGS, "-shared", "-cudart", "static", PROBE, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on the FP32 rate probe:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, probe_path())

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        probe = ex.submit(build_probe)
        objs = list(ex.map(compile_one, SOURCES))
        probe.result()
    tmp = lib_path() + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    v = "-v" in sys.argv
    flags = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []
    print(build(force=True, verbose=v or bool(flags), extra_flags=flags))
