"""FP64 CPU oracle for the regularised field-map estimator (arXiv 2005.08661).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may load it; the library's product path never does.  It shares no
code with the CUDA path.  See fm_oracle.c for what each function computes and the
paper passages it follows.

Pins: every function here is checked against something the paper or the
mathematics fixes (tests/test_oracle_*.py); the Polak-Ribiere step is pinned by the
conjugacy of successive directions on near-quadratic cases (tests/test_oracle_pr.py).
The fixed inner step count of the line search and its zero starting step follow the
readings stated in fm_oracle.c and are "parity unpinned" against the paper itself.
"""
from .oracle import (Oracle, build_oracle, curv_raw, get_threads, ic0_factor, ic0_solve, ict_factor, lib_path,
                     set_threads, voxel_r, voxel_terms, wf_gamma)

__all__ = ["Oracle", "build_oracle", "ic0_factor", "ic0_solve", "ict_factor", "voxel_terms", "voxel_r", "wf_gamma",
           "lib_path", "set_threads", "get_threads", "curv_raw"]
