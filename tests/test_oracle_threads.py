"""The oracle's OpenMP build: per-voxel loops spread over threads and sums taken in fixed
8192-voxel chunks added in chunk order, so every result is bitwise the same for any thread
count (the stored expected values and the GPU parity tests do not depend on it)."""
import numpy as np

from oracle import Oracle, get_threads, set_threads
from synth import make_volume


def test_results_do_not_depend_on_the_thread_count():
    vol = make_volume(40, 36, 12, ncoil=3, snr_db=15.0, seed=21, fmax_hz=150.0, nblobs=3)
    out = []
    try:
        for t in (1, 3, 8):
            set_threads(t)
            o = Oracle.from_volume(vol)
            r = o.solve(niter=3, nls=5)
            w = r["w"]
            out.append((r["cost"], r["alpha"], r["mu"], w, o.grad(w), o.curv(w), o.cost(w)))
            o.close()
    finally:
        set_threads(1)
    assert get_threads() == 1
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(np.asarray(a), np.asarray(b))


def test_curvature_from_raw_data_is_the_precomputed_oracles():
    """curv_raw (Eq. 10 formed voxel by voxel from y and s, for volumes whose precomputed r
    would not fit in memory) is the same computation as Oracle.curv, bitwise."""
    from oracle import curv_raw
    vol = make_volume(30, 26, 9, ncoil=4, snr_db=15.0, seed=22, fmax_hz=150.0, nblobs=3)
    rng = np.random.default_rng(1)
    w = (vol.omega_true + 0.03 * rng.standard_normal(vol.mask.shape)) * vol.mask
    ref = Oracle.from_volume(vol).curv(w)
    try:
        set_threads(4)
        d = curv_raw(vol.y, vol.smap, vol.te, vol.mask, w)
    finally:
        set_threads(1)
    assert np.array_equal(d, ref)
