#!/usr/bin/env python3
"""Throughput of the IC(0)-preconditioned NCG-MLS field-map solve on GB300.

One step = the whole hot path over one synthetic acquisition: fm_set_data (the
Algorithm box's precompute and the Eq. 6 initial map) followed by fm_solve with the
workload's outer-iteration count.  Metric: voxel-NCG-iterations per second =
N_v(grid) x N_outer / step time, summed over ranks.

Default workload: 256 x 256 x 128 voxels, 8 coils, 3 echoes (0/2/10 ms), beta = 2^-3,
100 outer iterations, 5 line-search steps, IC(0) preconditioner, FP32 voxel arithmetic
with FP64 reductions and pivots.  Inputs are seeded synthetic volumes (synth/) standing in
for the paper's datasets; each step streams 2.1 GB of inputs, far more than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torch.distributed.run; each rank solves its own
independent volume (weak scaling, no collective on the data path); the step time is
the maximum over ranks.  --impl reference times the FP64 CPU oracle on the host cores
(rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# ncu DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch, by (workload,
# kernel), from one ncu capture of the full workload (its summary sits with the committed
# profiles), each with the hash of the kernel sources it was measured on: a figure whose
# sources have changed since is reported as null.
KERNEL_SOURCES = {"ls": ("k_data.cu",), "grad": ("k_data.cu",), "ic_fwd": ("k_ic.cu",), "ic_bwd": ("k_ic.cu",)}
NCU_TRAFFIC_BYTES = {  # (bytes per launch, kernel_src_hash of the sources measured)
    ("full", "ls"): (2007300608 + 12793088, "4494fb0460a61f4d"),
    ("full", "grad"): (506223872 + 27680256, "4494fb0460a61f4d"),
    # the IC sweeps on the same 256x256x128 grid with one coil (their work does not depend on it)
    ("full", "ic_fwd"): (79724800 + 37426688, "355df626ce512b8a"),
    ("full", "ic_bwd"): (137366784 + 18694656, "355df626ce512b8a"),
}


def kernel_src_hash(kernel):
    """sha256 (16 hex digits) of the sources a kernel class is built from (its .cu and the
    shared device header)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_08661_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, ()) + ("fm_internal.h",):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel):
    e = NCU_TRAFFIC_BYTES.get((workload, kernel))
    if e is None or e[1] != kernel_src_hash(kernel):
        return None
    return e[0]

WORKLOADS = {
    "full": dict(desc="256x256x128 voxels, 8 coils, 3 echoes (0/2/10 ms), SNR 15 dB, beta=2^-3, "
                      "100 NCG iterations, N_ls=5, IC(0)", niter=100),
    "small": dict(desc="64x64x16 voxels, 1 coil, 3 echoes (0/2/10 ms), SNR 20 dB, beta=2^-3, "
                       "50 NCG iterations, N_ls=5, IC(0)", niter=50),
    "medium": dict(desc="128x128x64 voxels, 8 coils, 3 echoes (0/2/10 ms), SNR 20 dB, beta=2^-3, "
                        "100 NCG iterations, N_ls=5, IC(0)", niter=100),
    "full1": dict(desc="256x256x128 voxels, 1 coil, 3 echoes (0/2/10 ms), SNR 15 dB, beta=2^-3, "
                       "100 NCG iterations, N_ls=5, IC(0) (the full grid with one coil: the IC sweeps' "
                       "profiling case)", niter=100),
    "batch": dict(desc="32 independent volumes from 64x64x16 to 192x192x96, 1 or 8 coils, 3 echoes "
                       "(0/2/10 ms), SNR 10-25 dB, beta=2^-3, 50 NCG iterations each, N_ls=5, IC(0), one "
                       "CUDA graph launch per two iterations of all volumes", niter=50),
    "wf": dict(desc="water-fat: 192x192x64 voxels, 1 coil, 6 echoes (1.2..6.2 ms), seeded 6-peak fat spectrum "
                    "(-3.8..+0.6 ppm at 3 T), +-200 Hz smooth field, SNR 20 dB, beta=2^-7; per step: setup, "
                    "100-value voxel-wise sweep, 10 PWLS CG iterations, 100 NCG iterations (N_ls=5, IC(0)), "
                    "water/fat amplitudes", niter=100),
    "precond": dict(desc="preconditioner comparison: 74x74x10 voxels, 32 coils, 3 echoes (0/1/2.3 ms), SNR 20 dB, "
                         "beta=2^-3, FP32 NCG-MLS (N_ls=5) with IC(0) natural order, IC with drop tolerance "
                         "1e-3 H_max, IC(0) red-black, diagonal, none: iterations and time until the RMSD to the "
                         "converged map falls below 0.5 Hz",
                    niter=0),
    "diff": dict(desc="128x128x64 voxels, 8 coils, 3 echoes (0/2/10 ms), SNR 20 dB, beta=2^-3: "
                      "torch.autograd forward (100 NCG iterations) + backward (IC(0)-preconditioned adjoint "
                      "CG to 1e-6, dl/dbeta and dl/dy) of l = ||w^ - w_true||^2", niter=100),
}
CPU_SAMPLE = (64, 64, 32)  # oracle sample (all host cores): centred sub-volume of the same acquisition
CPU_SAMPLE_1CORE = (32, 32, 16)  # the one-thread figure, on a smaller centred sub-volume


def make_workload(name, seed_offset=0):
    from synth import diff_config, full1_config, full_config, small_config, wf_config
    if name == "full1":
        return full1_config(seed=1002 + seed_offset)
    if name == "wf":
        return wf_config(seed=1003 + seed_offset)
    if name == "full":
        return full_config(seed=1002 + seed_offset)
    if name == "medium":
        return diff_config(seed=1005 + seed_offset)
    return small_config(seed=1001 + seed_offset)


def sub_volume(vol, size):
    """Centred sub-block of a volume (same data, mask and coils) for oracle sampling."""
    from synth import Volume
    sx, sy, sz = min(size[0], vol.nx), min(size[1], vol.ny), min(size[2], vol.nz)
    x0, y0, z0 = (vol.nx - sx) // 2, (vol.ny - sy) // 2, (vol.nz - sz) // 2
    sl = (slice(z0, z0 + sz), slice(y0, y0 + sy), slice(x0, x0 + sx))
    return Volume(y=np.ascontiguousarray(vol.y[(slice(None), slice(None)) + sl]),
                  smap=None if vol.smap is None else np.ascontiguousarray(vol.smap[(slice(None),) + sl]),
                  mask=np.ascontiguousarray(vol.mask[sl]), te=vol.te, omega_true=vol.omega_true[sl],
                  beta=vol.beta, name=f"{vol.name}_sub{sx}x{sy}x{sz}",
                  meta={k: v for k, v in vol.meta.items() if k.startswith("fat_")})


# ------------------------------------------------------------------ flop / byte model

def data_eval_flops(nc, L, literal):
    """Algorithmic flops of one voxel's data-term evaluation (gradient + curvature), by the
    method's work count rather than the implementation's instructions: about 12 per echo-pair
    rotation (the phase of the pair term and its cost and gradient contributions, Eq. 2 and 8)
    and about 14 per wrapped-sinc curvature term (Eq. 10-11: phase, wrap into [-pi, pi],
    sin(u)/u, weighted accumulation) -- N_c^2 of them per pair for the literal curvature, one
    per pair for the coil-combined form."""
    P = L * (L - 1) // 2
    return P * (12 + 14 * (nc * nc if literal else 1))


def data_eval_bytes(nc, L, literal, ts=4):
    P = L * (L - 1) // 2
    b = P * 2 * ts + 1 + 2 * ts  # pair polar, mask bits, w and z
    if literal:
        b += L * nc * 2 * ts
    return b


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy peak is the roofline)


def fp32_probe(device):
    """Measured FP32 FMA rate of the GPU (paper_2005_08661_gb300/probe/fp32_rate.cu):
    (TFLOP/s, FMA lane-ops per SM per clock, SM MHz during the probe), or None."""
    import ctypes as C
    from paper_2005_08661_gb300 import build as fm_build
    try:
        lib = C.CDLL(fm_build.probe_path())
        f = lib.fmprobe_fp32_rate
        f.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        f.restype = C.c_int
        t, r, m = C.c_double(), C.c_double(), C.c_double()
        if f(int(device), C.byref(t), C.byref(r), C.byref(m)) != 0:
            return None
        return t.value, r.value, m.value
    except OSError:
        return None


def peak_numbers(sm_mhz, nsm, probe=None):
    """Roofline denominators: the measured HBM copy bandwidth, and the FP32 rate measured by the
    FMA probe scaled to the SM clock of the timed region (else derived from 128 lanes per SM)."""
    peaks = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mp = json.load(open(path))
        peaks["hbm_gbs"] = float(mp["hbm_gbs"])
        peaks["hbm_src"] = "of measured"
    else:
        peaks["hbm_gbs"] = 6800.0
        peaks["hbm_src"] = "of fallback"
    if probe is not None:
        tflops, per_clk, mhz = probe
        peaks["fp32_tflops"] = 2 * per_clk * nsm * sm_mhz * 1e6 / 1e12
        peaks["fp32_src"] = (f"of measured: FMA probe {per_clk:.1f} FP32 FMA/clk/SM ({tflops:.1f} TFLOP/s at "
                             f"{mhz:.0f} MHz), x {nsm} SMs x {sm_mhz:.0f} MHz of the timed region")
    else:
        peaks["fp32_tflops"] = 2 * 128 * nsm * sm_mhz * 1e6 / 1e12
        peaks["fp32_src"] = f"derived: 2 flops x 128 FP32 lanes x {nsm} SMs x {sm_mhz:.0f} MHz"
    return peaks


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ oracle (CPU baseline / reference arm)

def _oracle_child(p):
    """Runs in a spawned process (no CUDA context, its own OpenMP runtime): times the FP64
    oracle on one sub-volume, p["reps"] times; returns (seconds of each rep, threads used)."""
    from oracle import Oracle, set_threads, wf_gamma
    from synth import Volume
    used = set_threads(p["threads"])
    sub = Volume(y=p["y"], smap=p["smap"], mask=p["mask"], te=p["te"], omega_true=np.zeros(p["mask"].shape),
                 beta=p["beta"], name="sample", meta=p["meta"])
    out = []
    for _ in range(p["reps"]):
        if "fat_amps" in sub.meta:  # water-fat: the sweep + PWLS start, then the timed NCG iterations
            amps, freqs = sub.meta["fat_amps"], sub.meta["fat_freqs_khz"]
            o = Oracle.from_volume(sub)
            o.set_gamma(wf_gamma(sub.te, amps, freqs)[1])
            half = float(np.pi * abs(freqs[int(np.argmax(amps))]))
            w0 = o.pwls(o.wf_sweep(100, -half, half), 10)
            t0 = time.perf_counter()
            o.solve(w0=w0, niter=p["iters"], nls=5)
            out.append(time.perf_counter() - t0)
            o.close()
            continue
        t0 = time.perf_counter()
        o = Oracle.from_volume(sub)
        if p["curvature"] == "combined":
            o.set_curvature("combined")
        o.solve(niter=p["iters"], nls=5)
        out.append(time.perf_counter() - t0)
        o.close()
    return out, used


def oracle_sample(vol, iters, curvature="literal", threads=None, size=CPU_SAMPLE, reps=1):
    """Time the FP64 oracle (precompute + iters NCG-MLS iterations) on a centred sub-volume in a
    spawned process with `threads` host threads (default: all); returns (seconds per rep,
    voxel-iterations per rep, threads used, sub-volume)."""
    import multiprocessing as mp
    sub = sub_volume(vol, size)
    meta = {k: v for k, v in sub.meta.items() if k.startswith("fat_")}
    payload = dict(y=sub.y, smap=sub.smap, te=sub.te, mask=sub.mask, beta=sub.beta, meta=meta, iters=iters,
                   threads=threads or os.cpu_count() or 1, curvature=curvature, reps=reps)
    with mp.get_context("spawn").Pool(1) as pool:
        dts, used = pool.apply(_oracle_child, (payload,))
    return dts, sub.nvox * iters, used, sub


def sample_desc(sub, iters, threads, curvature, ncoil):
    return (f"FP64 C oracle, {threads} thread{'s' if threads > 1 else ''} (OpenMP, fixed-chunk sums), precompute + "
            f"{iters} NCG-MLS-IC(0) iteration{'s' if iters > 1 else ''} (N_ls=5) on the centred "
            f"{sub.nx}x{sub.ny}x{sub.nz} sub-volume of the workload ({ncoil} coils, {curvature} curvature), host "
            f"{cpu_desc()}, nproc {os.cpu_count()}")


def cpu_desc():
    model = ""
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "processor\t")) and "model name" in ln.lower():
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model or os.uname().machine


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    vol = make_workload(args.workload)
    # one step = the oracle's precompute + 1 NCG-MLS iteration on the sample, all host cores
    dts, units, used, sub = oracle_sample(vol, 1, args.curvature, reps=args.warmup + args.steps)
    times = dts[args.warmup:]
    t = sum(times) / len(times)
    value = units / t
    sample = sample_desc(sub, 1, used, args.curvature, vol.ncoil) + ", per step"
    line = {"metric": "voxel-NCG-iters/s", "value": value, "unit": "voxel-iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main arm

def run_ours(args, world, rank, local, quiet=False):
    import torch
    from paper_2005_08661_gb300 import FieldMap, build as fm_build
    fm_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vol = make_workload(args.workload, seed_offset=rank)
    niter = args.niter or WORKLOADS[args.workload]["niter"]
    prec = args.precision
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    rd = torch.float32 if prec == "fp32" else torch.float64
    y_h = torch.from_numpy(vol.y).to(cd).pin_memory()
    s_h = torch.from_numpy(vol.smap).to(cd).pin_memory() if vol.smap is not None else None
    m_h = torch.from_numpy(vol.mask).pin_memory()
    stream = torch.cuda.Stream(dev)
    y_d = torch.empty_like(y_h, device=dev)
    s_d = torch.empty_like(s_h, device=dev) if s_h is not None else None
    m_d = torch.empty_like(m_h, device=dev)
    with torch.cuda.stream(stream):
        y_d.copy_(y_h)
        if s_d is not None:
            s_d.copy_(s_h)
        m_d.copy_(m_h)
    stream.synchronize()
    nv = vol.nvox
    nmask = int(vol.mask.sum())
    fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision=prec, device=local,
                  stream=stream, curvature=args.curvature)
    fm.set_profiling(True)
    w = torch.empty(vol.mask.shape, dtype=rd, device=dev)
    w_h = torch.empty(vol.mask.shape, dtype=rd).pin_memory()
    wf = "fat_amps" in vol.meta
    if wf:  # water-fat: sweep + PWLS start, NCG from there, then the water and fat maps
        fm.set_fat_model(vol.meta["fat_amps"], vol.meta["fat_freqs_khz"])
        w_t = torch.empty_like(w)
        amp_w = torch.empty(vol.mask.shape, dtype=cd, device=dev)
        amp_f = torch.empty_like(amp_w)

    def solve_path(inputs=None):
        yb, sb, mb = inputs if inputs is not None else (y_d, s_d, m_d)
        fm.set_data(yb, sb, vol.te, mb, vol.beta)
        if wf:
            fm.wf_sweep(100, out=w_t)
            fm.pwls_init(w_t, 10, out=w)
            fm.solve_into(w, False, niter)
            fm.wf_amplitudes(w, out=(amp_w, amp_f))
        else:
            fm.solve_into(w, True, niter)

    def step():
        solve_path()

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1000.0 / args.steps
    kt = fm.kernel_times()
    t_step = max_over_ranks(t_step, world, dev)
    value = world * nv * niter / t_step

    # end to end through the C ABI's host-buffer calls (fm_set_data_host, fm_solve_host): every
    # step copies its images, coil maps and mask from page-locked host memory into the
    # library's staging buffers (its copy stream) and the field map back to host memory; the
    # upload of step k + 1 runs while step k is solved
    h2d = y_h.numel() * y_h.element_size() + m_h.numel() + (s_h.numel() * s_h.element_size() if s_h is not None else 0)
    d2h = w.numel() * w.element_size()
    e2e = None
    if not args.no_e2e and not wf:
        fm_io = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision=prec, device=local,
                         stream=stream, curvature=args.curvature)
        fm_io.set_profiling(True)

        def run_e2e(nsteps):
            for _ in range(nsteps):
                fm_io.set_data_host(y_h, s_h, vol.te, m_h, vol.beta)
                fm_io.solve_host(w_h, True, niter)

        run_e2e(2)
        fm_io.synchronize()
        barrier(world)
        nst = max(1, args.steps)
        e0.record(stream)
        run_e2e(nst)
        e1.record(stream)
        fm_io.synchronize()
        torch.cuda.synchronize(dev)
        barrier(world)
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1000.0 / nst, world, dev)
        kio = fm_io.kernel_times()
        h2d_ms, d2h_ms = kio["h2d"][0], kio["d2h"][0]
        fm_io.close()
        e2e = {"value": world * nv * niter / t_e2e, "unit": "voxel-iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * t_e2e,
               "h2d_ms_per_step": h2d_ms, "h2d_gbs": h2d / (h2d_ms * 1e-3) / 1e9 if h2d_ms > 0 else None,
               "d2h_ms_per_step": d2h_ms,
               "path": "C ABI fm_set_data_host + fm_solve_host on page-locked host buffers; the library's copy "
                       "stream uploads step k+1 while step k is solved"}

    # roofline of the kernel with the largest share of the outer iteration
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_run = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peaks = peak_numbers(sm_run, nsm, fp32_probe(local))
    per_iter = {k: v[0] for k, v in kt.items() if v[1] > 0 and k in ("grad", "ic_fwd", "ic_bwd", "ls")}
    dom = max(per_iter, key=per_iter.get) if per_iter else None
    literal = vol.ncoil > 1 and args.curvature == "literal"
    def kernel_roofline(name, ms):
        """Algorithmic work of one launch of kernel class `name` against its bound."""
        evals = {"grad": 1, "ls": 4}.get(name, 0)
        ts = 4 if prec == "fp32" else 8
        dir_bytes = nmask * (4 + 1 + 6 * ts) if name == "ls" else 0  # the line search's direction phase
        if evals and literal:
            flops = evals * nmask * data_eval_flops(vol.ncoil, vol.necho, True)
            ach = flops / (ms * 1e-3) / 1e12
            byts = evals * nmask * data_eval_bytes(vol.ncoil, vol.necho, literal, ts) + dir_bytes
            hbm = byts / (ms * 1e-3) / 1e9
            return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                    "frac": ach / peaks["fp32_tflops"], "peak_src": peaks["fp32_src"], "ms_per_launch": ms,
                    "algorithmic_flops_per_launch": flops,
                    "flop_count": "per mask voxel and evaluation: 12 per echo-pair rotation + 14 per wrapped-sinc "
                                  "term (N_c^2 per pair)",
                    "hbm": {"achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": hbm / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": byts},
                    "traffic": ncu_traffic(args.workload, name)}
        if evals:
            byts = evals * (nmask * data_eval_bytes(vol.ncoil, vol.necho, literal, ts) + nv) + dir_bytes
        elif name == "ic_fwd":  # per grid voxel: bits, d and g in, pivots and v out
            byts = nv * (1 + 2 * ts + 2 * ts)
        elif name == "ic_bwd":  # per grid voxel: bits, v, pivots, g, g_prev in, p out
            byts = nv * (1 + 2 * ts + 3 * ts)
        else:
            return None
        ach = byts / (ms * 1e-3) / 1e9
        out = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": ach / peaks["hbm_gbs"], "peak_src": peaks["hbm_src"], "ms_per_launch": ms,
               "algorithmic_bytes_per_launch": byts, "traffic": ncu_traffic(args.workload, name)}
        if name.startswith("ic"):
            out["note"] = "latency-bound wavefront: the HBM fraction is reported for reference only"
        return out

    roof = kernel_roofline(dom, per_iter[dom]) if dom is not None else None
    kernels = {}
    for k, v in kt.items():
        if v[1] > 0 and k in ("grad", "ic_fwd", "ic_bwd", "ls"):
            r = kernel_roofline(k, v[0])
            kernels[k] = {"ms_per_launch": v[0], "share_of_iteration": v[0] / sum(per_iter.values()),
                          "bound": r["bound"], "achieved": r["achieved"], "unit": r["unit"], "frac": r["frac"]}
            if "hbm" in r:
                kernels[k]["hbm_frac_algorithmic"] = r["hbm"]["frac"]
            tb = ncu_traffic(args.workload, k)
            if tb:  # ncu DRAM bytes of one launch over its CUDA-event time, against the HBM peak
                kernels[k]["hbm_traffic_frac"] = tb / (v[0] * 1e-3) / 1e9 / peaks["hbm_gbs"]
                kernels[k]["hbm_traffic_frac_nominal"] = tb / (v[0] * 1e-3) / 1e9 / HBM_NOMINAL_GBS

    # time to the oracle's final cost on the small workload and on the eight-coil 64x64x32
    # volume (oracle histories stored by tests/golden/make_golden.py)
    ttc = ttc8 = None
    if rank == 0 and not args.no_ttc:
        ttc = time_to_oracle_cost(prec, stream, "small")
        ttc8 = time_to_oracle_cost(prec, stream, "full8")

    # the batched, water-fat, differentiation and preconditioner forms, measured after the main
    # figures (short runs; each form's own workload line comes from --workload)
    batch = forms = None
    if rank == 0 and world == 1 and not args.no_forms and args.workload == "full":
        fm_keep = fm
        batch = batch_summary(local, prec, 3, 2)
        forms = forms_summary(local, prec)
        fm = fm_keep

    # the precision form against the plain FP64 GPU solve of the same workload (untimed)
    fp64cmp = None
    if rank == 0 and prec == "fp32" and not args.no_fp64_check:
        w32, c32 = fm.solve(None, niter=niter)
        w32 = w32.double()
        ref = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision="fp64", device=local,
                       stream=stream, curvature=args.curvature)
        ref.set_data(y_d.to(torch.complex128), s_d.to(torch.complex128) if s_d is not None else None, vol.te, m_d,
                     vol.beta)
        if wf:
            ref.set_fat_model(vol.meta["fat_amps"], vol.meta["fat_freqs_khz"])
            ref.set_data(y_d.to(torch.complex128), s_d.to(torch.complex128) if s_d is not None else None, vol.te,
                         m_d, vol.beta)
            w64_0 = ref.pwls_init(ref.wf_sweep(100), 10)
            w64, c64 = ref.solve(w64_0, niter=niter)
            w32_0 = fm.pwls_init(fm.wf_sweep(100), 10)
            w32, c32 = fm.solve(w32_0, niter=niter)
            w32 = w32.double()
        else:
            w64, c64 = ref.solve(None, niter=niter)
        ref.close()
        mk = m_d.bool()
        dhz = (w32 - w64)[mk].abs() * 1000.0 / (2 * math.pi)
        fp64cmp = {"final_cost_rel": abs(c32[-1] - c64[-1]) / abs(c64[-1]),
                   "rmse_hz": float(dhz.pow(2).mean().sqrt()), "max_abs_hz": float(dhz.max()),
                   "what": f"FP32 path vs the FP64 GPU path, {niter} iterations each, over the mask"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        iters = 8 if literal else 20
        dts, units, used, sub = oracle_sample(vol, iters, args.curvature)
        cpu = {"value": units / dts[0], "unit": "voxel-iter/s", "cores": used, "kind": "oracle",
               "sample": sample_desc(sub, iters, used, args.curvature, vol.ncoil) + f", {dts[0]:.1f} s"}
        dts1, units1, _, sub1 = oracle_sample(vol, 1, args.curvature, threads=1, size=CPU_SAMPLE_1CORE)
        cpu["one_core"] = {"value": units1 / dts1[0], "unit": "voxel-iter/s", "cores": 1,
                           "sample": sample_desc(sub1, 1, 1, args.curvature, vol.ncoil) + f", {dts1[0]:.1f} s"}

    # per step: mask count, chunk scan, setup; 4 kernels per outer iteration (gradient pass, IC
    # forward and back sweeps, direction + line search); the final update (water-fat adds the
    # sweep, the PWLS start and 2 kernels per PWLS iteration, the amplitudes)
    launches = args.steps * (3 + 4 * niter + 1 + ((1 + 1 + 2 * 10 + 1) if wf else 0))
    line = {"metric": "voxel-NCG-iters/s", "value": value, "unit": "voxel-iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "voxels": nv, "mask_voxels": nmask,
                       "niter": niter, "nls": 5, "precision": ("fp32 voxel arithmetic, fp64 reductions and IC "
                                                               "pivots" if prec == "fp32" else "fp64"),
                       "curvature": args.curvature,
                       "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (2.1 GB streamed per step)",
                       "masked_voxel_iters_per_s": world * nmask * niter / t_step},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "kernels": kernels, "clocks": clk,
            "cpu_baseline": cpu, "time_to_oracle_cost": ttc, "time_to_oracle_cost_8coil": ttc8,
            "fp32_vs_fp64_gpu": fp64cmp, "batch": batch, "forms": forms}
    if rank == 0 and not quiet:
        print(json.dumps(line), flush=True)
    fm.close()
    return line if quiet else 0


def batch_summary(local, precision, steps, warmup, rank=0):
    """The batched form's numbers for the main line: the 32-volume aggregate (one graph launch
    per two iterations of every volume) against the same volumes solved one after another."""
    class A:
        pass
    a = A()
    a.niter, a.precision, a.steps, a.warmup = 0, precision, steps, warmup
    line = run_batch(a, 1, rank, local, quiet=True)
    return {"workload": WORKLOADS["batch"]["desc"], "value": line["value"], "unit": "voxel-iter/s",
            "ms_per_step": line["ms_per_step"], "sequential": line["sequential"],
            "speedup_vs_sequential": line["speedup_vs_sequential"], "steps": steps, "warmup": warmup,
            "grid_fraction": line["config"]["grid_fraction"],
            "ic_bwd_blocks_per_sm": line["config"]["ic_bwd_blocks_per_sm"]}


def forms_summary(local, precision):
    """Short runs of the water-fat, differentiation and preconditioner-comparison workloads for
    the main line (each is its own line with --workload wf|diff|precond)."""
    class A:
        pass
    out = {}
    for name, fn in (("wf", run_ours), ("diff", run_diff), ("precond", run_precond)):
        a = A()
        a.workload, a.precision, a.curvature, a.niter = name, precision, "literal", 0
        a.steps, a.warmup = (1, 1) if name == "precond" else (3, 2)
        a.no_e2e = a.no_cpu_baseline = a.no_ttc = a.no_forms = True
        a.no_fp64_check = name != "wf"
        try:
            line = fn(a, 1, 0, local, quiet=True)
        except Exception as e:  # a form that fails is reported, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"}
            continue
        keep = {"workload": WORKLOADS[name]["desc"], "value": line["value"], "unit": line["unit"],
                "ms_per_step": line.get("ms_per_step")}
        for k in ("fp32_vs_fp64_gpu", "fp32_error_vs_fp64_gpu", "backward", "preconditioners"):
            if k in line:
                keep[k] = line[k]
        out[name] = keep
    return out


def run_batch(args, world, rank, local, quiet=False):
    """Config-4 form: aggregate voxel-NCG-iters/s of 32 uneven volumes solved together,
    against the same 32 volumes solved one after another with fm_solve."""
    import torch
    from paper_2005_08661_gb300 import FieldMap, FieldMapBatch, build as fm_build
    from synth import batch_configs, make_volume
    import ctypes as C
    fm_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    niter = args.niter or WORKLOADS["batch"]["niter"]
    cfgs = batch_configs(32, seed=1004 + rank)
    vols = [make_volume(c["nx"], c["ny"], c["nz"], ncoil=c["ncoil"], snr_db=c["snr_db"], seed=c["seed"],
                        fmax_hz=200.0, nblobs=4) for c in cfgs]
    cd = torch.complex64 if args.precision == "fp32" else torch.complex128
    dev_in = []
    for v in vols:
        y = torch.from_numpy(v.y).to(dev).to(cd)
        s = torch.from_numpy(v.smap).to(dev).to(cd) if v.smap is not None else None
        m = torch.from_numpy(v.mask).to(dev)
        dev_in.append((y, s, m))
    stream = torch.cuda.Stream(dev)
    nvox = sum(v.nvox for v in vols)
    b = FieldMapBatch([(v.nx, v.ny, v.nz, v.ncoil, v.necho) for v in vols], precision=args.precision, device=local,
                      stream=stream)
    for k, v in enumerate(vols):
        b.set_data(k, dev_in[k][0], dev_in[k][1], v.te, dev_in[k][2], v.beta)
    frac, _ = b.autotune(niter_probe=4)
    _, order_w = b.schedule()
    bwd_blocks = b.bwd_blocks_per_sm()
    ws = [b.empty(k) for k in range(len(vols))]
    ptrs = (C.c_void_p * len(vols))(*[w.data_ptr() for w in ws])

    def step_batch():
        for k, v in enumerate(vols):
            b.set_data(k, dev_in[k][0], dev_in[k][1], v.te, dev_in[k][2], v.beta)
        b.solve_into(ptrs, True, niter)

    singles = [FieldMap(v.nx, v.ny, v.nz, ncoil=v.ncoil, necho=v.necho, precision=args.precision, device=local,
                        stream=stream) for v in vols]

    def step_seq():
        for k, v in enumerate(vols):
            singles[k].set_data(dev_in[k][0], dev_in[k][1], v.te, dev_in[k][2], v.beta)
            singles[k].solve_into(ws[k], True, niter)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1000.0 / args.steps

    clocks = ClockSampler(local)
    t_b = max_over_ranks(timed(step_batch), world, dev)
    clk = clocks.stop()
    t_s = max_over_ranks(timed(step_seq), world, dev)

    # the batched FP32 maps against plain FP64 GPU solves of a sample of the volumes (untimed)
    cmp = None
    if rank == 0 and args.precision == "fp32" and not quiet:
        step_batch()
        torch.cuda.synchronize(dev)
        order = sorted(range(len(vols)), key=lambda k: vols[k].nvox)
        sample = sorted({order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]})
        worst = {"rmse_hz": 0.0, "max_abs_hz": 0.0}
        for k in sample:
            v = vols[k]
            ref = FieldMap(v.nx, v.ny, v.nz, ncoil=v.ncoil, necho=v.necho, precision="fp64", device=local,
                           stream=stream)
            s64 = dev_in[k][1].to(torch.complex128) if dev_in[k][1] is not None else None
            ref.set_data(dev_in[k][0].to(torch.complex128), s64, v.te, dev_in[k][2], v.beta)
            w64, _ = ref.solve(None, niter=niter, want_history=False)
            ref.close()
            mk = dev_in[k][2].bool()
            dhz = (ws[k].double() - w64)[mk].abs() * 1000.0 / (2 * math.pi)
            worst["rmse_hz"] = max(worst["rmse_hz"], float(dhz.pow(2).mean().sqrt()))
            worst["max_abs_hz"] = max(worst["max_abs_hz"], float(dhz.max()))
        cmp = dict(worst, volumes=[f"{vols[k].nx}x{vols[k].ny}x{vols[k].nz}_c{vols[k].ncoil}" for k in sample],
                   what=f"batched FP32 maps vs plain FP64 GPU solves, {niter} iterations, over the mask (worst)")
    line = {"metric": "voxel-NCG-iters/s", "value": world * nvox * niter / t_b, "unit": "voxel-iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"]["desc"], "volumes": len(vols), "voxels": nvox, "niter": niter,
                       "grid_fraction": frac, "ic_tile_order_weights": list(order_w),
                       "ic_bwd_blocks_per_sm": bwd_blocks,
                       "parallelism": f"replicas{world}"},
            "sequential": {"value": world * nvox * niter / t_s, "ms_per_step": 1000 * t_s,
                           "what": "the same 32 volumes, fm_set_data + fm_solve one after another"},
            "speedup_vs_sequential": t_s / t_b, "fp32_vs_fp64_gpu": cmp, "clocks": clk}
    if rank == 0 and not quiet:
        print(json.dumps(line), flush=True)
    for f in singles:
        f.close()
    b.close()
    return line if quiet else 0


def run_diff(args, world, rank, local, quiet=False):
    """Differentiation form: forward solve + implicit-gradient backward through
    torch.autograd, FP32 timed, with the FP64 GPU path as the accuracy reference."""
    import torch
    from paper_2005_08661_gb300 import FieldMap, build as fm_build, field_map_solve
    from synth import diff_config
    fm_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    niter = args.niter or WORKLOADS["diff"]["niter"]
    vol = diff_config(seed=1005 + rank)
    nv = vol.nvox
    stream = torch.cuda.Stream(dev)

    def setup(prec):
        cd = torch.complex64 if prec == "fp32" else torch.complex128
        rd = torch.float32 if prec == "fp32" else torch.float64
        y = torch.from_numpy(vol.y).to(dev).to(cd).contiguous()
        s = torch.from_numpy(vol.smap).to(dev).to(cd).contiguous()
        m = torch.from_numpy(vol.mask).to(dev)
        tgt = torch.from_numpy(vol.omega_true * vol.mask).to(dev).to(rd)
        fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision=prec, device=local,
                      stream=stream)
        return fm, y, s, m, tgt

    def fwd_bwd(fm, y, s, m, tgt, ev=None):
        yv = y.clone().requires_grad_(True)
        beta = torch.tensor(vol.beta, dtype=torch.float64, requires_grad=True)
        w = field_map_solve(yv, beta, fm, s, vol.te, m, niter=niter)
        loss = ((w - tgt) ** 2 * m).sum()
        if ev is not None:
            ev[0].record(stream)
        dy, db = torch.autograd.grad(loss, (yv, beta))
        if ev is not None:
            ev[1].record(stream)
        return w, dy, db

    res = {}
    with torch.cuda.stream(stream):
        for prec in ("fp64", "fp32"):
            fm, y, s, m, tgt = setup(prec)
            steps = args.steps if prec == "fp32" else 1
            for _ in range(args.warmup if prec == "fp32" else 1):
                fwd_bwd(fm, y, s, m, tgt)
            torch.cuda.synchronize(dev)
            clocks = ClockSampler(local) if prec == "fp32" else None
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            em = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            e0.record(stream)
            out = None
            for k in range(steps):
                out = fwd_bwd(fm, y, s, m, tgt, em[k])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            clk = clocks.stop() if clocks else None
            total = e0.elapsed_time(e1) / steps
            bwd = sum(a.elapsed_time(b) for a, b in em) / steps
            res[prec] = dict(ms=total, bwd_ms=bwd, w=out[0].detach().double(), dy=out[1].to(torch.complex128),
                             db=float(out[2]), adj=dict(fm.last_adjoint), clk=clk)
            fm.close()
    t_s = max_over_ranks(res["fp32"]["ms"] / 1000.0, world, dev)
    r32, r64 = res["fp32"], res["fp64"]
    err = {"dl_dbeta_rel": abs(r32["db"] - r64["db"]) / abs(r64["db"]),
           "dl_dy_rel_l2": float((r32["dy"] - r64["dy"]).norm() / r64["dy"].norm()),
           "w_hat_rms_hz": float(((r32["w"] - r64["w"]) ** 2 * torch.from_numpy(vol.mask).to(dev)).sum().div(
               float(vol.mask.sum())).sqrt()) * 1000.0 / (2 * math.pi)}
    line = {"metric": "voxel-NCG-iters/s", "value": world * nv * niter / t_s, "unit": "voxel-iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["diff"]["desc"], "voxels": nv, "mask_voxels": int(vol.mask.sum()),
                       "niter": niter, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (0.4 GB of pair/coil data streamed per evaluation)"},
            "backward": {"ms": r32["bwd_ms"], "adjoint_cg_iterations": r32["adj"]["iterations"],
                         "adjoint_relres": r32["adj"]["relres"],
                         "ms_per_cg_iteration": r32["bwd_ms"] / max(1, r32["adj"]["iterations"])},
            "fp64_gpu": {"ms_per_step": r64["ms"], "backward_ms": r64["bwd_ms"],
                         "adjoint_cg_iterations": r64["adj"]["iterations"], "adjoint_relres": r64["adj"]["relres"]},
            "fp32_error_vs_fp64_gpu": err, "clocks": r32["clk"]}
    if rank == 0:
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    return line if quiet else 0


def run_precond(args, world, rank, local, quiet=False):
    """Time for each preconditioner to bring the RMSD to the converged map below 0.5 Hz
    (the paper's phantom comparison), with the converged map from a long FP64 IC(0) solve."""
    import torch
    from paper_2005_08661_gb300 import FieldMap, FmError, build as fm_build
    from synth import phantom_config
    fm_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vol = phantom_config(seed=1006 + rank)
    stream = torch.cuda.Stream(dev)
    m = torch.from_numpy(vol.mask).to(dev)
    nmask = int(vol.mask.sum())

    def open_fm(prec, pc):
        cd = torch.complex64 if prec == "fp32" else torch.complex128
        fm = FieldMap(vol.nx, vol.ny, vol.nz, ncoil=vol.ncoil, necho=vol.necho, precision=prec, precond=pc,
                      device=local, stream=stream)
        fm.set_data(torch.from_numpy(vol.y).to(dev).to(cd), torch.from_numpy(vol.smap).to(dev).to(cd), vol.te, m,
                    vol.beta)
        return fm

    ref = open_fm("fp64", "ic0")
    w_inf, _ = ref.solve(niter=400, want_history=False)
    ref.close()
    w_inf = w_inf.double()
    hz = 1000.0 / (2 * math.pi)

    def rmsd_hz(w):
        return float(((w.double() - w_inf) ** 2 * m).sum().div(nmask).sqrt()) * hz

    def precond_row(pc):
        fm = open_fm("fp32", pc)
        cache = {}

        def rmsd_at(k):
            if k not in cache:
                w, _ = fm.solve(niter=k, want_history=False)
                cache[k] = rmsd_hz(w)
            return cache[k]
        try:
            kmax = 4096
            hi = 1
            while hi < kmax and rmsd_at(hi) >= 0.5:
                hi *= 2
            if rmsd_at(hi) >= 0.5:
                return {"iterations": None, "ms": None, "rmsd_hz_at_limit": rmsd_at(hi)}
            lo = hi // 2
            while hi - lo > 1:  # first k with RMSD < 0.5 Hz (RMSD falls monotonically here)
                mid = (lo + hi) // 2
                if rmsd_at(mid) < 0.5:
                    hi = mid
                else:
                    lo = mid
            k = hi
            w = torch.empty(vol.mask.shape, dtype=torch.float32, device=dev)
            for _ in range(max(3, args.warmup)):
                fm.solve_into(w, True, k)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(1, args.steps)
            e0.record(stream)
            for _ in range(reps):
                fm.solve_into(w, True, k)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return {"iterations": k, "ms": e0.elapsed_time(e1) / reps, "rmsd_hz": rmsd_at(k)}
        finally:
            fm.close()

    rows = {}
    for pc in ("ic0", "ict", "rb", "diag", "none"):
        try:
            rows[pc] = precond_row(pc)
        except FmError as e:  # FM_ERR_FILL: the kept fill needs more offsets than the factor holds
            rows[pc] = {"iterations": None, "ms": None, "error": str(e)}
    base = rows["ic0"]["ms"]
    for r in rows.values():
        r["vs_ic0"] = (r["ms"] / base) if (r.get("ms") and base) else None
    line = {"metric": "time to RMSD < 0.5 Hz", "value": base, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["precond"]["desc"], "voxels": vol.nvox, "mask_voxels": nmask,
                       "reference": "converged map: 400 FP64 IC(0) iterations", "parallelism": f"replicas{world}"},
            "preconditioners": rows}
    if rank == 0:
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    return line if quiet else 0


TTC_CASES = {
    "small": ("small_oracle_cost.json", WORKLOADS["small"]["desc"]),
    "full8": ("full8_oracle_cost.json", "64x64x32 voxels, 8 coils, 3 echoes (0/2/10 ms), +-250 Hz + 40 Hz step, "
                                        "SNR 15 dB, beta=2^-3 (the full workload's recipe), 100 NCG iterations, "
                                        "N_ls=5, IC(0)"),
}


def time_to_oracle_cost(prec, stream, case="small"):
    """Seconds (setup + solve, CUDA events) until the GPU solve's cost first falls to the FP64
    oracle's final cost x (1 + 1e-6), on the 64x64x16 one-coil workload or the 64x64x32
    eight-coil volume."""
    import torch
    from paper_2005_08661_gb300 import FieldMap
    from synth import full8_small_config
    fname, desc = TTC_CASES[case]
    path = os.path.join(ROOT, "tests", "golden", fname)
    if not os.path.exists(path):
        return None
    gold = json.load(open(path))
    target = gold["final_cost"] * (1 + 1e-6)
    vol = make_workload("small") if case == "small" else full8_small_config()
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    dev = torch.device("cuda", torch.cuda.current_device())
    y = torch.from_numpy(vol.y).to(dev).to(cd)
    s = torch.from_numpy(vol.smap).to(dev).to(cd) if vol.smap is not None else None
    m = torch.from_numpy(vol.mask).to(dev)
    fm = FieldMap(vol.nx, vol.ny, vol.nz, vol.ncoil, vol.necho, precision=prec, stream=stream)
    fm.set_data(y, s, vol.te, m, vol.beta)
    nmax = gold["niter"]
    _, cost = fm.solve(niter=nmax)
    hit = [i for i, c in enumerate(cost) if c <= target]
    if not hit:
        fm.close()
        return {"reached": False, "target": target, "final_cost": float(cost[-1])}
    i_star = hit[0]
    w = fm.empty()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        fm.set_data(y, s, vol.te, m, vol.beta)
        fm.solve_into(w, True, i_star)
    ts = []
    for _ in range(5):
        e0.record(stream)
        fm.set_data(y, s, vol.te, m, vol.beta)
        fm.solve_into(w, True, i_star)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1000.0)
    fm.close()
    return {"workload": desc, "precision": prec, "iterations": i_star, "seconds": statistics.median(ts),
            "oracle_cost": gold["final_cost"], "final_cost_rel": abs(cost[-1] - gold["final_cost"]) /
            abs(gold["final_cost"]), "target_rel": 1e-6}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="full")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--curvature", choices=["literal", "combined"], default="literal",
                    help="Huber curvature over every (c, d, m, n) term (the paper's) or from the "
                         "coil-combined pair weights (labelled variant, HBM-bound)")
    ap.add_argument("--niter", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttc", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave out the short runs of the batched, water-fat, differentiation and preconditioner "
                         "forms that the default line reports beside the main figures")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        if args.workload == "batch":
            return run_batch(args, world, rank, local)
        if args.workload == "diff":
            return run_diff(args, world, rank, local)
        if args.workload == "precond":
            return run_precond(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
