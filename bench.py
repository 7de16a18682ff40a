#!/usr/bin/env python3
"""Benchmark of the SU(Nc) chessboard link sweep on GB300.

Workload (the configuration the %-of-HBM metric is quoted on): SU(3) on a
48^3 x 96 lattice, beta = 6.2, cold start, sweeps of 1 heatbath + 5
overrelaxation steps (each step = 8 chessboard passes), FP32 links in two-row
(12-real) storage, FP64 reunitarization of every link once per sweep (inside
the update kernels of the sweep's last step), plaquette and Polyakov loop
measured after every sweep.  One benchmark step = one such sweep (the whole
hot path).

  value      link updates/s, device-resident lattice (2.0 GB, larger than L2),
             CUDA events on the lattice's stream, max over ranks
  e2e        the same metric through the C ABI with host buffers: every step
             imports the configuration from pinned host memory (compact
             format: the stored rows in FP32, 2.04 GB), sweeps, reads the
             observables and exports the configuration back
  roofline   the dominant kernel (overrelaxation pass): algorithmic bytes
             (8 link reads + 1 link write per update) / measured launch time
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload

--impl reference times the CPU oracle alone on the same workload and metric.
Multi-GPU: independent replicas (one lattice per rank), weak scaling.

--workload batched: 64 independent SU(3) chains, L drawn from {8,12,16,24},
beta uniform in [5.6, 6.4], Haar start, 50 sweeps (1 heatbath + 4
overrelaxation) of every chain per step, all chains in one batch (a captured
CUDA graph per batch sweep), against the same chains run one at a time.
--workload serving: a Poisson request trace (mean 20/s) of SU(Nc) chains,
Nc in {2,3,4,6}, L in {8..24}, 20..200 sweeps each, served by continuous
batching under a device-memory budget, against the same trace served one
request at a time; p50/p99 latency and throughput.
"""
import argparse
import hashlib
import glob
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NC, DIMS, BETA = 3, (48, 48, 48, 96), 6.2
N_HB, N_OR = 1, 5
METRIC = "link updates/s"
WORKLOAD_NAME = "SU(3) 48^3x96 beta=6.2 cold start, sweeps of 1 heatbath + 5 overrelaxation, FP32 links"


def volume(d):
    return d[0] * d[1] * d[2] * d[3]


def workload_config(world):
    """The workload both arms (this one and --impl reference) are measured on."""
    return {"workload": WORKLOAD_NAME, "nc": NC, "dims": list(DIMS), "beta": BETA, "start": "cold",
            "n_heatbath": N_HB, "n_overrelax": N_OR, "link_updates_per_step": updates_per_sweep(),
            "reunitarize": "FP64, every link once per sweep",
            "observables": "FP64 plaquette + Polyakov every sweep",
            "l2": "lattice (2.0 GB two-row FP32) larger than L2, no flush", "parallelism": f"replicas x{world}"}


def updates_per_sweep():
    return (N_HB + N_OR) * 4 * volume(DIMS)


def source_digest():
    """Digest of what defines the SU(3) update kernels' code: the device headers, the
    SU(3) instantiation units and the compiler flags (host-only sources excluded)."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1112_4533_gb300")
    files = [os.path.join(pkg, "csrc", n) for n in ("sun_device.cuh", "sun_kernels.cuh", "sun_runtime.h")]
    files += sorted(glob.glob(os.path.join(pkg, "csrc", "ops_su3*.cu"))) + [os.path.join(pkg, "build.py")]
    for p in files:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag):
    """dram bytes per launch from a committed ncu summary, if it was taken on the current sources."""
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read()
        m_k = re.search(r"^roofline_kernel:\s*(\S+)", text, re.M)
        m_t = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
        m_d = re.search(r"^source_digest:\s*(\S+)", text, re.M)
        if m_k and m_t and m_d and m_k.group(1) == kernel_tag:
            if m_d.group(1) == source_digest():
                return float(m_t.group(1))
            return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_selector(local):
    """nvidia-smi -i argument for this process's GPU (UUID, which ignores CUDA_VISIBLE_DEVICES remapping)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- CPU oracle ----

def oracle_sample(target_seconds=12.0, threads=None, max_slices=24):
    """Time the FP64 CPU oracle on a bounded sample of the workload: heatbath and
    overrelaxation passes over the first time slices of the cold 48^3 x 96
    lattice, each kind repeated over (direction, parity) for about half of
    target_seconds, rates combined 1:5 as in a sweep.  Returns (updates/s, cores, desc)."""
    import numpy as np
    import oracle as orc

    cores = orc.set_threads(threads or os.cpu_count() or 1)
    nx, ny, nz, nt = DIMS
    n_slab = max(1, min(max_slices, nt - 2))
    U = np.zeros((4, nt, nz, ny, nx, NC, NC), dtype=np.complex128)  # pages touched lazily
    for t in list(range(0, n_slab + 1)) + [nt - 1]:  # cold start on the slices the slab reads
        for a in range(NC):
            U[:, t, :, :, :, a, a] = 1.0
    per_pass = nx * ny * nz // 2 * n_slab

    def rate(mode, budget):
        n, t_used, k = 0, 0.0, 0
        while t_used < budget or k == 0:
            mu, par = (k // 2) % 4, k % 2
            t0 = time.perf_counter()
            orc.update_pass(U, BETA, mode, mu, par, 0, 1, 0, n_slab)
            t_used += time.perf_counter() - t0
            n += per_pass
            k += 1
        return n / t_used, n, t_used

    r_hb, n_hb, t_hb = rate(orc.HEATBATH, target_seconds / 2)
    r_or, n_or, t_or = rate(orc.OVERRELAX, target_seconds / 2)
    r = (N_HB + N_OR) / (N_HB / r_hb + N_OR / r_or)
    desc = (f"heatbath and overrelaxation passes over time slices [0,{n_slab}) of the cold 48^3x96 "
            f"lattice ({per_pass} link updates per pass): {n_hb} heatbath updates in {t_hb:.1f} s, "
            f"{n_or} overrelaxation updates in {t_or:.1f} s, rates combined 1:5 as in a sweep")
    return r, cores, desc


def oracle_input(threads=None):
    """The 48^3 x 96 configuration the oracle leg starts from, made by the oracle
    alone: a 16^3 x 32 lattice thermalised from a cold start (six sweeps of
    1 heatbath + 4 overrelaxation at beta 6.2), tiled 3 x 3 x 3 x 3 (a periodic
    configuration of the large lattice whose neighbourhoods are the small
    one's).  Returned in canonical order, complex128."""
    import numpy as np
    import oracle as orc

    orc.set_threads(threads or os.cpu_count() or 1)
    tile = (16, 16, 16, 32)
    U = orc.init(NC, tile, False, 13)
    for s in range(6):
        orc.sweep(U, BETA, 1, 4, True, 13, s)
    reps = tuple(d // t for d, t in zip(DIMS, tile))
    return np.tile(U, (1, reps[3], reps[2], reps[1], reps[0], 1, 1))


def oracle_leg(L, n_doubles, target_seconds=12.0, max_slices=24):
    """The CPU baseline with the agreement of the two stated.  The oracle makes
    its own thermalised 48^3 x 96 configuration (oracle_input); the GPU lattice
    is loaded with it (after the timed sweeps), and both measure its plaquette
    and Polyakov loop.  Then one heatbath pass and one overrelaxation pass:
    the GPU on the whole lattice, the oracle on the first time slices (same
    input, same Philox counters), each oracle pass timed (rates combined 1:5
    as in a sweep); the second pass starts from the oracle's result of the
    first.  Returns the cpu_baseline dict with an "agreement" entry."""
    import numpy as np
    import torch
    import oracle as orc
    import paper_1112_4533_gb300 as sun

    cores = orc.set_threads(os.cpu_count() or 1)
    nx, ny, nz, nt = DIMS
    shape = (4, nt, nz, ny, nx, NC, NC)
    t0 = time.perf_counter()
    U = oracle_input()
    t_input = time.perf_counter() - t0
    a = torch.empty(n_doubles, dtype=torch.float64).pin_memory()
    b = torch.empty(n_doubles, dtype=torch.float64).pin_memory()
    A = a.numpy().view(np.complex128).reshape(shape)
    B = b.numpy().view(np.complex128).reshape(shape)
    A[...] = U
    del U
    L.import_links_raw(a.data_ptr(), n_doubles)
    p_gpu = L.plaquette()
    l_gpu = L.polyakov_loop()
    t0 = time.perf_counter()
    p_orc = orc.plaquette(A)
    t_plaq = time.perf_counter() - t0
    l_orc = complex(orc.polyakov(A))
    step = 7
    L.heatbath_step = step
    n_slab = max(1, min(max_slices, nt - 2))
    per_pass = nx * ny * nz // 2 * n_slab

    def slab_diff(X, Y):
        return np.abs(X[:, :n_slab] - Y[:, :n_slab]).reshape(4, n_slab, -1, NC * NC).max(axis=-1)

    # heatbath pass (mu 1, even): GPU on the whole lattice, oracle on the slab
    L.update_pass(sun.HEATBATH, 1, 0)
    L.export_links_raw(b.data_ptr(), n_doubles)
    n_hb, t_hb = 0, 0.0
    t0 = time.perf_counter()
    orc.update_pass(A, BETA, orc.HEATBATH, 1, 0, step, 1, 0, n_slab)
    t_hb += time.perf_counter() - t0
    n_hb += per_pass
    d = slab_diff(A, B)
    flips = int((d > 1e-5).sum())
    hb_err = float(d[d <= 1e-5].max())
    # overrelaxation pass (mu 2, odd), both from the oracle's post-heatbath links
    L.import_links_raw(a.data_ptr(), n_doubles)
    L.update_pass(sun.OVERRELAX, 2, 1)
    L.export_links_raw(b.data_ptr(), n_doubles)
    t0 = time.perf_counter()
    orc.update_pass(A, BETA, orc.OVERRELAX, 2, 1, step, 1, 0, n_slab)
    t_or = time.perf_counter() - t0
    n_or = per_pass
    or_err = float(slab_diff(A, B).max())
    # more passes of each kind on the slab for a steadier rate (results not compared)
    k = 0
    while t_hb + t_or < target_seconds and k < 64:
        mu, par = (k // 2) % 4, k % 2
        t0 = time.perf_counter()
        orc.update_pass(A, BETA, orc.HEATBATH if k % 2 == 0 else orc.OVERRELAX, mu, par, step + 1, 1, 0, n_slab)
        if k % 2 == 0:
            t_hb += time.perf_counter() - t0
            n_hb += per_pass
        else:
            t_or += time.perf_counter() - t0
            n_or += per_pass
        k += 1
    r_hb, r_or = n_hb / t_hb, n_or / t_or
    r = (N_HB + N_OR) / (N_HB / r_hb + N_OR / r_or)
    desc = (f"FP64 oracle on its own thermalised 48^3x96 configuration (16^3x32, six sweeps from a cold start, "
            f"tiled 3x3x3x3; made in {t_input:.1f} s): heatbath and overrelaxation passes over time slices "
            f"[0,{n_slab}) ({per_pass} link updates per pass), {n_hb} heatbath updates in {t_hb:.1f} s, {n_or} "
            f"overrelaxation updates in {t_or:.1f} s, rates combined 1:5 as in a sweep; plaquette of the whole "
            f"lattice in {t_plaq:.1f} s")
    agreement = {
        "plaquette": {"gpu": p_gpu, "oracle": p_orc, "abs_err": abs(p_gpu - p_orc)},
        "polyakov": {"gpu": [l_gpu.real, l_gpu.imag], "oracle": [l_orc.real, l_orc.imag],
                     "abs_err": abs(l_gpu - l_orc)},
        "overrelaxation_pass": {"links": 4 * per_pass, "max_abs_err": or_err, "bound": 1e-5},
        "heatbath_pass": {"links": 4 * per_pass, "max_abs_err_where_branches_agree": hb_err,
                          "branch_flips": flips, "bound": "1e-5, flips <= 1e-6 of updates"},
        "note": "the GPU lattice loaded with the oracle's configuration; one pass from the same input; links of all "
                "four directions on the slab compared (only direction 1 / 2 changes)",
    }
    del A, B, a, b
    return {"value": r, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": desc,
            "plaquette_s": t_plaq, "agreement": agreement}


# ---------------------------------------------------------------- GPU arm ----

def dist_init(n_gpus):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    """Max of x over the ranks (the per-rank times of the timed region)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, ms_local, world):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    ms = allreduce_max(ms_local, world)
    return units_per_rank * world / (ms / 1e3), ms


def time_kernel(L, reps):
    """Average duration of one overrelaxation pass, CUDA events on the lattice's stream."""
    import torch
    import paper_1112_4533_gb300 as sun
    evs = []
    for r in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        mu, par = (r // 2) % 4, r % 2
        a.record(L.stream)
        L.update_pass(sun.OVERRELAX, mu, par)
        b.record(L.stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / reps


def time_pass(L, reps, heatbath=False):
    """Average duration of one pass of the given kind, CUDA events on the lattice's stream."""
    import torch
    import paper_1112_4533_gb300 as sun
    evs = []
    for r in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        mu, par = (r // 2) % 4, r % 2
        a.record(L.stream)
        L.update_pass(sun.HEATBATH if heatbath else sun.OVERRELAX, mu, par)
        b.record(L.stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / reps


def run_sweeps(L, steps):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(L.stream)
    plaq, poly = L.run(steps, N_HB, N_OR)
    b.record(L.stream)
    b.synchronize()
    return a.elapsed_time(b), plaq, poly


def gpu_arm(args):
    import torch
    import paper_1112_4533_gb300 as sun

    rank, world, local = dist_init(args.gpus)
    K, W = args.steps, args.warmup
    V = volume(DIMS)
    hbm_peak, peak_kind = measured_peaks()

    # ---- headline: FP32; kernel shape, storage format and re-unitarization
    # placement measured by the library's autotuner (outside the timed region)
    tuned = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tuned = sun.autotune(NC, DIMS, BETA, N_HB, N_OR, precision=32, storage=args.storage,
                             reunit_mode=args.reunit_mode, tune_storage=True, tune_reunit_mode=True, two_row=True)
        tuned["tuning_s"] = time.perf_counter() - t0
        args.storage, args.variant, args.reunit_mode = tuned["storage"], tuned["variant"], tuned["reunit_mode"]
        args.block, args.graph_sweeps = tuned["block_threads"], tuned["graph_sweeps"]
    kw = dict(precision=32, reunit_mode=args.reunit_mode, variant=args.variant, block_threads=args.block,
              graph_sweeps=args.graph_sweeps)
    L = sun.Lattice(NC, DIMS, BETA, hot_start=False, seed=1 + rank, storage=args.storage, **kw)
    L.run(W, N_HB, N_OR)
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    ms, plaq, poly = run_sweeps(L, K)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    value, ms_max = aggregate_rate(updates_per_sweep() * K, ms, world)

    # ---- dominant kernel, timed alone (events around each launch)
    k_ms = time_kernel(L, 32)
    link_bytes = L.link_bytes
    alg_bytes = (V // 2) * 9 * link_bytes
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    kernel_tag = f"or_pass_su3_{args.storage}real_fp32_48x48x48x96"
    traffic = profiled_traffic(kernel_tag)

    # ---- the other storage format, and the two-row staple products (variant bit 2)
    variants = {}
    if not args.no_variants:
        L.close()
        del L
        torch.cuda.empty_cache()
        alt = 18 if args.storage == 12 else 12
        other = "fp32_12real_full_staple" if args.variant & 2 else "fp32_12real_two_row_staple"
        for name, st, var in [(f"fp32_{alt}real", alt, args.variant & ~2),
                              (other, 12, (args.variant ^ 2) & ~8)]:
            if st == args.storage and var == args.variant:
                continue
            L2 = sun.Lattice(NC, DIMS, BETA, hot_start=False, seed=1 + rank, storage=st,
                             **dict(kw, variant=var))
            L2.run(max(1, W // 2), N_HB, N_OR)
            k2s = max(2, K // 2)
            ms2, _, _ = run_sweeps(L2, k2s)
            k2 = time_kernel(L2, 16)
            variants[name] = {
                "value": updates_per_sweep() * k2s / (ms2 / 1e3), "unit": METRIC, "storage_reals": st,
                "variant": var, "ms_per_step": ms2 / k2s, "or_pass_ms": k2,
                "or_pass_gbs": (V // 2) * 9 * L2.link_bytes / (k2 / 1e3) / 1e9}
            if var & 2:
                variants[name]["note"] = ("third row of each staple term taken as conj(row0 x row1), exact for "
                                          "SU(3) products; within 1e-5 of the oracle on thermalised links")
            else:
                variants[name]["note"] = "every staple term multiplied out in full (all three rows)"
            L2.close()
            del L2
            torch.cuda.empty_cache()
        L = sun.Lattice(NC, DIMS, BETA, hot_start=False, seed=1 + rank, storage=args.storage, **kw)

    # ---- end to end through the C ABI with pinned host buffers: every step the
    # configuration comes from and goes back to host memory in the compact format
    # (the stored rows in FP32, as configuration files hold them)
    e2e = None
    if not args.no_e2e:
        nbytes = L.links_bytes
        host_a = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        host_b = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        L.export_stored_raw(host_a.data_ptr(), nbytes)
        ke = max(2, min(K, args.e2e_steps))
        for _ in range(1):
            L.import_stored_raw(host_a.data_ptr(), nbytes)
            L.run(1, N_HB, N_OR)
            L.export_stored_raw(host_b.data_ptr(), nbytes)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(ke):
            src, dst = (host_a, host_b) if s % 2 == 0 else (host_b, host_a)
            L.import_stored_raw(src.data_ptr(), nbytes)
            L.run(1, N_HB, N_OR)
            L.export_stored_raw(dst.data_ptr(), nbytes)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = allreduce_max(dt, world)
        e2e = {"value": updates_per_sweep() * ke * world / dt, "unit": METRIC,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 3 * 8,
               "steps": ke, "ms_per_step": dt / ke * 1e3,
               "path": "sun_import_stored + sun_run(1 sweep, observables to host) + sun_export_stored: the "
                       "configuration in pinned host memory in the compact format (stored rows, FP32)"}
        del host_a, host_b

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_leg(L, 8 * NC * NC * V, args.cpu_seconds)

    L.close()
    del L
    torch.cuda.empty_cache()
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        for name, fn in [("c1_su2_8x8x8x8_fp64", lambda: measure_c1(local)),
                         ("c2_su3_16x16x16x16_fp32", lambda: measure_c2(local)),
                         ("su4_32x32x32x32_fp32", lambda: measure_su4(local, hbm_peak)),
                         ("c4_batched_64_chains", lambda: measure_batched(local, steps=3)),
                         ("c5_serving", lambda: measure_serving(local, n_requests=args.requests,
                                                                budget_gb=args.budget_gb,
                                                                work_cap_ms=args.work_cap_ms,
                                                                low_latency_cap_ms=args.low_latency_cap_ms))]:
            t0 = time.perf_counter()
            extra[name] = fn()
            extra[name]["measure_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
    # kernels per sweep: the passes (8 per step, or 4 wavefront launches with bit 8), the separate
    # re-unitarization (placement 0 only), plaquette, Polyakov loop, step counter
    passes_per_step = 4 if (args.variant & 8) and not (args.variant & 18) else 8
    launches_per_sweep = (N_HB + N_OR) * passes_per_step + (1 if args.reunit_mode == 0 else 0) + 3
    out = {
        "metric": METRIC,
        "value": value,
        "unit": METRIC,
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (cold start, Philox seed 1 + rank)",
        "config": workload_config(world),
        "kernel_config": {"storage_reals": args.storage, "kernel_variant": args.variant, "block_threads": args.block,
                          "graph_sweeps": args.graph_sweeps, "autotuned": tuned,
                          "reunit_placement": {0: "own pass after the sweep", 1: "in the update kernels of the last "
                                               "step", 2: "spread over the steps"}[args.reunit_mode]},
        "hbm_gbs_effective": updates_per_sweep() * 9 * link_bytes / (ms_max / K / 1e3) / 1e9,
        "plaquette_last": float(plaq[-1]),
        "polyakov_last": [float(poly[-1].real), float(poly[-1].imag)],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "kernel": ("overrelaxation pass, SU(3) FP32 %d-real, kernel variant %d, one thread per link"
                                % (args.storage, args.variant)),
                     "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": k_ms,
                     "peak_kind": peak_kind + " (hbm_gbs, copy kernel)"},
        "variants": variants,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches_per_sweep * K,
        "workloads": extra,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------- the other workloads ----
# C1, C2 (single chains shaped like the paper's runs), C4 (64 chains batched)
# and C5 (served request stream), measured in the default run beside the
# headline, each with CUDA-event timing and its own clock record.

def _timed(stream, fn):
    """Run fn() between two CUDA events on stream; returns (ms, fn's result)."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b), r


def measure_c1(local, reps=20):
    """SU(2) 8^4, beta 2.3, cold start, 10 sweeps of 1 heatbath + 4
    overrelaxation, FP64 quaternion links, Philox seed 1, plaquette after every
    sweep (the sweep re-unitarizes).  One run = the 10 sweeps from the cold
    start; its plaquette history is compared with the FP64 oracle's, both
    free-running and sweep by sweep from the oracle's links."""
    import numpy as np
    import oracle as orc
    import paper_1112_4533_gb300 as sun

    dims, beta, sweeps = (8, 8, 8, 8), 2.3, 10
    L = sun.Lattice(2, dims, beta, hot_start=False, seed=1, precision=64, storage=4, graph_sweeps=sweeps)
    cold = L.export_stored()
    upd = sweeps * 5 * 4 * volume(dims)

    def one_run():
        L.import_stored(cold)
        L.heatbath_step = 0
        return _timed(L.stream, lambda: L.run(sweeps, 1, 4))

    for _ in range(3):
        one_run()
    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    total, hist = 0.0, None
    for _ in range(reps):
        ms, (plaq, _) = one_run()
        total += ms
        hist = plaq
    clocks = sampler.stop()
    # the oracle's chain, and each GPU sweep from the oracle's links
    U = orc.init(2, dims, False, 1)
    o_hist, same = [], []
    for s in range(sweeps):
        L.import_links(U)
        L.heatbath_step = s
        p1, _ = L.run(1, 1, 4)
        got = L.export_links()
        orc.sweep(U, beta, 1, 4, True, 1, s)
        o_hist.append(orc.plaquette(U))
        same.append((abs(p1[0] - o_hist[-1]), float(np.abs(got - U).max())))
    L.close()
    o_hist = np.array(o_hist)
    return {"metric": METRIC, "value": upd * reps / (total / 1e3), "unit": METRIC, "ms_per_run": total / reps,
            "runs": reps, "link_updates_per_run": upd, "dtype": "f64",
            "workload": "SU(2) 8^4 beta=2.3 cold start, 10 sweeps of 1 heatbath + 4 overrelaxation (re-unitarized), "
                        "FP64 quaternion links, Philox seed 1, plaquette after each sweep",
            "bound": "L2-resident (512 KiB of links): launch and latency bound",
            "plaquette_history": [float(x) for x in hist],
            "oracle_plaquette_history": [float(x) for x in o_hist],
            "agreement": {
                "same_input_max_abs_err_plaquette": max(a for a, _ in same),
                "same_input_max_abs_err_links": max(b for _, b in same),
                "free_running_abs_err_per_sweep": [float(x) for x in np.abs(hist - o_hist)],
                "note": "same input: before each sweep the GPU lattice holds the oracle's links and heatbath step; "
                        "free running: both chains from the cold start (rounding-order differences grow ~30x per "
                        "sweep)"},
            "clocks": clocks}


def measure_c2(local, reps=3):
    """SU(3) 16^4, beta 6.0, Haar start (seed 2), 200 sweeps of 1 heatbath + 4
    overrelaxation, FP32 two-row links, FP64 re-unitarization every sweep and
    FP64 plaquette after every sweep; the re-unitarization placement and kernel
    shape measured by the autotuner.  Agreement: the first sweep from the
    oracle's Haar start against the oracle's sweep."""
    import numpy as np
    import oracle as orc
    import paper_1112_4533_gb300 as sun

    dims, beta, sweeps = (16, 16, 16, 16), 6.0, 200
    t = sun.autotune(3, dims, beta, 1, 4, precision=32, storage=12, reunit_mode=1, tune_storage=False,
                     tune_reunit_mode=True)
    kw = dict(precision=32, storage=12, variant=t["variant"], reunit_mode=t["reunit_mode"],
              block_threads=t["block_threads"], graph_sweeps=t["graph_sweeps"])
    L = sun.Lattice(3, dims, beta, hot_start=True, seed=2, **kw)
    hot = L.export_stored()
    upd = sweeps * 5 * 4 * volume(dims)

    def one_run():
        L.import_stored(hot)
        L.heatbath_step = 0
        return _timed(L.stream, lambda: L.run(sweeps, 1, 4, polyakov=False))

    one_run()
    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    total, hist = 0.0, None
    for _ in range(reps):
        ms, (plaq, _) = one_run()
        total += ms
        hist = plaq
    clocks = sampler.stop()
    # agreement with the oracle from its own Haar start: one heatbath and one
    # overrelaxation pass link by link, and the plaquette after one sweep
    U = orc.init(3, dims, True, 2)
    passes = {}
    for name, mode, mu, par in [("heatbath_pass", orc.HEATBATH, 0, 0), ("overrelaxation_pass", orc.OVERRELAX, 3, 1)]:
        L.import_links(U)
        L.heatbath_step = 0
        L.update_pass(mode, mu, par)
        got = L.export_links()
        want = U.copy()
        orc.update_pass(want, beta, mode, mu, par, 0, 2)
        d = np.abs(got - want).reshape(-1, 9).max(axis=1)
        passes[name] = {"max_abs_err": float(d.max()), "links_above_1e-5": int((d > 1e-5).sum()),
                        "links": int(d.size)}
    L.import_links(U)
    L.heatbath_step = 0
    p1, _ = L.run(1, 1, 4, polyakov=False)
    L.close()
    orc.sweep(U, beta, 1, 4, {0: True, 1: orc.REUNIT_FUSED, 2: orc.REUNIT_SPREAD}[kw["reunit_mode"]], 2, 0)
    tail = hist[100:]
    bins = tail.reshape(10, -1).mean(axis=1)
    return {"metric": METRIC, "value": upd * reps / (total / 1e3), "unit": METRIC, "ms_per_run": total / reps,
            "ms_per_sweep": total / reps / sweeps, "runs": reps, "link_updates_per_run": upd, "dtype": "f32",
            "workload": "SU(3) 16^4 beta=6.0 Haar start (seed 2), 200 sweeps of 1 heatbath + 4 overrelaxation, FP32 "
                        "two-row links, FP64 re-unitarization every sweep, FP64 plaquette after each sweep",
            "bound": "L2-resident (12 MiB of links)", "kernel_config": t,
            "plaquette": {"first": float(hist[0]), "last": float(hist[-1]),
                          "mean_sweeps_100_199": float(tail.mean()),
                          "binned_err": float(bins.std(ddof=1) / np.sqrt(len(bins)))},
            "agreement": dict(passes, first_sweep_abs_err_plaquette=abs(float(p1[0]) - orc.plaquette(U)),
                              note="from the oracle's Haar start: one pass of each kind link by link (a Haar start "
                                   "has nearly cancelling staples, where FP32 rounding is amplified by 1/k); the "
                                   "plaquette after one sweep (overrelaxation conserves the action, so it stays "
                                   "comparable while chained FP32 passes on such a start decorrelate the links "
                                   "themselves)"),
            "clocks": clocks}


def measure_su4(local, hbm_peak, sweeps=10):
    """SU(4) 32^4, beta 11.2 (0.7 Nc^2), Haar start, FP32 full storage, sweeps of
    1 heatbath + 4 overrelaxation with re-unitarization and observables, for the
    kernels the library has for Nc = 4: one thread per link with every loop over
    rows, columns and the six subgroups unrolled at compile time (variant 0),
    the same bounded to 128 registers (variant 1), and the row-parallel kernel
    shared with the generic SU(Nc) path (Nc threads per link, variant 4).  Each
    with its sweep rate and its passes' time and algorithmic HBM fraction (9
    link-sizes of 128 bytes per update)."""
    import paper_1112_4533_gb300 as sun

    dims, beta = (32, 32, 32, 32), 11.2
    V = volume(dims)
    upd = sweeps * 5 * 4 * V
    out = {}
    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    for name, var in [("per_link", 0), ("per_link_128_registers", 1), ("row_parallel", 4)]:
        L = sun.Lattice(4, dims, beta, hot_start=True, seed=4, precision=32, variant=var)
        L.run(1, 1, 4)
        ms, _ = _timed(L.stream, lambda: L.run(sweeps, 1, 4))
        alg = (V // 2) * 9 * L.link_bytes
        t_or = time_kernel(L, 16)
        t_hb = time_pass(L, 8, heatbath=True)
        L.close()
        out[name] = {"variant": var, "value": upd / (ms / 1e3), "unit": METRIC, "ms_per_sweep": ms / sweeps,
                     "or_pass_ms": t_or, "or_pass_hbm_frac": alg / (t_or / 1e3) / 1e9 / hbm_peak,
                     "hb_pass_ms": t_hb, "hb_pass_hbm_frac": alg / (t_hb / 1e3) / 1e9 / hbm_peak}
    clocks = sampler.stop()
    best = max(out, key=lambda k: out[k]["value"])
    return {"metric": METRIC, "value": out[best]["value"], "unit": METRIC, "kernel": best, "dtype": "f32",
            "workload": "SU(4) 32^4 beta=11.2 Haar start, sweeps of 1 heatbath + 4 overrelaxation, FP32 links, "
                        "FP64 re-unitarization and observables every sweep",
            "kernels": out, "clocks": clocks,
            "note": "per_link is the SU(4)-specialised kernel (compile-time Nc = 4); row_parallel is the generic "
                    "SU(Nc) mapping the paper's comparison of optimised SU(4) with generic SU(Nc) code refers to"}


def c4_chains():
    import numpy as np
    rng = np.random.default_rng(4)
    Ls = rng.choice([8, 12, 16, 24], size=64)
    betas = rng.uniform(5.6, 6.4, size=64)
    return [int(x) for x in Ls], [float(b) for b in betas]


def measure_batched(local, steps=3, tune=True, opts=None):
    """C4: 64 SU(3) chains, L drawn from {8,12,16,24}, beta uniform in
    [5.6, 6.4], Haar starts (seeds 100..163), 50 sweeps of 1 heatbath + 4
    overrelaxation each, FP32 update / FP64 re-unitarization, the shared kernel
    configuration measured by the autotuner.  All 50 sweeps of all 64 chains
    are one launch of a captured CUDA graph (per-pass kernels over all chains
    of the group).  Plain path: the same chains one at a time, sun_run of 50
    sweeps each (one graph launch per chain), same kernels.  Both timed with
    CUDA events on one stream, after an untimed run of each."""
    import numpy as np
    import torch
    import paper_1112_4533_gb300 as sun

    Ls, betas = c4_chains()
    sweeps = 50
    tuned = None
    o = dict(storage=12, variant=1, reunit_mode=1, block_threads=0)
    if opts:
        o.update(opts)
    if tune:
        t0 = time.perf_counter()
        tuned = sun.autotune_batch([(3, (L,) * 4, b) for L, b in zip(Ls, betas)], 1, 4, precision=32,
                                   storage=o["storage"], reunit_mode=o["reunit_mode"], tune_storage=True,
                                   tune_reunit_mode=True, two_row=True)
        tuned["tuning_s"] = time.perf_counter() - t0
        o.update({k: tuned[k] for k in ("storage", "variant", "reunit_mode", "block_threads")})
    kw = dict(precision=32, graph_sweeps=sweeps, **o)
    stream = torch.cuda.Stream()
    lats = [sun.Lattice(3, (L,) * 4, b, hot_start=True, seed=100 + i, stream=stream, **kw)
            for i, (L, b) in enumerate(zip(Ls, betas))]
    starts = [L.export_stored() for L in lats]

    def reset():
        for L, h in zip(lats, starts):
            L.import_stored(h)
            L.heatbath_step = 0

    updates = sum(5 * 4 * L ** 4 for L in Ls) * sweeps
    B = sun.Batch(lats, stream=stream, use_graphs=True)
    reset()
    B.run(sweeps, 1, 4)  # captures the 50-sweep graph
    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    tb = []
    for _ in range(steps):
        reset()
        ms, (plaq_b, _) = _timed(stream, lambda: B.run(sweeps, 1, 4))
        tb.append(ms)
    clocks = sampler.stop()
    B.close()
    # plain: each chain alone
    reset()
    for L in lats:
        L.run(sweeps, 1, 4)  # captures each chain's 50-sweep graph

    def plain():
        return [L.run(sweeps, 1, 4)[0] for L in lats]

    sampler = ClockSampler(gpu_selector(local))
    sampler.start()
    tp = []
    for _ in range(steps):
        reset()
        ms, plaq_p = _timed(stream, plain)
        tp.append(ms)
    clocks_p = sampler.stop()
    for L in lats:
        L.close()
    # links evolve bitwise as alone; the batch sums each chain's plaquette in its
    # own fixed order, so the histories agree to rounding
    hist_diff = max(float(np.abs(plaq_b[:, i] - plaq_p[i]).max()) for i in range(len(lats)))
    mb, mp = min(tb), min(tp)
    return {"metric": "chains/s", "value": 64 / (mb / 1e3), "unit": "chains/s", "ms_per_step": mb,
            "steps": steps, "link_updates_per_s": updates / (mb / 1e3), "link_updates_per_step": updates,
            "dtype": "f32",
            "workload": "64 SU(3) chains, L in {8,12,16,24} (seeded draw), beta U[5.6,6.4], Haar start, 50 sweeps of "
                        "1 heatbath + 4 overrelaxation each, FP32 links, FP64 re-unitarization every sweep",
            "L_counts": {str(v): Ls.count(v) for v in (8, 12, 16, 24)},
            "kernel_config": dict(o, graph_sweeps=sweeps, autotuned=tuned),
            "launch": "all 50 sweeps of all 64 chains: one launch of one captured CUDA graph",
            "plain": {"value": 64 / (mp / 1e3), "unit": "chains/s", "ms_per_step": mp,
                      "link_updates_per_s": updates / (mp / 1e3), "clocks": clocks_p,
                      "path": "each chain alone: sun_run of 50 sweeps (one graph launch per chain), same kernels"},
            "speedup_vs_plain": mp / mb,
            "plaquette_histories_max_abs_diff_vs_plain": hist_diff,
            "clocks": clocks}


def measure_serving(local, n_requests=80, budget_gb=64.0, policy="srpt", tick_ms=40.0, work_cap_ms=8.0,
                    low_latency_cap_ms=3.0, sweeps_per_tick=None, use_graphs=True):
    """C5: a Poisson request trace (mean 20/s, seed 7) of SU(Nc) chains, Nc in
    {2,3,4,6}, L in {8..24}, 20..200 sweeps each, served by continuous batching
    under a device-memory budget, with the server's per-Nc sweep costs measured
    on this GPU first.  Two server settings: "served" adds chains to a tick
    while one predicted sweep of the batch stays within work_cap_ms (fuller
    launches, for throughput), "served_low_latency" within low_latency_cap_ms
    (finer shortest-first scheduling).  Against the same trace served one
    request at a time, in arrival order (FIFO) and shortest request first
    (SRPT), so that the scheduling gain and the batching gain show separately.
    Each path's wall time is the interval between two CUDA events on the
    default stream around the whole trace (the server synchronises after
    every tick)."""
    import torch
    from paper_1112_4533_gb300 import serve

    trace = serve.poisson_trace(n_requests, rate=20.0, seed=7)
    budget = int(budget_gb * (1 << 30))
    warm = serve.poisson_trace(4, rate=50.0, seed=99, Ls=(8,), sweeps=(2, 3))
    serve.Server(budget).run(warm)
    serve.serve_plain(warm)
    costs = serve.measure_sweep_costs()
    upd = sum(r.n_sweeps * 5 * 4 * r.L ** 4 for r in trace)
    stream = torch.cuda.current_stream()

    servers = {}

    def server(cap, key):
        def run():
            servers[key] = serve.Server(budget, sweeps_per_tick=sweeps_per_tick, work_cap_ms=cap, tick_ms=tick_ms,
                                        policy=policy, costs=costs, use_graphs=use_graphs)
            return servers[key].run(trace)
        return run

    runs = [("served", server(work_cap_ms, "served")), ("served_low_latency", server(low_latency_cap_ms, "served_low_latency")),
            ("plain_fifo", lambda: serve.serve_plain(trace, order="fifo", costs=costs)[0]),
            ("plain_srpt", lambda: serve.serve_plain(trace, order="srpt", costs=costs)[0])]
    out = {}
    for name, fn in runs:
        sampler = ClockSampler(gpu_selector(local))
        sampler.start()
        ms, res = _timed(stream, fn)
        clocks = sampler.stop()
        st = serve.latency_stats(res)
        out[name] = {"p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
                     "completed": st["completed"], "wall_s": ms / 1e3, "requests_per_s": len(trace) / (ms / 1e3),
                     "link_updates_per_s": upd / (ms / 1e3), "clocks": clocks}
        if name in servers:
            out[name]["ticks"] = servers[name].ticks
            out[name]["batches_built"] = servers[name].batches_built
    s, sl, pf, ps = out["served"], out["served_low_latency"], out["plain_fifo"], out["plain_srpt"]
    return {"metric": "requests/s", "value": s["requests_per_s"], "unit": "requests/s",
            "p50_s": s["p50_s"], "p99_s": s["p99_s"], "dtype": "f32",
            "workload": f"{n_requests} requests, Poisson mean 20/s (seed 7), Nc in {{2,3,4,6}}, L in "
                        "{8,12,16,20,24}, 20..200 sweeps of 1 heatbath + 4 overrelaxation, FP32 links",
            "server": {"hbm_budget_gb": budget_gb, "policy": policy, "tick_ms": tick_ms, "work_cap_ms": work_cap_ms,
                       "low_latency_work_cap_ms": low_latency_cap_ms,
                       "sweep_ms_per_site_measured": {str(k): v for k, v in costs.items()}},
            "link_updates": upd, "served": s, "served_low_latency": sl, "plain_fifo": pf, "plain_srpt": ps,
            "throughput_vs_plain_fifo": s["requests_per_s"] / pf["requests_per_s"],
            "throughput_vs_plain_srpt": s["requests_per_s"] / ps["requests_per_s"],
            "low_latency_throughput_vs_plain_srpt": sl["requests_per_s"] / ps["requests_per_s"],
            "note": "plain_fifo: one request at a time in arrival order; plain_srpt: one at a time, the arrived "
                    "request with the least work first (scheduling without batching); served: continuous batching"}


def batched_arm(args):
    """--workload batched: the C4 measurement alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    opts = None
    if args.no_tune:
        opts = dict(storage=args.storage, variant=args.variant, reunit_mode=args.reunit_mode,
                    block_threads=args.block)
    r = measure_batched(0, steps=max(1, args.steps), tune=not args.no_tune, opts=opts)
    out = {"metric": "batched chains/s", "value": r["value"], "unit": "chains/s", "n_gpus": 1,
           "steps": r["steps"], "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (Haar starts, seeds 100..163)",
           "config": {"workload": r["workload"], "L_counts": r["L_counts"],
                      "link_updates_per_step": r["link_updates_per_step"]},
           "gpu_launches": None, "clocks": r["clocks"], "batched": r}
    print(json.dumps(out))


def serving_arm(args):
    """--workload serving: the C5 measurement alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    r = measure_serving(0, n_requests=args.requests, budget_gb=args.budget_gb, policy=args.policy,
                        tick_ms=args.tick_ms, work_cap_ms=args.work_cap_ms,
                        low_latency_cap_ms=args.low_latency_cap_ms, sweeps_per_tick=args.sweeps_per_tick or None,
                        use_graphs=not args.serve_no_graphs)
    out = {"metric": "served requests/s", "value": r["value"], "unit": "requests/s", "n_gpus": 1, "steps": 1,
           "warmup": 1, "ms_per_step": r["served"]["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic Poisson trace (seed 7)",
           "config": {"workload": r["workload"]}, "gpu_launches": None, "clocks": r["served"]["clocks"],
           "serving": r}
    print(json.dumps(out))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    per = max(1.0, min(args.cpu_seconds, 150.0 / max(1, K + W)))
    for _ in range(W):
        oracle_sample(per / 4)
    rates, cores, desc = [], 1, ""
    t0 = time.perf_counter()
    for _ in range(K):
        r, cores, desc = oracle_sample(per)
        rates.append(r)
    dt = time.perf_counter() - t0
    value = sum(rates) / len(rates)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": K,
           "warmup": W, "ms_per_step": dt / K * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (cold start)",
           "config": workload_config(args.gpus),
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", type=int, default=12, choices=[12, 18])
    ap.add_argument("--variant", type=int, default=3, choices=range(32),
                    help="update-kernel variant bits (with --no-tune): 1 = 5 blocks/SM register bound, "
                         "2 = two-row staple products")
    ap.add_argument("--reunit-mode", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="seconds of oracle work in the cpu_baseline leg, and the cap of one --impl reference step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="fixed configuration from the flags, no autotuning")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the C1, C2, batched (C4) and serving (C5) measurements of the default run")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the update kernels (0 = 128)")
    ap.add_argument("--graph-sweeps", type=int, default=0, help="sweeps captured per CUDA graph (0 = 1)")
    ap.add_argument("--workload", choices=["single", "batched", "serving"], default="single")
    ap.add_argument("--requests", type=int, default=80)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--sweeps-per-tick", type=int, default=0, help="cap on sweeps per serving tick (0 = none)")
    ap.add_argument("--tick-ms", type=float, default=40.0, help="predicted GPU time a serving tick aims at")
    ap.add_argument("--policy", choices=["srpt", "fifo"], default="srpt")
    ap.add_argument("--work-cap-ms", type=float, default=8.0,
                    help="serving: predicted ms of one batch sweep up to which chains are added to a tick")
    ap.add_argument("--serve-no-graphs", action="store_true",
                    help="serving: batches launch their kernels directly instead of capturing CUDA graphs")
    ap.add_argument("--low-latency-cap-ms", type=float, default=3.0,
                    help="serving: the same for the second, low-latency server setting")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "serving":
        serving_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
