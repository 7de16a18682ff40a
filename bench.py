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


def oracle_leg(L, n_doubles, target_seconds=12.0, max_slices=24):
    """The CPU baseline on the GPU's own configuration, with the agreement of
    the two stated: the FP64 oracle measures the plaquette and Polyakov loop of
    the configuration the GPU holds after the timed sweeps, then repeats one
    heatbath pass and one overrelaxation pass of the GPU (same input, same
    Philox counters) on the first time slices, timing each (rates combined 1:5
    as in a sweep).  Returns the cpu_baseline dict with an "agreement" entry."""
    import numpy as np
    import torch
    import oracle as orc
    import paper_1112_4533_gb300 as sun

    cores = orc.set_threads(os.cpu_count() or 1)
    nx, ny, nz, nt = DIMS
    shape = (4, nt, nz, ny, nx, NC, NC)
    a = torch.empty(n_doubles, dtype=torch.float64).pin_memory()
    b = torch.empty(n_doubles, dtype=torch.float64).pin_memory()
    A = a.numpy().view(np.complex128).reshape(shape)
    B = b.numpy().view(np.complex128).reshape(shape)
    L.export_links_raw(a.data_ptr(), n_doubles)
    p_gpu = L.plaquette()
    l_gpu = L.polyakov_loop()
    t0 = time.perf_counter()
    p_orc = orc.plaquette(A)
    t_plaq = time.perf_counter() - t0
    l_orc = orc.polyakov(A)
    l_orc = complex(l_orc[0], l_orc[1]) if isinstance(l_orc, tuple) else complex(l_orc)
    step = L.heatbath_step
    n_slab = max(1, min(max_slices, nt - 2))
    per_pass = nx * ny * nz // 2 * n_slab

    def slab_diff(X, Y):
        d = np.abs(X[:, :n_slab] - Y[:, :n_slab]).reshape(4, n_slab, -1, NC * NC).max(axis=-1)
        return d

    # heatbath pass (mu 1, even) from A: GPU on the whole lattice, oracle on the slab
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
    # overrelaxation pass (mu 2, odd) from the GPU's post-heatbath state B
    L.update_pass(sun.OVERRELAX, 2, 1)
    L.export_links_raw(a.data_ptr(), n_doubles)
    t0 = time.perf_counter()
    orc.update_pass(B, BETA, orc.OVERRELAX, 2, 1, step, 1, 0, n_slab)
    t_or = time.perf_counter() - t0
    n_or = per_pass
    or_err = float(slab_diff(A, B).max())
    # more passes of each kind on the slab for a steadier rate (results not compared)
    k = 0
    while t_hb + t_or < target_seconds and k < 64:
        mu, par = (k // 2) % 4, k % 2
        t0 = time.perf_counter()
        orc.update_pass(B, BETA, orc.HEATBATH if k % 2 == 0 else orc.OVERRELAX, mu, par, step + 1, 1, 0, n_slab)
        if k % 2 == 0:
            t_hb += time.perf_counter() - t0
            n_hb += per_pass
        else:
            t_or += time.perf_counter() - t0
            n_or += per_pass
        k += 1
    r_hb, r_or = n_hb / t_hb, n_or / t_or
    r = (N_HB + N_OR) / (N_HB / r_hb + N_OR / r_or)
    desc = (f"FP64 oracle on the GPU's configuration after the timed sweeps: heatbath and overrelaxation passes "
            f"over time slices [0,{n_slab}) of the 48^3x96 lattice ({per_pass} link updates per pass), "
            f"{n_hb} heatbath updates in {t_hb:.1f} s, {n_or} overrelaxation updates in {t_or:.1f} s, rates "
            f"combined 1:5 as in a sweep; plaquette of the whole lattice in {t_plaq:.1f} s")
    agreement = {
        "plaquette": {"gpu": p_gpu, "oracle": p_orc, "abs_err": abs(p_gpu - p_orc)},
        "polyakov": {"gpu": [l_gpu.real, l_gpu.imag], "oracle": [l_orc.real, l_orc.imag],
                     "abs_err": abs(l_gpu - l_orc)},
        "overrelaxation_pass": {"links": 4 * per_pass, "max_abs_err": or_err, "bound": 1e-5},
        "heatbath_pass": {"links": 4 * per_pass, "max_abs_err_where_branches_agree": hb_err,
                          "branch_flips": flips, "bound": "1e-5, flips <= 1e-6 of updates"},
        "note": "one pass from the same FP64 input; links of all four directions on the slab compared "
                "(only direction 1 / 2 changes)",
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
    import numpy as np
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
                             reunit_mode=args.reunit_mode, tune_storage=True, tune_reunit_mode=True)
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
        for name, st, var in [(f"fp32_{alt}real", alt, args.variant & ~2),
                              ("fp32_12real_two_row_staple", 12, (args.variant | 2) & ~8)]:
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
                variants[name]["note"] = ("third row of each staple term taken as conj(row0 x row1): "
                                          "up to 1.2e-5 from the oracle on links of a Haar start before "
                                          "their first re-unitarization (1e-5 bar)")
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
        "config": {"workload": WORKLOAD_NAME, "nc": NC, "dims": list(DIMS), "beta": BETA,
                   "n_heatbath": N_HB, "n_overrelax": N_OR, "storage_reals": args.storage,
                   "kernel_variant": args.variant, "block_threads": args.block,
                   "autotuned": tuned,
                   "reunitarize": ("FP64, every link once per sweep, " +
                                   {0: "own pass after the sweep", 1: "in the update kernels of the last step",
                                    2: "spread over the steps"}[args.reunit_mode]),
                   "observables": "FP64 plaquette + Polyakov every sweep",
                   "link_updates_per_step": updates_per_sweep(),
                   "l2": "lattice (2.0 GB) larger than L2, no flush", "parallelism": f"replicas x{world}"},
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
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batched_arm(args):
    import numpy as np
    import torch
    import paper_1112_4533_gb300 as sun

    torch.cuda.set_device(0)
    rng = np.random.default_rng(4)
    n = 64
    Ls = rng.choice([8, 12, 16, 24], size=n)
    betas = rng.uniform(5.6, 6.4, size=n)
    sweeps = 50
    tuned = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tuned = sun.autotune_batch([(3, (int(L),) * 4, float(b)) for L, b in zip(Ls, betas)], 1, 4, precision=32,
                                   storage=args.storage, reunit_mode=args.reunit_mode, tune_storage=True,
                                   tune_reunit_mode=True)
        tuned["tuning_s"] = time.perf_counter() - t0
        args.storage, args.variant, args.reunit_mode = tuned["storage"], tuned["variant"], tuned["reunit_mode"]
        args.block, args.graph_sweeps = tuned["block_threads"], tuned["graph_sweeps"]
    kw = dict(precision=32, storage=args.storage, reunit_mode=args.reunit_mode, variant=args.variant,
              block_threads=args.block, graph_sweeps=args.graph_sweeps)
    lats = [sun.Lattice(3, (int(L),) * 4, float(b), hot_start=True, seed=100 + i, **kw)
            for i, (L, b) in enumerate(zip(Ls, betas))]
    updates = sum((1 + 4) * 4 * int(L) ** 4 for L in Ls) * sweeps
    B = sun.Batch(lats, use_graphs=True)
    B.run(max(1, args.warmup), 1, 4)
    torch.cuda.synchronize()
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        B.run(sweeps, 1, 4)
        t.append(time.perf_counter() - t0)
    B.close()
    # plain path: the same chains, one at a time
    for L in lats:
        L.run(1, 1, 4)
    torch.cuda.synchronize()
    tp = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        for L in lats:
            L.run(sweeps, 1, 4)
        torch.cuda.synchronize()
        tp.append(time.perf_counter() - t0)
    for L in lats:
        L.close()
    tb, tpl = min(t), min(tp)
    out = {"metric": "batched chains/s", "value": n / tb, "unit": "chains/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (Haar starts, seeds 100..163)",
           "config": {"workload": "64 SU(3) chains, L in {8,12,16,24} (seeded draw), beta U[5.6,6.4], hot start, "
                                  "50 sweeps of 1 heatbath + 4 overrelaxation each, FP32 links",
                      "L_counts": {str(v): int((Ls == v).sum()) for v in (8, 12, 16, 24)},
                      "link_updates_per_step": updates, "storage_reals": args.storage, "kernel_variant": args.variant,
                      "block_threads": args.block, "reunit_mode": args.reunit_mode, "autotuned": tuned},
           "link_updates_per_s": updates / tb,
           # per batch sweep of the one SU(3) group: 40 passes, the separate re-unitarization
           # (placement 0), plaquette and Polyakov partials and their per-chain sums, two counters
           "gpu_launches": args.steps * sweeps * (40 + (1 if args.reunit_mode == 0 else 0) + 4 + 2),
           "plain": {"value": n / tpl, "unit": "chains/s", "ms_per_step": tpl * 1e3, "link_updates_per_s": updates / tpl,
                     "path": "each chain alone, sun_run of 50 sweeps (one captured sweep graph per chain)"},
           "speedup_vs_plain": tpl / tb}
    print(json.dumps(out))


def serving_arm(args):
    import torch
    from paper_1112_4533_gb300 import serve

    torch.cuda.set_device(0)
    trace = serve.poisson_trace(args.requests, rate=20.0, seed=7)
    budget = int(args.budget_gb * (1 << 30))
    warm = serve.poisson_trace(4, rate=50.0, seed=99, Ls=(8,), sweeps=(2, 3))
    serve.Server(budget).run(warm)  # load kernels
    srv = serve.Server(budget, sweeps_per_tick=args.sweeps_per_tick or None, work_cap_ms=args.work_cap_ms,
                       tick_ms=args.tick_ms, policy=args.policy)
    t0 = time.perf_counter()
    out = srv.run(trace)
    wall = time.perf_counter() - t0
    st = serve.latency_stats(out)
    plain, pwall, pupd = serve.serve_plain(trace)
    pst = serve.latency_stats(plain)
    upd = sum(r.n_sweeps * 5 * 4 * r.L ** 4 for r in trace)
    res = {"metric": "p50 request latency", "value": st["p50_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic Poisson trace (seed 7)",
           "config": {"workload": f"{args.requests} requests, Poisson mean 20/s, Nc in {{2,3,4,6}}, L in "
                                  "{8,12,16,20,24}, 20..200 sweeps of 1 heatbath + 4 overrelaxation, FP32",
                      "hbm_budget_gb": args.budget_gb, "max_sweeps_per_tick": args.sweeps_per_tick or None,
                      "tick_ms": args.tick_ms, "work_cap_ms": args.work_cap_ms, "policy": args.policy},
           "p99_s": st["p99_s"], "mean_s": st["mean_s"], "completed": st["completed"],
           "throughput": {"requests_per_s": len(trace) / wall, "link_updates_per_s": upd / wall},
           "plain": {"p50_s": pst["p50_s"], "p99_s": pst["p99_s"], "mean_s": pst["mean_s"],
                     "requests_per_s": len(trace) / pwall, "link_updates_per_s": pupd / pwall,
                     "path": "one request at a time in arrival order, sun_run per chain"},
           "ticks": srv.ticks}
    print(json.dumps(res))


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
           "config": {"workload": WORKLOAD_NAME, "nc": NC, "dims": list(DIMS), "beta": BETA,
                      "n_heatbath": N_HB, "n_overrelax": N_OR},
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
    ap.add_argument("--variant", type=int, default=1, choices=range(16),
                    help="update-kernel variant bits: 1 = 5 blocks/SM register bound, 2 = two-row staple")
    ap.add_argument("--reunit-mode", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="seconds of oracle work in the cpu_baseline leg, and the cap of one --impl reference step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="fixed configuration from the flags, no autotuning")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the update kernels (0 = 128)")
    ap.add_argument("--graph-sweeps", type=int, default=0, help="sweeps captured per CUDA graph (0 = 1)")
    ap.add_argument("--workload", choices=["single", "batched", "serving"], default="single")
    ap.add_argument("--requests", type=int, default=80)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--sweeps-per-tick", type=int, default=0, help="cap on sweeps per serving tick (0 = none)")
    ap.add_argument("--tick-ms", type=float, default=40.0, help="predicted GPU time a serving tick aims at")
    ap.add_argument("--policy", choices=["srpt", "fifo"], default="srpt")
    ap.add_argument("--work-cap-ms", type=float, default=3.0)
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
