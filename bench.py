#!/usr/bin/env python
"""Throughput bench of the heterogeneous power-law attenuation FDTD.

Workload (default): 3D seeded Voronoi tissue map 512^3, 8 classes, 2 % c/rho
jitter, N = 4 relaxation mechanisms per class calibrated on the host, 20-cell
absorbing layer, 3 MHz focused square aperture (65 536 source cells) and a
strided receiver grid; FP32 arithmetic and storage.

One bench step = one time step of the whole grid (velocity sweep, pressure
sweep, sources, receivers).  Metric: voxel-updates per second (Gvox/s, one
voxel advanced by one full time step).  The working set (~15 GB) is far
larger than L2, so no flush is needed between steps.

Other workloads: ``--workload twolayer2d`` (2D two-layer nonlinear medium,
2048^2), ``--workload serving`` (a stream of mixed 2D/3D requests through the
continuous-batching server: throughput, p50/p99 latency) and ``--workload
adjoint`` (whole gradients of a receiver functional on a 1024^2 medium).

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU
oracle (the paper ships no runnable code) on a crop of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--size", type=int, default=512, help="cube side (512 = the 3D Voronoi workload)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="streaming end-to-end steps (0: = --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-order", type=int, default=2, choices=[2, 4],
                    help="2: leapfrog; 4: the time-space stencil (Sec. 3.3)")
    ap.add_argument("--no-other-scheme", action="store_true",
                    help="skip the device-time line of the other time scheme")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="voronoi3d", choices=["voronoi3d", "twolayer2d", "serving", "adjoint"],
                    help="serving: the mixed 2D/3D request stream through the continuous-batching server")
    ap.add_argument("--requests", type=int, default=40, help="serving: requests in the stream (200 = full mix)")
    ap.add_argument("--gradients", type=int, default=3, help="adjoint: timed gradients")
    ap.add_argument("--slots", type=int, default=8, help="serving: admitted requests at once")
    ap.add_argument("--load", type=float, default=0.8, help="serving: offered load / one-at-a-time capacity")
    ap.add_argument("--no-capacity", action="store_true", help="serving: skip the all-at-once capacity arms")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: one independent simulation per GPU)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_value(units_per_rank, seconds_per_rank, ws):
    """Whole-job throughput of N independent replicas: the units all ranks
    processed divided by the slowest rank's time (weak scaling)."""
    return ws * units_per_rank / allmax(seconds_per_rank, ws)


def allmax(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# workload


def workload(args, n_steps):
    """The synthetic workload: the 3D Voronoi medium (default) or the 2D
    two-layer nonlinear medium; returns (spec, class map, class list for the
    calibration as (alpha0, y, c) triples, beta map or None)."""
    from synthetic import config_c2, config_c3
    if args.workload == "twolayer2d":
        spec = config_c2(n_steps=n_steps)
        la, lb = spec.extra["layer_a"], spec.extra["layer_b"]
        n = spec.shape[0]
        cls = ((np.arange(n)[:, None] >= spec.extra["interface"]) * np.ones(spec.shape)).astype(np.uint16)
        return spec, cls, [(la["alpha0"], la["y"], la["c"]), (lb["alpha0"], lb["y"], lb["c"])], spec.maps["beta"]
    n = args.size
    if n == 512:
        spec = config_c3(n_steps=n_steps)
    else:
        lo = (512 - n) // 2
        box = ((0, n), (lo, lo + n), (lo, lo + n))
        spec = config_c3(n_steps=n_steps, box=box)
    triples = list(zip(spec.classes["alpha0"], spec.classes["y"], spec.classes["c"]))
    return spec, spec.maps["class_idx"], triples, None


def fit_classes(triples):
    """Host FP64 calibration of every (alpha0, y, c) class (paper settings), one thread per class."""
    import paper_2606_11103_gb300 as fw
    out = [None] * len(triples)
    reps = [None] * len(out)

    def job(i):
        a, y, c = triples[i]
        out[i], reps[i] = fw.fit_relaxation(float(a), float(y), 4, c0=float(c))

    th = [threading.Thread(target=job, args=(i,)) for i in range(len(out))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out, reps


def alg_bytes(ndim, nmech, storage, nonlinear, wabs, shape, time_order=2):
    """Algorithmic bytes per voxel of each sweep and of the minimal single-pass
    step (every field read once and written once, maps read once).  The
    time-space stencil's per-cell weights need K dt in the velocity sweep and
    rho in the pressure sweep (4 B each); the single-pass minimum reads both
    maps once either way."""
    es = 4
    eps = {"f32": 4, "bf16": 2, "f16": 2}[storage]
    D = ndim
    n_axes = list(shape)

    def frac(half):
        f = []
        for n in n_axes:
            act = (2 * wabs - 1) if half else 2 * wabs
            f.append(min(act, n) / n if wabs > 0 else 0.0)
        return f

    pml_v = sum(frac(True)) * 2 * es
    pml_p = sum(frac(False)) * 2 * es
    vel = es + 2 * D * es + 2 * D * nmech * eps + es + 2 + pml_v
    pres = D * es + 2 * es + 2 * nmech * eps + es + (es if nonlinear else 0) + 2 + pml_p
    single = 2 * es + 2 * D * es + 2 * D * nmech * eps + 2 * nmech * eps + es + es + 2 + \
        (es if nonlinear else 0) + pml_v + pml_p
    if time_order == 4:
        vel += es
        pres += es
    return vel, pres, single


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("fw_kernels.cuh", "fw_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2606_11103_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(vox, key="velocity"):
    """DRAM bytes per launch of the sweep from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_sha") != kernel_source_sha() or key not in d:
        return None
    return d[key]["bytes_per_voxel"] * vox


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline leg and the reference arm)


ORACLE_CROP = {"voronoi3d": 128, "twolayer2d": 768}


def oracle_sample(kind):
    crop = ORACLE_CROP[kind]
    if kind == "twolayer2d":
        return "%d^2 two-layer medium of the same kind (N=4, nonlinear, 30-cell PML)" % crop
    return "%d^3 crop of the 512^3 Voronoi workload (N=4, 20-cell PML)" % crop


def oracle_sim(kind, n_steps=8, time_order=2):
    from oracle import fit
    from oracle.medium import OracleMedium
    from oracle.stepper import OracleSim
    from synthetic import config_c2, config_c3
    crop = ORACLE_CROP[kind]
    if kind == "twolayer2d":
        spec = config_c2(n=crop, n_steps=n_steps)
        la, lb = spec.extra["layer_a"], spec.extra["layer_b"]
        triples = [(la["alpha0"], la["y"]), (lb["alpha0"], lb["y"])]
        cls = ((np.arange(crop)[:, None] >= spec.extra["interface"]) * np.ones(spec.shape)).astype(np.int64)
        beta = spec.maps["beta"].astype(np.float64)
    else:
        lo = (512 - crop) // 2
        spec = config_c3(n_steps=n_steps, box=((0, crop), (lo, lo + crop), (lo, lo + crop)))
        triples = list(zip(spec.classes["alpha0"], spec.classes["y"]))
        cls = spec.maps["class_idx"].astype(np.int64)
        beta = None
    params = []
    for a, y in triples:
        p, _ = fit.fit_relaxation(float(a), float(y), 4, maxiter=200, w_list=(0.5,))
        params.append(p)
    med = OracleMedium(spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], cls, params, beta=beta,
                       pml=spec.pml, f0=spec.f0, time_order=time_order)
    sim = OracleSim(med)
    sim.set_sources(spec.src_mask, spec.src_waves.astype(np.float64), spec.src_wave_of)
    sim.set_receivers(spec.rcv_mask, n_steps)
    return sim, int(np.prod(spec.shape))


def time_oracle(budget_s, kind="voronoi3d", time_order=2):
    sim, vox = oracle_sim(kind, n_steps=4096, time_order=time_order)
    sim.run(1)                      # thread start-up
    t0 = time.perf_counter()
    sim.run(2)
    one = (time.perf_counter() - t0) / 2
    k = max(1, min(2000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    sim.run(k)
    dt = time.perf_counter() - t0
    from oracle import stepper
    cores = stepper.threads()
    return {"value": vox * k / dt / 1e9, "unit": "Gvoxel-updates/s", "cores": cores, "kind": "oracle",
            "sample": "FP64 C oracle, %s, %d time steps, %.1f s" % (oracle_sample(kind), k, dt)}


def metric_name(args):
    return "voxel-updates/s (2D FP32)" if args.workload == "twolayer2d" else "voxel-updates/s (3D FP32)"


def workload_config(args, l2, parallelism):
    """The config object both arms print (the reference arm times a crop of it)."""
    scheme = scheme_name(getattr(args, "time_order", 2))
    if args.workload == "twolayer2d":
        return {"workload": "2D two-layer 2048^2 (c 1580/1450, rho 1060/950, alpha0 1.09/0.6, y 1.0/1.5, "
                            "beta 3.5/6), N=4, 30-cell PML, 3 MHz line source",
                "voxels": 2048 ** 2, "storage": args.storage, "scheme": scheme, "l2": l2, "parallelism": parallelism}
    return {"workload": "3D seeded Voronoi %d^3, 8 classes, N=4, 20-cell PML, focused 3 MHz aperture" % args.size,
            "voxels": args.size ** 3, "storage": args.storage, "scheme": scheme, "l2": l2,
            "parallelism": parallelism}


def reference_config(args):
    """The config object of the reference arm: the crop of the workload the
    FP64 oracle actually runs (a throughput is per voxel-update, so the crop's
    rate stands beside the full workload's), naming the workload it is cut
    from."""
    crop = ORACLE_CROP[args.workload]
    full = workload_config(args, "host cores (FP64 CPU oracle)", "host threads")
    out = dict(full)
    out["workload"] = "%s (sampled from: %s)" % (oracle_sample(args.workload), full["workload"])
    out["voxels"] = crop ** 2 if args.workload == "twolayer2d" else crop ** 3
    out["storage"] = "f64"
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sim, vox = oracle_sim(args.workload, n_steps=args.warmup + args.steps + 1, time_order=args.time_order)
    sim.run(args.warmup)
    t0 = time.perf_counter()
    sim.run(args.steps)
    dt = time.perf_counter() - t0
    v = vox * args.steps / dt / 1e9
    from oracle import stepper
    cores = stepper.threads()
    out = {"impl": "reference", "metric": metric_name(args), "value": v, "unit": "Gvoxel-updates/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": reference_config(args),
           "cpu_baseline": {"value": v, "unit": "Gvoxel-updates/s", "cores": cores, "kind": "oracle",
                            "sample": "FP64 C oracle on a %s, %d timed steps after %d"
                                      % (oracle_sample(args.workload), args.steps, args.warmup)},
           "e2e": {"value": v, "unit": "Gvoxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=ws)
    torch.cuda.set_device(local)
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build as fwbuild
    if rank == 0:
        fwbuild.build()
    barrier(ws)
    L = fw.lib()

    K, W = args.steps, args.warmup
    K2 = args.e2e_steps or K
    n_total = W + K + K2 + 2
    t0 = time.perf_counter()
    spec, cls_map, triples, beta = workload(args, n_total)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    classes, reps = fit_classes(triples)
    t_fit = time.perf_counter() - t0
    log("workload %s generated in %.1fs, %d classes fitted in %.1fs (max NRMSE %.3f)" %
        (spec.name, t_gen, len(classes), t_fit, max(r.nrmse for r in reps)))
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls_map, classes,
                               dt=spec.dt, beta=beta, pml=spec.pml, f0=spec.f0, storage=args.storage,
                               time_order=args.time_order)
    m.set_sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
    m.set_receivers(spec.rcv_mask, n_total)
    t_create = time.perf_counter() - t0
    info = m.info()
    vox = int(np.prod(spec.shape))
    log("medium: %.2f GB on device, created in %.1fs, dt %.3e" % (info["device_bytes"] / 1e9, t_create, info["dt"]))

    # warm-up (graph path and the timed path)
    m.run(W)
    torch.cuda.synchronize()

    # ---- timed region: per-sweep CUDA events on the launch stream ----
    ms_v, ms_p, ms_io, ms_tot = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    nl = C.c_int()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        fw.check(L.fw_step_timed(m.h, K, C.c_void_p(stream.cuda_stream), C.byref(ms_v), C.byref(ms_p),
                                 C.byref(ms_io), C.byref(ms_tot), C.byref(nl)), "fw_step_timed")
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    # device time of the K steps: from the first kernel's start event to the
    # last one's end event (the outer torch events also contain host-side
    # set-up of fw_step_timed and are kept as a cross-check)
    ms_outer = ev0.elapsed_time(ev1)
    ms = allmax(ms_tot.value, ws)
    rc, pmax = m.status()
    if rc != 0:
        raise RuntimeError("unstable run: %s" % fw.FwError(rc))
    value = replica_value(vox * K, ms_tot.value / 1e3, ws) / 1e9

    # ---- end to end through the C ABI: per step, the step's waveform samples
    # go host->device from pinned memory and the step's receiver samples come
    # back device->host into pinned memory ----
    nw, nr = spec.src_waves.shape[0], int(info["n_rcv"])
    h_w = torch.from_numpy(np.ascontiguousarray(spec.src_waves.T)).pin_memory()   # [steps][n_wave]
    h_r = torch.empty((K2, nr), dtype=torch.float32).pin_memory()
    it0 = info["step"]
    sp = C.c_void_p(stream.cuda_stream)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(K2):
        it = it0 + j
        fw.check(L.fw_set_waveform_samples(m.h, it, 1, C.c_void_p(h_w[it].data_ptr()), sp), "waveforms")
        fw.check(L.fw_run(m.h, 1, sp), "fw_run")
        fw.check(L.fw_read_receivers_range(m.h, it, 1, C.c_void_p(h_r[j].data_ptr()), sp), "receivers")
    torch.cuda.synchronize()
    t_e2e = allmax(time.perf_counter() - t0, ws)
    e2e = ws * vox * K2 / t_e2e / 1e9
    assert np.isfinite(h_r.numpy()).all()

    # ---- roofline of the dominant kernel (velocity sweep) ----
    b_vel, b_pres, b_single = alg_bytes(len(spec.shape), 4, args.storage, beta is not None, spec.pml, spec.shape,
                                        args.time_order)
    peak, peak_kind = measured_peaks()
    t_vel = ms_v.value / K / 1e3
    t_pres = ms_p.value / K / 1e3
    ach = b_vel * vox / t_vel / 1e9
    tkey = "velocity" if args.storage == "f32" else "velocity_" + args.storage
    tkey += "_2d" if args.workload == "twolayer2d" else ""
    tkey += "_ts" if args.time_order == 4 else ""
    traffic = profiled_traffic(vox, tkey)
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": traffic, "kernel": "k_velocity (velocity sweep)",
            "peak_source": "%s hbm_gbs" % peak_kind}
    step_info = {
        "velocity_ms": round(t_vel * 1e3, 4), "pressure_ms": round(t_pres * 1e3, 4),
        "io_ms": round(ms_io.value / K, 4),
        "outer_events_ms_per_step": round(ms_outer / K, 4),
        "pressure_gbs": round(b_pres * vox / t_pres / 1e9, 1),
        "alg_bytes_per_voxel": {"velocity": round(b_vel, 2), "pressure": round(b_pres, 2),
                                "single_pass_min": round(b_single, 2)},
        "step_gbs_vs_single_pass_min": round(b_single * vox * K / (ms / 1e3) / 1e9, 1),
        "frac_step_vs_single_pass_min": round(b_single * vox * K / (ms / 1e3) / 1e9 / peak, 4),
    }
    out = {
        "metric": metric_name(args), "value": round(value, 3), "unit": "Gvoxel-updates/s",
        "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": round(ms / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else "f32/%s-psi" % args.storage,
        "data": "synthetic",
        "config": workload_config(args, "working set %.1f GB >> 129 MB L2, no flush needed" % (info["device_bytes"] / 1e9),
                                  "replicas" if ws > 1 else "single GPU"),
        "e2e": {"value": round(e2e, 3), "unit": "Gvoxel-updates/s", "h2d_bytes_per_step": nw * 4,
                "d2h_bytes_per_step": nr * 4, "steps": K2},
        "gpu_launches": int(nl.value),
        "roofline": roof,
        "step": step_info,
        "clocks": clk.summary(),
        "max_abs_p": pmax,
    }
    m.close()
    if not args.no_other_scheme:
        out["other_scheme"] = other_scheme(fw, L, args, spec, cls_map, classes, beta, n_total, stream, vox, peak)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = time_oracle(args.cpu_seconds, args.workload, args.time_order)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def scheme_name(order):
    return "time-space stencil (4th order in time, Sec. 3.3)" if order == 4 else "leapfrog (2nd order in time)"


def other_scheme(fw, L, args, spec, cls_map, classes, beta, n_total, stream, vox, peak):
    """Device time of the same workload with the other time scheme (same
    medium, sources and step count; CUDA events on the launch stream), for
    the comparison of the two schemes beside the headline line."""
    order = 6 - args.time_order
    m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls_map, classes,
                               dt=spec.dt, beta=beta, pml=spec.pml, f0=spec.f0, storage=args.storage,
                               time_order=order)
    m.set_sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
    m.set_receivers(spec.rcv_mask, n_total)
    m.run(args.warmup)
    ms_v, ms_p, ms_io, ms_tot = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    nl = C.c_int()
    fw.check(L.fw_step_timed(m.h, args.steps, C.c_void_p(stream.cuda_stream), C.byref(ms_v), C.byref(ms_p),
                             C.byref(ms_io), C.byref(ms_tot), C.byref(nl)), "fw_step_timed")
    rc, _ = m.status()
    m.close()
    if rc != 0:
        raise RuntimeError("unstable run (%s): %s" % (scheme_name(order), fw.FwError(rc)))
    K = args.steps
    b_vel, b_pres, b_single = alg_bytes(len(spec.shape), 4, args.storage, beta is not None, spec.pml, spec.shape,
                                        order)
    t_vel, t_pres = ms_v.value / K / 1e3, ms_p.value / K / 1e3
    return {"scheme": scheme_name(order), "value": round(vox * K / (ms_tot.value / 1e3) / 1e9, 3),
            "unit": "Gvoxel-updates/s", "ms_per_step": round(ms_tot.value / K, 4),
            "velocity_ms": round(t_vel * 1e3, 4), "pressure_ms": round(t_pres * 1e3, 4),
            "velocity_frac": round(b_vel * vox / t_vel / 1e9 / peak, 4),
            "pressure_frac": round(b_pres * vox / t_pres / 1e9 / peak, 4),
            "alg_bytes_per_voxel": {"velocity": round(b_vel, 2), "pressure": round(b_pres, 2)}}


# ---------------------------------------------------------------------------
# serving: continuous batching vs one request at a time


def _serving_arm(fw, media, classes, arrivals, budget, slots, streams, chunk=32, policy=0):
    """Replay the arrival stream through one server; returns per-request
    completions (tag -> dict) and the server-clock origin."""
    from synthetic.serving import DT, DX, F0, PML
    srv = fw.Server(budget, max_active=slots, chunk_steps=chunk, n_streams=streams, policy=policy)
    t0 = srv.now()
    done, i, n = {}, 0, len(media)
    last = time.perf_counter()
    while len(done) < n:
        now = srv.now() - t0
        while i < n and arrivals[i] <= now:
            q = media[i]
            srv.submit(q["shape"], DX, DT, q["c"], q["rho"], q["class_idx"], classes[i], q["n_steps"],
                       src_mask=q["src_mask"], waves=q["waves"], rcv_mask=q["rcv_mask"], pml=PML, f0=F0, tag=i)
            i += 1
        wait = (arrivals[i] - (srv.now() - t0)) if i < n else 0.5
        for d in srv.poll(timeout=max(0.0, min(wait, 0.5))):
            done[d["tag"]] = d
            last = time.perf_counter()
            if d["status"] != 0:
                log("  request %d %s: status %d" % (d["tag"], media[d["tag"]]["shape"], d["status"]))
        if time.perf_counter() - last > 300 and i == n:
            log("serving: no completion for 300 s, stats %s" % srv.stats())
            srv.close()
            raise RuntimeError("serving arm stalled")
    srv.close()
    return done, t0


def _arm_summary(done, t0, arrivals):
    lat = np.array([done[k]["t_done"] - done[k]["t_submit"] for k in sorted(done)])
    wait = np.array([done[k]["t_admit"] - done[k]["t_submit"] for k in sorted(done)])
    vs = sum(d["voxel_steps"] for d in done.values())
    span = max(d["t_done"] for d in done.values()) - (t0 + float(arrivals[0]))
    bad = {int(k): int(d["status"]) for k, d in done.items() if d["status"] != 0}
    return {"value": round(vs / span / 1e9, 3), "unit": "Gvoxel-updates/s", "makespan_s": round(span, 2),
            "p50_s": round(float(np.percentile(lat, 50)), 3), "p99_s": round(float(np.percentile(lat, 99)), 3),
            "mean_queue_s": round(float(wait.mean()), 3), "failed": bad}


def run_serving(args):
    """Mixed stream of 2D (512^2-4096^2) and 3D (128^3-384^3) requests with
    500-3000 steps (Poisson arrivals at args.load of the measured
    one-at-a-time capacity) through the continuous-batching server and
    through the same server limited to one request at a time; then the same
    stream submitted at once (capacity)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build as fwbuild
    from synthetic import serving_stream
    from synthetic.serving import DT, DX, F0, PML, lut_pairs, request_media
    fwbuild.build()
    pairs = lut_pairs()
    lut = [None] * len(pairs)

    def job(k):
        lut[k], _ = fw.fit_relaxation(pairs[k][0], pairs[k][1], 4, maxiter=3000, w=(0.1, 0.5, 0.9))

    t0 = time.perf_counter()
    th = [threading.Thread(target=job, args=(k,)) for k in range(len(pairs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    t_fit = time.perf_counter() - t0
    reqs = serving_stream(seed=3, n_req=args.requests, rate_hz=1.0)
    t0 = time.perf_counter()
    media = [request_media(r, len(pairs)) for r in reqs]
    torch.cuda.synchronize()
    classes = [[lut[k] for k in q["lut_idx"]] for q in media]
    log("serving: %d table pairs fitted in %.1fs, %d requests generated in %.1fs" %
        (len(pairs), t_fit, len(reqs), time.perf_counter() - t0))
    # one-at-a-time service rate per dimension, from one request of each
    rate = {}
    for nd in (2, 3):
        k = next(i for i, q in enumerate(media) if len(q["shape"]) == nd)
        q = media[k]
        m = fw.Medium.from_classes(q["shape"], DX, q["c"], q["rho"], q["class_idx"], classes[k], dt=DT, pml=PML, f0=F0)
        n = min(300, q["n_steps"])
        m.run(32)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        m.run(n)
        torch.cuda.synchronize()
        rate[nd] = int(np.prod(q["shape"])) * n / (time.perf_counter() - t1)
        m.close()
    work = np.array([int(np.prod(q["shape"])) * q["n_steps"] for q in media], np.float64)
    service = np.array([w / rate[len(q["shape"])] for w, q in zip(work, media)])
    lam = args.load / service.mean()
    gaps = np.diff([r["arrival"] for r in reqs], prepend=0.0)       # seeded Exp(1) gaps
    arrivals = np.cumsum(gaps) / lam
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(200e9, 0.8 * free))
    slots = args.slots
    with ClockSampler(0) as clk:
        batched, tb = _serving_arm(fw, media, classes, arrivals, budget, slots, slots, policy=0)
        log("serving: batched (size classes) done")
        shared, tsh = _serving_arm(fw, media, classes, arrivals, budget, slots, slots, policy=1)
        log("serving: batched (one priority) done")
        single, ts = _serving_arm(fw, media, classes, arrivals, budget, 1, 1, policy=1)
        log("serving: one at a time done")
    same = sum(int(batched[k]["status"] == 0 and np.array_equal(batched[k]["traces"], single[k]["traces"]))
               for k in batched)
    sb, ssh, ss = (_arm_summary(batched, tb, arrivals), _arm_summary(shared, tsh, arrivals),
                   _arm_summary(single, ts, arrivals))
    # latency by size class (short: voxels x steps <= the server's default bound)
    short = {k for k, q in enumerate(media) if np.prod(q["shape"]) * q["n_steps"] <= 5e9}
    for summ, res in ((sb, batched), (ssh, shared), (ss, single)):
        for name, keys in (("short", short), ("long", set(res) - short)):
            lat = [res[k]["t_done"] - res[k]["t_submit"] for k in keys if k in res]
            if lat:
                summ[name] = {"n": len(lat), "p50_s": round(float(np.percentile(lat, 50)), 3),
                              "p99_s": round(float(np.percentile(lat, 99)), 3)}
    cap = {}
    if not args.no_capacity:
        zero = np.zeros(len(media))
        cap_b, tcb = _serving_arm(fw, media, classes, zero, budget, slots, slots, policy=0)
        cap_s, tcs = _serving_arm(fw, media, classes, zero, budget, 1, 1, policy=1)
        cap = {"batched": _arm_summary(cap_b, tcb, zero), "one_at_a_time": _arm_summary(cap_s, tcs, zero)}
    out = {
        "metric": "serving throughput, mixed 2D/3D request stream",
        "value": cap["batched"]["value"] if cap else sb["value"], "unit": "Gvoxel-updates/s",
        "higher_is_better": True, "p50_s": sb["p50_s"], "p99_s": sb["p99_s"],
        "capacity": cap,
        "at_offered_load": {"batched": sb, "batched_one_priority": ssh, "one_at_a_time": ss},
        "n_requests": len(media), "identical_results": "%d/%d" % (same, len(media)),
        "offered_load": args.load, "service_rate_gvox_s": {"2d": round(rate[2] / 1e9, 2), "3d": round(rate[3] / 1e9, 2)},
        "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Poisson stream (seed 3) of %d requests: 2D 512^2-4096^2, 3D 128^3-384^3 Voronoi "
                               "media (8 classes from a 36-pair table, N=4), 500-3000 steps" % len(media),
                   "slots": args.slots, "streams": args.slots, "chunk_steps": 32, "hbm_budget_gb": round(budget / 1e9, 1),
                   "arrival_span_s": round(float(arrivals[-1]), 2)},
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# adjoint workload: gradients of a receiver misfit (fw_gradient)


def adjoint_alg_bytes(ndim, nmech, wabs, shape):
    """Algorithmic bytes per voxel and time step of one gradient: the forward
    run and the recomputation of each segment (two forward steps), the state
    image of every recomputed step written and read back once, the adjoint
    state read and written once, two FP64 gradient accumulators read and
    written once, the material maps and class index read once."""
    vel, pres, _ = alg_bytes(ndim, nmech, "f32", False, wabs, shape)
    state = (1 + ndim + ndim * nmech + nmech) * 4
    return 2 * (vel + pres) + 2 * state + 2 * state + 2 * 2 * 8 + (4 + 4 + 2)


def oracle_gradient_rate(budget_s):
    """FP64 oracle adjoint on a 192^2 crop of the adjoint workload (same
    classes and protocol), voxel-steps per second of the whole gradient."""
    from oracle import fit
    from oracle.adjoint import misfit_gradient
    from oracle import stepper
    from synthetic import config_c5
    n, steps = 192, 300
    spec = config_c5(n=n, n_steps=steps)
    params = [fit.fit_relaxation(float(a), float(y), 3, maxiter=200, w_list=(0.5,))[0]
              for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    cls = spec.maps["class_idx"].astype(np.int64)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((int(spec.rcv_mask.sum()), steps))
    t0 = time.perf_counter()
    misfit_gradient(spec.shape, spec.dx, spec.dt, spec.maps["c"].astype(np.float64),
                    spec.maps["rho"].astype(np.float64), cls, params, np.asarray(spec.classes["alpha0"]), steps,
                    spec.src_mask, spec.src_waves.astype(np.float64), spec.rcv_mask, G=G, pml=spec.pml, f0=spec.f0,
                    checkpoint=30)
    dt = time.perf_counter() - t0
    return {"value": n * n * steps / dt / 1e9, "unit": "Gvoxel-steps/s", "cores": stepper.threads(),
            "kind": "oracle", "sample": "FP64 oracle adjoint (Python driver, C stepper), %d^2 crop of the "
                                        "adjoint workload, %d steps, checkpoint 30, %.1f s" % (n, steps, dt)}


def run_adjoint(args):
    """Gradient of a receiver functional on the 1024^2 Voronoi adjoint
    workload (6 classes, N=3, 64 receivers, 3000 steps, checkpoint every
    100): whole gradients (forward with checkpoints, recomputation, adjoint)
    timed with device-resident G, alpha0 and outputs; e2e with host buffers."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build as fwbuild
    from synthetic import config_c5
    fwbuild.build()
    spec = config_c5()
    triples = list(zip(spec.classes["alpha0"], spec.classes["y"], spec.classes["c"]))
    t0 = time.perf_counter()
    out_cls = [None] * len(triples)

    def job(i):
        a, y, c = triples[i]
        out_cls[i] = fw.fit_relaxation(float(a), float(y), 3, c0=float(c))[0]

    th = [threading.Thread(target=job, args=(i,)) for i in range(len(triples))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    log("adjoint workload: %d classes fitted in %.1fs" % (len(triples), time.perf_counter() - t0))
    cls = spec.maps["class_idx"]
    m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls, out_cls, dt=spec.dt,
                               pml=spec.pml, f0=spec.f0)
    m.set_sources(spec.src_mask, spec.src_waves)
    n_steps = spec.n_steps
    m.set_receivers(spec.rcv_mask, n_steps)
    nr = int(m.info()["n_rcv"])
    rng = np.random.default_rng(6)
    G_h = rng.standard_normal((nr, n_steps)).astype(np.float32)
    a0_h = np.asarray(spec.classes["alpha0"], np.float32)[cls]
    dev = torch.device("cuda", local)
    G_d, a0_d = torch.from_numpy(G_h).to(dev), torch.from_numpy(a0_h).to(dev)
    out_d = (torch.empty(spec.shape, dtype=torch.float32, device=dev),
             torch.empty(spec.shape, dtype=torch.float32, device=dev))
    start = m.save_state(out=torch.empty(m.state_bytes(), dtype=torch.uint8, device=dev))
    stream = torch.cuda.current_stream()
    K, W = max(1, args.gradients), 1
    for _ in range(W):
        m.load_state(start)
        m.gradient(n_steps, G_d, alpha0=a0_d, checkpoint=100, out=out_d)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(K):
            m.load_state(start)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.gradient(n_steps, G_d, alpha0=a0_d, checkpoint=100, out=out_d)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    assert torch.isfinite(out_d[0]).all() and torch.isfinite(out_d[1]).all()
    # end to end: G and alpha0 from host memory, gradients back to host memory
    out_h = (np.empty(spec.shape, np.float32), np.empty(spec.shape, np.float32))
    m.load_state(start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.gradient(n_steps, G_h, alpha0=a0_h, checkpoint=100, out=out_h)
    t_e2e = time.perf_counter() - t0
    m.close()
    vox = int(np.prod(spec.shape))
    t = float(np.median(times))
    value = vox * n_steps / t / 1e9
    b = adjoint_alg_bytes(2, 3, spec.pml, spec.shape)
    peak, peak_kind = measured_peaks()
    ach = b * vox * n_steps / t / 1e9
    out = {"metric": "gradient voxel-steps/s (2D FP32 adjoint)", "value": round(value, 3), "unit": "Gvoxel-steps/s",
           "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": round(t * 1e3, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "2D Voronoi 1024^2, 6 classes, N=3, 20-cell PML, 64 receivers, 3000 steps per "
                                  "gradient, checkpoint every 100", "voxels": vox, "storage": "f32",
                      "l2": "state images %.1f GB >> 129 MB L2" % ((n_steps // 100 + 103) * m_state_gb(spec)),
                      "parallelism": "single GPU", "step": "one whole gradient"},
           "e2e": {"value": round(vox * n_steps / t_e2e / 1e9, 3), "unit": "Gvoxel-steps/s",
                   "h2d_bytes_per_step": G_h.nbytes + a0_h.nbytes, "d2h_bytes_per_step": 2 * out_h[0].nbytes},
           "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "traffic": None,
                        "kernel": "fw_gradient as a whole (%.1f B per voxel-step)" % b,
                        "peak_source": "%s hbm_gbs" % peak_kind},
           "gradient_s": [round(x, 4) for x in times],
           "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_gradient_rate(args.cpu_seconds)
    print(json.dumps(out), flush=True)


def m_state_gb(spec):
    # p, v (2), psi1 (2 x 3), psi2 (3) and the absorbing-layer memory, FP32
    return (1 + 2 + 6 + 3 + 4) * 4 * int(np.prod(spec.shape)) / 1e9


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
