#!/usr/bin/env python
"""Benchmark: first-hit ray tracing through hybrid voxel formats on one B300.

Workload (one "step"): the 512^3 seeded terrain volume (fBm heightfield with
fBm caves, RGBA8 materials) in the two formats R(4,4,4) S(2) G(3) and
R(3,3,3) R(3,3,3) R(3,3,3); for each format, a 1920x1080 pinhole view
(rays generated and traced in one kernel) and 2^21 incoherent rays (origins
uniform in the box, directions uniform on the sphere) resident in HBM.
value = rays traced / time, in Mrays/s, over the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun) every rank traces its own replica of the workload
(rays are independent; no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s per hybrid format vs bytes/voxel; batched+served p50/p99 vs plain"
UNIT = "Mrays/s"
N_VOL = 512
FORMATS = ["R(4,4,4) S(2) G(3)", "R(3,3,3) R(3,3,3) R(3,3,3)"]
WIDTH, HEIGHT = 1920, 1080
N_INC = 1 << 21
SEED = 2024
FLUSH_BYTES = 256 << 20  # > 126 MB L2
WORKLOAD = ("512^3 terrain (fBm heightfield + caves, RGBA8), formats R(4,4,4) S(2) G(3) and "
            "R(3,3,3) R(3,3,3) R(3,3,3); per format 1920x1080 pinhole view + 2^21 incoherent rays")


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_src_sha():
    h = hashlib.sha256()
    for name in ("trace.cuh", "fmt.hpp"):
        with open(os.path.join(ROOT, "paper_2410_14128_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    sha = kernel_src_sha()
    with open(p) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == sha:
                return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.out = os.path.join("/tmp", f"vx_clocks_{os.getpid()}.csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.out)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs():
    import synth
    grid = synth.terrain_volume(SEED, N_VOL)
    cam = synth.camera(SEED + 1, N_VOL, WIDTH, HEIGHT, mode="above")
    inc = synth.incoherent_rays(SEED + 2, N_VOL, N_INC)
    return grid, cam, inc


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(grid, cam, inc, budget_s: float, threads: int | None = None):
    """Times the FP64 oracle on an interleaved sample of the step's rays (half
    primary, half incoherent) until about budget_s seconds of wall time.
    The oracle is format-independent (it walks the uncompressed grid)."""
    import oracle
    prim = oracle.pinhole(cam)
    rng = np.random.default_rng(5)
    pi = rng.permutation(len(prim))
    ii = rng.permutation(len(inc))
    chunk = max(20000, 2048 * (os.cpu_count() or 1))
    done, t_used, used_threads, k = 0, 0.0, 1, 0
    while t_used < budget_s and (k + 1) * chunk <= min(len(prim), len(inc)):
        sample = np.concatenate([prim[pi[k * chunk:(k + 1) * chunk]], inc[ii[k * chunk:(k + 1) * chunk]]])
        t0 = time.perf_counter()
        _, used_threads = oracle.trace(grid, sample, threads=threads)
        t_used += time.perf_counter() - t0
        done += len(sample)
        k += 1
    return done / t_used / 1e6, used_threads, done, t_used


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return 0
    grid, cam, inc = make_inputs()
    import oracle
    oracle.lib()
    per_step = []
    # bounded sample per step, so that the whole run stays within a few minutes
    budget = max(0.05, min(args.ref_step_s, 150.0 / (args.steps + args.warmup)))
    for s in range(args.warmup + args.steps):
        v, thr, n, t = oracle_rate(grid, cam, inc, budget_s=budget)
        if s >= args.warmup:
            per_step.append((v, n, t))
    rays = sum(p[1] for p in per_step)
    secs = sum(p[2] for p in per_step)
    value = rays / secs / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "formats": FORMATS, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{rays} rays of the step (half pinhole, half incoherent) per run; the FP64 "
                                   f"oracle walks the uncompressed 512^3 grid, so one timing serves both formats"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2410_14128_b300 as vx

    grid, cam, inc_np = make_inputs()
    vols = [vx.Volume(s, grid) for s in FORMATS]
    inc = torch.from_numpy(inc_np).cuda()
    n_prim = WIDTH * HEIGHT
    hits_p = [vx.alloc_hits(n_prim) for _ in FORMATS]
    hits_i = [vx.alloc_hits(N_INC) for _ in FORMATS]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    rays_per_step = len(FORMATS) * (n_prim + N_INC)
    mode = {"auto": vx.MODE_AUTO, "plain": vx.MODE_PLAIN, "persistent": vx.MODE_PERSISTENT}[args.mode]

    # --- autotune the incoherent-ray trace per format (outside timing) ---
    tuned = []
    if mode == vx.MODE_AUTO and not args.no_tune:
        for v in vols:
            tuned.append(v.autotune(inc[: 1 << 19]))

    # --- algorithmic bytes per ray (instrumented kernels, outside timing) ---
    counts = {}
    prim_rays = vx.raygen_pinhole(cam)
    for k, v in enumerate(vols):
        for name, rays in (("render", prim_rays), ("trace", inc)):
            c = torch.zeros(3, dtype=torch.int64, device="cuda")
            tmp = vx.alloc_hits(rays.shape[0])
            v.trace_counted(rays, tmp, c)
            torch.cuda.synchronize()
            b, it, d = (int(x) for x in c.cpu())
            n = rays.shape[0]
            counts[(k, name)] = {"node_bytes_per_ray": b / n, "iters_per_ray": it / n, "fp64_per_ray": d / n}
    del prim_rays

    def step(evs=None, mode=mode):
        flush.zero_()
        for k, v in enumerate(vols):
            if evs is not None:
                evs[(k, "render")][0].record()
            v.render(cam, hits_p[k])
            if evs is not None:
                evs[(k, "render")][1].record()
                evs[(k, "trace")][0].record()
            v.trace(inc, hits_i[k], mode=mode)
            if evs is not None:
                evs[(k, "trace")][1].record()

    # the plain one-thread-per-ray kernel on the same step, for comparison
    plain_ms = None
    if mode != vx.MODE_PLAIN:
        for _ in range(2):
            step(mode=vx.MODE_PLAIN)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            step(mode=vx.MODE_PLAIN)
        b.record()
        torch.cuda.synchronize()
        plain_ms = a.elapsed_time(b) / 5

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    ev = {key: [] for key in counts}
    all_evs = []
    for _ in range(args.steps):
        e = {key: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for key in counts}
        all_evs.append(e)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_start.record()
    for s in range(args.steps):
        step(all_evs[s])
    t_end.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    for e in all_evs:
        for key, (a, b) in e.items():
            ev[key].append(a.elapsed_time(b))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * rays_per_step * args.steps / (total_ms / 1e3) / 1e6

    # --- per-format results and the roofline of the dominant kernel ---
    peak, peak_kind = load_peaks()
    per_format = []
    tot = {}
    for k, spec in enumerate(FORMATS):
        st = vols[k].stats()
        ms_r = float(np.mean(ev[(k, "render")]))
        ms_t = float(np.mean(ev[(k, "trace")]))
        tot[(k, "render")] = sum(ev[(k, "render")])
        tot[(k, "trace")] = sum(ev[(k, "trace")])
        per_format.append({
            "format": spec,
            "mrays_s_primary": round(n_prim / ms_r / 1e3, 2),
            "mrays_s_incoherent": round(N_INC / ms_t / 1e3, 2),
            "mrays_s": round((n_prim + N_INC) / (ms_r + ms_t) / 1e3, 2),
            "device_bytes": st["device_bytes"],
            "bytes_per_voxel": round(st["device_bytes"] / N_VOL ** 3, 5),
            "bytes_per_occupied_voxel": round(st["device_bytes"] / max(1, st["occupied_voxels"]), 4),
            "node_bytes_per_ray_primary": round(counts[(k, "render")]["node_bytes_per_ray"], 2),
            "node_bytes_per_ray_incoherent": round(counts[(k, "trace")]["node_bytes_per_ray"], 2),
            "iters_per_ray_incoherent": round(counts[(k, "trace")]["iters_per_ray"], 2),
            "fp64_decisions_per_ray_incoherent": round(counts[(k, "trace")]["fp64_per_ray"], 5),
            "specialized_kernel": st["specialized"],
            "tuned_trace_opts": tuned[k] if tuned else None,
        })
    dom = max(tot, key=tot.get)
    k, name = dom
    n_rays = n_prim if name == "render" else N_INC
    io = 16 + (32 if name == "trace" else 0)
    alg_bytes = n_rays * (counts[dom]["node_bytes_per_ray"] + io)
    avg_ms = float(np.mean(ev[dom]))
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    kernel_key = f"{name}:{FORMATS[k].replace(' ', '')}"
    traffic = ncu_traffic(kernel_key)
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": f"{'k_render' if name == 'render' else 'k_trace'} {FORMATS[k]}",
                "alg_bytes_per_launch": int(alg_bytes), "avg_launch_ms": round(avg_ms, 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}

    # --- end to end through the host-memory entry points ---
    e2e = None
    if not args.no_e2e:
        pin_rays = torch.from_numpy(inc_np).pin_memory().numpy()
        out_p = torch.empty((n_prim, 4), dtype=torch.int32).pin_memory().numpy().view(vx.HIT_DTYPE).reshape(-1)
        out_i = torch.empty((N_INC, 4), dtype=torch.int32).pin_memory().numpy().view(vx.HIT_DTYPE).reshape(-1)

        def e2e_step():
            for v in vols:
                v.render_host(cam, out=out_p)
                v.trace_host(pin_rays, out=out_i)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": round(world * rays_per_step * args.steps / dt / 1e6, 3), "unit": UNIT,
               "h2d_bytes_per_step": len(FORMATS) * N_INC * 32,
               "d2h_bytes_per_step": len(FORMATS) * (n_prim + N_INC) * 16,
               "api": "vx_render_host + vx_trace_host, pinned host buffers"}

    # --- CPU baseline: the oracle on a bounded sample ---
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, thr, n, t = oracle_rate(grid, cam, inc_np, budget_s=args.cpu_budget_s)
        cpu = {"value": round(v, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{n} rays of the step (half pinhole, half incoherent), {t:.1f} s of FP64 oracle on "
                         f"the uncompressed 512^3 grid; format-independent"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "formats": FORMATS, "rays_per_step": rays_per_step,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"flushed before each step by a {FLUSH_BYTES >> 20} MiB write (inside the timed region)",
                       "hit_layout": "full 16 B",
                       "mode": {"auto": "auto (vx_trace options autotuned per format on 2^19 of the rays)",
                                "plain": "plain (one thread per ray)",
                                "persistent": "persistent warps with ray refill"}[args.mode]},
            "plain_kernel_ms_per_step": round(plain_ms, 4) if plain_ms else None,
            "per_format": per_format,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * len(FORMATS) * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    for v in vols:
        v.free()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "plain", "persistent"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
