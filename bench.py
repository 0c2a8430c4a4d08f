#!/usr/bin/env python
"""Benchmark: first-hit ray tracing through hybrid voxel formats on one B300.

Default workload (one JSON line): the 2048^3 seeded primitive scene (20k
spheres, boxes and thin walls plus 64 stamped 64^3 prototypes, ~2% occupied).

  value      batched tracing: 64 ray sets of uneven size (2^16..2^23 rays,
             camera views and incoherent rays) over 4 resident formats, traced
             by one vx_trace_batch call per step, replayed as a CUDA graph;
             a "step" is one pass over all 64 sets (84.4 M rays), Mrays/s.
             Beside it: one plain launch per set, one persistent launch per set.
  per_format the Table 2 sweep at 2048^3: each format's size (bytes/voxel),
             Mrays/s on 8 camera views of 1920x1080 and on 8 ambient-occlusion
             rays per primary hit, and the achieved fraction of HBM bandwidth.
  serving    Poisson render requests over 6 resident formats (512^3 and
             2048^3): continuous batching against the serial plain path,
             throughput with p50/p99 latency.
  roofline   the dominant kernel of the batched step, timed with CUDA events
             on the stream it runs on, inside the timed region.
  e2e        the batched step through vx_trace_batch_host from pinned host
             memory (per-set vx_trace_host calls beside it).
  cpu_baseline  the FP64 oracle on the machine's host cores, on a sample of the
             same rays.
  terrain512 the 512^3 terrain step (two formats, a 1080p view and 2^21
             incoherent rays each) as a sub-object.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload {terrain512,formats512,sweep2048,batch,serve,dedup,buildmem}

For N > 1 (torchrun) every rank traces its own replica of the workload
(rays are independent; no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import datetime
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
WORKLOAD512 = ("512^3 terrain (fBm heightfield + caves, RGBA8), formats R(4,4,4) S(2) G(3) and "
               "R(3,3,3) R(3,3,3) R(3,3,3); per format 1920x1080 pinhole view + 2^21 incoherent rays")

# Table 2: the paper's label of each format (1-20 at 2048^3, 21-40 at 512^3).
TABLE2_2048 = {1: "D(4,4,4,6) D(3,3,3,6) G(4)", 2: "D(4,4,4,6) R(3,3,3) G(4)", 3: "R(4,4,4) R(3,3,3) G(4)",
               4: "R(4,4,4) S(3) G(4)", 5: "R(4,4,4) R(4,4,4) R(3,3,3)", 6: "D(4,4,4,6) S(7)",
               7: "D(4,4,4,6) G(7)", 8: "D(6,6,6,6) S(5)", 9: "D(6,6,6,6) G(5)", 10: "R(4,4,4) S(7)",
               11: "R(4,4,4) G(7)", 12: "R(6,6,6) S(5)", 13: "R(6,6,6) G(5)", 14: "R(3,3,3) G(8)",
               15: "R(8,8,8) G(3)", 16: "S(7) G(4)", 17: "S(5) G(6)", 18: "S(3) G(8)", 19: "S(11)", 20: "G(11)"}
TABLE2_512 = {21: "D(3,3,3,6) D(3,3,3,6) G(3)", 22: "D(3,3,3,6) R(3,3,3) G(3)", 23: "R(3,3,3) R(3,3,3) G(3)",
              24: "R(3,3,3) R(3,3,3) R(3,3,3)", 25: "R(4,4,4) R(1,1,1) R(4,4,4)", 26: "D(4,4,4,6) S(5)",
              27: "D(4,4,4,6) G(5)", 28: "R(4,4,4) S(5)", 29: "R(4,4,4) G(5)", 30: "R(2,2,2) G(7)",
              31: "R(7,7,7) G(2)", 32: "S(5) R(4,4,4)", 33: "G(5) R(4,4,4)", 34: "D(5,5,5,6) D(4,4,4,6)",
              35: "D(5,5,5,6) R(4,4,4)", 36: "R(5,5,5) R(4,4,4)", 37: "R(9,9,9)", 38: "D(9,9,9,6)", 39: "S(9)",
              40: "G(9)"}
# the 2048^3 sweep: all of Table 2's 2048^3 formats, plus one with 2^2 and 2^1 Raw levels
SWEEP_FORMATS = list(TABLE2_2048.values()) + ["R(2,2,2) R(1,1,1) S(4) G(4)"]
LABEL = {v: k for k, v in {**TABLE2_2048, **TABLE2_512}.items()}
BATCH_FORMATS = ["R(3,3,3) G(8)", "R(4,4,4) G(7)", "R(4,4,4) S(3) G(4)", "R(4,4,4) R(3,3,3) G(4)"]
SEED3 = 2048
N_SETS = 64
WORKLOAD = ("2048^3 primitive scene (20k seeded spheres/boxes/thin walls + 64 stamped 64^3 prototypes, "
            "~2% occupied); batched: 64 ray sets of 2^16..2^23 rays (even: camera views, odd: incoherent) over "
            "4 resident formats, one vx_trace_batch per step replayed as a CUDA graph")


def job_throughput(local_ms: float, rays_per_rank: int, world: int, dist=None):
    """Whole-job throughput: every rank traced rays_per_rank rays; the job
    took the slowest rank's time.  Returns (Mrays/s, max ms over ranks)."""
    total_ms = local_ms
    if dist is not None and world > 1:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * rays_per_rank / (total_ms / 1e3) / 1e6, total_ms


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


def ncu_counters(kernel_key: str):
    """Counters per launch of `kernel_key` ("<ray set>:<format>:<kernel>")
    from the committed ncu summary: {"dram_bytes", "warp_inst", "l2_hit_pct"}
    (a missing one is None), or {} when the kernel source changed since the
    capture or the kernel was not captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return {}
    sha = kernel_src_sha()
    with open(p) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split("#")[0].split()
            if len(parts) >= 4 and parts[0] == kernel_key and parts[1] == sha:
                num = [None if x == "-" else float(x) for x in parts[2:5]] + [None] * 3
                return {"dram_bytes": num[0], "warp_inst": num[1], "l2_hit_pct": num[2]}
    return {}


# Warp-instruction issue peak: 148 SMs x 4 schedulers x 1 warp instruction per
# cycle at the 2032 MHz maximum SM clock.
ISSUE_PEAK_GINST_S = 148 * 4 * 2.032
NOMINAL_HBM_GBS = 8000.0  # B300 HBM3e, nominal (the measured copy rate is the roofline's peak)


def trace_launches(opts: dict | None, log2_dim) -> int:
    """Kernels one vx_trace call launches: the trace, plus the coherence sort
    when the options ask for it (key histogram, tiled scan of the bins -- a
    second pass when there is more than one tile of 8192 -- scatter of the
    rays, and the gather that puts the hits back in order)."""
    g = opts.get("sort_cell_log2", 0) if opts else 0
    if not g:
        return 1
    nbins = 8 << sum(min(max(ld - g, 0), 5) for ld in log2_dim)
    return 1 + 4 + (1 if nbins > 8192 else 0)


def pcie_both_ways_gbs(nbytes: int = 256 << 20, reps: int = 5) -> float:
    """Host<->device copy rate (GB/s, both directions summed) with one
    pinned-host upload and one download in flight at once on two streams."""
    import torch
    h_up = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_dn = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_up = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_dn = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()

    def both():
        with torch.cuda.stream(s_up):
            d_up.copy_(h_up, non_blocking=True)
        with torch.cuda.stream(s_dn):
            h_dn.copy_(d_dn, non_blocking=True)

    both()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        both()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    del h_up, h_dn, d_up, d_dn
    return 2 * nbytes / dt / 1e9


def gpu_smi_index(local_rank: int):
    """nvidia-smi index of this process's GPU: the entry of
    CUDA_VISIBLE_DEVICES, else the GPU whose UUID torch reports, else None."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if local_rank < len(ids):
        return ids[local_rank]
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            idx, u = [x.strip() for x in line.split(",")[:2]]
            if u.endswith(uuid) or uuid.endswith(u.replace("GPU-", "")):
                return idx
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 50 ms; `stop()`
    summarises the samples taken between `mark_start()` and `mark_end()`
    (wall clock), i.e. during the timed region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None
        self.out = os.path.join("/tmp", f"vx_clocks_{os.getpid()}.csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if gpu_index is not None:
            cmd += ["-i", str(gpu_index)]
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # wait for the first sample, so that the timed region is covered
        t_end = time.time() + 10.0
        while self.proc is not None and time.time() < t_end and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.out) > 0:
                break
            time.sleep(0.05)

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f")
                    rows.append((ts, float(p[2]), float(p[3]), [n for n, v in zip(names, p[6:10])
                                                                 if v.lower().startswith("active")]))
                except ValueError:
                    continue
        os.unlink(self.out)
        if not rows:
            return None
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        window = "timed region"
        if not inside:  # region shorter than the sampling period: nearest samples
            inside = sorted(rows, key=lambda r: abs((r[0] - (self.t0 or r[0])).total_seconds()))[:3]
            window = "samples nearest the timed region"
        reasons = sorted({n for r in inside for n in r[3]})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": float(max(r[2] for r in inside)),
                "reasons": reasons, "samples": len(inside), "window": window,
                "gpu": "nvidia-smi index " + str(self.gpu) if self.gpu is not None else "all GPUs (index unknown)"}


def _timed(torch, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


# ---------------------------------------------------------------------------
# Inputs
# ---------------------------------------------------------------------------
def make_inputs():
    import synth
    grid = synth.terrain_volume(SEED, N_VOL)
    cam = synth.camera(SEED + 1, N_VOL, WIDTH, HEIGHT, mode="above")
    inc = synth.incoherent_rays(SEED + 2, N_VOL, N_INC)
    return grid, cam, inc


_SCENE = None


def _scene2048():
    global _SCENE
    if _SCENE is None:
        import synth
        sc = synth.PrimitiveScene(SEED3, 2048)
        g8 = sc.render_u8()
        _SCENE = (sc, g8)
    return _SCENE


def batch_recipe(scale: float = 1.0):
    """The 64 ray sets of the batched workload: (k, size, kind, parameter)
    with kind "view" (a camera of about `size` pixels, 16:9) or
    "incoherent" (synth.incoherent_rays seed); set k belongs to
    BATCH_FORMATS[k % 4].  scale < 1 shrinks every set (a small case of the
    same workload, for profiler captures)."""
    import synth
    rng = np.random.default_rng(SEED3 + 4)
    sizes = np.exp(rng.uniform(np.log(65536), np.log(8388608), N_SETS))
    sizes = np.maximum(1024, sizes * scale).astype(np.int64)
    out = []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            h = max(1, int(round((int(n) * 9 / 16) ** 0.5)))
            w = max(1, int(n) // h)
            out.append((k, w * h, "view", synth.camera(SEED3 + 100 + k, 2048, w, h, mode="sphere")))
        else:
            out.append((k, int(n), "incoherent", SEED3 + 100 + k))
    return out


def batch_rays_device(vx, torch, recipe):
    import synth
    rays = []
    for k, n, kind, prm in recipe:
        if kind == "view":
            rays.append(vx.raygen_pinhole(prm))
        else:
            rays.append(torch.from_numpy(synth.incoherent_rays(prm, 2048, n)).cuda())
    return rays


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate_2048(g8, palette, recipe, budget_s: float, threads: int | None = None, seed: int = 5):
    """Times the FP64 oracle on samples of the batched workload's rays until
    about budget_s seconds of wall time: rounds of 1024 rays from each of the
    64 sets (camera rays from the oracle's own FP64 pinhole twin, incoherent
    rays from the seeded generator), so every set and both ray kinds are in
    the sample.  Returns (Mrays/s, threads, rays, seconds)."""
    import oracle
    import synth
    rng = np.random.default_rng(seed)
    pools = []
    for k, n, kind, prm in recipe:
        if kind == "view":
            r = oracle.pinhole(prm)
        else:
            r = synth.incoherent_rays(prm, 2048, n)
        pools.append(r[rng.permutation(len(r))[:16384]])
    done, t_used, used_threads, k = 0, 0.0, 1, 0
    per = 1024 if threads != 1 else 64
    while t_used < budget_s and (k + 1) * per <= 16384:
        sample = np.concatenate([p[k * per:(k + 1) * per] for p in pools])
        t0 = time.perf_counter()
        _, used_threads = oracle.trace_pal(g8, palette, sample, threads=threads)
        t_used += time.perf_counter() - t0
        done += len(sample)
        k += 1
    return done / t_used / 1e6, used_threads, done, t_used


def oracle_rate_512(grid, cam, inc, budget_s: float, threads: int | None = None):
    """Times the FP64 oracle on an interleaved sample of the 512^3 step's rays
    (half primary, half incoherent) until about budget_s seconds."""
    import oracle
    prim = oracle.pinhole(cam)
    rng = np.random.default_rng(5)
    pi = rng.permutation(len(prim))
    ii = rng.permutation(len(inc))
    chunk = max(20000, 2048 * (threads or os.cpu_count() or 1))
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
    """The reference arm: the FP64 oracle on the host cores, timed on bounded
    samples of the default workload's rays (the 2048^3 batched sets)."""
    rank, _, world = rank_info()
    if rank != 0:
        return 0
    import oracle
    oracle.lib()
    sc, g8 = _scene2048()
    recipe = batch_recipe()
    per_step = []
    budget = max(0.05, min(args.ref_step_s, 150.0 / (args.steps + args.warmup)))
    for s in range(args.warmup + args.steps):
        v, thr, n, t = oracle_rate_2048(g8, sc.palette, recipe, budget_s=budget, seed=100 + s)
        if s >= args.warmup:
            per_step.append((v, n, t))
    rays = sum(p[1] for p in per_step)
    secs = sum(p[2] for p in per_step)
    value = rays / secs / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "formats": BATCH_FORMATS, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{rays} rays over {args.steps} steps: per step rounds of 1024 rays from each "
                                   f"of the 64 batched sets (~{budget:.1f} s); the FP64 oracle walks the "
                                   f"uncompressed 2048^3 grid, so one timing serves every format"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Default workload: the 2048^3 scene
# ---------------------------------------------------------------------------
def run_headline(args):
    import torch
    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2410_14128_b300 as vx
    peak, peak_kind = load_peaks()

    sc, g8 = _scene2048()
    vols = [vx.Volume(s, g8, palette=sc.palette) for s in BATCH_FORMATS]
    recipe = batch_recipe(args.batch_scale)
    rays = batch_rays_device(vx, torch, recipe)
    sets = [(vols[k % len(vols)], rays[k], vx.alloc_hits(rays[k].shape[0])) for k in range(N_SETS)]
    total = sum(r.shape[0] for r in rays)

    # --- autotune each format on a sample of its own sets (outside timing) ---
    tuned, tuned_batch = [], []
    if not args.no_tune:
        for i, v in enumerate(vols):
            own = torch.cat([rays[k][: 1 << 17] for k in range(i, N_SETS, len(vols))])
            tuned.append(v.autotune(own))
        # the batched kernel's options per format, timed on its own 16 sets
        chosen = vx.autotune_batch(sets)
        tuned_batch = [chosen[i] for i in range(len(vols))]

    # --- algorithmic bytes per ray and footprint (instrumented kernel, outside timing) ---
    node_bytes, iters = [], []
    sects = [v.alloc_sectors() for v in vols]
    for k, (v, r, _) in enumerate(sets):
        c = torch.zeros(4, dtype=torch.int64, device="cuda")
        tmp = vx.alloc_hits(r.shape[0])
        v.trace_counted(r, tmp, c, sectors=sects[k % len(vols)])
        torch.cuda.synchronize()
        node_bytes.append(int(c[0]))
        iters.append(int(c[1]))
        del tmp
    footprint = [vx.Volume.footprint_bytes(s) for s in sects]
    del sects

    # --- the per-set paths, for comparison ---
    ref = [vx.alloc_hits(r.shape[0]) for r in rays]

    def plain():
        for (v, r, _), h in zip(sets, ref):
            v.trace(r, h, mode=vx.MODE_PLAIN)

    def per_set_auto():
        for v, r, h in sets:
            v.trace(r, h)

    ms_plain = _timed(torch, plain, 3, 2)
    ms_auto = _timed(torch, per_set_auto, 3, 2)

    # --- the batched step: one graph per timed step, each with its own
    # timing events around every group's kernel (on the stream it runs on) ---
    n_groups = len(vols)
    vx.trace_batch(sets)  # creates the library's fork streams outside capture
    torch.cuda.synchronize()
    ok_same = all(torch.equal(h, r) for (_, _, h), r in zip(sets, ref))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * n_groups)] for _ in range(args.steps)]
    for row in evs:
        for e in row:
            e.record()
    torch.cuda.synchronize()
    graphs = []
    for s in range(args.steps):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            got = vx.trace_batch(sets, events=evs[s])
        assert got == n_groups, (got, n_groups)
        graphs.append(g)
    for w in range(args.warmup):
        graphs[w % len(graphs)].replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    clocks = ClockSampler(gpu_smi_index(local))
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.mark_start()
    torch.cuda.nvtx.range_push("vx_timed")  # lets a profiler select the timed launches
    t_start.record()
    for s in range(args.steps):
        step_ev[s][0].record()
        graphs[s].replay()
        step_ev[s][1].record()
    t_end.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks.mark_end()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    local_ms = t_start.elapsed_time(t_end)
    value, total_ms = job_throughput(local_ms, total * args.steps, world, dist)
    ms_per_step = total_ms / args.steps
    group_ms = [[evs[s][2 * k].elapsed_time(evs[s][2 * k + 1]) for s in range(args.steps)] for k in range(n_groups)]
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    ok_same = ok_same and all(torch.equal(h, r) for (_, _, h), r in zip(sets, ref))
    del graphs
    # each group's kernel alone (its 16 sets in one uncaptured call), for the
    # kernel's own speed: inside the step it shares the SMs with the others
    group_alone_ms = []
    for k in range(n_groups):
        own = [sets[i] for i in range(k, N_SETS, len(vols))]
        pair = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        for e in pair:
            e.record()
        ts = []
        for rep in range(6):
            vx.trace_batch(own, events=pair)
            torch.cuda.synchronize()
            if rep >= 1:
                ts.append(pair[0].elapsed_time(pair[1]))
        group_alone_ms.append(float(np.mean(ts)))

    # --- roofline of the dominant kernel: the group whose kernel takes longest
    # alone (inside the step the concurrent kernels' intervals overlap, so the
    # longest interval there can belong to a group with less work) ---
    dom = int(np.argmax(group_alone_ms)) if group_alone_ms else int(np.argmax([np.mean(m) for m in group_ms]))
    g_sets = list(range(dom, N_SETS, len(vols)))
    g_rays = sum(rays[k].shape[0] for k in g_sets)
    alg = sum(node_bytes[k] + 48 * rays[k].shape[0] for k in g_sets)
    avg_ms = float(np.mean(group_ms[dom]))
    achieved = alg / (avg_ms / 1e3) / 1e9
    key = f"batch:{BATCH_FORMATS[dom].replace(' ', '')}:k_trace_batch"
    cnt = ncu_counters(key)
    traffic = cnt.get("dram_bytes")
    compulsory = footprint[dom] + 48 * g_rays
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "dram_frac": round(traffic / (avg_ms / 1e3) / 1e9 / peak, 4) if traffic else None,
                "l2_hit_rate_pct": cnt.get("l2_hit_pct"),
                "compulsory_bytes_per_launch": int(compulsory),
                "kernel": f"k_trace_batch {BATCH_FORMATS[dom]} (group {dom}: {len(g_sets)} sets, {g_rays} rays)",
                "alg_bytes_per_launch": int(alg),
                "alg_bytes_per_ray": round(alg / g_rays, 2),
                "avg_launch_ms": round(avg_ms, 4),
                "avg_launch_ms_alone": round(group_alone_ms[dom], 4),
                "frac_alone": round(alg / (group_alone_ms[dom] / 1e3) / 1e9 / peak, 4),
                "group_launch_ms": [round(float(np.mean(m)), 4) for m in group_ms],
                "group_launch_ms_alone": [round(t, 4) for t in group_alone_ms],
                "timing": "CUDA events recorded by vx_trace_batch_timed on each group's stream, inside the "
                          "graphs replayed in the timed region",
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    insts = cnt.get("warp_inst")
    roofline_issue = None
    if insts:
        ach = insts / (avg_ms / 1e3) / 1e9
        ach_alone = insts / (group_alone_ms[dom] / 1e3) / 1e9
        roofline_issue = {"bound": "issue", "achieved": round(ach, 2), "peak": round(ISSUE_PEAK_GINST_S, 2),
                          "unit": "Gwarp-inst/s", "frac": round(ach / ISSUE_PEAK_GINST_S, 4),
                          "achieved_alone": round(ach_alone, 2),
                          "frac_alone": round(ach_alone / ISSUE_PEAK_GINST_S, 4),
                          "warp_inst_per_launch": insts,
                          "peak_source": "148 SMs x 4 schedulers x 1 warp-inst/cycle x 2032 MHz (nominal)"}

    # --- end to end: every set from pinned host memory, one vx_trace_batch_host per step ---
    e2e = None
    if not args.no_e2e:
        from concurrent.futures import ThreadPoolExecutor
        host_rays = [r.cpu().pin_memory().numpy() for r in rays]
        host_hits = [torch.empty((r.shape[0], 4), dtype=torch.int32).pin_memory().numpy()
                     .view(vx.HIT_DTYPE).reshape(-1) for r in rays]
        host_items = [(vols[k % len(vols)], host_rays[k], host_hits[k]) for k in range(N_SETS)]

        def e2e_step():
            vx.trace_batch_host(host_items)

        def timed_host(step_fn):
            step_fn()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            n_e2e = max(1, min(args.steps, args.e2e_steps))
            t0 = time.perf_counter()
            for _ in range(n_e2e):
                step_fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if dist:
                t = torch.tensor([dt], device="cuda")
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                dt = float(t.item())
            return n_e2e, dt

        n_e2e, dt = timed_host(e2e_step)
        same_host = all(np.array_equal(host_hits[k].view(np.int32).reshape(-1, 4), ref[k].cpu().numpy())
                        for k in range(N_SETS))
        # the same sets one vx_trace_host call each (one host thread per volume), for comparison
        pool = ThreadPoolExecutor(max_workers=len(vols))

        def one_volume(i):  # each volume has its own staging buffers and streams
            for k in range(i, N_SETS, len(vols)):
                vols[i].trace_host(host_rays[k], out=host_hits[k])

        def per_set_step():
            for f in [pool.submit(one_volume, i) for i in range(len(vols))]:
                f.result()

        n_ps, dt_ps = timed_host(per_set_step)
        pool.shutdown()
        h2d, d2h = 32 * total, 16 * total
        pcie = pcie_both_ways_gbs()
        bound = total / ((h2d + d2h) / (pcie * 1e9)) / 1e6
        e2e_value = world * total * n_e2e / dt / 1e6
        e2e = {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": n_e2e, "results_identical": same_host,
               "pcie": {"bound": "pcie", "peak_gbs_both_ways": round(pcie, 1), "bound_mrays_s": round(bound, 1),
                        "frac": round(e2e_value / world / bound, 4),
                        "peak_source": "256 MiB pinned-host copies, one up and one down at once, timed here"},
               "api": "vx_trace_batch_host: the 64 sets from pinned host memory in one call per step (waves of "
                      "2^21 rays: upload, batched kernels and download of four waves overlapping), hits back "
                      "to pinned host memory",
               "per_set_vx_trace_host_mrays_s": round(world * total * n_ps / dt_ps / 1e6, 3)}
        del host_rays, host_hits, host_items

    # --- CPU baseline: the oracle on a bounded sample of the same rays ---
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, thr, n, t = oracle_rate_2048(g8, sc.palette, recipe, budget_s=args.cpu_budget_s)
        v1, _, n1, t1 = oracle_rate_2048(g8, sc.palette, recipe, budget_s=min(5.0, args.cpu_budget_s), threads=1)
        cpu = {"value": round(v, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{n} rays ({t:.1f} s): rounds of 1024 rays from each of the 64 batched sets (camera rays "
                         f"from the oracle's FP64 pinhole twin); the FP64 oracle walks the uncompressed 2048^3 grid",
               "single_core": {"value": round(v1, 4), "sample": f"{n1} rays, {t1:.1f} s on one thread"}}

    batch_formats = []
    for i, (s, v) in enumerate(zip(BATCH_FORMATS, vols)):
        st = v.stats()
        own = list(range(i, N_SETS, len(vols)))
        batch_formats.append({"format": s, "table2": LABEL.get(s), "device_bytes": st["device_bytes"],
                              "bytes_per_voxel": round(st["device_bytes"] / 2048 ** 3, 6),
                              "sets": len(own), "rays": int(sum(rays[k].shape[0] for k in own)),
                              "node_bytes_per_ray": round(sum(node_bytes[k] for k in own) /
                                                          sum(rays[k].shape[0] for k in own), 2),
                              "iters_per_ray": round(sum(iters[k] for k in own) /
                                                     sum(rays[k].shape[0] for k in own), 2),
                              "ray_kind": "camera views" if i % 2 == 0 else "incoherent",
                              "footprint_bytes": footprint[i],
                              "kernel_ms": round(float(np.mean(group_ms[i])), 4),
                              "specialized_kernel": st["specialized"]})
    for v in vols:
        v.free()
    del sets, rays, ref
    torch.cuda.empty_cache()

    # --- the sweep, serving and the 512^3 step (rank 0, after the timed region) ---
    per_format = sweep_formats(args, vx, torch, sc, g8, peak) if (rank == 0 and not args.no_sweep) else None
    serving = serve_rows(args, vx, torch, sc, g8, rhos=args.rhos, requests=args.requests,
                         warm=args.warm_requests) if (rank == 0 and not args.no_serve) else None
    t512 = None
    if rank == 0 and not args.no_512:
        a2 = argparse.Namespace(**vars(args))
        a2.steps, a2.warmup, a2.no_cpu_baseline = args.steps512, max(3, args.warmup), True
        t512 = run_terrain512(a2, emit=False)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + (f" (sets scaled by {args.batch_scale:g})" if args.batch_scale != 1.0
                                               else ""),
                       "formats": BATCH_FORMATS, "rays_per_step": total, "sets": N_SETS,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2: {32 * total / 1e9:.2f} GB of rays and {16 * total / 1e9:.2f} GB "
                             f"of hits per step (L2 126 MB)",
                       "hit_layout": "full 16 B", "graph": "one CUDA graph per timed step (vx_trace_batch_timed)",
                       "occupancy": round(sc.occupied / 2048 ** 3, 5),
                       "tuned_trace_opts": tuned or None, "tuned_batch_opts": tuned_batch or None},
            "batched": {"mrays_s": round(value, 2), "step_ms_median": round(float(np.median(step_ms)), 4),
                        "results_identical_to_plain": ok_same, "groups": n_groups},
            "plain_mrays_s": round(total / ms_plain / 1e3, 2),
            "per_set_autotuned_mrays_s": round(total / ms_auto / 1e3, 2),
            "speedup_vs_plain": round(ms_plain / ms_per_step, 3),
            "batch_formats": batch_formats,
            "per_format": per_format,
            "serving": serving,
            "roofline": roofline,
            "roofline_issue": roofline_issue,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "terrain512": t512,
            "gpu_launches": args.steps * n_groups,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def sweep_formats(args, vx, torch, sc, g8, peak):
    """Every 2048^3 format of Table 2 (and one more): size, Mrays/s of 8
    1080p views (vx_render_views: one launch; and one vx_render per view)
    and of 8 AO rays per primary hit (vx_trace,
    autotuned), algorithmic bytes per ray from the instrumented kernel and the
    achieved fraction of HBM bandwidth; stack vs restarting traversal."""
    import synth
    cams = [synth.camera(SEED3 + 10 + v, 2048, WIDTH, HEIGHT, mode="sphere") for v in range(8)]
    n_prim = WIDTH * HEIGHT
    per = []
    budget = int(args.sweep_budget_gb * (1 << 30))
    for spec in SWEEP_FORMATS:
        t0 = time.perf_counter()
        try:
            v = vx.Volume(spec, g8, palette=sc.palette)
        except vx.VxError as e:  # e.g. over 2^32 words (Sec. 3.3's 16 GiB limit)
            per.append({"format": spec, "skipped": str(e)})
            continue
        build_s = time.perf_counter() - t0
        st = v.stats()
        if st["device_bytes"] > budget:
            per.append({"format": spec, "skipped": f"{st['device_bytes'] / 2**30:.1f} GiB over the budget"})
            v.free()
            continue
        hits = [vx.alloc_hits(n_prim) for _ in cams]
        rays = [vx.raygen_pinhole(c) for c in cams]
        for c, h in zip(cams, hits):
            v.render(c, h)
        ao = torch.cat([vx.raygen_ao(r, h, seed=SEED3, spp=8) for r, h in zip(rays, hits)])
        ao_hits = vx.alloc_hits(ao.shape[0])
        tune = v.autotune(ao[: 1 << 20]) if not args.no_tune else None
        # the 8 views in one vx_render_views call (one launch), and one vx_render per view
        ms_prim = _timed(torch, lambda: v.render_views(cams, hits), args.sweep_steps, 1)
        ms_prim_each = _timed(torch, lambda: [v.render(c, h) for c, h in zip(cams, hits)], args.sweep_steps, 1)
        ms_ao = _timed(torch, lambda: v.trace(ao, ao_hits), args.sweep_steps, 1)
        n_ao_live = int((ao[:, 7] > 0).sum().item())
        # algorithmic bytes: node words the instrumented kernel reads, plus
        # the hit write (16 B) and, for traced rays, the ray read (32 B)
        prim = torch.cat(rays)
        c = torch.zeros(4, dtype=torch.int64, device="cuda")
        tmp = vx.alloc_hits(prim.shape[0])
        v.trace_counted(prim, tmp, c)
        torch.cuda.synchronize()
        nb_prim = int(c[0]) / prim.shape[0]
        c.zero_()
        v.trace_counted(ao, ao_hits, c)
        torch.cuda.synchronize()
        nb_ao = int(c[0]) / ao.shape[0]
        del tmp
        alg_prim = prim.shape[0] * (nb_prim + 16)
        alg_ao = ao.shape[0] * (nb_ao + 48)
        frac_prim = alg_prim / (ms_prim / 1e3) / 1e9 / peak
        frac_ao = alg_ao / (ms_ao / 1e3) / 1e9 / peak
        frac_all = (alg_prim + alg_ao) / ((ms_prim + ms_ao) / 1e3) / 1e9 / peak
        # node stack vs restarting traversal (Sec. 4.4) on the same rays
        trav = {}
        if not args.sweep_fast:
            prim_hits = vx.alloc_hits(prim.shape[0])
            for rs in (False, True):
                mp = _timed(torch, lambda: v.trace(prim, prim_hits, mode=vx.MODE_PLAIN, restart=rs),
                            args.sweep_steps, 1)
                ma = _timed(torch, lambda: v.trace(ao, ao_hits, mode=vx.MODE_PERSISTENT, restart=rs),
                            args.sweep_steps, 1)
                trav["restart" if rs else "stack"] = {"mrays_s_primary_plain": round(prim.shape[0] / mp / 1e3, 1),
                                                      "mrays_s_ao_persistent": round(ao.shape[0] / ma / 1e3, 1)}
            del prim_hits
        cnt = ncu_counters(f"ao:{spec.replace(' ', '')}:trace")
        per.append({"format": spec, "table2": LABEL.get(spec), "build_s": round(build_s, 1),
                    "device_bytes": st["device_bytes"], "packed": st["packed"],
                    "bytes_per_voxel": round(st["device_bytes"] / 2048 ** 3, 6),
                    "bytes_per_occupied_voxel": round(st["device_bytes"] / max(1, st["occupied_voxels"]), 4),
                    "mrays_s_primary": round(len(cams) * n_prim / ms_prim / 1e3, 1),
                    "mrays_s_primary_view_per_launch": round(len(cams) * n_prim / ms_prim_each / 1e3, 1),
                    "mrays_s_ao": round(ao.shape[0] / ms_ao / 1e3, 1),
                    "mrays_s": round((len(cams) * n_prim + ao.shape[0]) / (ms_prim + ms_ao) / 1e3, 1),
                    "ao_rays": int(ao.shape[0]), "ao_rays_live": n_ao_live,
                    "node_bytes_per_ray_primary": round(nb_prim, 2), "node_bytes_per_ray_ao": round(nb_ao, 2),
                    "hbm_frac": round(frac_all, 5), "hbm_frac_primary": round(frac_prim, 5),
                    "hbm_frac_ao": round(frac_ao, 5), "l2_hit_rate_pct": cnt.get("l2_hit_pct"),
                    "specialized_kernel": st["specialized"], "tuned": tune, "traversal": trav or None})
        del hits, rays, ao, ao_hits, prim
        v.free()
        torch.cuda.empty_cache()
    return per


def serve_rows(args, vx, torch, sc, g8, rhos, requests, warm):
    """Serving: Poisson render requests over 6 resident formats of the 512^3
    and 2048^3 volumes; continuous batching vs the serial plain path."""
    import synth
    from paper_2410_14128_b300 import serve
    grid, _, _ = make_inputs()
    vols = {"t512 R4S2G3": vx.Volume("R(4,4,4) S(2) G(3)", grid),
            "t512 R3R3R3": vx.Volume("R(3,3,3) R(3,3,3) R(3,3,3)", grid),
            "t512 R4G5": vx.Volume("R(4,4,4) G(5)", grid),
            "s2048 R3G8": vx.Volume("R(3,3,3) G(8)", g8, palette=sc.palette),
            "s2048 R4G7": vx.Volume("R(4,4,4) G(7)", g8, palette=sc.palette),
            "s2048 R4S3G4": vx.Volume("R(4,4,4) S(3) G(4)", g8, palette=sc.palette)}
    del grid
    names = sorted(vols)
    res_choices = [(256, 256), (512, 512), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]

    def make(count, rate, seed):
        r = np.random.default_rng(seed)
        t = np.cumsum(r.exponential(1.0 / rate, count)) if rate else np.zeros(count)
        out = []
        for i in range(count):
            name = names[int(r.integers(0, len(names)))]
            w, h = res_choices[int(r.integers(0, len(res_choices)))]
            side = 512 if name.startswith("t512") else 2048
            cam = synth.camera(seed * 100000 + i, side, w, h, mode="above" if side == 512 else "sphere")
            out.append(serve.Request(i, name, float(t[i]), camera=cam))
        return out

    # plain-path capacity: mean service time of one request, alone
    cal = make(60, 0, 1)
    serve.serve_serial(vols, cal[:10])
    t0 = time.perf_counter()
    serve.serve_serial(vols, cal)
    cap = len(cal) / (time.perf_counter() - t0)
    rows = []
    budget = int(args.serve_budget_gb * (1 << 30))
    arena = serve.HostArena(budget)  # pinned download space, shared by the servers below
    for rho in rhos:
        rate = rho * cap
        reqs = make(requests + warm, rate, int(rho * 1000))
        srv = serve.Server(vols, mem_budget_bytes=budget, keep_hits=False, digest_every=10, host_arena=arena)
        res = srv.run(reqs, realtime=True)
        ser = serve.serve_serial(vols, reqs, keep_hits=False, digest_every=10)
        keep = [r.id for r in reqs[warm:]]
        rs = {i: res[i] for i in keep}
        ss = {i: ser[i] for i in keep}
        rays = sum(reqs[i].n for i in keep)
        span = max(r.done for r in rs.values()) - min(r.arrival for r in rs.values())
        span_s = max(r.done for r in ss.values()) - min(r.arrival for r in ss.values())
        same = all(res[i].digest == ser[i].digest for i in keep if i % 10 == 0)
        rows.append({"rho": rho, "rate_req_s": round(rate, 1), "requests": len(keep),
                     "served": {"mrays_s": round(rays / span / 1e6, 1), **serve.latency_stats(rs),
                                "epochs": srv.epochs, "max_inflight_seen": srv.max_inflight_seen},
                     "serial_plain": {"mrays_s": round(rays / span_s / 1e6, 1), **serve.latency_stats(ss)},
                     "results_identical": same})
    # saturated: every request due at t = 0 (throughput of both paths)
    reqs = make(requests, 0, 7)
    srv = serve.Server(vols, mem_budget_bytes=budget, keep_hits=False, digest_every=10, host_arena=arena)
    res = srv.run(reqs, realtime=False)
    ser = serve.serve_serial(vols, reqs, keep_hits=False, digest_every=10)
    rays = sum(r.n for r in reqs)
    rows.append({"rho": "saturated", "requests": len(reqs),
                 "served": {"mrays_s": round(rays / max(r.done for r in res.values()) / 1e6, 1),
                            **serve.latency_stats(res), "epochs": srv.epochs,
                            "max_inflight_seen": srv.max_inflight_seen},
                 "serial_plain": {"mrays_s": round(rays / max(r.done for r in ser.values()) / 1e6, 1),
                                  **serve.latency_stats(ser)},
                 "results_identical": all(res[i].digest == ser[i].digest for i in res if i % 10 == 0)})
    for v in vols.values():
        v.free()
    del arena
    torch.cuda.empty_cache()
    return {"workload": "Poisson render requests (256^2..3840x2160, uniform), random format among 6 resident "
                        "(3 on the 512^3 terrain, 3 on the 2048^3 scene); served = continuous batching "
                        f"({args.serve_budget_gb:g} GiB device budget), serial = one request at a time (plain)",
            "plain_capacity_req_s": round(cap, 1), "rows": rows}


# ---------------------------------------------------------------------------
# The 512^3 terrain step
# ---------------------------------------------------------------------------
def run_terrain512(args, emit=True):
    import torch
    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1 and emit:
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
    fixed = {"sort": args.sort} if args.sort and mode != vx.MODE_AUTO else {}  # fixed options (no autotuning)

    # --- autotune the incoherent-ray trace per format (outside timing) ---
    tuned = []
    if mode == vx.MODE_AUTO and not args.no_tune:
        for v in vols:
            tuned.append(v.autotune(inc))

    # --- algorithmic bytes per ray (instrumented kernels, outside timing) ---
    counts = {}
    prim_rays = vx.raygen_pinhole(cam)
    for k, v in enumerate(vols):
        for name, rays in (("render", prim_rays), ("trace", inc)):
            c = torch.zeros(4, dtype=torch.int64, device="cuda")
            sect = v.alloc_sectors()
            tmp = vx.alloc_hits(rays.shape[0])
            v.trace_counted(rays, tmp, c, sectors=sect)
            torch.cuda.synchronize()
            b, it, d, _ = (int(x) for x in c.cpu())
            n = rays.shape[0]
            counts[(k, name)] = {"node_bytes_per_ray": b / n, "iters_per_ray": it / n, "fp64_per_ray": d / n,
                                 "footprint_bytes": vx.Volume.footprint_bytes(sect)}
            del sect
    del prim_rays

    # The step's four launches are independent: the renders go on the main
    # stream and the traces on a second one, so a launch's tail (its last
    # warps, while most SMs have run out of rays) overlaps the next launch of
    # the other stream.  Both start after the L2 flush; the main stream waits
    # for the traces before the step ends.
    side = torch.cuda.Stream()

    def step(evs=None, mode=mode):
        flush.zero_()
        main = torch.cuda.current_stream()
        flushed = torch.cuda.Event()
        flushed.record(main)
        side.wait_event(flushed)
        for k, v in enumerate(vols):
            for name, st in (("render", main), ("trace", side)):
                with torch.cuda.stream(st):
                    if evs is not None:
                        evs[(k, name)][0].record(st)
                    if name == "render":
                        v.render(cam, hits_p[k])
                    else:
                        v.trace(inc, hits_i[k], mode=mode, **fixed)
                    if evs is not None:
                        evs[(k, name)][1].record(st)
        traced = torch.cuda.Event()
        traced.record(side)
        main.wait_event(traced)

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
    clocks = ClockSampler(gpu_smi_index(local)) if emit else None
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if clocks:
        clocks.mark_start()
    torch.cuda.nvtx.range_push("vx_timed")  # lets a profiler select the timed launches
    t_start.record()
    for s in range(args.steps):
        step(all_evs[s])
    t_end.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_end()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    local_ms = t_start.elapsed_time(t_end)
    for e in all_evs:
        for key, (a, b) in e.items():
            ev[key].append(a.elapsed_time(b))
    value, total_ms = job_throughput(local_ms, rays_per_step * args.steps, world, dist)
    ms_per_step = total_ms / args.steps

    # --- per-format results and the roofline of the dominant kernel ---
    peak, peak_kind = load_peaks()
    # Each launch alone (after the timed region; L2 flushed before each), for
    # the kernels' own speed: inside the step they share the GPU with the
    # other stream's launches.
    alone = {}
    for key in counts:
        k, name = key
        ts = []
        for r in range(12):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if name == "render":
                vols[k].render(cam, hits_p[k])
            else:
                vols[k].trace(inc, hits_i[k], mode=mode, **fixed)
            b.record()
            ts.append((a, b))
        torch.cuda.synchronize()
        alone[key] = float(np.mean([a.elapsed_time(b) for a, b in ts[2:]]))

    per_format = []
    tot = {}
    for k, spec in enumerate(FORMATS):
        st = vols[k].stats()
        ms_r = float(np.mean(ev[(k, "render")]))
        ms_t = float(np.mean(ev[(k, "trace")]))
        tot[(k, "render")] = sum(ev[(k, "render")])
        tot[(k, "trace")] = sum(ev[(k, "trace")])
        alg_r = n_prim * (counts[(k, "render")]["node_bytes_per_ray"] + 16)
        alg_t = N_INC * (counts[(k, "trace")]["node_bytes_per_ray"] + 48)
        per_format.append({
            "format": spec,
            "mrays_s_primary": round(n_prim / ms_r / 1e3, 2),
            "mrays_s_incoherent": round(N_INC / ms_t / 1e3, 2),
            "mrays_s": round((n_prim + N_INC) / (ms_r + ms_t) / 1e3, 2),
            "mrays_s_primary_alone": round(n_prim / alone[(k, "render")] / 1e3, 2),
            "mrays_s_incoherent_alone": round(N_INC / alone[(k, "trace")] / 1e3, 2),
            "hbm_frac": round((alg_r + alg_t) / ((ms_r + ms_t) / 1e3) / 1e9 / peak, 5),
            "device_bytes": st["device_bytes"],
            "bytes_per_voxel": round(st["device_bytes"] / N_VOL ** 3, 5),
            "bytes_per_occupied_voxel": round(st["device_bytes"] / max(1, st["occupied_voxels"]), 4),
            "node_bytes_per_ray_primary": round(counts[(k, "render")]["node_bytes_per_ray"], 2),
            "node_bytes_per_ray_incoherent": round(counts[(k, "trace")]["node_bytes_per_ray"], 2),
            "iters_per_ray_incoherent": round(counts[(k, "trace")]["iters_per_ray"], 2),
            "fp64_decisions_per_ray_incoherent": round(counts[(k, "trace")]["fp64_per_ray"], 5),
            "format_footprint_bytes_incoherent": counts[(k, "trace")]["footprint_bytes"],
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
    if name == "render":
        kname = "k_render"
    else:
        persistent = mode == vx.MODE_PERSISTENT or (mode == vx.MODE_AUTO and (not tuned or tuned[k]["mode"] == "persistent"))
        kname = "k_trace_persistent" if persistent else "k_trace"
        g_sort = tuned[k]["sort_cell_log2"] if tuned else fixed.get("sort", 0)
        if g_sort:
            # the sort key keeps at most 5 bits of the origin cell per axis, so
            # every g below log2(grid) - 5 gives the same key, permutation and
            # trace as g = log2(grid) - 5: name the counters by that g
            g_eff = max(g_sort, (N_VOL.bit_length() - 1) - 5)
            kname += f"+sort{g_eff}"  # the trace of the sorted copy of the rays
    # counters of the same kernel on the same format (a capture of another
    # kernel does not count)
    kernel_key = f"{name}:{FORMATS[k].replace(' ', '')}:{kname}"
    cnt = ncu_counters(kernel_key)
    traffic, insts = cnt.get("dram_bytes"), cnt.get("warp_inst")
    # compulsory bytes: the distinct 32-byte sectors of the format the launch
    # reads (sector bitmap of the instrumented kernel) plus the ray/hit I/O,
    # the least DRAM traffic a launch with cold caches can have
    compulsory = counts[dom]["footprint_bytes"] + n_rays * io
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "dram_frac": round(traffic / (avg_ms / 1e3) / 1e9 / peak, 4) if traffic else None,
                "l2_hit_rate_pct": cnt.get("l2_hit_pct"),
                "compulsory_bytes_per_launch": int(compulsory),
                "kernel": f"{kname} {FORMATS[k]}",
                "alg_bytes_per_launch": int(alg_bytes), "avg_launch_ms": round(avg_ms, 4),
                "avg_launch_ms_alone": round(alone[dom], 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    # The traversal is a chain of dependent small reads that mostly hit in L1/L2,
    # so the unit that limits it is instruction issue: warp instructions per
    # launch (same ncu capture) over the live launch time, against the peak.
    roofline_issue = None
    if insts:
        ach = insts / (avg_ms / 1e3) / 1e9
        ach_alone = insts / (alone[dom] / 1e3) / 1e9
        roofline_issue = {"bound": "issue", "achieved": round(ach, 2), "peak": round(ISSUE_PEAK_GINST_S, 2),
                          "unit": "Gwarp-inst/s", "frac": round(ach / ISSUE_PEAK_GINST_S, 4),
                          "achieved_alone": round(ach_alone, 2),
                          "frac_alone": round(ach_alone / ISSUE_PEAK_GINST_S, 4),
                          "warp_inst_per_launch": insts,
                          "peak_source": "148 SMs x 4 schedulers x 1 warp-inst/cycle x 2032 MHz (nominal)"}

    # --- end to end through the host-memory entry points ---
    e2e = None
    if not args.no_e2e:
        from concurrent.futures import ThreadPoolExecutor
        pin_rays = torch.from_numpy(inc_np).pin_memory().numpy()

        def pinned_hits(n):
            return torch.empty((n, 4), dtype=torch.int32).pin_memory().numpy().view(vx.HIT_DTYPE).reshape(-1)

        outs = [(pinned_hits(n_prim), pinned_hits(N_INC)) for _ in vols]
        # one host thread per volume: the calls block, and each volume has its
        # own staging buffers and streams (the library releases the GIL during
        # its calls).  A render only downloads and a trace mostly uploads, so
        # alternate volumes take them in opposite orders: one volume's render
        # downloads while the other's trace uploads, and both PCIe directions
        # stay busy for the whole step.
        pool = ThreadPoolExecutor(max_workers=len(vols))

        def one_volume(k):
            if k % 2 == 0:
                vols[k].render_host(cam, out=outs[k][0])
                vols[k].trace_host(pin_rays, out=outs[k][1])
            else:
                vols[k].trace_host(pin_rays, out=outs[k][1])
                vols[k].render_host(cam, out=outs[k][0])

        def e2e_step():
            for f in [pool.submit(one_volume, k) for k in range(len(vols))]:
                f.result()

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        n_e2e = min(args.steps, 50)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        h2d = len(FORMATS) * N_INC * 32
        d2h = len(FORMATS) * (n_prim + N_INC) * 16
        # The bound of this path is PCIe: the step's bytes over the copy rate
        # with both directions busy at once, measured here with plain copies.
        pcie = pcie_both_ways_gbs()
        bound = rays_per_step / ((h2d + d2h) / (pcie * 1e9)) / 1e6
        e2e_value = world * rays_per_step * n_e2e / dt / 1e6
        e2e = {"value": round(e2e_value, 3), "unit": UNIT,
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e,
               "pcie": {"bound": "pcie", "peak_gbs_both_ways": round(pcie, 1),
                        "bound_mrays_s": round(bound, 1), "frac": round(e2e_value / world / bound, 4),
                        "peak_source": "256 MiB pinned-host copies, one up and one down at once, timed here"},
               "api": "vx_render_host + vx_trace_host, pinned host buffers, one host thread per volume "
                      "(alternate volumes render first / trace first)"}
        pool.shutdown()

    # --- CPU baseline: the oracle on a bounded sample ---
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, thr, n, t = oracle_rate_512(grid, cam, inc_np, budget_s=args.cpu_budget_s)
        v1, _, n1, t1 = oracle_rate_512(grid, cam, inc_np, budget_s=min(5.0, args.cpu_budget_s), threads=1)
        cpu = {"value": round(v, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{n} rays of the step (half pinhole, half incoherent), {t:.1f} s of FP64 oracle on "
                         f"the uncompressed 512^3 grid; format-independent",
               "single_core": {"value": round(v1, 4), "sample": f"{n1} rays, {t1:.1f} s on one thread"}}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD512, "formats": FORMATS, "rays_per_step": rays_per_step,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"flushed before each step by a {FLUSH_BYTES >> 20} MiB write (inside the timed region)",
                   "hit_layout": "full 16 B",
                   "streams": "renders on one stream, traces on a second, overlapping within the step",
                   "mode": {"auto": "auto (vx_trace options autotuned per format on the incoherent rays, outside the timed region)",
                            "plain": "plain (one thread per ray)",
                            "persistent": "persistent warps with ray refill"}[args.mode]},
        "plain_kernel_ms_per_step": round(plain_ms, 4) if plain_ms else None,
        "plain_mrays_s": round(rays_per_step / plain_ms / 1e3, 2) if plain_ms else None,
        "per_format": per_format,
        "roofline": roofline,
        "roofline_issue": roofline_issue,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * sum(1 + trace_launches(tuned[k] if tuned else {"sort_cell_log2": fixed.get("sort", 0)},
                                                            vols[k].log2_dim)
                                         for k in range(len(FORMATS))),
        "clocks": clk,
    }
    for v in vols:
        v.free()
    del flush
    torch.cuda.empty_cache()
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return line if not emit else 0


# ---------------------------------------------------------------------------
# Other workloads (one JSON line each)
# ---------------------------------------------------------------------------
def run_sweep(args):
    """The 2048^3 Table 2 sweep as its own line."""
    import torch
    import paper_2410_14128_b300 as vx
    sc, g8 = _scene2048()
    peak, _ = load_peaks()
    per = sweep_formats(args, vx, torch, sc, g8, peak)
    ok = [p for p in per if "skipped" not in p]
    tot_rays = sum(8 * WIDTH * HEIGHT + p["ao_rays"] for p in ok)
    tot_ms = sum(8 * WIDTH * HEIGHT / p["mrays_s_primary"] / 1e3 + p["ao_rays"] / p["mrays_s_ao"] / 1e3 for p in ok)
    print(json.dumps({"metric": METRIC, "workload": "sweep2048", "value": round(tot_rays / tot_ms / 1e3, 2),
                      "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "2048^3 primitive scene (20k spheres/boxes/walls + 64 stamped 64^3 "
                                             "prototypes, ~2% occupied); 8 1920x1080 views + 8 AO rays per hit "
                                             "(cosine-weighted, tmax 32) per format",
                                 "occupancy": round(sc.occupied / 2048 ** 3, 5)},
                      "per_format": per}), flush=True)
    return 0


def run_formats512(args):
    """Every 512^3 format of Table 2 (plus the headline R(4,4,4) S(2) G(3)) on
    the 512^3 terrain: size, build time, and Mrays/s of the 1080p view and of
    the 2^21 incoherent rays (autotuned), so speed can be read against
    bytes per voxel as in the paper's trade-off plots."""
    import torch
    import paper_2410_14128_b300 as vx
    grid, cam, inc_np = make_inputs()
    inc = torch.from_numpy(inc_np).cuda()
    n_prim = WIDTH * HEIGHT
    hp, hi = vx.alloc_hits(n_prim), vx.alloc_hits(N_INC)
    per = []
    for spec in list(TABLE2_512.values()) + ["R(4,4,4) S(2) G(3)"]:
        t0 = time.perf_counter()
        v = vx.Volume(spec, grid)
        build_s = time.perf_counter() - t0
        st = v.stats()
        tune = v.autotune(inc) if not args.no_tune else None
        ms_r = _timed(torch, lambda: v.render(cam, hp), args.steps, args.warmup)
        ms_t = _timed(torch, lambda: v.trace(inc, hi), args.steps, args.warmup)
        c = torch.zeros(4, dtype=torch.int64, device="cuda")
        sect = v.alloc_sectors()
        v.trace_counted(inc, hi, c, sectors=sect)
        torch.cuda.synchronize()
        b, it, _, _ = (int(x) for x in c.cpu())
        per.append({"format": spec, "table2": LABEL.get(spec), "build_s": round(build_s, 2),
                    "format_footprint_bytes_incoherent": vx.Volume.footprint_bytes(sect),
                    "device_bytes": st["device_bytes"], "canonical_bytes": st["canonical_bytes"],
                    "bytes_per_voxel": round(st["device_bytes"] / N_VOL ** 3, 5),
                    "specialized_kernel": st["specialized"],
                    "mrays_s_primary": round(n_prim / ms_r / 1e3, 1), "mrays_s_incoherent": round(N_INC / ms_t / 1e3, 1),
                    "mrays_s": round((n_prim + N_INC) / (ms_r + ms_t) / 1e3, 1),
                    "node_bytes_per_ray_incoherent": round(b / N_INC, 2), "iters_per_ray_incoherent": round(it / N_INC, 2),
                    "tuned": tune})
        v.free()
        torch.cuda.empty_cache()
    tot_ms = sum((n_prim + N_INC) / p["mrays_s"] / 1e3 for p in per)
    print(json.dumps({"metric": METRIC, "workload": "formats512", "value": round(len(per) * (n_prim + N_INC) / tot_ms / 1e3, 2),
                      "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "512^3 terrain; every Table 2 512^3 format; per format one 1920x1080 "
                                             "view + 2^21 incoherent rays", "steps": args.steps},
                      "per_format": per}), flush=True)
    return 0


def run_dedup(args):
    """De-duplication scope (Sec. 4.3): every Table 2 format with an SVDAG
    level, built with one map per sub-volume (the paper's default) and with
    one map per level; sizes only (host build, no GPU)."""
    import paper_2410_14128_b300 as vx
    rows = []

    def measure(spec, grid, palette, scene):
        r = {"format": spec, "table2": LABEL.get(spec), "scene": scene}
        for name, scope in (("per_subvolume", vx.DEDUP_PER_SUBVOLUME), ("whole_level", vx.DEDUP_WHOLE_LEVEL)):
            t0 = time.perf_counter()
            v = vx.Volume(spec, grid, palette=palette, dedup=scope, upload=False)
            st = v.stats()
            r[name] = {"bytes": st["canonical_bytes"], "build_s": round(time.perf_counter() - t0, 2),
                       "level_bytes": [4 * w for w in st["level_words"]]}
            v.free()
        r["whole_over_per"] = round(r["whole_level"]["bytes"] / r["per_subvolume"]["bytes"], 4)
        rows.append(r)

    grid, _, _ = make_inputs()
    for spec in TABLE2_512.values():
        if "G(" in spec:
            measure(spec, grid, None, "512^3 terrain")
    del grid
    sc, g8 = _scene2048()
    for spec in TABLE2_2048.values():
        if "G(" in spec:
            measure(spec, g8, sc.palette, "2048^3 primitive scene")
    print(json.dumps({"workload": "dedup", "metric": "canonical bytes per de-duplication scope",
                      "data": "synthetic", "rows": rows}), flush=True)
    return 0


def _buildmem_one(spec: str):
    """Child process: builds `spec` from the 2048^3 scene brick by brick
    (the lazy voxelizer of Sec. 5) and prints its peak resident memory."""
    import resource
    import synth
    import paper_2410_14128_b300 as vx
    sc = synth.PrimitiveScene(SEED3, 2048)
    base = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss
    t0 = time.perf_counter()
    v = vx.Volume(spec, log2_dim=(11, 11, 11), fill_brick=sc.fill_brick_fn, block_empty=sc.block_empty_fn,
                  user=sc.handle, upload=False)
    dt = time.perf_counter() - t0
    st = v.stats()
    peak = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss
    print(json.dumps({"format": spec, "build_s": round(dt, 1), "canonical_bytes": st["canonical_bytes"],
                      "peak_rss_bytes": peak * 1024, "rss_before_build_bytes": base * 1024}), flush=True)
    return 0


def run_buildmem(args):
    """Out-of-core construction (Sec. 5): each 2048^3 format of the sweep is
    built in its own process from 64^3 bricks produced on demand, and the
    process's peak resident memory is recorded (the dense grid would take
    32 GiB as RGBA words)."""
    rows = []
    for spec in SWEEP_FORMATS:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--buildmem-spec", spec],
                             capture_output=True, text=True)
        if out.returncode != 0:
            rows.append({"format": spec, "error": out.stderr.strip().splitlines()[-1:]})
            continue
        r = json.loads(out.stdout.strip().splitlines()[-1])
        r["table2"] = LABEL.get(spec)
        rows.append(r)
    print(json.dumps({"workload": "buildmem", "metric": "peak resident memory of a brick-by-brick build",
                      "data": "synthetic", "dense_rgba_bytes": 4 * 2048 ** 3, "rows": rows}), flush=True)
    return 0


def run_serve(args):
    """The serving measurement as its own line."""
    import torch
    import paper_2410_14128_b300 as vx
    sc, g8 = _scene2048()
    out = serve_rows(args, vx, torch, sc, g8, rhos=args.rhos, requests=args.requests, warm=args.warm_requests)
    best = max(r["served"]["mrays_s"] for r in out["rows"])
    print(json.dumps({"metric": METRIC, "workload": "serve", "value": best, "unit": UNIT, "n_gpus": 1,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic", **out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="scene2048",
                    choices=["scene2048", "terrain512", "formats512", "sweep2048", "batch", "serve", "dedup",
                             "buildmem"])
    ap.add_argument("--mode", default="auto", choices=["auto", "plain", "persistent"],
                    help="terrain512: trace mode of the incoherent rays")
    ap.add_argument("--sort", type=int, default=0,
                    help="terrain512 with --mode plain/persistent: sort the incoherent rays by origin cells of side 2^G")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-512", action="store_true")
    ap.add_argument("--steps512", type=int, default=100)
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="shrink the 64 batched sets (a small case for profiler captures; the line says so)")
    ap.add_argument("--sweep-steps", type=int, default=3)
    ap.add_argument("--sweep-fast", action="store_true", help="skip the stack vs restart columns of the sweep")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--buildmem-spec", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--sweep-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--warm-requests", type=int, default=200)
    ap.add_argument("--rhos", type=float, nargs="+", default=[0.8])
    args = ap.parse_args()
    if args.buildmem_spec:
        return _buildmem_one(args.buildmem_spec)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "dedup":
        return run_dedup(args)
    if args.workload == "buildmem":
        return run_buildmem(args)
    if args.workload == "sweep2048":
        return run_sweep(args)
    if args.workload == "formats512":
        return run_formats512(args)
    if args.workload == "batch":
        a = argparse.Namespace(**vars(args))
        a.no_sweep = a.no_serve = a.no_512 = True
        return run_headline(a)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "terrain512":
        return run_terrain512(args)
    return run_headline(args)


if __name__ == "__main__":
    sys.exit(main())
