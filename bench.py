"""Benchmark of the fused two-species PM step (particle-steps per second).

Workload (default): two-level PM, 256^3 fine mesh, coarse ratio 4 (64^3
coarse mesh), 64 fine tiles of 64^3 interior + 16-cell buffer (96^3 FFTs),
128^3 Zel'dovich CDM + 256^3 Fermi-Dirac neutrinos (18.9M particles),
compressed state with 8-bit offsets and 8-bit velocities, float32 math.
One step = decompress + deposit, coarse and tile solves, interpolate + kick
+ drift + recompress of both species (pm_step), codes -> codes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
  python bench.py --workload largest1536 --tuning JSON   # 1536^3, 4.08e9 particles

Under torchrun each rank runs an independent replica of the workload (the
path shards by independent problems; no data-path collective): value is the
particle-steps of all ranks divided by the slowest rank's time.
--impl reference times the oracle (plain float64 numpy restatement of the
method) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "particle-steps/s (CDM+nu) per PM step"
UNIT = "particle-steps/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_rate(local_seconds, units_per_rank, world, device="cpu", dist=None):
    """Whole-job throughput of a weak-scaled replica run: the units of all ranks
    divided by the slowest rank's time (max over ranks).  Returns (rate, max_s)."""
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    worst = float(t.item())
    return units_per_rank * world / worst, worst


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def algorithmic_bytes(cfg, counts, vel_bits):
    """Algorithmic bytes per launch of each kernel kind: what the method itself
    must move (per-unit figures of the design notes), not the scratch or
    padding of this implementation."""
    nf, t, b = cfg["n_fine"], cfg["tile"], cfg["buffer"]
    T = t + 2 * b
    NH = T // 2 + 1
    vb = 2 if vel_bits == 16 else 1
    N = sum(counts)
    n_tiles = (nf // t) ** 3
    batch = min(cfg.get("tile_batch", 0) or 1024, n_tiles)
    nc = nf // cfg["coarse_ratio"]
    ncell = (nf // cfg["cmp_ratio"]) ** 3
    per_tile_a = T ** 3 * 4 + T * T * NH * 8
    per_tile_b = T * T * NH * 8 + 3 * t * T * NH * 8
    per_tile_c = 3 * t * T * NH * 8 + 3 * t ** 3 * 4
    return {
        "fft_a_tiles": batch * per_tile_a,
        "fft_b_tiles": batch * per_tile_b,
        "fft_c_tiles": batch * per_tile_c,
        # 3 B of position codes per particle and the count bytes read; fine + coarse density written
        "deposit": N * 3 + 2 * ncell + (nf ** 3 + nc ** 3) * 4,
        # position + velocity codes read, fine + coarse acceleration read
        "ikd_count": N * 3 * (1 + vb) + 12 * (nf ** 3 + nc ** 3),
        # position + velocity codes written
        "ikd_scatter": N * 3 * (1 + vb),
        # position codes read, one float32 acceleration triple written per particle
        "pp": N * 15,
    }


def step_model_bytes(cfg, counts, vel_bits):
    """Whole-step byte model of the method (per step): 3 B of position codes
    read by the deposit plus the codes read and written by the update (15 B
    per particle with 8-bit velocities, 21 B with 16-bit); 40 B per cell of
    every buffered tile and of the coarse mesh (density write + read,
    spectrum write + read, force write + read); the kernels read once (2 B per
    coarse cell, 3 x 4 x T^2 (T/2 + 1) B for the tile kernel)."""
    nf, t, b = cfg["n_fine"], cfg["tile"], cfg["buffer"]
    T = t + 2 * b
    per_particle = 3 + 2 * (3 + 3 * (2 if vel_bits == 16 else 1))
    if cfg.get("coarse_ratio", 1) > 1:
        nc = nf // cfg["coarse_ratio"]
        cells = (nf // t) ** 3 * T ** 3 + nc ** 3
        kernels = 2 * nc ** 3 + 3 * 4 * T * T * (T // 2 + 1)
    else:
        cells = nf ** 3
        kernels = 3 * 4 * nf * nf * (nf // 2 + 1)
    return sum(counts) * per_particle + 40 * cells + kernels


def csrc_digest():
    """Digest of the CUDA sources; ncu traffic figures apply only to the sources they were taken on."""
    import glob
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1611_01545_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind):
    """DRAM bytes per launch of a kernel kind from the committed ncu summary, or
    None when the kernels changed since that capture."""
    path = os.path.join(ROOT, "profiles", "step_kernels_two_level256_ncu.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    digest = csrc_digest()
    for ln in lines:
        parts = ln.split()
        if len(parts) == 4 and parts[0] == "traffic" and parts[1] == kind and parts[3] == f"csrc={digest}":
            return int(parts[2])
    return None


def build_state(pm, w, torch):
    import torch as _t  # noqa: F401
    codes = []
    for s in range(2):
        x = torch.from_numpy(w.x[s]).cuda()
        v = torch.from_numpy(w.v[s]).cuda()
        cap = max(64, w.x[s].shape[0] // 255 + 1)
        out = pm.empty_codes(w.x[s].shape[0], esc_cap=cap)
        pm.compress(s, x, v, out=out)
        codes.append(out)
        del x, v
    pm.check()
    spare = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in codes]
    return codes, spare


# Largest one-GPU workload: two-level PM on a 1536^3 fine mesh (384^3 coarse,
# 13,824 tiles of 64^3 + 16), 768^3 Zel'dovich CDM + 1536^3 Fermi-Dirac
# neutrinos (4.08e9 particles, 16-bit velocities), drawn on the device.
LARGEST = dict(n_fine=1536, coarse_ratio=4, tile=64, buffer=16, cmp_ratio=4, vel_bits=16, n_cdm=768, n_nu=1536,
               r_cut=14.0, seed=1619)


def largest_config(tile_batch=64):
    L = LARGEST
    return dict(n_fine=L["n_fine"], coarse_ratio=L["coarse_ratio"], tile=L["tile"], buffer=L["buffer"],
                cmp_ratio=L["cmp_ratio"], vel_bits=L["vel_bits"], G=1.0 / (4.0 * np.pi), mass=(8.0, 0.04),
                count=(L["n_cdm"] ** 3, L["n_nu"] ** 3), r_split=L["r_cut"] / 4.5, r_cut=L["r_cut"],
                tile_batch=tile_batch)


def build_largest_codes(pm, torch):
    """The largest workload's compressed state, built on the device: the CDM
    set compressed whole; the neutrinos one z slab of compression cells at a
    time (each slab's codes copied into place), with the species' v_max found
    over all slabs first.  No host array holds the particles."""
    from synth import device as dev
    L = LARGEST
    nf, ncmp = L["n_fine"], L["n_fine"] // L["cmp_ratio"]
    ncell_slab = ncmp * ncmp
    codes = []
    x, v = dev.zeldovich_lattice(L["seed"], L["n_cdm"], nf)
    c0 = pm.empty_codes(x.shape[0], esc_cap=x.shape[0] // 255 + 1)
    pm.compress(0, x, v, out=c0)
    del x, v
    codes.append(c0)
    n_nu = L["n_nu"] ** 3
    per = n_nu // ncmp
    seed = L["seed"] + 1
    vmax = torch.zeros(1, dtype=torch.float32, device="cuda")
    for k in range(ncmp):
        vmax = torch.maximum(vmax, dev.neutrino_slab(seed, k, ncmp, per, nf, velocities_only=True).abs().max())
    c1 = pm.empty_codes(n_nu, esc_cap=n_nu // 255 + 1)
    c1.vmax.copy_(vmax)
    slab = pm.empty_codes(per, esc_cap=per // 255 + 1)
    for k in range(ncmp):
        x, v = dev.neutrino_slab(seed, k, ncmp, per, nf)
        pm.compress(1, x, v, vmax=vmax, out=slab)
        lo = k * ncell_slab
        c1.cnt[lo:lo + ncell_slab].copy_(slab.cnt[lo:lo + ncell_slab])
        c1.pos[k * per:(k + 1) * per].copy_(slab.pos)
        c1.vel[k * per:(k + 1) * per].copy_(slab.vel)
        if int(slab.n_esc.item()) != 0:
            raise RuntimeError("a neutrino slab produced escape entries; the slab assembly does not merge them")
    del x, v, slab
    codes.append(c1)
    pm.check()
    return codes


def codes_bytes(c, vel_bits, packed=False):
    """Bytes of one species' codes: packed record bytes (3 + 3 or 6 per particle)
    or the padded in-memory words (4 + 4 or 8), plus counts, escapes and v_max."""
    vb = 2 if vel_bits == 16 else 1
    per = 3 * (1 + vb) if packed else 4 * (1 + vb)
    return c.cnt.numel() + c.esc.numel() * 4 + 4 + c.n * per + 4


def timed_loop(torch, stream, fn, steps: int) -> float:
    """Milliseconds of `steps` calls of fn, CUDA events on the launching stream."""
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def plain_step_ms(pm, w, codes, spare, torch, stream, steps: int) -> float:
    """The plain form of one step, one library call per stage: decompress each
    species, deposit (global float atomics), coarse + tile solve, interpolate +
    kick + drift, compress; like the fused step, every step maps `codes` to
    `spare`.  Returns milliseconds per step."""
    ac, af = pm.zeros_acc()
    rc, rf = pm.zeros_meshes()

    def one():
        xv = [pm.decompress(s, codes[s]) for s in range(2)]
        rf.zero_()
        if rc is not None:
            rc.zero_()
        for s in range(2):
            pm.deposit(s, xv[s][0], rc, rf)
        pm.solve(rc, rf, ac, af)
        for s in range(2):
            pm.kick_drift(xv[s][0], xv[s][1], ac, af, 1.0, 1.0)
            pm.compress(s, xv[s][0], xv[s][1], out=spare[s])

    ms = timed_loop(torch, stream, one, steps) / steps
    pm.check()
    return ms


def run_largest(args):
    """The largest one-GPU workload (1536^3, 4.08e9 particles): the fused step
    replayed from a graph, then per-stage CUDA-event times.  Inputs are built
    on the device; no host copy of the state is made, so there is no
    end-to-end number for this workload."""
    import torch

    from paper_1611_01545_gb300 import PM, _lib

    rank, world, local = dist_env()
    if world > 1:
        return None if rank else {"workload": "largest1536", "skipped": "one-GPU workload"}
    torch.cuda.set_device(local)
    cfg = largest_config(args.tile_batch or 64)
    cfg["vmax_mode"] = args.vmax_mode
    t0 = time.perf_counter()
    pm = PM(cfg)
    a = build_largest_codes(pm, torch)
    b = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in a]
    build_s = time.perf_counter() - t0
    if args.tuning:
        pm.set_tuning(json.loads(args.tuning))
    tuning = pm.get_tuning()
    n_total = sum(c.n for c in a)
    lib = _lib.load()
    stream = torch.cuda.current_stream()

    def one_step():
        pm.step(a, b, 1.0, 1.0)

    pm.set_graphs(True)
    for _ in range(args.warmup):
        one_step()
    pm.check()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    launches0 = lib.pm_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lib.pm_launch_count() - launches0
    sampler.stop()
    ms = e0.elapsed_time(e1)
    pm.check()
    pm.set_graphs(False)
    pm.set_timing(True)
    for _ in range(max(1, min(args.steps, 3))):
        one_step()
    torch.cuda.synchronize()
    pm.check()
    stages = pm.stage_times()
    pm.set_timing(False)
    free, total = torch.cuda.mem_get_info()
    alg = algorithmic_bytes(dict(cfg, tile_batch=tuning["tile_batch"]), [c.n for c in a], cfg["vel_bits"])
    result = {
        "metric": METRIC, "value": n_total * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (device-generated)",
        "config": {"workload": "largest1536", "n_fine": cfg["n_fine"], "coarse_ratio": 4, "tile": 64, "buffer": 16,
                   "tile_batch": tuning["tile_batch"], "particles": {"cdm": a[0].n, "nu": a[1].n},
                   "vel_bits": 16, "vmax_mode": args.vmax_mode, "l2": "working set > L2"},
        "e2e": None, "gpu_launches": int(launches), "tuning": tuning,
        "stages_ms": {k: round(v[0], 4) for k, v in stages.items()},
        "stage_launches": {k: v[1] for k, v in stages.items()},
        "stage_gbs": {k: round(alg[k] / (v[0] / 1e3) / 1e9, 1) for k, v in stages.items() if k in alg},
        "device_memory_used_gb": round((total - free) / 1e9, 1), "build_s": round(build_s, 1),
        "clocks": sampler.summary(),
    }
    pm.close()
    return result


def run_gb300(args):
    import torch
    import torch.distributed as dist

    if args.workload == "largest1536":
        return run_largest(args)

    from paper_1611_01545_gb300 import PM, _lib
    from synth import make_workload

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = make_workload(args.workload, seed=None)
    cfg = w.config()
    cfg["tile_batch"] = args.tile_batch
    cfg["vmax_mode"] = args.vmax_mode
    if args.pp:
        # Eq. 4 softening: 0.05 of the mean CDM inter-particle spacing, L / (20 n_p)
        n_p = round(w.counts[0] ** (1.0 / 3.0))
        cfg["pp"], cfg["r_soft"] = 1, w.n_fine / (20.0 * n_p)
    pm = PM(cfg)
    codes, spare = build_state(pm, w, torch)
    counts = w.counts
    n_total = sum(counts)
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    # Every step is one pass of the hot path over the same synthetic batch: the
    # initial state (the workload's initial conditions) is mapped to a new
    # state and is never overwritten, so every timed region measures the
    # configured workload and not a state evolved by c_k = c_d = 1 steps.
    a, b = codes, spare

    def one_step():
        pm.step(a, b, 1.0, 1.0)

    if args.tuning:
        pm.set_tuning(json.loads(args.tuning))
    tuning = pm.get_tuning()
    if not args.no_autotune and not args.tuning:
        # launch tuning picked by timing candidate cell blocks / launch forms / tile batches
        tuning = pm.autotune(a, b, 1.0, 1.0, reps=2)
    # headline: the step replayed from a captured CUDA graph
    pm.set_graphs(True)
    for _ in range(args.warmup):
        one_step()
    pm.check()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lib.pm_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = lib.pm_launch_count() - launches0
    sampler.stop()
    ms = e0.elapsed_time(e1)
    pm.check()
    value, worst_s = job_rate(ms / 1e3, n_total * args.steps, world, "cuda", dist)
    ms_max = worst_s * 1e3
    pm.set_graphs(False)

    # the same kernels launched directly, then with CUDA events around every
    # stage on the launching stream (per-kernel durations for the roofline)
    direct_ms = timed_loop(torch, stream, one_step, args.steps) / args.steps
    pm.set_timing(True)
    for _ in range(args.steps):
        one_step()
    torch.cuda.synchronize()
    pm.check()
    stages = pm.stage_times()
    pm.set_timing(False)
    plain_ms = plain_step_ms(pm, w, a, b, torch, stream, max(3, args.steps // 4))

    # end-to-end through the C ABI with host buffers (pinned), copies in the timed
    # region: the packed record form (pm_step_packed) and the padded in-memory
    # form (pm_step_host)
    pm.set_graphs(True)
    k_e2e = max(1, min(args.steps, 10))

    def e2e_run(fn, hin, hout):
        fn(hin, hout, 1.0, 1.0)           # first call allocates the library's staging buffers
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            fn(hin, hout, 1.0, 1.0)
        return time.perf_counter() - t0

    pk_in = [pm.pack(c).to("cpu", pin=True) for c in a]
    pk_out = [pm.pack(c).to("cpu", pin=True) for c in b]
    e2e_s = e2e_run(pm.step_packed, pk_in, pk_out)
    pad_s = e2e_run(pm.step_host, [c.to("cpu", pin=True) for c in a], [c.to("cpu", pin=True) for c in b])
    pm.set_graphs(False)
    e2e_value, _ = job_rate(e2e_s, n_total * k_e2e, world, "cuda", dist)
    pad_value, _ = job_rate(pad_s, n_total * k_e2e, world, "cuda", dist)
    h2d = sum(codes_bytes(c, w.vel_bits, packed=True) for c in a)
    d2h = h2d

    alg = algorithmic_bytes(dict(cfg, tile_batch=tuning["tile_batch"]), counts, w.vel_bits)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # dominant kernel: largest total time among kinds with an algorithmic byte model
    dom = None
    for k, (avg, cnt) in stages.items():
        if k in alg and (dom is None or avg * cnt > stages[dom][0] * stages[dom][1]):
            dom = k
    roofline = None
    if dom:
        avg_ms = stages[dom][0]
        achieved = alg[dom] / (avg_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                    "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                    "traffic": recorded_traffic(dom),
                    "alg_bytes_per_launch": alg[dom], "avg_launch_ms": round(avg_ms, 5)}
    step_ms = ms_max / args.steps
    model = step_model_bytes(cfg, counts, w.vel_bits)
    step_roofline = {"bound": "hbm", "bytes_per_step": model, "achieved": round(model / (step_ms / 1e3) / 1e9, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(model / (step_ms / 1e3) / 1e9 / hbm, 4),
                     "model": "whole step: 15 or 21 B per particle + 40 B per tile and coarse cell + kernels"}
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_fine": w.n_fine, "coarse_ratio": w.coarse_ratio,
                   "tile": w.tile, "buffer": w.buffer, "tile_batch": args.tile_batch,
                   "vmax_mode": args.vmax_mode, "pp": int(args.pp),
                   "particles": {"cdm": counts[0], "nu": counts[1]}, "vel_bits": w.vel_bits,
                   "global_batch": n_total * world, "parallelism": f"replicas{world}",
                   "l2": "working set > L2 (126 MB): codes 113 MB + meshes > 400 MB per step"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": k_e2e, "host_form": "packed record bytes (pm_step_packed)",
                "padded": {"value": pad_value, "bytes_per_step_each_way": sum(codes_bytes(c, w.vel_bits) for c in a),
                           "host_form": "padded in-memory words (pm_step_host)"}},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "step_roofline": step_roofline,
        "tuning": tuning,
        "launch_forms": {"graph_ms_per_step": round(ms_max / args.steps, 5),
                         "direct_ms_per_step": round(direct_ms, 5),
                         "plain_ms_per_step": round(plain_ms, 5),
                         "plain_value": n_total * world / (plain_ms / 1e3),
                         "plain": "one call per stage: decompress, deposit, solve, kick_drift, compress"},
        "stages_ms": {k: round(v[0], 5) for k, v in stages.items()},
        "stage_launches": {k: v[1] for k, v in stages.items()},
        "clocks": sampler.summary(),
    }
    if not args.no_adjoint:
        result["adjoint"] = adjoint_ratio(args.adjoint_workload)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, 1.0 / 64)
    if world > 1:
        dist.destroy_process_group()
    pm.close()
    return result if rank == 0 else None


def adjoint_ratio(workload: str, steps: int = 10, every: int = 2, reps: int = 3):
    """Adjoint/forward time of the differentiable trajectory: `steps` PM steps of
    a single-mesh workload from x0 = q + psi, loss sum (rho_K - target)^2, its
    gradient in psi by the reverse mode with checkpoints every `every` steps."""
    import numpy as np
    import torch

    from paper_1611_01545_gb300 import PM
    from paper_1611_01545_gb300.diff import trajectory_loss
    from synth import make_workload

    w = make_workload(workload)
    cfg = dict(w.config(), deposit_mode=1)
    pm = PM(cfg)
    q = torch.from_numpy(w.x[0]).cuda()
    rng = np.random.default_rng(9)
    psi = torch.from_numpy((rng.standard_normal(w.x[0].shape) * 0.2).astype(np.float32)).cuda()
    xnu = torch.from_numpy(w.x[1]).cuda()
    vnu = torch.from_numpy(w.v[1]).cuda()
    target = torch.zeros((w.n_fine,) * 3, device="cuda")
    fwd, bwd = [], []
    for r in range(reps + 1):
        p = psi.clone().requires_grad_(True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        L = trajectory_loss(pm, p, q, xnu, vnu, target, 0.0, steps, every, 1.0, 1.0)
        e1.record()
        L.backward()
        e2.record()
        torch.cuda.synchronize()
        if r:
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    pm.check()
    pm.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    return {"workload": workload, "particles": sum(w.counts), "steps": steps, "checkpoint_every": every,
            "forward_ms": round(f, 3), "adjoint_ms": round(b, 3), "ratio": round(b / f, 3),
            "note": "adjoint time includes the checkpointed recompute of each segment"}


def cpu_baseline(workload, frac: float = 1.0 / 64):
    """Times the oracle, as it stands, on a bounded sample of the workload.

    Sample: the oracle's particle stages (CIC deposit onto the coarse and the
    fine mesh, interpolation, kick-drift, codec) on a random subset of both
    species, one buffered fine-tile solve and the full coarse-mesh solve;
    the full-step time is extrapolated per particle and per tile.
    """
    from oracle import codec, mesh, solve, step
    from synth import make_workload

    w = make_workload(workload) if isinstance(workload, str) else workload
    nf, t, b = w.n_fine, w.tile, w.buffer
    T = t + 2 * b
    n_tiles = (nf // t) ** 3 if w.coarse_ratio > 1 else 0
    rng = np.random.default_rng(5)
    sub = []
    for s in range(2):
        n = w.x[s].shape[0]
        idx = rng.choice(n, max(1, int(n * frac)), replace=False)
        sub.append((w.x[s][idx], w.v[s][idx]))
    t0 = time.perf_counter()
    nc = nf // 4
    xs = []
    for s, (x, v) in enumerate(sub):
        c = codec.compress(x, v, nf, nc, w.vel_bits)
        xd, vd = codec.decompress(c, nf)
        xs.append((xd, vd))
    rho_f = sum(mesh.cic_deposit(x, m, nf) for (x, _), m in zip(xs, w.mass))
    if w.coarse_ratio > 1:
        rho_c = sum(mesh.cic_deposit(x.astype(np.float64) / w.coarse_ratio, m, nf // w.coarse_ratio)
                    for (x, _), m in zip(xs, w.mass))
    zero3 = np.zeros((3,) + rho_f.shape)
    for (x, v) in xs:
        a = mesh.cic_interp(zero3, x, nf)
        x1, v1 = step.kick_drift(x, v, a, 1.0, 1.0, nf)
        codec.compress(step.to_f32_positions(x1, nf), v1.astype(np.float32), nf, nc, w.vel_bits)
    t_particles = time.perf_counter() - t0
    t0 = time.perf_counter()
    if w.coarse_ratio > 1:
        solve.accel_periodic(rho_c, float(w.coarse_ratio), w.G, w.r_split)
    else:
        solve.accel_periodic(rho_f, 1.0, w.G)
    t_coarse = time.perf_counter() - t0
    t_tile = 0.0
    if n_tiles:
        K = solve.fine_kernel(T, w.G, w.r_split, w.r_cut)
        t0 = time.perf_counter()
        solve.accel_tile(rho_f[:T, :T, :T], K)
        t_tile = time.perf_counter() - t0
    n_total = sum(w.counts)
    est = t_particles / frac + t_coarse + t_tile * n_tiles
    return {"value": n_total / est, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle particle stages on {frac:.4f} of both species ({sum(len(x) for x, _ in sub)} "
                       f"particles, {t_particles:.1f} s), 1 of {n_tiles} tile solves ({t_tile:.1f} s), full coarse "
                       f"solve ({t_coarse:.1f} s); full step extrapolated to {est:.0f} s"),
            "seconds_measured": round(t_particles + t_coarse + t_tile, 2), "n_total": n_total}


def run_reference(args):
    """Reference arm: the oracle timed on the host cores, one bounded sample per step."""
    from synth import make_workload

    rank, world, _ = dist_env()
    if rank != 0:
        return None
    w = make_workload(args.workload)
    frac = 1.0 / 256
    samples = []
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        cpu_baseline(w, frac)
    for _ in range(args.steps):
        samples.append(cpu_baseline(w, frac))
    wall = time.perf_counter() - t0
    value = statistics.median(s["value"] for s in samples)
    cb = dict(samples[-1])
    cb["value"] = value
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["n_total"] / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="two_level256")
    p.add_argument("--tile-batch", type=int, default=0)
    p.add_argument("--vmax-mode", type=int, default=0, choices=[0, 1],
                   help="0: exact v_max' (the paper's definition); 1: bound from the force meshes")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--pp", action="store_true", help="add the particle-particle force of Eq. 4 to the step")
    p.add_argument("--tuning", default="", help="launch tuning as JSON (as printed under 'tuning'); skips the autotuner")
    p.add_argument("--adjoint-workload", default="diff128")
    args = p.parse_args()
    res = run_reference(args) if args.impl == "reference" else run_gb300(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
