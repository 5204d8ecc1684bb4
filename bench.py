"""Benchmark of the fused two-species PM step (particle-steps per second).

Workload (default): the largest one-GPU configuration, two-level PM on a
1536^3 fine mesh (384^3 coarse mesh, 13,824 tiles of 64^3 + 16-cell buffer,
96^3 FFTs), 768^3 Zel'dovich CDM + 1536^3 Fermi-Dirac neutrinos (4.08e9
particles, 16-bit velocity codes, about 37 GB of record bytes), drawn on the
device.  One step = decompress + deposit, coarse and tile solves,
interpolate + kick + drift + recompress of both species (pm_step), codes ->
codes.  The 256^3 workload (128^3 + 256^3 particles, 8-bit velocity codes)
is reported beside it under "two_level256".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
  python bench.py --workload two_level256        # the 256^3 workload alone

Under torchrun each rank runs an independent replica of the workload (the
path shards by independent problems; no data-path collective): value is the
particle-steps of all ranks divided by the slowest rank's time.
--impl reference times the oracle (plain float64 numpy restatement of the
method) on the host cores, one bounded sample of the workload per step.
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


# CUDA sources that define each kernel kind (its code and its launcher)
_PARTICLE_SOURCES = ("particles.cu", "particles.cuh", "pm_common.cuh")
_SOLVE_SOURCES = ("solve.cu", "fft.cuh", "tma.cuh", "pm_common.cuh")
KIND_SOURCES = {"deposit": _PARTICLE_SOURCES, "ikd_count": _PARTICLE_SOURCES, "ikd_scatter": _PARTICLE_SOURCES,
                "fft_a_tiles": _SOLVE_SOURCES, "fft_b_tiles": _SOLVE_SOURCES, "fft_c_tiles": _SOLVE_SOURCES}


def csrc_digest(kind=None):
    """Digest of the CUDA sources of a kernel kind (all sources for kind None);
    ncu traffic figures apply only to the sources they were taken on."""
    import glob
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1611_01545_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh")))
    if kind in KIND_SOURCES:
        files = [f for f in files if os.path.basename(f) in KIND_SOURCES[kind]]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind, workload, particles, vel_bits):
    """DRAM bytes (read + write) per launch of a kernel kind from the committed
    ncu record (profiles/traffic.json), or None when the kernels changed since
    that capture.  A record taken on a smaller workload of the same recipe and
    velocity width is scaled to this one by the particles processed (the
    particle passes move a fixed number of bytes per particle plus per-cell
    tables that grow with the mesh, i.e. in the same proportion for these
    workloads, which all hold 1.125 particles per fine cell)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    digest = csrc_digest(kind)
    best = None
    for e in rec.get("entries", []):
        if e.get("kind") != kind or e.get("csrc") != digest:
            continue
        if e.get("workload") == workload and e.get("vel_bits") == vel_bits:
            return {"bytes": int(e["bytes_per_launch"]), "captured_on": workload, "scaled": False}
        if e.get("scale") == "particles" and e.get("particles") and e.get("vel_bits") == vel_bits:
            best = {"bytes": int(round(e["bytes_per_launch"] * particles / e["particles"])),
                    "captured_on": e["workload"], "scaled": True}
    return best


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


# Launch tuning of the largest workload: the shapes the autotuner picks on
# the 256^3 workload of the same recipe (persistent 32x2x1-cell deposit
# blocks, 64x1x1 kick blocks with a new-cell window half-width of 1), and 256
# tiles per solve batch (measured: 8, 16, 32, 64, 128, 256 tiles per batch
# gave 392, 376, 365, 358, 355, 353 ms per step).  The autotuner itself would
# spend minutes at this size (each candidate is timed on whole steps).
LARGEST_TUNING = {"deposit_block": [32, 2, 1], "deposit_persistent": 1, "kick_block": [64, 1, 1],
                  "kick_window": 1, "kick_persistent": 0, "tile_batch": 256}


def measured_hbm():
    """HBM roofline denominator: the measured copy rate of this GPU pool, else the fallback figure."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    hbm = peaks.get("hbm_gbs")
    return (float(hbm), "measured") if hbm else (6800.0, "fallback")


def kernel_roofline(stages, alg, workload, particles, vel_bits):
    """Roofline of the dominant kernel kind (largest total time among the kinds
    with an algorithmic byte model): algorithmic bytes per launch / its mean
    CUDA-event launch duration, against the HBM copy peak."""
    hbm, src = measured_hbm()
    dom = None
    for k, (avg, cnt) in stages.items():
        if k in alg and (dom is None or avg * cnt > stages[dom][0] * stages[dom][1]):
            dom = k
    if dom is None:
        return None
    avg_ms = stages[dom][0]
    achieved = alg[dom] / (avg_ms / 1e3) / 1e9
    tr = recorded_traffic(dom, workload, particles, vel_bits)
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm, "peak_source": src,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": tr["bytes"] if tr else None,
            "traffic_source": tr, "alg_bytes_per_launch": alg[dom], "avg_launch_ms": round(avg_ms, 5),
            "note": f"frac of {src} HBM copy rate"}


def step_roofline(model_bytes, step_ms):
    hbm, src = measured_hbm()
    gbs = model_bytes / (step_ms / 1e3) / 1e9
    return {"bound": "hbm", "bytes_per_step": model_bytes, "achieved": round(gbs, 1), "peak": hbm,
            "peak_source": src, "unit": "GB/s", "frac": round(gbs / hbm, 4),
            "model": "whole step: 15 or 21 B per particle + 40 B per tile and coarse cell + kernels"}


def host_mem_available():
    """MemAvailable of this host in bytes (None where /proc/meminfo is absent)."""
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def cpu_model():
    """The host CPU's model name (lscpu), else /proc/cpuinfo's model or part field."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            low = ln.lower()
            if low.startswith("model name") or low.startswith("cpu part"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def pinned_like(t, torch):
    """An uninitialised pinned host tensor of t's shape and dtype."""
    return torch.empty(t.shape, dtype=t.dtype, pin_memory=True)


def to_pinned(codes, torch):
    """Device codes copied into freshly allocated pinned host tensors."""
    from paper_1611_01545_gb300.pm import Codes
    f = {k: pinned_like(getattr(codes, k), torch) for k in ("cnt", "esc", "n_esc", "pos", "vel", "vmax")}
    for k, t in f.items():
        t.copy_(getattr(codes, k))
    return Codes(codes.n, **f)


def empty_pinned_packed(pm, n, esc_cap, torch):
    """Pinned host codes for a step's output, written once here so that the
    timed copies do not pay for the first touch of their pages."""
    from paper_1611_01545_gb300.pm import Codes
    vdt = torch.int16 if pm.vel_bits == 16 else torch.uint8
    ncell = pm.n_cmp ** 3
    c = Codes(n=n, cnt=torch.empty(ncell, dtype=torch.uint8, pin_memory=True),
              esc=torch.zeros((esc_cap, 2), dtype=torch.int32).pin_memory(),
              n_esc=torch.zeros(1, dtype=torch.int32).pin_memory(),
              pos=torch.empty((n, 3), dtype=torch.uint8, pin_memory=True),
              vel=torch.empty((n, 3), dtype=vdt, pin_memory=True),
              vmax=torch.zeros(1, dtype=torch.float32).pin_memory())
    for t in (c.cnt, c.pos, c.vel):
        t.zero_()
    return c


def e2e_packed(pm, codes, spare, torch, steps, world, dist, n_total, warmup=1):
    """End to end through the C ABI (pm_step_packed) with the state in pinned
    host memory: each step copies the packed record bytes (3 B position + 3 or
    6 B velocity codes per particle, plus counts, escapes and v_max) host ->
    device, steps, and copies the new packed state device -> host; the first
    call (staging allocation, graph capture) is not timed.  The device codes
    `codes` / `spare` are released first (the library's own staging holds the
    state during the call), so the lists are emptied."""
    vb = 2 if pm.vel_bits == 16 else 1
    rec = sum(c.n for c in codes) * 3 * (1 + vb)
    avail = host_mem_available()
    if avail is not None and avail < 2.3 * rec * world:
        return {"value": None, "unit": UNIT, "skipped": f"host memory: {avail / 1e9:.0f} GB available, "
                f"{2 * rec * world / 1e9:.0f} GB of pinned buffers needed"}
    spare.clear()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    hin = []
    for i in range(len(codes)):
        pk = pm.pack(codes[i])
        hin.append(to_pinned(pk, torch))
        del pk
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    ncodes = [(c.n, c.esc.shape[0]) for c in codes]
    codes.clear()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    hout = [empty_pinned_packed(pm, n, cap, torch) for n, cap in ncodes]
    setup_s = time.perf_counter() - t0
    el, form, gaps = packed_steps(pm, hin, hout, steps, world, dist, warmup)
    value, worst = job_rate(el, n_total * steps, world, "cuda", dist)
    nbytes = sum(codes_bytes(c, pm.vel_bits, packed=True) for c in hin)
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": steps, "ms_per_step": round(worst / steps * 1e3, 3), **gap_summary(gaps),
            "host_form": f"packed record bytes in pinned host memory ({form})",
            "setup_s": round(setup_s, 1)}


def packed_steps(pm, hin, hout, steps, world, dist, warmup=1):
    """Seconds of `steps` end-to-end steps from packed pinned host codes to
    packed pinned host codes: pm_step_packed_async calls (each step's copies
    overlap the neighbouring steps' compute) closed by pm_check, which waits
    for the last output copies; pm_step_packed (synchronous, graph-replayed)
    where the extra packed input buffer does not fit.  `warmup` untimed
    steps (the first allocates) come first."""
    import torch

    from paper_1611_01545_gb300.pm import PMError
    form = "pm_step_packed_async"
    try:
        for _ in range(max(1, warmup)):
            pm.step_packed_async(hin, hout, 1.0, 1.0)
        pm.check()
    except PMError:
        form = "pm_step_packed"
        pm.set_graphs(True)
        for _ in range(max(1, warmup)):
            pm.step_packed(hin, hout, 1.0, 1.0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    st = torch.cuda.current_stream()
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t0 = time.perf_counter()
    ends[0].record(st)
    for i in range(steps):
        if form == "pm_step_packed_async":
            pm.step_packed_async(hin, hout, 1.0, 1.0)
        else:
            pm.step_packed(hin, hout, 1.0, 1.0)   # ends with pm_check
        ends[i + 1].record(st)
    pm.check()
    el = time.perf_counter() - t0
    pm.set_graphs(False)
    # time between the ends of consecutive steps' kernels on the step stream:
    # the first includes the pipeline fill (its whole input copy)
    gaps = [ends[i].elapsed_time(ends[i + 1]) for i in range(steps)]
    return el, form, gaps


def gap_summary(gaps):
    """First-step and steady-state (median of the rest) step intervals, ms."""
    rest = sorted(gaps[1:])
    return {"first_step_ms": round(gaps[0], 2),
            "steady_ms_per_step": round(rest[len(rest) // 2], 2) if rest else None}


def run_largest(args):
    """The largest one-GPU workload (1536^3, 4.08e9 particles): the fused step
    replayed from a graph (the headline), per-stage CUDA-event times, the
    dominant kernel's roofline, end to end through pm_step_packed, and the
    oracle's CPU baseline on a bounded sample."""
    import torch
    import torch.distributed as dist

    from paper_1611_01545_gb300 import PM, _lib

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tuning = dict(LARGEST_TUNING)
    if args.tuning:
        tuning.update(json.loads(args.tuning))
    if args.tile_batch:
        tuning["tile_batch"] = args.tile_batch
    cfg = largest_config(tuning["tile_batch"])
    cfg["vmax_mode"] = args.vmax_mode
    t0 = time.perf_counter()
    pm = PM(cfg)
    a = build_largest_codes(pm, torch)
    b = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in a]
    build_s = time.perf_counter() - t0
    pm.set_tuning(tuning)
    tuning = pm.get_tuning()
    counts = [c.n for c in a]
    n_total = sum(counts)
    lib = _lib.load()
    stream = torch.cuda.current_stream()

    def one_step():
        pm.step(a, b, 1.0, 1.0)

    # headline: the step replayed from a captured CUDA graph; inputs (4.08e9
    # particles, 49 GB of codes, 58 GB of meshes) are far larger than L2
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
    step_ms = worst_s * 1e3 / args.steps
    pm.set_graphs(False)
    # per-stage CUDA events on the launching stream (direct launches)
    pm.set_timing(True)
    for _ in range(2):
        one_step()
    torch.cuda.synchronize()
    pm.check()
    stages = pm.stage_times()
    pm.set_timing(False)
    free, total = torch.cuda.mem_get_info()
    alg = algorithmic_bytes(dict(cfg, tile_batch=tuning["tile_batch"]), counts, cfg["vel_bits"])
    e2e = None
    if not args.no_e2e:
        e2e = e2e_packed(pm, a, b, torch, max(1, min(args.steps, 20)), world, dist, n_total,
                         warmup=max(1, min(args.warmup, 5)))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (device-generated)",
        "config": {"workload": "largest1536", "n_fine": cfg["n_fine"], "coarse_ratio": 4, "tile": 64, "buffer": 16,
                   "tile_batch": tuning["tile_batch"], "particles": {"cdm": counts[0], "nu": counts[1]},
                   "vel_bits": 16, "vmax_mode": args.vmax_mode, "global_batch": n_total * world,
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2: 49 GB of codes, 58 GB of meshes"},
        "e2e": e2e, "gpu_launches": int(launches),
        "roofline": kernel_roofline(stages, alg, "largest1536", n_total, cfg["vel_bits"]),
        "step_roofline": step_roofline(step_model_bytes(cfg, counts, cfg["vel_bits"]), step_ms),
        "tuning": tuning,
        "stages_ms": {k: round(v[0], 4) for k, v in stages.items()},
        "stage_launches": {k: v[1] for k, v in stages.items()},
        "stage_gbs": {k: round(alg[k] / (v[0] / 1e3) / 1e9, 1) for k, v in stages.items() if k in alg},
        "device_memory_used_gb": round((total - free) / 1e9, 1), "build_s": round(build_s, 1),
        "clocks": sampler.summary(),
    }
    pm.close()
    del a, b
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    return result if rank == 0 else None


def run_workload(args, workload, adjoint=True, cpu=True):
    """One of the smaller workloads (two_level256 and the others of
    synth.generators): autotuned launch tuning, the graph-replayed step, the
    direct and plain forms, per-stage times, end to end (packed and padded
    host forms), the adjoint/forward ratio and the oracle's CPU baseline."""
    import torch
    import torch.distributed as dist

    from paper_1611_01545_gb300 import PM, _lib
    from synth import make_workload

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    own_group = world > 1 and not dist.is_initialized()
    if own_group:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = make_workload(workload, seed=None)
    cfg = w.config()
    cfg["tile_batch"] = args.tile_batch
    cfg["vmax_mode"] = args.vmax_mode
    vel_bits = args.vel_bits or w.vel_bits
    cfg["vel_bits"] = vel_bits
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
    # region: the packed record form (pm_step_packed_async) and the padded
    # in-memory form (pm_step_host)
    e2e = None
    if not args.no_e2e:
        e2e = small_e2e(pm, a, b, torch, args.steps, world, dist, n_total, vel_bits)

    alg = algorithmic_bytes(dict(cfg, tile_batch=tuning["tile_batch"]), counts, vel_bits)

    step_ms = ms_max / args.steps
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "n_fine": w.n_fine, "coarse_ratio": w.coarse_ratio,
                   "tile": w.tile, "buffer": w.buffer, "tile_batch": args.tile_batch,
                   "vmax_mode": args.vmax_mode, "pp": int(args.pp),
                   "particles": {"cdm": counts[0], "nu": counts[1]}, "vel_bits": vel_bits,
                   "global_batch": n_total * world, "parallelism": f"replicas{world}",
                   "l2": "working set > L2 (126 MB): codes + meshes > 400 MB per step"},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": kernel_roofline(stages, alg, workload, n_total, vel_bits),
        "step_roofline": step_roofline(step_model_bytes(cfg, counts, vel_bits), step_ms),
        "tuning": tuning,
        "launch_forms": {"graph_ms_per_step": round(step_ms, 5),
                         "direct_ms_per_step": round(direct_ms, 5),
                         "plain_ms_per_step": round(plain_ms, 5),
                         "plain_value": n_total * world / (plain_ms / 1e3),
                         "plain": "one call per stage: decompress, deposit, solve, kick_drift, compress"},
        "stages_ms": {k: round(v[0], 5) for k, v in stages.items()},
        "stage_launches": {k: v[1] for k, v in stages.items()},
        "clocks": sampler.summary(),
    }
    if "tile_count_max" in w.notes:
        result["config"]["tile_count"] = {"max": w.notes["tile_count_max"], "min": w.notes["tile_count_min"]}
    if adjoint and not args.no_adjoint:
        result["adjoint"] = adjoint_ratio(args.adjoint_workload)
    pm.close()
    del a, b, codes, spare
    torch.cuda.empty_cache()
    if cpu and rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(workload)
    if own_group:
        dist.destroy_process_group()
    return result if rank == 0 else None


def small_e2e(pm, a, b, torch, steps, world, dist, n_total, vel_bits):
    """End to end on a workload whose host copies fit beside the device state:
    packed record bytes (pm_step_packed_async) and the padded in-memory words
    (pm_step_host), pinned host buffers, copies inside the timed region."""
    k_e2e = max(1, min(steps, 50))

    def e2e_run(fn, hin, hout):
        fn(hin, hout, 1.0, 1.0)           # first call allocates the library's staging buffers
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            fn(hin, hout, 1.0, 1.0)
        return time.perf_counter() - t0

    pk_in = [to_pinned(pm.pack(c), torch) for c in a]
    pk_out = [to_pinned(pm.pack(c), torch) for c in b]
    e2e_s, e2e_form, _ = packed_steps(pm, pk_in, pk_out, k_e2e, world, dist)
    pm.set_graphs(True)
    pad_s = e2e_run(pm.step_host, [to_pinned(c, torch) for c in a], [to_pinned(c, torch) for c in b])
    pm.set_graphs(False)
    e2e_value, _ = job_rate(e2e_s, n_total * k_e2e, world, "cuda", dist)
    pad_value, _ = job_rate(pad_s, n_total * k_e2e, world, "cuda", dist)
    h2d = sum(codes_bytes(c, vel_bits, packed=True) for c in a)
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
            "steps": k_e2e, "host_form": f"packed record bytes ({e2e_form})",
            "padded": {"value": pad_value, "bytes_per_step_each_way": sum(codes_bytes(c, vel_bits) for c in a),
                       "host_form": "padded in-memory words (pm_step_host)"}}


def run_gb300(args):
    if args.workload != "largest1536":
        return run_workload(args, args.workload)
    res = run_largest(args)
    rank = dist_env()[0]
    if rank == 0 and res is not None and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline("largest1536")
    if not args.no_extra:
        # the 256^3 workload beside the headline (its own autotuned launch tuning)
        small = argparse.Namespace(**vars(args))
        small.tuning, small.tile_batch = "", 0
        extra = run_workload(small, "two_level256", adjoint=True, cpu=False)
        if res is not None and extra is not None:
            keep = ("value", "ms_per_step", "e2e", "roofline", "step_roofline", "tuning", "launch_forms",
                    "stages_ms", "adjoint", "clocks", "gpu_launches", "config")
            res["two_level256"] = {k: extra[k] for k in keep if k in extra}
    return res


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




# ---------------------------------------------------------------- oracle --
# The oracle's own stages, timed on the host cores on a bounded sample: whole
# fine tiles of the two-level step (decompress the tile's home particles,
# deposit them on the coarse mesh, deposit the tile's buffered window, solve
# the tile, interpolate the fine and coarse force at the home particles,
# kick, drift, recompress them).  Every tile of a two-level workload of this
# recipe (64^3 interior + 16-cell buffer, one CDM particle per 8 fine cells,
# one neutrino per fine cell) carries the same work, so the per-tile rate
# times the tile count gives the step; the coarse solve (one per step) is
# added from its own timing.

# workload -> (realisation of the recipe the sample tiles are cut from,
#              velocity bits, coarse mesh edge, tiles per step)
ORACLE_SAMPLES = {
    "largest1536": ("two_level256", 16, 384, 13824),
    "two_level256": ("two_level256", 8, 64, 64),
}


def _oracle_tile_inputs(workload, n_jobs, seed=5):
    """Per-tile inputs of the oracle sample, written to pickles in a temporary
    directory: the tile's home particles as codes, the decoded positions of the
    other particles of its buffered window, the tile kernel and the coarse
    force mesh (both precomputed once per run by the oracle).  Returns
    (paths, info)."""
    import pickle
    import tempfile

    from oracle import codec, solve
    from oracle import mesh as omesh
    from synth import make_workload

    recipe, vel_bits, nc_target, tiles_target = ORACLE_SAMPLES[workload]
    w = make_workload(recipe)
    n, t, b, rc = w.n_fine, w.tile, w.buffer, w.coarse_ratio
    T, nc, ncmp = t + 2 * b, n // rc, n // w.cmp_ratio
    nt = n // t
    cfg = dict(w.config(), vel_bits=vel_bits)
    K = solve.fine_kernel(T, w.G, w.r_split, w.r_cut)
    rng = np.random.default_rng(seed)
    picks = rng.choice(nt ** 3, size=min(n_jobs, nt ** 3), replace=False)
    # the coarse force the tiles interpolate from: the oracle's coarse solve of
    # the sampled tiles' home particles, timed (one coarse solve per step)
    cells = [np.floor(x).astype(np.int32) for x in w.x]          # fine cell of every particle
    tids = [(c[:, 0] // t) + nt * ((c[:, 1] // t) + nt * (c[:, 2] // t)) for c in cells]
    homes = []
    rho_c = np.zeros((nc, nc, nc))
    for tid in picks:
        idx = np.array([tid % nt, (tid // nt) % nt, tid // (nt * nt)])
        hs = []
        for s in range(2):
            sel = tids[s] == tid
            hs.append(sel)
            rho_c += omesh.cic_deposit(w.x[s][sel].astype(np.float64) / rc, w.mass[s], nc)
        homes.append((idx, hs))
    t0 = time.perf_counter()
    acc_c = solve.accel_periodic(rho_c, float(rc), w.G, w.r_split)
    t_coarse = time.perf_counter() - t0
    d = tempfile.mkdtemp(prefix="pm_oracle_sample_")
    paths = []
    for j, (idx, hs) in enumerate(homes):
        origin = idx * t - b
        job = {"cfg": cfg, "origin": origin.astype(np.float64), "K": K, "acc_c": acc_c, "home": [], "buf": []}
        for s in range(2):
            x, v = w.x[s], w.v[s]
            # window membership of the tile deposit: floor((x - origin) mod n) in [0, T - 2]
            win = np.ones(x.shape[0], dtype=bool)
            for ax in range(3):
                win &= ((cells[s][:, ax] - int(origin[ax])) % n) <= T - 2
            buf = win & ~hs[s]
            job["home"].append(codec.compress(x[hs[s]], v[hs[s]], n, ncmp, vel_bits))
            cb = codec.compress(x[buf], v[buf], n, ncmp, vel_bits)
            job["buf"].append(codec.decompress(cb, n)[0])
        p = os.path.join(d, f"tile{j}.pkl")
        with open(p, "wb") as fh:
            pickle.dump(job, fh, protocol=pickle.HIGHEST_PROTOCOL)
        paths.append(p)
    # the coarse solve at the target coarse mesh: measured here at nc^3 and
    # scaled by N^3 log N (the oracle's transforms are O(N^3 log N))
    scale = (nc_target / nc) ** 3 * np.log(nc_target ** 3) / np.log(nc ** 3)
    info = {"recipe": recipe, "vel_bits": vel_bits, "tiles_per_step": tiles_target, "coarse_edge": nc_target,
            "coarse_solve_s": t_coarse * scale, "coarse_measured_edge": nc, "coarse_measured_s": t_coarse,
            "dir": d}
    return paths, info


def _oracle_tile_step(path):
    """One tile of the oracle's step (the stages listed above); returns
    (seconds, home particles, window particles)."""
    import pickle

    from oracle import codec, solve
    from oracle import mesh as omesh
    from oracle import step as ostep

    with open(path, "rb") as fh:
        job = pickle.load(fh)
    cfg = job["cfg"]
    n, rc = cfg["n_fine"], cfg["coarse_ratio"]
    T = cfg["tile"] + 2 * cfg["buffer"]
    nc, ncmp = n // rc, n // cfg["cmp_ratio"]
    origin = job["origin"]
    t0 = time.perf_counter()
    xv = [codec.decompress(c, n) for c in job["home"]]
    rho_c = sum(omesh.cic_deposit(x.astype(np.float64) / rc, m, nc) for (x, _), m in zip(xv, cfg["mass"]))
    rho = sum(omesh.tile_deposit(np.concatenate([x, xb]), m, origin, T, n)
              for (x, _), xb, m in zip(xv, job["buf"], cfg["mass"]))
    a_t = solve.accel_tile(rho, job["K"])
    nh = 0
    for x, v in xv:
        a = omesh.tile_interp(a_t, np.mod(x.astype(np.float64) - origin, n)) + \
            omesh.cic_interp(job["acc_c"], x.astype(np.float64) / rc, nc)
        x1, v1 = ostep.kick_drift(x, v, a, 1.0, 1.0, n)
        codec.compress(ostep.to_f32_positions(x1, n), v1.astype(np.float32), n, ncmp, cfg["vel_bits"])
        nh += x.shape[0]
    el = time.perf_counter() - t0
    del rho_c
    return el, nh, nh + sum(xb.shape[0] for xb in job["buf"])


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


class OracleSampler:
    """The oracle's tile sample: inputs built once, then timed on one thread
    (in this process) or on every host core (a spawn pool, one tile per
    worker)."""

    def __init__(self, workload, n_jobs=None):
        self.cores = os.cpu_count() or 1
        n_jobs = n_jobs or max(2, self.cores)
        self.paths, self.info = _oracle_tile_inputs(workload, n_jobs)
        self.pool = None
        self.next = 0

    def one_thread(self, tiles):
        out = []
        for _ in range(tiles):
            out.append(_oracle_tile_step(self.paths[self.next % len(self.paths)]))
            self.next += 1
        return out

    def all_cores(self):
        import multiprocessing as mp
        if self.pool is None:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_single_thread_env)
            self.pool.map(_oracle_tile_step, self.paths[:self.cores])    # imports, first-touch
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_tile_step, [self.paths[i % len(self.paths)] for i in range(self.cores)])
        return time.perf_counter() - t0, res

    def close(self):
        import shutil
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
        shutil.rmtree(self.info["dir"], ignore_errors=True)


def cpu_baseline(workload):
    """The oracle, as it stands, timed on the host cores on a bounded sample
    of the workload (whole tiles, see ORACLE_SAMPLES): one thread and all
    cores.  value = the all-cores rate in particle-steps/s."""
    if workload not in ORACLE_SAMPLES:
        return None
    t0 = time.perf_counter()
    smp = OracleSampler(workload)
    setup_s = time.perf_counter() - t0
    try:
        one = smp.one_thread(2)
        wall, many = smp.all_cores()
    finally:
        smp.close()
    info = smp.info
    tiles, coarse = info["tiles_per_step"], info["coarse_solve_s"]
    home = np.mean([r[1] for r in one + many])
    n_step = home * tiles
    t1 = np.mean([r[0] for r in one])
    step1 = tiles * t1 + coarse
    stepN = tiles * wall / len(many) + coarse
    return {"value": n_step / stepN, "unit": UNIT, "cores": smp.cores, "kind": "oracle",
            "cpu": cpu_model(), "nproc": smp.cores,
            "one_thread": {"value": n_step / step1, "cores": 1, "tile_s": round(t1, 3)},
            "all_cores": {"value": n_step / stepN, "cores": smp.cores, "tiles": len(many), "wall_s": round(wall, 3)},
            "sample": (f"oracle stages of whole 96^3 tiles (64^3 + 16 buffer; decompress, coarse deposit, window "
                       f"deposit, tile solve, fine + coarse interpolation, kick-drift, recompress of the home "
                       f"particles, {vel_bits_note(info)}) cut from the {info['recipe']} realisation of the recipe "
                       f"({home:.0f} home particles per tile): {len(one)} tiles on 1 thread, {len(many)} tiles on "
                       f"{smp.cores} processes at once; per step x {tiles} tiles + the {info['coarse_edge']}^3 coarse "
                       f"solve ({coarse:.1f} s: measured at {info['coarse_measured_edge']}^3, scaled N^3 log N)"),
            "seconds_measured": round(sum(r[0] for r in one) + wall, 1), "setup_s": round(setup_s, 1)}


def vel_bits_note(info):
    return f"{info['vel_bits']}-bit velocity codes"


def run_reference(args):
    """Reference arm: the oracle timed on all host cores, one bounded sample per
    step (one tile per core of the workload's two-level recipe, plus the
    coarse solve's share of a step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    wl = args.workload if args.workload in ORACLE_SAMPLES else "two_level256"
    t0 = time.perf_counter()
    smp = OracleSampler(wl)
    setup_s = time.perf_counter() - t0
    info = smp.info
    share = info["coarse_solve_s"] / info["tiles_per_step"]
    steps = []
    try:
        for _ in range(args.warmup):
            smp.all_cores()
        for _ in range(args.steps):
            wall, res = smp.all_cores()
            steps.append((wall + share * len(res), sum(r[1] for r in res)))
    finally:
        smp.close()
    sec = statistics.median(s[0] for s in steps)
    units = statistics.median(s[1] for s in steps)
    value = units / sec
    cb = {"value": value, "unit": UNIT, "cores": smp.cores, "kind": "oracle", "cpu": cpu_model(), "nproc": smp.cores,
          "sample": (f"per step: {smp.cores} whole 96^3 tiles of the {info['recipe']} realisation of the recipe "
                     f"({info['vel_bits']}-bit velocity codes), one per process, through the oracle's stages, "
                     f"plus their share of the {info['coarse_edge']}^3 coarse solve ({share * 1e3:.1f} ms per tile)")}
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "sample_particles_per_step": int(units)}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": round(setup_s, 1)}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="largest1536")
    p.add_argument("--tile-batch", type=int, default=0)
    p.add_argument("--vel-bits", type=int, default=0, choices=[0, 8, 16],
                   help="velocity code width (0: the workload's own); not for the largest workload")
    p.add_argument("--vmax-mode", type=int, default=0, choices=[0, 1],
                   help="0: exact v_max' (the paper's definition); 1: bound from the force meshes")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end runs (host buffers)")
    p.add_argument("--no-extra", action="store_true", help="largest workload: skip the 256^3 workload beside it")
    p.add_argument("--pp", action="store_true", help="add the particle-particle force of Eq. 4 to the step")
    p.add_argument("--tuning", default="", help="launch tuning as JSON (as printed under 'tuning')")
    p.add_argument("--adjoint-workload", default="diff128")
    args = p.parse_args()
    res = run_reference(args) if args.impl == "reference" else run_gb300(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
