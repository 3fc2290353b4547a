#!/usr/bin/env python
"""Benchmark of the R^2-Gaussian hot path on B300: fwd+bwd Gaussian-pixel evals/s.

Headline step (differentiation at scale): 500,000 anisotropic, rotated Gaussians
sampled from a seeded 40-ellipsoid 256^3 phantom (per-axis scales log-uniform in
[0.002, 0.05]); cone beam with source-to-origin 1000 mm and source-to-detector
1500 mm; all 75 views of 512^2 at 0.8 mm rasterized in one launch against
projections with Poisson noise (1e5 photons per ray); L1 + 0.25 D-SSIM over the
75 views; 8 random 32^3 TV patches (weight 0.05) voxelized, with their TV; the
full 256^3 volume voxelized (forward); the full backward through the rasterizer
and the patches, and the fused Adam step -- one r2g_train_step call, all in
libr2g.so.  The metric counts the (pixel, Gaussian) and (voxel, Gaussian) pairs
that pass the gates in that step, once, over the device time of the whole step.
The one-scan step (50,000 Gaussians, one view and one TV patch per iteration) is
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (one scan per rank, no data
exchange: the path has nothing to reduce across scans); value = all ranks'
pairs / the slowest rank's time.  --impl reference times the FP64 CPU oracle on
the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Gaussian-pixel evals/s"
N_VIEWS, M_GAUSS, D_TV, N_OUT = 50, 50_000, 32, 256
SCALE_M, SCALE_V, SCALE_NP = 500_000, 75, 8     # the headline (differentiation-at-scale) workload
SCALE_TILES = ((16, 16), (32, 32), (8, 8), (32, 8))
SM_COUNT = 148
MUFU_PER_CLK = 16          # ex2 per SM per clock
FP32_PER_CLK = 128         # FP32 lanes per SM per clock
# FP32 operations charged per gated pair (the scope table's count of the work a pair
# needs: forward ~10 -- 2 FADD, 5 FMUL/FFMA for q, a compare, the -1/2 log2(e) fold,
# the accumulate; backward ~20 -- the recomputed forward and ~10 FFMA for the six
# moments); the kernels' own reduced counts (incremental quadratics) beside them
OPS_FWD, OPS_BWD = 10, 20
OWN_OPS_FWD, OWN_OPS_BWD = 6, 14
# FP32 lane operations per voxel and orientation of the slice SSIM: 11-tap horizontal
# and vertical passes over five moment maps (110 FMAs), three products, ~16 for the
# SSIM ratio
SSIM_OPS_PER_VOXEL = 129


def peaks():
    p = {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p.update(hbm_gbs=float(m["hbm_gbs"]), sm_max_mhz=float(m.get("sm_max_mhz", 2032.0)), source="measured")
    except Exception:
        pass
    return p


# ----------------------------------------------------------------------------- workload


def make_workload(seed: int, device):
    """The one-scan workload: phantom, init, geometry and measured projections."""
    from paper_2405_20693_b300 import inputs as I

    ph, vol = I.normalised_phantom(seed, N_OUT)
    G = I.init_from_volume(vol, I.cube_grid(N_OUT), M_GAUSS, seed)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(N_VIEWS), I.CONE_L_SO)
    meas = I.phantom_projections(ph, views, cam, device=device).astype(np.float32)
    return G, cam, views, meas


N_DISTINCT = 64  # distinct (view, TV patch) pairs the steps cycle through


def step_sequence(seed: int, n: int):
    """(view index, patch offset) of the first n steps: a seeded list of
    N_DISTINCT pairs, repeated."""
    g = np.random.Generator(np.random.PCG64(seed + 2))
    vs = g.integers(0, N_VIEWS, N_DISTINCT)
    offs = g.integers(0, N_OUT - D_TV + 1, (N_DISTINCT, 3))
    base = [(int(vs[k]), tuple(int(x) for x in offs[k])) for k in range(N_DISTINCT)]
    return [base[k % N_DISTINCT] for k in range(n)]


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """SM clock, its maximum, power and the clock-event (throttle) reasons, sampled
    every 200 ms through NVML (read-only queries; nothing is set) while the timed
    region runs.  Falls back to one nvidia-smi query per sample if NVML is missing.
    (A long-running `nvidia-smi -lms` whose stdout is a pipe buffers its lines and
    loses them when it is terminated, which left no samples.)"""

    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4), ("hw_power_brake_slowdown", 0x80))

    def __init__(self, gpu_uuid: str | None, index: int = 0, period_s: float = 0.2):
        self.uuid, self.index, self.period = gpu_uuid, index, period_s
        self.samples = []   # (sm_mhz, sm_max_mhz, power_w, reasons bitmask)
        self._stop = threading.Event()
        self._t = None
        self._nvml = None
        self._h = None
        self.source = None

    def _open(self):
        try:
            import pynvml

            pynvml.nvmlInit()
            h = None
            if self.uuid:
                try:
                    h = pynvml.nvmlDeviceGetHandleByUUID(self.uuid)
                except Exception:
                    h = None
            if h is None:
                h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self._nvml, self._h, self.source = pynvml, h, "nvml"
        except Exception:
            self._nvml, self.source = None, "nvidia-smi"

    def _one(self):
        if self._nvml is not None:
            n, h = self._nvml, self._h
            sm = n.nvmlDeviceGetClockInfo(h, n.NVML_CLOCK_SM)
            smax = n.nvmlDeviceGetMaxClockInfo(h, n.NVML_CLOCK_SM)
            pw = n.nvmlDeviceGetPowerUsage(h) / 1000.0
            rs = n.nvmlDeviceGetCurrentClocksEventReasons(h)
            return float(sm), float(smax), float(pw), int(rs)
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
        target = self.uuid or str(self.index)
        out = subprocess.run(["nvidia-smi", f"--id={target}", f"--query-gpu={q}", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=5).stdout.strip().split(",")
        return float(out[0]), float(out[1]), float(out[2]), int(out[3].strip(), 16)

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self._one())
            except Exception:
                pass
            self._stop.wait(self.period)

    def start(self):
        self._open()
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t is not None:
            self._t.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "source": self.source,
                    "reasons": ["no clock samples"]}
        sm = [x[0] for x in self.samples]
        reasons = sorted({name for name, bit in self.REASONS for x in self.samples if x[3] & bit})
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": max(x[1] for x in self.samples),
                "power_w_max": max(x[2] for x in self.samples), "samples": len(sm), "source": self.source,
                "period_ms": int(1000 * self.period), "reasons": reasons}


# ----------------------------------------------------------------------------- reference arm / CPU baseline


def oracle_steps(G, cam, views, meas, seq, n_steps, budget_s=None):
    """Full training steps of the FP64 oracle (forward, losses, adjoints) on the host:
    returns (pairs, seconds, steps run).  Stops early once budget_s has elapsed."""
    from oracle import core, losses
    from paper_2405_20693_b300 import inputs as I

    pairs, t0, done = 0, time.perf_counter(), 0
    for k in range(n_steps):
        if budget_s is not None and done > 0 and time.perf_counter() - t0 > budget_s:
            break
        v, off = seq[k % len(seq)]
        img, pp = core.render(G, views[v:v + 1], cam, Q=9.0)
        L, dimg = losses.projection_loss(img, meas[v:v + 1].astype(np.float64), 0.25)
        gd = I.patch_grid(off, D_TV, N_OUT)
        vol, vp = core.voxelize(G, gd, 11.345)
        Ltv, dvol = losses.tv3d(vol.reshape(D_TV, D_TV, D_TV), 0.05)
        core.render_backward(G, views[v:v + 1], cam, dimg, Q=9.0)
        core.voxelize_backward(G, gd, dvol.ravel(), 11.345)
        pairs += pp + vp
        done += 1
    return pairs, time.perf_counter() - t0, done


def make_scale_workload(seed: int, device):
    """The headline workload: 500k Gaussians sampled from the phantom's support
    (per-axis scales log-U[0.002, 0.05], uniform random rotations, rho = 0.15 V(p)),
    75 cone-beam views of 512^2, and (with a device for the chord evaluation) the
    measured projections with Poisson noise at 1e5 photons per ray."""
    from paper_2405_20693_b300 import inputs as I

    ph, vol = I.normalised_phantom(seed, N_OUT)
    G = I.init_from_volume(vol, I.cube_grid(N_OUT), SCALE_M, seed + 3, scale_override=(0.002, 0.05), random_rot=True)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(SCALE_V), I.CONE_L_SO)
    meas = None
    if device is not None:
        clean = I.phantom_projections(ph, views, cam, device=device)
        meas = I.poisson_noise(clean, seed + 3, 1e5).astype(np.float32)
    return G, cam, views, meas


def scale_patch_origins(seed: int, n_steps: int) -> np.ndarray:
    """Origins of the 8 TV patches of each step, [n_steps, 8, 3] float32: offsets
    U{0..224}^3 voxels of the 256^3 grid over [-1, 1]^3 (seeded)."""
    g = np.random.Generator(np.random.PCG64(seed + 4))
    offs = g.integers(0, N_OUT - D_TV + 1, (n_steps, SCALE_NP, 3))
    return (-1.0 + offs * (2.0 / N_OUT)).astype(np.float32)


def host_cpu():
    """(threads this process may use, CPU model)."""
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return n, model


# worker side of the oracle sample: the upstream gradients are drawn once per process
_SAMPLE_CACHE = {}


def _oracle_sample_shard(task):
    """One shard of the oracle sample: forward and backward of the sampled Gaussians
    over all views (render, render_backward with a seeded dL/dI), and the voxelizer
    forward of the patches and the full volume with the patches' backward (seeded
    dL/dV).  Returns (pairs, seconds)."""
    from oracle import core
    from paper_2405_20693_b300 import inputs as I

    G, views, cam, patch_gd, full_gd = task
    key = (views.shape[0], cam.H, cam.W, patch_gd.shape[0])
    if key not in _SAMPLE_CACHE:
        g = np.random.default_rng(11)
        _SAMPLE_CACHE[key] = (g.standard_normal((views.shape[0], cam.H, cam.W)) * 1e-6,
                              g.standard_normal(patch_gd.shape[0] * D_TV ** 3) * 1e-4)
    dimg, dvol = _SAMPLE_CACHE[key]
    t0 = time.perf_counter()
    _, pp = core.render(G, views, cam, Q=9.0)
    core.render_backward(G, views, cam, dimg, Q=9.0)
    _, vp = core.voxelize(G, patch_gd, 11.345)
    core.voxelize_backward(G, patch_gd, dvol, 11.345)
    _, fp = core.voxelize(G, full_gd, 11.345)
    return pp + vp + fp, time.perf_counter() - t0


class OracleSampler:
    """Times the FP64 oracle on bounded samples of the headline workload on the host
    cores: each sample is a seeded subset of the Gaussians, split over a spawned
    process pool (one shard per worker) or run in this process (cores = 1).  The
    oracle runs as it stands; only the Gaussians are partitioned across processes.
    The projection loss (a fixed per-pixel cost, small next to the pairs at this
    size) is not part of the sample."""

    def __init__(self, G, views, cam, workers: int):
        from paper_2405_20693_b300 import inputs as I

        self.G, self.views, self.cam = G, views, cam
        self.full_gd = np.asarray(I.cube_grid(N_OUT), np.float64)
        self.workers = max(1, int(workers))
        self.pool = None
        if self.workers > 1:
            import multiprocessing as mp

            self.pool = mp.get_context("spawn").Pool(self.workers)

    def patch_grids(self, origins):
        from paper_2405_20693_b300 import inputs as I

        return np.stack([np.asarray(I.grid_desc(o, (2.0 / N_OUT,) * 3, (D_TV,) * 3), np.float64) for o in origins])

    def run(self, n_gauss: int, seed: int, origins):
        """(pairs, wall seconds) of one sample of n_gauss Gaussians."""
        idx = np.sort(np.random.default_rng(seed).choice(self.G.M, size=n_gauss, replace=False))
        sub = self.G.subset(idx).astype(np.float64)
        gd = self.patch_grids(origins)
        if self.pool is None:
            p, _ = _oracle_sample_shard((sub, self.views, self.cam, gd, self.full_gd))
            return p, None
        shards = np.array_split(np.arange(n_gauss), self.workers)
        tasks = [(sub.subset(s), self.views, self.cam, gd, self.full_gd) for s in shards if len(s)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_sample_shard, tasks)
        return sum(r[0] for r in res), time.perf_counter() - t0

    def timed(self, n_gauss: int, seed: int, origins):
        t0 = time.perf_counter()
        p, wall = self.run(n_gauss, seed, origins)
        return p, (wall if wall is not None else time.perf_counter() - t0)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def cpu_baseline_scale(G, views, cam, n_gauss=6000):
    """The oracle's pairs/s on one bounded sample of the headline workload, on all the
    host's cores and on one core (same sample)."""
    cores, model = host_cpu()
    origins = scale_patch_origins(0, 1)[0]
    out = {"unit": "pairs/s", "kind": "oracle", "cpu_model": model, "nproc": cores}
    one = OracleSampler(G, views, cam, 1)
    one.timed(200, 1, origins)  # loads the library
    p1, s1 = one.timed(n_gauss, 2, origins)
    out["single_core"] = {"value": p1 / s1, "cores": 1, "seconds": s1, "pairs": p1}
    if cores > 1:
        w = min(cores, 32)
        allc = OracleSampler(G, views, cam, w)
        allc.timed(w * 4, 1, origins)  # spawns and warms the workers
        pa, sa = allc.timed(n_gauss, 2, origins)
        allc.close()
        out["all_cores"] = {"value": pa / sa, "cores": w, "seconds": sa, "pairs": pa}
    best = out.get("all_cores", out["single_core"])
    out.update(value=best["value"], cores=best["cores"],
               sample=f"{n_gauss} seeded Gaussians of the 500k set (the same subset on 1 core and on "
                      f"{best['cores']} processes, Gaussians split evenly): FP64 oracle render + adjoint over all "
                      f"75 views of 512^2 with a seeded dL/dI, voxelize + adjoint of 8 32^3 patches, voxelize of "
                      f"the 256^3 volume; the projection loss is not in the sample")
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    G, cam, views, _ = make_scale_workload(0, None)
    cores, model = host_cpu()
    w = min(cores, 32)
    smp = OracleSampler(G, views, cam, w)
    n_step = 400 * w  # about a second of oracle work per step on each worker
    origins = scale_patch_origins(0, args.warmup + args.steps)
    for k in range(args.warmup):
        smp.timed(n_step, 1000 + k, origins[k])
    pairs, secs = 0, 0.0
    for k in range(args.steps):
        p, t = smp.timed(n_step, 2000 + k, origins[args.warmup + k])
        pairs += p
        secs += t
    smp.close()
    value = pairs / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": SCALE_WORKLOAD, "oracle": "FP64 C++ scatter form, one process per core"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": w, "kind": "oracle", "nproc": cores,
                             "cpu_model": model,
                             "sample": f"each step {n_step} seeded Gaussians of the 500k set split over {w} "
                                       "processes: render + adjoint over all 75 views, voxelize + adjoint of the "
                                       "step's 8 TV patches, voxelize of the 256^3 volume (no projection loss)"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SCALE_WORKLOAD = ("differentiation at scale: 500k Gaussians (per-axis scales log-U[0.002, 0.05], random rotations) "
                  "from a seeded 40-ellipsoid 256^3 phantom; cone beam L_SO 1000 mm, L_SD 1500 mm; all 75 views x "
                  "512^2 at 0.8 mm in one launch against Poisson-noised projections (1e5 photons/ray), L1 + 0.25 "
                  "D-SSIM; 8 random 32^3 TV patches (0.05) and the full 256^3 volume voxelized; full backward; Adam")


def _has_cuda():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


# ----------------------------------------------------------------------------- our arm


# the source file of each profiled kernel (with every shared .cuh header)
KERNEL_SOURCES = {"splat_bwd": "raster.cu", "splat_fwd": "raster.cu", "project_bwd": "raster.cu", "project": "raster.cu",
                  "loss": "loss.cu", "fdk_bp": "fdk.cu", "fdk_filter": "fdk.cu", "init_knn": "fdk.cu",
                  "init_select_hist": "fdk.cu", "metrics": "metrics.cu", "densify": "densify.cu"}


def _included(csrc: str, name: str, seen: set):
    """name and the local headers it includes (#include "..."), transitively."""
    if name in seen or not os.path.exists(os.path.join(csrc, name)):
        return
    seen.add(name)
    with open(os.path.join(csrc, name)) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith('#include "'):
                _included(csrc, os.path.basename(line.split('"')[1]), seen)


def source_hash(kernel: str | None = None):
    """Hash of the sources a kernel is built from: its .cu file and the local headers
    it includes (all of csrc when kernel is None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2405_20693_b300", "csrc")
    files = set(os.listdir(csrc))
    if kernel is not None:
        files = set()
        _included(csrc, KERNEL_SOURCES[kernel], files)
    for f in sorted(files):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_summary():
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            return json.load(f)
    except Exception:
        return None


def _entry(t, kernel: str, workload: str | None):
    """The summary's (source hash, per-workload section) for a kernel: the headline
    and one-scan kernels under "workloads", the auxiliary kernels under "other"."""
    if not t:
        return None, None
    if workload is not None:
        return t.get("source_hashes", {}).get(kernel), t.get("workloads", {}).get(workload, {})
    o = t.get("other", {})
    return o.get("source_hashes", {}).get(kernel), o


def _current(t, kernel: str, workload: str | None) -> bool:
    h, _ = _entry(t, kernel, workload)
    return kernel in KERNEL_SOURCES and h is not None and h == source_hash(kernel)


def ncu_traffic(kernel: str, workload: str | None = None):
    """DRAM bytes per launch from the committed ncu summary of the workload ("scale":
    the headline step, "one_scan"; None: the auxiliary kernels), if it was taken on
    the kernel's current sources; else None."""
    t = _ncu_summary()
    return _entry(t, kernel, workload)[1].get("kernels", {}).get(kernel) if _current(t, kernel, workload) else None


def ncu_pipes(kernel: str, workload: str | None = None):
    """FMA and XU (MUFU) pipe utilisation (% of peak sustained) of the kernel from the
    committed ncu summary of the workload, if it was taken on the kernel's current
    sources; else None."""
    t = _ncu_summary()
    return _entry(t, kernel, workload)[1].get("pipes", {}).get(kernel) if _current(t, kernel, workload) else None


def measure_batched(dev, rounds=20, n_scans=16, seed=5):
    """Scans/hour of the uneven 16-scan workload: one scan at a time (each scan's
    fused training step, eagerly, scan after scan) against all scans batched (one
    CUDA graph per round, one branch per scan on its own stream).  Both run the same
    per-scan arithmetic; the scans/hour figures assume 30,000 iterations per scan."""
    import torch

    from paper_2405_20693_b300 import engine, r2g
    from paper_2405_20693_b300 import inputs as I

    specs = I.batched_specs(n_scans, seed)
    scans = []
    for sp in specs:
        G, cam, views, meas, _ = I.make_scan(sp, device=dev)
        scans.append(engine.Scan(G, views, meas, cam, n_out=sp.n_out, D=D_TV, device=dev, seed=sp.seed))
    # each scan's tile shape by measurement (its fused step alone, state restored); both
    # legs below use the chosen shapes
    tuned = [sc.autotune_tile() for sc in scans]
    # one scan at a time: each scan's steps back to back on one stream, their entries
    # preloaded in a device table so the host only issues the calls
    stream = torch.cuda.current_stream()
    elem = engine.ctypes_sizeof_entry()
    per_scan_ms = []
    for sc in scans:
        t = np.zeros((rounds + 3, 8), np.int32)
        f = t.view(np.float32)
        for k in range(rounds + 3):
            v, it, origin = sc.next_entry()
            t[k, 0], t[k, 1] = v, it
            f[k, 2:5] = origin
        tdev = torch.as_tensor(t, device=dev)
        evs = []
        for k in range(rounds + 3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r2g.r2g_train_step(sc.job, tdev.data_ptr() + k * elem, stream)
            e1.record(stream)
            if k >= 3:
                evs.append((e0, e1))
        torch.cuda.synchronize()
        per_scan_ms.append(sum(a.elapsed_time(b) for a, b in evs) / rounds)
    plain_ms = sum(per_scan_ms)
    # all scans batched: one graph per round
    bt = engine.BatchTrainer(scans, graph=True, device=dev)
    for _ in range(3):
        bt.round()
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(rounds):
        stream.synchronize()
        bt._fill()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.graph.replay()
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    batched_ms = ms / rounds
    overflow = any(sc.overflowed() for sc in scans)
    iters = 30000
    return {"workload": f"{n_scans} uneven cone-beam scans (seed {seed}): M log-U[5k, 300k], 25/50/75 views, "
                        "256^2/512^2 detectors, 128^3/256^3 volumes, random init; one training iteration each per round",
            "gaussians": [sp.M for sp in specs],
            "tiles": ["%dx%d" % min(t, key=t.get) for t in tuned],
            "tile_note": "per scan, the tile shape with the shortest fused step among 8x8, 16x16, 32x8, 32x32 "
                         "(4 timed steps each on a restored copy of the state)",
            "plain_ms_per_iteration_of_all_scans": plain_ms, "batched_ms_per_round": batched_ms,
            "scans_per_hour_plain": n_scans * 3600.0 / (iters * plain_ms * 1e-3),
            "scans_per_hour_batched": n_scans * 3600.0 / (iters * batched_ms * 1e-3),
            "speedup": plain_ms / batched_ms, "iterations_per_scan": iters, "list_overflow": overflow,
            "timing": f"CUDA events, mean of {rounds} rounds after 3 warm-up rounds"}


def measure_serving(dev, n_requests=16, mean_interarrival_s=0.25, max_iters=500, check_every=250, seed=5):
    """p50/p99 time-to-volume and scans/hour of the continuous-batching server on a
    seeded Poisson stream of requests with the uneven multi-scan size mix.  Scanner
    data is prepared before the clock starts (a server receives projections, it
    does not synthesise them).  Arrivals are compressed in time and iterations
    capped (max_iters, PSNR target 35 dB checked every check_every) so the run takes
    seconds; both are stated in the output."""
    from paper_2405_20693_b300 import inputs as I
    from paper_2405_20693_b300 import serve

    specs = I.batched_specs(n_requests, seed=seed)
    reqs = serve.poisson_requests(n_requests, mean_interarrival_s, seed=6, specs=specs, max_iters=max_iters,
                                  psnr_target=35.0, check_every=check_every)
    for r in reqs:
        r.data = I.make_scan(r.spec, device=dev)
    import torch

    budget = int(0.5 * torch.cuda.get_device_properties(dev).total_memory)
    srv = serve.Server(budget, D=D_TV, device=dev)
    res = srv.run(reqs)
    out = serve.summarize(res, srv.wall)
    its = [r.iters for r in res]
    out.update({"arrivals": f"Poisson, mean inter-arrival {mean_interarrival_s} s (seed 6), compressed from the "
                            "2/min stream", "iterations_cap": max_iters, "psnr_target_db": 35.0,
                "iterations_per_request": {"p50": float(np.percentile(its, 50)), "p99": float(np.percentile(its, 99)),
                                           "max": int(max(its)), "mean": float(np.mean(its))},
                "check_every": check_every, "hbm_budget_bytes": budget, "max_resident": srv.max_active,
                "rounds": srv.rounds, "mean_final_psnr_db": float(np.mean([r.psnr for r in res]))})
    return out


LSU_PER_CLK = 32   # load/store lanes per SM per clock
BP_LOADS = 4       # detector reads per (voxel, view): one bilinear interpolation


def measure_fdk_init(dev, views_np, meas_np, cam, reps=10, cpu=True):
    """Sec. 4.1 initialisation of the workload's scan on the device: FDK of the 50
    measured views onto the 256^3 output grid, then the draw of 50k Gaussians (tau
    0.05, k 0.15) with their 3-NN scales.  Device time per kernel (event pairs over
    `reps` runs after 3 warm-up runs), the whole initialisation's device time, and the
    back-projection's roofline: (voxel, view) updates per second against the issue
    rate of its 4 detector reads per update on the SMs' load/store lanes.  With cpu,
    the FP64 oracle back-projects one z slice of the same grid on the host."""
    import torch

    from oracle import fdk as ofdk
    from paper_2405_20693_b300 import engine, r2g
    from paper_2405_20693_b300 import inputs as I

    vd = torch.as_tensor(np.ascontiguousarray(views_np, np.float32), device=dev)
    md = torch.as_tensor(np.ascontiguousarray(meas_np, np.float32), device=dev)
    gd = I.cube_grid(N_OUT)

    def once():
        vol = engine.fdk_volume(vd, md, cam, gd, device=dev)
        return vol, engine.init_gaussians(vol, gd, M_GAUSS, device=dev)

    for _ in range(3):
        once()
    torch.cuda.synchronize()
    ids = [r2g.PROFILE_KERNELS.index(n) for n in ("fdk_filter", "fdk_bp", "init_select", "init_knn")]
    r2g.r2g_profile_enable(True, 16 * reps + 16)
    r2g.r2g_profile_select(sum(1 << k for k in ids))
    r2g.r2g_profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        vol, G = once()
    e1.record()
    torch.cuda.synchronize()
    ks = {}
    for k in ids:
        n, t = r2g.r2g_profile_read(k)
        ks[r2g.PROFILE_KERNELS[k]] = t / max(n, 1)
    r2g.r2g_profile_enable(False)
    total_ms = e0.elapsed_time(e1) / reps
    updates = float(N_OUT) ** 3 * views_np.shape[0]
    pk = peaks()
    lsu_peak = SM_COUNT * LSU_PER_CLK * pk["sm_max_mhz"] * 1e6 / BP_LOADS
    ach = updates / (ks["fdk_bp"] * 1e-3)
    out = {"ms_per_init": total_ms, "kernels_ms": ks, "gaussians": int(G[0].shape[0]),
           "grid": f"{N_OUT}^3", "views": int(views_np.shape[0]),
           "roofline": {"kernel": "fdk_bp", "bound": "lsu", "achieved": ach / 1e9, "peak": lsu_peak / 1e9,
                        "unit": "G voxel-view updates/s", "frac": ach / lsu_peak, "traffic": ncu_traffic("fdk_bp"),
                        "peak_note": f"{LSU_PER_CLK} load lanes/clk/SM / {BP_LOADS} reads per update x {SM_COUNT} "
                                     f"SMs x {pk['sm_max_mhz']:.0f} MHz"},
           "note": "ms_per_init: device time of the whole initialisation (FDK filter + back-projection + draw + "
                   "3-NN) incl. the host's read of the drawn count"}
    if cpu:
        t0 = time.perf_counter()
        filt = ofdk.fdk_filter(meas_np[:2], cam)
        t_filt = (time.perf_counter() - t0) / 2
        sl = np.asarray(gd, np.float64).copy()
        sl[2] = -1.0 + (N_OUT // 2) * (2.0 / N_OUT)
        sl[8] = 1
        F = np.repeat(filt[:1], views_np.shape[0], axis=0)
        t0 = time.perf_counter()
        ofdk.fdk_backproject(F, views_np, cam, sl, 2 * np.pi / views_np.shape[0])
        t_bp = time.perf_counter() - t0
        upd = float(N_OUT) ** 2 * views_np.shape[0]
        out["cpu_baseline"] = {"value": upd / t_bp / 1e9, "unit": "G voxel-view updates/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"FP64 oracle back-projection of one {N_OUT}^2 z slice from "
                                         f"{views_np.shape[0]} views ({t_bp:.2f} s); filter "
                                         f"{t_filt * 1e3:.0f} ms per 512^2 view"}
    return out


def measure_metrics(dev, reps=20):
    """r2g_volume_metrics (3D PSNR and SSIM over axial, coronal and sagittal slices)
    of two 256^3 volumes: device time per call (CUDA events, after 3 warm-up calls)
    and its HBM roofline with the algorithmic bytes = both volumes read once."""
    import torch

    from paper_2405_20693_b300 import engine, r2g
    from paper_2405_20693_b300 import inputs as I

    ref = torch.as_tensor(I.normalised_phantom(0, N_OUT)[1].astype(np.float32), device=dev)
    g = torch.Generator(device=dev).manual_seed(1)
    est = (ref + 0.05 * torch.randn(ref.shape, generator=g, device=dev)).clamp(0, 1)
    out = torch.empty(6, dtype=torch.float64, device=dev)
    ws = torch.empty(r2g.r2g_metrics_workspace_size(N_OUT, N_OUT, N_OUT), dtype=torch.uint8, device=dev)
    for _ in range(3):
        r2g.r2g_volume_metrics(est, ref, out, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        r2g.r2g_volume_metrics(est, ref, out, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    algo = 2 * 4 * N_OUT ** 3
    pk = peaks()
    vals = dict(zip(engine.METRIC_KEYS, out.cpu().tolist()))
    # the bound that binds: per voxel and orientation the window's separable passes over
    # the five moment maps (2 x 5 x 11 FMAs), the three products and ~16 operations of
    # the SSIM ratio, ~129 FP32 lane operations, at 128 per clock per SM; reading both
    # volumes once (128 MB) would take a tenth of that time at the measured HBM rate
    units = 3.0 * N_OUT ** 3
    peak = SM_COUNT * FP32_PER_CLK * pk["sm_max_mhz"] * 1e6 / SSIM_OPS_PER_VOXEL
    ach = units / (ms * 1e-3)
    return {"ms_per_call": ms, "volume": f"{N_OUT}^3", "values_noisy_phantom": vals,
            "roofline": {"kernel": "slice_ssim", "bound": "alu", "achieved": ach / 1e9, "peak": peak / 1e9,
                         "unit": "G voxel-orientations/s", "frac": ach / peak, "ops_per_unit": SSIM_OPS_PER_VOXEL,
                         "traffic": ncu_traffic("metrics"),
                         "hbm": {"algorithmic_bytes": algo, "achieved_gbs": algo / (ms * 1e-3) / 1e9,
                                 "peak_gbs": pk["hbm_gbs"], "frac": algo / (ms * 1e-3) / 1e9 / pk["hbm_gbs"]},
                         "peak_note": f"FP32 {FP32_PER_CLK}/clk/SM / {SSIM_OPS_PER_VOXEL} ops x {SM_COUNT} SMs x "
                                      f"{pk['sm_max_mhz']:.0f} MHz (of measured sm_max_mhz)"}}


def measure_limited_angle(dev, iters=3000):
    """App. E's limited-angle setting: 100 cone-beam views over 0-150, 0-120 and
    0-90 degrees and a full-circle control (12k Gaussians, 128^2 detector, 64^3
    volume, same random initialisation), trained together by the batched fused step;
    the volumes' PSNR and 3D SSIM against the phantom (r2g_volume_metrics)."""
    import torch

    from paper_2405_20693_b300 import engine
    from paper_2405_20693_b300 import inputs as I

    spans = (360.0, 150.0, 120.0, 90.0)
    scans, gts = [], []
    for sp in spans:
        G, cam, views, meas, vol = I.make_scan(I.ScanSpec(230, 12000, 100, 128, 64, span=sp), device=dev)
        scans.append(engine.Scan(G, views, meas, cam, n_out=64, D=16, total_iters=iters, seed=3, device=dev))
        gts.append(torch.as_tensor(vol.astype(np.float32), device=dev))
    bt = engine.BatchTrainer(scans, graph=True, device=dev)
    for _ in range(iters):
        bt.round()
    torch.cuda.synchronize()
    vox = engine.Voxelizer(12000, I.cube_grid(64), device=dev)
    out = {}
    for sp, sc, gt in zip(spans, scans, gts):
        m = engine.volume_metrics(vox.forward(*sc.state.params()).view(64, 64, 64), gt, device=dev)
        out[f"{sp:g}deg"] = {"psnr": m["psnr"], "ssim": m["ssim"]}
    return {"iterations": iters, "views": 100, "results": out}


def measure_adaptive(dev, iters=3000):
    """Adaptive density control (Sec. 4.2.3) on one scan of the uneven workload's kind
    (seed 242: 20k Gaussians from the random initialisation, 50 views of 256^2, 128^3
    volume), trained with and without it for `iters` fused iterations (one batched
    round each), densifying every 100 iterations from 500 to iters / 2 (the paper's
    500..15k of 30k, compressed): Gaussian counts, the volumes' PSNR / 3D SSIM, and the
    device time of r2g_densify with its HBM roofline (algorithmic bytes: the four
    11-float state arrays read for every input Gaussian and written for every output
    one, plus the two statistics arrays)."""
    import torch

    from paper_2405_20693_b300 import engine, r2g
    from paper_2405_20693_b300 import inputs as I

    spec = I.ScanSpec(242, 20000, 50, 256, 128)
    G, cam, views, meas, vol = I.make_scan(spec, device=dev)
    gt = torch.as_tensor(vol.astype(np.float32), device=dev)
    plain = engine.Scan(G, views, meas, cam, n_out=128, D=32, total_iters=iters, seed=1, device=dev)
    ac = engine.Scan(G, views, meas, cam, n_out=128, D=32, total_iters=iters, seed=1, device=dev)
    ac.enable_adaptive(10 * G.M, start=500, stop=iters // 2, every=100)
    bt = engine.BatchTrainer([plain, ac], graph=True, device=dev)
    kid = r2g.PROFILE_KERNELS.index("densify")
    r2g.r2g_profile_enable(True, 4096)
    r2g.r2g_profile_select(1 << kid)
    r2g.r2g_profile_reset()
    counts, ins = [], []
    for _ in range(iters):
        m_before = ac.M
        bt.round()
        if ac.M != m_before or (ac.it % 100 == 0 and 500 <= ac.it <= iters // 2):
            counts.append((ac.it, ac.M))
            ins.append((m_before, ac.M))
    torch.cuda.synchronize()
    n, t = r2g.r2g_profile_read(kid)
    r2g.r2g_profile_enable(False)
    out = {"iterations": iters, "densify_every": 100, "densify_from_to": [500, iters // 2],
           "gaussians": {"start": G.M, "end": ac.M, "trajectory": counts}}
    for name, sc in (("without", plain), ("with", ac)):
        vox = engine.Voxelizer(sc.M, I.cube_grid(128), device=dev)
        m = engine.volume_metrics(vox.forward(*sc.state.params()).view(128, 128, 128), gt, device=dev)
        out[name] = {"psnr": m["psnr"], "ssim": m["ssim"], "gaussians": sc.M}
    if n:
        ms = t / n
        algo = sum(4 * 11 * 4 * (a + b) + 8 * a for a, b in ins) / max(1, len(ins))
        pk = peaks()
        out["densify_kernel"] = {"calls": n, "ms_per_call": ms,
                                 "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9,
                                              "peak": pk["hbm_gbs"], "unit": "GB/s",
                                              "frac": algo / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], "traffic": None}}
    return out


def voxel_box_counter(sc):
    """Voxels of each Gaussian's box (|x_k - p_k| <= sqrt(Q3 Sigma_kk), voxel centres)
    inside a D^3 TV patch at a given offset, summed over Gaussians: FP64 on the host
    from the parameters at the start of the timed region."""
    mean, scale, quat, rho = (t.detach().double().cpu().numpy() for t in sc.state.params())
    q = quat / np.linalg.norm(quat, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(-1, 3, 3)
    sig_kk = np.einsum('nkj,nkj->nk', R * scale[:, None, :], R * scale[:, None, :])
    vs = 2.0 / N_OUT
    ext = np.sqrt(11.345 * sig_kk) / vs

    def count(off):
        c = (mean - (-1.0 + np.asarray(off) * vs)) / vs - 0.5
        lo = np.maximum(0, np.ceil(c - ext))
        hi = np.minimum(D_TV - 1, np.floor(c + ext))
        n = np.clip(hi - lo + 1, 0, None)
        return int(np.prod(n, axis=1).sum())
    return count


def job_totals(dist, ms: float, pairs: float, device):
    """Whole-job (device ms, pairs) of a timed region across ranks: the slowest rank's
    time and every rank's pairs (independent replicas; one process per GPU).  dist =
    torch.distributed with an initialised process group, or None for one process."""
    if dist is None:
        return ms, pairs
    import torch

    tt = torch.tensor([ms, pairs], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


def slowest(dist, seconds: float, device) -> float:
    """The largest of a per-rank wall time over ranks (dist None: as is)."""
    if dist is None:
        return seconds
    import torch

    tt = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt[0])


def splat_roofline(name: str, units: float, avg_ms: float, pk: dict, workload: str) -> dict:
    """ALU roofline of a splat kernel: units (gated pairs per launch) / mean launch
    time, against min(MUFU ex2 rate, FP32 rate / ops per pair) at the maximum SM
    clock, charging the scope table's ops per pair (forward 10, backward 20); the
    fraction on the kernel's own reduced count is reported beside it."""
    f = pk["sm_max_mhz"] * 1e6
    mufu = SM_COUNT * MUFU_PER_CLK * f
    fp32 = SM_COUNT * FP32_PER_CLK * f
    fwd = name.endswith("fwd")
    ops, own = (OPS_FWD, OWN_OPS_FWD) if fwd else (OPS_BWD, OWN_OPS_BWD)
    peak = min(mufu, fp32 / ops) / 1e9
    peak_own = min(mufu, fp32 / own) / 1e9
    ach = units / (avg_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpair/s", "frac": ach / peak,
            "ops_per_pair": ops, "frac_own_ops": ach / peak_own, "own_ops_per_pair": own,
            "ms_per_launch": avg_ms, "units_per_launch": units,
            "traffic": ncu_traffic(name, workload), "pipes_pct_of_peak": ncu_pipes(name, workload),
            "peak_note": f"min(MUFU ex2 {MUFU_PER_CLK}/clk/SM, FP32 {FP32_PER_CLK}/clk/SM / {ops} ops) x {SM_COUNT} "
                         f"SMs x {pk['sm_max_mhz']:.0f} MHz (of measured sm_max_mhz; no FP32 peak is measured)"}


def _profile_breakdown(step, ks, n_brk):
    """Event pairs around every kernel group over the steps ks (untimed)."""
    import torch

    from paper_2405_20693_b300 import r2g

    r2g.r2g_profile_enable(True, 64 * n_brk + 64)
    r2g.r2g_profile_select(0xFFFFFFFF)
    r2g.r2g_profile_reset()
    for k in ks:
        step(k)
    torch.cuda.synchronize()
    out = {}
    for kid, name in enumerate(r2g.PROFILE_KERNELS):
        n, t = r2g.r2g_profile_read(kid)
        if n:
            out[name] = t / len(ks)
    r2g.r2g_profile_enable(False)
    return out


def measure_scale(args, dev, dist, seed, world):
    """The headline: the batch form of r2g_train_step on the differentiation-at-scale
    workload (see the module docstring).  Per step: all 75 views, the step's 8 TV
    patches (seeded origins), the full volume.  Returns the fields of the JSON line."""
    import torch

    from paper_2405_20693_b300 import engine, r2g

    G, cam, views_np, meas_np = make_scale_workload(seed, dev)
    n_brk = min(args.steps, 5)
    n_all = args.warmup + n_brk + args.steps
    origins = torch.as_tensor(scale_patch_origins(seed, n_all), device=dev)
    tab = np.zeros((n_all, 8), np.int32)
    tab[:, 1] = np.arange(n_all)
    table = torch.as_tensor(tab, device=dev)
    sc = engine.Scan(G, views_np, meas_np, cam, n_out=N_OUT, D=D_TV, device=dev, headroom=1.25, all_views=True,
                     n_patches=SCALE_NP, full_volume=True, tile=(16, 16))
    # tile shape by measurement (the fused step per shape, on a restored copy of the state)
    tiles = sc.autotune_tile(tiles=SCALE_TILES, steps=2)
    elem = engine.ctypes_sizeof_entry()
    stream = torch.cuda.current_stream()
    org0, org_row = origins.data_ptr(), 4 * 3 * SCALE_NP

    def step(k):
        sc.job.patch_origins = org0 + k * org_row
        r2g.r2g_train_step(sc.job, table.data_ptr() + k * elem, stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    assert not sc.overflowed(), "list capacity overflow in the warm-up"
    breakdown = _profile_breakdown(step, range(args.warmup, args.warmup + n_brk), n_brk)
    dom = max(breakdown, key=breakdown.get)
    t0_steps = args.warmup + n_brk
    # algorithmic pairs (counting runs, untimed, on the parameters at the start of the
    # timed region): all views, each step's 8 patches, the full volume
    from paper_2405_20693_b300 import inputs as I

    mean, scale, quat, rho = sc.state.params()
    sc.rast.forward(mean, scale, quat, rho, sc.views, sc.image, check=True, count=True)
    pix = sc.rast.pair_count()
    org_np = origins.cpu().numpy()
    vox = []
    for k in range(t0_steps, t0_steps + args.steps):
        sc.vox.set_grids([I.grid_desc(o, (2.0 / N_OUT,) * 3, (D_TV,) * 3) for o in org_np[k]])
        sc.vox.forward(mean, scale, quat, rho, sc.vol, check=True, count=True)
        vox.append(sc.vox.pair_count())
    sc.full_vox.forward(mean, scale, quat, rho, sc.full_vol.view(-1), check=True, count=True)
    full = sc.full_vox.pair_count()
    # the superset the raster kernels walk: every record's pixel box (stated FP32 bounds)
    proj = torch.empty((SCALE_V, sc.M, 8), dtype=torch.float32, device=dev)
    prect = torch.empty((SCALE_V, sc.M, 4), dtype=torch.int32, device=dev)
    r2g.r2g_project(mean, scale, quat, rho, sc.views, sc.rast.cam, sc.rast.opts, proj, prect)
    rc = prect.long()
    box_pix = int(((rc[..., 1] - rc[..., 0] + 1) * (rc[..., 3] - rc[..., 2] + 1))[proj[..., 7] == 1.0].sum())
    del proj, prect, rc
    sc.job = sc._make_job()  # a checked run that had to regrow a workspace moved it
    total_pairs = float(args.steps * pix + sum(vox) + args.steps * full)
    st = sc.state
    start_state = [t.clone() for t in (st.raw, st.act, st.m, st.v)]

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kf, kb = r2g.PROFILE_KERNELS.index("splat_fwd"), r2g.PROFILE_KERNELS.index("splat_bwd")
    kd = r2g.PROFILE_KERNELS.index(dom)
    r2g.r2g_profile_enable(True, 8 * args.steps + 64)
    r2g.r2g_profile_select((1 << kf) | (1 << kb) | (1 << kd))
    r2g.r2g_profile_reset()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clock = ClockSampler(gpu_id, dev.index or 0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clock.start()
    launches0 = r2g.r2g_launch_count()
    for j in range(args.steps):
        evs[j][0].record(stream)
        step(t0_steps + j)
        evs[j][1].record(stream)
    torch.cuda.synchronize()
    launches = r2g.r2g_launch_count() - launches0
    clocks = clock.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    assert not sc.overflowed(), "list capacity overflow inside the timed region"
    prof = {}
    for name, kid in (("splat_fwd", kf), ("splat_bwd", kb), (dom, kd)):
        n, t = r2g.r2g_profile_read(kid)
        prof[name] = (n, t)
    r2g.r2g_profile_enable(False)
    r2g.r2g_profile_select(0xFFFFFFFF)
    ms_job, pairs_job = job_totals(dist, ms, total_pairs, dev)
    value = pairs_job / (ms_job * 1e-3)

    # end to end through the public API: every step's 75 measured views, their geometry
    # rows, the 8 patch origins and the round entry go host -> device from pinned memory
    # (one r2g_train_step_host_batch call, staged on a copy stream), the losses come back
    NS = 2
    meas_host = torch.from_numpy(np.ascontiguousarray(meas_np, np.float32)).pin_memory()
    views_host = torch.from_numpy(np.ascontiguousarray(views_np, np.float32)).pin_memory()
    ent_host = torch.from_numpy(tab.copy()).pin_memory()
    org_host = torch.from_numpy(org_np.copy()).pin_memory()
    feed = engine.HostFeed(sc, meas_host, views_host, n_slots=NS, stream=stream)
    for j in range(NS):                            # creates the copy stream and events
        feed.step(0, ent_host.data_ptr() + 32 * j, org_host.data_ptr() + org_row * j)
    feed.finish()
    for t, saved in zip((st.raw, st.act, st.m, st.v), start_state):
        t.copy_(saved)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    loss_sum, n_read = 0.0, 0
    t0 = time.perf_counter()
    for j in range(args.steps):
        k = t0_steps + j
        out = feed.step(0, ent_host.data_ptr() + 32 * k, org_host.data_ptr() + org_row * k)
        if out is not None:
            loss_sum += out[0]
            n_read += 1
    for out in feed.finish():
        loss_sum += out[0]
        n_read += 1
    e2e_s = time.perf_counter() - t0
    assert n_read == args.steps and np.isfinite(loss_sum)
    e2e_s = slowest(dist, e2e_s, dev)
    # the memory-tight form of the same step: views 15 at a time through a workspace for
    # one chunk, every chunk's lists but the last rebuilt in the backward (timed apart)
    rc_out = None
    if not args.no_recompute:
        chunk = 15
        tile = (sc.rast.opts.tile_w, sc.rast.opts.tile_h)
        sc2 = engine.Scan(G, views_np, meas_np, cam, n_out=N_OUT, D=D_TV, device=dev, headroom=1.25,
                          all_views=True, n_patches=SCALE_NP, full_volume=True, tile=tile, view_chunk=chunk)

        def step2(k):
            sc2.job.patch_origins = org0 + k * org_row
            r2g.r2g_train_step(sc2.job, table.data_ptr() + k * elem, stream)

        for k in range(args.warmup):
            step2(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n2 = min(args.steps, 5)
        e0.record(stream)
        for j in range(n2):
            step2(t0_steps + j)
        e1.record(stream)
        torch.cuda.synchronize()
        assert not sc2.overflowed()
        rc_out = {"view_chunk": chunk, "ms_per_step": e0.elapsed_time(e1) / n2, "steps": n2,
                  "raster_ws_bytes": int(sc2.rast.ws.numel()), "raster_ws_bytes_all_views": int(sc.rast.ws.numel()),
                  "note": "the same step with r2g_raster_opts.view_chunk = 15: a workspace for 15 views, the backward "
                          "rebuilding the records and lists of 4 of its 5 chunks; device time per step over the "
                          "first steps of the timed sequence from the warmed-up state of that scan"}
        del sc2
        torch.cuda.empty_cache()
    pk = peaks()
    roofs = {}
    for name in ("splat_fwd", "splat_bwd"):
        n, t = prof[name]
        if n:
            roofs[name] = splat_roofline(name, float(pix), t / n, pk, "scale")
    if dom in roofs:
        roof = roofs[dom]
    else:
        n, t = prof[dom]
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": ncu_traffic(dom, "scale"), "ms_per_launch": t / max(n, 1)}
    return {
        "value": value, "ms_per_step": ms_job / args.steps, "pairs_per_step": total_pairs / args.steps,
        "e2e": {"value": pairs_job / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": feed.bytes_in,
                "d2h_bytes_per_step": 8,
                "note": "per step, one r2g_train_step_host_batch call (engine.HostFeed): the 75 measured views "
                        "(78.6 MB), their geometry rows, the 8 patch origins and the round entry copied from "
                        "pinned host memory into one of two device slots on a copy stream (overlapping the step "
                        "before it), the fused step, the two losses read back to pinned host memory and read by "
                        "the host; the same steps as the device-timed leg, from the same starting state"},
        "gpu_launches": int(launches), "roofline": roof, "splat_rooflines": roofs, "kernels_ms_per_step": breakdown,
        "clocks": clocks, "recompute_lists": rc_out,
        "config": {"workload": SCALE_WORKLOAD, "gaussians": int(sc.M), "views_per_step": SCALE_V,
                   "detector": "512x512", "tv_patches_per_step": SCALE_NP, "full_volume": f"{N_OUT}^3",
                   "pixel_pairs_per_step": pix, "voxel_pairs_per_step_patches": sum(vox) / args.steps,
                   "voxel_pairs_per_step_full_volume": full, "box_pixel_pairs_per_step": box_pix,
                   "gated_over_box_pixels": pix / max(1, box_pix),
                   "tile": "%dx%d" % (sc.rast.opts.tile_w, sc.rast.opts.tile_h),
                   "tile_autotune_ms_per_step": {"%dx%d" % t: v for t, v in tiles.items()},
                   "bricks": "8^3", "l2": "not flushed: each step's working set (records 1.2 GB, lists, 79 MB of "
                                         "images) is far larger than the 126 MB L2",
                   "parallelism": f"replicas x{world}",
                   "kernels_note": f"breakdown: event pairs around every kernel group over {n_brk} untimed steps; "
                                   "timed region: events around the two splat kernels (and the dominant kernel)"},
        "_sc": sc, "_G": G, "_views": views_np, "_cam": cam,
    }


def measure_one_scan(args, dev, dist, seed):
    """The one-scan step (one view and one 32^3 TV patch per iteration, 50k Gaussians):
    device-timed value with an L2 flush before every step, end to end through
    r2g_train_step_host, the per-kernel breakdown and the splat rooflines."""
    import torch

    from paper_2405_20693_b300 import engine, r2g
    from paper_2405_20693_b300 import inputs as I

    G, cam, views_np, meas_np = make_workload(seed, dev)
    sc = engine.Scan(G, views_np, meas_np, cam, n_out=N_OUT, D=D_TV, device=dev)
    n_brk = min(args.steps, 200)
    n_all = args.warmup + n_brk + args.steps
    seq = step_sequence(seed, n_all)
    tab = np.zeros((n_all, 8), np.int32)
    for k, (v, off) in enumerate(seq):
        tab[k, 0], tab[k, 1] = v, k
        tab[k, 2:5] = np.asarray([-1.0 + o * (2.0 / N_OUT) for o in off], np.float32).view(np.int32)
    table = torch.as_tensor(tab, device=dev)
    elem = engine.ctypes_sizeof_entry()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def step(k):
        r2g.r2g_train_step(sc.job, table.data_ptr() + k * elem, stream)

    def flushed_step(k):
        flush.zero_()
        step(k)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    assert not sc.overflowed(), "list capacity overflow in the warm-up"
    breakdown = _profile_breakdown(flushed_step, range(args.warmup, args.warmup + n_brk), n_brk)
    t0_steps = args.warmup + n_brk
    mean, scale, quat, rho = sc.state.params()
    counted = {}
    for k in range(t0_steps, t0_steps + args.steps):
        v, off = seq[k]
        if (v, off) in counted:
            continue
        sc.rast.forward(mean, scale, quat, rho, sc.views[v:v + 1], sc.image, check=True, count=True)
        pp = sc.rast.pair_count()
        sc.vox.set_grids(I.patch_grid(off, D_TV, N_OUT))
        sc.vox.forward(mean, scale, quat, rho, sc.vol, check=True, count=True)
        counted[(v, off)] = (pp, sc.vox.pair_count())
    sc.job = sc._make_job()
    pix = [counted[seq[k]][0] for k in range(t0_steps, t0_steps + args.steps)]
    voxp = [counted[seq[k]][1] for k in range(t0_steps, t0_steps + args.steps)]
    total_pairs = float(sum(pix) + sum(voxp))
    st = sc.state
    start_state = [t.clone() for t in (st.raw, st.act, st.m, st.v)]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kf, kb = r2g.PROFILE_KERNELS.index("splat_fwd"), r2g.PROFILE_KERNELS.index("splat_bwd")
    r2g.r2g_profile_enable(True, 4 * args.steps + 64)
    r2g.r2g_profile_select((1 << kf) | (1 << kb))
    r2g.r2g_profile_reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for j in range(args.steps):
        flush.zero_()
        evs[j][0].record(stream)
        step(t0_steps + j)
        evs[j][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    assert not sc.overflowed(), "list capacity overflow inside the timed region"
    prof = {name: r2g.r2g_profile_read(kid) for name, kid in (("splat_fwd", kf), ("splat_bwd", kb))}
    r2g.r2g_profile_enable(False)
    r2g.r2g_profile_select(0xFFFFFFFF)
    ms_job, pairs_job = job_totals(dist, ms, total_pairs, dev)
    NS = 3
    meas_host = torch.from_numpy(np.ascontiguousarray(meas_np, np.float32)).pin_memory()
    views_host = torch.from_numpy(np.ascontiguousarray(views_np, np.float32)).pin_memory()
    ent_host = torch.from_numpy(tab.copy()).pin_memory()
    ent0 = ent_host.data_ptr()
    feed = engine.HostFeed(sc, meas_host, views_host, n_slots=NS, stream=stream)
    for j in range(NS):
        feed.step(seq[j][0], ent0 + 32 * j)
    feed.finish()
    for t, saved in zip((st.raw, st.act, st.m, st.v), start_state):
        t.copy_(saved)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    loss_sum, n_read = 0.0, 0
    t0 = time.perf_counter()
    for j in range(args.steps):
        k = t0_steps + j
        out = feed.step(seq[k][0], ent0 + 32 * k)
        if out is not None:
            loss_sum += out[0]
            n_read += 1
    for out in feed.finish():
        loss_sum += out[0]
        n_read += 1
    e2e_s = slowest(dist, time.perf_counter() - t0, dev)
    assert n_read == args.steps and np.isfinite(loss_sum)
    pk = peaks()
    per_step_pix = sum(pix) / args.steps
    roofs = {name: splat_roofline(name, per_step_pix, t / n, pk, "one_scan") for name, (n, t) in prof.items() if n}
    return {"value": pairs_job / (ms_job * 1e-3), "unit": "pairs/s", "ms_per_step": ms_job / args.steps,
            "e2e": {"value": pairs_job / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": feed.bytes_in,
                    "d2h_bytes_per_step": 8},
            "workload": "one cone-beam scan: 50k Gaussians from a seeded 40-ellipsoid 256^3 phantom, L_SO 1000 mm, "
                        "L_SD 1500 mm, 50 views x 512^2 at 0.8 mm; per step 1 view (L1+0.25 D-SSIM) + one 32^3 TV "
                        "patch (0.05), full backward, Adam",
            "pixel_pairs_per_step": per_step_pix, "voxel_pairs_per_step": sum(voxp) / args.steps,
            "splat_rooflines": roofs, "kernels_ms_per_step": breakdown, "tile": "32x32",
            "l2": "flushed (256 MB write) before every timed step",
            "step_cycle": f"{N_DISTINCT} seeded (view, patch) pairs, repeated",
            "_G": G, "_cam": cam, "_views": views_np, "_meas": meas_np, "_seq": seq[t0_steps:]}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2405_20693_b300 import build

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    seed = rank * 1000
    if args.extras_only:
        if rank == 0:
            print(json.dumps({"volume_metrics": measure_metrics(dev), "limited_angle": measure_limited_angle(dev),
                              "adaptive_control": measure_adaptive(dev)}), flush=True)
        return
    if args.profile_step:
        # the headline step with a chosen number of views, tile 32 x 32, for profiler captures:
        # --warmup steps, then --steps steps inside an NVTX range named "step"
        import torch

        from paper_2405_20693_b300 import engine, r2g

        one = args.profile_workload == "one_scan"
        if one:  # the one-scan step: 50k Gaussians, one view and one patch per step, 32 x 32 tiles
            G, cam, views_np, meas_np = make_workload(seed, dev)
            sc = engine.Scan(G, views_np, meas_np, cam, n_out=N_OUT, D=D_TV, device=dev)
        else:
            G, cam, views_np, meas_np = make_scale_workload(seed, dev)
            keep = np.linspace(0, SCALE_V - 1, args.scale_views).round().astype(int)
            views_np, meas_np = views_np[keep], meas_np[keep]
            sc = engine.Scan(G, views_np, meas_np, cam, n_out=N_OUT, D=D_TV, device=dev, headroom=1.25,
                             all_views=True, n_patches=SCALE_NP, full_volume=True, tile=(32, 32))
        n = args.warmup + args.steps
        origins = torch.as_tensor(scale_patch_origins(seed, n), device=dev)
        tab = torch.zeros((n, 8), dtype=torch.int32, device=dev)
        tab[:, 1] = torch.arange(n, dtype=torch.int32, device=dev)
        if one:  # the one-scan step sequence: view and patch origin per step
            seq = step_sequence(seed, n)
            tnp = np.zeros((n, 8), np.int32)
            for k, (v, off) in enumerate(seq):
                tnp[k, 0], tnp[k, 1] = v, k
                tnp[k, 2:5] = np.asarray([-1.0 + o * (2.0 / N_OUT) for o in off], np.float32).view(np.int32)
            tab = torch.as_tensor(tnp, device=dev)
        stream = torch.cuda.current_stream()
        for k in range(n):
            if k == args.warmup:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("step")
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            if not one:
                sc.job.patch_origins = origins.data_ptr() + k * 12 * SCALE_NP
            r2g.r2g_train_step(sc.job, tab.data_ptr() + 32 * k, stream)
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        # gated pixel pairs of the last step's view set (a counting run after the range)
        mean, scale, quat, rho = sc.state.params()
        vsel = sc.views[seq[n - 1][0]:seq[n - 1][0] + 1] if one else sc.views
        sc.rast.forward(mean, scale, quat, rho, vsel, sc.image, check=True, count=True)
        if rank == 0:
            print(json.dumps({"profile_step": {"workload": args.profile_workload,
                                               "views": 1 if one else int(args.scale_views),
                                               "ms_per_step": e0.elapsed_time(e1) / args.steps,
                                               "pixel_pairs": int(sc.rast.pair_count()),
                                               "overflow": bool(sc.overflowed())}}), flush=True)
        return
    if args.serving_full:
        if rank == 0:
            out = measure_serving(dev, n_requests=64, mean_interarrival_s=2.0, max_iters=30000, check_every=500)
            out["note"] = ("64 requests with the uneven size mix, each to 35 dB (checked every 500 iterations) or "
                           "30,000 iterations; arrivals compressed 15x (mean 2 s instead of 30 s); each request's "
                           "service is seconds, so at the uncompressed 2/min rate the requests would meet no queue "
                           "and time-to-volume would be the service time alone")
            print(json.dumps({"serving_config5": out}), flush=True)
        return
    if args.fdk_only:
        if rank == 0:
            G, cam, views_np, meas_np = make_workload(seed, dev)
            print(json.dumps({"fdk_init": measure_fdk_init(dev, views_np, meas_np, cam, reps=args.steps,
                                                           cpu=not args.no_cpu_baseline)}), flush=True)
        return
    head = measure_scale(args, dev, dist, seed, world)
    sc = head.pop("_sc")
    Gs, views_s, cam_s = head.pop("_G"), head.pop("_views"), head.pop("_cam")
    del sc
    torch.cuda.empty_cache()
    one = None
    if not args.no_one_scan:
        one = measure_one_scan(args, dev, dist, seed)
    if rank == 0:
        extras = {}
        if world == 1 and not args.no_batched:
            G2, cam2, views2, meas2 = one["_G"], one["_cam"], one["_views"], one["_meas"]
            extras = {"batched": measure_batched(dev), "serving": measure_serving(dev),
                      "fdk_init": measure_fdk_init(dev, views2, meas2, cam2, cpu=not args.no_cpu_baseline),
                      "volume_metrics": measure_metrics(dev), "limited_angle": measure_limited_angle(dev),
                      "adaptive_control": measure_adaptive(dev)}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_scale(Gs, views_s, cam_s)
            if one is not None:
                p, s_, _ = oracle_steps(one["_G"], one["_cam"], one["_views"], one["_meas"], one["_seq"], 2)
                one["cpu_baseline"] = {"value": p / s_, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                                       "sample": "2 full training steps of the one-scan workload (FP64 oracle, "
                                                 "single thread)"}
        if one is not None:
            for k in ("_G", "_cam", "_views", "_meas", "_seq"):
                one.pop(k, None)
        line = {
            "metric": METRIC, "value": head["value"], "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": head["config"],
            "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "roofline": head["roofline"],
            "splat_rooflines": head["splat_rooflines"], "kernels_ms_per_step": head["kernels_ms_per_step"],
            "pairs_per_step": head["pairs_per_step"],
            "step_call": "r2g_train_step, batch form (one C call per step; all views, 8 patch origins and the "
                         "full volume from the job, iteration from a device table)",
            "recompute_lists": head["recompute_lists"],
            "cpu_baseline": cpu, "one_scan": one, **extras, "clocks": head["clocks"],
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-one-scan", action="store_true", help="skip the one-scan (50k Gaussians, 1 view) leg")
    ap.add_argument("--no-recompute", action="store_true", help="skip the view-chunked (recomputed lists) timing")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the multi-scan scans/hour, serving and FDK-initialisation measurements")
    ap.add_argument("--fdk-only", action="store_true",
                    help="time only the FDK initialisation of the workload's scan (--steps runs)")
    ap.add_argument("--profile-step", action="store_true",
                    help="run only the headline step (--scale-views views, tile 32x32) for profiler captures")
    ap.add_argument("--scale-views", type=int, default=SCALE_V, help="views of the --profile-step workload")
    ap.add_argument("--profile-workload", choices=["scale", "one_scan"], default="scale",
                    help="the --profile-step workload: the headline step or the one-scan step")
    ap.add_argument("--serving-full", action="store_true",
                    help="run only the 64-request serving stream to 35 dB or 30k iterations (minutes)")
    ap.add_argument("--extras-only", action="store_true",
                    help="run only the volume-metrics, limited-angle and adaptive-control legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
