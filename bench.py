#!/usr/bin/env python
"""Benchmark of the R^2-Gaussian hot path on B300: fwd+bwd Gaussian-pixel evals/s.

One step = one training iteration of the one-scan cone-beam workload (50,000
Gaussians initialised from a seeded 40-ellipsoid 256^3 phantom; source-to-origin
1000 mm, source-to-detector 1500 mm, 50 views over 360 deg, 512^2 detector at
0.8 mm): rasterize one view, L1 + 0.25 D-SSIM, voxelize a random 32^3 TV patch
with weight 0.05, full backward through both, fused Adam -- all in libr2g.so.
The metric counts the (pixel, Gaussian) and (voxel, Gaussian) pairs that pass
the gates in that step, once, over the device time of the whole step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (one scan per rank, no data
exchange: the path has nothing to reduce across scans); value = all ranks'
pairs / the slowest rank's time.  --impl reference times the FP64 CPU oracle on
the same workload (a bounded number of full steps) on the host cores.
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
SM_COUNT = 148
MUFU_PER_CLK = 16          # ex2 per SM per clock
FP32_PER_CLK = 128         # FP32 lanes per SM per clock
OPS_FWD, OPS_BWD = 6, 14   # algorithmic FP32 ops per gated pair (forward, backward)


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
    """nvidia-smi samples every 100 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.idx = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
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
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


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


def run_reference(args, rank, world):
    if rank != 0:
        return
    G, cam, views, meas = make_workload(0, None if not _has_cuda() else "cuda")
    seq = step_sequence(0, args.warmup + args.steps)
    # each oracle step is a full training step (~5 s single-threaded); the run is
    # bounded by time: one warm-up step, then timed steps until K or 120 s
    oracle_steps(G, cam, views, meas, seq, 1)
    pairs, secs, done = oracle_steps(G, cam, views, meas, seq[args.warmup:], args.steps, budget_s=120.0)
    value = pairs / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": done, "warmup": 1, "ms_per_step": 1e3 * secs / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "one cone-beam scan, 50k Gaussians, 512^2 x 50 views, 1 view + 32^3 TV patch "
                                   "per step", "oracle": "FP64 C++ scatter form + numpy losses, single thread"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} full training steps of the same workload (time-bounded at 120 s "
                                       f"of the {args.steps} asked)"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


def _current(t, kernel: str) -> bool:
    return bool(t) and kernel in KERNEL_SOURCES and t.get("source_hashes", {}).get(kernel) == source_hash(kernel)


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the kernel's current sources; else None."""
    t = _ncu_summary()
    return t["kernels"].get(kernel) if _current(t, kernel) else None


def ncu_pipes(kernel: str):
    """FMA and XU (MUFU) pipe utilisation (% of peak sustained) of the kernel from the
    committed ncu summary, if it was taken on the kernel's current sources; else None."""
    t = _ncu_summary()
    return t.get("pipes", {}).get(kernel) if _current(t, kernel) else None


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


def measure_serving(dev, n_requests=16, mean_interarrival_s=0.25, max_iters=500, check_every=250):
    """p50/p99 time-to-volume and scans/hour of the continuous-batching server on a
    seeded Poisson stream of requests with the uneven multi-scan size mix.  Scanner
    data is prepared before the clock starts (a server receives projections, it
    does not synthesise them).  Arrivals are compressed in time and iterations
    capped (max_iters, PSNR target 35 dB checked every check_every) so the run takes
    seconds; both are stated in the output."""
    from paper_2405_20693_b300 import inputs as I
    from paper_2405_20693_b300 import serve

    specs = I.batched_specs(n_requests, seed=5)
    reqs = serve.poisson_requests(n_requests, mean_interarrival_s, seed=6, specs=specs, max_iters=max_iters,
                                  psnr_target=35.0, check_every=check_every)
    for r in reqs:
        r.data = I.make_scan(r.spec, device=dev)
    import torch

    budget = int(0.5 * torch.cuda.get_device_properties(dev).total_memory)
    srv = serve.Server(budget, D=D_TV, device=dev)
    res = srv.run(reqs)
    out = serve.summarize(res, srv.wall)
    out.update({"arrivals": f"Poisson, mean inter-arrival {mean_interarrival_s} s (seed 6), compressed from the "
                            "2/min stream", "iterations_cap": max_iters, "psnr_target_db": 35.0,
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
    return {"ms_per_call": ms, "volume": f"{N_OUT}^3", "values_noisy_phantom": vals,
            "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": algo / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                         "note": "algorithmic bytes = both volumes read once (128 MB); the kernel reads them "
                                 "once per orientation plus once for the MSE, with 5-voxel halos"}}


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


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2405_20693_b300 import build, engine, r2g

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    seed = rank * 1000
    G, cam, views_np, meas_np = make_workload(seed, dev)
    if args.extras_only:
        if rank == 0:
            print(json.dumps({"volume_metrics": measure_metrics(dev), "limited_angle": measure_limited_angle(dev),
                              "adaptive_control": measure_adaptive(dev)}), flush=True)
        return
    if args.fdk_only:
        if rank == 0:
            print(json.dumps({"fdk_init": measure_fdk_init(dev, views_np, meas_np, cam, reps=args.steps,
                                                           cpu=not args.no_cpu_baseline)}), flush=True)
        return
    # the scan's parameters, Adam state, views, measured projections, step buffers and
    # workspaces stay resident; one step = one r2g_train_step call reading its view,
    # iteration and TV patch origin from a device table holding every step's entry
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

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    assert not sc.overflowed(), "list capacity overflow in the warm-up"

    # per-kernel breakdown, untimed: event pairs around every kernel group of n_brk
    # steps; it names the dominant kernel, the only one bracketed in the timed region
    r2g.r2g_profile_enable(True, 64 * n_brk + 64)
    r2g.r2g_profile_select(0xFFFFFFFF)
    r2g.r2g_profile_reset()
    for k in range(args.warmup, args.warmup + n_brk):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    breakdown = {}
    for kid, name in enumerate(r2g.PROFILE_KERNELS):
        n, t = r2g.r2g_profile_read(kid)
        if n:
            breakdown[name] = t / n_brk
    dom = max(breakdown, key=breakdown.get)
    t0_steps = args.warmup + n_brk

    # algorithmic pairs of every distinct (view, patch) of the timed steps (counting
    # runs, untimed, on the parameters at the start of the timed region)
    from paper_2405_20693_b300 import inputs as I

    mean, scale, quat, rho = sc.state.params()
    # the superset the kernels walk: each Gaussian's pixel box (the projection's
    # stated FP32 bounds) and voxel box inside the patch
    proj = torch.empty((1, sc.M, 8), dtype=torch.float32, device=dev)
    prect = torch.empty((1, sc.M, 4), dtype=torch.int32, device=dev)
    vox_box = voxel_box_counter(sc)
    counted = {}
    for k in range(t0_steps, t0_steps + args.steps):
        v, off = seq[k]
        if (v, off) in counted:
            continue
        sc.rast.forward(mean, scale, quat, rho, sc.views[v:v + 1], sc.image, check=True, count=True)
        pp = sc.rast.pair_count()
        sc.vox.set_grids(I.patch_grid(off, D_TV, N_OUT))
        sc.vox.forward(mean, scale, quat, rho, sc.vol, check=True, count=True)
        r2g.r2g_project(mean, scale, quat, rho, sc.views[v:v + 1], sc.rast.cam, sc.rast.opts, proj, prect)
        rc = prect[0].long()
        ok = proj[0, :, 7] == 1.0
        box_p = int(((rc[:, 1] - rc[:, 0] + 1) * (rc[:, 3] - rc[:, 2] + 1))[ok].sum())
        counted[(v, off)] = (pp, sc.vox.pair_count(), box_p, vox_box(off))
    sc.job = sc._make_job()  # a checked run that had to regrow a workspace moved it
    pix_pairs = [counted[seq[k]][0] for k in range(t0_steps, t0_steps + args.steps)]
    vox_pairs = [counted[seq[k]][1] for k in range(t0_steps, t0_steps + args.steps)]
    box_pairs = [counted[seq[k]][2] + counted[seq[k]][3] for k in range(t0_steps, t0_steps + args.steps)]
    total_pairs = float(sum(pix_pairs) + sum(vox_pairs))
    # the state at the start of the timed region: the end-to-end leg restarts from it,
    # so that both legs run the same steps on the same parameters (the same pairs)
    st = sc.state
    start_state = [t.clone() for t in (st.raw, st.act, st.m, st.v)]

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    r2g.r2g_profile_enable(True, 2 * args.steps + 64)
    r2g.r2g_profile_select(1 << r2g.PROFILE_KERNELS.index(dom))
    r2g.r2g_profile_reset()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    clock = ClockSampler(gpu_id)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clock.start()
    launches0 = r2g.r2g_launch_count()
    for j in range(args.steps):
        flush.zero_()
        evs[j][0].record(stream)
        step(t0_steps + j)
        evs[j][1].record(stream)
    torch.cuda.synchronize()
    launches = r2g.r2g_launch_count() - launches0
    clocks = clock.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    assert not sc.overflowed(), "list capacity overflow inside the timed region"
    n_dom, t_dom = r2g.r2g_profile_read(r2g.PROFILE_KERNELS.index(dom))
    r2g.r2g_profile_enable(False)
    r2g.r2g_profile_select(0xFFFFFFFF)

    ms_job, pairs_job = job_totals(dist, ms, total_pairs, dev)
    value = pairs_job / (ms_job * 1e-3)

    # end to end through the public API (engine.HostFeed over r2g_train_step_host):
    # every step's inputs -- its measured view (H x W floats), the view's geometry
    # row and its round entry -- go host -> device from pinned memory into one of NS
    # staging slots on a copy stream, the fused step runs once its slot has arrived,
    # and its losses come back to pinned host memory; copies overlap the steps
    # before them, and the host reads step k's losses after queueing step k + NS - 1
    NS = 3
    meas_host = torch.from_numpy(np.ascontiguousarray(meas_np, np.float32)).pin_memory()
    views_host = torch.from_numpy(np.ascontiguousarray(views_np, np.float32)).pin_memory()
    ent_host = torch.from_numpy(tab.copy()).pin_memory()
    ent0 = ent_host.data_ptr()
    feed = engine.HostFeed(sc, meas_host, views_host, n_slots=NS, stream=stream)
    for j in range(NS):                            # creates the copy stream and events
        feed.step(seq[j][0], ent0 + 32 * j)
    feed.finish()
    for t, saved in zip((st.raw, st.act, st.m, st.v), start_state):
        t.copy_(saved)
    loss_sum, n_read = 0.0, 0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
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
    assert n_read == args.steps
    e2e_s = time.perf_counter() - t0
    assert np.isfinite(loss_sum)
    e2e_s = slowest(dist, e2e_s, dev)
    e2e_value = pairs_job / e2e_s

    if rank == 0:
        pk = peaks()
        f = pk["sm_max_mhz"] * 1e6
        mufu_peak = SM_COUNT * MUFU_PER_CLK * f
        fp32_peak = SM_COUNT * FP32_PER_CLK * f
        per_step_pix = sum(pix_pairs) / args.steps
        per_step_vox = sum(vox_pairs) / args.steps
        # roofline of the kernel with the largest device time (timed live, alone)
        roof = None
        if dom in ("splat_fwd", "splat_bwd", "vox_fwd", "vox_bwd"):
            units = per_step_pix if dom.startswith("splat") else per_step_vox
            ops = OPS_FWD if dom.endswith("fwd") else OPS_BWD
            peak = min(mufu_peak, fp32_peak / ops) / 1e9
            avg_s = t_dom / n_dom * 1e-3
            ach = units / avg_s / 1e9
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpair/s",
                    "frac": ach / peak, "traffic": ncu_traffic(dom), "pipes_pct_of_peak": ncu_pipes(dom),
                    "peak_note": f"min(MUFU ex2 {MUFU_PER_CLK}/clk/SM, FP32 {FP32_PER_CLK}/clk/SM / {ops} ops) "
                                 f"x {SM_COUNT} SMs x {pk['sm_max_mhz']:.0f} MHz"}
        elif dom is not None:
            roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": None, "traffic": ncu_traffic(dom)}
        batched = None
        serving = None
        fdk_init = metrics = limited = adaptive = None
        if world == 1 and not args.no_batched:
            batched = measure_batched(dev)
            serving = measure_serving(dev)
            fdk_init = measure_fdk_init(dev, views_np, meas_np, cam, cpu=not args.no_cpu_baseline)
            metrics = measure_metrics(dev)
            limited = measure_limited_angle(dev)
            adaptive = measure_adaptive(dev)
        cpu = None
        # CPU baseline: the oracle on two full steps of the same workload
        if world == 1 and not args.no_cpu_baseline:
            p, s, _ = oracle_steps(G, cam, views_np, meas_np, seq[t0_steps:], 2)
            cpu = {"value": p / s, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                   "sample": "2 full training steps of the same workload (FP64 oracle, single thread, "
                             "initial parameters)"}
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_job / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "one cone-beam scan: 50k Gaussians from a seeded 40-ellipsoid 256^3 phantom, "
                                   "L_SO 1000 mm, L_SD 1500 mm, 50 views x 512^2 at 0.8 mm; per step 1 view "
                                   "(L1+0.25 D-SSIM) + one 32^3 TV patch (0.05), full backward, Adam",
                       "pixel_pairs_per_step": per_step_pix, "voxel_pairs_per_step": per_step_vox,
                       "box_pairs_per_step": sum(box_pairs) / args.steps,
                       "gated_over_box": total_pairs / max(1.0, float(sum(box_pairs))),
                       "step_cycle": f"{N_DISTINCT} seeded (view, patch) pairs, repeated",
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{world}",
                       "tile": "32x32", "bricks": "8^3"},
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": 4 * cam.H * cam.W + 48 + 32,
                    "d2h_bytes_per_step": 8,
                    "note": "per step, one r2g_train_step_host call (engine.HostFeed): the measured view, its "
                            "geometry row and its round entry copied from pinned host memory into one of three "
                            "device slots on a copy stream (overlapping the steps before it), the fused step, the "
                            "two losses read back to pinned host memory and read by the host; the same steps as the "
                            "device-timed leg, from the same starting state"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "kernels_ms_per_step": breakdown,
            "kernels_note": f"breakdown: event pairs around every kernel group over {n_brk} untimed steps; "
                            f"timed region: events around {dom} only",
            "step_call": "r2g_train_step (one C call per step; entries from a device table)",
            "cpu_baseline": cpu,
            "batched": batched,
            "serving": serving,
            "fdk_init": fdk_init,
            "volume_metrics": metrics,
            "limited_angle": limited,
            "adaptive_control": adaptive,
            "clocks": clocks,
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
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the multi-scan scans/hour, serving and FDK-initialisation measurements")
    ap.add_argument("--fdk-only", action="store_true",
                    help="time only the FDK initialisation of the workload's scan (--steps runs)")
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
