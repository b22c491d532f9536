#!/usr/bin/env python
"""Benchmark of the 4D GSUBSURF segmentation hot path on GB300.

One bench step = one whole segmentation of the large synthetic workload
(512x512x128 space x 48 frames = 1.61G voxels, one nucleus per 40^3 voxels,
20 semi-implicit steps), with the image already resident in HBM: set-up
(thresholding, two presmoothing solves, face coefficients, u0) and
20 x {coefficients, red-black SOR solve to the stopping rule, rescale}, all
through the C ABI.

metric: voxel-sweeps/s = voxels x red-black sweeps (every solve, set-up
included) / wall time of the whole segmentation.  The roofline object is for
the dominant kernel (the red-black half sweep): algorithmic bytes per launch /
its CUDA-event time on the launching stream, against the measured HBM peak.

Further legs: the medium workload (128x128x64 x 32 frames, 50 steps) in FP32
and in mixed precision, a grid of the paper's largest stack on a lean handle,
the batched per-nucleus windows, and serving.

--impl reference times the FP64 CPU oracle (the reference of this project) on
a bounded crop of the same workload.  Multi-GPU (torchrun): independent
replicas, one per GPU (the full-grid path does not shard: replicas only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per voxel-sweep of the sweep as launched: the FP32 solve
# sweeps its correction system in symmetrically scaled form, reading the
# correction (r + w 8), its right-hand side (4) and four FP32 face weights
# per voxel (16); the lean handle's unscaled sweep also reads gamma = c/D (4).
ALG_BYTES_SCALED = 28.0
ALG_BYTES_UNSCALED = 32.0
FALLBACK_HBM_GBS = 6800.0
SWEEP_KERNEL = "k_sweep_vec (one colour of a red-black sweep per launch, 2 voxels/thread)"
# DRAM traffic of the sweep comes from a committed ncu summary: its
# "bench-record:" line gives the bytes per voxel update and the hash of the
# kernel sources at capture time; a record whose hash differs from the
# current sources is stale and gives no traffic figure.
SWEEP_SOURCES = ["solve_kernels.cu", "stencil.cuh", "seg4d_internal.cuh"]


def sweep_src_sha():
    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2111_11866_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def sweep_traffic_record(profile):
    """(bytes per voxel update, record) from profiles/<profile>, or (None,
    reason) when the record is missing or was taken on other sources."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        with open(path) as fh:
            text = fh.read()
    except OSError:
        return None, f"no {profile}"
    m = re.search(r"bench-record: kernel=(\S+) src_sha=(\S+) bytes_per_voxel_update=([0-9.]+)",
                  text)
    if not m:
        return None, f"no bench-record line in {profile}"
    if m.group(2) != sweep_src_sha():
        return None, f"{profile}: captured on other kernel sources (src_sha {m.group(2)})"
    return float(m.group(3)), f"{profile} ({m.group(1)}, src_sha {m.group(2)})"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (timed regions end with the slowest rank);
    x itself when the job runs on one process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: all ranks' units over the
    slowest rank's time."""
    return world * units_per_rank / seconds


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


CROP = (64, 64, 32, 8)   # (n1, n2, n3, n4) of the CPU baselines' sample


def _crop_box(seeds, dims, n=CROP):
    """Origin of an n-sized box around the seed nearest the grid centre."""
    import numpy as np
    c = np.array(dims[:3], float) / 2
    s = seeds[np.argmin(((seeds[:, :3] - c) ** 2).sum(1))]
    return [int(min(max(0, round(s[d]) - n[d] // 2), dims[d] - n[d])) for d in range(3)]


def _crop_seeds(seeds, org, n=CROP):
    import numpy as np
    sh = seeds.copy()
    sh[:, :3] -= np.array(org, float)
    keep = ((sh[:, 0] >= 0) & (sh[:, 0] < n[0]) & (sh[:, 1] >= 0) & (sh[:, 1] < n[1]) &
            (sh[:, 2] >= 0) & (sh[:, 2] < n[2]) & (sh[:, 3] < n[3]))
    return sh[keep]


def large_crop(img=None, frames=48, depth=128, n=CROP):
    """The CPU baselines' sample of the large workload: an n-sized crop (first
    n4 frames) around the nucleus nearest the grid centre.  From the device
    image when given, else the first n4 frames generated on the host by the
    same seeded generator.  Returns (image (n4, n3, n2, n1) numpy, seeds,
    description)."""
    import numpy as np
    from paper_2111_11866_gb300 import synth
    dims = (512, 512, depth, frames)
    n = tuple(min(a, b) for a, b in zip(n, dims))
    seeds, count, gen = synth.nuclei_frames(3, dims, 1.0 / 40 ** 3, "cpu" if img is None else
                                            img.device)
    x0, y0, z0 = _crop_box(seeds, dims, n)
    n1, n2, n3, n4 = n
    if img is not None:
        crop = img[:n4, z0:z0 + n3, y0:y0 + n2, x0:x0 + n1].cpu().numpy().copy()
    else:
        crop = np.empty((n4, n3, n2, n1), np.float32)
        for l, f in enumerate(gen):
            crop[l] = f[z0:z0 + n3, y0:y0 + n2, x0:x0 + n1].numpy()
            if l + 1 == n4:
                break
    desc = (f"{n1}x{n2}x{n3}x{n4} crop at ({x0},{y0},{z0},0) of the large "
            f"512x512x{depth}x{frames} grid")
    return crop, _crop_seeds(seeds, (x0, y0, z0), n), desc


def _host_cpu():
    """nproc, architecture and CPU model of the host the CPU baselines ran on."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "processor name") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def oracle_sample(img, seeds, where, params, nsteps=2, omp=False):
    """The FP64 oracle, as it stands, on a crop of the workload: returns
    (voxel-sweeps per second, description, seconds, threads).  omp: its OpenMP
    build (the paper's frame-split red-black sweeps on all host cores)."""
    import numpy as np
    import oracle as O
    P = O.OracleParams(h=tuple(params.h), tau=params.tau, eps=params.eps, K=params.K,
                       delta=params.delta, vartheta=params.vartheta, lambda_th=params.lambda_th,
                       r_ball=params.r_ball, R_init=params.R_init, v_init=params.v_init,
                       sigma_t=params.sigma_t, tol=1e-12)
    t0 = time.perf_counter()
    u, info = O.segment(img.astype(np.float64), seeds, P, nsteps=nsteps, omp=omp)
    dt = time.perf_counter() - t0
    sweeps = sum(info["iters"])
    how = (f"OpenMP build, {O.threads(True)} threads, frame-split red-black sweeps" if omp
           else "1 thread")
    desc = (f"oracle (plain C, FP64, {how}) full pipeline on a {where} ({len(seeds)} seeds), "
            f"{nsteps} step(s) solved to 1e-12; counts step-solve sweeps, times set-up too")
    return img.size * sweeps / dt, desc, dt, (O.threads(True) if omp else 1)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample (a crop, one time step) of the large workload."""
    if rank != 0:
        return
    from paper_2111_11866_gb300._lib import Params
    import oracle
    oracle.build()
    img, seeds, where = large_crop()
    params = Params()
    for _ in range(args.warmup):
        oracle_sample(img, seeds, where, params)
    vals, times = [], []
    desc = ""
    for _ in range(args.steps):
        v, desc, dt, _ = oracle_sample(img, seeds, where, params)
        vals.append(v)
        times.append(dt)
    value = statistics.mean(vals)
    cfg = _config_large()
    cfg["sample"] = f"each step: {where}, 2 time steps (the full workload takes the oracle days)"
    line = {"impl": "reference", "metric": "voxel-sweeps/s", "value": value,
            "unit": "voxel-sweeps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "voxel-sweeps/s", "cores": 1,
                             "kind": "oracle", "sample": desc, "host": _host_cpu()},
            "e2e": {"value": value, "unit": "voxel-sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config_large(frames=48, nsteps=20, depth=128):
    return {"workload": f"large full grid 512x512x{depth}x{frames}, 1 nucleus per 40^3 voxels, "
                        f"{nsteps} steps", "n1": 512, "n2": 512, "n3": depth, "n4": frames,
            "voxels": 512 * 512 * depth * frames, "time_steps": nsteps,
            "parallelism": "replicas",
            "l2": "inputs larger than L2 (about 200 GB resident)"}


def _plain_window(img_d, seeds, nsteps, params):
    """The plain per-instance FP32 path: one handle per window."""
    from paper_2111_11866_gb300 import _lib
    n4, n3, n2, n1 = img_d.shape
    import torch
    out = torch.empty_like(img_d)
    with _lib.Seg4D((n1, n2, n3, n4), stream=torch.cuda.current_stream(), params=params) as s:
        s.set_image(img_d)
        s.set_seeds(seeds)
        s.step(nsteps)
        s.read_u(out)
    return out


def _mixed(params):
    import copy
    pm = copy.copy(params)
    pm.precision = 1
    return pm


def _roofline(nvox, sweeps, sweep_ms, sweep_launches, alg_bytes, kernel, traffic_rec=None):
    """Roofline of the sweep: algorithmic bytes of one launch (alg_bytes per
    voxel-sweep x the voxel-sweeps of a launch) / the launch's average
    CUDA-event time, against the measured HBM peak; traffic = DRAM bytes of
    one launch from the committed capture record, when it is current."""
    peak, peak_kind = _peaks()
    per_launch_sweeps = sweeps / max(sweep_launches, 1)
    per_launch_bytes = alg_bytes * nvox * per_launch_sweeps
    launch_ms = sweep_ms / max(sweep_launches, 1)
    achieved = per_launch_bytes / (launch_ms / 1000.0) / 1e9 if launch_ms > 0 else None
    out = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak if achieved else None, "traffic": None,
           "peak_kind": peak_kind, "alg_bytes_per_voxel_sweep": alg_bytes,
           "alg_bytes_per_launch": per_launch_bytes, "sweeps_per_launch": per_launch_sweeps,
           "avg_launch_ms": launch_ms}
    if traffic_rec is not None:
        b_upd, src = traffic_rec
        out["traffic_source"] = src
        if b_upd is not None:
            # a launch updates the voxels of one colour: per_launch_sweeps x nvox updates x 2
            out["traffic"] = b_upd * nvox * per_launch_sweeps * 2.0
            out["traffic_bytes_per_voxel_update"] = b_upd
    return out


def run_headline(args, params, local, dist, world):
    """The large workload (512x512x128 x 48 frames, 1.61G voxels, 20 steps),
    built on the device: W warm-up and K timed whole segmentations with the
    image resident in HBM, then the same through the ABI from pinned host
    memory with u read back (e2e), and the CPU baselines on a crop."""
    import numpy as np
    import torch
    from paper_2111_11866_gb300 import _lib, synth

    img_d, seeds, nsteps, meta = synth.large("cuda", frames=args.large_frames,
                                             depth=args.large_depth)
    if args.time_steps is not None:
        nsteps = args.time_steps
    dims = tuple(reversed(img_d.shape))
    nvox = img_d.numel()
    crop = large_crop(img_d, frames=args.large_frames, depth=args.large_depth)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    seg = _lib.Seg4D(dims, stream=stream, params=params)

    def one_step(src):
        seg.set_image(src)
        seg.set_seeds(seeds)
        return seg.step(nsteps)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    try:
        for _ in range(max(args.warmup, 0)):
            one_step(img_d)
        sampler = ClockSampler(local)
        barrier()
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sweeps = launches = sweep_launches = 0
        sweep_ms = 0.0
        infos = []
        e0.record(stream)
        for _ in range(args.steps):
            info = one_step(img_d)
            infos.append(info)
            sweeps += info["sweeps_total"]
            sweep_ms += info["sweep_ms"]
            sweep_launches += info["sweep_launches"]
            launches += info["launches"] + 1      # + the image split kernel of set_image
        e1.record(stream)
        barrier()
        clocks = sampler.stop()
        elapsed_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        value = job_rate(world, nvox * sweeps, elapsed_ms / 1000.0)

        # end to end through the same ABI with host buffers: the image comes
        # from pinned host memory and u goes back to it, copies timed
        img_h = torch.empty(img_d.shape, dtype=torch.float32, pin_memory=True)
        img_h.copy_(img_d)
        out_h = torch.empty(img_d.shape, dtype=torch.float32, pin_memory=True)
        del img_d
        torch.cuda.empty_cache()
        barrier()
        t0 = time.perf_counter()
        e2e_sweeps = 0
        e2e_steps = 1
        for _ in range(e2e_steps):
            info = one_step(img_h)
            e2e_sweeps += info["sweeps_total"]
            seg.read_u(out_h)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": job_rate(world, nvox * e2e_sweeps, e2e_s), "unit": "voxel-sweeps/s",
               "h2d_bytes_per_step": img_h.nbytes, "d2h_bytes_per_step": out_h.nbytes,
               "steps": e2e_steps}
        last = infos[-1]
        res = {"value": value, "elapsed_ms": elapsed_ms, "nvox": nvox, "sweeps": sweeps,
               "launches": launches, "clocks": clocks, "e2e": e2e, "crop": crop,
               "config": _config_large(args.large_frames, nsteps, args.large_depth),
               "meta": meta,
               "sweep_rate": nvox * sweeps / (sweep_ms / 1000.0) if sweep_ms > 0 else None,
               "roofline": _roofline(nvox, sweeps, sweep_ms, sweep_launches, ALG_BYTES_SCALED,
                                     SWEEP_KERNEL,
                                     sweep_traffic_record("k_sweep_vec_large_planes.md")),
               "sweeps_per_segmentation": sweeps / args.steps,
               "ms_per_time_step": elapsed_ms / args.steps / nsteps,
               "last_solve": {"res_rel": last["res_rel"],
                              "res_inf_rel": last["res_inf"] / max(last["bmax"], 1e-300)},
               "device_gb": _lib.Seg4D.device_bytes(dims) / 1e9}
        return res
    finally:
        seg.close()
        torch.cuda.empty_cache()


def run_medium(args, params, local):
    """The medium workload (128x128x64 x 32 frames, 33.5M voxels, 50 steps):
    whole segmentations in FP32 and in mixed precision on one handle, the
    image resident in HBM, with the sweep's roofline and the mixed result's
    difference from the FP32 one."""
    import numpy as np
    import torch
    from paper_2111_11866_gb300 import _lib, synth

    case = synth.medium()
    nvox = int(np.prod(case.dims))
    stream = torch.cuda.current_stream()
    img_d = torch.from_numpy(case.image).cuda()
    out = {"workload": f"medium full grid 128x128x64x32, {case.meta['count']} nuclei, "
                       f"{case.nsteps} steps", "voxels": nvox}
    with _lib.Seg4D(case.dims, stream=stream, params=params) as seg:
        def run(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            sw = sl = 0
            sms = 0.0
            e0.record(stream)
            for _ in range(k):
                seg.set_image(img_d)
                seg.set_seeds(case.seeds)
                info = seg.step(case.nsteps)
                sw += info["sweeps_total"]
                sms += info["sweep_ms"]
                sl += info["sweep_launches"]
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), sw, sms, sl, info

        run(1)
        ms, sw, sms, sl, info = run(args.medium_steps)
        out.update({"value": nvox * sw / (ms / 1000.0), "unit": "voxel-sweeps/s",
                    "ms_per_segmentation": ms / args.medium_steps,
                    "sweeps_per_segmentation": sw / args.medium_steps,
                    "sweep_rate": nvox * sw / (sms / 1000.0),
                    "roofline": _roofline(nvox, sw, sms, sl, ALG_BYTES_SCALED,
                                          SWEEP_KERNEL,
                                          sweep_traffic_record("k_sweep_vec_medium.md"))})
        u_plain = seg.read_u()
        if args.mixed_steps > 0:
            seg.set_params(precision=1)
            run(1)
            ms, sw, sms, sl, info = run(args.mixed_steps)
            u_mixed = seg.read_u()
            seg.set_params(precision=0)
            out["mixed_precision"] = {
                "value": nvox * sw / (ms / 1000.0), "unit": "voxel-sweeps/s",
                "ms_per_segmentation": ms / args.mixed_steps,
                "sweeps_per_segmentation": sw / args.mixed_steps,
                "sweep_rate": nvox * sw / (sms / 1000.0),
                "max_rel_diff_vs_f32": float(np.abs(u_mixed - u_plain).max() /
                                             max(np.abs(u_plain).max(), 1e-30)),
                "dtype": "bf16 sweep weights, f32 sweeps and defect passes, f64 norms"}
    del img_d
    torch.cuda.empty_cache()
    return out


def run_paper_scale(nsteps, params, local, mixed_steps=0):
    """A grid of the size of the paper's largest stack (567x577x147 x 70
    frames, 3.37G voxels; the paper ran it on six nodes with 1012 GB) on one
    GPU with a lean handle (80 B/voxel): synthetic nuclei made frame by frame
    on the device into a host buffer, set-up, then `nsteps` time steps."""
    import numpy as np
    import torch
    from paper_2111_11866_gb300 import _lib, synth

    dims, seeds, count, frames = synth.paper_scale("cuda")
    n1, n2, n3, n4 = dims
    stream = torch.cuda.current_stream()
    seg = _lib.Seg4D(dims, stream=stream, params=params, lean=True)
    try:
        host = np.empty((n4, n3, n2, n1), np.float32)
        t0 = time.perf_counter()
        for l, f in enumerate(frames):
            host[l] = f.cpu().numpy()
        t_gen = time.perf_counter() - t0
        torch.cuda.empty_cache()
        seg.set_image(host)
        del host
        seg.set_seeds(seeds)
        t0 = time.perf_counter()
        info0 = seg.setup()
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = seg.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        nvox = n1 * n2 * n3 * n4
        sweeps = info["sweeps_total"]
        peak, peak_kind = _peaks()
        rate = nvox * sweeps / (info["sweep_ms"] / 1000.0)
        # the same handle continues in mixed precision (BF16 sweep weights,
        # FP32 defect passes): the weights fit beside the lean grid
        mixed = None
        if mixed_steps > 0:
            seg.set_params(precision=1)
            e0.record(stream)
            infm = seg.step(mixed_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            msm = e0.elapsed_time(e1)
            mixed = {"steps": mixed_steps, "value": nvox * infm["sweeps_total"] / (msm / 1000.0),
                     "unit": "voxel-sweeps/s", "ms_per_time_step": msm / mixed_steps,
                     "sweeps_per_time_step": infm["sweeps_total"] / mixed_steps,
                     "sweep_rate": nvox * infm["sweeps_total"] / (infm["sweep_ms"] / 1000.0),
                     "last_res_rel": infm["res_rel"],
                     "device_used_gb": (lambda fr: (fr[1] - fr[0]) / 1e9)(
                         torch.cuda.mem_get_info())}
        return {"workload": f"567x577x147x70 ({nvox} voxels, {count} nuclei), {nsteps} steps, "
                            f"lean handle", "voxels": nvox, "mixed_precision": mixed,
                "device_gb": _lib.Seg4D.device_bytes(dims, lean=True) / 1e9,
                "value": nvox * sweeps / (ms / 1000.0), "unit": "voxel-sweeps/s",
                "ms_per_time_step": ms / nsteps, "sweeps_per_time_step": sweeps / nsteps,
                "sweep_rate": rate,
                "roofline_frac": ALG_BYTES_UNSCALED * rate / 1e9 / peak,
                "alg_bytes_per_voxel_sweep": ALG_BYTES_UNSCALED,
                "peak_kind": peak_kind, "last_res_rel": info["res_rel"],
                "u_range": [info["umin"], info["umax"]], "setup_s": t_setup,
                "setup_sweeps": info0["sweeps_total"], "generate_s": t_gen, "clocks": clocks,
                "data": "synthetic, generated on the device frame by frame (seeded)"}
    finally:
        seg.close()
        torch.cuda.empty_cache()


def run_batched(nwin, nsteps, params, plain_sample=48):
    """Per-nucleus windows (edge U[24,64], 8-16 frames) advanced by the batch
    engine in mixed precision (BF16 sweep weights, FP32 defect passes) with
    continuous admission under a device budget, against the plain per-window
    FP32 path on a sample of the same windows, at the same tolerance."""
    import numpy as np
    import torch
    from paper_2111_11866_gb300 import _lib, serve, synth
    pm = _mixed(params)
    ws = synth.windows(nwin, nsteps=nsteps)
    dev = [torch.from_numpy(w[0]).cuda() for w in ws]
    need = sum(_lib.Batch.window_bytes((w[0].shape[3], w[0].shape[2], w[0].shape[1],
                                        w[0].shape[0]), 1, 1) for w in ws)
    budget = int(min(need * 1.05 + (64 << 20), 200e9))
    reqs = [serve.Request(k, 0.0, dev[k], ws[k][1], nsteps) for k in range(nwin)]
    torch.cuda.synchronize()
    with serve.Server(budget, min(nwin, 8192), params=pm) as srv:
        t0 = time.perf_counter()
        st = srv.run(reqs, sync=None)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
    nplain = min(plain_sample, nwin)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_out = [_plain_window(dev[k], ws[k][1], nsteps, params) for k in range(nplain)]
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    # accuracy check on a few windows: batched result vs plain result
    maxdiff = 0.0
    with _lib.Batch(int(need / nwin * 8 + (64 << 20)), 8, params=pm) as b:
        for k in range(min(4, nplain)):
            wid = b.add(dev[k], ws[k][1], nsteps)
            for _ in range(nsteps):
                b.advance()
            u = b.read_u(wid)
            ref = plain_out[k].cpu().numpy()
            maxdiff = max(maxdiff, float(np.abs(u - ref).max() / max(np.abs(ref).max(), 1e-30)))
            b.remove(wid)
    vox = sum(w[0].size for w in ws)
    return {"workload": f"{nwin} per-nucleus windows, edge U[24,64], 8-16 frames, {nsteps} steps",
            "voxels": vox, "budget_gb": budget / 1e9, "seconds": tb,
            "seg_per_s": st.served / tb, "window_sweeps": st.window_sweeps, "launches": st.launches,
            "max_resident": st.max_resident, "failed": st.failed,
            "plain": {"windows": nplain, "seconds": tp, "seg_per_s": nplain / tp},
            "speedup_vs_plain": (st.served / tb) / (nplain / tp),
            "max_rel_diff_vs_plain": maxdiff,
            "dtype": "mixed: bf16 sweep weights, f32 sweeps and defect passes, f64 norms"}


def run_serving(rate, seconds, budget_gb, params, pool=24):
    """Open-loop Poisson requests (window edge log-uniform 16..96, frames =
    edge/4), continuous batching under a device budget; p50/p99 latency and
    seg/s at the offered rate, the closed-loop capacity (every pool request
    arriving at once), then p50/p99 at half that capacity.  The comparison is
    sequential plain FP32 solves of the same pool of requests, one at a time."""
    import torch
    from paper_2111_11866_gb300 import serve, synth
    sizes = synth.request_sizes(pool)
    imgs = []
    for k, (e, _, _, f) in enumerate(sizes):
        img, seeds, nsteps = synth.request_window(1000 + k, e, f, nsteps=30)
        imgs.append((torch.from_numpy(img).cuda(), seeds, nsteps))

    def requests(r, horizon, seed):
        t = serve.poisson_arrivals(r, max(1, int(r * horizon)), seed)
        return [serve.Request(k, float(t[k]), *imgs[k % pool]) for k in range(len(t))]

    budget = int(budget_gb * 1e9)
    out = {"workload": f"open-loop Poisson, window edge log-uniform 16..96 (frames edge/4), "
                       f"30 steps, {budget_gb:g} GB admission budget, pool of {pool} images; "
                       f"the offered rate saturates the GPU, so latency there is queueing: "
                       f"stats cover requests completed within the {seconds:g} s horizon"}
    _plain_window(*imgs[0], params)   # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(pool):
        _plain_window(*imgs[k], params)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    out["sequential_plain"] = {"requests": pool, "seg_per_s": pool / tp,
                               "mean_ms": 1e3 * tp / pool}
    pm = _mixed(params)
    with serve.Server(budget, 8192, params=pm) as srv:
        st = srv.run([serve.Request(k, 0.0, *imgs[k % pool]) for k in range(2 * pool)])
        cap = st.served / st.wall_s
        out["capacity"] = {"requests": 2 * pool, "seg_per_s": cap,
                           "speedup_vs_sequential_plain": cap * tp / pool}
    with serve.Server(budget, 8192, params=pm) as srv:
        st = srv.run(requests(rate, seconds, 11), horizon_s=seconds)
        s = st.summary()
        s["offered_rate"] = rate
        s["seg_per_s"] = st.served / seconds
        out["at_offered_rate"] = s
    with serve.Server(budget, 8192, params=pm) as srv:
        st = srv.run(requests(0.5 * cap, seconds, 12), horizon_s=seconds + 20.0)
        s = st.summary()
        s["offered_rate"] = 0.5 * cap
        out["at_half_capacity"] = s
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3,
                    help="timed whole segmentations of the large workload")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--large-frames", type=int, default=48,
                    help="frames of the large grid (fewer: the same planes, for profiling)")
    ap.add_argument("--large-depth", type=int, default=128,
                    help="z-planes of the large grid (fewer: the same rows, for profiling)")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="override the large workload's 20 time steps (profiling runs only)")
    ap.add_argument("--medium-steps", type=int, default=3,
                    help="timed segmentations of the medium workload (0 = skip)")
    ap.add_argument("--mixed-steps", type=int, default=3,
                    help="segmentations of the medium workload in mixed precision (0 = skip)")
    ap.add_argument("--paper-steps", type=int, default=5,
                    help="time steps of the 567x577x147x70 grid with a lean handle (0 = skip)")
    ap.add_argument("--paper-mixed-steps", type=int, default=3,
                    help="further time steps of that grid in mixed precision (0 = skip)")
    ap.add_argument("--batched-windows", type=int, default=4096,
                    help="per-nucleus windows of the batched measurement (0 = skip)")
    ap.add_argument("--batched-steps", type=int, default=30)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="offered requests/s")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="arrival horizon of the serving measurement (0 = skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_11866_gb300 import _lib

    params = _lib.Params.defaults()
    head = run_headline(args, params, local, dist, world)

    cpu = cpu_omp = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        img, seeds, where = head["crop"]
        v, desc, _, _ = oracle_sample(img, seeds, where, params)
        cpu = {"value": v, "unit": "voxel-sweeps/s", "cores": 1, "kind": "oracle", "sample": desc,
               "host": _host_cpu()}
        try:
            v, desc, _, cores = oracle_sample(img, seeds, where, params, omp=True)
            cpu_omp = {"value": v, "unit": "voxel-sweeps/s", "cores": cores,
                       "kind": "oracle, OpenMP build", "sample": desc}
        except Exception as e:   # noqa: BLE001 -- no OpenMP toolchain on the host
            cpu_omp = {"unavailable": f"OpenMP build of the oracle failed: {e}"[:200]}

    medium = paper = batched = serving = None
    if args.medium_steps > 0:
        medium = run_medium(args, params, local)
    if args.paper_steps > 0:
        paper = run_paper_scale(args.paper_steps, params, local, args.paper_mixed_steps)
    if args.batched_windows > 0:
        batched = run_batched(args.batched_windows, args.batched_steps, params)
    if args.serve_seconds > 0:
        serving = run_serving(args.serve_rate, args.serve_seconds, args.serve_budget_gb, params)

    if rank == 0:
        line = {
            "metric": "voxel-sweeps/s", "value": head["value"], "unit": "voxel-sweeps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["elapsed_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": head["config"],
            "sweeps_per_segmentation": head["sweeps_per_segmentation"],
            "ms_per_time_step": head["ms_per_time_step"],
            "sweep_rate": head["sweep_rate"],
            "roofline": head["roofline"],
            "last_solve": head["last_solve"],
            "device_gb": head["device_gb"],
            "cpu_baseline": cpu,
            "cpu_baseline_omp": cpu_omp,
            "e2e": head["e2e"],
            "gpu_launches": head["launches"],
            "clocks": head["clocks"],
            "medium": medium,
            "paper_scale": paper,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
