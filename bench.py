#!/usr/bin/env python3
"""Benchmark of the DVNR hot path (arXiv 2304.10516) on GB300.

Metric: INR training samples/s (and decode samples/s) at equal PSNR to the
plain FP32 path. One *step* is one training iteration of the whole hot path
over one batch: sampling, trilinear targets, hash-grid encoding, MLP forward,
L1 loss, backward, gradient scatter and Adam (plus, reported beside it,
decoding and ray-marching of the trained model).

Workload (default): the 256^3 spectral-field model -- hash grid L=16, F=2,
T=2^19, N_min=16, b=1.38, MLP 32->64->64->64->1, batch 2^18 samples/step.
Inputs are seeded synthetic fields resident in HBM before the timed region.
The per-step working set (tables, gradients, Adam moments, volume) is larger
than the 129 MB L2, so no explicit flush is needed between steps.

Under torchrun (N > 1) every rank trains its own partition model with no
exchange between ranks (the paper's model parallelism, Sec. 3.1): weak
scaling, timed with a barrier and the max over ranks.

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
tier) on the same workload, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_10516_gb300 import shard  # noqa: E402

WORKLOADS = {
    "spectral256": dict(desc="256^3 spectral k^-5/3 field, L=16 F=2 T=2^19 N0=16 b=1.38, "
                             "MLP 32-64-64-64-1, batch 2^18",
                        shape=(256, 256, 256), seed=1002, L=16, F=2, log2T=19, base=16, growth=1.38,
                        width=64, hidden=3, batch=1 << 18, steps_full=2000, lam=0.0, lr=1e-2),
    "blocks64": dict(desc="1024x1024x512 spectral field, 64 uneven blocks (4x4x4 over [0,512)^3, edges "
                          "96-160, 1 ghost layer), one INR each (L=16 F=2 T=2^17 N0=16 b=1.38, MLP "
                          "32-64-64-64-1), 2^14 samples/model/step, lambda 0.15",
                     shape=(512, 1024, 1024), seed=1004, L=16, F=2, log2T=17, base=16, growth=1.38,
                     width=64, hidden=3, batch=1 << 14, steps_full=2000, lam=0.15, lr=1e-2),
    "insitu512": dict(desc="16 advected 512^3 spectral steps through a window of 8 (warm start, "
                           "500 iterations each, older steps frozen to FP16), decode 512^3, ray-march "
                           "1024x1024x512 (L=16 F=2 T=2^19, MLP 32-64-64-64-1, batch 2^18, lambda 0.15)",
                      shape=(512, 512, 512), seed=1005, L=16, F=2, log2T=19, base=16, growth=1.38,
                      width=64, hidden=3, batch=1 << 18, steps_full=500, lam=0.15, lr=1e-2, t_steps=16,
                      window=8),
    "blobs64": dict(desc="64^3 Gaussian blobs, L=8 F=2 T=2^15 N0=4 b=1.5, MLP 16-32-32-1, batch 4096",
                    shape=(64, 64, 64), seed=1001, L=8, F=2, log2T=15, base=4, growth=1.5,
                    width=32, hidden=2, batch=4096, steps_full=200, lam=0.0, lr=1e-2),
}

LEGS = ("roofline", "decode", "render", "render_inr", "e2e", "gain", "cpu", "batched", "insitu")

SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="spectral256", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default="auto", choices=["auto", "fp16", "fp32"])
    p.add_argument("--no-extras", action="store_true",
                   help="skip the e2e, decode, render and CPU-baseline legs")
    p.add_argument("--legs", default="all",
                   help="comma list of the extra legs to run, from " + ",".join(LEGS)
                        + " (default all; e2e includes the FP32 path and PSNR, gain needs e2e); "
                          "blocks64 takes all or roofline")
    return p.parse_args()


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="dvnr_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------- algorithmic bytes/flops ---
def kernel_bytes(name, w, n_params, batch):
    """Algorithmic bytes of one launch of kernel `name`: the kernel's bytes
    per unit (a sample, a parameter) times the units one launch processes."""
    L, F, W, H = w["L"], w["F"], w["width"], w["hidden"]
    D = L * F
    if name == "adam":
        return 34 * n_params  # read g, theta, m, v; write theta, m, v, fp16 copy, zeroed g
    if name == "train_fused_fp16":
        # per sample: 8 fp32 volume reads, 8 fp16 corner reads and 8 fp32 corner
        # gradient read-modify-writes per feature and level
        return batch * (8 * 4 + L * 8 * F * 2 + L * 8 * F * 4)
    if name == "fp32_sample_encode":
        return batch * (8 * 4 + L * 8 * F * 4 + D * 4 + 12 + 4)
    if name == "fp32_scatter":
        return batch * (L * 8 * F * 4 + D * 4 + 12)
    return None


# ------------------------------------------------------------ our arm -------
def graph_stats(A):
    import ctypes as C

    c, r, e = C.c_int64(), C.c_int64(), C.c_int64()
    A.call("dvnr_graph_stats", C.byref(c), C.byref(r), C.byref(e))
    return c.value, r.value, e.value


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2304_10516_gb300 import _abi as A
    from paper_2304_10516_gb300 import model as dv
    from paper_2304_10516_gb300 import volumes

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS[args.workload]
    lib = A.load()
    prec = args.precision
    if prec == "auto":
        prec = "fp16"
    precision = A.DVNR_FP16 if prec == "fp16" else A.DVNR_FP32

    vol_np = volumes.spectral(w["shape"], seed=w["seed"] + rank) if args.workload == "spectral256" \
        else volumes.blobs(w["shape"][0], seed=w["seed"] + rank)
    vol = torch.from_numpy(vol_np).to(dev)
    nz, ny, nx = vol_np.shape
    enc = dv.EncodingConfig(w["L"], w["F"], w["log2T"], w["base"], w["growth"])
    mlp = dv.MLPConfig(w["width"], w["hidden"])

    def new_model(seed, enc_=enc):
        return dv.Model((0, 0, 0), (nx, ny, nz), 0, enc_, mlp, seed=seed)

    def cfg(steps, prec_code=precision, seed=7 + rank):
        return dv.TrainConfig(batch=w["batch"], steps=steps, lr=w["lr"], lambda_bnd=w["lam"],
                              precision=prec_code, seed=seed)

    model = new_model(100 + rank)
    stream = torch.cuda.current_stream()
    gpu_index = local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0
    # clocks sampled from the warm-up through the timed region (a 20-step
    # timed call lasts about 9 ms, shorter than the sampling interval)
    clocks = ClockSampler(gpu_index)
    # warm-up (untimed): W steps, then one call of the timed step count, which
    # captures the step graphs that count replays (a capture never falls in
    # the timed region)
    dv.train([model], [vol], cfg(max(args.warmup, 3)), sync=True)
    dv.train([model], [vol], cfg(args.steps), sync=True)
    dv.train([model], [vol], cfg(max(args.steps, 200)), sync=True)  # under load while sampling
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lib.dvnr_launch_count()
    g0 = graph_stats(A)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dv.train([model], [vol], cfg(args.steps), stream=stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    g1 = graph_stats(A)
    launches = lib.dvnr_launch_count() - launches0
    clk = clocks.stop()
    ms = shard.max_over_ranks(e0.elapsed_time(e1))  # the slowest rank's time
    samples = w["batch"] * args.steps * world
    value = samples / (ms / 1e3)
    result = {
        "metric": "INR train samples/s and decode samples/s at equal PSNR vs plain FP32 path",
        "value": value, "unit": "train samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f16" if precision == A.DVNR_FP16 else "f32",
        "data": "synthetic (seeded random-phase k^-5/3 spectral field)",
        "config": {"workload": w["desc"], "global_batch": w["batch"] * world,
                   "parallelism": f"{world} independent partition models (no exchange)",
                   "precision": prec, "l2": "working set > L2 (no flush needed)",
                   "warmup_extra": f"after the warm-up, one untimed call of {args.steps} steps "
                                   "(captures the step graphs the timed call replays) and one of "
                                   f"{max(args.steps, 200)} steps (load while the clocks are sampled)"},
        "clocks": clk, "gpu_launches": int(launches),
        "graph": {"captures_in_timed_region": g1[0] - g0[0], "graph_launches": g1[1] - g0[1],
                  "eager_steps": g1[2] - g0[2],
                  "layout": "graphs of 32, 16, 8 and 4 steps for the binary digits of the step "
                            "count; fewer than 4 remaining steps launched directly"},
    }
    if rank != 0:
        return None
    legs = set() if args.no_extras else (set(LEGS) if args.legs == "all" else set(args.legs.split(",")))
    if legs - set(LEGS):
        raise SystemExit(f"unknown legs {sorted(legs - set(LEGS))}; choose from {','.join(LEGS)}")
    if not legs:
        return result
    import ctypes as C

    # ---- dominant-kernel roofline: per-launch CUDA events on the launching stream
    if "roofline" in legs:
        result["roofline"] = roofline_leg(A, dv, model, vol, cfg, w, args)
    # ---- decode and render of the trained model
    torch.cuda.synchronize()
    ex, ey, ez = nx, ny, nz
    if legs & {"decode", "render", "render_inr"}:
        out = torch.empty((ez, ey, ex), device=dev)
        model.decode_grid(out)
        torch.cuda.synchronize()
    if "decode" in legs:
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        d0.record(stream)
        for _ in range(reps):
            model.decode_grid(out)
        d1.record(stream)
        torch.cuda.synchronize()
        dec_ms = d0.elapsed_time(d1) / reps
        result["decode"] = {"value": ex * ey * ez / (dec_ms / 1e3), "unit": "decode samples/s",
                            "ms": dec_ms, "points": ex * ey * ez}
    if legs & {"render", "render_inr"}:
        tf = dv.make_tf(alpha_max=0.05)
        img = dv.render([model], tf, 1024, 1024, 512)
        torch.cuda.synchronize()
    if "render" in legs:
        A.call("dvnr_profile_enable", 1)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        dv.render([model], tf, 1024, 1024, 512, out=img)
        r1.record(stream)
        torch.cuda.synchronize()
        tms, cnt = C.c_double(), C.c_int64()
        A.call("dvnr_profile_read", b"render", C.byref(tms), C.byref(cnt))
        A.call("dvnr_profile_enable", 0)
        result["render"] = {"value": 1024 * 1024 * 512 / (tms.value / 1e3), "unit": "ray samples/s",
                            "march_ms": tms.value, "decode_plus_march_ms": r0.elapsed_time(r1),
                            "image": [1024, 1024], "samples_per_ray": 512}
    # ---- the same frame marched through the network itself (no decoded grid)
    if "render_inr" in legs:
        result["render_inr"] = render_inr_leg(model, tf, img, out, stream)
    model.close()
    if "e2e" in legs:
        e2e_legs(result, dv, A, w, vol, vol_np, new_model, cfg, precision, gpu_index, rank,
                 "gain" in legs)
    # ---- CPU baseline: the FP64 oracle on a bounded sample of the workload
    if "cpu" in legs:
        result["cpu_baseline"] = cpu_baseline(w, vol_np)
    # ---- the other two workloads of the metric, measured in the same run:
    # 64 uneven partitions in one grouped launch, and the in situ time series
    if "batched" in legs and args.workload == "spectral256":
        del vol
        torch.cuda.empty_cache()
        result["batched"] = blocks_measure(args, rank, world, local_rank, compact=True)
    if "insitu" in legs and args.workload == "spectral256":
        torch.cuda.empty_cache()
        result["insitu"] = insitu_measure(args, rank, world, local_rank, compact=True)
    return result


def roofline_leg(A, dv, model, vol, cfg, w, args):
    import ctypes as C

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    A.call("dvnr_profile_enable", 1)
    nprof = min(args.steps, 50)
    dv.train([model], [vol], cfg(nprof), sync=True)
    kern = {}
    names = ["train_fused_fp16", "mp_schedule", "adam", "minmax", "fp32_sample_encode",
             "fp32_gemm", "fp32_out_loss", "fp32_scatter"]
    for n in names:
        tms, cnt = C.c_double(), C.c_int64()
        A.call("dvnr_profile_read", n.encode(), C.byref(tms), C.byref(cnt))
        if cnt.value:
            kern[n] = (tms.value, cnt.value)
    A.call("dvnr_profile_enable", 0)
    out = _roofline(kern, w, model.n_params, w["batch"], hbm_peak, bool(peaks), nprof)
    dom = out["kernel"]
    out["traffic"], out["traffic_source"] = measured_traffic(dom, args.workload)
    if dom == "train_fused_fp16" and w["F"] == 2:
        out["request_ceiling"] = request_ceiling(A, model, vol, w, out["kernel_ms_per_step"])
    return out


def request_ceiling(A, model, vol, w, kernel_ms):
    """The resource that binds the training kernel is the rate of scattered
    L1/L2 requests, for which no datasheet figure exists: measure it. The
    library's probe issues the training step's exact requests (samples,
    volume corners, staged table gathers, gradient reductions) without the
    MLP at 1 to 8 CTAs of 128 threads per SM; its fastest launch is the
    ceiling of that request pattern here, and the kernel's time is reported
    as a fraction of it."""
    import ctypes as C

    rows = {}
    for ctas in (1, 2, 3, 4, 6, 8):
        ms = (C.c_double * 2)()
        A.call("dvnr_probe_requests", model.handle, vol.data_ptr(), w["batch"], ctas, 7, 10,
               C.cast(ms, C.c_void_p))
        rows[str(int(ms[1]))] = ms[0]
    parts = {}
    for name, mode in (("gathers", 1), ("reductions", 2), ("volume", 4)):
        ms = (C.c_double * 2)()
        A.call("dvnr_probe_requests", model.handle, vol.data_ptr(), w["batch"], 2, mode, 10,
               C.cast(ms, C.c_void_p))
        parts[name] = ms[0]
    best = min(rows.values())
    return {"probe_ms_by_ctas_per_sm": rows, "best_ms": best, "kernel_ms": kernel_ms,
            "frac": best / kernel_ms, "parts_ms_at_2_ctas_per_sm": parts,
            "what": "the training step's memory requests alone (no MLP), fastest launch shape"}


def _mean_se(xs):
    m = statistics.fmean(xs)
    se = statistics.stdev(xs) / math.sqrt(len(xs)) if len(xs) > 1 else float("nan")
    return m, se


def e2e_legs(result, dv, A, w, vol, vol_np, new_model, cfg, precision, gpu_index, rank, gain,
             seeds=4):
    """End to end through the public API, then the "equal PSNR" statistic:
    the production path and the plain FP32 path each trained from the same
    `seeds` seeded initialisations and sample streams for the full step count;
    mean PSNR difference with its standard error (paired by seed)."""
    import torch

    # ---- end to end: host volume -> device -> train -> loss to host
    pinned = torch.from_numpy(vol_np).pin_memory()
    dvol = torch.empty_like(vol)
    steps_full = w["steps_full"]

    def psnr_of(m):
        sse, mx = dv.error_stats(m.decode_grid(), vol)
        return 10 * math.log10(1.0 / (sse / vol.numel())), mx

    clocks_e2e = ClockSampler(gpu_index)
    m = new_model(100 + rank)
    w0 = m.get_weights()
    t_e2e = []
    for r in range(2):
        if r:
            m.set_weights(w0)  # same initial weights and fresh optimiser state
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dvol.copy_(pinned, non_blocking=True)
        dv.train([m], [dvol], cfg(steps_full), sync=True)
        t_e2e.append(time.perf_counter() - t0)
    result["clocks_e2e"] = clocks_e2e.stop()
    result["e2e"] = {"value": steps_full * w["batch"] / min(t_e2e), "unit": "train samples/s",
                     "h2d_bytes_per_step": int(vol.numel() * 4), "d2h_bytes_per_step": 4,
                     "step": f"upload volume, {steps_full} training iterations, read loss"}
    m.close()
    del dvol, pinned
    # ---- equal PSNR: `seeds` paired runs of both paths on the resident volume
    runs = []
    t_mp = t_32 = 0.0
    trained = None
    for k in range(seeds):
        row = {"init_seed": 100 + rank + k, "sample_seed": 7 + rank + k}
        for name, code in (("path", precision), ("fp32_path", A.DVNR_FP32)):
            m = new_model(row["init_seed"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dv.train([m], [vol], cfg(steps_full, code, seed=row["sample_seed"]), sync=True)
            dt = time.perf_counter() - t0
            if code == precision:
                t_mp += dt
            else:
                t_32 += dt
            row[name], row[name + "_max_abs"] = psnr_of(m)
            if k == 0 and code == precision and gain:
                trained = m
            else:
                m.close()
        runs.append(row)
    d = [r["path"] - r["fp32_path"] for r in runs]
    dm, dse = _mean_se(d)
    pm, pse = _mean_se([r["path"] for r in runs])
    fm, fse = _mean_se([r["fp32_path"] for r in runs])
    result["psnr"] = {"path_mean": pm, "path_se": pse, "fp32_path_mean": fm, "fp32_path_se": fse,
                      "delta_db_mean": dm, "delta_db_se": dse, "equal_psnr": abs(dm) <= 0.2,
                      "gate_db": 0.2, "runs": runs, "steps": steps_full, "seeds": seeds,
                      "note": "delta = FP16 path - plain FP32 path, paired by seed; PSNR over "
                              "all voxels from the FP64 error reduction"}
    result["fp32_path"] = {"value": seeds * steps_full * w["batch"] / t_32, "unit": "train samples/s",
                           "speedup": t_32 / t_mp}
    # ---- what the learned network gains: against the untrained network and
    # against the raw-grid fallback (trilinear) at the model's FP16 byte size
    if gain:
        result["learned_gain"] = learned_gain(trained, new_model(100 + rank), vol, dv, w, new_model, cfg)


def _profile(A, names):
    import ctypes as C

    out = {}
    for n in names:
        tms, cnt = C.c_double(), C.c_int64()
        A.call("dvnr_profile_read", n.encode(), C.byref(tms), C.byref(cnt))
        if cnt.value:
            out[n] = (tms.value, cnt.value)
    return out


def _roofline(kern, w, n_params, units, hbm_peak, have_peaks, steps):
    """Roofline of the dominant kernel over `steps` profiled steps: its
    algorithmic bytes per step (per unit x units of a step) over its device
    time per step. A step is one training launch, or one per wave when the
    step interleaves Adam wave by wave, so the time is taken per step."""
    total = sum(v[0] for v in kern.values())
    dom = max(kern, key=lambda k: kern[k][0])
    dms, dcnt = kern[dom]
    byt = kernel_bytes(dom, w, n_params, units)
    per_step = dms / steps
    ach = byt / (per_step / 1e3) / 1e9 if byt else None
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": (ach / hbm_peak) if ach else None, "traffic": None,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if have_peaks else "fallback",
            "kernel_ms_per_step": per_step, "launches_per_step": dcnt / steps,
            "avg_launch_ms": dms / dcnt, "algorithmic_bytes_per_step": byt,
            "share": {k: round(v[0] / total, 4) for k, v in kern.items()}}


def measured_traffic(kernel, workload):
    """(DRAM bytes per launch, provenance) of the training kernel from the
    committed ncu summary, if that summary was taken on the current kernel
    revision (else None)."""
    import re

    if kernel != "train_fused_fp16" or workload != "spectral256":
        return None, None
    path = os.path.join("profiles", "k_mp_train_fp16_spectral256.md")
    try:
        src = open(os.path.join(ROOT, "paper_2304_10516_gb300", "csrc", "mp_path.cu")).read()
        rev = int(re.search(r"kTrainKernelRevision = (\d+);", src).group(1))
        prof = open(os.path.join(ROOT, path)).read()
        prev = int(re.search(r"kernel revision: (\d+)", prof).group(1))
        traffic = int(re.search(r"traffic_bytes_per_launch: (\d+)", prof).group(1))
    except Exception:
        return None, None
    if rev != prev:
        return None, f"{path} was taken on kernel revision {prev}, the kernel is at {rev}"
    return traffic, f"one ncu capture committed in {path} (kernel revision {rev}), not this run"


def _peaks():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p.get("hbm_gbs", 6800.0)), True
    except Exception:
        return 6800.0, False


def blocks_measure(args, rank, world, local_rank, compact=False):
    """The partitioned workload: 64 uneven blocks of a 1024x1024x512 field,
    one INR each, all of a GPU's blocks trained by one grouped launch per
    step. Under torchrun the ranks split the one global decomposition by
    longest-processing-time on voxel count (Sec. 3.1: no exchange while
    training), so the total work is fixed (strong scaling); the frame is
    rendered per rank and composited sort-last, the PSNR reduced over ranks.
    compact: the sub-object of the default run (throughput, roofline, PSNR
    of the production path and of the plain FP32 path, decode)."""
    import torch

    from paper_2304_10516_gb300 import _abi as A
    from paper_2304_10516_gb300 import model as dv
    from paper_2304_10516_gb300 import volumes

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS["blocks64"]
    lib = A.load()
    field = volumes.spectral_torch(w["shape"], seed=w["seed"], device=dev)
    boxes_all = volumes.uneven_boxes((512, 512, 512), (4, 4, 4), (96, 160), seed=w["seed"])
    costs = [int(np.prod([h - l + 2 for l, h in zip(lo, hi)])) for lo, hi in boxes_all]
    mine = shard.rank_partitions(costs, world, rank)
    boxes = [boxes_all[i] for i in mine]
    vols = [volumes.extract_block(field, lo, hi, 1) for lo, hi in boxes]
    enc = dv.EncodingConfig(w["L"], w["F"], w["log2T"], w["base"], w["growth"])
    mlp = dv.MLPConfig(w["width"], w["hidden"])

    def fresh():
        return [dv.Model(lo, hi, 1, enc, mlp, seed=100 + i) for i, (lo, hi) in zip(mine, boxes)]

    models = fresh()
    n = len(models)

    def cfg(steps, prec=A.DVNR_FP16):
        return dv.TrainConfig(batch=w["batch"], steps=steps, lr=w["lr"], lambda_bnd=w["lam"],
                              sigma_bnd=0.005, precision=prec, seed=7)

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0 if "CUDA_VISIBLE_DEVICES" in os.environ else local_rank)
    # warm-up, then one untimed call of the timed step count (step graphs)
    dv.train(models, vols, cfg(max(args.warmup, 3)))
    dv.train(models, vols, cfg(args.steps))
    dv.train(models, vols, cfg(max(args.steps, 64)))  # under load while sampling
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    l0 = lib.dvnr_launch_count()
    g0 = graph_stats(A)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dv.train(models, vols, cfg(args.steps), sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    g1 = graph_stats(A)
    ms = shard.max_over_ranks(e0.elapsed_time(e1))
    launches = lib.dvnr_launch_count() - l0
    clk = clocks.stop()
    samples = len(boxes_all) * w["batch"] * args.steps  # all ranks together
    res = {
        "metric": "INR train samples/s and decode samples/s at equal PSNR vs plain FP32 path",
        "value": samples / (ms / 1e3), "unit": "train samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded random-phase k^-5/3 spectral field)",
        "config": {"workload": w["desc"], "models": len(boxes_all), "models_this_rank": n,
                   "global_batch": len(boxes_all) * w["batch"],
                   "parallelism": f"64 partition models split over {world} GPU(s) by LPT on voxel "
                                  "count, one grouped launch per step per GPU",
                   "l2": "working set > L2 (no flush needed)",
                   "warmup_extra": f"after the warm-up, one untimed call of {args.steps} steps "
                                   "(captures the step graphs the timed call replays) and one of "
                                   f"{max(args.steps, 64)} steps (load while the clocks are sampled)"},
        "clocks": clk, "gpu_launches": int(launches),
        "graph": {"captures_in_timed_region": g1[0] - g0[0], "graph_launches": g1[1] - g0[1],
                  "eager_steps": g1[2] - g0[2]}}
    if args.no_extras:
        return res if rank == 0 else None
    if rank == 0:
        hbm, have = _peaks()
        A.call("dvnr_profile_enable", 1)
        nprof = min(args.steps, 20)
        dv.train(models, vols, cfg(nprof))
        kern = _profile(A, ["train_fused_fp16", "mp_schedule", "adam", "minmax"])
        A.call("dvnr_profile_enable", 0)
        res["roofline"] = _roofline(kern, w, models[0].n_params * n, n * w["batch"], hbm, have, nprof)
        if args.legs == "roofline" and not compact:  # the roofline leg alone (profiling)
            return res
    # full training from fresh models, then decode and PSNR over owned voxels
    for m in models:
        m.close()
    models = fresh()
    # end to end: the blocks (with ghosts) come from pinned host memory inside
    # the timed region, as a simulation rank would hand them over
    pinned = [v.cpu().pin_memory() for v in vols]
    dvols = [torch.empty_like(v) for v in vols]
    h2d = sum(v.numel() * 4 for v in vols)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for dst, src in zip(dvols, pinned):
        dst.copy_(src, non_blocking=True)
    dv.train(models, dvols, cfg(w["steps_full"]))
    t_full = shard.max_over_ranks(time.perf_counter() - t0)
    del dvols, pinned
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    grids = [torch.empty(tuple(h - l for l, h in zip(lo, hi))[::-1], device=dev) for lo, hi in boxes]
    d0.record(stream)
    for m, g in zip(models, grids):
        m.decode_grid(g)
    d1.record(stream)
    torch.cuda.synchronize()
    dec_ms = shard.max_over_ranks(d0.elapsed_time(d1))

    def block_sse(grids_):
        sse, vox = 0.0, 0
        for (lo, hi), g in zip(boxes, grids_):
            ref = field[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].contiguous()
            s_, _ = dv.error_stats(g, ref)
            sse += s_
            vox += g.numel()
        return sse, vox

    sse, vox = block_sse(grids)
    psnr, _, vox_all = shard.global_psnr(sse, vox)
    res["decode"] = {"value": vox_all / (dec_ms / 1e3), "unit": "decode samples/s", "ms": dec_ms,
                     "points": int(vox_all)}
    res["e2e"] = {"value": len(boxes_all) * w["batch"] * w["steps_full"] / t_full,
                  "unit": "train samples/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 4 * n,
                  "step": f"upload the blocks, {w['steps_full']} grouped iterations of all models, "
                          "read losses"}
    # the same blocks through the plain FP32 path (one model after another),
    # full length, for the equal-PSNR comparison
    f32 = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dv.train(f32, vols, cfg(w["steps_full"], A.DVNR_FP32))
    t32 = shard.max_over_ranks(time.perf_counter() - t0)
    g32 = [m.decode_grid() for m in f32]
    sse32, _ = block_sse(g32)
    psnr32, _, _ = shard.global_psnr(sse32, vox)
    del g32
    for m in f32:
        m.close()
    res["psnr"] = {"path": psnr, "fp32_path": psnr32, "delta_db": psnr - psnr32,
                   "equal_psnr": abs(psnr - psnr32) <= 0.2, "gate_db": 0.2,
                   "steps": w["steps_full"], "voxel_weighted": True}
    v32 = len(boxes_all) * w["batch"] * w["steps_full"] / t32
    res["fp32_path"] = {"value": v32, "unit": "train samples/s", "speedup": res["e2e"]["value"] / v32,
                        "note": "both full 2000-iteration calls, host upload included on the FP16 side"}
    # the frame of all blocks: each rank marches its blocks in the global
    # frame one depth layer at a time, the layers of all ranks are gathered
    # and blended front to back (sort-last, Sec. 4.3)
    tf = dv.make_tf(alpha_max=0.05)
    lo_f, hi_f = (0, 0, 0), (512, 512, 512)
    layers = sorted({lo[2] for lo, _ in boxes_all})
    torch.cuda.synchronize()
    r0 = time.perf_counter()

    def render_layer(z):
        sel = [m for m, (lo, _) in zip(models, boxes) if lo[2] == z]
        if not sel:
            return torch.zeros((512, 512, 4), device=dev)
        return dv.render_in_frame(sel, lo_f, hi_f, tf, 512, 512, 256)

    img = shard.sort_last_frame(layers, render_layer, lambda ims, ds: dv.composite(ims, ds))
    torch.cuda.synchronize()
    res["render"] = {"ms": shard.max_over_ranks((time.perf_counter() - r0) * 1e3),
                     "image": [512, 512], "samples_per_ray": 256,
                     "composite": f"{len(layers)} depth layers x {world} rank(s), sort-last",
                     "alpha_mean": float(img[..., 3].mean())}
    if rank != 0:
        return None
    if compact:
        for k in ("metric", "n_gpus", "higher_is_better", "vs_baseline", "data"):
            res.pop(k, None)
        return res
    # iteration budget proportional to each block's voxel count (Sec. 3.2,
    # N_epoch = 16), then the same with the early stop at the median of the
    # moving-average losses that run ended with: models leave the grouped
    # launch at different steps
    res["adaptive_budget"] = adaptive_budget(models, vols, boxes, enc, mlp, w, rank)
    res["cpu_baseline"] = cpu_baseline(w, vols[0].cpu().numpy())
    return res


def insitu_measure(args, rank, world, local_rank, compact=False):
    """In situ time series: each step of an advected 512^3 field is compressed
    by an INR warm-started from the previous step's weights (Sec. 3.5),
    decoded back to the grid and ray-marched. compact: the sub-object of the
    default run (per-step figures summarised)."""
    import torch

    from paper_2304_10516_gb300 import _abi as A
    from paper_2304_10516_gb300 import model as dv
    from paper_2304_10516_gb300 import volumes

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS["insitu512"]
    lib = A.load()
    enc = dv.EncodingConfig(w["L"], w["F"], w["log2T"], w["base"], w["growth"])
    mlp = dv.MLPConfig(w["width"], w["hidden"])
    n3 = w["shape"][0]
    tf = dv.make_tf(alpha_max=0.05)
    clocks = ClockSampler(0 if "CUDA_VISIBLE_DEVICES" in os.environ else local_rank)
    stream = torch.cuda.current_stream()

    def cfg(steps):
        return dv.TrainConfig(batch=w["batch"], steps=steps, lr=w["lr"], lambda_bnd=w["lam"],
                              sigma_bnd=0.005, precision=A.DVNR_FP16, seed=7 + rank)

    # warm-up of the code paths on a throw-away model
    warm = dv.Model((0, 0, 0), (n3, n3, n3), 0, enc, mlp, seed=1)
    f0 = volumes.advected_torch(w["shape"], w["seed"] + rank, 0.0, device=dev)
    dv.train([warm], [f0], cfg(max(args.warmup, 3)))
    warm.close()
    grid = torch.empty((n3, n3, n3), device=dev)
    img = torch.empty((1024, 1024, 4), device=dev)
    # the series goes through a temporal window (Sec. 4.2): each push warm-
    # starts the new step from the newest one, trains it and freezes the
    # previous one; the window keeps the last w["window"] steps
    win = dv.Window([((0, 0, 0), (n3, n3, n3))], w["window"], enc, mlp, ghost=0, seed=100)
    per = []
    l0 = lib.dvnr_launch_count()
    t_train = t_dec = t_ren = t_e2e = 0.0
    img_host = torch.empty((1024, 1024, 4), pin_memory=True)
    for t in range(w["t_steps"]):
        field = volumes.advected_torch(w["shape"], w["seed"] + rank, float(t), device=dev)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        w0 = time.perf_counter()
        ev[0].record(stream)
        win.push([field], cfg(w["steps_full"]), sync=False)
        ev[1].record(stream)
        m = win.model(t, 0)
        m.decode_grid(grid)
        ev[2].record(stream)
        dv.render([m], tf, 1024, 1024, 512, out=img)
        ev[3].record(stream)
        img_host.copy_(img, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e += time.perf_counter() - w0
        tr, de, re_ = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])
        t_train += tr
        t_dec += de
        t_ren += re_
        sse, _ = dv.error_stats(grid, field)
        mb, db = win.bytes()
        per.append({"t": t, "push_ms": tr, "decode_ms": de, "render_ms": re_,
                    "psnr": 10 * math.log10(1.0 / (sse / grid.numel())),
                    "last_loss": m.state()["last_loss"], "window_device_bytes": db})
        del field
    # the whole window visualised at the last step, straight from the cached
    # networks (frozen FP16 models, no decoded grids)
    first, last = win.range()
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for s_ in range(first, last + 1):
        dv.render_inr([win.model(s_, 0)], tf, 1024, 1024, 512, out=img)
    r1.record(stream)
    torch.cuda.synchronize()
    mb, db = win.bytes()
    window = {"capacity": w["window"], "steps_cached": last - first + 1,
              "model_bytes_fp16": mb, "device_bytes": db,
              "raw_grid_bytes_same_steps": (last - first + 1) * n3 ** 3 * 4,
              "render_inr_ms_per_cached_step": r0.elapsed_time(r1) / (last - first + 1)}
    win.close()
    launches = lib.dvnr_launch_count() - l0
    clk = clocks.stop()
    t_train = shard.max_over_ranks(t_train)
    T = w["t_steps"]
    samples = T * w["steps_full"] * w["batch"] * world
    res = {
        "metric": "INR train samples/s and decode samples/s at equal PSNR vs plain FP32 path",
        "value": samples / (t_train / 1e3), "unit": "train samples/s", "n_gpus": world,
        "steps": T * w["steps_full"], "warmup": args.warmup,
        "ms_per_step": t_train / (T * w["steps_full"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded advected k^-5/3 spectral field)",
        "config": {"workload": w["desc"], "global_batch": w["batch"] * world,
                   "parallelism": "one model per GPU"},
        "clocks": clk, "gpu_launches": int(launches),
        "decode": {"value": T * n3 ** 3 / (t_dec / 1e3), "unit": "decode samples/s",
                   "ms_per_step": t_dec / T},
        "render": {"value": T * 1024 * 1024 * 512 / (t_ren / 1e3), "unit": "ray samples/s",
                   "ms_per_step_incl_decode": t_ren / T},
        "window": window,
        "e2e": {"value": samples / t_e2e if world == 1 else None, "unit": "train samples/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 1024 * 1024 * 4 * 4,
                "step": "one time step through the public API: window push (new model, warm start, "
                        f"{w['steps_full']} iterations, freeze), decode 512^3, ray-march 1024x1024x512, "
                        "image to pinned host memory; the field is produced on the device, as by a "
                        "simulation sharing the GPU"},
        "per_step": per,
    }
    if compact:
        ps = [r["psnr"] for r in per]
        res["psnr"] = {"min": min(ps), "max": max(ps), "mean": statistics.fmean(ps)}
        res["push_ms"] = {"min": min(r["push_ms"] for r in per), "max": max(r["push_ms"] for r in per)}
        for k in ("metric", "n_gpus", "higher_is_better", "vs_baseline", "data", "per_step"):
            res.pop(k, None)
    return res


def render_inr_leg(model, tf, img_grid, grid, stream):
    """Direct INR ray-march of the benchmark frame: time, image PSNR against
    the decoded-grid march and the device memory each needs beyond the
    model (decoded grid vs per-segment composites)."""
    import torch

    from paper_2304_10516_gb300 import model as dv

    w = h = 1024
    spr = 512
    img = dv.render_inr([model], tf, w, h, spr)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        dv.render_inr([model], tf, w, h, spr, out=img)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    mse = float(((img - img_grid) ** 2).mean())
    return {"value": w * h * spr / (ms / 1e3), "unit": "ray samples/s (network inferences/s)",
            "ms": ms, "psnr_vs_grid_march_db": 10 * math.log10(1.0 / max(mse, 1e-30)),
            "max_abs_vs_grid_march": float((img - img_grid).abs().max()),
            "work_bytes": w * h * 16 + min(w * h, (1 << 24) // spr) * spr * 4,
            "grid_bytes": grid.numel() * 4,
            "model_bytes_fp16": model.n_params * 2}


def adaptive_budget(models, vols, boxes, enc, mlp, w, rank):
    """Grouped training with per-model budgets ceil(N_vox / B) * 16 and then
    with early stop as well; throughput counts the iterations each model ran."""
    import statistics

    import torch

    from paper_2304_10516_gb300 import _abi as A
    from paper_2304_10516_gb300 import model as dv

    for m in models:
        m.close()
    out = {}
    stop = 0.0
    for name in ("budget", "budget_and_stop"):
        ms_ = [dv.Model(lo, hi, 1, enc, mlp, seed=100 + i) for i, (lo, hi) in enumerate(boxes)]
        cfg = dv.TrainConfig(batch=w["batch"], epochs=16, lr=w["lr"], lambda_bnd=w["lam"],
                             sigma_bnd=0.005, precision=A.DVNR_FP16, seed=7 + rank,
                             stop_loss=stop, stop_decay=0.9)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dv.train(ms_, vols, cfg, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = [m.state() for m in ms_]
        iters = [s_["iter"] for s_ in st]
        sse, vox = 0.0, 0
        for m, v in zip(ms_, vols):
            ref = v[1:-1, 1:-1, 1:-1].contiguous()
            s2, _ = dv.error_stats(m.decode_grid(), ref)
            sse += s2
            vox += ref.numel()
        out[name] = {"value": sum(iters) * w["batch"] / (ms / 1e3), "unit": "train samples/s",
                     "ms": ms, "iterations_min": min(iters), "iterations_max": max(iters),
                     "iterations_sum": sum(iters), "stopped_models": sum(s_["stopped"] for s_ in st),
                     "psnr": 10 * math.log10(1.0 / (sse / vox))}
        if name == "budget":
            stop = statistics.median(s_["loss_ema"] for s_ in st)
            out["stop_loss"] = stop
        for m in ms_:
            m.close()
    return out


def _grid_same_bytes(vol, n_bytes):
    """PSNR of the raw-grid fallback at n_bytes of FP16: the volume
    downsampled to that many voxels and read back trilinearly (voxel centres
    aligned)."""
    import torch.nn.functional as Fn

    side = int(math.floor((n_bytes / 2) ** (1.0 / 3.0)))
    v5 = vol[None, None]
    small = Fn.interpolate(v5, size=(side,) * 3, mode="trilinear", align_corners=True).half().float()
    back = Fn.interpolate(small, size=tuple(vol.shape), mode="trilinear", align_corners=True)[0, 0]
    return back.contiguous(), side


def learned_gain(model, untrained, vol, dv, w, new_model, cfg):
    """PSNR of the trained INR vs the untrained one and vs a grid of the same
    FP16 byte budget (the fallback): the memory the representation saves and
    what that memory buys when spent on a plain grid instead. Then the same
    comparison over the table size T and the step count, to show where the
    learned representation overtakes the fallback."""
    import torch

    def psnr_of(dec):
        sse, mx = dv.error_stats(dec, vol)
        return 10 * math.log10(1.0 / (sse / vol.numel())), mx

    p_inr, mx_inr = psnr_of(model.decode_grid())
    p_init, _ = psnr_of(untrained.decode_grid())
    inr_bytes = model.n_params * 2
    back, side = _grid_same_bytes(vol, inr_bytes)
    p_grid, mx_grid = psnr_of(back)
    model.close()
    untrained.close()
    raw = vol.numel() * 4
    out = {"inr_bytes_fp16": inr_bytes, "raw_bytes_fp32": raw, "compression_ratio": raw / inr_bytes,
           "psnr_inr": p_inr, "max_abs_inr": mx_inr, "psnr_untrained": p_init,
           "psnr_grid_same_bytes": p_grid, "max_abs_grid_same_bytes": mx_grid,
           "grid_side_same_bytes": side}
    curve = []
    for log2T, steps in ((19, 8000), (18, 2000), (17, 2000), (16, 2000), (16, 8000), (14, 2000),
                         (12, 2000), (12, 8000)):
        enc = dv.EncodingConfig(w["L"], w["F"], log2T, w["base"], w["growth"])
        m = new_model(100, enc)
        dv.train([m], [vol], cfg(steps), sync=True)
        p, _ = psnr_of(m.decode_grid())
        b = m.n_params * 2
        g, gs = _grid_same_bytes(vol, b)
        pg, _ = psnr_of(g)
        curve.append({"log2_T": log2T, "steps": steps, "inr_bytes_fp16": b,
                      "compression_ratio": raw / b, "psnr_inr": p, "psnr_grid_same_bytes": pg,
                      "gain_db": p - pg, "grid_side": gs})
        m.close()
    out["curve"] = curve
    # the same comparison on a field with a sharp, localised feature (a thin
    # wrinkled front), which the spectral field lacks
    from paper_2304_10516_gb300 import volumes

    fr = torch.from_numpy(volumes.front(tuple(vol.shape))).to(vol.device)

    def psnr_fr(dec):
        sse, _ = dv.error_stats(dec, fr)
        return 10 * math.log10(1.0 / (sse / fr.numel()))

    fcurve = []
    for log2T in (19, 16, 14, 12):
        enc = dv.EncodingConfig(w["L"], w["F"], log2T, w["base"], w["growth"])
        m = new_model(100, enc)
        dv.train([m], [fr], cfg(w["steps_full"]), sync=True)
        p = psnr_fr(m.decode_grid())
        b = m.n_params * 2
        g, gs = _grid_same_bytes(fr, b)
        pg = psnr_fr(g)
        fcurve.append({"log2_T": log2T, "steps": w["steps_full"], "inr_bytes_fp16": b,
                       "compression_ratio": raw / b, "psnr_inr": p, "psnr_grid_same_bytes": pg,
                       "gain_db": p - pg, "grid_side": gs})
        m.close()
    out["front_field"] = {"field": "thin wrinkled front (tanh, 1.5 voxels) over a gentle background, "
                                   f"{'x'.join(str(v) for v in vol.shape)}", "curve": fcurve}
    return out


def _oracle_steps(orc, w, vol_np, batch, budget_s, max_steps):
    """FP64 training iterations of the workload's model at `batch` until
    budget_s of wall time (at least one); returns (steps, seconds)."""
    oc = orc.Config(w["L"], w["F"], w["log2T"], w["base"], w["growth"], w["width"], w["hidden"])
    th = orc.init_params(oc, 100)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    tc = orc.TrainConfig(batch=batch, lr=w["lr"], seed=7, lambda_bnd=w["lam"])
    st = orc.State()
    vmin, vmax = float(vol_np.min()), float(vol_np.max())
    t0 = time.perf_counter()
    steps = 0
    while True:
        orc.train(oc, tc, st, th, m1, m2, vol_np, vmin, vmax, 1)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= max_steps:
            break
    return steps, time.perf_counter() - t0, oc.n_params


def cpu_baseline(w, vol_np, budget_s=12.0):
    """The FP64 oracle on the host cores at the workload's own batch (all
    cores), and single-threaded on a smaller batch."""
    import oracle as orc

    cores = orc.set_threads(os.cpu_count() or 1)
    steps, dt, P = _oracle_steps(orc, w, vol_np, w["batch"], budget_s, 50)
    out = {"value": steps * w["batch"] / dt, "unit": "train samples/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{steps} FP64 training iterations of the same model at the full batch "
                     f"{w['batch']} (Adam over all {P} parameters each iteration), {dt:.1f} s"}
    b1 = min(w["batch"], 1 << 12)
    orc.set_threads(1)
    try:
        s1, d1, _ = _oracle_steps(orc, w, vol_np, b1, 5.0, 50)
    finally:
        orc.set_threads(cores)
    out["single_thread"] = {"value": s1 * b1 / d1, "unit": "train samples/s", "cores": 1,
                            "sample": f"{s1} FP64 training iterations at batch {b1} "
                                      f"(Adam over all {P} parameters each iteration), {d1:.1f} s"}
    return out


# ------------------------------------------------------ reference arm ------
def run_reference(args):
    """The FP64 oracle timed on the host cores on the workload of our arm:
    the same model, volume and batch (2^18 for the 256^3 workload) while the
    whole run stays within about 60 full steps; beyond that the batch is
    scaled down by a power of two and the sample says so."""
    import oracle as orc

    from paper_2304_10516_gb300 import volumes

    w = WORKLOADS[args.workload]
    vol_np = volumes.spectral(w["shape"], seed=w["seed"]) if args.workload == "spectral256" \
        else volumes.blobs(w["shape"][0], seed=w["seed"])
    oc = orc.Config(w["L"], w["F"], w["log2T"], w["base"], w["growth"], w["width"], w["hidden"])
    th = orc.init_params(oc, 100)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    total = args.steps + max(args.warmup, 1)
    batch = w["batch"]
    while batch > 1024 and total * batch > 60 * w["batch"]:
        batch //= 2
    tc = orc.TrainConfig(batch=batch, lr=w["lr"], seed=7, lambda_bnd=w["lam"])
    st = orc.State()
    cores = orc.set_threads(os.cpu_count() or 1)
    vmin, vmax = float(vol_np.min()), float(vol_np.max())
    orc.train(oc, tc, st, th, m1, m2, vol_np, vmin, vmax, max(args.warmup, 1))
    t0 = time.perf_counter()
    orc.train(oc, tc, st, th, m1, m2, vol_np, vmin, vmax, args.steps)
    dt = time.perf_counter() - t0
    value = args.steps * batch / dt
    sample = (f"each step one FP64 training iteration of the same model at batch {batch}"
              + (" (the full step)" if batch == w["batch"] else
                 f" (a bounded sample of the {w['batch']}-sample step)"))
    return {
        "impl": "reference", "metric": "INR train samples/s and decode samples/s at equal PSNR "
        "vs plain FP32 path", "value": value, "unit": "train samples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random-phase k^-5/3 spectral field)",
        "config": {"workload": w["desc"], "global_batch": batch, "parallelism": "1 CPU process"},
        "cpu_baseline": {"value": value, "unit": "train samples/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "train samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "blocks64":
        res = blocks_measure(args, rank, world, local_rank)
    elif args.workload == "insitu512":
        res = insitu_measure(args, rank, world, local_rank)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
