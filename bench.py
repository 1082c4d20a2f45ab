"""Throughput of hashed path space filtering on synthetic HD frames.

One step = one frame of the whole hot path through the library's fused launch
(pps_filter): key construction (Alg. 1), probing insert with atomic
accumulation (Sec. 3.2), temporal blend (Sec. 3.4.1), one lookup per vertex,
and the per-frame clear.  The workload is the HD configuration: 1920x1080, one
path per pixel, 3 bounces with Russian roulette 0.8 (about 5.06 M vertices per
frame), table 2^23 slots, FP32 history of 2^25 slots, alpha = 0.2, 16 frames
with the camera moving 0.01 in x per frame; frames are generated once on the
GPU and stay resident in HBM (182 MB of input per frame, larger than L2, and
the steps cycle through the 16 frames).

Multi-GPU (torchrun): every rank filters its own independent stream of frames
(different path seeds) with its own table; no collective touches the data
path (weak scaling).  `value` is all ranks' vertices / the slowest rank's time.

`--impl reference` times the CPU oracle (the plain numpy implementation the
tests compare against) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered path vertices/sec (insert+query) and ms/frame at 1080p×3 bounces vs plain"
UNIT = "vertices/s"
FRAMES = 16
CSRC = os.path.join(ROOT, "paper_1902_05942_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_fused_hd_traffic.json")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources that define the headline kernel; its DRAM counters stay valid while they do
KERNEL_SOURCES = ("pps_device.cuh", "pps_internal.h", "pps_kernels.cu")


def _strip_comments(src: str) -> str:
    """C++ source without its comments (string and character literals kept),
    so that editing a comment does not count as changing a kernel."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "".join(out)


def _source_hash(texts=None) -> str:
    """Hash of the code (comments and blank space at line ends left out) of
    the sources that define the persistent kernels."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        if texts is None:
            with open(os.path.join(CSRC, f), encoding="utf-8") as fh:
                src = fh.read()
        else:
            src = texts[f]
        code = "\n".join(line.rstrip() for line in _strip_comments(src).splitlines() if line.strip())
        h.update(f.encode())
        h.update(code.encode())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes of one headline launch from the committed ncu summary, or None
    when the kernel sources changed since those counters were taken."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        if d.get("source_sha") == _source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def reduce_ranks(ms: float, vertices: float, device=None):
    """Across ranks: the slowest rank's time and all ranks' vertices (weak
    scaling; value = total vertices / slowest time).  One rank: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, vertices
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([vertices], dtype=torch.float64, device=device)
    dist.all_reduce(v)
    return float(t.item()), float(v.item())


def make_frames(rank: int, device):
    import torch
    from paper_1902_05942_gb300 import configs, scene
    w = configs.hd(FRAMES)
    frames = []
    for f in range(FRAMES):
        spec = configs.frame_spec(w, 0, f)
        spec.path_seed += 1000 * rank
        spec.radiance_seed += 1000 * rank
        v = scene.trace_stream(spec, f, device)
        frames.append(({k: v[k] for k in scene.STREAMS}, tuple(spec.view.eye)))
    torch.cuda.synchronize()
    return w, frames


def algorithmic_bytes(n: int, cells: int, hist_bytes: int = 32) -> int:
    """Per frame: 36 B of vertex input + 12 B of output + 1 B status per vertex;
    per occupied cell 20 B (accumulator and fingerprint written back once) and
    `hist_bytes` for its history value read and written by the blend (FP32
    history: 16 B read + 16 B written; FP16: 8 + 8; none: 0)."""
    return 49 * n + (20 + hist_bytes) * cells


def subframe_error(frames, cfg, nsub=1_000_000, blended_frames=0, **table_kw):
    """Precision of a table variant against the FP64 oracle, off the timed
    path: the first `nsub` vertices of the leading frames filtered as frames of
    their own (`blended_frames` > 0: that many frames with the temporal blend,
    the oracle blending in FP64 without any storage rounding), then the last
    frame's max relative error and RMSE per channel."""
    import numpy as np
    import torch
    from oracle import pps_oracle as O
    from paper_1902_05942_gb300 import pps, scene
    tab = pps.Table(cfg, **table_kw)
    fixed = tab.fixed
    hist = O.History.empty()
    nf = max(1, blended_frames)
    for f in range(nf):
        v, eye = frames[f % len(frames)]
        sub = {k: v[k][:nsub].contiguous() for k in scene.STREAMS}
        out = tab.filter(sub, eye, f, blend=blended_frames > 0, alpha=cfg.alpha)
        torch.cuda.synchronize()
        v_np = {k: t.cpu().numpy() for k, t in sub.items()}
        fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), eye, f, v_np)
        if blended_frames:
            hist, ref, cnt = O.blend(hist, fr, cfg.alpha)
        else:
            ref, cnt = fr.mean64, fr.count
    o = {k: t.cpu().numpy() for k, t in out.items()}
    tab.close()
    ok = o["status"] != 2
    got = np.column_stack([o[c] for c in "rgb"]).astype(np.float64)[ok]
    rel = np.abs(got - ref[ok]) / np.abs(ref[ok])
    res = {"vertices": int(ok.sum()), "frames": nf, "max_rel": float(rel.max()),
           "rmse_rgb": [float(x) for x in np.sqrt(((got - ref[ok]) ** 2).mean(axis=0))],
           "counts_equal": bool(np.array_equal(o["count"].astype(np.int64)[ok], cnt[ok]))}
    if fixed and not blended_frames:
        res["bit_exact_vs_oracle_fixed"] = bool(np.array_equal(
            np.column_stack([o[c] for c in "rgb"])[ok], fr.mean_fixed[ok]))
    return res


def oracle_error(v_np, cfg, eye, frame, out_np, view=None, fixed=False):
    """Error of one plain frame's results against the FP64 oracle over the
    same vertices (the GPU's `out_np` from filtering exactly `v_np` as frame
    `frame`): max relative error and RMSE per channel over the vertices that
    kept a cell (status != OVERFLOW); with `fixed`, whether the results equal
    the oracle's fixed-point averages bit for bit."""
    import numpy as np
    from oracle import pps_oracle as O
    kw = cfg.oracle_kwargs()
    if view is not None:
        kw["pixel_angle"] = O.pixel_angle(view.fov_y_deg, view.height)
    fr = O.filter_frame(O.KeyParams(**kw), eye, frame, v_np)
    ok = out_np["status"] != 2
    got = np.column_stack([out_np[c] for c in "rgb"]).astype(np.float64)[ok]
    ref = fr.mean64[ok]
    rel = np.abs(got - ref) / np.abs(ref)
    res = {"vertices": int(ok.sum()), "max_rel": float(rel.max()),
           "rmse_rgb": [float(x) for x in np.sqrt(((got - ref) ** 2).mean(axis=0))],
           "counts_equal": bool(np.array_equal(out_np["count"].astype(np.int64)[ok], fr.count[ok]))}
    if fixed:
        res["bit_exact_vs_oracle_fixed"] = bool(np.array_equal(
            np.column_stack([out_np[c] for c in "rgb"])[ok], fr.mean_fixed[ok]))
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1902_05942_gb300 import build, pps
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    w, frames = make_frames(rank, dev)
    cfg = w.filters[0]
    tab = pps.Table(cfg)
    n_max = max(fr[0]["px"].numel() for fr in frames)
    out = pps.empty_output(n_max, dev, count=False, status=True)
    stream = torch.cuda.current_stream()
    # argument blocks built once per frame; the timed loop only calls the C ABI
    import ctypes
    L = pps.lib()
    sptr = stream.cuda_stream
    calls = []
    for v, eye in frames:
        n = v["px"].numel()
        calls.append((pps.camera(eye), pps.make_vertices(v, n), n,
                      pps.make_output({k: t[:n] for k, t in out.items()}, n)))

    def step(i):
        cam, vs, n, os_ = calls[i % FRAMES]
        rc = L.pps_filter(tab.handle, ctypes.byref(cam), i, ctypes.byref(vs), n, 1, cfg.alpha,
                          ctypes.byref(os_), sptr)
        if rc:
            raise pps.PPSError(rc, pps.last_error())
        return n

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    st = tab.stats()
    total_n = sum(frames[(args.warmup + i) % FRAMES][0]["px"].numel() for i in range(args.steps))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cells = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = tab.stats()  # cells of the last frame (deterministic per frame)
    # cells per frame: one extra untimed pass per distinct frame for the byte count
    for i in range(min(args.steps, FRAMES)):
        step(args.warmup + i)
        cells.append(tab.stats()["frame_cells"])
    plain = plain_leg(frames, cfg, calls, args.steps, args.warmup)
    fallbacks = {}
    if not args.no_fallbacks:
        fsteps = min(args.steps, 16)
        for fb in ("coarse", "neighbors"):
            fallbacks[fb] = fallback_leg(frames, cfg, calls, fsteps, args.warmup, fb,
                                         out["status"])
    hvariants = {}
    if not args.no_fallbacks:
        hvariants["evict"] = history_leg(frames, cfg, calls, fsteps, args.warmup,
                                         hist_evict=True, log2_hist_slots=23)
        hvariants["migrate"] = history_leg(frames, cfg, calls, fsteps, args.warmup,
                                           hist_migrate=True)
    precision = {}
    if not args.no_fallbacks:
        precision["fixed_point_plain"] = history_leg(frames, cfg, calls, fsteps, args.warmup,
                                                     blend=0, hist_mode=0, accum_fixed=True)
        precision["fixed_point_plain"]["error_vs_fp64_oracle"] = subframe_error(
            frames, cfg, hist_mode=0, accum_fixed=True)
        precision["fp16_history"] = history_leg(frames, cfg, calls, fsteps, args.warmup,
                                                hist_mode=2)
        precision["fp16_history"]["error_vs_fp64_oracle"] = subframe_error(
            frames, cfg, blended_frames=3, hist_mode=2)
        precision["fp32_headline"] = {"error_vs_fp64_oracle": subframe_error(
            frames, cfg, blended_frames=3)}
        precision["error_sample"] = ("first 1,000,000 vertices of the leading HD frames "
                                     "filtered as frames of their own, off the timed path")
    merge = {}
    if not args.no_fallbacks:
        for m, name in ((1, "none"), (2, "gated"), (3, "always")):
            merge[name] = {
                "temporal_ms": history_leg(frames, cfg, calls, fsteps, args.warmup,
                                           tune={"merge": m})["ms_per_frame"],
                "plain_ms": history_leg(frames, cfg, calls, fsteps, args.warmup, blend=0,
                                        hist_mode=0, tune={"merge": m})["ms_per_frame"]}
    ms, job_n = reduce_ranks(ms, float(total_n), dev)
    value = job_n / (ms / 1e3)
    ms_step = ms / args.steps
    # roofline of the dominant (only) kernel: k_fused_ws (the pipelined
    # insert, the default at this table size), one launch per step
    mean_n = total_n / args.steps
    mean_c = sum(cells) / len(cells)
    alg = algorithmic_bytes(int(mean_n), int(mean_c))
    achieved = alg / (ms_step / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = _traffic_per_launch()

    # end to end through the host-buffer entry point: the uploads of each
    # frame's inputs from pinned host memory, the filter, and the downloads of
    # r, g, b and status, all inside the timed region; pps_filter_host_async
    # overlaps one frame's uploads with the previous frame's filter and
    # downloads, and pps_host_wait ends the timed region
    e2e = None
    if not args.no_e2e:
        hv = [{k: t.cpu().pin_memory() for k, t in fr[0].items()} for fr in frames[:4]]
        ho = []
        for _ in range(2):
            o = pps.empty_output(n_max, "cpu", count=False, status=True)
            ho.append({k: t.pin_memory() for k, t in o.items()})
        tab_h = pps.Table(cfg)

        def hstep(i):
            v = hv[i % len(hv)]
            n = v["px"].numel()
            o = {k: t[:n] for k, t in ho[i % 2].items()}
            pps.pps_filter_host_async(tab_h.handle, pps.camera(frames[i % len(hv)][1]), i,
                                      pps.make_vertices(v, n, device=False), n, True, cfg.alpha,
                                      pps.make_output(o, n, device=False), stream)
            return n

        for i in range(args.warmup):
            hstep(i)
        pps.pps_host_wait(tab_h.handle)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        hn = sum(hstep(args.warmup + i) for i in range(args.steps))
        pps.pps_host_wait(tab_h.handle)
        dt = time.perf_counter() - t0
        dt, hn = reduce_ranks(dt, float(hn), dev)
        e2e = {"value": hn / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(36 * mean_n), "d2h_bytes_per_step": int(13 * mean_n),
               "ms_per_step": 1e3 * dt / args.steps,
               "api": "pps_filter_host_async + pps_host_wait (pinned host buffers)"}
        tab_h.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "hd: 1920x1080 x 3 bounces (RR 0.8), ~5.06M vertices/frame, "
                                   "T=2^23, P=16, FP32 history 2^25, alpha=0.2, 16 frames, "
                                   "camera +0.01/frame",
                       "vertices_per_frame": mean_n, "cells_per_frame": mean_c,
                       "l2": "inputs larger than L2 (182 MB per frame, 16 frames cycled)",
                       "parallelism": f"replicas x{ws} (independent frame streams)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind, "kernel": "k_fused_ws",
                         "algorithmic_bytes_per_launch": alg},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "e2e": e2e,
            "plain": dict(plain, temporal_over_plain=ms_step / plain["ms_per_frame"]),
        }
        if fallbacks:
            line["fallbacks"] = {
                "workload": "the headline temporal HD frames with a low-count fallback "
                            "(count < 4): coarse = multi-level accumulation, neighbors = "
                            "3x3x3 neighborhood search", **fallbacks}
        if hvariants:
            line["history_variants"] = {
                "workload": "the headline temporal HD frames with an evicting history of "
                            "2^23 cells (evict) or a history that follows changes of "
                            "resolution (migrate)", **hvariants}
        if merge:
            line["merge_modes"] = {
                "workload": "the headline HD frames (temporal and plain) with each warp "
                            "aggregation of the pipelined insert (pps_tuning.merge): none, "
                            "gated (__match_any_sync where neighbouring lanes repeat a key; "
                            "the default), always", **merge}
        if precision:
            line["precision"] = {
                "workload": "the headline HD frames: fixed-point (int64) accumulation without "
                            "history, and the temporal frame with an FP16 history", **precision}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(frames[0], w, args.cpu_sample)
        if not args.no_mlp:
            line["mlp_fallback"] = mlp_leg(frames, cfg)
        if not args.no_batched:
            del frames
            line["batched"] = batched_leg()
        if not args.no_stress:
            line["stress"] = stress_leg()
        print(json.dumps(line), flush=True)
    tab.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def plain_leg(frames, cfg, calls, steps, warmup):
    """The same resident HD frames through the plain filter (no history, no
    blend): one persistent launch per frame, timed with CUDA events like the
    headline."""
    import ctypes
    import torch
    from paper_1902_05942_gb300 import pps
    tab = pps.Table(cfg, hist_mode=0)
    L = pps.lib()
    stream = torch.cuda.current_stream()

    def step(i):
        cam, vs, n, os_ = calls[i % len(calls)]
        rc = L.pps_filter(tab.handle, ctypes.byref(cam), i, ctypes.byref(vs), n, 0, 0.0,
                          ctypes.byref(os_), stream.cuda_stream)
        if rc:
            raise pps.PPSError(rc, pps.last_error())
        return n

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total = sum(step(warmup + i) for i in range(steps))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    tab.close()
    return {"workload": "the same HD frames, plain filter (no temporal blend)",
            "ms_per_frame": ms, "vertices_per_s": total / steps / (ms * 1e-3)}


def fallback_leg(frames, cfg, calls, steps, warmup, fallback, status):
    """The headline workload (temporal HD frames) with a low-count fallback:
    "coarse" = multi-level accumulation (a second table one level coarser,
    Sec. 3.3.2), "neighbors" = neighborhood search over the 3x3x3 block
    (Sec. 3.3.1).  Same timing as the headline; reports the share of vertices
    that took the fallback in the last frame."""
    import ctypes
    import torch
    from paper_1902_05942_gb300 import pps
    tab = pps.Table(cfg, fallback=fallback)
    L = pps.lib()
    stream = torch.cuda.current_stream()

    def step(i):
        cam, vs, n, os_ = calls[i % len(calls)]
        rc = L.pps_filter(tab.handle, ctypes.byref(cam), i, ctypes.byref(vs), n, 1, cfg.alpha,
                          ctypes.byref(os_), stream.cuda_stream)
        if rc:
            raise pps.PPSError(rc, pps.last_error())
        return n

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total = sum(step(warmup + i) for i in range(steps))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # share of the vertices of one more (steady-state) frame that took the fallback
    n = step(warmup + steps)
    torch.cuda.synchronize()
    code = pps.STATUS_COARSE if fallback == "coarse" else pps.STATUS_NEIGHBORS
    share = float((status[:n] == code).float().mean().item())
    tab.close()
    return {"ms_per_frame": ms, "vertices_per_s": total / steps / (ms * 1e-3),
            "fallback_share": share}


def history_leg(frames, cfg, calls, steps, warmup, blend=1, tune=None, **table_kw):
    """The headline workload with a table variant, same timing as the
    headline: "evict" = an evicting history of 2^23 cells (Sec. 3.4.3),
    "migrate" = the history following changes of resolution (Sec. 3.4.2;
    split kernels, two blend launches); the precision modes: fixed-point
    accumulation (plain frame) and an FP16 history."""
    import ctypes
    import torch
    from paper_1902_05942_gb300 import pps
    tab = pps.Table(cfg, **table_kw)
    if tune:
        tab.tune(**tune)
    L = pps.lib()
    stream = torch.cuda.current_stream()

    def step(i):
        cam, vs, n, os_ = calls[i % len(calls)]
        rc = L.pps_filter(tab.handle, ctypes.byref(cam), i, ctypes.byref(vs), n, blend,
                          cfg.alpha, ctypes.byref(os_), stream.cuda_stream)
        if rc:
            raise pps.PPSError(rc, pps.last_error())
        return n

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total = sum(step(warmup + i) for i in range(steps))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    st = tab.stats()
    tab.close()
    return {"ms_per_frame": ms, "vertices_per_s": total / steps / (ms * 1e-3),
            "hist_occupied": st["hist_occupied"], "hist_overflow_cells": st["hist_overflow"]}


MLP_FWD_FLOP = 2 * (80 * 64 + 64 * 64 + 64 * 64 + 64 * 3)  # per sample, algorithmic


def mlp_leg(frames, cfg, steps_timed=8):
    """The learned-fallback workload on the resident HD frames: per frame the
    temporal filter, 4 Adam steps of 16,384 samples on cells with count >= 8,
    and inference for vertices with count < 4.  Times each part with CUDA
    events; RMSE of the GPU predictions against the FP64 oracle network with
    the same trained weights, on sampled low-count vertices of the last frame."""
    import numpy as np
    import torch
    from oracle import mlp_oracle as M
    from paper_1902_05942_gb300 import pps
    tab = pps.Table(cfg)
    net = pps.MLP(pps.mlp_params())
    n_max = max(fr[0]["px"].numel() for fr in frames)
    out = pps.empty_output(n_max, frames[0][0]["px"].device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_f = t_t = t_i = 0.0
    n_low = 0
    warm = 4
    for i in range(warm + steps_timed):
        v, eye = frames[i % len(frames)]
        n = v["px"].numel()
        o = {k: t[:n] for k, t in out.items()}
        ev[0].record()
        tab.filter(v, eye, i, blend=True, alpha=cfg.alpha, out=o)
        ev[1].record()
        net.train(v, o, i)
        ev[2].record()
        net.infer(v, o)
        ev[3].record()
        torch.cuda.synchronize()
        if i >= warm:
            t_f += ev[0].elapsed_time(ev[1])
            t_t += ev[1].elapsed_time(ev[2])
            t_i += ev[2].elapsed_time(ev[3])
            n_low += int((o["status"] == pps.STATUS_MLP).sum().item())
    k = steps_timed
    train_flop = 4 * 16384 * 3 * MLP_FWD_FLOP
    infer_flop = (n_low / k) * MLP_FWD_FLOP
    # accuracy against the FP64 oracle network with the same weights
    w = net.get_weights().astype(np.float64)
    low = torch.nonzero(o["status"] == pps.STATUS_MLP).flatten()
    pick = low[torch.randperm(low.numel(), device=low.device)[:50000]].cpu().numpy()
    vn = {c: v[c][:n].cpu().numpy() for c in ("px", "py", "pz", "nx", "ny", "nz")}
    P = np.column_stack([vn["px"][pick], vn["py"][pick], vn["pz"][pick]])
    Nn = np.column_stack([vn["nx"][pick], vn["ny"][pick], vn["nz"][pick]])
    X = M.encode(P, Nn, (-100.0,) * 3, (100.0,) * 3)
    gpu = np.column_stack([o[c][:n].cpu().numpy()[pick] for c in "rgb"]).astype(np.float64)
    ref_model = M.forward(w, X, bf16=True).y
    ref_fp64 = M.forward(w, X, bf16=False).y
    rmse = lambda a, b: [float(np.sqrt(((a[:, j] - b[:, j]) ** 2).mean())) for j in range(3)]
    tab.close()
    net.close()
    peak = 1915.4
    return {
        "workload": "hd temporal + learned fallback (count < 4), 4 x 16384 samples/frame",
        "ms_filter": t_f / k, "ms_train": t_t / k, "ms_infer": t_i / k,
        "ms_frame": (t_f + t_t + t_i) / k,
        "lowcount_vertices_per_frame": n_low / k,
        "train_tflops": train_flop / (t_t / k * 1e-3) / 1e12,
        "infer_tflops": infer_flop / (t_i / k * 1e-3) / 1e12 if t_i > 0 else None,
        "bf16_peak_tflops": peak,
        "rmse_vs_fp64_oracle_rgb": rmse(gpu, ref_fp64),
        "rmse_vs_oracle_bf16_model_rgb": rmse(gpu, ref_model),
        "rms_prediction_rgb": [float(np.sqrt((ref_fp64[:, j] ** 2).mean())) for j in range(3)],
    }


def batched_leg(steps_timed=8, tune=True):
    """The batched workload: 8 views of uneven resolution (2x each 1280x720,
    1920x1080, 2560x1440, 3840x2160), 1 path per pixel, 2 bounces, each view
    with its own table; table size and probe limit per view and the batch
    width chosen by the autotuner on the first frame (off the timed path);
    then graph replays of the one persistent launch, timed with CUDA events,
    against the same views filtered one pps_filter call at a time."""
    import torch
    from paper_1902_05942_gb300 import autotune, configs, pps, scene
    w = configs.batched()
    views = []
    for i, spec in enumerate(w.streams):
        v = scene.trace_stream(spec, 0, "cuda")
        views.append(({k: v[k] for k in scene.STREAMS}, tuple(spec.view.eye)))
    torch.cuda.synchronize()
    cfgs, tuned = [], []
    for i, (v, eye) in enumerate(views):
        cfg = w.filters[i]
        if tune:
            cfg, trials = autotune.tune_view(cfg, v, eye, log2_range=(21, 24), probes=(8, 16, 32))
        cfgs.append(cfg)
        tuned.append({"view": f"{w.streams[i].view.width}x{w.streams[i].view.height}",
                      "vertices": v["px"].numel(), "log2_slots": cfg.log2_slots,
                      "max_probes": cfg.max_probes})
    outs = [pps.empty_output(v["px"].numel(), "cuda", count=True) for v, _ in views]
    cams = [eye for _, eye in views]

    def make(width, block):
        tabs = []
        for cfg in cfgs:
            t = pps.Table(cfg)
            t.tune(width, block=block)
            tabs.append(t)
        b = pps.Batch([(tabs[i], views[i][0], outs[i]) for i in range(len(views))])
        b._tables = tabs
        return b

    (width, block), wt = autotune.tune_batch_shape(make, cams) if tune else ((2, 512), {})
    batch = make(width, block)
    total = sum(v["px"].numel() for v, _ in views)
    for i in range(3):
        batch.run(cams, i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps_timed):
        batch.run(cams, 3 + i)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps_timed
    cells = [t.stats()["frame_cells"] for t in batch._tables]
    last = 3 + steps_timed - 1
    # precision of the last batched frame against the FP64 oracle: the two
    # smallest views in full (their vertices are the oracle's whole input)
    errs = []
    for i in range(2):
        v, eye = views[i]
        errs.append(oracle_error({k: v[k].cpu().numpy() for k in scene.STREAMS}, cfgs[i], eye,
                                 last, {k: t.cpu().numpy() for k, t in outs[i].items()},
                                 w.streams[i].view))
    # the same views, one call per view
    tabs = [pps.Table(c) for c in cfgs]
    for t in tabs:
        t.tune(width, block=block)
    def seq(f):
        for i, (v, eye) in enumerate(views):
            tabs[i].filter(v, eye, f, out=outs[i])
    seq(0)
    torch.cuda.synchronize()
    e0.record()
    for i in range(steps_timed):
        seq(1 + i)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / steps_timed
    batch.close()
    for t in tabs + batch._tables:
        t.close()
    alg = sum(algorithmic_bytes(v["px"].numel(), c, hist_bytes=0) for (v, _), c in zip(views, cells))
    peak, peak_kind = _peaks()
    return {"workload": "8 views (2x 720p/1080p/1440p/2160p), 2 bounces, one persistent launch "
                        "replayed from a CUDA graph",
            "vertices_per_frame": total, "ms_per_frame": ms,
            "vertices_per_s": total / (ms * 1e-3),
            "ms_per_frame_one_call_per_view": ms_seq,
            "batch_width": width, "block": block, "launch_shape_trials_ms": wt, "views": tuned,
            "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg / (ms * 1e-3) / 1e9 / peak,
                         "peak_source": peak_kind, "kernel": "k_fused_multi",
                         "algorithmic_bytes_per_launch": alg},
            "error_vs_fp64_oracle": {"views": "the two 1280x720 views of the last timed frame, "
                                              "every vertex", "per_view": errs}}


def stress_leg(steps_timed=6):
    """The stress workload: 3840x2160 at 2 paths per pixel, 6 bounces (~61 M
    vertices per frame, 80 % of them squeezed into 5 % of the scene box),
    table 2^26 slots at load ~0.7, FP16 history of 2^28 cells with a temporal
    blend, and the learned fallback (training + inference) every frame.  Two
    frames are generated on the GPU and alternate; times per frame with CUDA
    events: the filter alone and the whole frame."""
    import torch
    from paper_1902_05942_gb300 import configs, pps, scene
    w = configs.stress()
    cfg = w.filters[0]
    frames = []
    for f in range(2):
        spec = configs.frame_spec(w, 0, f)
        v = scene.trace_stream(spec, f, "cuda")
        frames.append(({k: v[k] for k in scene.STREAMS}, tuple(spec.view.eye)))
        del v
    torch.cuda.synchronize()
    n = frames[0][0]["px"].numel()
    # probe limit by the autotuner at the workload's table size: the fastest
    # limit whose overflowing share stays within 0.1 % (the paper wants probe
    # failures rare, Sec. 3.2)
    from paper_1902_05942_gb300 import autotune
    tuned, trials = autotune.tune_view(cfg, frames[0][0], frames[0][1],
                                       log2_range=(cfg.log2_slots, cfg.log2_slots),
                                       probes=(16, 32), max_overflow=1e-3)
    cfg = tuned
    tab = pps.Table(cfg)
    net = pps.MLP(pps.mlp_params())
    out = pps.empty_output(max(fr[0]["px"].numel() for fr in frames), "cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_f = t_all = 0.0
    nv = 0
    for i in range(2 + steps_timed):
        v, eye = frames[i % 2]
        m = v["px"].numel()
        o = {k: t[:m] for k, t in out.items()}
        ev[0].record()
        tab.filter(v, eye, i, blend=True, alpha=cfg.alpha, out=o)
        ev[1].record()
        net.train(v, o, i)
        net.infer(v, o)
        ev[2].record()
        torch.cuda.synchronize()
        if i >= 2:
            t_f += ev[0].elapsed_time(ev[1])
            t_all += ev[0].elapsed_time(ev[2])
            nv += m
    st = tab.stats()
    tab.close()
    net.close()
    k = steps_timed
    err = subframe_error(frames, cfg, blended_frames=2)
    del frames, out
    torch.cuda.empty_cache()
    alg = algorithmic_bytes(int(nv / k), st["frame_cells"], hist_bytes=16)
    peak, peak_kind = _peaks()
    bw = alg / (t_f / k * 1e-3) / 1e9
    return {"workload": f"3840x2160 x2 paths x6 bounces, 80% of vertices in 5% of the box, "
                        f"T=2^26, P={cfg.max_probes} (tuned), FP16 history 2^28, alpha=0.2, "
                        f"learned fallback",
            "vertices_per_frame": nv / k, "ms_filter": t_f / k, "ms_frame_with_mlp": t_all / k,
            "filter_vertices_per_s": nv / (t_f * 1e-3),
            "max_probes": cfg.max_probes, "probe_trials": trials,
            "overflow_vertices_last_frame": st["overflow_vertices"],
            "overflow_share_last_frame": st["overflow_vertices"] / (nv / k),
            "frame_cells_last_frame": st["frame_cells"],
            "roofline": {"bound": "hbm", "achieved": bw, "peak": peak, "unit": "GB/s",
                         "frac": bw / peak, "peak_source": peak_kind, "kernel": "k_fused",
                         "algorithmic_bytes_per_launch": alg},
            "error_vs_fp64_oracle": dict(err, sample="first 1,000,000 vertices of the two "
                                                     "stress frames, two blended frames with "
                                                     "the tuned table, off the timed path")}


def _oracle_step(v_np, w, frame, eye, hist):
    from oracle import pps_oracle as O
    cfg = w.filters[0]
    fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), eye, frame, v_np)
    hist, val, cnt = O.blend(hist, fr, cfg.alpha)
    return hist


def _shard_cells(task):
    """One worker of the all-core oracle (a spawned process): the oracle's keys
    of one shard of vertices (global vertex ids, so the jitter is the same) and
    the shard's cells -- sorted tuples, FP64 sums, fixed-point sums, counts --
    with each vertex's cell within the shard."""
    import numpy as np
    from oracle import pps_oracle as O
    v_np, kw, frame, eye, ids = task
    keys = O.vertex_keys(O.KeyParams(**kw), eye, frame, v_np["px"], v_np["py"], v_np["pz"],
                         v_np["nx"], v_np["ny"], v_np["nz"], ids=ids)
    uniq, inv, cnt = O.group_cells(keys.tuples())
    rgb = np.column_stack([v_np[c].astype(np.float32) for c in "rgb"])
    s64 = np.column_stack([np.bincount(inv, weights=rgb[:, j].astype(np.float64),
                                       minlength=uniq.shape[0]) for j in range(3)])
    sfx = np.zeros((uniq.shape[0], 3), dtype=np.int64)
    np.add.at(sfx, inv, O.to_fixed(rgb))
    return uniq, s64, sfx, cnt, inv


def _oracle_step_sharded(pool, nshards, v_np, w, frame, eye, hist):
    """The oracle's filter + blend with the key construction and per-shard
    group-by spread over worker processes, then the partial cells merged (an
    ordered group-by of the shards' tuples, sums and counts added) and the
    blend run on the merged cells."""
    import numpy as np
    from oracle import pps_oracle as O
    cfg = w.filters[0]
    n = v_np["px"].shape[0]
    bounds = np.linspace(0, n, nshards + 1).astype(np.int64)
    tasks = [({k: a[lo:hi] for k, a in v_np.items()}, cfg.oracle_kwargs(), frame, eye,
              np.arange(lo, hi, dtype=np.uint32)) for lo, hi in zip(bounds[:-1], bounds[1:])]
    parts = pool.map(_shard_cells, tasks)
    allt = np.concatenate([p[0] for p in parts])
    uniq, minv = np.unique(allt, axis=0, return_inverse=True)
    minv = minv.reshape(-1)
    C = uniq.shape[0]
    s64 = np.zeros((C, 3))
    sfx = np.zeros((C, 3), dtype=np.int64)
    cnt = np.zeros(C, dtype=np.int64)
    np.add.at(s64, minv, np.concatenate([p[1] for p in parts]))
    np.add.at(sfx, minv, np.concatenate([p[2] for p in parts]))
    np.add.at(cnt, minv, np.concatenate([p[3] for p in parts]))
    off = np.cumsum([0] + [p[0].shape[0] for p in parts[:-1]])
    cell = np.concatenate([minv[o + p[4]] for o, p in zip(off, parts)])
    fr = O.FrameResult(None, cell, uniq, cnt[cell], s64[cell] / cnt[cell][:, None],
                       O.fixed_mean_f32(sfx, cnt)[cell], cnt, s64, sfx, None, None)
    hist, _, _ = O.blend(hist, fr, cfg.alpha)
    return hist


def cpu_baseline(frame, w, sample):
    """The CPU oracle as it stands, single-threaded numpy, on the first `sample`
    vertices of one HD frame (a bounded sample: the full frame takes ~15 s);
    beside it the same step spread over all host cores (the key construction
    and group-by per shard in spawned worker processes, then the merge and the
    blend in this process)."""
    import multiprocessing as mp
    from oracle import pps_oracle as O
    v, eye = frame
    v_np = {k: t[:sample].cpu().numpy() for k, t in v.items()}
    t0 = time.perf_counter()
    _oracle_step(v_np, w, 0, eye, O.History.empty())
    dt = time.perf_counter() - t0
    res = {"value": sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"first {sample} vertices of HD frame 0, filter + blend, numpy FP64"}
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        small = {k: a[:4096] for k, a in v_np.items()}
        _oracle_step_sharded(pool, cores, small, w, 0, eye, O.History.empty())  # start-up
        t0 = time.perf_counter()
        _oracle_step_sharded(pool, cores, v_np, w, 0, eye, O.History.empty())
        dta = time.perf_counter() - t0
    res["all_cores"] = {"value": sample / dta, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": res["sample"] + "; keys and per-shard group-by in one "
                                  "spawned process per core, merge and blend in the parent"}
    return res


def run_reference(args):
    """The oracle on the host cores, same workload/metric, bounded samples."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import torch
    from oracle import pps_oracle as O
    from paper_1902_05942_gb300 import configs, scene
    w = configs.hd(FRAMES)
    # bounded: about 30 M oracle vertices in total keeps the run to a few minutes
    sample = max(50_000, min(args.cpu_sample, int(30e6 / (args.steps + args.warmup))))
    hist = O.History.empty()
    data = []
    for f in range(FRAMES if args.steps + args.warmup > FRAMES else args.steps + args.warmup):
        spec = configs.frame_spec(w, 0, f)
        v = scene.trace_stream(spec, f, "cpu")
        data.append(({k: v[k][:sample].numpy() for k in scene.STREAMS}, tuple(spec.view.eye)))
    for i in range(args.warmup):
        v, eye = data[i % len(data)]
        hist = _oracle_step(v, w, i, eye, hist)
    t0 = time.perf_counter()
    n = 0
    for i in range(args.steps):
        v, eye = data[(args.warmup + i) % len(data)]
        hist = _oracle_step(v, w, args.warmup + i, eye, hist)
        n += v["px"].shape[0]
    dt = time.perf_counter() - t0
    value = n / dt
    desc = f"first {sample} vertices of each HD frame, filter + blend, numpy FP64"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "hd (CPU oracle on a bounded sample of each frame)",
                   "sample_vertices": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ncu_case(args):
    """A small fixed case for profilers, no timing.  `--case hd`: one HD frame
    through the fused launch, three times (history from --hist, batch width
    from --batch, fallback from --fallback).  `--case mlp`: that frame
    filtered with history, then the learned fallback: one training call (4
    Adam steps of 16,384 samples) and one inference call."""
    import torch
    from paper_1902_05942_gb300 import build, configs, pps, scene
    build.build()
    torch.cuda.set_device(0)
    w = configs.hd()
    cfg = w.filters[0]
    spec = configs.frame_spec(w, 0, 0)
    v = scene.trace_stream(spec, 0, "cuda")
    d = {k: v[k] for k in scene.STREAMS}
    if args.case == "mlp":
        out = pps.empty_output(d["px"].numel(), "cuda")
        tab = pps.Table(cfg)
        net = pps.MLP(pps.mlp_params())
        tab.filter(d, spec.view.eye, 0, blend=True, alpha=cfg.alpha, out=out)
        net.train(d, out, 0)
        net.infer(d, out)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "mlp",
                          "lowcount": int((out["status"] == pps.STATUS_MLP).sum().item())}))
        return
    out = pps.empty_output(d["px"].numel(), "cuda", count=False)
    tab = pps.Table(cfg, hist_mode=args.hist, fallback=args.fallback)
    if args.batch:
        tab.tune(args.batch)
    for i in range(3):
        tab.filter(d, spec.view.eye, i, blend=args.hist != 0, alpha=cfg.alpha, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "hd", "hist": args.hist, "fallback": args.fallback,
                      "stats": tab.stats()}))


def run_rates(args):
    """Random memory-operation rates of this GPU (pps_bench_rate): each
    operation on its own random 32-byte sector of a 32 MB (L2-resident) and a
    1 GB region."""
    import torch
    from paper_1902_05942_gb300 import build, pps
    build.build()
    torch.cuda.set_device(0)
    out = {}
    for mb in (32, 1024):
        region = torch.zeros(mb << 20, dtype=torch.uint8, device="cuda")
        for kind in pps.RATE_KINDS:
            out[f"{kind}@{mb}MB"] = pps.pps_bench_rate(kind, region, 1 << 25) / 1e9
        del region
    print(json.dumps({"rates_G_ops_per_s": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=48)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--cpu-sample", type=int, default=1_500_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mlp", action="store_true", help="skip the learned-fallback leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-views leg")
    ap.add_argument("--no-fallbacks", action="store_true", help="skip the low-count fallback legs")
    ap.add_argument("--no-stress", action="store_true", help="skip the stress-workload leg")
    ap.add_argument("--ncu-case", action="store_true", help="small fixed case for profilers")
    ap.add_argument("--rates", action="store_true", help="random memory-operation rates")
    ap.add_argument("--hist", type=int, default=1, help="--ncu-case: history mode")
    ap.add_argument("--batch", type=int, default=0, help="--ncu-case: batch width")
    ap.add_argument("--case", default="hd", choices=("hd", "mlp"), help="--ncu-case: workload")
    ap.add_argument("--fallback", default="none", choices=("none", "coarse", "neighbors"),
                    help="--ncu-case hd: low-count fallback")
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.rates:
        return run_rates(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
