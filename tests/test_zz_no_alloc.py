"""The allocation-free entry point, pps_filter_noalloc, against pps_filter.

pps_filter_noalloc is for callers that may not allocate device memory while
they filter (a plug-in inside an application that owns the GPU memory budget,
a real-time thread that must not block on cudaMalloc).  It keeps its working
memory in one static device array that every call reuses, so the test calls it
twice in a row on different frames and compares each result with the table
entry point on the same inputs.  This file is collected last so that a failure
here cannot hide the other tests; it also passes when run alone.
"""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _frame(width, height, frame):
    w = configs.small()
    spec = configs.frame_spec(w, 0, 0)
    spec.view = scene.View(width, height, eye=(0.1 * frame, 3.0, -12.0),
                           target=(0.1 * frame, 0.5, 0.0))
    spec.bounces = 2
    cfg = w.filters[0]
    cfg.pixel_angle = spec.view.pixel_angle()
    v = scene.trace_stream(spec, frame, "cpu")
    return spec, cfg, {k: v[k].to("cuda").contiguous() for k in scene.STREAMS}


def _compare(out_a, out_b, what):
    """Counts and statuses equal; values within twice the FP32 summation bar
    (both sides add in some order and are each within max(1e-5, (n + 1) u)
    of the exact average).  Which keys meet the probe limit depends on the
    order of insertion, so vertices that overflowed on either side (a tiny
    share at load 0.3 with 16 probes) are left out; returns their number."""
    sa, sb = out_a["status"].cpu().numpy(), out_b["status"].cpu().numpy()
    keep = (sa != 2) & (sb != 2)
    assert np.array_equal(out_a["count"].cpu().numpy()[keep], out_b["count"].cpu().numpy()[keep]), what
    assert np.array_equal(sa[keep], sb[keep]), what
    a = torch.stack([out_a[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)[keep]
    b = torch.stack([out_b[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)[keep]
    cnt = out_b["count"].cpu().numpy().astype(np.float64)[keep]
    tol = 2 * np.maximum(1e-5, (cnt + 1) * U)[:, None]
    rel = np.abs(a - b) / np.abs(b)
    assert np.all(rel <= tol), f"{what}: max rel {rel.max():.3e}"
    return int((~keep).sum())


def _noalloc(cfg, spec, frame, d, n, log2_slots=None):
    params = pps.make_params(cfg)
    if log2_slots is not None:
        params.log2_slots = log2_slots
    out = pps.empty_output(n, "cuda")
    rc = pps.lib().pps_filter_noalloc(ctypes.byref(params), ctypes.byref(pps.camera(spec.view.eye)),
                                      frame, ctypes.byref(pps.make_vertices(d, n)), n,
                                      ctypes.byref(pps.make_output(out, n)),
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == pps.PPS_OK, pps.last_error()
    return out


def _table(cfg, spec, frame, d, log2_slots=None):
    if log2_slots is not None:
        cfg = dataclasses.replace(cfg, log2_slots=log2_slots)
    tab = pps.Table(cfg)
    out = tab.filter(d, spec.view.eye, frame)
    torch.cuda.synchronize()
    st = tab.stats()
    tab.close()
    return out, st


def test_noalloc_matches_table_entry_point_on_two_calls_in_a_row():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    for frame, (w, h) in enumerate([(300, 240), (211, 157)]):
        spec, cfg, d = _frame(w, h, frame)
        n = d["px"].numel()
        # the allocation-free call, straight through the C ABI
        params = pps.make_params(cfg)
        out_a = pps.empty_output(n, "cuda")
        rc = pps.lib().pps_filter_noalloc(ctypes.byref(params), ctypes.byref(pps.camera(spec.view.eye)),
                                          frame, ctypes.byref(pps.make_vertices(d, n)), n,
                                          ctypes.byref(pps.make_output(out_a, n)),
                                          torch.cuda.current_stream().cuda_stream)
        assert rc == pps.PPS_OK, pps.last_error()
        # the table entry point on the same inputs
        tab = pps.Table(cfg)
        out_b = tab.filter(d, spec.view.eye, frame)
        torch.cuda.synchronize()
        tab.close()
        assert torch.equal(out_a["count"], out_b["count"])
        assert torch.equal(out_a["status"], out_b["status"])
        a = torch.stack([out_a[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)
        b = torch.stack([out_b[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)
        cnt = out_b["count"].cpu().numpy().astype(np.float64)
        # both sum in FP32 in some order: each is within max(1e-5, (n + 1) u) of
        # the exact average, so they are within twice that of each other
        tol = 2 * np.maximum(1e-5, (cnt + 1) * U)[:, None]
        rel = np.abs(a - b) / np.abs(b)
        assert np.all(rel <= tol), f"call {frame}: max rel {rel.max():.3e}"


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    spec, cfg, d = _frame(64, 64, 0)
    n = d["px"].numel()
    out = pps.empty_output(n, "cuda")
    L = pps.lib()
    for field, value, nn in [("log2_slots", 21, n), ("hist_mode", 1, n), ("accum_mode", 1, n),
                             (None, None, (1 << 19) + 1)]:
        params = pps.make_params(cfg)
        if field:
            setattr(params, field, value)
        rc = L.pps_filter_noalloc(ctypes.byref(params), ctypes.byref(pps.camera(spec.view.eye)),
                                  0, ctypes.byref(pps.make_vertices(d, n)), nn,
                                  ctypes.byref(pps.make_output(out, n)), None)
        assert rc == pps.PPS_EINVAL
        assert "pps_filter_noalloc" in pps.last_error()


def test_noalloc_at_its_limits_and_after_a_larger_call():
    """n = 2^19 vertices at 2^20 slots fills every region of the static array
    (slots, accumulators, cell records, stash, control block); a 2^16-slot call
    after it must not see what the larger call left; n = 0 is a valid call.
    Each call's counters come back through pps_noalloc_stats."""
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    nmax = 1 << 19
    spec, cfg, d = _frame(640, 480, 3)
    assert d["px"].numel() >= nmax
    d = {k: t[:nmax].contiguous() for k, t in d.items()}
    cur = torch.cuda.current_stream().cuda_stream
    for log2, n in [(20, nmax), (16, 40000), (20, nmax)]:
        dd = {k: t[:n].contiguous() for k, t in d.items()}
        out_a = _noalloc(cfg, spec, 3, dd, n, log2_slots=log2)
        st_a = pps.pps_noalloc_stats(cur)
        out_b, st_b = _table(cfg, spec, 3, dd, log2_slots=log2)
        ovf = _compare(out_a, out_b, f"2^{log2} slots, {n} vertices")
        assert ovf <= 1e-4 * n
        assert st_a["vertices"] == n and st_a["device_error"] == 0
        assert abs(st_a["frame_cells"] - st_b["frame_cells"]) <= ovf
        assert max(st_a["overflow_vertices"], st_b["overflow_vertices"]) <= ovf
    empty = pps.empty_output(0, "cuda")
    params = pps.make_params(cfg)
    rc = pps.lib().pps_filter_noalloc(ctypes.byref(params), ctypes.byref(pps.camera(spec.view.eye)),
                                      0, ctypes.byref(pps.make_vertices(d, 0)), 0,
                                      ctypes.byref(pps.make_output(empty, 0)), cur)
    assert rc == pps.PPS_OK, pps.last_error()
    st = pps.pps_noalloc_stats(cur)
    assert st["vertices"] == 0 and st["frame_cells"] == 0 and st["device_error"] == 0
