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
