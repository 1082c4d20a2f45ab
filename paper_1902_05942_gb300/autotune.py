"""Autotuner for table size, probe limit and launch shape.

Off the timed path, on a sample frame of each view: for every candidate table
size (2^lo .. 2^hi slots) and probe limit, filter the view a few times with the
library's fused launch, time it with CUDA events and read the overflow count;
keep the fastest candidate whose overflowing share of vertices stays below
`max_overflow` (if none does, the one with the least overflow), candidates
within 3 % of the fastest counting as ties that the smaller table and probe
limit win.  Then choose the launch shape of a batched launch -- batch width
(vertices per thread per insert step) and block shape (threads per CTA) -- by
timing the whole batch with each.  The paper sizes the table in
proportion to the image (Sec. 4); the candidate range brackets that choice.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import torch

from . import pps


def _time(fn, reps: int) -> float:
    fn()  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def choose(trials: List[dict], max_overflow: float, tie: float = 0.03) -> dict:
    """Among the trials whose overflowing share of vertices is at most
    `max_overflow`, those within `tie` (relative) of the fastest count as equally
    fast -- timing noise of a few per cent must not decide -- and of those the
    one with the smallest table, then the smallest probe limit, then the
    smallest launch-shape key wins, so that identical views get identical
    choices.  If no trial qualifies, the one with the least overflow (ties: the
    fastest)."""
    if not trials:
        raise ValueError("no trials")
    ok = [t for t in trials if t["overflow"] <= max_overflow]
    if ok:
        best = min(t["ms"] for t in ok)
        near = [t for t in ok if t["ms"] <= best * (1.0 + tie)]
        return min(near, key=lambda t: (t.get("log2_slots", 0), t.get("max_probes", 0),
                                        t.get("shape", 0), t["ms"]))
    return min(trials, key=lambda t: (t["overflow"], t["ms"]))


def tune_view(cfg, v: Dict[str, torch.Tensor], eye, log2_range=(21, 24),
              probes: Sequence[int] = (8, 16, 32), reps: int = 3, max_overflow: float = 1e-5):
    """Best (log2_slots, max_probes) for one view; returns (config, table of trials)."""
    n = v["px"].numel()
    out = pps.empty_output(n, v["px"].device, count=False)
    trials = []
    for lg in range(log2_range[0], log2_range[1] + 1):
        for P in probes:
            c = dataclasses.replace(cfg, log2_slots=lg, max_probes=P, hist_mode=0)
            tab = pps.Table(c)
            ms = _time(lambda: tab.filter(v, eye, 0, out=out), reps)
            ovf = tab.stats()["overflow_vertices"] / max(n, 1)
            tab.close()
            trials.append({"log2_slots": lg, "max_probes": P, "ms": ms, "overflow": ovf})
    best = choose(trials, max_overflow)
    return dataclasses.replace(cfg, log2_slots=best["log2_slots"], max_probes=best["max_probes"]), trials


def tune_batch_shape(make_batch, cams, reps: int = 3,
                     shapes: Sequence[Tuple[int, int]] = ((2, 512), (4, 512), (2, 256), (4, 256))
                     ) -> Tuple[Tuple[int, int], Dict[str, float]]:
    """Launch shape of a batched launch: batch width (vertices per thread per
    insert step) and block shape (threads per CTA), timed on the whole batch;
    `make_batch(width, block)` builds it.  Shapes within 3 % of the fastest
    count as equally fast and the first of them in `shapes` wins."""
    times = {}
    for w, blk in shapes:
        b = make_batch(w, blk)
        times[(w, blk)] = _time(lambda: b.run(cams, 0), reps)
        b.close()
    trials = [{"ms": times[s], "overflow": 0.0, "shape": i} for i, s in enumerate(shapes)]
    best = choose(trials, 1.0)
    return shapes[best["shape"]], {f"{w}x{blk}": ms for (w, blk), ms in times.items()}
