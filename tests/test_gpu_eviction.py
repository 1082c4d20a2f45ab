"""GPU checks of the evicting history (Sec. 3.4.3).

Which entries a full table evicts depends on the order in which the GPU's
threads reach them, so the checks are: without pressure, the evicting table
gives exactly the oracle's blend (keys, counts, values within the FP32 bar);
under pressure, every vertex gets either its blend with the previous frame's
history (count N_old + N_new) or a fresh start (count N_new), both matched to
the oracle; recently used entries survive where an evicting table has room
only for them; and priorities survive the rebase of the 8-bit epoch.
"""
import numpy as np
import pytest
import torch

from oracle import pps_oracle as O
from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


def _cfg(**kw):
    w = configs.small()
    cfg = w.filters[0]
    cfg.pixel_angle = scene.View(128, 96).pixel_angle()
    cfg.hist_mode = 1
    cfg.hist_evict = True
    for k, v in kw.items():
        setattr(cfg, k, v)
    return w, cfg


def _frame(w, f, eye_x=0.0, width=128, height=96, bounces=2):
    spec = configs.frame_spec(w, 0, f)
    spec.view = scene.View(width, height, eye=(eye_x + 0.05 * f, 3.0, -12.0),
                           target=(eye_x + 0.05 * f, 0.5, 0.0))
    spec.bounces = bounces
    v = scene.trace_stream(spec, f, "cpu")
    return spec, {k: v[k] for k in scene.STREAMS}


def _dev(v):
    return {k: v[k].to("cuda").contiguous() for k in scene.STREAMS}


def _np(v):
    return {k: v[k].numpy() for k in scene.STREAMS}


def _rgb(out):
    return torch.stack([out[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)


def _close(got, ref, count, frames):
    tol = np.maximum(1e-5, (count + 1) * U)[:, None] + 8 * U * frames
    return np.all(np.abs(got - ref) <= tol * np.abs(ref), axis=1)


@pytest.mark.parametrize("fused", [True, False])
def test_without_pressure_eviction_equals_the_plain_history(fused):
    w, cfg = _cfg(log2_hist_slots=19)
    tab = pps.Table(cfg)
    p = O.KeyParams(**cfg.oracle_kwargs())
    hist = O.History.empty()
    for f in range(4):
        spec, v = _frame(w, f)
        d = _dev(v)
        if fused:
            out = tab.filter(d, spec.view.eye, f, blend=True, alpha=0.2)
        else:
            tab.build(spec.view.eye, f)
            slots = torch.empty(d["px"].numel(), dtype=torch.int32, device="cuda")
            tab.insert(d, slots)
            tab.blend(0.2)
            out = tab.query(d, slots)
        fr = O.filter_frame(p, spec.view.eye, f, _np(v))
        hist, val, cnt = O.blend(hist, fr, 0.2)
        assert np.array_equal(out["count"].cpu().numpy().astype(np.int64), cnt)
        assert np.all(_close(_rgb(out), val, fr.count, f + 1))
    st = tab.stats()
    assert st["hist_overflow"] == 0 and st["hist_occupied"] == hist.tuples.shape[0]
    tab.close()


def test_under_pressure_each_vertex_blends_or_starts_afresh():
    w, cfg = _cfg(log2_hist_slots=13)  # 8,192 history cells for ~16,000 cells per frame
    tab = pps.Table(cfg)
    p = O.KeyParams(**cfg.oracle_kwargs())
    hist = O.History.empty()
    for f in range(2):
        spec, v = _frame(w, f)
        out = tab.filter(_dev(v), spec.view.eye, f, blend=True, alpha=0.2)
        fr = O.filter_frame(p, spec.view.eye, f, _np(v))
        hist, val, cnt = O.blend(hist, fr, 0.2)
        got, gcnt = _rgb(out), out["count"].cpu().numpy().astype(np.int64)
        fresh = (gcnt == fr.count) & _close(got, fr.mean64, fr.count, 1)
        blended = (gcnt == cnt) & _close(got, val, fr.count, 2)
        assert np.all(fresh | blended)
        if f == 0:
            assert fresh.all()
        else:
            had = cnt > fr.count  # cells with a frame-0 entry in the oracle's history
            assert (blended & had).sum() > 1000 and (fresh & had & ~blended).sum() > 1000
    assert tab.stats()["hist_occupied"] <= 8192
    tab.close()


def test_recently_used_entries_survive():
    """Frames 0-1 look at one part of the scene, frames 2-3 at another; the
    history (8,192 cells) holds about one view's cells (~7,500 per frame).
    At frame 3 the evicting table blends the second view's vertices whose
    frame-2 entries replaced older ones; without eviction the table is full of
    the first view's cells and the second view's cells found no room."""
    shares = {}
    for evict in (True, False):
        w, cfg = _cfg(log2_hist_slots=13, hist_evict=evict)
        tab = pps.Table(cfg)
        p = O.KeyParams(**cfg.oracle_kwargs())
        for f in range(4):
            spec, v = _frame(w, f, eye_x=-8.0 if f < 2 else 8.0, bounces=1)
            out = tab.filter(_dev(v), spec.view.eye, f, blend=True, alpha=0.2)
        fr = O.filter_frame(p, spec.view.eye, 3, _np(v))
        shares[evict] = float((out["count"].cpu().numpy() > fr.count).mean())
        tab.close()
    assert shares[True] > 0.35 and shares[True] > shares[False] + 0.15, shares


def test_priorities_survive_the_epoch_rebase():
    """300 blends on a table with room for every cell: the 8-bit epoch runs
    out at 255 and every priority drops by 128, yet no entry may be lost, so
    the evicting table's counts equal those of a table without eviction
    frame after frame."""
    w, cfg = _cfg(log2_hist_slots=15)
    tabs = [pps.Table(cfg, hist_evict=True), pps.Table(cfg, hist_evict=False)]
    spec, v = _frame(w, 0, width=48, height=32, bounces=1)
    d = _dev(v)
    for f in range(300):
        outs = [t.filter(d, spec.view.eye, f, blend=True, alpha=0.2) for t in tabs]
        if f in (100, 254, 255, 256, 299):
            assert torch.equal(outs[0]["count"], outs[1]["count"]), f
            got, ref = _rgb(outs[0]), _rgb(outs[1])
            assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref)), f
    assert outs[0]["count"].max().item() > 200
    for t in tabs:
        st = t.stats()
        assert st["device_error"] == 0 and st["hist_overflow"] == 0
        t.close()
