"""GPU parity of the history's migration across changes of resolution (Sec.
3.4.2) against the oracle: a cell whose history entry is new takes the pooled
history of its finer children, or its coarser parent's.

Bars (per vertex): counts bit-exact; values as for the temporal blend (the
frame bar plus 8 u per blended frame, u = 2^-24) plus 40 u for a migrated old
value (its pooled sum of up to eight products and the division, all
non-negative); FP16 history: one binary16 rounding step.
"""
import numpy as np
import pytest
import torch

from oracle import pps_oracle as O
from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
CAM = (0.0, 2.0, -9.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


def _cfg(**kw):
    cfg = configs.small().filters[0]
    cfg.voxel_scale = 3.0
    cfg.pixel_angle = 0.0013
    cfg.jitter = False
    cfg.hist_mode = 1
    cfg.log2_hist_slots = 18
    cfg.hist_migrate = True
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    p = (rng.normal(0, 0.06, (n, 3)) + np.array([0.3, 1.0, 1.0])).astype(np.float32)
    nrm = np.array([[0, 1, 0], [0.6, 0.8, 0]], dtype=np.float32)[rng.integers(0, 2, n)]
    rgb = rng.lognormal(-1, 1.0, (n, 3)).astype(np.float32)
    arrs = [p[:, 0], p[:, 1], p[:, 2], nrm[:, 0], nrm[:, 1], nrm[:, 2], rgb[:, 0], rgb[:, 1],
            rgb[:, 2]]
    return {k: np.ascontiguousarray(a) for k, a in zip(scene.STREAMS, arrs)}


def _dev(v):
    return {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in v.items()}


def _rgb(out):
    return torch.stack([out[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)


def _check(out, val, cnt, fr, frames, fp16=False):
    """Counts exact; FP32 values within the temporal bar, where the history a
    cell starts from may have come from other cells' samples.

    The blended value is a non-negative weighted average of the old value and
    this frame's average, so its relative error is at most the larger of
    theirs plus the blend's three roundings (8 u per blended frame covers
    them).  This frame's average is within max(1e-5, (n + 1) u).  The old
    value was averaged over at most 8 N_old samples: its own history (N_old),
    its children's summed (sum N_i = N_old), or its parent's (N_p <= 8
    ceil(N_p / 8) = 8 N_old); so it is within max(1e-5, (8 N_old + 1) u) plus
    the earlier frames' 8 u each.  Migrating from children adds eight FP32
    products N_i c_i, seven additions and one division of non-negative terms:
    at most 9 u more (recursive summation, Higham 2002, Sec. 3.1); from a
    parent the value passes unchanged.  Hence the bar below, 10 u for the
    migration."""
    got_cnt = out["count"].cpu().numpy().astype(np.int64)
    assert np.array_equal(got_cnt, cnt)
    rel = np.abs(_rgb(out) - val) / np.abs(val)
    if fp16:
        tol = 2.0 ** -10 + 1e-5
    else:
        n_old = cnt - fr.count
        nref = np.maximum(fr.count, 8 * n_old)
        tol = np.maximum(1e-5, (nref + 1) * U)[:, None] + 8 * U * frames + 10 * U
    assert np.all(rel <= tol), f"max rel {rel.max():.3e}"


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("coarser", [True, False])
def test_level_change_matches_oracle(coarser, split):
    """The same cloud at one level, then one level coarser (the finer
    children's history added up) or one level finer (the parent's)."""
    cfg = _cfg()
    par = O.KeyParams(**cfg.oracle_kwargs())
    tab = pps.Table(cfg)
    hist = O.History.empty()
    v = _cloud(6000, 1)
    d0 = O.camera_distance(*CAM, v["px"], v["py"], v["pz"])
    dists = [d0, (2 * d0).astype(np.float32)] if coarser else [(2 * d0).astype(np.float32), d0]
    alpha = 0.25 if coarser else -1.0
    for f, dist in enumerate(dists):
        vf = {**_cloud(6000, 10 + f), **{k: v[k] for k in ("px", "py", "pz", "nx", "ny", "nz")}}
        vf["dist"] = dist
        d = _dev(vf)
        if split:
            tab.build(CAM, f)
            tab.insert(d)
            tab.blend(alpha)
            out = tab.query(d)
        else:
            out = tab.filter(d, CAM, f, blend=True, alpha=alpha)
        fr = O.filter_frame(par, CAM, f, vf)
        hist, val, cnt = O.blend(hist, fr, alpha, migrate=True)
        _check(out, val, cnt, fr, f + 1)
        if f == 1:  # every cell of the second frame migrated
            assert np.all(cnt > fr.count)
    assert tab.stats()["hist_overflow"] == 0
    tab.close()


@pytest.mark.parametrize("hist_mode", [1, 2])
def test_camera_moving_away_matches_oracle(hist_mode):
    """Small-scene frames with the camera backing off by a quarter per frame
    (jitter on): cells change level along the way; some take their children's
    or parent's history, the rest blend with their own."""
    w = configs.small()
    cfg = _cfg(jitter=True, hist_mode=hist_mode, log2_hist_slots=19)
    spec0 = configs.frame_spec(w, 0, 0)
    cfg.pixel_angle = scene.View(128, 96).pixel_angle()
    par = O.KeyParams(**cfg.oracle_kwargs())
    tab = pps.Table(cfg)
    hist = O.History.empty()
    migrated = 0
    for f in range(4):
        spec = configs.frame_spec(w, 0, f)
        back = 1.25 ** f
        spec.view = scene.View(128, 96, eye=(0.0, 3.0 * back, -12.0 * back), target=(0.0, 0.5, 0.0))
        spec.bounces = 2
        vt = scene.trace_stream(spec, f, "cpu")
        v = {k: vt[k].numpy() for k in scene.STREAMS}
        out = tab.filter(_dev(v), spec.view.eye, f, blend=True, alpha=0.2)
        fr = O.filter_frame(par, spec.view.eye, f, v)
        kw = dict(fp16=hist_mode == 2, n_cap=65535 if hist_mode == 2 else None)
        _, _, cnt_plain = O.blend(hist, fr, 0.2, **kw)
        hist, val, cnt = O.blend(hist, fr, 0.2, migrate=True, **kw)
        _check(out, val, cnt, fr, f + 1, fp16=hist_mode == 2)
        migrated += int((cnt != cnt_plain).sum())
    assert migrated > 2000, migrated
    assert tab.stats()["hist_overflow"] == 0
    tab.close()
    del spec0


def test_migrating_tables_refuse_batches_and_extra_words():
    cfg = _cfg()
    tab = pps.Table(cfg)
    v = _cloud(1000, 3)
    d = _dev(v)
    out = pps.empty_output(1000, "cuda")
    with pytest.raises(pps.PPSError) as e:
        pps.Batch([(tab, d, out)])
    assert e.value.code == pps.PPS_EINVAL
    d["extra"] = torch.zeros(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(pps.PPSError) as e:
        tab.filter(d, CAM, 0, blend=True, alpha=0.2)
    assert e.value.code == pps.PPS_EINVAL
    tab.close()
