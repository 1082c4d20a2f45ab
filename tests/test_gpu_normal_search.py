"""GPU parity of the similar-normal search (Sec. 3.2.2) against the oracle:
with the normal only in the fingerprint, each lookup walks its voxel's probe
window and pools the cells whose quantized normal is within r steps of its
own.  Through pps_filter and the split calls, FP32 and fixed point, with and
without a temporal blend.

Bars (per vertex): counts and statuses bit-exact; fixed point bit-exact
(pooled int64 sums); FP32 the summation bound (n + 1) 2^-24 relative (at
least 1e-5) plus one rounding per pooled cell (at most P = 64 of them); after
a blend, 8 2^-24 per blended frame on top.

With the normal only in the fingerprint, a voxel on a curved surface can hold
more distinct quantized normals than the probe window has slots, so a few keys
overflow even at P = 64.  Which ones depends on the order of insertion:
overflow is all-or-none per key (checked), the overflowed vertices keep their
own contribution, and the oracle then runs on the other vertices (same jitter
counters) -- the cells the table does hold."""
import numpy as np
import pytest
import torch

from oracle import pps_oracle as O
from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
P = 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


def _setup(radius, width=160, height=120, **fkw):
    w = configs.small()
    spec = configs.frame_spec(w, 0, 0)
    spec.view.width, spec.view.height = width, height
    spec.bounces = 2
    cfg = w.filters[0]
    cfg.pixel_angle = spec.view.pixel_angle()
    cfg.normal_in_home_hash = False
    cfg.max_probes = P
    cfg.normal_search = radius + 1
    for k, v in fkw.items():
        setattr(cfg, k, v)
    return w, spec, cfg


def _gen(spec, frame=0):
    v = scene.trace_stream(spec, frame, "cpu")
    return {k: v[k] for k in scene.STREAMS}


def _dev(v):
    return {k: v[k].to("cuda").contiguous() for k in scene.STREAMS}


def _np(v):
    return {k: v[k].numpy() for k in scene.STREAMS}


def _rgb(out):
    return torch.stack([out[c] for c in "rgb"], 1).cpu().numpy()


def _oracle_on_table_cells(cfg, eye, frame, vn, out):
    """The oracle over the vertices whose key the table holds: overflow is
    all-or-none per key and such vertices return their own contribution."""
    st = out["status"].cpu().numpy()
    ovf = st == 2
    full = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), eye, frame, vn)
    for c in np.unique(full.cell[ovf]):
        assert np.all(ovf[full.cell == c])
    own = np.column_stack([vn[c] for c in "rgb"])
    assert np.array_equal(_rgb(out)[ovf], own[ovf])
    assert ovf.mean() < 2e-3
    keep = np.nonzero(~ovf)[0]
    fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), eye, frame,
                        {k: a[keep] for k, a in vn.items()}, ids=keep.astype(np.uint32))
    return fr, keep


def _run(tab, d, eye, frame, fused, blend=False, alpha=0.2):
    if fused:
        return tab.filter(d, eye, frame, blend=blend, alpha=alpha)
    tab.build(eye, frame)
    slots = torch.empty(d["px"].numel(), dtype=torch.int32, device="cuda")
    tab.insert(d, slots)
    if blend:
        tab.blend(alpha)
    return tab.query(d, slots)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("fixed", [False, True])
@pytest.mark.parametrize("radius", [0, 2, 6])
def test_similar_normals_match_oracle(radius, fixed, fused):
    _, spec, cfg = _setup(radius, accum_fixed=fixed)
    v = _gen(spec)
    tab = pps.Table(cfg)
    out = _run(tab, _dev(v), spec.view.eye, 2, fused)
    fr, keep = _oracle_on_table_cells(cfg, spec.view.eye, 2, _np(v), out)
    val64, valfx, cnt = O.similar_normals(fr, radius)
    assert tab.stats()["device_error"] == 0
    if radius:
        assert (cnt > fr.count).mean() > 0.05  # the search pools other normals' cells
    assert np.array_equal(out["count"].cpu().numpy().astype(np.int64)[keep], cnt)
    assert np.array_equal(out["status"].cpu().numpy()[keep], np.where(cnt < 4, 1, 0))
    got = _rgb(out)[keep]
    if fixed:
        assert np.array_equal(got, valfx)
    else:
        tol = np.maximum(1e-5, (cnt + 1) * U)[:, None] + P * U
        rel = np.abs(got.astype(np.float64) - val64) / np.abs(val64)
        assert np.all(rel <= tol), f"max rel {rel.max():.3e}"
    tab.close()


def test_radius_zero_equals_the_plain_lookup():
    """r = 0 pools only the vertex's own cell: the same results, bit for bit
    in fixed point, as the table without the search, on the vertices whose key
    neither run lost to the probe limit (which keys overflow depends on the
    order of insertion)."""
    _, spec, cfg = _setup(0, accum_fixed=True)
    d = _dev(_gen(spec))
    tab = pps.Table(cfg)
    a = tab.filter(d, spec.view.eye, 1)
    cfg.normal_search = 0
    tab2 = pps.Table(cfg)
    b = tab2.filter(d, spec.view.eye, 1)
    torch.cuda.synchronize()
    keep = (a["status"] != 2) & (b["status"] != 2)
    assert (~keep).float().mean().item() < 4e-3
    for c in ("r", "g", "b", "count", "status"):
        assert torch.equal(a[c][keep], b[c][keep]), c
    tab.close()
    tab2.close()


@pytest.mark.parametrize("fused", [True, False])
def test_similar_normals_after_temporal_blend(fused):
    """Three blended frames.  Voxels of a quarter of the default edge keep the
    number of normals per voxel well below the window, so that no history
    window overflows (the oracle's blend has no history limit)."""
    w, _, cfg = _setup(3, hist_mode=1, log2_hist_slots=20, voxel_scale=1.0)
    alpha = 0.2
    tab = pps.Table(cfg)
    p = O.KeyParams(**cfg.oracle_kwargs())
    hist = O.History.empty()
    for f in range(3):
        spec = configs.frame_spec(w, 0, f)
        spec.view = scene.View(160, 120, eye=(0.05 * f, 3.0, -12.0), target=(0.05 * f, 0.5, 0.0))
        spec.bounces = 2
        v = _gen(spec, f)
        out = _run(tab, _dev(v), spec.view.eye, f, fused, blend=True, alpha=alpha)
        st = tab.stats()
        assert st["hist_overflow"] == 0 and st["device_error"] == 0, st
        fr, keep = _oracle_on_table_cells(cfg, spec.view.eye, f, _np(v), out)
        hist, val, cnt = O.blend(hist, fr, alpha)
        cv = np.zeros((fr.tuples.shape[0], 3))
        cw = np.zeros(fr.tuples.shape[0], dtype=np.int64)
        cv[fr.cell] = val
        cw[fr.cell] = cnt
        ref, _, rcnt = O.similar_normals(fr, 3, cell_value=cv, cell_weight=cw)
        got_n = out["count"].cpu().numpy().astype(np.int64)[keep]
        assert np.array_equal(got_n, rcnt), (f, int((got_n != rcnt).sum()))
        tol = np.maximum(1e-5, (rcnt + 1) * U)[:, None] + 8 * U * (f + 1) + 2 * P * U
        rel = np.abs(_rgb(out)[keep].astype(np.float64) - ref) / np.abs(ref)
        assert np.all(rel <= tol), f"frame {f}: max rel {rel.max():.3e}"
    assert tab.stats()["hist_overflow"] == 0
    tab.close()


def test_batch_and_noalloc_reject_normal_search():
    import ctypes
    _, spec, cfg = _setup(2, width=64, height=64)
    d = _dev(_gen(spec))
    n = d["px"].numel()
    tab = pps.Table(cfg)
    out = pps.empty_output(n, "cuda")
    with pytest.raises(pps.PPSError) as e:
        pps.Batch([(tab, d, out)])
    assert e.value.code == pps.PPS_EINVAL
    tab.close()
    params = pps.make_params(cfg)
    rc = pps.lib().pps_filter_noalloc(ctypes.byref(params), ctypes.byref(pps.camera(spec.view.eye)),
                                      0, ctypes.byref(pps.make_vertices(d, n)), n,
                                      ctypes.byref(pps.make_output(out, n)), None)
    assert rc == pps.PPS_EINVAL
