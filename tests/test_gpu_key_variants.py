"""GPU parity of the key variants (a given distance for the level of detail,
an extra key word; Sec. 3.1.1, 3.1.2 and the caption of Algorithm 1) against
the oracle: keys bit-exact, cells and counts bit-exact, fixed-point values
bit-exact, FP32 values within the summation bar."""
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


def _setup(**kw):
    w = configs.small()
    spec = configs.frame_spec(w, 0, 0)
    spec.view.width, spec.view.height = 128, 96
    spec.bounces = 2
    cfg = w.filters[0]
    cfg.pixel_angle = spec.view.pixel_angle()
    for k, v in kw.items():
        setattr(cfg, k, v)
    v = scene.trace_stream(spec, 0, "cpu")
    v = {k: v[k] for k in scene.STREAMS}
    n = v["px"].numel()
    rng = np.random.default_rng(11)
    eye = np.array(spec.view.eye, dtype=np.float32)
    p = np.column_stack([v[c].numpy() for c in ("px", "py", "pz")])
    d = np.linalg.norm(p - eye, axis=1).astype(np.float32)
    # a path-length-like distance: the camera distance stretched per vertex
    v["dist"] = torch.from_numpy((d * rng.uniform(1.0, 3.0, n)).astype(np.float32))
    v["extra"] = torch.from_numpy(rng.integers(0, 3, n).astype(np.int32))
    return spec, cfg, v


def _np(v):
    out = {k: t.numpy() for k, t in v.items()}
    if "extra" in out:
        out["extra"] = out["extra"].view(np.uint32)
    return out


def _dev(v):
    return {k: t.to("cuda").contiguous() for k, t in v.items()}


@pytest.mark.parametrize("use", ["dist", "extra", "both"])
def test_keys_bit_exact(use):
    spec, cfg, v = _setup()
    keep = {"dist": ["dist"], "extra": ["extra"], "both": ["dist", "extra"]}[use]
    vv = {k: t for k, t in v.items() if k in scene.STREAMS or k in keep}
    tab = pps.Table(cfg)
    tab.build(spec.view.eye, 3)
    h, f = tab.keys(_dev(vv))
    kw = cfg.oracle_kwargs()
    kw["log2_slots"] = 32
    a = _np(vv)
    k = O.vertex_keys(O.KeyParams(**kw), spec.view.eye, 3, *(a[c] for c in ("px", "py", "pz", "nx", "ny", "nz")),
                      dist=a.get("dist"), extra=a.get("extra"))
    assert np.array_equal(h.cpu().numpy().view(np.uint32), k.home)
    assert np.array_equal(f.cpu().numpy().view(np.uint32), k.fp)
    tab.close()


@pytest.mark.parametrize("fixed", [False, True])
def test_filter_with_key_variants_matches_oracle(fixed):
    spec, cfg, v = _setup(accum_fixed=fixed)
    tab = pps.Table(cfg)
    out = tab.filter(_dev(v), spec.view.eye, 2)
    fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), spec.view.eye, 2, _np(v))
    assert np.array_equal(out["count"].cpu().numpy().astype(np.int64), fr.count)
    got = torch.stack([out[c] for c in "rgb"], 1).cpu().numpy()
    if fixed:
        assert np.array_equal(got, fr.mean_fixed)
    else:
        tol = np.maximum(1e-5, (fr.count + 1) * U)[:, None]
        assert np.all(np.abs(got - fr.mean64) <= tol * np.abs(fr.mean64))
    tab.close()


def test_neighborhood_search_keeps_extra_words_apart():
    spec, cfg, v = _setup(accum_fixed=True, fallback="neighbors")
    del v["dist"]
    tab = pps.Table(cfg)
    out = tab.filter(_dev(v), spec.view.eye, 1)
    fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), spec.view.eye, 1, _np(v))
    _, valfx, cnt, st = O.neighborhood(fr, 4)
    assert np.array_equal(out["count"].cpu().numpy().astype(np.int64), cnt)
    assert np.array_equal(out["status"].cpu().numpy(), st)
    assert np.array_equal(torch.stack([out[c] for c in "rgb"], 1).cpu().numpy(), valfx)
    tab.close()


def test_variants_rejected_where_unsupported():
    spec, cfg, v = _setup()
    d = _dev(v)
    tab = pps.Table(cfg)
    out = pps.empty_output(d["px"].numel(), "cuda")
    with pytest.raises(pps.PPSError) as e:
        pps.Batch([(tab, d, out)])
    assert e.value.code == pps.PPS_EINVAL
    tab.close()
