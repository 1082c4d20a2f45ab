"""Pins of the oracle's key variants (no GPU): a given per-vertex distance for
the level of detail, and an extra 32-bit key word (Sec. 3.1.1, 3.1.2 and the
caption of Algorithm 1)."""
import math

import numpy as np
import pytest

from oracle import pps_oracle as O

CAM = (0.5, 2.0, -7.0)


def _verts(n, seed):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=(n, 3)) * 25).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return p, nrm


def _params(jitter=True, nih=True):
    return O.KeyParams(log2_slots=20, max_probes=16, voxel_scale=3.0, pixel_angle=0.0013,
                       jitter=jitter, normal_in_home_hash=nih)


def _keys(par, p, nrm, **kw):
    return O.vertex_keys(par, CAM, 9, *(p[:, i] for i in range(3)), *(nrm[:, i] for i in range(3)),
                         **kw)


def test_camera_distance_as_given_distance_reproduces_algorithm_1():
    """d = |p_cam - x| (the same FP32 operations) gives d' = |p_cam - x'|
    exactly, so every key equals the plain one."""
    p, nrm = _verts(5000, 1)
    par = _params()
    d = O.camera_distance(*CAM, p[:, 0], p[:, 1], p[:, 2])
    a, b = _keys(par, p, nrm), _keys(par, p, nrm, dist=d)
    for f in ("xq", "lod", "lod0", "home", "fp", "xj"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_given_distance_sets_the_level():
    """Twice the camera distance raises the level by exactly one (without
    jitter); a distance of 2^m / k gives level m (float64 log2 cross-check)."""
    p, nrm = _verts(5000, 2)
    par = _params(jitter=False)
    d = O.camera_distance(*CAM, p[:, 0], p[:, 1], p[:, 2])
    a, b = _keys(par, p, nrm), _keys(par, p, nrm, dist=(2 * d).astype(np.float32))
    free = (a.lod > par.lod_min) & (a.lod + 1 < par.lod_max)
    assert free.mean() > 0.99 and np.array_equal(b.lod[free], a.lod[free] + 1)
    k = float(O.footprint_scale(par))
    rng = np.random.default_rng(3)
    m = rng.integers(-6, 8, 5000)
    dist = (rng.uniform(1.05, 1.95, 5000) * 2.0 ** m / k).astype(np.float32)
    c = _keys(par, p, nrm, dist=dist)
    ref = np.array([math.floor(math.log2(k * float(x))) for x in dist])
    assert np.array_equal(c.lod0, ref)


def test_extra_word_is_hashed_last_into_both_hashes():
    """Against the library MurmurHash3: home = hash(X, Y, Z, L, NQ, E) and
    fingerprint = hash2(X, Y, Z, L, NQ, E), E the extra word."""
    sk = pytest.importorskip("sklearn.utils")
    p, nrm = _verts(300, 4)
    par = _params()
    ex = np.random.default_rng(5).integers(0, 2 ** 32, 300, dtype=np.uint64).astype(np.uint32)
    kk = _keys(O.KeyParams(**{**par.__dict__, "log2_slots": 32}), p, nrm, extra=ex)
    for j in range(300):
        nq = int(kk.nq[j, 0]) | (int(kk.nq[j, 1]) << 8) | (int(kk.nq[j, 2]) << 16)
        words = [int(x) & 0xFFFFFFFF for x in kk.xq[j]] + [int(kk.lod[j]) & 0xFFFFFFFF, nq, int(ex[j])]
        msg = np.array(words, dtype="<u4").tobytes()
        assert int(kk.home[j]) == sk.murmurhash3_32(msg, seed=par.hash_seed_home, positive=True)
        f = sk.murmurhash3_32(msg, seed=par.hash_seed_fp, positive=True)
        assert int(kk.fp[j]) == (f if f else 1)


def test_extra_word_splits_cells():
    """Cells are the groups of equal (tuple, extra word), counted by a plain
    dictionary over the vertices."""
    rng = np.random.default_rng(6)
    # a small cloud ~12 units from the camera (voxel edge 2^-5) with two normals
    p = (rng.normal(0, 0.05, (4000, 3)) + np.array([0.5, 2.0, 5.0])).astype(np.float32)
    nrm = np.array([[0, 1, 0], [0.6, 0.8, 0]], dtype=np.float32)[rng.integers(0, 2, 4000)]
    ex = rng.integers(0, 3, 4000).astype(np.uint32)
    rgb = np.ones((4000, 3), dtype=np.float32)
    v = {"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "nx": nrm[:, 0], "ny": nrm[:, 1],
         "nz": nrm[:, 2], "r": rgb[:, 0], "g": rgb[:, 1], "b": rgb[:, 2], "extra": ex}
    fr = O.filter_frame(_params(jitter=False), CAM, 0, v)
    k = _keys(_params(jitter=False), p, nrm)
    groups = {}
    for j in range(4000):
        key = (tuple(k.xq[j]), int(k.lod[j]), tuple(k.nq[j]), int(ex[j]))
        groups[key] = groups.get(key, 0) + 1
    ref = np.array([groups[(tuple(k.xq[j]), int(k.lod[j]), tuple(k.nq[j]), int(ex[j]))]
                    for j in range(4000)])
    assert np.array_equal(fr.count, ref)
    assert fr.tuples.shape[0] == len(groups) and fr.count.max() > 3
