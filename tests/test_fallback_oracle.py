"""Pins of the oracle's low-density fallbacks (no GPU): multi-level
accumulation (Sec. 3.3.2) and neighborhood search (Sec. 3.3.1).

The pins do not reuse the oracle's grouping: brute-force loops over tiny
inputs compute levels with float64 logarithms and cells with float64 floors,
and closed forms cover the constant field, the threshold that switches the
fallbacks off and the weighting of blended values."""
import math

import numpy as np

from oracle import pps_oracle as O

CAM = (0.0, 0.0, 0.0)


def _shell(n, k, a, rng, sigma=1.0):
    """Six clusters of points at distance 1.5 * 2^a / k from the camera, so
    that the footprint k * d stays inside [1.2, 1.8] * 2^a (floor(log2(k d))
    = a, and a + 1 for 2k, far from any rounding boundary); each cluster is a
    Gaussian of `sigma` voxel edges (2^a) so that cells hold a few vertices."""
    dirs = rng.normal(size=(6, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    centers = dirs * (1.5 * 2.0 ** a / k)
    pts = centers[rng.integers(0, 6, n)] + rng.normal(0, sigma * 2.0 ** a, (n, 3))
    return pts.astype(np.float32)


def _normals(n, rng):
    """A few distinct unit normals, so that the quantized normal splits cells."""
    pool = np.array([[0, 1, 0], [0.6, 0.8, 0], [0, 0, -1]], dtype=np.float32)
    return pool[rng.integers(0, 3, n)]


def _verts(p, nrm, rgb):
    return {"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "nx": nrm[:, 0], "ny": nrm[:, 1],
            "nz": nrm[:, 2], "r": rgb[:, 0], "g": rgb[:, 1], "b": rgb[:, 2]}


def _params(jitter=False, scale=2.0):
    return O.KeyParams(log2_slots=12, max_probes=16, voxel_scale=scale, pixel_angle=0.002,
                       jitter=jitter)


def _brute_cells(p, nrm, k, rgb):
    """Cells by float64 arithmetic: l = floor(log2(k d)), x~ = floor(x / 2^l),
    q(n) = floor((n + 1) 128) -> {key: [vertex indices]}."""
    cells = {}
    for j in range(p.shape[0]):
        d = math.sqrt(sum(float(c) ** 2 for c in p[j]))
        l = math.floor(math.log2(k * d))
        x = tuple(math.floor(float(c) / 2.0 ** l) for c in p[j])
        q = tuple(min(255, max(0, math.floor((float(c) + 1.0) * 128.0))) for c in nrm[j])
        cells.setdefault((x, l, q), []).append(j)
    return cells


def test_coarse_params_raise_every_level_by_one():
    rng = np.random.default_rng(1)
    p = (rng.normal(size=(4000, 3)) * 30).astype(np.float32)
    nrm = rng.normal(size=(4000, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    fine = _params(jitter=True)
    coarse = O.coarse_params(fine)
    kf = O.vertex_keys(fine, CAM, 3, *(p[:, i] for i in range(3)), *(nrm[:, i] for i in range(3)))
    kc = O.vertex_keys(coarse, CAM, 3, *(p[:, i] for i in range(3)), *(nrm[:, i] for i in range(3)))
    free = (kf.lod0 > fine.lod_min) & (kf.lod0 + 1 < fine.lod_max)
    assert free.mean() > 0.99
    assert np.array_equal(kc.lod0[free], kf.lod0[free] + 1)
    # same jitter draw, twice the offset: x'_c - x = 2 (x'_f - x) up to one rounding of each sum
    off_f = kf.xj.astype(np.float64) - p
    off_c = kc.xj.astype(np.float64) - p
    tol = 2.0 * np.spacing(np.abs(p).max(axis=1, keepdims=True).astype(np.float32))
    assert np.all(np.abs(off_c - 2.0 * off_f) <= 3 * tol)
    # without jitter the coarse cell is the parent of the fine cell
    fine0 = _params(jitter=False)
    k0 = O.vertex_keys(fine0, CAM, 3, *(p[:, i] for i in range(3)), *(nrm[:, i] for i in range(3)))
    k1 = O.vertex_keys(O.coarse_params(fine0), CAM, 3, *(p[:, i] for i in range(3)),
                       *(nrm[:, i] for i in range(3)))
    free = (k0.lod > fine0.lod_min) & (k0.lod + 1 < fine0.lod_max)
    assert np.array_equal(k1.lod[free], k0.lod[free] + 1)
    assert np.array_equal(k1.xq[free], np.floor_divide(k0.xq[free], 2))


def test_multilevel_matches_brute_force():
    rng = np.random.default_rng(2)
    par = _params(jitter=False)
    k = float(O.footprint_scale(par))
    p = _shell(400, k, 1, rng, sigma=0.4)
    nrm = _normals(400, rng)
    rgb = rng.lognormal(-1, 1.5, (400, 3)).astype(np.float32)
    v = _verts(p, nrm, rgb)
    fine = O.filter_frame(par, CAM, 0, v)
    coarse = O.filter_frame(O.coarse_params(par), CAM, 0, v)
    val, cnt, st = O.multilevel_select(fine.mean64, fine.count, coarse.mean64, coarse.count, 4)
    bf_f = _brute_cells(p, nrm, k, rgb)
    bf_c = _brute_cells(p, nrm, 2 * k, rgb)
    mean_of = {}
    for cells in (bf_f, bf_c):
        for key, js in cells.items():
            for j in js:
                mean_of.setdefault(j, []).append((len(js), rgb[js].astype(np.float64).mean(axis=0)))
    n_low = 0
    for j in range(400):
        (nf, mf), (nc, mc) = mean_of[j]
        assert nc >= nf  # the coarse cell contains the fine one
        if nf < 4:
            n_low += 1
            assert st[j] == O.STATUS_COARSE and cnt[j] == nc
            assert np.allclose(val[j], mc, rtol=1e-12)
        else:
            assert st[j] == O.STATUS_OK and cnt[j] == nf
            assert np.allclose(val[j], mf, rtol=1e-12)
    assert 20 < n_low < 380


def test_neighborhood_matches_brute_force():
    rng = np.random.default_rng(3)
    par = _params(jitter=False)
    k = float(O.footprint_scale(par))
    p = _shell(500, k, 0, rng, sigma=0.7)
    nrm = _normals(500, rng)
    rgb = rng.lognormal(-1, 1.5, (500, 3)).astype(np.float32)
    fr = O.filter_frame(par, CAM, 0, _verts(p, nrm, rgb))
    val, valfx, cnt, st = O.neighborhood(fr, 3)
    cells = _brute_cells(p, nrm, k, rgb)
    n_low = 0
    for (x, l, q), js in cells.items():
        for j in js:
            if len(js) >= 3:
                assert st[j] == O.STATUS_OK and cnt[j] == len(js)
                continue
            n_low += 1
            pool = []
            for (x2, l2, q2), js2 in cells.items():
                if l2 == l and q2 == q and all(abs(a - b) <= 1 for a, b in zip(x, x2)):
                    pool += js2
            assert st[j] == O.STATUS_NEIGHBORS and cnt[j] == len(pool)
            assert np.allclose(val[j], rgb[pool].astype(np.float64).mean(axis=0), rtol=1e-12)
            # fixed point: exact integer sums, one FP32 division
            s = sum(int(O.to_fixed(rgb[i:i + 1])[0, 0]) for i in pool)
            ref = np.float32(np.float32(float(s)) * np.float32(2.0 ** -24)) / np.float32(len(pool))
            assert valfx[j, 0] == ref
    assert 20 < n_low < 480


def test_fallbacks_keep_a_constant_field_and_switch_off_at_zero():
    rng = np.random.default_rng(4)
    par = _params(jitter=True)
    p = (rng.normal(size=(3000, 3)) * 20).astype(np.float32)
    nrm = _normals(3000, rng)
    rgb = np.full((3000, 3), 0.75, dtype=np.float32)
    v = _verts(p, nrm, rgb)
    fine = O.filter_frame(par, CAM, 1, v)
    coarse = O.filter_frame(O.coarse_params(par), CAM, 1, v)
    val, cnt, st = O.multilevel_select(fine.mean64, fine.count, coarse.mean64, coarse.count, 4)
    assert np.all(val == 0.75) and (st == O.STATUS_COARSE).any()
    val, valfx, cnt, st = O.neighborhood(fine, 4)
    assert np.all(val == 0.75) and np.all(valfx == np.float32(0.75))
    assert (st == O.STATUS_NEIGHBORS).any()
    # threshold 0: nothing is low, both fallbacks return the plain filter
    val, cnt, st = O.multilevel_select(fine.mean64, fine.count, coarse.mean64, coarse.count, 0)
    assert np.array_equal(val, fine.mean64) and not st.any()
    val, valfx, cnt, st = O.neighborhood(fine, 0)
    assert np.array_equal(val, fine.mean64) and np.array_equal(valfx, fine.mean_fixed)
    assert np.array_equal(cnt, fine.count) and not st.any()


def test_neighborhood_weights_blended_values_by_their_counts():
    """Three cells in a row at one level and normal, blended values c and
    counts N: a low cell's pooled value is sum(N c) / sum(N) over the block."""
    rng = np.random.default_rng(5)
    par = _params(jitter=False)
    k = float(O.footprint_scale(par))
    # one vertex per cell, cells x~ = (0, 0, 0), (1, 0, 0), (3, 0, 0) at level l
    d = 1.5 / k
    l = math.floor(math.log2(k * d))
    e = 2.0 ** l
    # points on the camera's +z axis at distance ~d, offset in x by whole voxels
    base = np.array([0.25 * e, 0.25 * e, d], dtype=np.float64)
    base[2] = (math.floor(d / e) + 0.5) * e
    pts = np.array([base, base + [e, 0, 0], base + [3 * e, 0, 0]], dtype=np.float32)
    nrm = np.tile(np.array([[0, 1, 0]], dtype=np.float32), (3, 1))
    rgb = rng.uniform(0.1, 1.0, (3, 3)).astype(np.float32)
    fr = O.filter_frame(par, CAM, 0, _verts(pts, nrm, rgb))
    assert fr.tuples.shape[0] == 3 and len(set(fr.tuples[:, 3])) == 1
    c = np.array([[1.0, 2.0, 3.0], [5.0, 7.0, 11.0], [13.0, 17.0, 19.0]])
    N = np.array([2, 6, 1])
    order = fr.cell  # vertex j lives in cell fr.cell[j]
    cv = np.zeros((3, 3))
    cw = np.zeros(3, dtype=np.int64)
    cv[order] = c
    cw[order] = N
    val, _, cnt, st = O.neighborhood(fr, 4, cell_value=cv, cell_weight=cw)
    # vertex 0 (x~ 0, N 2) pools cells x~ 0 and 1; vertex 1 (N 6) is not low;
    # vertex 2 (x~ 3, N 1) finds no neighbour (x~ 2 and 4 are empty)
    assert np.allclose(val[0], (2 * c[0] + 6 * c[1]) / 8, rtol=1e-15) and cnt[0] == 8
    assert np.array_equal(val[1], c[1]) and cnt[1] == 6
    assert np.allclose(val[2], c[2], rtol=1e-15) and cnt[2] == 1
    assert list(st) == [O.STATUS_NEIGHBORS, O.STATUS_OK, O.STATUS_NEIGHBORS]


def test_neighborhood_for_a_subset_equals_the_full_search():
    """Searching only for some vertices gives those vertices the same results
    as the search over all of them."""
    rng = np.random.default_rng(23)
    p = (rng.normal(0, 0.3, (3000, 3)) + np.array([0.0, 1.0, 2.0])).astype(np.float32)
    nrm = np.tile(np.array([[0.0, 1.0, 0.0]], dtype=np.float32), (3000, 1))
    rgb = rng.lognormal(-1, 1.0, (3000, 3)).astype(np.float32)
    v = {"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "nx": nrm[:, 0], "ny": nrm[:, 1],
         "nz": nrm[:, 2], "r": rgb[:, 0], "g": rgb[:, 1], "b": rgb[:, 2]}
    par = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=2.0, pixel_angle=0.002,
                      jitter=False, normal_in_home_hash=False)
    fr = O.filter_frame(par, (0.0, 2.0, -6.0), 0, v)
    full = O.neighborhood(fr, 4)
    sub = rng.choice(3000, 700, replace=False)
    part = O.neighborhood(fr, 4, only=sub)
    assert (full[3][sub] == O.STATUS_NEIGHBORS).sum() > 100
    for a, b in zip(full, part):
        assert np.array_equal(a[sub], b[sub])
