"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test ties one oracle function to something other than itself: published
known-answer vectors, a library routine, a closed form, an invariant, or brute
force on tiny inputs.  A plausible slip in the oracle (a dropped term, a wrong
level, a transposed operand, a wrong rounding) fails at least one of these.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import pps_oracle as O

F32 = np.float32


# --------------------------------------------------------------- Philox / Murmur
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:], row


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 2 ** 32, size=(4, 64), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2 ** 32, size=(2, 64), dtype=np.uint64).astype(np.uint32)
    vec = O.philox4x32_10(c[0], c[1], c[2], c[3], k[0], k[1])
    for j in range(0, 64, 7):
        sc = O.philox4x32_10(c[0, j], c[1, j], c[2, j], c[3, j], k[0, j], k[1, j])
        assert [int(vec[i][j]) for i in range(4)] == [int(x) for x in sc]


def test_murmur3_published_vectors():
    for msg, seed, h in read_golden("murmur3_x86_32_vectors.txt"):
        b = b"" if msg == "-" else bytes.fromhex(msg)
        words = [np.uint32(int.from_bytes(b[i:i + 4], "little")) for i in range(0, len(b), 4)]
        assert int(O.murmur3_32(words, int(seed, 16))) == int(h, 16), (msg, seed)


def test_murmur3_matches_library_on_random_key_words():
    sk = pytest.importorskip("sklearn.utils")
    rng = np.random.default_rng(11)
    for nw in (4, 5):
        W = rng.integers(0, 2 ** 32, size=(200, nw), dtype=np.uint64).astype(np.uint32)
        seed = int(rng.integers(0, 2 ** 32))
        ours = O.murmur3_32([W[:, j] for j in range(nw)], seed)
        for r in range(200):
            ref = sk.murmurhash3_32(W[r].astype("<u4").tobytes(), seed=seed, positive=True)
            assert int(ours[r]) == ref


# --------------------------------------------------------------- conversions
def test_int64_to_f32_rn_matches_exact_double_route():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.integers(-2 ** 52, 2 ** 52, 5000),
                        rng.integers(-2 ** 30, 2 ** 30, 5000),
                        np.array([0, 1, -1, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1, 2 ** 24 + 2,
                                  2 ** 24 + 3, 2 ** 25 + 2, 2 ** 25 + 6])])
    ref = v.astype(np.float64).astype(F32)  # exact double, one rounding to f32
    assert np.array_equal(O.int64_to_f32_rn(v), ref)


def test_int64_to_f32_rn_ties_and_extremes():
    cases = {2 ** 24 + 1: 2 ** 24, 2 ** 24 + 3: 2 ** 24 + 4, 2 ** 25 + 2: 2 ** 25,
             2 ** 25 + 6: 2 ** 25 + 8, 2 ** 62 + 2 ** 38: 2 ** 62,
             2 ** 62 + 2 ** 38 + 1: 2 ** 62 + 2 ** 39, -(2 ** 63): -(2 ** 63),
             2 ** 63 - 1: 2 ** 63}
    for k, want in cases.items():
        assert float(O.int64_to_f32_rn(np.array([k]))[0]) == float(want), k


def test_to_fixed_is_round_to_nearest_of_scaled_value():
    v = np.array([0.75, 1.0, 2.0 ** -24, 1.5 * 2.0 ** -24, 2.5 * 2.0 ** -24, 3.0e-8, 123.456],
                 dtype=F32)
    got = O.to_fixed(v)
    want = [round(float(x) * 2 ** 24) for x in v]  # Python round: half to even
    assert got.tolist() == want


# --------------------------------------------------------------- key pieces
def test_lod_matches_floor_log2_from_frexp():
    rng = np.random.default_rng(7)
    x = rng.uniform(-50, 50, (3, 4000)).astype(F32)
    cam = (F32(1.5), F32(3.0), F32(-12.0))
    k = F32(0.00427)
    l = O.level_of_detail(*cam, x[0], x[1], x[2], k, -24, 24)
    for j in range(0, 4000, 13):
        dx = F32(cam[0]) - x[0, j]
        dy = F32(cam[1]) - x[1, j]
        dz = F32(cam[2]) - x[2, j]
        d = np.sqrt(F32(F32(F32(dx * dx) + F32(dy * dy)) + F32(dz * dz)))
        F = float(F32(k * d))
        m, e = math.frexp(F)  # F = m 2^e, m in [0.5, 1)
        assert l[j] == max(-24, min(24, e - 1))


def test_lod_clamps_zero_distance():
    z = np.zeros(1, dtype=F32)
    assert O.level_of_detail(0, 0, 0, z, z, z, F32(0.01), -24, 24)[0] == -24
    big = np.full(1, 3e38, dtype=F32)
    assert O.level_of_detail(0, 0, 0, big, z, z, F32(10.0), -24, 24)[0] == 24


def _unit_normals(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v = v.astype(F32)
    special = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                        [0, 1, -0.0], [1, 0, -0.0]], dtype=F32)
    return np.concatenate([special, v])


def test_orthonormal_basis_is_right_handed_orthonormal():
    n = _unit_normals(5000, 1)
    t, b = O.orthonormal_basis(n[:, 0], n[:, 1], n[:, 2])
    T = np.column_stack(t).astype(np.float64)
    B = np.column_stack(b).astype(np.float64)
    N = n.astype(np.float64)
    assert np.all(np.isfinite(T)) and np.all(np.isfinite(B))
    tol = 4e-6
    assert np.abs((T * N).sum(1)).max() < tol
    assert np.abs((B * N).sum(1)).max() < tol
    assert np.abs((T * B).sum(1)).max() < tol
    assert np.abs(np.linalg.norm(T, axis=1) - 1).max() < tol
    assert np.abs(np.linalg.norm(B, axis=1) - 1).max() < tol
    assert np.abs(np.cross(T, B) - N).max() < 1e-5  # t x b = n


def test_quantize_normal_special_values():
    c = np.array([-1.0, -0.9999999, 0.0, 0.5, 1.0, 0.99999994, -0.0078125, 1.5, -2.0],
                 dtype=F32)
    want = [0, 0, 128, 192, 255, 255, 127, 255, 0]
    assert O.quantize_normal(c).tolist() == want


def test_jitter_uniform_chi_square():
    ids = np.arange(200000, dtype=np.uint32)
    u, w = O.jitter_uw(ids, 0, 1234, 7)
    assert u.min() >= -0.5 and u.max() < 0.5 and w.min() >= -0.5 and w.max() < 0.5
    for x in (u, w):
        h, _ = np.histogram(x, bins=64, range=(-0.5, 0.5))
        e = ids.size / 64
        chi2 = ((h - e) ** 2 / e).sum()
        assert chi2 < 120  # 63 dof: p ~ 1e-5
    # different frames give independent draws
    u2, _ = O.jitter_uw(ids, 0, 1234, 8)
    assert abs(np.corrcoef(u, u2)[0, 1]) < 0.01


def _cloud(n, seed, spread=20.0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-spread, spread, (n, 3)).astype(F32)
    nn = _unit_normals(n, seed + 1)[:n]
    return p, nn


def test_keys_jitter_in_tangent_plane_and_voxel_contains_point():
    p, n = _cloud(20000, 2)
    kp = O.KeyParams(log2_slots=20, max_probes=16, voxel_scale=4.0, pixel_angle=0.001069)
    cam = (0.0, 3.0, -12.0)
    k = O.vertex_keys(kp, cam, 3, p[:, 0], p[:, 1], p[:, 2], n[:, 0], n[:, 1], n[:, 2])
    off = k.xj.astype(np.float64) - p.astype(np.float64)
    E = np.exp2(k.lod0.astype(np.float64))
    # jitter lies in the tangent plane of n and within half a voxel per tangent axis
    assert np.abs((off * n.astype(np.float64)).sum(1)).max() <= 1e-5 * (E.max() + 1)
    assert np.all(np.linalg.norm(off, axis=1) <= E * math.sqrt(0.5) * (1 + 1e-5) + 1e-5)
    # the voxel at level l' contains the jittered point: x~ 2^l' <= x' < (x~ + 1) 2^l'
    El = np.exp2(k.lod.astype(np.float64))[:, None]
    lo = k.xq.astype(np.float64) * El
    assert np.all(lo <= k.xj) and np.all(k.xj < lo + El)
    # l' is the level at the jittered point, l the level at the original one
    kk = O.footprint_scale(kp)
    assert np.array_equal(O.level_of_detail(*cam, k.xj[:, 0], k.xj[:, 1], k.xj[:, 2], kk, -24, 24),
                          k.lod)
    assert np.array_equal(O.level_of_detail(*cam, p[:, 0], p[:, 1], p[:, 2], kk, -24, 24), k.lod0)
    assert np.any(k.lod != k.lod0)  # the sample crosses level boundaries
    assert np.all(k.fp != 0)
    assert np.all(k.home < (1 << 20))


def test_home_and_fingerprint_are_murmur_of_key_words():
    sk = pytest.importorskip("sklearn.utils")
    p, n = _cloud(50, 4)
    for nih in (False, True):
        kp = O.KeyParams(log2_slots=12, max_probes=16, voxel_scale=4.0, pixel_angle=0.002,
                         normal_in_home_hash=nih)
        k = O.vertex_keys(kp, (0, 3, -12), 0, p[:, 0], p[:, 1], p[:, 2], n[:, 0], n[:, 1],
                          n[:, 2])
        for j in range(50):
            nq = int(k.nq[j, 0]) | int(k.nq[j, 1]) << 8 | int(k.nq[j, 2]) << 16
            words = [int(x) & 0xFFFFFFFF for x in k.xq[j]] + [int(k.lod[j]) & 0xFFFFFFFF]
            hw = words + ([nq] if nih else [])
            msg = lambda ws: b"".join(w.to_bytes(4, "little") for w in ws)
            h1 = sk.murmurhash3_32(msg(hw), seed=kp.hash_seed_home, positive=True)
            h2 = sk.murmurhash3_32(msg(words + [nq]), seed=kp.hash_seed_fp, positive=True)
            assert int(k.home[j]) == h1 & 0xFFF
            assert int(k.fp[j]) == (h2 or 1)


# --------------------------------------------------------------- grouping (Eq. 7)
def _vertices(p, n, rgb):
    return {"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "nx": n[:, 0], "ny": n[:, 1],
            "nz": n[:, 2], "r": rgb[:, 0], "g": rgb[:, 1], "b": rgb[:, 2]}


def test_zero_jitter_constant_level_matches_brute_force_pairs():
    rng = np.random.default_rng(9)
    N = 300
    p = rng.uniform(-3, 3, (N, 3)).astype(F32)
    choices = np.array([[0, 1, 0], [1, 0, 0], [0, 0, -1], [0.6, 0.8, 0]], dtype=F32)
    n = choices[rng.integers(0, 4, N)]
    rgb = rng.lognormal(-1, 1.5, (N, 3)).astype(F32)
    L = -1  # constant resolution s(k): voxel edge 1/2
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=1.0, pixel_angle=0.01,
                     jitter=False, lod_min=L, lod_max=L)
    fr = O.filter_frame(kp, (0, 3, -12), 0, _vertices(p, n, rgb))
    # brute force: chi_V(k, k') = 1 iff floor(x / 2^L) and the normal codes agree
    vox = np.floor(p.astype(np.float64) / 2.0 ** L).astype(np.int64)
    code = np.floor((n.astype(np.float64) + 1.0) * 128.0).clip(0, 255).astype(np.int64)
    for a in range(N):
        same = [b for b in range(N) if np.array_equal(vox[a], vox[b])
                and np.array_equal(code[a], code[b])]
        assert fr.count[a] == len(same)
        assert all(fr.cell[b] == fr.cell[a] for b in same)
        want = rgb[same].astype(np.float64).sum(0) / len(same)
        assert np.allclose(fr.mean64[a], want, rtol=1e-15, atol=0)


def test_counts_sum_to_vertex_count_and_partition():
    p, n = _cloud(5000, 12, spread=5.0)
    rgb = np.random.default_rng(1).lognormal(-1, 1.5, (5000, 3)).astype(F32)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=8.0, pixel_angle=0.002)
    fr = O.filter_frame(kp, (0, 3, -12), 1, _vertices(p, n, rgb))
    assert fr.cell_count.sum() == 5000
    assert np.array_equal(np.bincount(fr.cell), fr.cell_count)
    # transitivity: every vertex's tuple equals its cell's tuple
    assert np.array_equal(fr.tuples[fr.cell], fr.keys.tuples())


@pytest.mark.parametrize("c", [0.75, 0.3])
def test_constant_field_returns_itself(c):
    p, n = _cloud(4000, 13, spread=4.0)
    rgb = np.full((4000, 3), c, dtype=F32)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=4.0, pixel_angle=0.002)
    fr = O.filter_frame(kp, (0, 3, -12), 0, _vertices(p, n, rgb))
    assert np.all(fr.mean64 == np.float64(F32(c)))  # n * c exact for n < 2^29
    if c == 0.75:  # dyadic: exact in fixed point too
        assert np.all(fr.mean_fixed == F32(c))


def test_one_voxel_covering_everything_returns_global_mean():
    rng = np.random.default_rng(14)
    N = 3000
    p = rng.uniform(0, 500, (N, 3)).astype(F32)
    n = np.tile(np.array([[0, 1, 0]], dtype=F32), (N, 1))
    rgb = rng.lognormal(-1, 1.5, (N, 3)).astype(F32)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=1.0, pixel_angle=0.01,
                     jitter=False, lod_min=10, lod_max=10)  # voxel [0, 1024)^3
    fr = O.filter_frame(kp, (0, 3, -12), 0, _vertices(p, n, rgb))
    assert fr.tuples.shape[0] == 1 and np.all(fr.count == N)
    g = rgb.astype(np.float64).mean(0)
    assert np.allclose(fr.mean64, g[None, :], rtol=1e-14)


def test_fixed_point_is_order_free_and_close_to_fp64():
    p, n = _cloud(6000, 15, spread=3.0)
    rgb = np.random.default_rng(2).lognormal(-1, 1.5, (6000, 3)).astype(F32)
    ids = np.arange(6000, dtype=np.uint32)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=16.0, pixel_angle=0.002)
    fr = O.filter_frame(kp, (0, 3, -12), 2, _vertices(p, n, rgb), ids=ids)
    perm = np.random.default_rng(3).permutation(6000)
    vp = _vertices(p[perm], n[perm], rgb[perm])
    fr2 = O.filter_frame(kp, (0, 3, -12), 2, vp, ids=ids[perm])
    assert np.array_equal(fr.tuples, fr2.tuples)
    assert np.array_equal(fr.cell_fixed, fr2.cell_fixed)
    assert np.array_equal(fr.mean_fixed[perm], fr2.mean_fixed)
    # |fixed - fp64| <= n * 2^-25 / n (input rounding) + 2 ulp (two FP32 roundings)
    err = np.abs(fr.mean_fixed.astype(np.float64) - fr.mean64)
    ulp = np.spacing(np.abs(fr.mean_fixed)).astype(np.float64)
    assert np.all(err <= 2.0 ** -25 + 2 * ulp)


# --------------------------------------------------------------- temporal (Sec. 3.4.1)
def _frames(F, N=3000, seed=20):
    p, n = _cloud(N, seed, spread=3.0)
    rng = np.random.default_rng(seed + 5)
    return p, n, [rng.lognormal(-1, 1.5, (N, 3)).astype(F32) for _ in range(F)]


def test_integration_weight_gives_pooled_mean():
    F = 5
    p, n, rgbs = _frames(F)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=8.0, pixel_angle=0.002)
    h = O.History.empty()
    allt, allv = [], []
    for f in range(F):
        fr = O.filter_frame(kp, (0, 3, -12), f, _vertices(p, n, rgbs[f]))
        h, val, cnt = O.blend(h, fr, alpha=-1.0)
        allt.append(fr.keys.tuples())
        allv.append(rgbs[f].astype(np.float64))
    # closed form: the mean of all samples ever accumulated into each tuple
    T = np.concatenate(allt)
    V = np.concatenate(allv)
    uq, inv = np.unique(T, axis=0, return_inverse=True)[:2]
    inv = inv.reshape(-1)
    pooled = np.column_stack([np.bincount(inv, V[:, j]) for j in range(3)]) / \
        np.bincount(inv)[:, None]
    assert np.array_equal(uq, h.tuples)
    assert np.allclose(h.c, pooled, rtol=1e-12)
    assert np.array_equal(h.n, np.bincount(inv))
    last = inv[-p.shape[0]:]
    assert np.allclose(val, pooled[last], rtol=1e-12)


def test_ema_limits_and_constant_invariance():
    F = 3
    p, n, rgbs = _frames(F, seed=30)
    kp = O.KeyParams(log2_slots=16, max_probes=16, voxel_scale=8.0, pixel_angle=0.002)
    h0 = O.History.empty()
    frs = [O.filter_frame(kp, (0, 3, -12), f, _vertices(p, n, rgbs[f])) for f in range(F)]
    h, _, _ = O.blend(h0, frs[0], 0.2)
    h1, v_new, _ = O.blend(h, frs[1], 0.0)  # alpha = 0: only the current frame
    assert np.allclose(v_new, frs[1].mean64, rtol=1e-15)
    h2, v_old, _ = O.blend(h, frs[1], 1.0)  # alpha = 1: cells with history keep it
    idx = {tuple(t): i for i, t in enumerate(h.tuples)}
    for j in range(0, p.shape[0], 37):
        t = tuple(frs[1].tuples[frs[1].cell[j]])
        if t in idx:
            assert np.allclose(v_old[j], h.c[idx[t]])
        else:
            assert np.allclose(v_old[j], frs[1].mean64[j])
    # explicit formula for one cell present in both frames
    common = [j for j in range(p.shape[0]) if tuple(frs[1].tuples[frs[1].cell[j]]) in idx]
    j = common[0]
    _, v, _ = O.blend(h, frs[1], 0.2)
    c_old = h.c[idx[tuple(frs[1].tuples[frs[1].cell[j]])]]
    assert np.allclose(v[j], 0.2 * c_old + 0.8 * frs[1].mean64[j], rtol=1e-15)
    # constant field stays constant under any alpha
    cst = [np.full_like(r, 0.5) for r in rgbs]
    hc = O.History.empty()
    for f in range(F):
        fr = O.filter_frame(kp, (0, 3, -12), f, _vertices(p, n, cst[f]))
        hc, vc, _ = O.blend(hc, fr, 0.37)
        assert np.all(vc == 0.5)


# --------------------------------------------------------------- table audit helpers
def test_ambiguous_cells_window_rule():
    home = np.array([100, 115, 500, 516, 7, 65535], dtype=np.uint32)
    fp = np.array([9, 9, 4, 4, 3, 3], dtype=np.uint32)
    amb = O.ambiguous_cells(home, fp, 16, 16)
    # distance 15 < P overlaps; distance 16 does not; 7 and 65535 wrap (distance 8)
    assert amb.tolist() == [True, True, False, False, True, True]


def test_overflow_window_full():
    t = np.zeros(32, dtype=np.uint32)
    t[30:32] = 5
    t[0:2] = 6
    assert O.overflow_window_full(t, 30, 7, 4)
    assert not O.overflow_window_full(t, 30, 6, 4)  # f present in window
    t[1] = 0
    assert not O.overflow_window_full(t, 30, 7, 4)  # an empty slot in window


def test_linear_probing_mean_probes_match_knuth():
    # Knuth: successful search at load a costs about (1 + 1/(1 - a)) / 2 probes
    rng = np.random.default_rng(17)
    lg = 16
    T = 1 << lg
    for a in (0.3, 0.5):
        m = int(a * T)
        home = rng.integers(0, T, m).astype(np.uint32)
        fp = np.arange(1, m + 1, dtype=np.uint32)
        slot, probes, table = O.simulate_linear_probing(home, fp, lg, T)
        want = 0.5 * (1 + 1 / (1 - a))
        assert abs(probes.mean() - want) < 0.05 * want
        assert np.all(slot >= 0) and (table != 0).sum() == m


def test_fingerprint_collisions_follow_the_birthday_bound():
    """hash2 behaves like a random 32-bit function on distinct key tuples:
    among m distinct keys the number of colliding pairs has mean
    m (m - 1) / 2 / 2^32 (Poisson), here 116.4 for m = 10^6."""
    rng = np.random.default_rng(23)
    m = 1_000_000
    words = rng.integers(0, 2 ** 32, size=(4, 3 * m // 2), dtype=np.uint64).astype(np.uint32)
    t = np.unique(words.T, axis=0)[:m].T  # distinct 4-word keys
    assert t.shape[1] == m
    f = O.murmur3_32([t[0], t[1], t[2], t[3]], 0x2F0F1D3B)
    _, c = np.unique(f, return_counts=True)
    pairs = int((c * (c - 1) // 2).sum())
    mean = m * (m - 1) / 2 / 2 ** 32
    assert abs(pairs - mean) < 5 * np.sqrt(mean), (pairs, mean)


def _one_cell_frame(tuple7, c_new, n_new):
    """A frame of one cell (one vertex per member) with average c_new."""
    return O.FrameResult(None, np.zeros(n_new, dtype=np.int64), np.array([tuple7], dtype=np.int64),
                         np.full(n_new, n_new), np.tile(c_new, (n_new, 1)), None,
                         np.array([n_new]), np.array([np.array(c_new) * n_new]), None, None, None)


def test_fp16_history_rounds_to_binary16():
    """FP16 history (Sec. 3.4.1 with half-precision storage): the stored and
    returned value is the binary16 nearest to the blend.  0.1 = 1.6 * 2^-4 and
    1.6 * 1024 = 1638.4 rounds to 1638, so binary16(0.1) = 1638 / 1024 * 2^-4 =
    0.0999755859375; 0.75 is representable and survives every frame exactly."""
    t = (1, 2, 3, 4, 5, 6, 7)
    hist, val, _ = O.blend(O.History.empty(), _one_cell_frame(t, [0.1, 0.75, 2.0], 3), 0.2,
                           fp16=True)
    assert val[0, 0] == 0.0999755859375 and val[0, 1] == 0.75 and val[0, 2] == 2.0
    for _ in range(5):
        hist, val, _ = O.blend(hist, _one_cell_frame(t, [0.1, 0.75, 2.0], 3), 0.2, fp16=True)
        assert val[0, 1] == 0.75 and val[0, 2] == 2.0
        assert abs(val[0, 0] - 0.1) <= 2.0 ** -14  # within half a binary16 step at 0.1


def test_count_cap_saturates_but_weight_uses_true_counts():
    """N = N_old + N_new saturates at the cap (65535 for a 16-bit count) while
    the integrating weight alpha = N_old / (N_old + N_new) uses the counts
    before the cap."""
    t = (0, 0, 0, 1, 2, 3, 4)
    hist = O.History(np.array([t], dtype=np.int64), np.array([[1.0, 1.0, 1.0]]), np.array([65000]))
    hist2, val, cnt = O.blend(hist, _one_cell_frame(t, [2.0, 2.0, 2.0], 1000), -1.0,
                              n_cap=65535)
    a = 65000 / 66000
    assert cnt[0] == 65535 and hist2.n[0] == 65535
    assert np.allclose(val[0], a * 1.0 + (1 - a) * 2.0, rtol=1e-15)


def test_pow2_matches_ldexp_over_the_normal_range():
    """2^l built from the exponent bits equals the library's ldexp for every
    integer l of the normal FP32 range."""
    ls = np.arange(-126, 128)
    assert np.array_equal(O.pow2_f32(ls), np.ldexp(np.float32(1), ls).astype(np.float32))


def test_level_at_a_given_distance_matches_frexp():
    """floor(log2(k d)) for given distances, against the library's frexp of the
    FP32 product (frexp returns e with 2^(e-1) <= x < 2^e), and clamped."""
    rng = np.random.default_rng(17)
    d = (rng.uniform(0.5, 1.0, 4000) * 2.0 ** rng.integers(-20, 30, 4000)).astype(np.float32)
    k = np.float32(0.0039)
    F = (k * d).astype(np.float32)
    ref = np.clip(np.frexp(F)[1] - 1, -24, 24)
    assert np.array_equal(O.level_of_detail_at(d, k, -24, 24), ref)


def test_fixed_point_mean_of_dyadic_values_is_exact():
    """Fixed-point sums of a dyadic value c (c 2^24 an integer) are exact, so
    the average fl32(fl32(sum) 2^-24) / fl32(n) is c itself for any count."""
    for c in (0.75, 3.5, 0.0009765625):
        for n in (1, 3, 1000, 12345):
            s = np.array([[round(c * 2 ** 24) * n] * 3], dtype=np.int64)
            assert np.all(O.fixed_mean_f32(s, np.array([n])) == np.float32(c)), (c, n)


def test_pixel_angle_closed_forms():
    """theta_px = 2 tan(fov_y / 2) / height: tan 30 deg = 1 / sqrt 3 and
    tan 45 deg = 1 give closed forms; the vertical field of view pairs with
    the image height (a width, or a slip between degrees and radians, moves
    the value by a large factor)."""
    assert math.isclose(O.pixel_angle(60.0, 1080), 2.0 / (math.sqrt(3.0) * 1080), rel_tol=1e-15)
    assert math.isclose(O.pixel_angle(90.0, 512), 2.0 / 512, rel_tol=1e-15)
    assert math.isclose(O.pixel_angle(60.0, 256), 2.0 / (math.sqrt(3.0) * 256), rel_tol=1e-15)
    # the angle between the rays through the top and bottom edges of the
    # central pixel row, 2 atan(tan(fov / 2) / H), is theta_px up to the
    # small-angle term theta^2 / 12
    for fov, h in [(60.0, 1080), (60.0, 720), (45.0, 2160)]:
        th = O.pixel_angle(fov, h)
        edge = 2.0 * math.atan(math.tan(math.radians(fov) / 2.0) / h)
        assert abs(edge - th) <= th ** 3 / 12 * 1.01 + 1e-18
