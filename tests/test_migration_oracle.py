"""Pins of the oracle's resolution migration across frames (Sec. 3.4.2), no
GPU.  Levels are moved by exactly one with the given-distance key variant
(twice the distance is one level coarser, without jitter), so the migrated
history has a plain definition: the vertices of the earlier frame grouped on
the grid of the later frame's level."""
import numpy as np

from oracle import pps_oracle as O

CAM = (0.0, 2.0, -9.0)


def _params():
    return O.KeyParams(log2_slots=20, max_probes=16, voxel_scale=3.0, pixel_angle=0.0013,
                       jitter=False, normal_in_home_hash=False)


def _cloud(n, seed):
    """A cloud ~10 units from the camera, two normals, lognormal radiance."""
    rng = np.random.default_rng(seed)
    p = (rng.normal(0, 0.06, (n, 3)) + np.array([0.3, 1.0, 1.0])).astype(np.float32)
    nrm = np.array([[0, 1, 0], [0.6, 0.8, 0]], dtype=np.float32)[rng.integers(0, 2, n)]
    rgb = rng.lognormal(-1, 1.0, (n, 3)).astype(np.float32)
    v = {"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "nx": nrm[:, 0], "ny": nrm[:, 1],
         "nz": nrm[:, 2], "r": rgb[:, 0], "g": rgb[:, 1], "b": rgb[:, 2]}
    return v, p, nrm, rgb


def _frame(par, v, dist, frame):
    return O.filter_frame(par, CAM, frame, {**v, "dist": dist})


def _grid_mean(p, nrm, rgb, level, par):
    """Mean radiance and count of the vertices in each cell (floor(x 2^-l),
    l, q(n)) of one level: a plain dictionary over the vertices."""
    inv = np.float32(2.0 ** -level)
    xq = np.floor(p * inv).astype(np.int64)
    nq = np.clip(np.floor((nrm + np.float32(1)) * np.float32(128)), 0, 255).astype(np.int64)
    acc = {}
    for j in range(p.shape[0]):
        k = (*xq[j], level, *nq[j])
        s, c = acc.get(k, (np.zeros(3), 0))
        acc[k] = (s + rgb[j].astype(np.float64), c + 1)
    return acc


def test_sum_down_adds_the_finer_childrens_sums_and_counts():
    """Frame 0 at level l, frame 1 (same vertices) at l + 1: every frame-1
    cell's history is the frame-0 vertices of its coarser voxel pooled, i.e.
    their mean and their count; alpha = 0.25 blends it with frame 1."""
    par = _params()
    v, p, nrm, rgb = _cloud(6000, 1)
    d0 = O.camera_distance(*CAM, p[:, 0], p[:, 1], p[:, 2])
    f0 = _frame(par, v, d0, 0)
    l0 = int(f0.keys.lod[0])
    assert np.all(f0.keys.lod == l0)  # one level for the whole cloud
    hist, _, _ = O.blend(O.History.empty(), f0, 0.25, migrate=True)
    v1, _, _, rgb1 = _cloud(6000, 2)  # new radiance, same points' distribution
    v1 = {**v1, **{k: v[k] for k in ("px", "py", "pz", "nx", "ny", "nz")}}
    f1 = _frame(par, v1, (2 * d0).astype(np.float32), 1)
    assert np.all(f1.keys.lod == l0 + 1)
    _, val, cnt = O.blend(hist, f1, 0.25, migrate=True)
    coarse = _grid_mean(p, nrm, rgb, l0 + 1, par)
    for j in range(0, 6000, 37):
        k = (*f1.keys.xq[j].astype(np.int64), l0 + 1, *f1.keys.nq[j].astype(np.int64))
        s_old, n_old = coarse[k]
        assert cnt[j] == n_old + f1.count[j]
        ref = 0.25 * s_old / n_old + 0.75 * f1.mean64[j]
        assert np.allclose(val[j], ref, rtol=1e-12, atol=0)
    # without migration the coarser cells start afresh
    _, val2, cnt2 = O.blend(hist, f1, 0.25)
    assert np.array_equal(cnt2, f1.count) and np.allclose(val2, f1.mean64, rtol=1e-12)


def test_split_up_passes_the_parent_average_and_an_eighth_of_its_count():
    """Frame 0 at level l + 1, frame 1 at l: a frame-1 cell without finer
    history takes its parent's average, count ceil(N_parent / 8)."""
    par = _params()
    v, p, nrm, rgb = _cloud(6000, 3)
    d0 = O.camera_distance(*CAM, p[:, 0], p[:, 1], p[:, 2])
    f0 = _frame(par, v, (2 * d0).astype(np.float32), 0)
    l1 = int(f0.keys.lod[0])
    hist, _, _ = O.blend(O.History.empty(), f0, -1.0, migrate=True)
    f1 = _frame(par, v, d0, 1)
    assert np.all(f1.keys.lod == l1 - 1)
    _, val, cnt = O.blend(hist, f1, -1.0, migrate=True)
    parent = _grid_mean(p, nrm, rgb, l1, par)
    for j in range(0, 6000, 41):
        xq = f1.keys.xq[j].astype(np.int64)
        k = (*(xq // 2), l1, *f1.keys.nq[j].astype(np.int64))
        s_p, n_p = parent[k]
        n_old = -(-n_p // 8)
        assert cnt[j] == n_old + f1.count[j]
        a = n_old / (n_old + f1.count[j])  # the integrating weight
        ref = a * s_p / n_p + (1 - a) * f1.mean64[j]
        assert np.allclose(val[j], ref, rtol=1e-12, atol=0)


def test_own_history_wins_and_children_win_over_the_parent():
    """Hand-made history: a cell with its own entry ignores its relatives; a
    cell with both finer children and a coarser parent in the history takes
    the children."""
    t = np.array([[4, 6, -2, 3, 10, 20, 30]], dtype=np.int64)  # the frame's one cell
    kids = np.array([[8, 12, -4, 2, 10, 20, 30], [9, 13, -3, 2, 10, 20, 30],
                     [8, 12, -4, 2, 10, 20, 31]], dtype=np.int64)  # last: other normal
    parent = np.array([[2, 3, -1, 4, 10, 20, 30]], dtype=np.int64)
    h = O.History(np.concatenate([kids, parent]), np.array([[1.0, 2, 3], [3, 4, 5], [9, 9, 9],
                                                          [7, 7, 7]]),
                  np.array([1, 3, 5, 16]))
    c, n, found = O.migrated_history(h, t)
    assert found[0] and n[0] == 4 and np.allclose(c[0], [(1 + 9) / 4, (2 + 12) / 4, (3 + 15) / 4])
    c, n, found = O.migrated_history(O.History(parent, np.array([[7.0, 7, 7]]), np.array([17])), t)
    assert found[0] and n[0] == 3 and np.allclose(c[0], 7.0)
    # negative coordinates: the parent of -3 is floor(-3 / 2) = -2
    c, n, found = O.migrated_history(O.History(np.array([[-2, 0, 0, 1, 0, 0, 0]]),
                                               np.array([[5.0, 5, 5]]), np.array([8])),
                                     np.array([[-3, 1, 0, 0, 0, 0, 0]]))
    assert found[0] and n[0] == 1
    # a cell with its own history is not migrated (blend uses it as is)
    fr_t = t
    own = O.History(np.concatenate([t, kids]), np.array([[2.0, 2, 2], [1, 2, 3], [3, 4, 5],
                                                         [9, 9, 9]]), np.array([6, 1, 3, 5]))
    fr = O.FrameResult(None, np.zeros(1, dtype=np.int64), fr_t, np.array([2]),
                       np.array([[4.0, 4, 4]]), None, np.array([2]), np.array([[8.0, 8, 8]]),
                       None, None, None)
    _, val, cnt = O.blend(own, fr, 0.5, migrate=True)
    assert cnt[0] == 8 and np.allclose(val[0], 0.5 * 2 + 0.5 * 4)
