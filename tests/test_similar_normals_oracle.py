"""Pins of the oracle's similar-normal search (Sec. 3.2.2), no GPU: brute force
over all vertex pairs on tiny inputs, the plain lookup at radius 0, the whole
voxel at radius 255, and the count-weighted form for blended values."""
import numpy as np
import pytest

from oracle import pps_oracle as O


def _frame(seed, n=400):
    """Vertices in a handful of voxels with normals scattered around a few
    directions, so that one voxel holds several quantized normals."""
    rng = np.random.default_rng(seed)
    centers = np.array([[0.31, 0.02, 4.1], [0.33, 0.02, 4.1], [2.5, 0.9, 6.0], [-1.2, 0.4, 5.0]])
    base = np.array([[0.0, 1.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.6, -0.8]])
    c = centers[rng.integers(0, len(centers), n)] + rng.uniform(-1e-4, 1e-4, (n, 3))
    nb = base[rng.integers(0, len(base), n)] + rng.normal(0, 0.03, (n, 3))
    nb /= np.linalg.norm(nb, axis=1, keepdims=True)
    rgb = rng.lognormal(-1, 1.0, (n, 3))
    v = {k: a.astype(np.float32) for k, a in zip(
        ("px", "py", "pz", "nx", "ny", "nz", "r", "g", "b"),
        (c[:, 0], c[:, 1], c[:, 2], nb[:, 0], nb[:, 1], nb[:, 2], rgb[:, 0], rgb[:, 1], rgb[:, 2]))}
    kp = O.KeyParams(log2_slots=12, max_probes=16, voxel_scale=64.0, pixel_angle=0.002, jitter=False)
    return O.filter_frame(kp, (0.0, 1.0, -3.0), 0, v), v


def _brute(fr, v, radius):
    """For every vertex, the members of every vertex k in its voxel whose
    quantized normal is within `radius` steps on every axis, summed directly."""
    t = fr.keys.tuples()
    rgb = np.column_stack([v[c].astype(np.float64) for c in "rgb"])
    fx = O.to_fixed(np.column_stack([v[c] for c in "rgb"]))
    same = (t[:, None, :4] == t[None, :, :4]).all(axis=2)
    near = np.abs(t[:, None, 4:7] - t[None, :, 4:7]).max(axis=2) <= radius
    m = same & near
    cnt = m.sum(axis=1)
    return (m.astype(np.float64) @ rgb) / cnt[:, None], m.astype(np.int64) @ fx, cnt


@pytest.mark.parametrize("radius", [0, 1, 3, 8, 255])
def test_similar_normals_match_brute_force(radius):
    fr, v = _frame(radius + 1)
    assert fr.tuples.shape[0] > 20  # several cells ...
    vox = np.unique(fr.tuples[:, :4], axis=0).shape[0]
    assert vox < fr.tuples.shape[0]  # ... with several normals per voxel
    val, vfx, cnt = O.similar_normals(fr, radius)
    ref, sfx, rc = _brute(fr, v, radius)
    assert np.array_equal(cnt, rc)
    assert np.allclose(val, ref, rtol=1e-12, atol=0)
    assert np.array_equal(vfx, O.fixed_mean_f32(sfx, rc))


def test_radius_zero_is_the_plain_lookup_and_255_the_whole_voxel():
    fr, v = _frame(11)
    val, vfx, cnt = O.similar_normals(fr, 0)
    assert np.array_equal(cnt, fr.count)
    assert np.array_equal(vfx, fr.mean_fixed)
    val, _, cnt = O.similar_normals(fr, 255)
    t = fr.keys.tuples()
    _, inv, vc = np.unique(t[:, :4], axis=0, return_inverse=True, return_counts=True)
    assert np.array_equal(cnt, vc[inv.reshape(-1)])
    # a wider radius never pools fewer vertices
    c1 = O.similar_normals(fr, 1)[2]
    c4 = O.similar_normals(fr, 4)[2]
    assert np.all(fr.count <= c1) and np.all(c1 <= c4) and np.all(c4 <= cnt)


def test_blended_values_are_pooled_by_their_counts():
    fr, v = _frame(12)
    rng = np.random.default_rng(3)
    C = fr.tuples.shape[0]
    cval = rng.uniform(0.1, 2.0, (C, 3))
    N = rng.integers(1, 30, C)
    val, vfx, cnt = O.similar_normals(fr, 3, cell_value=cval, cell_weight=N)
    assert vfx is None
    t = fr.tuples
    for j in range(0, fr.cell.shape[0], 37):
        c = fr.cell[j]
        sel = (t[:, :4] == t[c, :4]).all(axis=1) & (np.abs(t[:, 4:7] - t[c, 4:7]).max(axis=1) <= 3)
        assert cnt[j] == N[sel].sum()
        assert np.allclose(val[j], (cval[sel] * N[sel, None]).sum(0) / N[sel].sum(), rtol=1e-12)
