"""CPU oracle for hashed path space filtering (Binder, Fricke, Keller 2019).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only the tests, the package's smoke check and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA library
and imports nothing from the package.

What it computes, and from which passage
----------------------------------------
* Key construction (Algorithm 1, Sec. 3.1.4 jittering in the tangent plane,
  Sec. 3.1.2 key components position + normal): level of detail from the
  camera distance, a tangent-plane jitter scaled by the voxel edge of that
  level, a second level of detail at the jittered point, the quantized
  position, and the two hashes: the home index i = hash(x~, ...) mod T and the
  32-bit fingerprint f = hash2(x~, n, ...) with the sentinel 0 excluded
  (Sec. 3.2, Sec. 3.2.1).
* Voxel membership (Eq. 7, with the transitivity argument right after it):
  two vertices share a cell iff their full quantized tuples are equal.  The
  oracle therefore groups vertices by the tuple (x~x, x~y, x~z, l', qx, qy, qz)
  in an ordered (sorted) map, which is the "gather per voxel" form that opens
  Sec. 3.2, and averages with weight w = 1 (Eq. 8/9): the cell value is the sum
  of the members' contributions divided by their count.  This is the plain
  definition the GPU's scatter form (atomic sums and counters, Sec. 3.2 and
  Sec. 3.3.1) reaches up to summation order.
* Temporal blending (Sec. 3.4.1): c = alpha c_old + (1 - alpha) c_new, or the
  integrating weight alpha = N_old / (N_old + N_new).
* Changes in resolution across frames (Sec. 3.4.2): a cell without history
  of its own adds up the sums and counts of its eight finer children, or else
  takes its coarser parent's average with the parent's count shared among
  eight children.
* Overflow audit (Sec. 3.2: the probe limit, after which a vertex keeps its
  own unfiltered contribution): a helper that checks a table dump.
* History eviction (Sec. 3.4.3): a sequential model of a history table whose
  fingerprint words carry a priority (the frame of last use) in their top
  bits, so that a cell without room replaces the least recently used entry
  of its probe window.
* Searching similar normals by linear probing (Sec. 3.2.2): with the normal
  only in the fingerprint, a lookup pools the cells of its voxel whose
  quantized normal lies within a given number of steps of its own.
* Fallbacks for cells with few vertices (Sec. 3.3.1 neighborhood search,
  Sec. 3.3.2 multi-level accumulation): the pooled average of the 3x3x3
  block of cells around a vertex's cell, and the average of the next coarser
  resolution, both taken only where the vertex's own cell has fewer than a
  threshold of members.

Readings where the paper is silent:
* LOD: l(d) = floor(log2(s * theta_px * d)) read from the exponent bits of the
  FP32 product, clamped to [lod_min, lod_max]; the voxel edge is 2^l, i.e. the
  "s * 2^l" of Algorithm 1 with the projected-pixel footprint folded in, so the
  voxel is always a power of two (Sec. 3.1.1 and Sec. 4).
* Jitter: (u, w) in [-0.5, 0.5) from Philox4x32-10 (Salmon et al., SC'11) keyed
  by (seed, frame), counter (vertex id, stream id, 0, 0); tangent frame from
  Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 2017).
* Hashes: MurmurHash3_x86_32 (Appleby) over the key's 32-bit words, with two
  different seeds for hash and hash2.
* Normal quantization: q(c) = clamp(floor((c + 1) * 128), 0, 255).
* All key arithmetic is FP32 with round-to-nearest-even per operation, in the
  order written below (numpy never fuses multiply-add), so the integer keys are
  reproducible bit for bit.

Sums are FP64 (the reference value) and, separately, fixed point
(round-to-nearest of v * 2^24 into int64), which is exact and order-free.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

F32 = np.float32
U32 = np.uint32
MASK32 = np.uint64(0xFFFFFFFF)

# ----------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy
# as 1, 2, 3", SC'11): a 10-round counter-based generator.  Each round takes
# two 32x32->64 products of counter words with fixed multipliers, swaps and
# xors the halves with the key, and the key is bumped by two Weyl constants
# between rounds.
# ----------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds; all arguments uint32 arrays (broadcastable)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(U32) for x in (c0, c1, c2, c3))


# ----------------------------------------------------------------------------
# MurmurHash3_x86_32 (Austin Appleby, public-domain reference algorithm) over
# a message made of whole little-endian 32-bit words, so there is no tail.
# ----------------------------------------------------------------------------
_MM_C1 = np.uint64(0xCC9E2D51)
_MM_C2 = np.uint64(0x1B873593)


def _rotl32(x, r):
    return ((x << np.uint64(r)) | (x >> np.uint64(32 - r))) & MASK32


def murmur3_32(words: Sequence, seed: int) -> np.ndarray:
    """MurmurHash3_x86_32 of the words (each a uint32 array) with `seed`."""
    words = [np.asarray(w).astype(np.uint64) & MASK32 for w in words]
    shape = np.broadcast(*words).shape if words else ()
    h = np.zeros(shape, dtype=np.uint64) + np.uint64(seed & 0xFFFFFFFF)
    for k in words:
        k = (k * _MM_C1) & MASK32
        k = _rotl32(k, 15)
        k = (k * _MM_C2) & MASK32
        h = h ^ k
        h = _rotl32(h, 13)
        h = (h * np.uint64(5) + np.uint64(0xE6546B64)) & MASK32
    h = h ^ np.uint64(4 * len(words))
    h = h ^ (h >> np.uint64(16))
    h = (h * np.uint64(0x85EBCA6B)) & MASK32
    h = h ^ (h >> np.uint64(13))
    h = (h * np.uint64(0xC2B2AE35)) & MASK32
    h = h ^ (h >> np.uint64(16))
    return h.astype(U32)


# ----------------------------------------------------------------------------
# Key construction, Algorithm 1.
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class KeyParams:
    """Parameters of key construction and of the table (Alg. 1, Sec. 3.2)."""

    log2_slots: int
    max_probes: int
    voxel_scale: float  # s: voxel edge in multiples of the projected pixel (Sec. 4)
    pixel_angle: float  # theta_px = 2 tan(fov_y / 2) / height
    jitter: bool = True
    seed: int = 0x0051F15E
    hash_seed_home: int = 0x9747B28C
    hash_seed_fp: int = 0x2F0F1D3B
    normal_in_home_hash: bool = False
    lod_min: int = -24
    lod_max: int = 24


def pixel_angle(fov_y_deg: float, height: int) -> float:
    """theta_px: the height of one pixel's footprint at unit distance from a
    pinhole camera, 2 tan(fov_y / 2) / height (fov_y the vertical field of
    view in degrees, height the image height in pixels), in FP64.  Sec. 4
    sizes voxels as s times "the projected size of a pixel"; with square
    pixels the vertical extent fixes it."""
    import math
    return 2.0 * math.tan(math.radians(float(fov_y_deg)) / 2.0) / float(height)


def pow2_f32(l) -> np.ndarray:
    """2^l as float32, exact for integer l in [-126, 127] (built from the bits)."""
    l = np.asarray(l, dtype=np.int64)
    return ((l + 127) << 23).astype(U32).view(F32)


def footprint_scale(p: KeyParams) -> np.float32:
    """k = fl32(s * theta_px): world size of the voxel at unit distance."""
    return F32(p.voxel_scale) * F32(p.pixel_angle)


def level_of_detail(cx, cy, cz, x, y, z, k, lod_min, lod_max) -> np.ndarray:
    """Alg. 1 level_of_detail(|p_cam - x|) = floor(log2(k * d)), clamped.

    d = sqrt(((dx*dx) + (dy*dy)) + (dz*dz)) with d = p_cam - x, each FP32 op
    rounded to nearest; floor(log2 F) of the positive FP32 F = k * d is its
    unbiased exponent field (0 and subnormals read as -127 and clamp to
    lod_min; inf/NaN read as 128 and clamp to lod_max)."""
    # FP32 overflow to inf is part of the definition (it reads as level 128)
    with np.errstate(over="ignore"):
        dx = F32(cx) - x
        dy = F32(cy) - y
        dz = F32(cz) - z
        d2 = (dx * dx + dy * dy) + dz * dz
        d = np.sqrt(d2)
        F = F32(k) * d
    e = ((F.view(U32) >> U32(23)) & U32(0xFF)).astype(np.int32) - 127
    return np.clip(e, lod_min, lod_max).astype(np.int32)


def orthonormal_basis(nx, ny, nz):
    """Tangent frame (t, b) of a unit normal n, after Duff et al. (JCGT 2017).

    s = sign(nz) (copysign, so -0 gives -1); a = -1 / (s + nz);
    q = (nx * ny) * a;  t = (1 + s*((nx*nx)*a), s*q, -(s*nx));
    b = (q, s + (ny*ny)*a, -ny)."""
    s = np.copysign(F32(1.0), nz).astype(F32)
    a = F32(-1.0) / (s + nz)
    q = (nx * ny) * a
    tx = F32(1.0) + s * ((nx * nx) * a)
    ty = s * q
    tz = -(s * nx)
    bx = q
    by = s + (ny * ny) * a
    bz = -ny
    return (tx, ty, tz), (bx, by, bz)


def jitter_uw(ids, stream, seed, frame):
    """(u, w) in [-0.5, 0.5): top 24 bits of the first two Philox words."""
    ids = np.asarray(ids, dtype=U32)
    zero = np.zeros_like(ids)
    x0, x1, _, _ = philox4x32_10(ids, np.full_like(ids, stream), zero, zero,
                                 np.full_like(ids, seed), np.full_like(ids, frame))
    u = (x0 >> U32(8)).astype(F32) * F32(2.0 ** -24) - F32(0.5)
    w = (x1 >> U32(8)).astype(F32) * F32(2.0 ** -24) - F32(0.5)
    return u, w


def quantize_normal(c) -> np.ndarray:
    """q(c) = clamp(floor((c + 1) * 128), 0, 255): 8 bits per normal axis."""
    q = np.floor((c + F32(1.0)) * F32(128.0))
    q = np.fmin(np.fmax(q, F32(0.0)), F32(255.0))
    return q.astype(np.int32)


_QMIN = F32(-2147483648.0)
_QMAX = F32(2147483520.0)  # largest float32 below 2^31


@dataclass
class Keys:
    xq: np.ndarray  # (N, 3) int32 quantized position x~
    lod: np.ndarray  # (N,) int32 l' (level at the jittered point)
    lod0: np.ndarray  # (N,) int32 l (level before jittering)
    nq: np.ndarray  # (N, 3) int32 quantized normal
    home: np.ndarray  # (N,) uint32 i = hash & (T - 1)
    fp: np.ndarray  # (N,) uint32 fingerprint, never 0
    xj: np.ndarray  # (N, 3) float32 jittered position x'

    def tuples(self) -> np.ndarray:
        """Full quantized tuple (x~x, x~y, x~z, l', qx, qy, qz) per vertex."""
        return np.column_stack([self.xq.astype(np.int64), self.lod.astype(np.int64),
                                self.nq.astype(np.int64)])


def camera_distance(cx, cy, cz, x, y, z) -> np.ndarray:
    """|p_cam - x| in FP32: sqrt(((dx*dx) + (dy*dy)) + (dz*dz)), each op rounded."""
    dx = F32(cx) - x
    dy = F32(cy) - y
    dz = F32(cz) - z
    return np.sqrt((dx * dx + dy * dy) + dz * dz)


def level_of_detail_at(d, k, lod_min, lod_max) -> np.ndarray:
    """floor(log2(k * d)) for a given FP32 distance d (exponent bits), clamped."""
    F = F32(k) * np.asarray(d, dtype=F32)
    e = ((F.view(U32) >> U32(23)) & U32(0xFF)).astype(np.int32) - 127
    return np.clip(e, lod_min, lod_max).astype(np.int32)


def vertex_keys(p: KeyParams, cam, frame: int, px, py, pz, nx, ny, nz,
                ids=None, stream: int = 0, dist=None, extra=None) -> Keys:
    """Algorithm 1 for every vertex.

    l  <- level_of_detail(|p_cam - x|)
    x' <- x + jitter(n) * 2^l          (tangent plane of n; skipped if no jitter)
    l' <- level_of_detail(|p_cam - x'|)
    x~ <- floor(x' * 2^-l')            (exact scaling by a power of two)
    i  <- hash(x~, l') mod T,   f <- hash2(x~, l', q(n)), 0 replaced by 1.

    Key variants (Sec. 3.1.2, 3.1.1 and the caption of Algorithm 1, which
    lets the hashed arguments be extended):
    * `dist`: a per-vertex distance d (e.g. the length of the path to the
      vertex) replaces the camera distance in the first level of detail; the
      second uses d' = (d - |p_cam - x|) + |p_cam - x'|, the same distance
      moved by the jitter's change of camera distance (with d = |p_cam - x|,
      d' = |p_cam - x'| exactly, and the keys are those of Algorithm 1).
    * `extra`: a per-vertex 32-bit word (e.g. a material or layer id, a
      quantized incident direction) hashed after the other words into both
      hashes."""
    px, py, pz, nx, ny, nz = (np.asarray(a, dtype=F32) for a in (px, py, pz, nx, ny, nz))
    n = px.shape[0]
    if ids is None:
        ids = np.arange(n, dtype=np.uint64).astype(U32)
    cx, cy, cz = (F32(c) for c in cam)
    k = footprint_scale(p)
    if dist is None:
        l0 = level_of_detail(cx, cy, cz, px, py, pz, k, p.lod_min, p.lod_max)
    else:
        dist = np.asarray(dist, dtype=F32)
        l0 = level_of_detail_at(dist, k, p.lod_min, p.lod_max)
    if p.jitter:
        u, w = jitter_uw(ids, stream, p.seed, frame)
        (tx, ty, tz), (bx, by, bz) = orthonormal_basis(nx, ny, nz)
        E = pow2_f32(l0)
        jx = u * tx + w * bx
        jy = u * ty + w * by
        jz = u * tz + w * bz
        xj = px + jx * E
        yj = py + jy * E
        zj = pz + jz * E
        if dist is None:
            l1 = level_of_detail(cx, cy, cz, xj, yj, zj, k, p.lod_min, p.lod_max)
        else:
            d1 = (dist - camera_distance(cx, cy, cz, px, py, pz)) + \
                camera_distance(cx, cy, cz, xj, yj, zj)
            l1 = level_of_detail_at(d1, k, p.lod_min, p.lod_max)
    else:
        xj, yj, zj = px, py, pz
        l1 = l0
    inv = pow2_f32(-l1.astype(np.int64))
    q = [np.fmin(np.fmax(np.floor(c * inv), _QMIN), _QMAX).astype(np.int32)
         for c in (xj, yj, zj)]
    xq = np.column_stack(q)
    nq = np.column_stack([quantize_normal(c) for c in (nx, ny, nz)])
    X, Y, Z = (c.view(U32) for c in q)
    L = l1.astype(np.int32).view(U32)
    NQ = (nq[:, 0] | (nq[:, 1] << 8) | (nq[:, 2] << 16)).astype(U32)
    EX = [] if extra is None else [np.asarray(extra, dtype=U32)]
    home_words = [X, Y, Z, L] + ([NQ] if p.normal_in_home_hash else []) + EX
    h1 = murmur3_32(home_words, p.hash_seed_home)
    home = h1 & U32((1 << p.log2_slots) - 1)
    f = murmur3_32([X, Y, Z, L, NQ] + EX, p.hash_seed_fp)
    f = np.where(f == 0, U32(1), f).astype(U32)
    return Keys(xq, l1, l0, nq, home.astype(U32), f, np.column_stack([xj, yj, zj]))


# ----------------------------------------------------------------------------
# Exact conversions used by the fixed-point mode.
# ----------------------------------------------------------------------------
FIXED_SHIFT = 24


def to_fixed(v) -> np.ndarray:
    """Round-to-nearest-even of v * 2^24 into int64 (v * 2^24 is exact)."""
    v = np.asarray(v, dtype=F32).astype(np.float64) * float(2 ** FIXED_SHIFT)
    return np.rint(v).astype(np.int64)


def _bit_length_u64(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64)
    bl = np.zeros(a.shape, dtype=np.int64)
    for s in (32, 16, 8, 4, 2, 1):
        m = a >= (np.uint64(1) << np.uint64(s))
        bl += np.where(m, s, 0)
        a = np.where(m, a >> np.uint64(s), a)
    return bl + (a > 0)


def int64_to_f32_rn(v) -> np.ndarray:
    """Correctly rounded (nearest, ties to even) int64 -> float32.

    Keep the top 24 significant bits of |v|; round up when the dropped part
    exceeds half a unit of the kept part, or equals it and the kept part is odd."""
    v = np.asarray(v, dtype=np.int64)
    neg = v < 0
    a = np.where(neg, -(v + 1), v).astype(np.uint64) + neg.astype(np.uint64)  # |v|
    bl = _bit_length_u64(a)
    shift = np.maximum(bl - 24, 0).astype(np.uint64)
    q = a >> shift
    rem = a - (q << shift)
    sm1 = np.where(shift > 0, shift - np.uint64(1), np.uint64(0))
    half = np.where(shift > 0, np.uint64(1) << sm1, np.uint64(0))
    up = (shift > 0) & ((rem > half) | ((rem == half) & ((q & np.uint64(1)) == 1)))
    q = q + up.astype(np.uint64)
    mag = q.astype(np.float64) * np.exp2(shift.astype(np.float64))
    return np.where(neg, -mag, mag).astype(F32)


# ----------------------------------------------------------------------------
# Accumulation and lookup, Eq. 8/9 with w = 1, in the gather form.
# ----------------------------------------------------------------------------
@dataclass
class FrameResult:
    keys: Keys
    cell: np.ndarray  # (N,) cell index into the sorted tuple list
    tuples: np.ndarray  # (C, 7) sorted distinct tuples
    count: np.ndarray  # (N,) int64 members of the vertex's cell
    mean64: np.ndarray  # (N, 3) float64 cell average (reference value)
    mean_fixed: np.ndarray  # (N, 3) float32 average from fixed-point sums
    cell_count: np.ndarray  # (C,)
    cell_sum64: np.ndarray  # (C, 3)
    cell_fixed: np.ndarray  # (C, 3) int64
    cell_home: np.ndarray  # (C,) uint32
    cell_fp: np.ndarray  # (C,) uint32


def group_cells(tuples: np.ndarray):
    """Ordered-map group-by over the full tuple: (sorted tuples, inverse, counts)."""
    uniq, inv, cnt = np.unique(tuples, axis=0, return_inverse=True, return_counts=True)
    return uniq, inv.reshape(-1), cnt


def fixed_mean_f32(sum_fixed: np.ndarray, count: np.ndarray) -> np.ndarray:
    """fl32(fl32(sum) * 2^-24) / fl32(n): the fixed-point mode's cell average.

    `sum_fixed` is (C, 3) int64 and `count` (C,); the product by 2^-24 is exact
    and the division is one FP32 round-to-nearest."""
    s = int64_to_f32_rn(sum_fixed) * F32(2.0 ** -FIXED_SHIFT)
    return (s / count.astype(F32)[:, None]).astype(F32)


def filter_frame(p: KeyParams, cam, frame: int, v: Dict[str, np.ndarray],
                 ids=None, stream: int = 0) -> FrameResult:
    """One frame of hashed path space filtering over the vertex arrays `v`
    (optional entries "dist" and "extra": the key variants of vertex_keys;
    the extra word then joins the grouping tuple)."""
    keys = vertex_keys(p, cam, frame, v["px"], v["py"], v["pz"], v["nx"], v["ny"], v["nz"],
                       ids=ids, stream=stream, dist=v.get("dist"), extra=v.get("extra"))
    tuples = keys.tuples()
    if v.get("extra") is not None:
        tuples = np.column_stack([tuples, np.asarray(v["extra"], dtype=np.uint32).astype(np.int64)])
    uniq, inv, cnt = group_cells(tuples)
    C = uniq.shape[0]
    rgb = np.column_stack([np.asarray(v[c], dtype=F32) for c in ("r", "g", "b")])
    sum64 = np.column_stack([np.bincount(inv, weights=rgb[:, j].astype(np.float64), minlength=C)
                             for j in range(3)])
    fx = to_fixed(rgb)
    sumfx = np.zeros((C, 3), dtype=np.int64)
    np.add.at(sumfx, inv, fx)
    count = cnt[inv].astype(np.int64)
    mean64 = sum64[inv] / count[:, None]
    mean_fixed = fixed_mean_f32(sumfx, cnt)[inv]
    # one representative vertex per cell gives the cell's home and fingerprint
    rep = np.zeros(C, dtype=np.int64)
    rep[inv] = np.arange(inv.shape[0])
    return FrameResult(keys, inv, uniq, count, mean64, mean_fixed, cnt.astype(np.int64),
                       sum64, sumfx, keys.home[rep], keys.fp[rep])


# ----------------------------------------------------------------------------
# Temporal filtering / integration, Sec. 3.4.1.
# ----------------------------------------------------------------------------
@dataclass
class History:
    """Per-cell history: sorted tuples, blended averages c and sample counts N."""

    tuples: np.ndarray
    c: np.ndarray
    n: np.ndarray

    @staticmethod
    def empty() -> "History":
        return History(np.zeros((0, 7), dtype=np.int64), np.zeros((0, 3)),
                       np.zeros(0, dtype=np.int64))


def migrated_history(history: History, tuples: np.ndarray):
    """Changes in resolution across frames (Sec. 3.4.2) for cells `tuples`
    that have no history entry of their own, read from `history` as it was
    before this frame.

    Resolution decreased (the cell is coarser than before): its eight finer
    children (2 x~ + d, d in {0, 1}^3, level l' - 1, the other tuple entries
    equal) that have history are added up -- sums and counts, so the value is
    sum(N_i c_i) / sum(N_i) and the count sum(N_i).  Otherwise, resolution
    increased (the cell is finer than before): its coarser parent (floor(x~ /
    2), level l' + 1) passes on its average, its count shared among its eight
    children, ceil(N / 8).  Returns (c_old (m, 3), n_old (m,), found (m,))."""
    m = tuples.shape[0]
    c = np.zeros((m, 3))
    n = np.zeros(m, dtype=np.int64)
    if history.tuples.shape[0] == 0 or m == 0:
        return c, n, np.zeros(m, dtype=bool)
    hk = _row_keys(history.tuples)
    order = np.argsort(hk, kind="stable")
    sk = hk[order]

    def lookup(q):
        qk = _row_keys(q)
        pos = np.searchsorted(sk, qk)
        posc = np.minimum(pos, sk.shape[0] - 1)
        hit = (pos < sk.shape[0]) & (sk[posc] == qk)
        return np.where(hit, order[posc], -1)

    sum_nc = np.zeros((m, 3))
    sum_n = np.zeros(m, dtype=np.int64)
    for d in np.array([(dx, dy, dz) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]):
        q = tuples.copy()
        q[:, :3] = 2 * q[:, :3] + d
        q[:, 3] -= 1
        idx = lookup(q)
        hit = idx >= 0
        sum_nc[hit] += history.n[idx[hit], None] * history.c[idx[hit]]
        sum_n[hit] += history.n[idx[hit]]
    kids = sum_n > 0
    c[kids] = sum_nc[kids] / sum_n[kids, None]
    n[kids] = sum_n[kids]
    q = tuples.copy()
    q[:, :3] = np.floor_divide(q[:, :3], 2)
    q[:, 3] += 1
    idx = lookup(q)
    par = ~kids & (idx >= 0)
    c[par] = history.c[idx[par]]
    n[par] = (history.n[idx[par]] + 7) // 8
    return c, n, kids | par


def blend(history: History, fr: FrameResult, alpha: float, fp16: bool = False,
          n_cap: Optional[int] = None, migrate: bool = False, c_new=None
          ) -> Tuple[History, np.ndarray, np.ndarray]:
    """c = alpha c_old + (1 - alpha) c_new per cell present in this frame.

    alpha < 0 selects the integrating weight N_old / (N_old + N_new).  A cell
    without history takes c_new; cells absent this frame keep their history.
    N <- N_old + N_new (capped at `n_cap` if given).  With `fp16` the stored
    average is rounded to binary16, as a half-precision history store does.
    With `migrate` a cell without history of its own takes the one of its
    finer children or coarser parent (migrated_history) as (c_old, N_old).
    `c_new` (C, 3), if given, is this frame's average per cell instead of the
    FP64 sum / count -- e.g. the fixed-point mode's average, which is what a
    fixed-point table blends.
    Returns (new history, blended value per vertex (N, 3), count per vertex)."""
    H = history.tuples.shape[0]
    allk = np.concatenate([history.tuples, fr.tuples]) if H else fr.tuples
    uniq, inv = np.unique(allk, axis=0, return_inverse=True)[:2]
    inv = inv.reshape(-1)
    U = uniq.shape[0]
    io, inw = inv[:H], inv[H:]
    has_old = np.zeros(U, dtype=bool)
    has_old[io] = True
    c = np.zeros((U, 3))
    N = np.zeros(U, dtype=np.int64)
    c[io] = history.c
    N[io] = history.n
    if c_new is None:
        c_new = fr.cell_sum64 / fr.cell_count[:, None]
    else:
        c_new = np.asarray(c_new, dtype=np.float64)
    n_new = fr.cell_count
    c_old = c[inw]
    n_old = N[inw]
    had = has_old[inw]
    if migrate and not had.all():
        need = np.nonzero(~had)[0]
        mc, mn, mf = migrated_history(history, fr.tuples[need])
        c_old[need[mf]] = mc[mf]
        n_old[need[mf]] = mn[mf]
        had[need[mf]] = True
    if alpha < 0:
        a = (n_old / np.maximum(n_old + n_new, 1))[:, None]
    else:
        a = float(alpha)
    out = np.where(had[:, None], a * c_old + (1.0 - a) * c_new, c_new)
    if fp16:
        out = out.astype(np.float16).astype(np.float64)
    c[inw] = out
    N[inw] = n_old + n_new
    if n_cap is not None:
        N = np.minimum(N, n_cap)
    new = History(uniq, c, N)
    return new, out[fr.cell], N[inw][fr.cell]


# ----------------------------------------------------------------------------
# Table audit: fingerprint ambiguity and probe-limit overflow (Sec. 3.2, 3.2.1).
# ----------------------------------------------------------------------------
def ambiguous_cells(cell_home: np.ndarray, cell_fp: np.ndarray, log2_slots: int,
                    max_probes: int) -> np.ndarray:
    """Cells whose fingerprint equals another cell's while their homes lie
    closer than P slots (mod T), so that their probe windows overlap.  The
    table may merge such cells, which the paper accepts as the price of
    fingerprints (Sec. 3.2.1); cells further apart can never meet."""
    T = 1 << log2_slots
    order = np.argsort(cell_fp, kind="stable")
    fs = cell_fp[order]
    starts = np.nonzero(np.r_[True, fs[1:] != fs[:-1]])[0]
    ends = np.r_[starts[1:], fs.shape[0]]
    amb = np.zeros(cell_fp.shape[0], dtype=bool)
    for s, e in zip(starts[ends - starts > 1], ends[ends - starts > 1]):
        members = order[s:e]
        hs = cell_home[members].astype(np.int64)
        for a in range(members.shape[0]):
            for b in range(a + 1, members.shape[0]):
                d = (hs[b] - hs[a]) % T
                if min(d, T - d) < max_probes:
                    amb[members[a]] = amb[members[b]] = True
    return amb


def overflow_window_full(fp_table: np.ndarray, home: int, f: int, max_probes: int) -> bool:
    """True iff slots home .. home+P-1 (mod T) are all occupied by fingerprints
    other than f: the only state in which an insert may legally give up."""
    T = fp_table.shape[0]
    idx = (home + np.arange(max_probes)) % T
    w = fp_table[idx]
    return bool(np.all((w != 0) & (w != f)))


def simulate_linear_probing(home: np.ndarray, fp: np.ndarray, log2_slots: int,
                            max_probes: int):
    """Sequential insert-only linear probing of distinct keys in the given order.

    Returns (slot per key or -1 on overflow, probes used per key, final table)."""
    T = 1 << log2_slots
    table = np.zeros(T, dtype=U32)
    slot = np.full(home.shape[0], -1, dtype=np.int64)
    probes = np.zeros(home.shape[0], dtype=np.int64)
    for j in range(home.shape[0]):
        h = int(home[j])
        f = int(fp[j])
        for s in range(max_probes):
            q = (h + s) & (T - 1)
            cur = int(table[q])
            if cur == 0:
                table[q] = f
                slot[j] = q
                probes[j] = s + 1
                break
            if cur == f:
                slot[j] = q
                probes[j] = s + 1
                break
        else:
            probes[j] = max_probes
    return slot, probes, table


# ----------------------------------------------------------------------------
# Fallbacks for cells with few vertices (Sec. 3.3): neighborhood search
# (Sec. 3.3.1) and multi-level accumulation (Sec. 3.3.2).  Both replace the
# value of a vertex only where its own cell has fewer than `threshold`
# members.
# ----------------------------------------------------------------------------
STATUS_OK = 0
STATUS_LOWCOUNT = 1
STATUS_COARSE = 4
STATUS_NEIGHBORS = 5


def coarse_params(p: KeyParams) -> KeyParams:
    """The next coarser resolution: the footprint scale s doubled.

    fl32(2 s * theta) = 2 fl32(s * theta) exactly, so every level of detail
    grows by exactly one (before the clamp), the jitter draw (u, w) stays the
    same and its offset is scaled by the coarser voxel edge 2^(l+1)."""
    return dataclasses.replace(p, voxel_scale=float(F32(2.0) * F32(p.voxel_scale)))


def multilevel_select(fine_value, fine_count, coarse_value, coarse_count, threshold: int):
    """Multi-level accumulation (Sec. 3.3.2): every vertex is accumulated at
    its own resolution and at the next coarser one; a vertex whose own cell
    has fewer than `threshold` members takes the coarser cell's value and
    count instead (status COARSE).  Works on per-vertex arrays, so the
    values may be plain averages or temporally blended ones.

    Returns (value (N, 3), count (N,), status (N,) uint8)."""
    low = np.asarray(fine_count) < threshold
    value = np.where(low[:, None], coarse_value, fine_value)
    count = np.where(low, coarse_count, fine_count)
    status = np.where(low, STATUS_COARSE, STATUS_OK).astype(np.uint8)
    return value, count, status


NEIGHBOR_OFFSETS = np.array([(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1)
                             for dz in (-1, 0, 1)], dtype=np.int64)


def _row_keys(t: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(t, dtype=np.int64).view(np.dtype((np.void, 8 * t.shape[1]))).ravel()


def neighbor_cells(tuples: np.ndarray, centers: np.ndarray) -> np.ndarray:
    """For each center tuple (x~x, x~y, x~z, l', qx, qy, qz) the indices of the
    27 cells (x~ + o, l', q), o in {-1, 0, 1}^3, among `tuples` (-1 where no
    such cell exists)."""
    keys = _row_keys(tuples)
    order = np.argsort(keys, kind="stable")
    sk = keys[order]
    out = np.full((centers.shape[0], NEIGHBOR_OFFSETS.shape[0]), -1, dtype=np.int64)
    for i, o in enumerate(NEIGHBOR_OFFSETS):
        q = centers.copy()
        q[:, :3] += o
        qk = _row_keys(q)
        pos = np.searchsorted(sk, qk)
        posc = np.minimum(pos, sk.shape[0] - 1)
        hit = (pos < sk.shape[0]) & (sk[posc] == qk)
        out[hit, i] = order[posc[hit]]
    return out


def neighborhood(fr: FrameResult, threshold: int, cell_value=None, cell_weight=None, only=None):
    """Neighborhood search (Sec. 3.3.1): a vertex whose own cell has fewer
    than `threshold` members takes the pooled average of the 3 x 3 x 3 block of
    cells around its cell at the same level and with the same quantized
    normal, i.e. the members of all those cells averaged together (cells that
    hold no vertex add nothing); its count becomes the block's member count
    and its status NEIGHBORS.

    Without `cell_value` the pooled average is (sum of the block's sums) /
    (sum of its counts), in FP64 and in the fixed-point reading
    fl32(fl32(sum of fixed sums) * 2^-24) / fl32(count).  With per-cell
    `cell_value` (C, 3) and `cell_weight` (C,) -- blended values and their
    counts N after a temporal blend -- it is sum(N c) / sum(N) in FP64, and
    the low-count test reads N.

    `only` (vertex indices): search only for those vertices (the others keep
    their own cell's values); the results for them are the same.

    Returns (value64 (N, 3), value_fixed (N, 3) or None, count (N,), status)."""
    if cell_value is None:
        w = fr.cell_count
    else:
        w = np.asarray(cell_weight, dtype=np.int64)
    own = w[fr.cell]
    low = own < threshold
    if cell_value is None:
        value64 = fr.mean64.copy()
        value_fx = fr.mean_fixed.copy()
    else:
        value64 = np.asarray(cell_value, dtype=np.float64)[fr.cell].copy()
        value_fx = None
    count = own.copy()
    status = np.zeros(fr.cell.shape[0], dtype=np.uint8)
    status[low] = STATUS_NEIGHBORS
    idx = np.nonzero(low)[0]
    if only is not None:
        idx = np.intersect1d(idx, np.asarray(only, dtype=np.int64))
    if idx.size == 0:
        return value64, value_fx, count, status
    nb = neighbor_cells(fr.tuples, fr.tuples[fr.cell[idx]])
    ok = nb >= 0
    nbc = np.where(ok, nb, 0)
    wn = np.where(ok, w[nbc], 0)
    tot = wn.sum(axis=1)
    count[idx] = tot
    if cell_value is None:
        s64 = np.where(ok[:, :, None], fr.cell_sum64[nbc], 0.0).sum(axis=1)
        sfx = np.where(ok[:, :, None], fr.cell_fixed[nbc], 0).sum(axis=1)
        value64[idx] = s64 / tot[:, None]
        value_fx[idx] = fixed_mean_f32(sfx, tot)
    else:
        cv = np.asarray(cell_value, dtype=np.float64)
        s64 = np.where(ok[:, :, None], cv[nbc] * wn[:, :, None], 0.0).sum(axis=1)
        value64[idx] = s64 / tot[:, None]
    return value64, value_fx, count, status


def similar_normals(fr: FrameResult, radius: int, cell_value=None, cell_weight=None):
    """Searching similar normals by linear probing (Sec. 3.2.2).  With the
    normal in the fingerprint only, all cells of one voxel share their home
    slot, so a lookup can walk the probe window past mismatching fingerprints
    and pool, besides its own cell, the cells of the same voxel whose normal
    is similar.  Reading: the cells pooled for a vertex are those with the
    same x~ and l' (and the same extra key word, if any) whose quantized
    normal lies within `radius` quantization steps of the vertex's own on
    every axis (max_a |q_a - q'_a| <= radius: an integer test, so every
    implementation decides membership identically).  radius 0 is the plain
    lookup; radius 255 pools the whole voxel whatever the normal.

    Without `cell_value`: the pooled sums over the pooled counts, in FP64 and
    in the fixed-point reading fl32(fl32(sum of fixed sums) * 2^-24) /
    fl32(count).  With per-cell `cell_value` (C, 3) and `cell_weight` (C,) --
    blended values and their counts N after a temporal blend -- sum(N c) /
    sum(N) in FP64.  Returns (value64 (N, 3), value_fixed (N, 3) or None,
    count (N,))."""
    T = fr.tuples
    C = T.shape[0]
    w = fr.cell_count if cell_value is None else np.asarray(cell_weight, dtype=np.int64)
    cv = None if cell_value is None else np.asarray(cell_value, dtype=np.float64)
    vox = np.concatenate([T[:, :4], T[:, 7:]], axis=1)  # x~, l' and any extra word
    _, vinv = np.unique(vox, axis=0, return_inverse=True)
    vinv = vinv.reshape(-1)
    order = np.argsort(vinv, kind="stable")
    starts = np.r_[0, np.nonzero(np.diff(vinv[order]))[0] + 1, C]
    pw = np.zeros(C, dtype=np.int64)
    p64 = np.zeros((C, 3))
    pfx = np.zeros((C, 3), dtype=np.int64)
    for a, b in zip(starts[:-1], starts[1:]):
        cells = order[a:b]
        q = T[cells, 4:7]
        near = np.abs(q[:, None, :] - q[None, :, :]).max(axis=2) <= radius  # (k, k)
        pw[cells] = near.astype(np.int64) @ w[cells]
        if cv is None:
            p64[cells] = near.astype(np.float64) @ fr.cell_sum64[cells]
            pfx[cells] = near.astype(np.int64) @ fr.cell_fixed[cells]
        else:
            p64[cells] = near.astype(np.float64) @ (cv[cells] * w[cells][:, None])
    count = pw[fr.cell]
    value64 = p64[fr.cell] / count[:, None]
    value_fx = None
    if cv is None:
        value_fx = fixed_mean_f32(pfx, pw)[fr.cell]
    return value64, value_fx, count


# ----------------------------------------------------------------------------
# History eviction, Sec. 3.4.3: the most significant bits of a history
# fingerprint word hold a priority -- here the blend epoch (frame) of the
# entry's last use, 1..255 -- and the low 24 bits the fingerprint, so that one
# word compare orders entries by recency.  0 is an empty cell.
# ----------------------------------------------------------------------------
EVICT_FP_BITS = 24
EVICT_FP_MASK = (1 << EVICT_FP_BITS) - 1


def evict_word(rank: int, f) -> np.ndarray:
    """Priority `rank` (1..255) over the low 24 fingerprint bits."""
    return ((np.uint32(rank) << np.uint32(EVICT_FP_BITS)) |
            (np.asarray(f, dtype=U32) & U32(EVICT_FP_MASK))).astype(U32)


def history_evict_step(table: np.ndarray, home: np.ndarray, fp: np.ndarray, rank: int,
                       max_probes: int):
    """One frame of an evicting history table, cells in the given order.

    For each cell (home h, fingerprint f): scan h .. h+P-1; the first empty
    word is claimed (fresh entry); a word whose low 24 bits equal f's is the
    cell's entry (kept, its priority set to `rank`); if the window is full,
    the entry with the smallest word (oldest priority, then smallest
    fingerprint) is replaced when its priority is older than `rank` (fresh
    entry), otherwise the cell has no history this frame.

    Updates `table` (uint32 words) in place and returns, per cell, the slot
    (-1: none) and whether the entry is fresh (no usable history)."""
    T = table.shape[0]
    slot = np.full(home.shape[0], -1, dtype=np.int64)
    fresh = np.zeros(home.shape[0], dtype=bool)
    f24 = (np.asarray(fp, dtype=np.uint64) & EVICT_FP_MASK).astype(np.int64)
    nw = evict_word(rank, fp).astype(np.int64)
    for j in range(home.shape[0]):
        victim, vword = -1, None
        for p in range(max_probes):
            q = (int(home[j]) + p) % T
            w = int(table[q])
            if w == 0:
                table[q] = nw[j]
                slot[j], fresh[j] = q, True
                break
            if (w & EVICT_FP_MASK) == f24[j]:
                table[q] = nw[j]
                slot[j] = q
                break
            if vword is None or w < vword:
                victim, vword = q, w
        else:
            if (vword >> EVICT_FP_BITS) < rank:
                table[victim] = nw[j]
                slot[j], fresh[j] = victim, True
    return slot, fresh


def history_age(table: np.ndarray, by: int = 128) -> None:
    """Rebase the priorities when the epoch counter runs out: every non-empty
    word's priority drops by `by` (at least 1 stays), keeping the order of
    entries used within the last 255 - by epochs."""
    nz = table != 0
    r = (table >> U32(EVICT_FP_BITS)).astype(np.int64)
    r = np.maximum(r - by, 1)
    table[nz] = ((r[nz].astype(np.uint64) << EVICT_FP_BITS) |
                 (table[nz].astype(np.uint64) & EVICT_FP_MASK)).astype(U32)
