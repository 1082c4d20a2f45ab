"""Named workload presets (plain numbers; no arithmetic of the method).

Each preset fixes the synthetic scene/stream recipe, the table geometry and the
filter options of one workload:

* ``small``   256x256, one primary-hit vertex per pixel (65,536 vertices),
              table 2^18 slots, 16 probes.
* ``hd``      1920x1080, one path per pixel, 3 bounces, Russian-roulette
              survival 0.8 (about 5.06 M vertices), table 2^23 slots, temporal
              blend alpha = 0.2 over 16 frames while the camera moves 0.01 in x
              per frame.
* ``hd_mlp``  the HD workload with the learned fallback for cells with count < 4.
* ``batched`` eight views of uneven resolution (two each at 1280x720,
              1920x1080, 2560x1440, 3840x2160), 2 bounces, about 37 M vertices.
* ``stress``  3840x2160 at 2 paths per pixel, 6 bounces (about 61 M vertices),
              80 % of the vertices squeezed into 5 % of the scene box, table
              2^26 slots, FP16 history, temporal blend over 8 frames.

`voxel_scale` (the s of "s times the projected size of a pixel", Sec. 4) was
calibrated once with the oracle so that the HD table load is about 0.3, then
frozen; the stress value was calibrated for a load of about 0.7.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

from .scene import StreamSpec, View

# Default constants shared by every preset (table seeds and LOD clamp).
JITTER_SEED = 0x0051F15E
HASH_SEED_HOME = 0x9747B28C
HASH_SEED_FP = 0x2F0F1D3B
LOD_MIN = -24
LOD_MAX = 24


@dataclass
class FilterConfig:
    """Table geometry and filter options (mirrors the C parameter block)."""

    log2_slots: int
    max_probes: int
    voxel_scale: float
    pixel_angle: float
    jitter: bool = True
    seed: int = JITTER_SEED
    hash_seed_home: int = HASH_SEED_HOME
    hash_seed_fp: int = HASH_SEED_FP
    # Normal quantization in both hashes: with 8-bit normals on curved surfaces,
    # the fingerprint-only layout printed in Algorithm 1 piles the differently
    # oriented keys of a voxel onto one home slot and overflows 16 probes for
    # about 1% of the HD cells; in both hashes, none overflow.  Membership is
    # identical either way.
    normal_in_home_hash: bool = True
    lod_min: int = LOD_MIN
    lod_max: int = LOD_MAX
    accum_fixed: bool = False
    hist_mode: int = 0  # 0 none, 1 FP32 history, 2 FP16 history
    log2_hist_slots: int = 0
    lowcount_threshold: int = 4
    alpha: Optional[float] = None  # temporal blend weight of the old value (< 0: integrate)
    fallback: str = "none"  # low-count vertices: "none", "coarse" (Sec. 3.3.2), "neighbors" (3.3.1)
    hist_evict: bool = False  # history evicts its least recently used entries (Sec. 3.4.3)
    hist_migrate: bool = False  # history follows changes of resolution (Sec. 3.4.2)
    # searching similar normals by linear probing (Sec. 3.2.2): 0 off, r + 1 =
    # lookups pool the voxel's cells whose quantized normal is within r steps
    normal_search: int = 0

    def oracle_kwargs(self) -> dict:
        """Plain keyword arguments for the oracle's key parameters."""
        return dict(log2_slots=self.log2_slots, max_probes=self.max_probes,
                    voxel_scale=self.voxel_scale, pixel_angle=self.pixel_angle,
                    jitter=self.jitter, seed=self.seed, hash_seed_home=self.hash_seed_home,
                    hash_seed_fp=self.hash_seed_fp,
                    normal_in_home_hash=self.normal_in_home_hash,
                    lod_min=self.lod_min, lod_max=self.lod_max)


@dataclass
class Workload:
    name: str
    streams: List[StreamSpec]
    filters: List[FilterConfig]
    frames: int = 1
    camera_step: float = 0.0  # camera translation in x per frame
    mlp: bool = False
    description: str = ""


HD_VOXEL_SCALE = 4.0
SMALL_VOXEL_SCALE = 4.0
STRESS_VOXEL_SCALE = 0.5  # load 0.70 at 2^26 slots (47.1 M cells of 61.2 M vertices)


def _pixel_angle(v: View) -> float:
    return v.pixel_angle()


def small() -> Workload:
    v = View(256, 256)
    s = StreamSpec(view=v, bounces=1, survival=0.8)
    f = FilterConfig(log2_slots=18, max_probes=16, voxel_scale=SMALL_VOXEL_SCALE,
                     pixel_angle=_pixel_angle(v))
    return Workload("small", [s], [f], frames=1,
                    description="256x256, 1 primary vertex/pixel, T=2^18, P=16")


def hd(frames: int = 16) -> Workload:
    v = View(1920, 1080)
    s = StreamSpec(view=v, bounces=3, survival=0.8)
    f = FilterConfig(log2_slots=23, max_probes=16, voxel_scale=HD_VOXEL_SCALE,
                     pixel_angle=_pixel_angle(v), hist_mode=1, log2_hist_slots=25,
                     alpha=0.2)
    return Workload("hd", [s], [f], frames=frames, camera_step=0.01,
                    description="1920x1080x3 bounces (RR 0.8), T=2^23, P=16, "
                                "temporal alpha=0.2 over 16 frames, camera +0.01/frame")


def hd_mlp(frames: int = 16) -> Workload:
    w = hd(frames)
    w.name = "hd_mlp"
    w.mlp = True
    w.description += ", MLP fallback for count<4"
    return w


BATCHED_VIEWS: Tuple[Tuple[int, int], ...] = (
    (1280, 720), (1280, 720), (1920, 1080), (1920, 1080),
    (2560, 1440), (2560, 1440), (3840, 2160), (3840, 2160))
BATCHED_SURVIVAL = 0.2355  # second-vertex survival that yields about 37 M vertices


def batched() -> Workload:
    streams, filters = [], []
    import math
    for j, (w_, h_) in enumerate(BATCHED_VIEWS):
        ang = 2.0 * math.pi * j / len(BATCHED_VIEWS)
        eye = (12.4 * math.sin(ang), 3.0, -12.4 * math.cos(ang))
        v = View(w_, h_, eye=eye, target=(0.0, 0.5, 0.0))
        streams.append(StreamSpec(view=v, bounces=2, survival=BATCHED_SURVIVAL,
                                  path_seed=2 + 101 * j, radiance_seed=3 + 101 * j))
        log2 = 21 if w_ * h_ <= 1_000_000 else 22 if w_ * h_ <= 2_100_000 else \
            23 if w_ * h_ <= 3_700_000 else 24
        filters.append(FilterConfig(log2_slots=log2, max_probes=16,
                                    voxel_scale=HD_VOXEL_SCALE, pixel_angle=_pixel_angle(v)))
    return Workload("batched", streams, filters, frames=1,
                    description="8 views (2x each 720p/1080p/1440p/2160p), 2 bounces")


def stress(frames: int = 8) -> Workload:
    v = View(3840, 2160, paths_per_pixel=2)
    s = StreamSpec(view=v, bounces=6, survival=0.8, cluster_fraction=0.8,
                   cluster_volume=0.05)
    f = FilterConfig(log2_slots=26, max_probes=16, voxel_scale=STRESS_VOXEL_SCALE,
                     pixel_angle=_pixel_angle(v), hist_mode=2, log2_hist_slots=28,
                     alpha=0.2)
    return Workload("stress", [s], [f], frames=frames, camera_step=0.01, mlp=True,
                    description="3840x2160x2ppp x6 bounces, 80% in 5% volume, T=2^26, "
                                "FP16 history, MLP, temporal over 8 frames")


PRESETS = {"small": small, "hd": hd, "hd_mlp": hd_mlp, "batched": batched, "stress": stress}


def get(name: str, **kw) -> Workload:
    return PRESETS[name](**kw)


def frame_view(w: Workload, stream: int, frame: int) -> View:
    """The camera of stream `stream` at `frame` (translated along x)."""
    v = w.streams[stream].view
    return v.shifted(w.camera_step * frame) if w.camera_step else v


def frame_spec(w: Workload, stream: int, frame: int) -> StreamSpec:
    return replace(w.streams[stream], view=frame_view(w, stream, frame))
