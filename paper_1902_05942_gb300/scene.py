"""Seeded synthetic path-vertex streams (stand-in for the path-generation phase).

The filter of Sec. 3 runs in a second phase over vertices stored by an ordinary
path tracer (Sec. 3, first two paragraphs).  The paper's scenes are not
available, so this module traces a small procedural scene instead: a pinhole
camera with a vertical field of view, a ground plane y = 0, a set of seeded
spheres and an enclosing inward-facing dome, so that every path that survives
Russian roulette produces a vertex.  Each vertex carries

* position (px, py, pz) and unit normal (nx, ny, nz), FP32;
* an RGB "contribution" (the product L_i f_i cos of Eq. 9), drawn i.i.d.
  lognormal(mu, sigma) per channel with a small fraction of fireflies scaled up,
  or, with ``radiance="field"``, that noise times a smooth procedural field.

Vertices are laid out bounce-major (all first vertices in pixel order, then all
surviving second vertices, ...), like the per-bounce buffers of a wavefront
path tracer; the first block is the coherent primary-hit case and the later
blocks the incoherent case that Sec. 4 distinguishes.

This module holds none of the filter's arithmetic (no keys, hashes, jitter or
averages).  It is shared, as plain input generation, by the CPU oracle tests and
by the GPU path; it runs on any torch device (CPU for tests, CUDA for large
benchmark inputs) and is deterministic for a given (seed, frame, device).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import torch

STREAMS = ("px", "py", "pz", "nx", "ny", "nz", "r", "g", "b")

DOME_RADIUS = 100.0
_RAY_EPS = 1e-4
_CHUNK = 1 << 22


@dataclass(frozen=True)
class Spheres:
    centers: torch.Tensor  # (S, 3) float32
    radii: torch.Tensor  # (S,) float32


@dataclass
class View:
    """One pinhole camera and its image."""

    width: int
    height: int
    eye: Tuple[float, float, float] = (0.0, 3.0, -12.0)
    target: Tuple[float, float, float] = (0.0, 0.5, 0.0)
    fov_y_deg: float = 60.0
    paths_per_pixel: int = 1

    def pixel_angle(self) -> float:
        """Angle subtended by one pixel at unit distance: 2 tan(fov/2) / height."""
        return 2.0 * math.tan(math.radians(self.fov_y_deg) * 0.5) / self.height

    def shifted(self, dx: float) -> "View":
        e, t = self.eye, self.target
        return View(self.width, self.height, (e[0] + dx, e[1], e[2]),
                    (t[0] + dx, t[1], t[2]), self.fov_y_deg, self.paths_per_pixel)


@dataclass
class StreamSpec:
    """Everything that determines one synthetic vertex stream."""

    view: View
    bounces: int = 3
    survival: float = 0.8
    scene_seed: int = 1
    path_seed: int = 2
    radiance_seed: int = 3
    sphere_count: int = 16
    mu: float = -1.0
    sigma: float = 1.5
    firefly_prob: float = 0.01
    firefly_scale: float = 100.0
    radiance: str = "iid"  # "iid" | "field" | "constant"
    constant: float = 0.75
    cluster_fraction: float = 0.0  # fraction of vertices squeezed into a small box
    cluster_volume: float = 0.05  # that box's volume as a fraction of the AABB's
    cluster_seed: int = 4
    primary_only_jitter: bool = False  # unused by the generator; kept for configs


def make_spheres(seed: int = 1, count: int = 16) -> Spheres:
    """Seeded sphere set: radius U[0.2, 1.5], centre (U[-10,10], r, U[-10,10])."""
    g = torch.Generator().manual_seed(int(seed))
    radii = 0.2 + 1.3 * torch.rand(count, generator=g, dtype=torch.float64)
    cx = -10.0 + 20.0 * torch.rand(count, generator=g, dtype=torch.float64)
    cz = -10.0 + 20.0 * torch.rand(count, generator=g, dtype=torch.float64)
    centers = torch.stack([cx, radii, cz], dim=1)
    return Spheres(centers.float(), radii.float())


def _normalize(v: torch.Tensor) -> torch.Tensor:
    return v / torch.linalg.vector_norm(v, dim=-1, keepdim=True)


def camera_rays(view: View, device) -> Tuple[torch.Tensor, torch.Tensor]:
    """Primary rays through pixel centres, row-major, `paths_per_pixel` copies each."""
    eye = torch.tensor(view.eye, dtype=torch.float64, device=device)
    tgt = torch.tensor(view.target, dtype=torch.float64, device=device)
    fwd = _normalize(tgt - eye)
    up0 = torch.tensor((0.0, 1.0, 0.0), dtype=torch.float64, device=device)
    right = _normalize(torch.linalg.cross(fwd, up0))
    up = torch.linalg.cross(right, fwd)
    th = math.tan(math.radians(view.fov_y_deg) * 0.5)
    aspect = view.width / view.height
    ys = (torch.arange(view.height, device=device, dtype=torch.float64) + 0.5) / view.height
    xs = (torch.arange(view.width, device=device, dtype=torch.float64) + 0.5) / view.width
    sy = (1.0 - 2.0 * ys) * th
    sx = (2.0 * xs - 1.0) * th * aspect
    d = (fwd[None, None, :] + sx[None, :, None] * right[None, None, :]
         + sy[:, None, None] * up[None, None, :])
    d = _normalize(d).reshape(-1, 3)
    if view.paths_per_pixel > 1:
        d = d.repeat_interleave(view.paths_per_pixel, dim=0)
    o = eye.expand_as(d)
    return o.float().contiguous(), d.float().contiguous()


def _intersect(o: torch.Tensor, d: torch.Tensor, sph: Spheres) -> Tuple[torch.Tensor, torch.Tensor]:
    """Nearest hit of rays (o, d) with plane y=0, the spheres and the dome.

    Returns hit position and the normal facing the incoming ray's side
    (outward for spheres and the plane's top, inward for the dome)."""
    M = o.shape[0]
    dev = o.device
    inf = torch.full((M,), float("inf"), device=dev)
    # dome (origin-centred, rays start inside): far root
    b = (o * d).sum(1)
    c = (o * o).sum(1) - DOME_RADIUS * DOME_RADIUS
    disc = (b * b - c).clamp_min(0.0)
    t_best = -b + torch.sqrt(disc)
    kind = torch.zeros(M, dtype=torch.int64, device=dev)  # 0 dome, 1 plane, 2+s sphere s
    # plane y = 0, approached from above
    tp = torch.where(d[:, 1] < 0, -o[:, 1] / d[:, 1], inf)
    tp = torch.where((o[:, 1] > 0) & (tp > _RAY_EPS), tp, inf)
    better = tp < t_best
    t_best = torch.where(better, tp, t_best)
    kind = torch.where(better, torch.ones_like(kind), kind)
    # spheres
    c_s = sph.centers.to(dev)
    r_s = sph.radii.to(dev)
    oc = o[:, None, :] - c_s[None, :, :]  # (M, S, 3)
    bs = (oc * d[:, None, :]).sum(2)
    cs = (oc * oc).sum(2) - r_s[None, :] ** 2
    ds = bs * bs - cs
    sq = torch.sqrt(ds.clamp_min(0.0))
    t0 = -bs - sq
    t1 = -bs + sq
    inf2 = torch.full_like(t0, float("inf"))
    ts = torch.where(t0 > _RAY_EPS, t0, torch.where(t1 > _RAY_EPS, t1, inf2))
    ts = torch.where(ds > 0, ts, inf2)
    tmin, arg = ts.min(dim=1)
    better = tmin < t_best
    t_best = torch.where(better, tmin, t_best)
    kind = torch.where(better, arg + 2, kind)
    p = o + t_best[:, None] * d
    n = torch.empty_like(p)
    dome = kind == 0
    plane = kind == 1
    sphere = kind >= 2
    n[dome] = -p[dome] / DOME_RADIUS
    n[plane] = torch.tensor((0.0, 1.0, 0.0), device=dev)
    si = (kind[sphere] - 2)
    n[sphere] = (p[sphere] - c_s[si]) / r_s[si][:, None]
    n = _normalize(n)
    return p, n


def _cosine_directions(n: torch.Tensor, u1: torch.Tensor, u2: torch.Tensor) -> torch.Tensor:
    """Cosine-weighted directions about n (any orthonormal frame will do here)."""
    a = torch.where(n[:, 0:1].abs() > 0.9,
                    torch.tensor((0.0, 1.0, 0.0), device=n.device).expand_as(n),
                    torch.tensor((1.0, 0.0, 0.0), device=n.device).expand_as(n))
    t = _normalize(torch.linalg.cross(a, n))
    b = torch.linalg.cross(n, t)
    rad = torch.sqrt(u1)
    phi = 2.0 * math.pi * u2
    x = rad * torch.cos(phi)
    y = rad * torch.sin(phi)
    z = torch.sqrt((1.0 - u1).clamp_min(0.0))
    return _normalize(x[:, None] * t + y[:, None] * b + z[:, None] * n)


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _mix_seed(*words: int) -> int:
    h = 0x243F6A8885A308D3
    for w in words:
        h = ((h ^ (int(w) & 0xFFFFFFFFFFFFFFFF)) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 29
    return h & 0x7FFFFFFFFFFFFFFF


def smooth_field(p: torch.Tensor, n: torch.Tensor) -> torch.Tensor:
    """Smooth procedural RGB field g(x, n) used as ground truth by the gain test.

    A clamped cosine towards a fixed point light plus an ambient term, tinted by
    slowly varying sinusoids of position; positive and bounded."""
    light = torch.tensor((4.0, 12.0, -3.0), device=p.device)
    l = _normalize(light[None, :] - p)
    cos = (l * n).sum(1).clamp_min(0.0)
    tint = torch.stack([
        0.6 + 0.4 * torch.sin(0.31 * p[:, 0] + 0.2),
        0.6 + 0.4 * torch.sin(0.27 * p[:, 2] + 1.1),
        0.6 + 0.4 * torch.cos(0.23 * (p[:, 0] + p[:, 2])),
    ], dim=1)
    return tint * (0.15 + 0.85 * cos[:, None])


def trace_stream(spec: StreamSpec, frame: int = 0, device="cpu") -> Dict[str, torch.Tensor]:
    """Trace `spec` for one frame; return SoA float32 streams plus metadata.

    Keys: the nine STREAMS (contiguous float32, length N), ``bounce_counts``
    (list of ints), and for ``radiance="field"`` also ``truth_r/g/b`` (the
    expected contribution g(x, n) * E[noise])."""
    device = torch.device(device)
    sph = make_spheres(spec.scene_seed, spec.sphere_count)
    o, d = camera_rays(spec.view, device)
    gp = _gen(device, _mix_seed(spec.path_seed, frame))
    pos: List[torch.Tensor] = []
    nrm: List[torch.Tensor] = []
    counts: List[int] = []
    for bounce in range(spec.bounces):
        if o.shape[0] == 0:
            counts.append(0)
            continue
        ps, ns = [], []
        for s in range(0, o.shape[0], _CHUNK):
            p_, n_ = _intersect(o[s:s + _CHUNK], d[s:s + _CHUNK], sph)
            ps.append(p_)
            ns.append(n_)
        p = torch.cat(ps)
        n = torch.cat(ns)
        pos.append(p)
        nrm.append(n)
        counts.append(p.shape[0])
        if bounce + 1 == spec.bounces:
            break
        alive = torch.rand(p.shape[0], generator=gp, device=device) < spec.survival
        p = p[alive]
        n = n[alive]
        u1 = torch.rand(p.shape[0], generator=gp, device=device)
        u2 = torch.rand(p.shape[0], generator=gp, device=device)
        d = _cosine_directions(n, u1, u2)
        o = p + _RAY_EPS * 10.0 * n
    P = torch.cat(pos) if pos else torch.zeros((0, 3), device=device)
    Nn = torch.cat(nrm) if nrm else torch.zeros((0, 3), device=device)
    N = P.shape[0]
    if spec.cluster_fraction > 0.0 and N > 0:
        P = _cluster(P, spec, device)
    out: Dict[str, torch.Tensor] = {}
    out["px"], out["py"], out["pz"] = (P[:, 0].contiguous(), P[:, 1].contiguous(),
                                       P[:, 2].contiguous())
    out["nx"], out["ny"], out["nz"] = (Nn[:, 0].contiguous(), Nn[:, 1].contiguous(),
                                       Nn[:, 2].contiguous())
    rgb, truth = _radiance(spec, frame, P, Nn, device)
    out["r"], out["g"], out["b"] = (rgb[:, 0].contiguous(), rgb[:, 1].contiguous(),
                                    rgb[:, 2].contiguous())
    if truth is not None:
        out["truth_r"], out["truth_g"], out["truth_b"] = (truth[:, 0].contiguous(),
                                                          truth[:, 1].contiguous(),
                                                          truth[:, 2].contiguous())
    for k in STREAMS:
        out[k] = out[k].to(torch.float32).contiguous()
    out["bounce_counts"] = counts
    return out


def _radiance(spec: StreamSpec, frame: int, P, Nn, device):
    N = P.shape[0]
    if spec.radiance == "constant":
        return torch.full((N, 3), float(spec.constant), device=device), None
    gr = _gen(device, _mix_seed(spec.radiance_seed, frame))
    z = torch.randn((N, 3), generator=gr, device=device)
    eps = torch.exp(spec.mu + spec.sigma * z)
    fire = torch.rand(N, generator=gr, device=device) < spec.firefly_prob
    eps = torch.where(fire[:, None], eps * spec.firefly_scale, eps)
    # keep every value a normal float well above FLT_MIN
    eps = eps.clamp_min(2.0 ** -100)
    if spec.radiance == "iid":
        return eps, None
    if spec.radiance == "field":
        g = smooth_field(P, Nn)
        mean_eps = math.exp(spec.mu + 0.5 * spec.sigma ** 2) * (
            1.0 + spec.firefly_prob * (spec.firefly_scale - 1.0))
        return g * eps, g * mean_eps
    raise ValueError(f"unknown radiance mode {spec.radiance!r}")


def _cluster(P: torch.Tensor, spec: StreamSpec, device) -> torch.Tensor:
    """Squeeze a seeded fraction of vertices affinely into a small sub-box.

    The sub-box has `cluster_volume` of the axis-aligned bounding box's volume
    and a seeded placement inside it; this concentrates vertices to stress
    the hash table (adversarial clustering)."""
    gc = _gen(device, _mix_seed(spec.cluster_seed, 0))
    lo = P.min(0).values
    hi = P.max(0).values
    ext = hi - lo
    side = spec.cluster_volume ** (1.0 / 3.0)
    off = torch.rand(3, generator=gc, device=device) * (1.0 - side)
    sel = torch.rand(P.shape[0], generator=gc, device=device) < spec.cluster_fraction
    Q = lo + (off + (P - lo) / ext * side) * ext
    return torch.where(sel[:, None], Q, P)


def camera_position(view: View) -> Tuple[float, float, float]:
    return tuple(float(x) for x in view.eye)


def concat_streams(parts: Sequence[Dict[str, torch.Tensor]]) -> Dict[str, torch.Tensor]:
    out = {k: torch.cat([p[k] for p in parts]).contiguous() for k in STREAMS}
    out["bounce_counts"] = [sum(p["bounce_counts"][i] for p in parts)
                            for i in range(len(parts[0]["bounce_counts"]))]
    return out
