"""Python binding of the C ABI in include/pps.h (argument marshalling only).

The functions carry the C names (``pps_create``, ``pps_build``, ``pps_insert``,
``pps_blend``, ``pps_query``, ``pps_filter``, ...) and take torch tensors,
whose device pointers are handed to the library unchanged; every step of the
filter runs in the CUDA library.  ``Table`` is a small convenience wrapper.

The library is ``libpps.so`` next to this file (built by ``build.py``).  If it
is missing, loading raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpps.so")

PPS_OK, PPS_EINVAL, PPS_ENOMEM, PPS_ECUDA, PPS_EDEVICE, PPS_ESTATE = range(6)
STATUS_OK, STATUS_LOWCOUNT, STATUS_OVERFLOW, STATUS_MLP = 0, 1, 2, 3
STATUS_COARSE, STATUS_NEIGHBORS = 4, 5
FALLBACK_NONE, FALLBACK_COARSE, FALLBACK_NEIGHBORS = 0, 1, 2
FALLBACKS = {"none": FALLBACK_NONE, "coarse": FALLBACK_COARSE, "neighbors": FALLBACK_NEIGHBORS}
MLP_PARAMS = 13699
ACCUM_FP32, ACCUM_FIXED = 0, 1
HIST_NONE, HIST_FP32, HIST_FP16 = 0, 1, 2
OVERFLOW_SLOT = 0xFFFFFFFF

_u32, _i32, _f32 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_float
_vp = ctypes.c_void_p


class pps_params(ctypes.Structure):
    _fields_ = [("log2_slots", _u32), ("max_probes", _u32), ("voxel_scale", _f32),
                ("pixel_angle", _f32), ("jitter", _u32), ("seed", _u32),
                ("hash_seed_home", _u32), ("hash_seed_fp", _u32),
                ("normal_in_home_hash", _u32), ("lod_min", _i32), ("lod_max", _i32),
                ("accum_mode", _u32), ("hist_mode", _u32), ("lowcount_threshold", _u32),
                ("log2_hist_slots", _u32), ("fallback", _u32), ("hist_evict", _u32),
                ("hist_migrate", _u32), ("normal_search", _u32)]


class pps_camera(ctypes.Structure):
    _fields_ = [("pos", _f32 * 3)]


class pps_vertices(ctypes.Structure):
    _fields_ = [("px", _vp), ("py", _vp), ("pz", _vp), ("nx", _vp), ("ny", _vp), ("nz", _vp),
                ("r", _vp), ("g", _vp), ("b", _vp), ("id", _vp), ("id_base", _u32),
                ("stream_id", _u32), ("dist", _vp), ("extra", _vp)]


class pps_output(ctypes.Structure):
    _fields_ = [("r", _vp), ("g", _vp), ("b", _vp), ("count", _vp), ("status", _vp)]


class pps_tuning(ctypes.Structure):
    _fields_ = [("batch", _u32), ("insert", _u32), ("key_warps", _u32), ("block", _u32),
                ("merge", _u32), ("reserved", _u32 * 3)]


class pps_stats_t(ctypes.Structure):
    _fields_ = [("frame_cells", ctypes.c_uint64), ("overflow_vertices", ctypes.c_uint64),
                ("occupied_slots", ctypes.c_uint64), ("vertices", ctypes.c_uint64),
                ("hist_overflow", ctypes.c_uint64), ("hist_occupied", ctypes.c_uint64),
                ("device_error", _u32), ("frame", _u32)]


class pps_view(ctypes.Structure):
    _fields_ = [("table", _vp), ("v", pps_vertices), ("n", ctypes.c_size_t), ("out", pps_output)]


class pps_mlp_params(ctypes.Structure):
    _fields_ = [("box_min", _f32 * 3), ("box_max", _f32 * 3), ("lr", _f32), ("beta1", _f32),
                ("beta2", _f32), ("eps", _f32), ("batch", _u32), ("steps", _u32),
                ("train_min_count", _u32), ("infer_max_count", _u32), ("seed", _u32),
                ("reserved", _u32 * 3)]


# Every exported function and its argument types.
SIGNATURES = {
    "pps_version": ([], ctypes.c_char_p),
    "pps_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "pps_create": ([ctypes.POINTER(_vp), ctypes.POINTER(pps_params)], ctypes.c_int),
    "pps_destroy": ([_vp], ctypes.c_int),
    "pps_build": ([_vp, ctypes.POINTER(pps_camera), _u32, _vp], ctypes.c_int),
    "pps_insert": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t, _vp, _vp], ctypes.c_int),
    "pps_blend": ([_vp, _f32, _vp], ctypes.c_int),
    "pps_query": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t, _vp,
                   ctypes.POINTER(pps_output), _vp], ctypes.c_int),
    "pps_filter": ([_vp, ctypes.POINTER(pps_camera), _u32, ctypes.POINTER(pps_vertices),
                    ctypes.c_size_t, ctypes.c_int, _f32, ctypes.POINTER(pps_output), _vp],
                   ctypes.c_int),
    "pps_filter_host": ([_vp, ctypes.POINTER(pps_camera), _u32, ctypes.POINTER(pps_vertices),
                         ctypes.c_size_t, ctypes.c_int, _f32, ctypes.POINTER(pps_output), _vp],
                        ctypes.c_int),
    "pps_filter_host_async": ([_vp, ctypes.POINTER(pps_camera), _u32,
                               ctypes.POINTER(pps_vertices), ctypes.c_size_t, ctypes.c_int, _f32,
                               ctypes.POINTER(pps_output), _vp], ctypes.c_int),
    "pps_host_wait": ([_vp], ctypes.c_int),
    "pps_keys": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t, _vp, _vp, _vp],
                 ctypes.c_int),
    "pps_stats": ([_vp, ctypes.POINTER(pps_stats_t), _vp], ctypes.c_int),
    "pps_set_tuning": ([_vp, ctypes.POINTER(pps_tuning)], ctypes.c_int),
    "pps_filter_noalloc": ([ctypes.POINTER(pps_params), ctypes.POINTER(pps_camera), _u32,
                            ctypes.POINTER(pps_vertices), ctypes.c_size_t,
                            ctypes.POINTER(pps_output), _vp], ctypes.c_int),
    "pps_noalloc_stats": ([ctypes.POINTER(pps_stats_t), _vp], ctypes.c_int),
    "pps_get_tuning": ([_vp, ctypes.POINTER(pps_tuning)], ctypes.c_int),
    "pps_table_dump": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "pps_mlp_create": ([ctypes.POINTER(_vp), ctypes.POINTER(pps_mlp_params), _vp], ctypes.c_int),
    "pps_mlp_destroy": ([_vp], ctypes.c_int),
    "pps_mlp_set_weights": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pps_mlp_get_weights": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pps_mlp_train": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t,
                       ctypes.POINTER(pps_output), _u32, _vp], ctypes.c_int),
    "pps_mlp_infer": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t,
                       ctypes.POINTER(pps_output), _vp], ctypes.c_int),
    "pps_mlp_forward": ([_vp, ctypes.POINTER(pps_vertices), ctypes.c_size_t, _vp, _vp, _vp, _vp],
                        ctypes.c_int),
    "pps_mlp_gradient": ([_vp, ctypes.POINTER(pps_vertices), _vp, _vp, _vp, _vp, _u32, _vp, _vp],
                         ctypes.c_int),
    "pps_batch_create": ([ctypes.POINTER(_vp), ctypes.POINTER(pps_view), _u32, ctypes.c_int, _f32],
                         ctypes.c_int),
    "pps_batch_run": ([_vp, ctypes.POINTER(pps_camera), _u32, _vp], ctypes.c_int),
    "pps_batch_destroy": ([_vp], ctypes.c_int),
    "pps_selftest_wait": ([ctypes.c_int, _u32, ctypes.POINTER(_u32)], ctypes.c_int),
    "pps_bench_rate": ([ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, _vp, _vp,
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
}

_lib: Optional[ctypes.CDLL] = None


class PPSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pps error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libpps.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1902_05942_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().pps_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != PPS_OK:
        raise PPSError(rc, last_error())


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: Optional[torch.Tensor], n: int, dtype, name: str, device=True) -> Optional[int]:
    if t is None:
        return None
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{name}: need a contiguous {dtype} tensor of >= {n} elements")
    if device and not t.is_cuda:
        raise ValueError(f"{name}: need a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError(f"{name}: need a host tensor")
    return t.data_ptr()


STREAM_NAMES = ("px", "py", "pz", "nx", "ny", "nz", "r", "g", "b")


def make_vertices(v: Dict[str, torch.Tensor], n: Optional[int] = None, ids=None, id_base=0,
                  stream_id=0, device=True) -> pps_vertices:
    n = v["px"].numel() if n is None else n
    ptrs = [_ptr(v[k], n, torch.float32, k, device) for k in STREAM_NAMES]
    return pps_vertices(*ptrs, _ptr(ids, n, torch.int32, "id", device) if ids is not None
                        else None, id_base & 0xFFFFFFFF, stream_id & 0xFFFFFFFF,
                        _ptr(v.get("dist"), n, torch.float32, "dist", device),
                        _ptr(v.get("extra"), n, torch.int32, "extra", device))


def make_output(out: Dict[str, torch.Tensor], n: int, device=True) -> pps_output:
    return pps_output(_ptr(out["r"], n, torch.float32, "r", device),
                      _ptr(out["g"], n, torch.float32, "g", device),
                      _ptr(out["b"], n, torch.float32, "b", device),
                      _ptr(out.get("count"), n, torch.int32, "count", device),
                      _ptr(out.get("status"), n, torch.uint8, "status", device))


def make_params(cfg, hist_mode: Optional[int] = None, accum_fixed: Optional[bool] = None,
                log2_hist_slots: Optional[int] = None, fallback: Optional[str] = None,
                hist_evict: Optional[bool] = None,
                hist_migrate: Optional[bool] = None) -> pps_params:
    """pps_params from a FilterConfig-like object (attribute names as in configs.py)."""
    hm = cfg.hist_mode if hist_mode is None else hist_mode
    fx = cfg.accum_fixed if accum_fixed is None else accum_fixed
    lh = cfg.log2_hist_slots if log2_hist_slots is None else log2_hist_slots
    fb = getattr(cfg, "fallback", "none") if fallback is None else fallback
    ev = getattr(cfg, "hist_evict", False) if hist_evict is None else hist_evict
    mg = getattr(cfg, "hist_migrate", False) if hist_migrate is None else hist_migrate
    return pps_params(cfg.log2_slots, cfg.max_probes, cfg.voxel_scale, cfg.pixel_angle,
                      int(cfg.jitter), cfg.seed & 0xFFFFFFFF, cfg.hash_seed_home & 0xFFFFFFFF,
                      cfg.hash_seed_fp & 0xFFFFFFFF, int(cfg.normal_in_home_hash), cfg.lod_min,
                      cfg.lod_max, ACCUM_FIXED if fx else ACCUM_FP32, hm,
                      cfg.lowcount_threshold, lh, FALLBACKS[fb], int(bool(ev)), int(bool(mg)),
                      int(getattr(cfg, "normal_search", 0)))


def camera(pos: Sequence[float]) -> pps_camera:
    return pps_camera((_f32 * 3)(*[float(x) for x in pos]))


# ---------------------------------------------------------------- C-named calls
def pps_version() -> str:
    return lib().pps_version().decode()


def pps_selftest_wait(kind: int, limit_us: int) -> int:
    """Run one bounded device wait on a condition that never comes true
    (0: grid barrier, 1: tensor-core mbarrier) and return the device error
    word it left (1 when the wait gave up as it should)."""
    w = _u32(0)
    _check(lib().pps_selftest_wait(int(kind), int(limit_us), ctypes.byref(w)))
    return int(w.value)


def pps_create(params: pps_params) -> int:
    h = _vp()
    _check(lib().pps_create(ctypes.byref(h), ctypes.byref(params)))
    return h.value


def pps_destroy(handle: int):
    _check(lib().pps_destroy(handle))


def pps_build(handle, cam: pps_camera, frame: int, stream=None):
    _check(lib().pps_build(handle, ctypes.byref(cam), frame & 0xFFFFFFFF, _stream(stream)))


def pps_insert(handle, v: pps_vertices, n: int, slot_out: Optional[torch.Tensor] = None,
               stream=None):
    _check(lib().pps_insert(handle, ctypes.byref(v), n,
                            _ptr(slot_out, n, torch.int32, "slot_out"), _stream(stream)))


def pps_blend(handle, alpha: float, stream=None):
    _check(lib().pps_blend(handle, float(alpha), _stream(stream)))


def pps_query(handle, v: pps_vertices, n: int, slot_in: Optional[torch.Tensor],
              out: pps_output, stream=None):
    _check(lib().pps_query(handle, ctypes.byref(v), n, _ptr(slot_in, n, torch.int32, "slot_in"),
                           ctypes.byref(out), _stream(stream)))


def pps_filter(handle, cam: pps_camera, frame: int, v: pps_vertices, n: int, blend: bool,
               alpha: float, out: pps_output, stream=None):
    _check(lib().pps_filter(handle, ctypes.byref(cam), frame & 0xFFFFFFFF, ctypes.byref(v), n,
                            1 if blend else 0, float(alpha), ctypes.byref(out), _stream(stream)))


def pps_filter_host(handle, cam: pps_camera, frame: int, v: pps_vertices, n: int, blend: bool,
                    alpha: float, out: pps_output, stream=None):
    _check(lib().pps_filter_host(handle, ctypes.byref(cam), frame & 0xFFFFFFFF, ctypes.byref(v),
                                 n, 1 if blend else 0, float(alpha), ctypes.byref(out),
                                 _stream(stream)))


def pps_filter_host_async(handle, cam: pps_camera, frame: int, v: pps_vertices, n: int,
                          blend: bool, alpha: float, out: pps_output, stream=None):
    _check(lib().pps_filter_host_async(handle, ctypes.byref(cam), frame & 0xFFFFFFFF,
                                       ctypes.byref(v), n, 1 if blend else 0, float(alpha),
                                       ctypes.byref(out), _stream(stream)))


def pps_host_wait(handle):
    _check(lib().pps_host_wait(handle))


def pps_filter_noalloc(params: pps_params, cam: pps_camera, frame: int, v: pps_vertices, n: int,
                       out: pps_output, stream=None):
    _check(lib().pps_filter_noalloc(ctypes.byref(params), ctypes.byref(cam), frame & 0xFFFFFFFF,
                                    ctypes.byref(v), n, ctypes.byref(out), _stream(stream)))


def pps_noalloc_stats(stream=None) -> dict:
    s = pps_stats_t()
    _check(lib().pps_noalloc_stats(ctypes.byref(s), _stream(stream)))
    return {k: getattr(s, k) for k, _ in pps_stats_t._fields_}


def pps_keys(handle, v: pps_vertices, n: int, h_out: torch.Tensor, f_out: torch.Tensor,
             stream=None):
    _check(lib().pps_keys(handle, ctypes.byref(v), n, _ptr(h_out, n, torch.int32, "h_out"),
                          _ptr(f_out, n, torch.int32, "f_out"), _stream(stream)))


def pps_set_tuning(handle, batch: int = 0, insert: int = 0, key_warps: int = 0, block: int = 0,
                   merge: int = 0):
    _check(lib().pps_set_tuning(handle, ctypes.byref(pps_tuning(batch, insert, key_warps, block,
                                                                merge))))


def pps_get_tuning(handle) -> dict:
    t = pps_tuning()
    _check(lib().pps_get_tuning(handle, ctypes.byref(t)))
    return {"batch": t.batch, "insert": t.insert, "key_warps": t.key_warps, "block": t.block,
            "merge": t.merge}


def pps_stats(handle, stream=None) -> dict:
    s = pps_stats_t()
    _check(lib().pps_stats(handle, ctypes.byref(s), _stream(stream)))
    return {k: getattr(s, k) for k, _ in pps_stats_t._fields_}


def pps_table_dump(handle, T: int, fixed: bool, stream=None):
    fp = np.zeros(T, dtype=np.uint32)
    acc = np.zeros((T, 4), dtype=np.int64 if fixed else np.float32)
    _check(lib().pps_table_dump(handle, fp.ctypes.data, acc.ctypes.data, _stream(stream)))
    return fp, acc


RATE_KINDS = {"red_v4_f32": 0, "cas_b32": 1, "red_f32": 2, "gather_v4": 3}


def pps_bench_rate(kind: str, region: torch.Tensor, ops: int, stream=None) -> float:
    """Random memory operations per second of `kind` over the device tensor
    `region` (its contents are overwritten)."""
    out = ctypes.c_double()
    rc = lib().pps_bench_rate(RATE_KINDS[kind], region.numel() * region.element_size(), ops,
                              region.data_ptr(), _stream(stream), ctypes.byref(out))
    if rc:
        raise PPSError(rc, "pps_bench_rate failed")
    return out.value


# ---------------------------------------------------------------- batched views
class Batch:
    """Several views in one persistent launch replayed from a CUDA graph.

    views: list of (Table, vertex dict, output dict).  The arrays must stay
    alive (and in place) for the batch's lifetime."""

    def __init__(self, views, blend=False, alpha=0.2):
        self._keep = views
        arr = (pps_view * len(views))()
        for i, (tab, v, out) in enumerate(views):
            n = v["px"].numel()
            arr[i] = pps_view(tab.handle, make_vertices(v, n), n, make_output(out, n))
        h = _vp()
        _check(lib().pps_batch_create(ctypes.byref(h), arr, len(views), 1 if blend else 0,
                                      float(alpha)))
        self.handle = h.value
        self.n = len(views)

    def run(self, cams, frame, stream=None):
        c = (pps_camera * self.n)(*[camera(x) for x in cams])
        _check(lib().pps_batch_run(self.handle, c, frame & 0xFFFFFFFF, _stream(stream)))

    def close(self):
        if self.handle:
            lib().pps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned fallback
def mlp_params(box_min=(-100.0, -100.0, -100.0), box_max=(100.0, 100.0, 100.0), lr=1e-3,
               beta1=0.9, beta2=0.999, eps=1e-8, batch=16384, steps=4, train_min_count=8,
               infer_max_count=4, seed=7) -> pps_mlp_params:
    return pps_mlp_params((_f32 * 3)(*box_min), (_f32 * 3)(*box_max), lr, beta1, beta2, eps,
                          batch, steps, train_min_count, infer_max_count, seed, (_u32 * 3)())


class MLP:
    """The learned fallback network on the current device."""

    def __init__(self, params: Optional[pps_mlp_params] = None, init=None):
        self.params = params or mlp_params()
        h = _vp()
        w = None
        if init is not None:
            w = np.ascontiguousarray(init, dtype=np.float32)
            assert w.size == MLP_PARAMS
        _check(lib().pps_mlp_create(ctypes.byref(h), ctypes.byref(self.params),
                                    w.ctypes.data if w is not None else None))
        self.handle = h.value

    def close(self):
        if self.handle:
            lib().pps_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib().pps_mlp_set_weights(self.handle, w.ctypes.data, w.size))

    def get_weights(self) -> np.ndarray:
        w = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(lib().pps_mlp_get_weights(self.handle, w.ctypes.data, w.size))
        return w

    def train(self, v, filtered, frame, stream=None, ids=None):
        n = v["px"].numel()
        _check(lib().pps_mlp_train(self.handle, ctypes.byref(make_vertices(v, n, ids)), n,
                                   ctypes.byref(make_output(filtered, n)), frame & 0xFFFFFFFF,
                                   _stream(stream)))

    def infer(self, v, out, stream=None):
        n = v["px"].numel()
        _check(lib().pps_mlp_infer(self.handle, ctypes.byref(make_vertices(v, n)), n,
                                   ctypes.byref(make_output(out, n)), _stream(stream)))

    def forward(self, v, stream=None):
        n = v["px"].numel()
        o = {c: torch.empty(n, dtype=torch.float32, device=v["px"].device) for c in "rgb"}
        _check(lib().pps_mlp_forward(self.handle, ctypes.byref(make_vertices(v, n)), n,
                                     o["r"].data_ptr(), o["g"].data_ptr(), o["b"].data_ptr(),
                                     _stream(stream)))
        return o

    def gradient(self, v, targets, idx: torch.Tensor, stream=None) -> torch.Tensor:
        n = v["px"].numel()
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=v["px"].device)
        _check(lib().pps_mlp_gradient(self.handle, ctypes.byref(make_vertices(v, n)),
                                      targets["r"].data_ptr(), targets["g"].data_ptr(),
                                      targets["b"].data_ptr(), _ptr(idx, idx.numel(), torch.int32,
                                                                    "idx"),
                                      idx.numel(), g.data_ptr(), _stream(stream)))
        return g


# ---------------------------------------------------------------- convenience
def empty_output(n: int, device="cuda", count=True, status=True) -> Dict[str, torch.Tensor]:
    o = {c: torch.empty(n, dtype=torch.float32, device=device) for c in ("r", "g", "b")}
    if count:
        o["count"] = torch.empty(n, dtype=torch.int32, device=device)
    if status:
        o["status"] = torch.empty(n, dtype=torch.uint8, device=device)
    return o


class Table:
    """One filter table (frame table plus optional history) on the current device."""

    def __init__(self, cfg, hist_mode: Optional[int] = None, accum_fixed: Optional[bool] = None,
                 log2_hist_slots: Optional[int] = None, fallback: Optional[str] = None,
                 hist_evict: Optional[bool] = None, hist_migrate: Optional[bool] = None):
        self.params = make_params(cfg, hist_mode, accum_fixed, log2_hist_slots, fallback,
                                  hist_evict, hist_migrate)
        self.handle = pps_create(self.params)
        self.T = 1 << self.params.log2_slots
        self.fixed = self.params.accum_mode == ACCUM_FIXED

    def close(self):
        if self.handle:
            pps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def filter(self, v, cam, frame, blend=False, alpha=0.2, out=None, stream=None, ids=None,
               id_base=0, stream_id=0):
        n = v["px"].numel()
        out = empty_output(n, v["px"].device) if out is None else out
        pps_filter(self.handle, camera(cam), frame, make_vertices(v, n, ids, id_base, stream_id),
                   n, blend, alpha, make_output(out, n), stream)
        return out

    def build(self, cam, frame, stream=None):
        pps_build(self.handle, camera(cam), frame, stream)

    def insert(self, v, slot_out=None, stream=None, ids=None, id_base=0, stream_id=0):
        n = v["px"].numel()
        pps_insert(self.handle, make_vertices(v, n, ids, id_base, stream_id), n, slot_out, stream)

    def blend(self, alpha, stream=None):
        pps_blend(self.handle, alpha, stream)

    def query(self, v, slot_in=None, out=None, stream=None, ids=None, id_base=0, stream_id=0):
        n = v["px"].numel()
        out = empty_output(n, v["px"].device) if out is None else out
        pps_query(self.handle, make_vertices(v, n, ids, id_base, stream_id), n, slot_in,
                  make_output(out, n), stream)
        return out

    def keys(self, v, stream=None, ids=None, id_base=0, stream_id=0):
        n = v["px"].numel()
        h = torch.empty(n, dtype=torch.int32, device=v["px"].device)
        f = torch.empty(n, dtype=torch.int32, device=v["px"].device)
        pps_keys(self.handle, make_vertices(v, n, ids, id_base, stream_id), n, h, f, stream)
        return h, f

    def stats(self, stream=None) -> dict:
        return pps_stats(self.handle, stream)

    def tune(self, batch: int = 0, insert: int = 0, key_warps: int = 0, block: int = 0,
             merge: int = 0):
        pps_set_tuning(self.handle, batch, insert, key_warps, block, merge)

    def dump(self, stream=None):
        return pps_table_dump(self.handle, self.T, self.fixed, stream)
