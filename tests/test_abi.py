"""The C-ABI library loads, exports every function include/pps.h declares, and
its host-side argument checks answer without a GPU.  The ctypes layouts of the
binding are checked against a C program compiled from the header."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", h) for h in ("pps.h", "pps_bench.h")]


def _lib():
    from paper_1902_05942_gb300 import build, pps
    build.build()
    return pps, pps.lib()


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pps_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("pps_build", "pps_insert", "pps_query", "pps_blend", "pps_create", "pps_destroy",
              "pps_filter", "pps_stats"):
        assert n in names


def test_library_exports_every_declared_symbol():
    pps, L = _lib()
    out = subprocess.run(["nm", "-D", "--defined-only", pps.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (pps_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert n in pps.SIGNATURES, f"binding lacks {n}"
        getattr(L, n)


def test_struct_layouts_match_the_header(tmp_path):
    pps, _ = _lib()
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pps.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        " sizeof(pps_params), sizeof(pps_camera), sizeof(pps_vertices), sizeof(pps_output),"
        " sizeof(pps_stats_t), offsetof(pps_params, log2_hist_slots),"
        " offsetof(pps_vertices, id_base), sizeof(pps_tuning), offsetof(pps_tuning, merge),"
        " sizeof(pps_mlp_params), offsetof(pps_mlp_params, seed));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(pps.pps_params), ctypes.sizeof(pps.pps_camera),
            ctypes.sizeof(pps.pps_vertices), ctypes.sizeof(pps.pps_output),
            ctypes.sizeof(pps.pps_stats_t), pps.pps_params.log2_hist_slots.offset,
            pps.pps_vertices.id_base.offset, ctypes.sizeof(pps.pps_tuning),
            pps.pps_tuning.merge.offset, ctypes.sizeof(pps.pps_mlp_params),
            pps.pps_mlp_params.seed.offset]
    assert got == want


def _params(pps, **kw):
    from paper_1902_05942_gb300 import configs
    cfg = configs.small().filters[0]
    p = pps.make_params(cfg)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [("log2_slots", 3), ("log2_slots", 31),
                                         ("max_probes", 0), ("max_probes", 5000),
                                         ("voxel_scale", 0.0), ("voxel_scale", float("nan")),
                                         ("pixel_angle", -1.0), ("lod_min", -126),
                                         ("lod_max", 127), ("accum_mode", 2), ("hist_mode", 3),
                                         ("jitter", 2), ("log2_hist_slots", 2)])
def test_create_rejects_bad_parameters_without_touching_the_gpu(field, value):
    pps, L = _lib()
    p = _params(pps, **{field: value})
    h = ctypes.c_void_p()
    rc = L.pps_create(ctypes.byref(h), ctypes.byref(p))
    assert rc == pps.PPS_EINVAL
    assert h.value is None
    assert pps.last_error()


@pytest.mark.parametrize("bad", [dict(normal_search=257), dict(normal_search=3, normal_in_home_hash=1),
                                 dict(normal_search=1, normal_in_home_hash=0, fallback=2)])
def test_normal_search_checks(bad):
    pps, L = _lib()
    p = _params(pps)
    for k, v in bad.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    assert L.pps_create(ctypes.byref(h), ctypes.byref(p)) == pps.PPS_EINVAL
    assert "normal_search" in pps.last_error()


def test_set_tuning_needs_a_table():
    pps, L = _lib()
    t = pps.pps_tuning()
    assert L.pps_set_tuning(None, ctypes.byref(t)) == pps.PPS_EINVAL
    assert "table" in pps.last_error()


def test_null_arguments_are_rejected():
    pps, L = _lib()
    assert L.pps_create(None, None) == pps.PPS_EINVAL
    assert L.pps_build(None, None, 0, None) == pps.PPS_EINVAL
    assert L.pps_insert(None, None, 0, None, None) == pps.PPS_EINVAL
    assert L.pps_query(None, None, 0, None, None, None) == pps.PPS_EINVAL
    assert L.pps_blend(None, 0.2, None) == pps.PPS_EINVAL
    assert L.pps_destroy(None) == pps.PPS_OK
    assert pps.pps_version().startswith("pps-gb300")


def test_bad_fallback_is_rejected():
    pps, L = _lib()
    p = _params(pps)
    p.fallback = 3
    h = ctypes.c_void_p()
    assert L.pps_create(ctypes.byref(h), ctypes.byref(p)) == pps.PPS_EINVAL
    assert "fallback" in pps.last_error()


def test_eviction_needs_a_history():
    pps, L = _lib()
    p = _params(pps)
    p.hist_evict = 1
    p.hist_mode = 0
    h = ctypes.c_void_p()
    assert L.pps_create(ctypes.byref(h), ctypes.byref(p)) == pps.PPS_EINVAL
    assert "hist_evict" in pps.last_error()


@pytest.mark.parametrize("bad", [dict(hist_migrate=2), dict(hist_migrate=1, hist_mode=0),
                                 dict(hist_migrate=1, hist_mode=1, hist_evict=1)])
def test_migration_needs_a_plain_history(bad):
    pps, L = _lib()
    p = _params(pps)
    for k, v in bad.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    assert L.pps_create(ctypes.byref(h), ctypes.byref(p)) == pps.PPS_EINVAL
    assert "hist_migrate" in pps.last_error()


@pytest.mark.parametrize("kind, limit", [(2, 1000), (-1, 1000), (0, 0), (1, 2000001)])
def test_selftest_wait_checks_its_arguments(kind, limit):
    pps, L = _lib()
    w = ctypes.c_uint32(7)
    assert L.pps_selftest_wait(kind, limit, ctypes.byref(w)) == pps.PPS_EINVAL


@pytest.mark.parametrize("field,value", [("voxel_scale", float("inf")), ("pixel_angle", float("inf")),
                                         ("log2_slots", 21), ("max_probes", 0), ("jitter", 2),
                                         ("hist_mode", 1), ("accum_mode", 1)])
def test_noalloc_checks_parameters_like_create_without_touching_the_gpu(field, value):
    """pps_filter_noalloc applies pps_create's parameter checks (an infinite
    voxel scale or pixel angle is refused as there) plus its own limits, each
    message naming the call."""
    pps, L = _lib()
    p = _params(pps, **{field: value})
    rc = L.pps_filter_noalloc(ctypes.byref(p), ctypes.byref(pps.pps_camera()), 0,
                              ctypes.byref(pps.pps_vertices()), 0,
                              ctypes.byref(pps.pps_output()), None)
    assert rc == pps.PPS_EINVAL
    assert pps.last_error().startswith("pps_filter_noalloc:")


def test_noalloc_null_arguments_name_the_call():
    pps, L = _lib()
    assert L.pps_filter_noalloc(None, None, 0, None, 0, None, None) == pps.PPS_EINVAL
    assert pps.last_error().startswith("pps_filter_noalloc:")
    assert L.pps_noalloc_stats(None, None) == pps.PPS_EINVAL
    assert pps.last_error().startswith("pps_noalloc_stats:")
