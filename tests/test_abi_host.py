"""Host-side checks of the C ABI (CPU only, no GPU compute).

The library must build for sm_103a, load, export every entry point that
include/rg.h declares, and reject bad arguments before touching the GPU.
"""
import ctypes as C
import os
import re

import pytest

from paper_2608_15785_gb300 import binding
from paper_2608_15785_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return binding.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["rg_scene_create", "rg_scene_destroy", "rg_render", "rg_render_batch", "rg_backward",
                 "rg_submit", "rg_poll", "rg_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert sorted(binding.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n


def test_version_and_error_string(L):
    assert L.rg_version() == 100
    assert isinstance(L.rg_last_error(), bytes)


def test_bad_arguments_are_rejected_without_a_gpu(L):
    out = C.c_void_p()
    assert L.rg_scene_create(None, None, C.byref(out)) == 1  # RG_ERR_INVALID_ARG
    assert b"NULL" in L.rg_last_error()
    d = binding.RgSceneDesc()
    d.n = -5
    assert L.rg_scene_create(C.byref(d), None, C.byref(out)) == 1
    d.n, d.sh_degree = 10, 4
    assert L.rg_scene_create(C.byref(d), None, C.byref(out)) == 1
    d.sh_degree = 3
    assert L.rg_scene_create(C.byref(d), None, C.byref(out)) == 1  # NULL attribute pointers
    assert L.rg_render(None, None, None, None, None, None) == 1
    assert L.rg_render_batch(None, None, None, 0, None, None, None) == 0  # empty batch
    assert L.rg_render_batch(None, None, None, 2, None, None, None) == 1
    assert L.rg_backward(None, None, None, None, None, None) == 1  # NULL arguments
    assert L.rg_submit(None, None, 0, None) == 1
    assert L.rg_poll(None, 0, None) == 1
    assert L.rg_server_create(None, 0, None, None) == 1
    assert L.rg_server_destroy(None) == 0
    assert L.rg_eval_fast_exp(None, None, -1, None) == 1
    assert L.rg_stage_times(None, None, None) == 1
    assert L.rg_scene_destroy(None) == 0


def test_scene_files_are_validated_before_touching_a_gpu(L, tmp_path):
    import struct
    out = C.c_void_p()
    assert L.rg_scene_save(None, b"x") == 1
    assert L.rg_scene_load(None, None, C.byref(out)) == 1
    assert L.rg_scene_load(str(tmp_path / "missing.rgs").encode(), None, C.byref(out)) == 1
    junk = tmp_path / "junk.rgs"
    junk.write_bytes(b"not a scene file at all" * 10)
    assert L.rg_scene_load(str(junk).encode(), None, C.byref(out)) == 1
    assert b"magic" in L.rg_last_error()
    # a valid header (n = 10, compact storage) whose buffers are missing
    hdr = b"RGSCENE1" + struct.pack("<IIqii", 1, 2, 10, 3, 0) + struct.pack("<12f", *([0.1] * 12)) + bytes(32)
    short = tmp_path / "short.rgs"
    short.write_bytes(hdr + bytes(100))
    assert L.rg_scene_load(str(short).encode(), None, C.byref(out)) == 1
    assert b"size" in L.rg_last_error()
    assert not out.value


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the public structs have the C compiler's sizes and offsets."""
    import subprocess
    structs = {"rg_camera": binding.RgCamera, "rg_scene_desc": binding.RgSceneDesc,
               "rg_render_opts": binding.RgOpts, "rg_stats": binding.RgStats, "rg_grads": binding.RgGrads,
               "rg_server_config": binding.RgServerConfig, "rg_server_stats_t": binding.RgServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_noalloc_sort_rejects_misaligned_arrays_before_any_launch(L):
    """rg_sort_pairs_noalloc reads keys 16 bytes at a time: pointers off a 16-byte boundary
    are refused on the host (no CUDA call is made, so this runs without a GPU; the
    addresses are never dereferenced)."""
    for keys, vals in ((0x10004, 0x20000), (0x10000, 0x20008), (0x1000c, 0x2000c)):
        st = L.rg_sort_pairs_noalloc(C.c_void_p(keys), C.c_void_p(vals), 1000, 32, None, None)
        assert st == 1, st  # RG_ERR_INVALID_ARG
        assert b"16-byte" in L.rg_last_error()
    assert L.rg_sort_pairs_noalloc(C.c_void_p(0x10000), C.c_void_p(0x20000), -1, 32, None, None) == 1
    assert L.rg_sort_pairs_noalloc(C.c_void_p(0x10000), C.c_void_p(0x20000), 10, 12, None, None) == 1


def test_binding_constants_match_the_header():
    """Every RG_* integer constant of include/rg.h has the same value in the binding."""
    src = open(os.path.join(ROOT, "include", "rg.h")).read()
    consts = {}
    for name, expr in re.findall(r"#define (RG_[A-Z0-9_]+)\s+(\(1u << \d+\)|\d+u?)(?=\s|$)", src):
        m = re.match(r"\(1u << (\d+)\)", expr)
        consts[name] = (1 << int(m.group(1))) if m else int(expr.rstrip("u"))
    assert "RG_FLAG_ORDERED_FRONT_END" in consts and "RG_INSPECT_KEYS" in consts
    for name, v in consts.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == v, name
    flags = [n for n in consts if n.startswith("RG_FLAG_")]
    assert all(hasattr(binding, n) for n in flags), [n for n in flags if not hasattr(binding, n)]
    assert len({consts[n] for n in flags}) == len(flags)  # no two flags share a bit
