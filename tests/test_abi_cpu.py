"""The C-ABI library loads on a machine without a GPU, exports every entry point
that include/m3e.h declares, and rejects bad parameters before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "m3e.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(m3e_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401
    from paper_2206_11535_gb300 import build
    return C.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("m3e_create", "m3e_destroy", "m3e_select_frames", "m3e_select_frames_plain",
              "m3e_select_frames_host", "m3e_select_frames_debug", "m3e_check", "m3e_last_error_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_config_checks_run_before_cuda(lib, cfg):
    from paper_2206_11535_gb300 import m3e
    h = C.c_void_p()
    bad = m3e.config_from_json(cfg)
    bad.size = 7
    assert m3e.lib.m3e_create(C.byref(bad), 0, C.byref(h)) == m3e.EINVAL
    assert b"size" in m3e.lib.m3e_last_error_string()
    for field, val in (("max_hits", 5000), ("max_triplets", 2000), ("max_tracks", 300), ("max_combos", 99999)):
        c = m3e.config_from_json(cfg, **{field: val})
        assert m3e.lib.m3e_create(C.byref(c), 0, C.byref(h)) == m3e.EINVAL, field
    c = m3e.config_from_json(cfg)
    c.r_mm[2] = 20.0
    assert m3e.lib.m3e_create(C.byref(c), 0, C.byref(h)) == m3e.EINVAL
    assert m3e.lib.m3e_select_frames(None, None, None, 0, None, None, None, None) == m3e.EINVAL
    assert m3e.lib.m3e_version() == 100


def test_config_struct_layout_matches_header():
    """Offsets of the ctypes mirror follow the C declaration order."""
    from paper_2206_11535_gb300 import m3e
    names = [f[0] for f in m3e.Config._fields_]
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = txt[txt.index("typedef struct {\n  uint32_t size;"):txt.index("} m3e_config;")]
    decl = re.findall(r"(\w+)(?:\[\d+\])?\s*[,;]", body)
    assert [n for n in decl if n in names] == names


def _c_layout(struct: str, fields: list[str], tmp_path) -> list[int]:
    """sizeof and offsetof of a header struct, from a C program compiled here with gcc."""
    import subprocess
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "m3e.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                           str(src), "-o", str(exe)])
    return [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]


@pytest.mark.parametrize("name,struct", [("Result", "m3e_result"), ("StreamParams", "m3e_stream_params"),
                                         ("StreamStatus", "m3e_stream_status"), ("ReplayStats", "m3e_replay_stats"),
                                         ("Tuning", "m3e_tuning"), ("Config", "m3e_config"),
                                         ("Dump", "m3e_dump")])
def test_ctypes_mirrors_match_the_c_layout(name, struct, tmp_path):
    import shutil
    if not shutil.which("gcc") or not os.path.exists("/usr/local/cuda/include/cuda_runtime.h"):
        pytest.skip("gcc or the CUDA headers are missing")
    from paper_2206_11535_gb300 import m3e
    cls = getattr(m3e, name)
    fields = [f[0] for f in cls._fields_]
    want = _c_layout(struct, fields, tmp_path)
    got = [C.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_stream_entry_points_check_arguments(lib):
    from paper_2206_11535_gb300 import m3e
    L = m3e.lib
    slot = m3e.Result()
    assert L.m3e_stream_submit(None, None, 0, 0, C.addressof(slot)) == m3e.EINVAL
    assert L.m3e_stream_poll(None, None) == m3e.EINVAL
    assert L.m3e_stream_drain(None, 0) == m3e.EINVAL
    assert L.m3e_stream_close(None) == m3e.EINVAL
    assert L.m3e_stream_open(None, None) == m3e.EINVAL
    assert L.m3e_stream_replay(None, None, None, 0, 1.0, 0, None, None, None, None, None) == m3e.EINVAL


def test_stats_buffer_matches_the_c_layout(tmp_path):
    """m3e_stats is read as an int64 buffer in STATS_FIELDS order, then reasons[8]."""
    import shutil
    if not shutil.which("gcc") or not os.path.exists("/usr/local/cuda/include/cuda_runtime.h"):
        pytest.skip("gcc or the CUDA headers are missing")
    from paper_2206_11535_gb300 import m3e
    fields = list(m3e.STATS_FIELDS) + ["reasons"]
    want = _c_layout("m3e_stats", fields, tmp_path)
    assert want == [8 * m3e.N_STATS] + [8 * k for k in range(len(fields))]
