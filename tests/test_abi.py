"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/lt.h
declares; host-only calls and argument validation work without a GPU (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def liblt():
    from paper_2609_32920_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lt_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(liblt):
    syms = declared_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(liblt, s), f"{s} declared in lt.h but not exported"
    from paper_2609_32920_gb300 import lt
    assert sorted(lt.EXPORTS) == syms


def test_built_for_sm_103a():
    from paper_2609_32920_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_kernels_compiled_replay_exact():
    """Every pass of a method must take the same discrete decisions for a path (the replay
    regenerates it from its seed): the path kernels are compiled without multiply-add
    contraction, so an expression rounds the same in every kernel it is inlined into."""
    from paper_2609_32920_gb300 import build
    kernels = [u for u in build.UNITS if u[0] == "lt_kernels.cu"]
    assert len(kernels) == 3
    for _, _, extra in kernels:
        assert "-fmad=false" in extra
        assert not any(f.startswith("--use_fast_math") or f.startswith("-use_fast_math") for f in extra)
    assert not any("fast_math" in f for f in build.FLAGS)


def test_host_only_calls(liblt):
    from paper_2609_32920_gb300 import lt
    liblt.lt_version.restype = C.c_char_p
    assert b"sm_103a" in liblt.lt_version()
    o = lt.lt_render_opts()
    o.n_paths, o.max_depth = 1000, 16
    liblt.lt_record_size.restype = C.c_size_t
    liblt.lt_naive_workspace_bytes.restype = C.c_size_t
    assert liblt.lt_record_size(C.byref(o)) == 32
    assert liblt.lt_naive_workspace_bytes(C.byref(o)) == 4096 + 1000 * 16 * 32


def test_argument_validation_without_gpu(liblt):
    liblt.lt_last_error.restype = C.c_char_p
    out = C.c_void_p()
    assert liblt.lt_scene_create(None, None, C.byref(out)) == 1
    assert b"desc" in liblt.lt_last_error()
    assert liblt.lt_scene_create(None, None, None) == 1
    assert liblt.lt_primal(None, None, None, 0, None, None, 0, None) == 1
    assert liblt.lt_backward_lrb3(None, None, None, None, None, None) == 1
    assert liblt.lt_backward_reslrb(None, None, None, None, None, None, None) == 1
    assert liblt.lt_backward_naive(None, None, None, None, None, 0, None, None) == 1
    assert liblt.lt_film_l2(None, None, 0, None, None, None) == 1
    assert liblt.lt_scene_refit(None, None, None) == 1
    assert liblt.lt_sync_status(None, None) == 1


def test_size_queries_refuse_path_counts_that_would_wrap(liblt):
    """Byte counts are derived from n_paths; beyond LT_MAX_PATHS (2^40) the size queries
    return 0 instead of a wrapped-around size (and every call rejects the opts)."""
    from paper_2609_32920_gb300 import lt
    liblt.lt_naive_workspace_bytes.restype = C.c_size_t
    liblt.lt_lrb2_buffer_bytes.restype = C.c_size_t
    liblt.lt_lrb3_state_bytes.restype = C.c_size_t
    o = lt.lt_render_opts()
    o.max_depth = 64
    o.n_paths = 1 << 40
    assert liblt.lt_naive_workspace_bytes(C.byref(o)) == 256 * ((4 * (1 << 40) + 255) // 256) + (1 << 40) * 64 * 32
    for n in ((1 << 40) + 1, 1 << 62):
        o.n_paths = n
        assert liblt.lt_naive_workspace_bytes(C.byref(o)) == 0
        assert liblt.lt_lrb2_buffer_bytes(C.byref(o)) == 0
        assert liblt.lt_lrb3_state_bytes(C.byref(o)) == 0


def test_lrb3_state_is_constant_in_depth_and_48_bytes_per_path(liblt):
    """The separate-kernel LRB-3 state (Sec. 4.3; Results, "Memory Scaling"): per path the validity
    mask, delta_total, a list entry, the first connection and the path order (48 B), plus the
    counting sort's fixed 4.2 MB; nothing grows with the path depth."""
    from paper_2609_32920_gb300 import lt
    liblt.lt_lrb3_state_bytes.restype = C.c_size_t
    o = lt.lt_render_opts()
    sizes = {}
    for n in (1 << 20, 1 << 24):
        per_depth = set()
        for D in (1, 8, 64):
            o.n_paths, o.max_depth = n, D
            per_depth.add(liblt.lt_lrb3_state_bytes(C.byref(o)))
        assert len(per_depth) == 1, per_depth
        sizes[n] = per_depth.pop()
    assert sizes[1 << 24] - sizes[1 << 20] == 48 * ((1 << 24) - (1 << 20))
    fixed = sizes[1 << 20] - 48 * (1 << 20)
    sort_area = 4 * 4096 * 257
    assert sort_area <= fixed <= sort_area + 8 * 256


def test_binding_structs_match_the_header_layout(tmp_path):
    """The binding's ctypes structures and include/lt.h describe the same bytes: every field
    the binding names exists in the C struct at the same offset, and the sizes agree (so
    the C struct has no field the binding lacks).  Compiled with the host C compiler."""
    import subprocess
    from paper_2609_32920_gb300 import lt
    structs = [lt.lt_scene_desc, lt.lt_params, lt.lt_render_opts, lt.lt_grads, lt.lt_batch_item,
               lt.lt_bidir_opts, lt.lt_batch_config]
    lines = ["#include <stdio.h>", '#include "lt.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'  printf("%s size %zu\\n", "{S.__name__}", sizeof({S.__name__}));')
        for name, _ in S._fields_:
            lines.append(f'  printf("%s.%s %zu\\n", "{S.__name__}", "{name}", offsetof({S.__name__}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for S in structs:
        assert int(got[f"{S.__name__} size"]) == C.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert int(got[f"{S.__name__}.{name}"]) == getattr(S, name).offset, (S.__name__, name)
