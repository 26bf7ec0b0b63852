"""C ABI checks that need no GPU: the library loads, exports every entry point the header
declares, its structs have the layout the binding assumes, and argument errors are
reported before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2408_11929_gb300 as hh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hh.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return hh.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", hh.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hh_\w+)", out))
    for name in names:
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(hh.EXPORTS) == set(names)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hh.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(hh_opts), sizeof(hh_result),'
                    ' sizeof(hh_stats), offsetof(hh_opts, stream), offsetof(hh_stats, sweep_steps),'
                    ' offsetof(hh_result, status), offsetof(hh_stats, gemm_flops), offsetof(hh_stats, gs_flops),'
                    ' offsetof(hh_opts, twisted), offsetof(hh_stats, twisted));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(hh.hh_opts), ctypes.sizeof(hh.hh_result), ctypes.sizeof(hh.hh_stats),
                    hh.hh_opts.stream.offset, hh.hh_stats.sweep_steps.offset, hh.hh_result.status.offset,
                    hh.hh_stats.gemm_flops.offset, hh.hh_stats.gs_flops.offset, hh.hh_opts.twisted.offset,
                    hh.hh_stats.twisted.offset]


def test_default_opts(lib):
    o = hh.default_opts()
    assert o.precision == hh.HH_PREC_FP64 and o.maxit == 200 and o.deflate_eta == 1e-10
    assert o.use_graph == 1 and o.timeout_cycles > 0 and o.bcr_depth == 0 and o.gs_passes == 2
    assert o.serve_slots == 8 and o.tensor_cores == 1 and o.autotune == 1 and o.fuse_chains == 1
    assert o.overlap_steps == 1 and o.twisted == 1


@pytest.mark.parametrize("k,n,strips,dirs,kw", [
    (10.0, 30, 4, 15, {}),          # n not a multiple of strips
    (10.0, 32, 32, 15, {}),         # one node line per strip
    (-1.0, 32, 4, 15, {}),          # k <= 0
    (10.0, 32, 4, 0, {}),           # no direction
    (10.0, 32, 4, 16, {}),          # unknown direction bit
    (10.0, 32, 4, 15, {"maxit": 0}),
    (10.0, 32, 4, 15, {"bcr_depth": 4}),   # R = 8 allows at most 3 levels of cyclic reduction
    (10.0, 32, 4, 15, {"interface_form": 2}),
    (10.0, 36, 4, 15, {"bcr_depth": 2}),   # R = 9 is odd: no cyclic reduction
    (10.0, 32, 4, 15, {"bcr_depth": -2}),
    (10.0, 32, 4, 15, {"gs_passes": 3}),
    (10.0, 32, 4, 15, {"gs_tensor": 2}),
    (10.0, 32, 4, 15, {"twisted": 2}),
    (10.0, 32, 4, 15, {"twisted": -2}),
    (10.0, 32, 4, 15, {"discretization": 2}),
    (10.0, 32, 4, 15, {"discretization": 1, "precision": 1}),   # the five-point mode is FP64 only
    (10.0, 32, 4, 15, {"serve_slots": 0}),
    (10.0, 32, 4, 15, {"serve_slots": 257}),
    (10.0, 1, 1, 15, {}),
])
def test_setup_rejects_bad_arguments(lib, k, n, strips, dirs, kw):
    o = hh.default_opts(**kw)
    h = ctypes.c_void_p()
    st = lib.hh_setup(k, n, strips, dirs, ctypes.byref(o), ctypes.byref(h))
    assert st == hh.HH_EINVAL
    assert h.value is None
    assert lib.hh_last_error()


def test_null_arguments(lib):
    o = hh.default_opts()
    assert lib.hh_setup(10.0, 32, 4, 15, ctypes.byref(o), None) == hh.HH_EINVAL
    assert lib.hh_solve(None, None, None, 1e-8, None) == hh.HH_EINVAL
    assert lib.hh_solve_batch(None, 1, None, None, 1e-8, None) == hh.HH_EINVAL
    assert lib.hh_apply_operator(None, 1, None, None) == hh.HH_EINVAL
    assert lib.hh_gram_schmidt_pass(None, 1, None, 1, None, None) == hh.HH_EINVAL
    assert lib.hh_get_stats(None, None) == hh.HH_EINVAL
    res = hh.hh_result()
    assert lib.hh_poll(ctypes.c_uint64(987654321), ctypes.byref(res)) == hh.HH_EINVAL
    lib.hh_destroy(None)


def test_dirs_mask():
    assert hh.dirs_mask("LR+RL+BT+TB") == 15
    assert hh.dirs_mask("LR+BT") == hh.HH_DIR_LR | hh.HH_DIR_BT
    assert hh.dirs_mask(4) == 4
