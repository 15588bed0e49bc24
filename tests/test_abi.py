"""Host-side checks of the C ABI boundary (no GPU needed): the shared library
builds for sm_103a, loads, exports every function include/spgemm1d.h declares,
and the ctypes structures of the binding have the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spgemm1d.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2408_14558_gb300 import build
    build.build()
    import paper_2408_14558_gb300 as g
    return g.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spgemm_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spgemm_plan", "spgemm_symbolic", "spgemm_numeric", "spgemm_1d_multiply",
                     "spgemm_plan_stats", "spgemm_plan_destroy", "spgemm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    import paper_2408_14558_gb300 as g
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "spgemm1d.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(spg_csc), sizeof(spg_options), sizeof(spg_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(spg_csc, colptr), offsetof(spg_options, stream),
         offsetof(spg_options, learned_slack), offsetof(spg_stats, ms_plan));
  printf("%zu %zu\\n", sizeof(spg_outer_stats), offsetof(spg_outer_stats, ms_split));
  printf("%zu %zu\\n", offsetof(spg_options, mask), offsetof(spg_options, mask_complement));
  printf("%zu %zu\\n", sizeof(spg_bc_stats), offsetof(spg_bc_stats, nnzC_total));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = list(map(int, out))
    assert sizes[0] == ctypes.sizeof(g.spg_csc)
    assert sizes[1] == ctypes.sizeof(g.spg_options)
    assert sizes[2] == ctypes.sizeof(g.spg_stats)
    assert sizes[3] == g.spg_csc.colptr.offset
    assert sizes[4] == g.spg_options.stream.offset
    assert sizes[5] == g.spg_options.learned_slack.offset
    assert sizes[6] == g.spg_stats.ms_plan.offset
    assert sizes[7] == ctypes.sizeof(g.spg_outer_stats)
    assert sizes[8] == g.spg_outer_stats.ms_split.offset
    assert sizes[9] == g.spg_options.mask.offset
    assert sizes[10] == g.spg_options.mask_complement.offset
    assert sizes[11] == ctypes.sizeof(g.spg_bc_stats)
    assert sizes[12] == g.spg_bc_stats.nnzC_total.offset


def test_default_options(lib):
    import paper_2408_14558_gb300 as g
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    assert (o.P, o.b, o.validate, o.sizing) == (1, 1024, 1, g.SPG_SIZING_EXACT)


def test_argument_errors_need_no_gpu(lib):
    """Argument checks run before any CUDA call."""
    import paper_2408_14558_gb300 as g
    A = g.spg_csc(4, 5, 0, 0, 0, 0, 0, 1, None, None)
    B = g.spg_csc(6, 3, 0, 0, 0, 0, 0, 1, None, None)      # 5 != 6
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    h = ctypes.c_void_p()
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    assert "dimension mismatch" in g.spgemm_last_error()
    B.nrows = 5
    o.P = 0
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    o.P = 2
    B.val_type = g.SPG_VAL_I64
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    assert not h.value


def test_outer_multiply_argument_errors_need_no_gpu(lib):
    """spgemm_outer_multiply rejects bad arguments before any CUDA call."""
    import paper_2408_14558_gb300 as g
    A = g.spg_csc(4, 5, 0, 0, 0, 0, 0, 1, None, None)
    B = g.spg_csc(6, 3, 0, 0, 0, 0, 0, 1, None, None)      # 5 != 6
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    C = g.spg_csc()
    f = lib.spgemm_outer_multiply
    f.argtypes = [ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_options),
                  ctypes.POINTER(g.spg_csc), ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(C), None) == g.SPG_INVALID_ARGUMENT
    B.nrows = 5
    o.P = 0
    assert f(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(C), None) == g.SPG_INVALID_ARGUMENT
    assert f(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), None, None) == g.SPG_INVALID_ARGUMENT


def test_split_and_block_argument_errors_need_no_gpu(lib):
    import paper_2408_14558_gb300 as g
    assert lib.spgemm_plan_blocks(None, None, None, None, None) == g.SPG_INVALID_ARGUMENT
    A = g.spg_csc(4, 5, 0, 0, 0, 0, 0, 1, None, None)
    B = g.spg_csc(5, 3, 0, 0, 0, 0, 0, 1, None, None)
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    o.split = 7
    h = ctypes.c_void_p()
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    assert "split" in g.spgemm_last_error()


def test_bc_argument_errors_need_no_gpu(lib):
    import paper_2408_14558_gb300 as g
    A = g.spg_csc(4, 5, 0, 0, 0, 0, 0, 1, None, None)       # not square, no arrays
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    f = lib.spgemm_bc_batch
    f.argtypes = [ctypes.POINTER(g.spg_csc), ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(g.spg_options),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(A), None, 0, ctypes.byref(o), None, None, 0, None) == g.SPG_INVALID_ARGUMENT
    fake = ctypes.c_double(0.0)
    assert f(ctypes.byref(A), None, 0, ctypes.byref(o), ctypes.addressof(fake), None, 0, None) == g.SPG_INVALID_ARGUMENT
    A.nrows = 5
    assert f(ctypes.byref(A), None, 3, ctypes.byref(o), ctypes.addressof(fake), None, 0, None) == g.SPG_INVALID_ARGUMENT


def test_mask_argument_errors_need_no_gpu(lib):
    """A mask with too few words per column, a complement flag other than
    0 / 1, or a mask with learned sizing, the outer-product form or the
    betweenness batch is rejected before any CUDA call."""
    import paper_2408_14558_gb300 as g
    A = g.spg_csc(70, 5, 0, 0, 0, 0, 0, 1, None, None)
    B = g.spg_csc(5, 3, 0, 0, 0, 0, 0, 1, None, None)
    words = (ctypes.c_uint32 * 16)()
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    assert o.mask is None and o.mask_words == 0 and o.mask_complement == 0
    o.mask = ctypes.addressof(words)
    o.mask_words = 2                         # 70 rows need 3 words
    h = ctypes.c_void_p()
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    assert "mask_words" in g.spgemm_last_error()
    o.mask_words = 3
    o.mask_complement = 2
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    o.mask_complement = 1
    o.sizing = g.SPG_SIZING_LEARNED
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_INVALID_ARGUMENT
    assert "learned" in g.spgemm_last_error()
    assert not h.value
    o.sizing = g.SPG_SIZING_EXACT
    C = g.spg_csc()
    f = lib.spgemm_outer_multiply
    f.argtypes = [ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_options),
                  ctypes.POINTER(g.spg_csc), ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(C), None) == g.SPG_INVALID_ARGUMENT
    assert "outer" in g.spgemm_last_error()
    fb = lib.spgemm_bc_batch
    fb.argtypes = [ctypes.POINTER(g.spg_csc), ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(g.spg_options),
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    fb.restype = ctypes.c_int
    G = g.spg_csc(5, 5, 0, 0, 0, 0, 0, 1, None, None)
    fake = ctypes.c_double(0.0)
    assert fb(ctypes.byref(G), None, 0, ctypes.byref(o), ctypes.addressof(fake), None, 0, None) == g.SPG_INVALID_ARGUMENT
    assert "mask" in g.spgemm_last_error()


def test_host_multiply_argument_errors_need_no_gpu(lib):
    """spgemm_1d_multiply_host checks its arguments (and the host column
    pointers' first and last entries) before any CUDA call."""
    import numpy as np
    import paper_2408_14558_gb300 as g
    f = lib.spgemm_1d_multiply_host
    f.argtypes = [ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_csc), ctypes.POINTER(g.spg_options), ctypes.c_int32,
                  g.HOST_ALLOC_FN, g.HOST_FREE_FN, ctypes.c_void_p, ctypes.POINTER(g.spg_csc)]
    f.restype = ctypes.c_int
    cp = np.array([0, 2, 3], dtype=np.int64)
    ri = np.array([0, 1, 1], dtype=np.int32)
    va = np.ones(3)
    A = g.spg_csc(2, 2, 3, 1, 0, 0, 0, cp.ctypes.data, ri.ctypes.data, va.ctypes.data)
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    C = g.spg_csc()
    never = g.HOST_ALLOC_FN(lambda n, ctx: None)
    nofree = g.HOST_FREE_FN(lambda p, n, ctx: None)
    null_alloc = ctypes.cast(None, g.HOST_ALLOC_FN)
    assert f(ctypes.byref(A), ctypes.byref(A), ctypes.byref(o), 1, null_alloc, nofree, None, ctypes.byref(C)) \
        == g.SPG_INVALID_ARGUMENT
    assert f(ctypes.byref(A), ctypes.byref(A), ctypes.byref(o), 0, never, nofree, None, ctypes.byref(C)) \
        == g.SPG_INVALID_ARGUMENT
    bad = np.array([0, 2, 2], dtype=np.int64)                   # last pointer != nnz
    Ab = g.spg_csc(2, 2, 3, 1, 0, 0, 0, bad.ctypes.data, ri.ctypes.data, va.ctypes.data)
    assert f(ctypes.byref(Ab), ctypes.byref(A), ctypes.byref(o), 1, never, nofree, None, ctypes.byref(C)) \
        == g.SPG_INVALID_ARGUMENT
    B3 = g.spg_csc(3, 2, 3, 1, 0, 0, 0, cp.ctypes.data, ri.ctypes.data, va.ctypes.data)   # 2 != 3
    assert f(ctypes.byref(A), ctypes.byref(B3), ctypes.byref(o), 1, never, nofree, None, ctypes.byref(C)) \
        == g.SPG_INVALID_ARGUMENT
    assert "dimension mismatch" in g.spgemm_last_error()
    o.sizing = g.SPG_SIZING_LEARNED
    assert f(ctypes.byref(A), ctypes.byref(A), ctypes.byref(o), 1, never, nofree, None, ctypes.byref(C)) \
        == g.SPG_INVALID_ARGUMENT
    assert C.colptr is None


def test_host_csc_marshalling():
    """The host-buffer call's descriptors: addresses, sizes and type codes of
    numpy arrays and CPU tensors."""
    import numpy as np
    import torch
    import paper_2408_14558_gb300 as g
    import synth
    M = synth.random_sparse(7, 5, 0.4, np.random.default_rng(0), values="i64")
    d = g._host_csc(M)
    assert (d.nrows, d.ncols, d.nnz) == (7, 5, M.nnz)
    assert (d.ptr_type, d.idx_type, d.val_type) == (g.SPG_IDX_I64, g.SPG_IDX_I32, g.SPG_VAL_I64)
    assert d.colptr == M.colptr.ctypes.data and d.rowidx == M.rowidx.ctypes.data
    T = synth.CSC(7, 5, torch.from_numpy(M.colptr.astype(np.int32)), torch.from_numpy(M.rowidx.astype(np.int64)),
                  torch.from_numpy(M.vals.astype(np.float64)))
    d = g._host_csc(T)
    assert (d.ptr_type, d.idx_type, d.val_type) == (g.SPG_IDX_I32, g.SPG_IDX_I64, g.SPG_VAL_F64)
    assert d.vals == T.vals.data_ptr()
    E = synth.CSC(3, 2, np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(0))
    d = g._host_csc(E)
    assert d.nnz == 0 and d.rowidx is None and d.vals is None


def test_semiring_other_than_plus_times_is_unsupported(lib):
    import paper_2408_14558_gb300 as g
    A = g.spg_csc(4, 5, 0, 0, 0, 0, 0, 1, None, None)
    B = g.spg_csc(5, 3, 0, 0, 0, 0, 0, 1, None, None)
    o = g.spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    assert o.semiring == g.SPG_SEMIRING_PLUS_TIMES
    o.semiring = 1
    h = ctypes.c_void_p()
    assert lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), ctypes.byref(o), ctypes.byref(h)) == g.SPG_UNSUPPORTED
    assert "semiring" in g.spgemm_last_error() and not h.value
