"""Python binding of the GB300 sparsity-aware 1D SpGEMM library (libspgemm1d.so).

Argument marshalling only: every step of C = A*B runs in the CUDA kernels behind
the C ABI declared in ``include/spgemm1d.h``.  PyTorch provides device memory
(through the allocator callbacks, so the library's workspace comes from the
caching allocator) and the stream (torch's current stream).  The functions keep
the C names:

    spgemm_plan, spgemm_symbolic, spgemm_numeric, spgemm_1d_multiply,
    spgemm_plan_stats, spgemm_plan_destroy, spgemm_last_error,
    spgemm_plan_export

There is no CPU fallback: if the shared library is missing or fails to load,
the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspgemm1d.so")

SPG_OK, SPG_INVALID_ARGUMENT, SPG_INVALID_INPUT, SPG_OUT_OF_MEMORY = 0, 1, 2, 3
SPG_CUDA_ERROR, SPG_TIMEOUT, SPG_UNSUPPORTED, SPG_OVERFLOW_RECOMPUTED = 4, 5, 6, 7
SPG_IDX_I32, SPG_IDX_I64 = 0, 1
SPG_VAL_F64, SPG_VAL_I32, SPG_VAL_I64 = 0, 1, 2
SPG_SIZING_EXACT, SPG_SIZING_LEARNED = 0, 1
SPG_SPLIT_UNIFORM, SPG_SPLIT_FLOPS = 0, 1
SPG_SEMIRING_PLUS_TIMES = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARGUMENT", 2: "INVALID_INPUT", 3: "OUT_OF_MEMORY",
                4: "CUDA_ERROR", 5: "TIMEOUT", 6: "UNSUPPORTED", 7: "OVERFLOW_RECOMPUTED"}


class SpgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class spg_csc(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("ptr_type", ctypes.c_int32), ("idx_type", ctypes.c_int32),
                ("val_type", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class spg_options(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("sizing", ctypes.c_int32), ("b", ctypes.c_int64),
                ("validate", ctypes.c_int32), ("light_max", ctypes.c_int32),
                ("slab_rows", ctypes.c_int32), ("split", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("model", ctypes.c_void_p),
                ("learned_slack", ctypes.c_double), ("mask", ctypes.c_void_p), ("mask_words", ctypes.c_int64),
                ("mask_complement", ctypes.c_int32), ("semiring", ctypes.c_int32)]


class spg_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "m", "k", "n", "nnzA", "nnzB", "P", "b", "products", "nnzC", "sum_H", "sum_dtilde",
        "fetch_blocks_total", "fetch_blocks_chosen", "gathered_nnz_exact", "gathered_nnz_block",
        "light_columns", "heavy_columns", "heavy_items", "empty_columns", "recomputed_columns",
        "nnzB_heavy", "nnzC_heavy", "kernel_launches", "learned_capacity")] + [
        (name, ctypes.c_double) for name in ("ms_plan", "ms_symbolic", "ms_numeric", "ms_gather", "ms_sym_light",
                                             "ms_sym_heavy", "ms_num_light", "ms_num_heavy")] + [
        ("gathered_nnz_remote", ctypes.c_int64)]


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libspgemm1d.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} is missing: build it with paper_2408_14558_gb300.build.build()")
            lib = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.spgemm_default_options.argtypes = [ctypes.POINTER(spg_options)]
            lib.spgemm_default_options.restype = None
            lib.spgemm_plan.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                        ctypes.POINTER(spg_options), ctypes.POINTER(vp)]
            lib.spgemm_symbolic.argtypes = [vp, vp, ctypes.POINTER(i64)]
            lib.spgemm_numeric.argtypes = [vp, ctypes.POINTER(spg_csc)]
            lib.spgemm_1d_multiply.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                               ctypes.POINTER(spg_options), ctypes.POINTER(spg_csc)]
            lib.spgemm_plan_stats.argtypes = [vp, ctypes.POINTER(spg_stats)]
            lib.spgemm_plan_destroy.argtypes = [vp]
            lib.spgemm_last_error.restype = ctypes.c_char_p
            lib.spgemm_plan_export.argtypes = [vp, i32, vp, vp, ctypes.POINTER(i64), vp, vp, vp, vp, vp]
            lib.spgemm_count_noalloc.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc), vp, vp]
            for name in ("spgemm_plan", "spgemm_symbolic", "spgemm_numeric", "spgemm_1d_multiply",
                         "spgemm_plan_stats", "spgemm_plan_destroy", "spgemm_plan_export",
                         "spgemm_count_noalloc"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def spgemm_last_error() -> str:
    return load_library().spgemm_last_error().decode()


def _check(status: int):
    if status not in (SPG_OK, SPG_OVERFLOW_RECOMPUTED):
        raise SpgError(status, spgemm_last_error())
    return status


# ------------------------------------------------------------------ matrices

_IDX = {torch.int32: SPG_IDX_I32, torch.int64: SPG_IDX_I64}
_VAL = {torch.float64: SPG_VAL_F64, torch.int32: SPG_VAL_I32, torch.int64: SPG_VAL_I64}


@dataclass
class DeviceCSC:
    """A CSC matrix whose three arrays are CUDA tensors."""
    nrows: int
    ncols: int
    colptr: torch.Tensor
    rowidx: torch.Tensor
    vals: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    def as_c(self) -> spg_csc:
        for t in (self.colptr, self.rowidx, self.vals):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("DeviceCSC arrays must be contiguous CUDA tensors")
        if self.colptr.numel() < self.ncols + 1 or self.vals.numel() != self.rowidx.numel():
            raise ValueError(f"DeviceCSC needs ncols + 1 = {self.ncols + 1} column pointers (has "
                             f"{self.colptr.numel()}) and one value per row id ({self.vals.numel()} values, "
                             f"{self.rowidx.numel()} row ids)")
        return spg_csc(self.nrows, self.ncols, self.nnz, _IDX[self.colptr.dtype], _IDX[self.rowidx.dtype],
                       _VAL[self.vals.dtype], 0, self.colptr.data_ptr(),
                       self.rowidx.data_ptr() if self.nnz else None, self.vals.data_ptr() if self.nnz else None)

    def to_host(self):
        """(colptr, rowidx, vals) as numpy arrays."""
        return self.colptr.cpu().numpy(), self.rowidx.cpu().numpy(), self.vals.cpu().numpy()


def to_device(M, device="cuda", ptr_dtype=None, idx_dtype=None, val_dtype=None, pin=False) -> DeviceCSC:
    """Copy a host CSC (anything with nrows, ncols, colptr, rowidx, vals numpy
    arrays) to the GPU, optionally converting the array types."""
    def conv(a, dt):
        t = torch.from_numpy(a)
        if dt is not None:
            t = t.to(dt)
        if pin:
            t = t.pin_memory()
        return t.to(device, non_blocking=pin)
    return DeviceCSC(int(M.nrows), int(M.ncols), conv(M.colptr, ptr_dtype), conv(M.rowidx, idx_dtype),
                     conv(M.vals, val_dtype))


# --------------------------------------------------------- allocator bridge

class _TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        self.device = device
        self.live = {}
        self.lock = threading.Lock()
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx, stream):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except RuntimeError:
            return None
        with self.lock:
            self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, nbytes, ctx, stream):
        with self.lock:
            self.live.pop(ptr, None)

    def adopt(self, ptr: int, nbytes: int, dtype, count: int) -> torch.Tensor:
        """Turn an allocation made through the callback into a typed tensor."""
        with self.lock:
            t = self.live.pop(ptr)
        return t[: count * torch.empty(0, dtype=dtype).element_size()].view(dtype) if count else \
            torch.empty(0, dtype=dtype, device=self.device)


def _mask_fields(mask, nrows, ncols):
    """(pointer, words per column) of an output mask: a CUDA int32 tensor of
    shape (ncols of C, words >= ceil(nrows / 32)), row-major, bit r of row j's
    words = row r of column j (least significant bit first)."""
    if mask is None:
        return None, 0
    if mask.dtype != torch.int32 or mask.dim() != 2 or not mask.is_cuda or not mask.is_contiguous():
        raise ValueError("mask must be a contiguous 2-D CUDA int32 tensor (columns x words)")
    if mask.shape[1] < (nrows + 31) // 32 or mask.shape[0] < ncols:
        raise ValueError(f"mask needs {ncols} columns of >= {(nrows + 31) // 32} words, has shape "
                         f"{tuple(mask.shape)}")
    return mask.data_ptr(), int(mask.shape[1])


def make_options(P=1, b=1024, stream=None, validate=True, light_max=0, slab_rows=0, sizing=SPG_SIZING_EXACT,
                 model=None, learned_slack=0.0, allocator=None, split=0, mask=None, mask_words=0,
                 mask_complement=False) -> spg_options:
    lib = load_library()
    o = spg_options()
    lib.spgemm_default_options(ctypes.byref(o))
    o.P, o.b, o.validate = int(P), int(b), 1 if validate else 0
    o.light_max, o.slab_rows, o.sizing, o.split = int(light_max), int(slab_rows), int(sizing), int(split)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    if allocator is not None:
        o.alloc, o.free = allocator.c_alloc, allocator.c_free
    o.model = model
    if learned_slack:
        o.learned_slack = float(learned_slack)
    if mask is not None:
        o.mask, o.mask_words, o.mask_complement = mask, int(mask_words), 1 if mask_complement else 0
    return o


# ----------------------------------------------------------------- the API

class Plan:
    """Handle of an spg_plan (steps 1-4 done).  Destroy it explicitly with
    spgemm_plan_destroy, or let garbage collection do it."""

    def __init__(self, handle, A, B, opts, allocator):
        self.handle = handle
        self._keep = (A, B, opts, allocator)   # inputs must outlive the plan
        self.A, self.B = A, B
        self.nnzC = None
        self.colptr = None

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load_library().spgemm_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def spgemm_plan(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, stream=None, validate=True, light_max=0,
                slab_rows=0, split=0, mask=None, mask_complement=False) -> Plan:
    """Steps 1-4 of Algorithm 1; split = SPG_SPLIT_UNIFORM or SPG_SPLIT_FLOPS;
    mask = an optional output mask (a CUDA int32 tensor, columns x words, bit
    r of column j's words = row r), kept alive with the plan; mask_complement
    keeps the rows whose bit is clear."""
    lib = load_library()
    alloc = _TorchAllocator(A.colptr.device)
    mp, mw = _mask_fields(mask, A.nrows, B.ncols)
    opts = make_options(P, b, stream, validate, light_max, slab_rows, allocator=alloc, split=split, mask=mp,
                        mask_words=mw, mask_complement=mask_complement)
    a, bb = A.as_c(), B.as_c()
    h = ctypes.c_void_p()
    _check(lib.spgemm_plan(ctypes.byref(a), ctypes.byref(bb), ctypes.byref(opts), ctypes.byref(h)))
    plan = Plan(h, A, B, opts, alloc)
    plan._mask = mask  # the plan's passes read it
    return plan


def spgemm_symbolic(plan: Plan):
    """Returns (colptr int64 tensor of n+1, nnz(C))."""
    lib = load_library()
    colptr = torch.empty(plan.B.ncols + 1, dtype=torch.int64, device=plan.B.colptr.device)
    nnz = ctypes.c_int64()
    _check(lib.spgemm_symbolic(plan.handle, colptr.data_ptr(), ctypes.byref(nnz)))
    plan.nnzC, plan.colptr = int(nnz.value), colptr
    return colptr, int(nnz.value)


def spgemm_numeric(plan: Plan, colptr: torch.Tensor | None = None) -> DeviceCSC:
    lib = load_library()
    if plan.nnzC is None:
        spgemm_symbolic(plan)
    colptr = plan.colptr if colptr is None else colptr
    dev = plan.B.colptr.device
    idx_dt = plan.A.rowidx.dtype
    val_dt = torch.float64 if plan.A.vals.dtype == torch.float64 else torch.int64
    rowidx = torch.empty(plan.nnzC, dtype=idx_dt, device=dev)
    vals = torch.empty(plan.nnzC, dtype=val_dt, device=dev)
    c = spg_csc(0, 0, 0, 0, 0, 0, 0, colptr.data_ptr(), rowidx.data_ptr() if plan.nnzC else None,
                vals.data_ptr() if plan.nnzC else None)
    _check(lib.spgemm_numeric(plan.handle, ctypes.byref(c)))
    return DeviceCSC(plan.A.nrows, plan.B.ncols, colptr, rowidx, vals)


def _c_out(C: DeviceCSC) -> spg_csc:
    return spg_csc(0, 0, 0, 0, 0, 0, 0, C.colptr.data_ptr(), C.rowidx.data_ptr() if C.nnz else None,
                   C.vals.data_ptr() if C.nnz else None)


def spgemm_numeric_refresh(plan: Plan, C: DeviceCSC) -> DeviceCSC:
    """Recompute C in place after new values were written into the plan's A
    and B tensors (same patterns); needs one spgemm_numeric on the plan."""
    c = _c_out(C)
    _check(load_library().spgemm_numeric_refresh(plan.handle, ctypes.byref(c)))
    return C


def spgemm_plan_capture(plan: Plan, C: DeviceCSC):
    """Record spgemm_numeric_refresh(plan, C) as a CUDA graph on the plan's
    stream (create the plan on a non-default stream)."""
    c = _c_out(C)
    plan._graph_out = C            # the graph writes into C's arrays
    _check(load_library().spgemm_plan_capture(plan.handle, ctypes.byref(c)))


def spgemm_plan_replay(plan: Plan):
    _check(load_library().spgemm_plan_replay(plan.handle))


def spgemm_plan_stats(plan: Plan) -> dict:
    lib = load_library()
    st = spg_stats()
    _check(lib.spgemm_plan_stats(plan.handle, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in spg_stats._fields_}


def spgemm_last_multiply_stats() -> dict:
    """Counters of the last spgemm_1d_multiply on this thread."""
    lib = load_library()
    lib.spgemm_last_multiply_stats.argtypes = [ctypes.POINTER(spg_stats)]
    lib.spgemm_last_multiply_stats.restype = ctypes.c_int
    st = spg_stats()
    _check(lib.spgemm_last_multiply_stats(ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in spg_stats._fields_}


def spgemm_plan_destroy(plan: Plan):
    if plan.handle:
        _check(load_library().spgemm_plan_destroy(plan.handle))
        plan.handle = None


def spgemm_1d_multiply(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, stream=None, validate=True, light_max=0,
                       slab_rows=0, sizing=SPG_SIZING_EXACT, model=None, learned_slack=0.0, split=0, mask=None,
                       mask_complement=False):
    """plan + symbolic + numeric + destroy in one C call; C's arrays come from
    torch's allocator through the callbacks.  Returns (C, status)."""
    lib = load_library()
    alloc = _TorchAllocator(A.colptr.device)
    mp, mw = _mask_fields(mask, A.nrows, B.ncols)
    opts = make_options(P, b, stream, validate, light_max, slab_rows, sizing,
                        model.handle if model is not None else None, learned_slack, allocator=alloc, split=split,
                        mask=mp, mask_words=mw, mask_complement=mask_complement)
    a, bb, c = A.as_c(), B.as_c(), spg_csc()
    st = _check(lib.spgemm_1d_multiply(ctypes.byref(a), ctypes.byref(bb), ctypes.byref(opts), ctypes.byref(c)))
    idx_dt = torch.int64 if c.idx_type == SPG_IDX_I64 else torch.int32
    val_dt = torch.float64 if c.val_type == SPG_VAL_F64 else torch.int64
    colptr = alloc.adopt(c.colptr, 0, torch.int64, c.ncols + 1)
    rowidx = alloc.adopt(c.rowidx, 0, idx_dt, c.nnz)
    vals = alloc.adopt(c.vals, 0, val_dt, c.nnz)
    return DeviceCSC(c.nrows, c.ncols, colptr, rowidx, vals), st


class spg_outer_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "P", "products", "nnzB_moved", "partial_nnz", "partial_moved", "nnzC")] + [
        (name, ctypes.c_double) for name in ("ms_split", "ms_local", "ms_merge")]


# ----------------------------------------------------- host-buffer multiply

HOST_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
HOST_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_HOST_IDX = {np.dtype(np.int32): SPG_IDX_I32, np.dtype(np.int64): SPG_IDX_I64}
_HOST_VAL = {np.dtype(np.float64): SPG_VAL_F64, np.dtype(np.int32): SPG_VAL_I32, np.dtype(np.int64): SPG_VAL_I64}


def _host_array(a):
    """(address, numpy dtype, length) of a contiguous CPU torch tensor or numpy array."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host arrays must be contiguous CPU tensors")
        return a.data_ptr(), np.dtype(str(a.dtype).replace("torch.", "")), a.numel()
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a.dtype, a.size


def _host_csc(M) -> spg_csc:
    cp, cpt, _ = _host_array(M.colptr)
    ri, rit, nnz = _host_array(M.rowidx)
    va, vat, _ = _host_array(M.vals)
    return spg_csc(int(M.nrows), int(M.ncols), int(nnz), _HOST_IDX[cpt], _HOST_IDX[rit], _HOST_VAL[vat], 0, cp,
                   ri if nnz else None, va if nnz else None)


class HostPool:
    """Pinned host memory carved into the arrays of a host-buffer product:
    reused from call to call (the previous result's arrays are overwritten).
    Exactly `nbytes` are page-locked (a host buffer registered with CUDA);
    torch's pinned allocator, which rounds sizes up to a power of two, is the
    fallback when registration fails."""

    def __init__(self, nbytes: int):
        nbytes = int(nbytes)
        self._host = None
        self.used = 0
        host = np.empty(nbytes, dtype=np.uint8)
        rt = torch.cuda.cudart()
        if nbytes > 0 and int(rt.cudaHostRegister(host.ctypes.data, nbytes, 0)) == 0:
            self._host, self._rt = host, rt
            self.buf = torch.from_numpy(host)
        else:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)

    def __del__(self):
        if getattr(self, "_host", None) is not None:
            try:
                self._rt.cudaHostUnregister(self._host.ctypes.data)
            except Exception:
                pass
            self._host = None

    def take(self, nbytes: int):
        start = (self.used + 255) & ~255
        if start + nbytes > self.buf.numel():
            return None
        self.used = start + nbytes
        return self.buf[start:start + nbytes]


class HostCSC:
    """A product in host memory: colptr (int64), rowidx (the inputs' index
    type) and vals (double or int64) as CPU tensors over pinned buffers."""

    def __init__(self, nrows, ncols, colptr, rowidx, vals, keep):
        self.nrows, self.ncols = nrows, ncols
        self.colptr, self.rowidx, self.vals = colptr, rowidx, vals
        self._keep = keep

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    @property
    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.colptr, self.rowidx, self.vals))


def spgemm_host_writable(t: torch.Tensor) -> bool:
    """True when the library's kernels can store into the CPU tensor t's
    memory directly (page-locked memory the GPU addresses with the same
    pointer)."""
    lib = load_library()
    lib.spgemm_host_writable.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    lib.spgemm_host_writable.restype = ctypes.c_int32
    return bool(lib.spgemm_host_writable(t.data_ptr(), t.numel() * t.element_size()))


def spgemm_1d_multiply_host(A, B, P=1, b=1024, chunks=4, stream=None, validate=True, light_max=0, slab_rows=0,
                            split=0, pool: HostPool | None = None, mask=None, mask_complement=False,
                            pinned: bool = True) -> HostCSC:
    """C = A * B for host matrices (objects with nrows, ncols and colptr /
    rowidx / vals as CPU tensors or numpy arrays; pinned memory for full copy
    speed) through spgemm_1d_multiply_host: the copies to and from the GPU
    happen inside the call, C's part of one group of column blocks streaming
    back while the next group computes.  C's arrays come from `pool` when
    given (its earlier contents are overwritten), else from fresh pinned
    tensors (pageable ones with pinned=False: C then always comes back through
    the copy engine).  mask: an optional output mask on the GPU (as for
    spgemm_plan)."""
    lib = load_library()
    lib.spgemm_1d_multiply_host.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                            ctypes.POINTER(spg_options), ctypes.c_int32, HOST_ALLOC_FN,
                                            HOST_FREE_FN, ctypes.c_void_p, ctypes.POINTER(spg_csc)]
    lib.spgemm_1d_multiply_host.restype = ctypes.c_int
    alloc = _TorchAllocator(torch.device("cuda", torch.cuda.current_device()))
    mp, mw = _mask_fields(mask, int(A.nrows), int(B.ncols))
    opts = make_options(P, b, stream, validate, light_max, slab_rows, allocator=alloc, split=split, mask=mp,
                        mask_words=mw, mask_complement=mask_complement)
    if pool is not None:
        pool.used = 0
    held = {}

    def host_alloc(nbytes, ctx):
        t = pool.take(nbytes) if pool is not None else torch.empty(int(nbytes), dtype=torch.uint8, pin_memory=pinned)
        if t is None:
            return None
        held[t.data_ptr()] = t
        return t.data_ptr()

    def host_free(ptr, nbytes, ctx):
        held.pop(ptr, None)

    ha, hb = _host_csc(A), _host_csc(B)
    c = spg_csc()
    fa, ff = HOST_ALLOC_FN(host_alloc), HOST_FREE_FN(host_free)
    _check(lib.spgemm_1d_multiply_host(ctypes.byref(ha), ctypes.byref(hb), ctypes.byref(opts), int(chunks), fa, ff,
                                       None, ctypes.byref(c)))
    idx_dt = torch.int64 if c.idx_type == SPG_IDX_I64 else torch.int32
    val_dt = torch.float64 if c.val_type == SPG_VAL_F64 else torch.int64

    def view(addr, dt, count):
        base = held[addr]
        return base[: count * torch.tensor([], dtype=dt).element_size()].view(dt)
    return HostCSC(c.nrows, c.ncols, view(c.colptr, torch.int64, c.ncols + 1), view(c.rowidx, idx_dt, c.nnz),
                   view(c.vals, val_dt, c.nnz), (held, pool))


def spgemm_outer_multiply(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, stream=None, validate=True, light_max=0,
                          slab_rows=0):
    """Outer-product 1D SpGEMM (Algorithm 3): B redistributed by P row blocks,
    the P partial products by the column 1D path, then their merge.  C's arrays
    come from torch's allocator.  Returns (C, stats dict)."""
    lib = load_library()
    lib.spgemm_outer_multiply.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                          ctypes.POINTER(spg_options), ctypes.POINTER(spg_csc),
                                          ctypes.POINTER(spg_outer_stats)]
    lib.spgemm_outer_multiply.restype = ctypes.c_int
    alloc = _TorchAllocator(A.colptr.device)
    opts = make_options(P, b, stream, validate, light_max, slab_rows, SPG_SIZING_EXACT, None, 0.0, allocator=alloc)
    a, bb, c, st = A.as_c(), B.as_c(), spg_csc(), spg_outer_stats()
    _check(lib.spgemm_outer_multiply(ctypes.byref(a), ctypes.byref(bb), ctypes.byref(opts), ctypes.byref(c),
                                     ctypes.byref(st)))
    idx_dt = torch.int64 if c.idx_type == SPG_IDX_I64 else torch.int32
    val_dt = torch.float64 if c.val_type == SPG_VAL_F64 else torch.int64
    colptr = alloc.adopt(c.colptr, 0, torch.int64, c.ncols + 1)
    rowidx = alloc.adopt(c.rowidx, 0, idx_dt, c.nnz)
    vals = alloc.adopt(c.vals, 0, val_dt, c.nnz)
    return DeviceCSC(c.nrows, c.ncols, colptr, rowidx, vals), {n: getattr(st, n) for n, _ in spg_outer_stats._fields_}


class spg_bc_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "levels", "frontier_nnz", "products_forward", "products_backward")] + [
        (name, ctypes.c_double) for name in ("ms_forward", "ms_backward", "ms_plan", "ms_sym_light", "ms_sym_heavy",
                                             "ms_num_light", "ms_num_heavy", "ms_gather")] + [
        (name, ctypes.c_int64) for name in ("multiplies", "nnzC_total")]


def spgemm_bc_batch(A: DeviceCSC, sources: torch.Tensor, P=1, b=1024, bc: torch.Tensor | None = None, stream=None,
                    validate=True, max_levels=256):
    """Batched Brandes betweenness (Section 3.2): adds, for the given source
    vertices (a CUDA int32 tensor), the dependencies delta_s(v) into bc (a CUDA
    float64 tensor of n, zeros if not given).  Returns (bc, level sizes, stats)."""
    lib = load_library()
    lib.spgemm_bc_batch.argtypes = [ctypes.POINTER(spg_csc), ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(spg_options), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.c_int32, ctypes.POINTER(spg_bc_stats)]
    lib.spgemm_bc_batch.restype = ctypes.c_int
    dev = A.colptr.device
    src = sources.to(device=dev, dtype=torch.int32).contiguous()
    if bc is None:
        bc = torch.zeros(A.ncols, dtype=torch.float64, device=dev)
    alloc = _TorchAllocator(dev)
    opts = make_options(P, b, stream, validate, allocator=alloc)
    lv = (ctypes.c_int64 * max_levels)()
    st = spg_bc_stats()
    a = A.as_c()
    _check(lib.spgemm_bc_batch(ctypes.byref(a), src.data_ptr(), int(src.numel()), ctypes.byref(opts), bc.data_ptr(),
                               lv, max_levels, ctypes.byref(st)))
    stats = {n: getattr(st, n) for n, _ in spg_bc_stats._fields_}
    return bc, [int(lv[i]) for i in range(min(stats["levels"], max_levels))], stats


def spgemm_plan_blocks(plan: Plan) -> dict:
    """Per-block diagnostics: bounds (P + 1), flops, gathered and remote A~
    nonzeros (P each, numpy int64), and cv_mem_a = mean remote / nnz(A) (the
    Discussion's CV/memA)."""
    import numpy as np
    lib = load_library()
    P = plan._keep[2].P
    out = {q: np.zeros(P + (1 if q == "bounds" else 0), dtype=np.int64)
           for q in ("bounds", "flops", "gathered", "remote")}
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    lib.spgemm_plan_blocks.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 4
    lib.spgemm_plan_blocks.restype = ctypes.c_int
    _check(lib.spgemm_plan_blocks(plan.handle, ptr(out["bounds"]), ptr(out["flops"]), ptr(out["gathered"]),
                                  ptr(out["remote"])))
    nnz_a = max(int(plan.A.rowidx.numel()), 1)
    out["cv_mem_a"] = float(out["remote"].mean()) / nnz_a if P else 0.0
    return out


def spgemm_plan_export(plan: Plan, block: int) -> dict:
    """Planning quantities of one column block as CUDA tensors (for tests)."""
    lib = load_library()
    dev = plan.B.colptr.device
    k, n = plan.B.nrows, plan.B.ncols
    P = plan._keep[2].P
    b = plan._keep[2].b
    W = (k + 31) // 32
    nfb = (k + b - 1) // b
    bounds = spgemm_plan_blocks(plan)["bounds"]
    c0, c1 = int(bounds[block]), int(bounds[block + 1])
    H = torch.zeros(max(W, 1), dtype=torch.int32, device=dev)
    nd = ctypes.c_int64()
    _check(lib.spgemm_plan_export(plan.handle, block, H.data_ptr(), None, ctypes.byref(nd), None, None, None,
                                  None, None))
    nd = int(nd.value)
    dt = torch.zeros(max(nd, 1), dtype=torch.int32, device=dev)
    fetch = torch.zeros(max(nfb, 1), dtype=torch.uint8, device=dev)
    acp = torch.zeros(nd + 1, dtype=torch.int64, device=dev)
    fl = torch.zeros(max(c1 - c0, 1), dtype=torch.int64, device=dev)
    _check(lib.spgemm_plan_export(plan.handle, block, None, dt.data_ptr(), None, fetch.data_ptr(),
                                  acp.data_ptr(), None, None, fl.data_ptr()))
    vol = int((acp[-1] - acp[0]).item())
    rows = torch.zeros(max(vol, 1), dtype=torch.int32, device=dev)
    vdt = torch.float64 if plan.A.vals.dtype == torch.float64 else torch.int64
    vals = torch.zeros(max(vol, 1), dtype=vdt, device=dev)
    _check(lib.spgemm_plan_export(plan.handle, block, None, None, None, None, None, rows.data_ptr(),
                                  vals.data_ptr(), None))
    return {"H_bits": H[:W], "dtilde": dt[:nd], "fetch": fetch[:nfb], "At_colptr": acp - acp[0],
            "At_rowidx": rows[:vol], "At_vals": vals[:vol], "flops": fl[: c1 - c0]}


def multiply(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, **kw) -> DeviceCSC:
    """Convenience: plan, symbolic, allocate C with torch, numeric, destroy."""
    plan = spgemm_plan(A, B, P, b, **kw)
    try:
        spgemm_symbolic(plan)
        return spgemm_numeric(plan)
    finally:
        spgemm_plan_destroy(plan)


def spgemm_count_noalloc(A: DeviceCSC, B: DeviceCSC, nnz_out: torch.Tensor | None = None, stream=None):
    """nnz(C(:,j)) of C = A*B through the entry point that allocates nothing.

    For callers that may not allocate device memory: the library keeps its
    scratch in one fixed 8 MiB array per GPU, so A may have at most 1,048,576
    rows, and calls that overlap on the GPU race (order them on one stream).
    The output array is the caller's (allocated here by torch if not given)."""
    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    for name, M in (("A", A), ("B", B)):
        for t in (M.colptr, M.rowidx):
            if t.device != dev:
                raise ValueError(f"{name} must be on the current device {dev} (the scratch array is looked up "
                                 f"for the current device), not {t.device}")
    if nnz_out is None:
        nnz_out = torch.empty(max(B.ncols, 1), dtype=torch.int64, device=dev)
    elif (nnz_out.dtype != torch.int64 or nnz_out.device != dev or not nnz_out.is_contiguous()
          or nnz_out.numel() < B.ncols):
        raise ValueError(f"nnz_out must be a contiguous int64 tensor on {dev} with at least {B.ncols} entries "
                         f"(got {nnz_out.dtype}, {nnz_out.device}, {nnz_out.numel()} entries, "
                         f"contiguous={nnz_out.is_contiguous()})")
    if stream is None:
        stream = torch.cuda.current_stream()
    a, b = A.as_c(), B.as_c()
    _check(lib.spgemm_count_noalloc(ctypes.byref(a), ctypes.byref(b), nnz_out.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))))
    return nnz_out[: B.ncols]


# ------------------------------------------------- one-launch small multiply

SMALL_RESULT_FIELDS = ("nnzC", "status", "products", "sum_H", "sum_dtilde", "gathered_nnz_exact",
                       "gathered_nnz_block", "fetch_blocks_chosen")


def _small_lib():
    lib = load_library()
    if not getattr(lib, "_small_ready", False):
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.spgemm_small_bound.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc), vp, vp]
        lib.spgemm_small_workspace.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc), i32, i64, i32,
                                               ctypes.POINTER(ctypes.c_size_t)]
        lib.spgemm_small_multiply.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc), i32, i64, i32, vp,
                                              ctypes.c_size_t, vp, vp, vp, i64, vp, i64, vp]
        for name in ("spgemm_small_bound", "spgemm_small_workspace", "spgemm_small_multiply"):
            getattr(lib, name).restype = ctypes.c_int
        lib._small_ready = True
    return lib


class SmallProduct:
    """Buffers of the one-launch multiply of A * B (spgemm_small_multiply):
    device workspace, C's arrays with room for `capacity` entries and the
    8-entry result block, allocated once with torch; `run()` only enqueues the
    call (two clears and one kernel), so it can be captured in a CUDA graph.

    The set-up reads spgemm_small_bound once (one synchronisation): the
    largest column bound picks the table class (8 when it is <= 128, else 10),
    and their sum is C's default capacity.  table_log forces a class."""

    def __init__(self, A: DeviceCSC, B: DeviceCSC, P=1, b=1024, capacity=None, timeout_ns=1_000_000_000,
                 table_log=None):
        lib = _small_lib()
        self.A, self.B, self.P, self.b = A, B, int(P), int(b)
        self._a, self._b = A.as_c(), B.as_c()
        dev = A.colptr.device
        bound = torch.zeros(2, dtype=torch.int64, device=dev)
        _check(lib.spgemm_small_bound(ctypes.byref(self._a), ctypes.byref(self._b), bound.data_ptr(),
                                      _stream_ptr(None)))
        self.max_bound, self.nnz_bound = (int(x) for x in bound.cpu())
        self.table_log = int(table_log) if table_log is not None else (8 if self.max_bound <= 128 else 10)
        nbytes = ctypes.c_size_t()
        _check(lib.spgemm_small_workspace(ctypes.byref(self._a), ctypes.byref(self._b), self.P, self.b,
                                          self.table_log, ctypes.byref(nbytes)))
        self.capacity = int(self.nnz_bound if capacity is None else capacity)
        self.workspace = torch.empty(max(int(nbytes.value), 1), dtype=torch.uint8, device=dev)
        val_dt = torch.float64 if A.vals.dtype == torch.float64 else torch.int64
        self.colptr = torch.empty(B.ncols + 1, dtype=torch.int64, device=dev)
        self.rowidx = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.vals = torch.empty(max(self.capacity, 1), dtype=val_dt, device=dev)
        self.result = torch.zeros(len(SMALL_RESULT_FIELDS), dtype=torch.int64, device=dev)
        self.timeout_ns = int(timeout_ns)

    def run(self, stream=None):
        """Enqueue C = A * B on `stream` (torch's current stream by default)."""
        _check(_small_lib().spgemm_small_multiply(
            ctypes.byref(self._a), ctypes.byref(self._b), self.P, self.b, self.table_log, self.workspace.data_ptr(),
            self.workspace.numel(), self.colptr.data_ptr(), self.rowidx.data_ptr(), self.vals.data_ptr(),
            self.capacity, self.result.data_ptr(), self.timeout_ns, _stream_ptr(stream)))
        return self

    def stats(self) -> dict:
        """The result block (synchronises with the device)."""
        return dict(zip(SMALL_RESULT_FIELDS, (int(x) for x in self.result.cpu())))

    def C(self) -> DeviceCSC:
        """C after the call (synchronises; raises SpgError on a device-side failure)."""
        st = self.stats()
        if st["status"]:
            raise SpgError(st["status"], f"one-launch multiply failed on the device (nnz(C) = {st['nnzC']}, "
                                         f"capacity {self.capacity})")
        n = st["nnzC"]
        return DeviceCSC(self.A.nrows, self.B.ncols, self.colptr, self.rowidx[:n], self.vals[:n])


def spgemm_small_multiply(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, capacity=None, stream=None) -> DeviceCSC:
    """One call of the one-launch multiply (buffers allocated for this call)."""
    return SmallProduct(A, B, P, b, capacity).run(stream).C()


# ------------------------------------------------------ learned nnz sizing

SPG_MODEL_NPARAMS = 1249


class Model:
    """Handle of an spg_model (the nnz-prediction MLP, parameters on the GPU)."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load_library().spgemm_model_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def _model_lib():
    lib = load_library()
    if not getattr(lib, "_model_ready", False):
        vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
        fp = ctypes.POINTER(ctypes.c_float)
        lib.spgemm_model_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(vp)]
        lib.spgemm_model_destroy.argtypes = [vp]
        lib.spgemm_model_set_params.argtypes = [vp, fp, i64]
        lib.spgemm_model_get_params.argtypes = [vp, fp, i64]
        lib.spgemm_model_train.argtypes = [vp, vp, vp, i64, i32, i32, f32, vp, fp]
        lib.spgemm_model_predict.argtypes = [vp, vp, i64, vp, vp]
        lib.spgemm_model_gradient.argtypes = [vp, vp, vp, i64, fp, fp, vp]
        lib.spgemm_model_save.argtypes = [vp, ctypes.c_char_p]
        lib.spgemm_model_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        lib.spgemm_plan_features.argtypes = [vp, vp]
        lib.spgemm_plan_labels.argtypes = [vp, vp]
        for name in ("spgemm_model_create", "spgemm_model_destroy", "spgemm_model_set_params",
                     "spgemm_model_get_params", "spgemm_model_train", "spgemm_model_predict",
                     "spgemm_model_gradient", "spgemm_model_save", "spgemm_model_load",
                     "spgemm_plan_features", "spgemm_plan_labels"):
            getattr(lib, name).restype = ctypes.c_int
        lib._model_ready = True
    return lib


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def spgemm_model_create(seed: int = 0) -> Model:
    h = ctypes.c_void_p()
    _check(_model_lib().spgemm_model_create(ctypes.c_uint64(seed), ctypes.byref(h)))
    return Model(h)


def spgemm_model_load(path: str) -> Model:
    h = ctypes.c_void_p()
    _check(_model_lib().spgemm_model_load(path.encode(), ctypes.byref(h)))
    return Model(h)


def spgemm_model_save(model: Model, path: str):
    _check(_model_lib().spgemm_model_save(model.handle, path.encode()))


def spgemm_model_get_params(model: Model):
    import numpy as np
    out = np.zeros(SPG_MODEL_NPARAMS, dtype=np.float32)
    _check(_model_lib().spgemm_model_get_params(model.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                SPG_MODEL_NPARAMS))
    return out


def spgemm_model_set_params(model: Model, params):
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(_model_lib().spgemm_model_set_params(model.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))


def spgemm_model_train(model: Model, X: torch.Tensor, y: torch.Tensor, epochs=10, batch=4096, lr=1e-3, stream=None):
    """Train in place on device tensors X (n, 4) and y (n,); returns the final MSE."""
    loss = ctypes.c_float()
    X, y = X.contiguous().float(), y.contiguous().float()
    _check(_model_lib().spgemm_model_train(model.handle, X.data_ptr(), y.data_ptr(), y.numel(), int(epochs),
                                           int(batch), float(lr), _stream_ptr(stream), ctypes.byref(loss)))
    return float(loss.value)


def spgemm_model_predict(model: Model, X: torch.Tensor, stream=None) -> torch.Tensor:
    X = X.contiguous().float()
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(_model_lib().spgemm_model_predict(model.handle, X.data_ptr(), X.shape[0], out.data_ptr(),
                                             _stream_ptr(stream)))
    return out


def spgemm_model_gradient(model: Model, X: torch.Tensor, y: torch.Tensor, stream=None):
    """(gradient of the MSE as a float32 numpy vector, loss)."""
    import numpy as np
    g = np.zeros(SPG_MODEL_NPARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    X, y = X.contiguous().float(), y.contiguous().float()
    _check(_model_lib().spgemm_model_gradient(model.handle, X.data_ptr(), y.data_ptr(), y.numel(),
                                              g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss),
                                              _stream_ptr(stream)))
    return g, float(loss.value)


def spgemm_plan_features(plan: Plan) -> torch.Tensor:
    X = torch.empty((max(plan.B.ncols, 1), 4), dtype=torch.float32, device=plan.B.colptr.device)
    _check(_model_lib().spgemm_plan_features(plan.handle, X.data_ptr()))
    return X[: plan.B.ncols]


def spgemm_plan_labels(plan: Plan) -> torch.Tensor:
    y = torch.empty(max(plan.B.ncols, 1), dtype=torch.float32, device=plan.B.colptr.device)
    _check(_model_lib().spgemm_plan_labels(plan.handle, y.data_ptr()))
    return y[: plan.B.ncols]


# --------------------------------------------------------- batched products

class spg_batch_options(ctypes.Structure):
    _fields_ = [("task_cols", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32), ("timeout_ns", ctypes.c_int64),
                ("stall_instance", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _batch_lib():
    lib = load_library()
    if not getattr(lib, "_batch_ready", False):
        vp = ctypes.c_void_p
        lib.spgemm_batch_default_options.argtypes = [ctypes.POINTER(spg_batch_options)]
        lib.spgemm_batch_default_options.restype = None
        lib.spgemm_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                            ctypes.POINTER(spg_batch_options), ctypes.POINTER(vp)]
        lib.spgemm_batch_execute.argtypes = [vp, vp]
        lib.spgemm_batch_status.argtypes = [vp, vp]
        lib.spgemm_batch_result.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(spg_csc)]
        lib.spgemm_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int32)]
        lib.spgemm_batch_destroy.argtypes = [vp]
        for name in ("spgemm_batch_create", "spgemm_batch_execute", "spgemm_batch_status", "spgemm_batch_result",
                     "spgemm_batch_info", "spgemm_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        lib._batch_ready = True
    return lib


class Batch:
    """Handle of an spg_batch; keeps its inputs alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load_library().spgemm_batch_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def spgemm_batch_create(As, Bs, task_cols=64, warps_per_cta=8, timeout_ns=2_000_000_000, stall_instance=-1) -> Batch:
    lib = _batch_lib()
    n = len(As)
    a = (spg_csc * n)(*[X.as_c() for X in As])
    b = (spg_csc * n)(*[X.as_c() for X in Bs])
    o = spg_batch_options()
    lib.spgemm_batch_default_options(ctypes.byref(o))
    o.task_cols, o.warps_per_cta, o.timeout_ns, o.stall_instance = task_cols, warps_per_cta, timeout_ns, stall_instance
    h = ctypes.c_void_p()
    _check(lib.spgemm_batch_create(n, a, b, ctypes.byref(o), ctypes.byref(h)))
    return Batch(h, (list(As), list(Bs)))


def spgemm_batch_execute(batch: Batch, stream=None):
    _check(_batch_lib().spgemm_batch_execute(batch.handle, _stream_ptr(stream)))


def spgemm_batch_status(batch: Batch, stream=None) -> int:
    """Synchronise and return the status of the last execution (raises on error)."""
    return _check(_batch_lib().spgemm_batch_status(batch.handle, _stream_ptr(stream)))


def spgemm_batch_result(batch: Batch, i: int):
    """(colptr, rowidx, vals) of instance i as CUDA tensors (copies)."""
    lib = _batch_lib()
    c = spg_csc()
    _check(lib.spgemm_batch_result(batch.handle, i, ctypes.byref(c)))
    dev = batch._keep[0][i].colptr.device
    val_dt = torch.float64 if c.val_type == SPG_VAL_F64 else torch.int64
    colptr = torch.empty(c.ncols + 1, dtype=torch.int64, device=dev)
    rowidx = torch.empty(max(c.nnz, 1), dtype=torch.int32, device=dev)
    vals = torch.empty(max(c.nnz, 1), dtype=val_dt, device=dev)
    lib.spgemm_batch_copy_result.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]
    lib.spgemm_batch_copy_result.restype = ctypes.c_int
    _check(lib.spgemm_batch_copy_result(batch.handle, i, colptr.data_ptr(), rowidx.data_ptr(), vals.data_ptr(),
                                        _stream_ptr(None)))
    return colptr, rowidx[: c.nnz], vals[: c.nnz]


def spgemm_batch_info(batch: Batch):
    nt, pool, grid = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(_batch_lib().spgemm_batch_info(batch.handle, ctypes.byref(nt), ctypes.byref(pool), ctypes.byref(grid)))
    return {"tasks": nt.value, "pool_entries": pool.value, "grid": grid.value}


def spgemm_batch_autotune(As, Bs, sample=0, cache_path=None) -> dict:
    """Fastest (task_cols, warps_per_cta) for this batch (cached in cache_path)."""
    lib = _batch_lib()
    lib.spgemm_batch_autotune.argtypes = [ctypes.c_int32, ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc),
                                          ctypes.c_int32, ctypes.c_char_p, ctypes.POINTER(spg_batch_options),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.spgemm_batch_autotune.restype = ctypes.c_int
    n = len(As)
    a = (spg_csc * n)(*[X.as_c() for X in As])
    b = (spg_csc * n)(*[X.as_c() for X in Bs])
    o = spg_batch_options()
    ms = ctypes.c_double()
    _check(lib.spgemm_batch_autotune(n, a, b, int(sample), cache_path.encode() if cache_path else None,
                                     ctypes.byref(o), ctypes.byref(ms)))
    return {"task_cols": o.task_cols, "warps_per_cta": o.warps_per_cta, "ms": ms.value}


def spgemm_autotune(A: DeviceCSC, B: DeviceCSC, P=1, b=1024, cache_path=None, stream=None) -> dict:
    """Fastest (light_max, slab_rows) of the plain path for A*B (cached in cache_path)."""
    lib = load_library()
    lib.spgemm_autotune.argtypes = [ctypes.POINTER(spg_csc), ctypes.POINTER(spg_csc), ctypes.POINTER(spg_options),
                                    ctypes.c_char_p, ctypes.POINTER(spg_options), ctypes.POINTER(ctypes.c_double)]
    lib.spgemm_autotune.restype = ctypes.c_int
    alloc = _TorchAllocator(A.colptr.device)
    base = make_options(P, b, stream, True, allocator=alloc)
    best = spg_options()
    ms = ctypes.c_double()
    a, bb = A.as_c(), B.as_c()
    _check(lib.spgemm_autotune(ctypes.byref(a), ctypes.byref(bb), ctypes.byref(base),
                               cache_path.encode() if cache_path else None, ctypes.byref(best), ctypes.byref(ms)))
    return {"light_max": best.light_max, "slab_rows": best.slab_rows, "ms": ms.value}


def spgemm_batch_destroy(batch: Batch):
    if batch.handle:
        _check(_batch_lib().spgemm_batch_destroy(batch.handle))
        batch.handle = None
