"""Distributed 1D SpGEMM across processes (Section 3.1, Algorithm 1 with P
processes; Algorithm 2 for what each process fetches).

Process i owns column block i of A (columns ``own_A[i]:own_A[i+1]``), of B and
of C.  To multiply its block, C_i = A * B_i, it needs the columns of A named
by the nonzero rows H_i of B_i that are nonempty (D~_i = H_i AND D), fetched
from their owners in blocks of ``b`` consecutive column ids.  One call of
``multiply_distributed`` on every process runs:

1. an agreement through the process group's key-value store that every
   process has reached this call (a late or missing peer turns into an
   ``SpgError`` with status ``SPG_TIMEOUT`` on every process, before any
   collective is entered);
2. an all-gather of the owners' column counts of A: the metadata Algorithm 1
   needs (the set D and where each column's entries start);
3. H_i and the chosen fetch blocks (``spgemm_dist_fetch_blocks``);
4. the requests: the chosen blocks cut at owner boundaries and merged into
   column ranges (``plan_requests``), sent to the owners (all-to-all of the
   range counts, then of the ranges);
5. the data plane: each owner packs the requested ranges of its A_j into one
   buffer in requester order (``spgemm_dist_pack``) and an all-to-all-v moves
   row ids and values into every requester's own memory;
6. the requester's fetched matrix A_f (column c = A(:, c) if c's block was
   chosen, else empty; ``spgemm_dist_fetched_colptr``) and the local multiply
   C_i = A_f * B_i by the column 1D path (A_f * B_i = A * B_i).

C stays distributed by column blocks; nothing is reduced (Section 3.1).

The device steps are the library's CUDA kernels (``CudaSteps``); the
collectives go through a ``Comm`` (``TorchComm``: ``torch.distributed`` with
NCCL for CUDA tensors, gloo for CPU tensors).  Both are parameters so that the
host logic (planning, request protocol, agreement, assembly order) can be
exercised by processes without a GPU.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (DeviceCSC, SPG_TIMEOUT, SpgError, _check, load_library, multiply)

__all__ = ["plan_requests", "request_entries", "TorchComm", "CudaSteps", "ExchangeInfo", "multiply_distributed",
           "owner_bounds"]


def owner_bounds(ncols: int, P: int) -> np.ndarray:
    """Column block i of P is [floor(i*ncols/P), floor((i+1)*ncols/P)) (the
    partition of Algorithm 1 for A, B and C alike)."""
    return np.array([(i * ncols) // P for i in range(P + 1)], dtype=np.int64)


def plan_requests(fetch: np.ndarray, b: int, k: int, own: np.ndarray) -> list[np.ndarray]:
    """The column ranges a process requests from each owner.

    ``fetch[t]`` = 1 when fetch block t (column ids [t*b, min((t+1)*b, k))) is
    chosen (Algorithm 2).  A block is cut at the owners' boundaries ``own``
    (P + 1 ascending column ids from 0 to k); adjacent pieces with one owner
    are merged.  Returns, per owner j, an int64 array of shape (r_j, 2) of
    GLOBAL column ranges [lo, hi), ascending."""
    fetch = np.asarray(fetch).astype(bool)
    own = np.asarray(own, dtype=np.int64)
    P = own.shape[0] - 1
    chosen = np.flatnonzero(fetch)
    lo = chosen * b
    hi = np.minimum(lo + b, k)
    out = []
    for j in range(P):
        a, e = int(own[j]), int(own[j + 1])
        cl, ch = np.maximum(lo, a), np.minimum(hi, e)
        keep = cl < ch
        cl, ch = cl[keep], ch[keep]
        if cl.size:
            # merge pieces that touch (consecutive chosen blocks)
            start = np.ones(cl.size, dtype=bool)
            start[1:] = cl[1:] != ch[:-1]
            first = np.flatnonzero(start)
            last = np.append(first[1:], cl.size) - 1
            cl, ch = cl[first], ch[last]
        out.append(np.stack([cl, ch], axis=1).astype(np.int64) if cl.size else np.zeros((0, 2), np.int64))
    return out


def request_entries(ranges: np.ndarray, gcolptr: np.ndarray) -> np.ndarray:
    """Entries of A in each global column range [lo, hi)."""
    if ranges.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    return gcolptr[ranges[:, 1]] - gcolptr[ranges[:, 0]]


# ------------------------------------------------------------ collectives

class TorchComm:
    """Collectives of one process group of ``torch.distributed``.

    Tensors live on ``device`` (CUDA for NCCL, CPU for gloo).  The agreement
    uses the group's key-value store: process 0 declares "go" once every
    process has arrived; a process that waits past its timeout declares
    "abort".  The first declaration wins (compare-and-set), so every process
    takes the same decision and none enters a collective that a peer will not
    join."""

    def __init__(self, device, group=None, store=None, prefix="spgemm1d"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = torch.device(device)
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.store = store if store is not None else dist.distributed_c10d._get_default_store()
        self.prefix = prefix
        self.calls = 0

    def all_gather(self, t: torch.Tensor) -> list[torch.Tensor]:
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return out

    def all_to_all(self, out: torch.Tensor, inp: torch.Tensor, out_splits, in_splits):
        self.dist.all_to_all_single(out, inp, [int(x) for x in out_splits], [int(x) for x in in_splits],
                                    group=self.group)

    def agree(self, timeout_s: float, poll_s: float = 0.005):
        tag = f"{self.prefix}/{self.calls}"
        self.calls += 1
        return agree(self.store, tag, self.rank, self.world, timeout_s, poll_s)


def agree(store, tag: str, rank: int, world: int, timeout_s: float, poll_s: float = 0.005):
    """Every process of the group calls this with the same tag; returns when
    all have (process 0's "go"), else raises SpgError(SPG_TIMEOUT) on every
    process that calls it, including a late one."""
    store.set(f"{tag}/arrived/{rank}", "1")
    key = f"{tag}/decision"
    deadline = time.monotonic() + timeout_s
    arrived = {rank}
    while True:
        if store.check([key]):
            decision = store.get(key)
            break
        if rank == 0:
            for r in range(world):
                if r not in arrived and store.check([f"{tag}/arrived/{r}"]):
                    arrived.add(r)
            if len(arrived) == world:
                decision = store.compare_set(key, "", "go")
                break
        if time.monotonic() > deadline:
            decision = store.compare_set(key, "", f"abort: process {rank} waited {timeout_s:g} s")
            break
        time.sleep(poll_s)
    decision = decision.decode() if isinstance(decision, bytes) else str(decision)
    if decision != "go":
        missing = "" if rank != 0 else f" (arrived: {sorted(arrived)} of {world})"
        raise SpgError(SPG_TIMEOUT, f"distributed SpGEMM call {tag}: not every process arrived in time "
                                    f"({decision}){missing}")


# ------------------------------------------------------------ device steps

def _stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class CudaSteps:
    """The device steps, through the C ABI of libspgemm1d.so."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        lib = load_library()
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        from . import spg_csc
        lib.spgemm_dist_fetch_blocks.argtypes = [ctypes.POINTER(spg_csc), vp, i64, vp, vp, vp, vp]
        lib.spgemm_dist_pack.argtypes = [ctypes.POINTER(spg_csc), vp, vp, i64, i64, vp, vp, vp, vp]
        lib.spgemm_dist_fetched_colptr.argtypes = [vp, vp, i64, i64, vp, vp]
        for name in ("spgemm_dist_fetch_blocks", "spgemm_dist_pack", "spgemm_dist_fetched_colptr"):
            getattr(lib, name).restype = ctypes.c_int
        self.lib = lib
        self.flag = torch.zeros(1, dtype=torch.int32, device=self.device)

    def _bad(self, what):
        if int(self.flag.item()):
            raise SpgError(2, f"{what}: an index lay outside its matrix (entries skipped)")

    def fetch_blocks(self, B: DeviceCSC, gcolptr: torch.Tensor, b: int) -> torch.Tensor:
        k = int(B.nrows)
        H = torch.empty(max((k + 31) // 32, 1), dtype=torch.int32, device=self.device)
        fetch = torch.empty(max((k + b - 1) // b, 1), dtype=torch.uint8, device=self.device)
        bc = B.as_c()
        _check(self.lib.spgemm_dist_fetch_blocks(ctypes.byref(bc), gcolptr.data_ptr(), int(b), H.data_ptr(),
                                                 fetch.data_ptr(), self.flag.data_ptr(), _stream_ptr()))
        self._bad("spgemm_dist_fetch_blocks (B)")
        return fetch[: (k + b - 1) // b]

    def pack(self, A: DeviceCSC, ranges: np.ndarray, sizes: np.ndarray):
        nr = int(ranges.shape[0])
        out_off = np.zeros(nr + 1, dtype=np.int64)
        np.cumsum(sizes, out=out_off[1:])
        total = int(out_off[-1])
        rows = torch.empty(total, dtype=A.rowidx.dtype, device=self.device)
        vals = torch.empty(total, dtype=A.vals.dtype, device=self.device)
        if nr and total:
            r = torch.from_numpy(np.ascontiguousarray(ranges.reshape(-1))).to(self.device)
            o = torch.from_numpy(out_off).to(self.device)
            ac = A.as_c()
            _check(self.lib.spgemm_dist_pack(ctypes.byref(ac), r.data_ptr(), o.data_ptr(), nr, total,
                                             rows.data_ptr(), vals.data_ptr(), self.flag.data_ptr(), _stream_ptr()))
            self._bad("spgemm_dist_pack")
        return rows, vals

    def fetched_colptr(self, gcolptr: torch.Tensor, fetch: torch.Tensor, k: int, b: int) -> torch.Tensor:
        out = torch.empty(k + 1, dtype=torch.int64, device=self.device)
        _check(self.lib.spgemm_dist_fetched_colptr(gcolptr.data_ptr(), fetch.data_ptr() if k else None, int(k),
                                                   int(b), out.data_ptr(), _stream_ptr()))
        return out

    def multiply(self, A_f: DeviceCSC, B: DeviceCSC, P: int, b: int) -> DeviceCSC:
        return multiply(A_f, B, P, b, validate=False)


# ------------------------------------------------------------------- driver

@dataclass
class ExchangeInfo:
    """What one process moved (entries of A; a row id and a value each)."""
    rank: int = 0
    fetch_blocks_chosen: int = 0
    requested_ranges: list = field(default_factory=list)   # per owner: (r_j, 2) global column ranges
    received: np.ndarray = None      # entries received from each owner (own share included)
    sent: np.ndarray = None          # entries sent to each requester (own share included)
    ms: dict = field(default_factory=dict)

    @property
    def received_remote(self) -> int:
        return int(self.received.sum() - self.received[self.rank])


def multiply_distributed(A_i: DeviceCSC, B_i: DeviceCSC, own_A, comm, b: int = 1024, P_local: int = 1,
                         steps=None, timeout_s: float = 300.0):
    """C_i = A * B_i on every process of ``comm`` (see the module docstring).

    A_i: this process's columns own_A[i]:own_A[i+1] of the m x k matrix A
    (local column pointers starting at 0).  B_i: this process's column block
    of B, k rows (global column ids of A).  own_A: P + 1 ascending column ids
    of A from 0 to k, the same on every process.  P_local: column blocks of
    the local multiply.  Returns (C_i, ExchangeInfo)."""
    steps = steps if steps is not None else CudaSteps()
    dev = steps.device
    own = np.asarray(own_A, dtype=np.int64)
    P, rank = comm.world, comm.rank
    if own.shape[0] != P + 1 or own[0] != 0 or np.any(np.diff(own) < 0):
        raise ValueError(f"own_A must hold P + 1 = {P + 1} ascending column ids starting at 0")
    k = int(own[-1])
    if int(B_i.nrows) != k or int(A_i.ncols) != int(own[rank + 1] - own[rank]):
        raise ValueError(f"process {rank}: A_i has {A_i.ncols} columns for its block of "
                         f"{int(own[rank + 1] - own[rank])}, B_i has {B_i.nrows} rows for k = {k}")
    info = ExchangeInfo(rank=rank)
    t0 = time.perf_counter()
    comm.agree(timeout_s)
    info.ms["agree"] = 1e3 * (time.perf_counter() - t0)

    # 1. the owners' column counts of A (padded to the widest block)
    t1 = time.perf_counter()
    widths = np.diff(own)
    kmax = int(widths.max()) if P else 0
    cnt = torch.zeros(max(kmax, 1), dtype=torch.int64, device=dev)
    if int(A_i.ncols):
        cnt[: int(A_i.ncols)] = torch.diff(A_i.colptr.to(torch.int64))
    parts = comm.all_gather(cnt)
    counts = np.concatenate([parts[j][: int(widths[j])].cpu().numpy() for j in range(P)]) if k else np.zeros(0, np.int64)
    gcol = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(counts, out=gcol[1:])
    gcol_dev = torch.from_numpy(gcol).to(dev)

    # 2. H_i and the chosen fetch blocks; 3. requests per owner
    fetch_dev = steps.fetch_blocks(B_i, gcol_dev, b)
    fetch = fetch_dev.cpu().numpy()
    info.fetch_blocks_chosen = int(fetch.astype(bool).sum())
    req = plan_requests(fetch, b, k, own)
    info.requested_ranges = req
    want = np.array([int(request_entries(r, gcol).sum()) for r in req], dtype=np.int64)
    nreq = torch.tensor([r.shape[0] for r in req], dtype=torch.int64, device=dev)
    nreq_in = torch.empty(P, dtype=torch.int64, device=dev)
    comm.all_to_all(nreq_in, nreq, [1] * P, [1] * P)
    nin = nreq_in.cpu().numpy()
    send_ranges = np.concatenate([(r - own[j]).reshape(-1) for j, r in enumerate(req)]) if P else np.zeros(0, np.int64)
    rin = torch.empty(int(2 * nin.sum()), dtype=torch.int64, device=dev)
    comm.all_to_all(rin, torch.from_numpy(send_ranges.astype(np.int64)).to(dev), 2 * nin,
                    [2 * r.shape[0] for r in req])
    asked = rin.cpu().numpy().reshape(-1, 2)          # local column ranges, requester after requester
    info.ms["plan"] = 1e3 * (time.perf_counter() - t1)

    # 4. data plane: pack what every requester asked for, all-to-all-v
    t2 = time.perf_counter()
    gl = asked + own[rank]
    sizes = request_entries(gl, gcol) if asked.shape[0] else np.zeros(0, np.int64)
    if asked.shape[0] and (np.any(asked[:, 0] < 0) or np.any(asked[:, 1] > int(A_i.ncols))
                           or np.any(asked[:, 0] > asked[:, 1])):
        raise SpgError(1, f"process {rank}: a request lies outside its columns of A")
    bounds = np.zeros(P + 1, dtype=np.int64)
    np.cumsum(nin, out=bounds[1:])
    sent = np.array([int(sizes[bounds[r]:bounds[r + 1]].sum()) for r in range(P)], dtype=np.int64)
    rows_s, vals_s = steps.pack(A_i, asked, sizes)
    total_in = int(want.sum())
    rows_r = torch.empty(total_in, dtype=A_i.rowidx.dtype, device=dev)
    vals_r = torch.empty(total_in, dtype=A_i.vals.dtype, device=dev)
    comm.all_to_all(rows_r, rows_s, want, sent)
    comm.all_to_all(vals_r, vals_s, want, sent)
    info.received, info.sent = want, sent
    info.ms["exchange"] = 1e3 * (time.perf_counter() - t2)

    # 5. the fetched matrix and the local multiply
    t3 = time.perf_counter()
    colptr_f = steps.fetched_colptr(gcol_dev, fetch_dev, k, b)
    if int(colptr_f[-1]) != total_in:
        raise SpgError(4, f"process {rank}: fetched column pointers end at {int(colptr_f[-1])}, "
                          f"received {total_in} entries")
    A_f = DeviceCSC(int(A_i.nrows), k, colptr_f, rows_r, vals_r)
    C_i = steps.multiply(A_f, B_i, P_local, b)
    info.ms["local_multiply"] = 1e3 * (time.perf_counter() - t3)
    return C_i, info
