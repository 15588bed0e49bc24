"""The distributed 1D SpGEMM (Section 3.1, Algorithm 1 with P processes;
Algorithm 2 for the fetch requests) run by 2 and 3 gloo processes on the CPU.

The host logic of ``paper_2408_14558_gb300.dist1d`` -- the all-gather of A's
column counts, the request planning and exchange, the owners' replies in
requester order, the all-to-all-v data plane, the assembly of the fetched
matrix and the agreement that turns a late or missing peer into SPG_TIMEOUT
-- runs here unchanged.  Its device steps (fetch blocks, pack, fetched column
pointers, local multiply) are replaced by host stand-ins defined below, built
on the CPU oracle; the CUDA versions are compared with the oracle in
tests/test_gpu_dist.py.  Every process checks that its block of C equals the
oracle's columns of A*B exactly, and that what it received equals the chosen
fetch blocks' share of each owner (the exact D~ volume when b = 1)."""
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth
from paper_2408_14558_gb300 import DeviceCSC, SPG_TIMEOUT, SpgError
from paper_2408_14558_gb300 import dist1d


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cpu_csc(M, c0=None, c1=None):
    """Columns c0:c1 of a host CSC as CPU tensors (local column pointers)."""
    cp = np.asarray(M.colptr, dtype=np.int64)
    c0 = 0 if c0 is None else c0
    c1 = M.ncols if c1 is None else c1
    s, e = int(cp[c0]), int(cp[c1])
    return DeviceCSC(M.nrows, c1 - c0, torch.from_numpy(cp[c0:c1 + 1] - s),
                     torch.from_numpy(np.asarray(M.rowidx[s:e]).copy()), torch.from_numpy(np.asarray(M.vals[s:e]).copy()))


class _View:
    def __init__(self, nrows, ncols, colptr, rowidx, vals):
        self.nrows, self.ncols, self.colptr, self.rowidx, self.vals = nrows, ncols, colptr, rowidx, vals


class HostSteps:
    """Host stand-ins for the device steps: fetch blocks from the oracle's
    Algorithm 1/2 planning of this block, plain slicing for the owners'
    replies, a cumulative sum for the fetched column pointers and the oracle
    for the local multiply."""

    device = torch.device("cpu")

    def __init__(self, A, B, c0, c1):
        self.A, self.B, self.c0, self.c1 = A, B, c0, c1

    def fetch_blocks(self, B_i, gcolptr, b):
        # the all-gathered column pointers must be A's
        assert np.array_equal(gcolptr.numpy(), np.asarray(self.A.colptr, dtype=np.int64))
        return torch.from_numpy(oracle.plan_block(self.A, self.B, self.c0, self.c1, b)["fetch"].copy())

    def pack(self, A_i, ranges, sizes):
        cp = A_i.colptr.numpy().astype(np.int64)
        rows = [A_i.rowidx[int(cp[lo]):int(cp[hi])] for lo, hi in ranges]
        vals = [A_i.vals[int(cp[lo]):int(cp[hi])] for lo, hi in ranges]
        for r, (lo, hi), n in zip(rows, ranges, sizes):
            assert r.numel() == n
        cat = lambda xs, t: torch.cat(xs) if xs else torch.zeros(0, dtype=t.dtype)
        return cat(rows, A_i.rowidx), cat(vals, A_i.vals)

    def fetched_colptr(self, gcolptr, fetch, k, b):
        g = gcolptr.numpy()
        take = np.repeat(fetch.numpy().astype(bool), b)[:k]
        out = np.zeros(k + 1, dtype=np.int64)
        np.cumsum(np.where(take, np.diff(g), 0), out=out[1:])
        return torch.from_numpy(out)

    def multiply(self, A_f, B_i, P, b):
        Af = _View(A_f.nrows, A_f.ncols, A_f.colptr.numpy(), A_f.rowidx.numpy(), A_f.vals.numpy())
        Bi = _View(B_i.nrows, B_i.ncols, B_i.colptr.numpy(), B_i.rowidx.numpy(), B_i.vals.numpy())
        return oracle.spgemm(Af, Bi)


def _expected_received(A, fetch, b, own):
    """Entries of A in the chosen fetch blocks, per owner: a loop over columns."""
    cp = np.asarray(A.colptr, dtype=np.int64)
    out = np.zeros(own.shape[0] - 1, dtype=np.int64)
    for c in range(A.ncols):
        if fetch[c // b]:
            j = int(np.searchsorted(own, c, side="right") - 1)
            out[j] += cp[c + 1] - cp[c]
    return out


def _case(name):
    rng = np.random.default_rng({"random": 11, "rmat": 12, "tiny": 13}[name])
    if name == "random":
        A = synth.random_sparse(90, 70, 0.06, rng, values="small")
        B = synth.random_sparse(70, 80, 0.05, rng, values="small")
    elif name == "rmat":
        A = synth.rmat_symmetric(8, 8, seed=2)
        B = A
    elif name == "tiny":          # more processes than columns of A: an owner of nothing
        A = synth.random_sparse(5, 2, 0.9, rng, values="i64", min_per_col=1)
        B = synth.random_sparse(2, 4, 0.9, rng, values="i64", min_per_col=1)
    else:
        raise ValueError(name)
    return A, B


def _worker(rank, world, port, cases):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = dist1d.TorchComm("cpu")
    for name, b, uneven in cases:
        A, B = _case(name)
        own = dist1d.owner_bounds(A.ncols, world)
        if uneven and A.ncols > 3:
            own = np.array([0] + sorted(np.random.default_rng(5).choice(np.arange(1, A.ncols), world - 1,
                                                                         replace=False).tolist()) + [A.ncols])
        cb = oracle.block_bounds(B.ncols, world)
        c0, c1 = int(cb[rank]), int(cb[rank + 1])
        A_i = _cpu_csc(A, int(own[rank]), int(own[rank + 1]))
        B_i = _cpu_csc(B, c0, c1)
        C_i, info = dist1d.multiply_distributed(A_i, B_i, own, comm, b=b, steps=HostSteps(A, B, c0, c1),
                                                timeout_s=60)
        ref = oracle.spgemm(A, B, cols=np.arange(c0, c1))
        where = f"{name} b={b} rank {rank}/{world}"
        assert np.array_equal(C_i["colptr"], ref["colptr"]), where
        assert np.array_equal(C_i["rowidx"], ref["rowidx"]), where
        assert np.array_equal(C_i["vals"], ref["vals"]), where
        pl = oracle.plan_block(A, B, c0, c1, b)
        assert np.array_equal(info.received, _expected_received(A, pl["fetch"], b, own)), where
        assert int(info.received.sum()) == pl["vol_block"], where
        vol = oracle.block_volumes(A, B, cb, b)
        if b == 1:               # one column per fetch block: exactly D~_i
            assert int(info.received.sum()) == pl["vol_exact"] == vol["gathered"][rank], where
        # every entry received was sent by its owner: totals agree across processes
        t = torch.tensor([int(info.received.sum()), int(info.sent.sum())], dtype=torch.int64)
        dist.all_reduce(t)
        assert int(t[0]) == int(t[1]), where
    dist.barrier()
    dist.destroy_process_group()


def _run(world, cases):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.exitcode is None:
            p.kill()
    assert codes == [0] * world, f"process exit codes {codes}"


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_product_equals_oracle(world):
    _run(world, [("random", 8, False), ("random", 1, True), ("rmat", 16, False), ("rmat", 1, False),
                 ("tiny", 1, False), ("tiny", 4, False)])


def test_plan_requests_cuts_blocks_at_owners():
    """Chosen blocks 0, 1 and 3 of width 4 over k = 14, owners [0, 6), [6, 9),
    [9, 14): owner 0 gets [0, 6), owner 1 gets [6, 8), owner 2 gets [12, 14)."""
    fetch = np.array([1, 1, 0, 1], dtype=np.uint8)
    req = dist1d.plan_requests(fetch, 4, 14, np.array([0, 6, 9, 14]))
    assert [r.tolist() for r in req] == [[[0, 6]], [[6, 8]], [[12, 14]]]
    g = np.arange(15, dtype=np.int64) * 2
    assert dist1d.request_entries(req[1], g).tolist() == [4]
    assert [r.tolist() for r in dist1d.plan_requests(np.zeros(4, np.uint8), 4, 14, np.array([0, 7, 14]))] == [[], []]


def _late_worker(rank, world, port, mode):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = dist1d.TorchComm("cpu", prefix=f"late-{mode}")
    A, B = _case("random")
    own = dist1d.owner_bounds(A.ncols, world)
    cb = oracle.block_bounds(B.ncols, world)
    c0, c1 = int(cb[rank]), int(cb[rank + 1])
    args = (_cpu_csc(A, int(own[rank]), int(own[rank + 1])), _cpu_csc(B, c0, c1), own, comm)
    steps = HostSteps(A, B, c0, c1)
    late = rank == world - 1
    if late and mode == "never":
        time.sleep(2.0)           # never joins this call; leaves without entering a collective
        comm.calls += 1           # (keeps its call count in step for the call that follows)
    else:
        if late:
            time.sleep(2.0)       # arrives after the others gave up
        t0 = time.monotonic()
        try:
            dist1d.multiply_distributed(*args, b=4, steps=steps, timeout_s=0.5)
            raise AssertionError("expected SPG_TIMEOUT")
        except SpgError as e:
            assert e.status == SPG_TIMEOUT, e
        assert time.monotonic() - t0 < 30
    # the group is still usable: the next call, joined by all, succeeds
    C_i, _ = dist1d.multiply_distributed(*args, b=4, steps=steps, timeout_s=60)
    ref = oracle.spgemm(A, B, cols=np.arange(c0, c1))
    assert np.array_equal(C_i["rowidx"], ref["rowidx"]) and np.array_equal(C_i["vals"], ref["vals"])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["late", "never"])
@pytest.mark.parametrize("world", [2, 3])
def test_late_or_missing_peer_times_out_on_every_process(world, mode):
    """A process that reaches the call 2 s late, or not at all, against a
    0.5 s limit: every process that calls gets SPG_TIMEOUT before any
    collective starts, and the next call joined by all succeeds."""
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_late_worker, args=(r, world, port, mode)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.exitcode is None:
            p.kill()
    assert codes == [0] * world, f"process exit codes {codes}"
