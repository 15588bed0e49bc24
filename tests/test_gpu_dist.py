"""The device steps of the distributed 1D SpGEMM (Section 3.1, Algorithm 1
with P processes; Algorithm 2) through the C ABI, against the oracle:

* spgemm_dist_fetch_blocks against oracle.plan_block's chosen fetch blocks,
  for every column block of several partitions;
* spgemm_dist_pack and spgemm_dist_fetched_colptr against plain slicing and
  counting of the host arrays;
* the whole of dist1d.multiply_distributed on one GPU with P host threads as
  the processes (their collectives are host-side copies between the threads'
  tensors, taken after a device synchronisation; no kernel waits on another),
  every block of C against the oracle;
* the same through torch.distributed with NCCL and one process."""
import os
import socket
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2408_14558_gb300 as g
from paper_2408_14558_gb300 import dist1d
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


def _dev_block(M, c0, c1, **kw):
    cp = np.asarray(M.colptr, dtype=np.int64)
    s, e = int(cp[c0]), int(cp[c1])
    sub = synth.CSC(M.nrows, c1 - c0, cp[c0:c1 + 1] - s, np.asarray(M.rowidx[s:e]), np.asarray(M.vals[s:e]))
    return g.to_device(sub, **kw)


def _cases():
    rng = np.random.default_rng(3)
    yield "random", synth.random_sparse(300, 257, 0.03, rng), synth.random_sparse(257, 203, 0.03, rng)
    R = synth.rmat_symmetric(11, 8, seed=4)
    yield "rmat", R, R
    U = synth.uniform_columns(3000, 6, seed=2, values="i32")
    yield "uniform-i32", U, U


@pytest.mark.parametrize("P,b", [(1, 64), (3, 1), (4, 32), (7, 1000)])
def test_fetch_blocks_match_oracle(P, b):
    steps = dist1d.CudaSteps()
    for name, A, B in _cases():
        gcol = torch.from_numpy(np.asarray(A.colptr, dtype=np.int64)).cuda()
        cb = oracle.block_bounds(B.ncols, P)
        for i in range(P):
            B_i = _dev_block(B, int(cb[i]), int(cb[i + 1]))
            got = steps.fetch_blocks(B_i, gcol, b).cpu().numpy()
            want = oracle.plan_block(A, B, int(cb[i]), int(cb[i + 1]), b)["fetch"]
            assert np.array_equal(got, want), f"{name} P={P} b={b} block {i}"


@pytest.mark.parametrize("idx", [torch.int32, torch.int64])
def test_pack_and_fetched_colptr(idx):
    steps = dist1d.CudaSteps()
    rng = np.random.default_rng(9)
    A = synth.random_sparse(500, 400, 0.02, rng, values="i64")
    dA = g.to_device(A, idx_dtype=idx)
    cp = np.asarray(A.colptr, dtype=np.int64)
    ranges = np.array([[0, 3], [3, 3], [10, 57], [57, 58], [399, 400], [120, 390]], dtype=np.int64)
    sizes = cp[ranges[:, 1]] - cp[ranges[:, 0]]
    rows, vals = steps.pack(dA, ranges, sizes)
    want_r = np.concatenate([A.rowidx[cp[lo]:cp[hi]] for lo, hi in ranges])
    want_v = np.concatenate([A.vals[cp[lo]:cp[hi]] for lo, hi in ranges])
    assert rows.dtype == idx and np.array_equal(rows.cpu().numpy(), want_r)
    assert np.array_equal(vals.cpu().numpy(), want_v)
    for b in (1, 7, 64, 400, 1000):
        nblk = (A.ncols + b - 1) // b
        fetch = (rng.random(nblk) < 0.5).astype(np.uint8)
        got = steps.fetched_colptr(torch.from_numpy(cp).cuda(), torch.from_numpy(fetch).cuda(), A.ncols, b)
        take = np.repeat(fetch.astype(bool), b)[: A.ncols]
        want = np.zeros(A.ncols + 1, dtype=np.int64)
        np.cumsum(np.where(take, np.diff(cp), 0), out=want[1:])
        assert np.array_equal(got.cpu().numpy(), want), f"b={b}"


class ThreadComm:
    """P host threads as the processes of a group, on one GPU: every
    collective meets at a barrier; each thread then copies its share out of
    the other threads' (device-synchronised) input tensors."""

    class Shared:
        def __init__(self, world):
            self.world = world
            self.bar = threading.Barrier(world, timeout=120)
            self.slots = [None] * world

    def __init__(self, shared, rank):
        self.sh, self.rank, self.world = shared, rank, shared.world
        self.device = torch.device("cuda")

    def _publish(self, item):
        torch.cuda.synchronize()
        self.sh.slots[self.rank] = item
        self.sh.bar.wait()
        items = list(self.sh.slots)
        self.sh.bar.wait()
        return items

    def all_gather(self, t):
        return [x.clone() for x in self._publish(t)]

    def all_to_all(self, out, inp, out_splits, in_splits):
        items = self._publish((inp, np.asarray(in_splits, dtype=np.int64)))
        pos = 0
        for j, (x, sp) in enumerate(items):
            start = int(sp[: self.rank].sum())
            n = int(sp[self.rank])
            assert n == int(out_splits[j])
            out[pos:pos + n].copy_(x[start:start + n])
            pos += n
        torch.cuda.synchronize()
        self.sh.bar.wait()

    def agree(self, timeout_s):
        self.sh.bar.wait()


@pytest.mark.parametrize("world,b,P_local", [(2, 64, 1), (3, 1, 2), (4, 16, 3)])
def test_threads_as_processes_match_oracle(world, b, P_local):
    for name, A, B in _cases():
        own = dist1d.owner_bounds(A.ncols, world)
        cb = oracle.block_bounds(B.ncols, world)
        shared = ThreadComm.Shared(world)
        results, errors = [None] * world, []

        def run(r):
            try:
                torch.cuda.set_device(0)
                A_i = _dev_block(A, int(own[r]), int(own[r + 1]))
                B_i = _dev_block(B, int(cb[r]), int(cb[r + 1]))
                results[r] = dist1d.multiply_distributed(A_i, B_i, own, ThreadComm(shared, r), b=b,
                                                         P_local=P_local)
            except BaseException as e:      # reported by the main thread
                errors.append(e)
                shared.bar.abort()

        threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert not errors, errors[0]
        sent = received = 0
        for r in range(world):
            C_i, info = results[r]
            ref = oracle.spgemm(A, B, cols=np.arange(int(cb[r]), int(cb[r + 1])))
            assert_full_parity(C_i, ref, f"{name} world={world} process {r}")
            pl = oracle.plan_block(A, B, int(cb[r]), int(cb[r + 1]), b)
            assert int(info.received.sum()) == pl["vol_block"]
            sent += int(info.sent.sum())
            received += int(info.received.sum())
        assert sent == received


def test_nccl_single_process():
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        A = synth.rmat_symmetric(12, 8, seed=6)
        dA = g.to_device(A)
        comm = dist1d.TorchComm("cuda")
        C, info = dist1d.multiply_distributed(dA, dA, dist1d.owner_bounds(A.ncols, 1), comm, b=256, P_local=4,
                                              timeout_s=60)
        torch.cuda.synchronize()
        assert_full_parity(C, oracle.spgemm(A, A), "nccl world=1")
        assert info.received_remote == 0
    finally:
        dist.destroy_process_group()
