// One-launch multiply for small products: every step of Algorithm 1 on one
// GPU (Section 3.1) in a single cooperative persistent kernel, so that a
// product of a few MFLOP costs one kernel instead of tens of launches and host
// read-backs, and the whole call can be captured in a CUDA graph.
//
// Every CTA owns a contiguous chunk of columns.  Phases, separated by two grid
// barriers (a counter each; every wait is bounded by a %globaltimer limit and
// gives up with SPG_TIMEOUT, never hangs):
//   1. warp per column j of the chunk: mark H_i (bit k of the block's bitmap
//      for every row k of B(:,j), Table 1), count flops_j (Section 3.2), then
//      the symbolic pass: a shared-memory hash of the rows of its products
//      gives nnz(C(:,j)); the CTA sums its chunk
//   2. H_i AND D, the chosen fetch blocks and the volumes of D~_i (Algorithm 1
//      and 2, reported as statistics); C's column pointers: each CTA scans its
//      chunk from the sum of the earlier chunks' totals
//   3. the chosen blocks' volume (statistics); numeric pass: warp per column,
//      hash of (row, value), compaction and a warp sort, written at the
//      column's offset
// The gather of A~_i is fused into the product loads: each required column of
// A is read in place when the B entry that needs it is processed (one GPU
// holds all of A), so the arithmetic is that of A~_i * B_i.
//
// Limits of this form (SPG_UNSUPPORTED otherwise): 32-bit row ids of A, and
// every column's bound min(flops_j, m) at most half the warp's table (128 or
// 512 by table class).
// C's arrays come from the caller with a capacity; a product that needs more
// reports its nnz and SPG_OUT_OF_MEMORY in the result block and writes no rows.
#include <algorithm>

#include "block_ops.cuh"
#include "spg_internal.cuh"

namespace spg {
void clear_error();

namespace {

// Table classes: 2^8 slots per warp and 32 warps per CTA (column bounds up to
// 128), or 2^10 slots and 8 warps (bounds up to 512); one CTA per SM.
constexpr int kSmallClassLog[2] = {8, 10};
constexpr int kSmallClassWarps[2] = {32, 8};
constexpr int kNumBarriers = 2;

// result block (device int64, caller-owned)
enum { kResNnz = 0, kResStatus, kResProducts, kResSumH, kResSumDt, kResGathered, kResGatheredBlock, kResFetch,
       kResCount };

struct SmallArgs {
    const void *Acp;
    int ap64;
    const int32_t *Arow;
    const void *Aval;
    int avt;
    const void *Bcp;
    int bp64;
    const void *Brow;
    int bi64;
    const void *Bval;
    int bvt;
    int64_t m, k, n;
    int P;
    int64_t b, W, nfb;
    unsigned *bar;           // kNumBarriers counters
    uint32_t *H;             // P * W
    uint8_t *fetch;          // P * nfb
    int64_t *cnt;            // n: flops_j, then nnz_j
    long long *chunk;        // gridDim.x CTA partial sums
    int64_t *Ccp;
    int32_t *Crow;
    void *Cval;
    int64_t capacity;
    long long *res;
    long long timeout_ns;
};

__device__ __forceinline__ long long now_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Record the first device-side failure (an spg_status code).
__device__ __forceinline__ void fail(long long *res, int code) {
    atomicCAS((unsigned long long *)(res + kResStatus), 0ull, (unsigned long long)code);
}

// Grid barrier number `idx`: every CTA adds one to its counter, then thread 0
// waits (bounded) until all CTAs have.  Returns false when the wait gave up
// or an earlier phase failed: the caller's CTA then returns.
__device__ bool grid_barrier(const SmallArgs &a, int idx) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.bar + idx, 1u);
        const long long t0 = now_ns();
        int ok = 1;
        while (*(volatile unsigned *)(a.bar + idx) < gridDim.x) {
            if (now_ns() - t0 > a.timeout_ns) {
                fail(a.res, SPG_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok_sh = ok && *(volatile long long *)(a.res + kResStatus) == 0;
    }
    __syncthreads();
    return ok_sh;
}

template <typename Acc>
__device__ __forceinline__ Acc ld_val(const void *p, int vt, int64_t i);
template <>
__device__ __forceinline__ double ld_val<double>(const void *p, int, int64_t i) {
    return __ldg((const double *)p + i);
}
template <>
__device__ __forceinline__ long long ld_val<long long>(const void *p, int vt, int64_t i) {
    return vt == SPG_VAL_I32 ? (long long)__ldg((const int *)p + i) : (long long)__ldg((const long long *)p + i);
}

__device__ __forceinline__ int table_log(int64_t U) {
    int lg = 5;
    while ((int64_t(1) << lg) < 2 * U) lg++;
    return lg;
}

// Column bounds min(flops_j, m): their maximum and their sum (an upper bound
// of nnz(C)), for choosing the table class and C's capacity.
__global__ void k_small_bound(const void *Acp, int ap64, const void *Bcp, int bp64, const void *Brow, int bi64,
                              int64_t m, int64_t k, int64_t n, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mx = 0, sum = 0;
    for (int64_t j = gw; j < n; j += nwarps) {
        const int64_t p0 = ld_ptr(Bcp, bp64, j), p1 = ld_ptr(Bcp, bp64, j + 1);
        long long f = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t kk = ld_ptr(Brow, bi64, p);
            if ((uint64_t)kk < (uint64_t)k) f += ld_ptr(Acp, ap64, kk + 1) - ld_ptr(Acp, ap64, kk);
        }
        f = warp_sum_ll(f);
        const unsigned long long u = (unsigned long long)min((int64_t)f, m);
        mx = max(mx, u);
        sum += u;
    }
    if (lane == 0) {
        if (mx) atomicMax(out, mx);
        if (sum) atomicAdd(out + 1, sum);
    }
}

// The kernel of the one-launch multiply.  CTA c owns the columns
// [c * L, (c + 1) * L) (L = ceil(n / gridDim.x)); its WARPS warps take them in
// turn, each with a shared table of 2^LOGS slots.
template <int LOGS, int WARPS, typename Acc>
__global__ void __launch_bounds__(WARPS * 32) k_small_multiply(SmallArgs a) {
    constexpr int kSlots = 1 << LOGS, kMaxU = kSlots / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSeg<Acc> *segs = (WarpSeg<Acc> *)smem_raw;
    int *keys_all = (int *)(segs + WARPS);
    int *slots_all = keys_all + WARPS * kSlots;
    Acc *vals_all = (Acc *)(slots_all + WARPS * kSlots);
    int *hist_all = (int *)(vals_all + WARPS * kSlots);
    __shared__ long long red[WARPS], red2[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *keys = keys_all + wid * kSlots;
    int *slots = slots_all + wid * kSlots;
    Acc *vals = vals_all + wid * kSlots;
    int *hist = hist_all + wid * 256;
    const int64_t L = (a.n + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = min((int64_t)blockIdx.x * L, a.n), j1 = min(j0 + L, a.n);

    // ---- 1: per column of this CTA's chunk: H_i and flops_j, then the
    // symbolic pass (a hash of the rows of its products gives nnz(C(:,j)))
    long long prod = 0, nz = 0;
    for (int64_t j = j0 + wid; j < j1; j += WARPS) {
        const int i = block_of(j, a.n, a.P);
        const int64_t p0 = ld_ptr(a.Bcp, a.bp64, j), p1 = ld_ptr(a.Bcp, a.bp64, j + 1);
        long long f = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t kk = ld_ptr(a.Brow, a.bi64, p);
            if ((uint64_t)kk >= (uint64_t)a.k) {
                fail(a.res, SPG_INVALID_INPUT);
                continue;
            }
            atomicOr(a.H + (int64_t)i * a.W + (kk >> 5), 1u << (kk & 31));
            f += ld_ptr(a.Acp, a.ap64, kk + 1) - ld_ptr(a.Acp, a.ap64, kk);
        }
        f = warp_sum_ll(f);
        prod += f;
        const int64_t U = min((int64_t)f, a.m);
        int c = 0;
        if (U > kMaxU) {
            if (lane == 0) fail(a.res, SPG_UNSUPPORTED);  // the column's bound exceeds this table class
        } else if (U > 0) {
            const int lg = table_log(U), S = 1 << lg;
            for (int s = lane; s < S; s += 32) keys[s] = kEmptyKey;
            __syncwarp();
            bool full = false;
            warp_products_v<false, 4, Acc>(
                p0, p1, lane, segs[wid], a.Arow,
                [&](int64_t p, long long &st, int &len, Acc &) {
                    const int64_t kk = ld_ptr(a.Brow, a.bi64, p);
                    if ((uint64_t)kk < (uint64_t)a.k) {
                        st = ld_ptr(a.Acp, a.ap64, kk);
                        len = (int)(ld_ptr(a.Acp, a.ap64, kk + 1) - st);
                    }
                },
                [&](long long) { return Acc(0); },
                [&](int r, Acc) {
                    bool fresh;
                    if (hash_insert(keys, lg, r, &fresh) < 0) full = true;
                    c += fresh ? 1 : 0;
                });
            c = warp_sum_i(c);
            if (__any_sync(kFull, full) && lane == 0) fail(a.res, SPG_CUDA_ERROR);
            __syncwarp();
        }
        if (lane == 0) a.cnt[j] = c;
        nz += c;
    }
    if (lane == 0) {
        red[wid] = nz;
        red2[wid] = prod;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0, t2 = 0;
        for (int w = 0; w < WARPS; w++) {
            t += red[w];
            t2 += red2[w];
        }
        a.chunk[blockIdx.x] = t;
        a.chunk[gridDim.x + blockIdx.x] = t2;
    }
    if (!grid_barrier(a, 0)) return;

    // ---- 2: D~_i = H_i AND D and the chosen fetch blocks (statistics), then
    // C's column pointers: the chunk's offset is the sum of the earlier chunks
    {
        long long sh = 0, sdt = 0, gat = 0;
        const int64_t nword = (int64_t)a.P * a.W;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nword;
             t += (int64_t)gridDim.x * blockDim.x) {
            uint32_t x = a.H[t];
            sh += __popc(x);
            const int64_t i = t / a.W, k0 = (t % a.W) * 32;
            while (x) {
                const int64_t kk = k0 + __ffs(x) - 1;
                x &= x - 1u;
                const int64_t len = ld_ptr(a.Acp, a.ap64, kk + 1) - ld_ptr(a.Acp, a.ap64, kk);
                if (len > 0) {
                    sdt++;
                    gat += len;
                    a.fetch[i * a.nfb + kk / a.b] = 1;
                }
            }
        }
        sh = warp_sum_ll(sh);
        sdt = warp_sum_ll(sdt);
        gat = warp_sum_ll(gat);
        if (lane == 0) {
            if (sh) atomicAdd((unsigned long long *)(a.res + kResSumH), (unsigned long long)sh);
            if (sdt) atomicAdd((unsigned long long *)(a.res + kResSumDt), (unsigned long long)sdt);
            if (gat) atomicAdd((unsigned long long *)(a.res + kResGathered), (unsigned long long)gat);
        }
    }
    {
        long long off = 0, total = 0, ptot = 0;
        for (int c = lane; c < (int)gridDim.x; c += 32) {
            const long long v = a.chunk[c];
            total += v;
            ptot += a.chunk[gridDim.x + c];
            if (c < (int)blockIdx.x) off += v;
        }
        off = warp_sum_ll(off);
        total = warp_sum_ll(total);
        ptot = warp_sum_ll(ptot);
        for (int64_t t0 = j0; t0 < j1; t0 += blockDim.x) {
            const int64_t j = t0 + threadIdx.x;
            const long long v = j < j1 ? a.cnt[j] : 0;
            long long inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) red[wid] = inc;
            __syncthreads();
            long long before = 0, tile = 0;
            for (int w = 0; w < WARPS; w++) {
                const long long y = red[w];
                if (w < wid) before += y;
                tile += y;
            }
            if (j < j1) a.Ccp[j] = off + before + inc - v;
            off += tile;
            __syncthreads();
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.Ccp[a.n] = total;
            a.res[kResNnz] = total;
            a.res[kResProducts] = ptot;
            if (total > a.capacity) fail(a.res, SPG_OUT_OF_MEMORY);
        }
    }
    if (!grid_barrier(a, 1)) return;

    // ---- 3: volume of the chosen fetch blocks (statistics), then the numeric
    // pass over this CTA's chunk
    {
        long long nb = 0, vb = 0;
        const int64_t nf = (int64_t)a.P * a.nfb;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf;
             t += (int64_t)gridDim.x * blockDim.x) {
            if (a.fetch[t]) {
                const int64_t f = t % a.nfb, lo = f * a.b, hi = min(lo + a.b, a.k);
                nb++;
                vb += ld_ptr(a.Acp, a.ap64, hi) - ld_ptr(a.Acp, a.ap64, lo);
            }
        }
        nb = warp_sum_ll(nb);
        vb = warp_sum_ll(vb);
        if (lane == 0) {
            if (nb) atomicAdd((unsigned long long *)(a.res + kResFetch), (unsigned long long)nb);
            if (vb) atomicAdd((unsigned long long *)(a.res + kResGatheredBlock), (unsigned long long)vb);
        }
    }
    Acc *Cval = (Acc *)a.Cval;
    for (int64_t j = j0 + wid; j < j1; j += WARPS) {
        const int64_t base = a.Ccp[j], want = a.Ccp[j + 1] - base;
        if (want == 0) continue;
        const int lg = table_log(want), S = 1 << lg;
        // values of the table's S slots (int64 as two 32-bit halves)
        const HeavyAcc<Acc> acc(vals, S);
        for (int s = lane; s < S; s += 32) {
            keys[s] = kEmptyKey;
            acc.zero(s);
        }
        __syncwarp();
        const int64_t p0 = ld_ptr(a.Bcp, a.bp64, j), p1 = ld_ptr(a.Bcp, a.bp64, j + 1);
        bool full = false;
        warp_products_v<true, 4, Acc>(
            p0, p1, lane, segs[wid], a.Arow,
            [&](int64_t p, long long &st, int &len, Acc &bv) {
                const int64_t kk = ld_ptr(a.Brow, a.bi64, p);
                if ((uint64_t)kk < (uint64_t)a.k) {
                    st = ld_ptr(a.Acp, a.ap64, kk);
                    len = (int)(ld_ptr(a.Acp, a.ap64, kk + 1) - st);
                    bv = ld_val<Acc>(a.Bval, a.bvt, p);
                }
            },
            [&](long long e) { return ld_val<Acc>(a.Aval, a.avt, e); },
            [&](int r, Acc v) {
                bool fresh;
                const int slot = hash_insert(keys, lg, r, &fresh);
                if (slot < 0)
                    full = true;
                else
                    acc.add(slot, v);
            });
        __syncwarp();
        // compact the occupied slots to the front (row ids, and the slot
        // holding each row's value), sort by row, then read the values out
        int nout = 0;
        for (int c0 = 0; c0 < S; c0 += 32) {
            const int kk = keys[c0 + lane];
            const bool occ = kk != kEmptyKey;
            const unsigned bal = __ballot_sync(kFull, occ);
            __syncwarp();
            if (occ) {
                const int pos = nout + __popc(bal & ((1u << lane) - 1u));
                keys[pos] = kk;
                slots[pos] = c0 + lane;
            }
            nout += __popc(bal);
            __syncwarp();
        }
        if (nout != want || full) {
            if (lane == 0) fail(a.res, SPG_CUDA_ERROR);
            continue;
        }
        warp_sort_pairs<int>(keys, slots, nout, S, hist, lane);
        for (int s = lane; s < nout; s += 32) {
            a.Crow[base + s] = keys[s];
            Cval[base + s] = acc.get(slots[s]);
        }
        __syncwarp();
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t bar, H, fetch, zero_bytes, cnt, chunk, total;
};

Layout layout_of(int64_t k, int64_t n, int P, int64_t b, int grid) {
    Layout L;
    const int64_t W = (k + 31) / 32, nfb = (k + b - 1) / b;
    size_t o = 0;
    L.bar = o;
    o = align256(o + sizeof(unsigned) * kNumBarriers);
    L.H = o;
    o = align256(o + sizeof(uint32_t) * (size_t)(P * W));
    L.fetch = o;
    o = align256(o + (size_t)(P * nfb));
    L.zero_bytes = o;  // everything above is cleared before each launch
    L.cnt = o;
    o = align256(o + sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1));
    L.chunk = o;  // per CTA: its chunk's nnz, then its products
    o = align256(o + sizeof(long long) * 2 * (size_t)grid);
    L.total = o;
    return L;
}

template <int LOGS, int WARPS, typename Acc>
size_t smem_of() {
    return WARPS * (sizeof(WarpSeg<Acc>) + (size_t(1) << LOGS) * (2 * sizeof(int) + sizeof(Acc)) + 256 * sizeof(int));
}

template <int LOGS, int WARPS, typename Acc>
spg_status grid_of_class(int sms, int *grid) {
    const size_t smem = smem_of<LOGS, WARPS, Acc>();
    spg_status s = cuda_check(cudaFuncSetAttribute(k_small_multiply<LOGS, WARPS, Acc>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              "smem attribute");
    int occ = 0;
    if (!s) s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_small_multiply<LOGS, WARPS, Acc>,
                                                                         WARPS * 32, smem), "occupancy");
    if (s) return s;
    if (occ < 1) {
        set_error("the one-launch multiply does not fit an SM");
        return SPG_UNSUPPORTED;
    }
    *grid = sms * occ;
    return SPG_OK;
}

// Co-resident CTAs of the kernel of this class on this device (the
// cooperative grid).
spg_status small_grid(int cls, bool f64, int *grid) {
    int dev = 0, sms = 0;
    spg_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (!s) s = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (s) return s;
    if (cls == 0)
        return f64 ? grid_of_class<8, 32, double>(sms, grid) : grid_of_class<8, 32, long long>(sms, grid);
    return f64 ? grid_of_class<10, 8, double>(sms, grid) : grid_of_class<10, 8, long long>(sms, grid);
}

int class_of(int32_t table_log) { return table_log == kSmallClassLog[0] ? 0 : table_log == kSmallClassLog[1] ? 1 : -1; }

template <int LOGS, int WARPS, typename Acc>
spg_status launch_class(int grid, cudaStream_t st, const SmallArgs &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(WARPS * 32);
    cfg.dynamicSmemBytes = smem_of<LOGS, WARPS, Acc>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_check(cudaLaunchKernelEx(&cfg, k_small_multiply<LOGS, WARPS, Acc>, a), "one-launch multiply");
}

bool bad_header(const spg_csc *M) {
    return !M || !M->colptr || (M->nnz > 0 && (!M->rowidx || !M->vals)) || M->ptr_type < 0 || M->ptr_type > 1 ||
           M->idx_type < 0 || M->idx_type > 1 || M->val_type < 0 || M->val_type > 2 || M->nrows < 0 ||
           M->ncols < 0 || M->nnz < 0;
}

spg_status check_small(const spg_csc *A, const spg_csc *B, int32_t P, int64_t b) {
    if (bad_header(A) || bad_header(B) || P < 1 || b < 1) {
        set_error("one-launch multiply: NULL pointer, bad header, P < 1 or b < 1");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A has %lld columns, B has %lld rows", (long long)A->ncols, (long long)B->nrows);
        return SPG_INVALID_ARGUMENT;
    }
    if ((A->val_type == SPG_VAL_F64) != (B->val_type == SPG_VAL_F64)) {
        set_error("A and B must both hold doubles or both integers");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->idx_type != SPG_IDX_I32 || A->nrows >= (int64_t(1) << 31)) {
        set_error("the one-launch multiply needs 32-bit row ids of A");
        return SPG_UNSUPPORTED;
    }
    return SPG_OK;
}

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" spg_status spgemm_small_bound(const spg_csc *A, const spg_csc *B, int64_t *bound, void *stream) {
    clear_error();
    if (bad_header(A) || bad_header(B) || !bound) {
        set_error("spgemm_small_bound: NULL pointer or bad header");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A has %lld columns, B has %lld rows", (long long)A->ncols, (long long)B->nrows);
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    spg_status s = cuda_check(cudaMemsetAsync(bound, 0, 2 * sizeof(int64_t), st), "bound clear");
    if (s || B->ncols == 0) return s;
    int64_t blocks = (B->ncols + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_small_bound<<<(int)blocks, 256, 0, st>>>(A->colptr, A->ptr_type == SPG_IDX_I64, B->colptr,
                                                B->ptr_type == SPG_IDX_I64, B->rowidx, B->idx_type == SPG_IDX_I64,
                                                A->nrows, B->nrows, B->ncols, (unsigned long long *)bound);
    return cuda_check(cudaGetLastError(), "spgemm_small_bound launch");
}

extern "C" spg_status spgemm_small_workspace(const spg_csc *A, const spg_csc *B, int32_t P, int64_t b,
                                             int32_t table_log, size_t *bytes) {
    clear_error();
    spg_status s = check_small(A, B, P, b);
    if (s) return s;
    const int cls = class_of(table_log);
    if (!bytes || cls < 0) {
        set_error("bytes must not be NULL; table_log must be 8 or 10");
        return SPG_INVALID_ARGUMENT;
    }
    int grid = 0;
    s = small_grid(cls, A->val_type == SPG_VAL_F64, &grid);
    if (s) return s;
    *bytes = layout_of(B->nrows, B->ncols, P, b, grid).total;
    return SPG_OK;
}

extern "C" spg_status spgemm_small_multiply(const spg_csc *A, const spg_csc *B, int32_t P, int64_t b,
                                            int32_t table_log, void *workspace, size_t workspace_bytes,
                                            int64_t *C_colptr, int32_t *C_rowidx, void *C_vals, int64_t capacity,
                                            int64_t *result, int64_t timeout_ns, void *stream) {
    clear_error();
    spg::PhaseRange nvtx_range("spgemm_small_multiply");
    spg_status s = check_small(A, B, P, b);
    if (s) return s;
    const int cls = class_of(table_log);
    if (!workspace || !C_colptr || !result || capacity < 0 || (capacity > 0 && (!C_rowidx || !C_vals)) ||
        timeout_ns <= 0 || cls < 0) {
        set_error("one-launch multiply: NULL workspace / C / result, negative capacity, timeout_ns <= 0 or "
                  "table_log not 8 or 10");
        return SPG_INVALID_ARGUMENT;
    }
    const bool f64 = A->val_type == SPG_VAL_F64;
    int grid = 0;
    s = small_grid(cls, f64, &grid);
    if (s) return s;
    const Layout L = layout_of(B->nrows, B->ncols, P, b, grid);
    if (workspace_bytes < L.total) {
        set_error("workspace of %zu bytes, %zu needed (spgemm_small_workspace)", workspace_bytes, L.total);
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    s = cuda_check(cudaMemsetAsync(ws, 0, L.zero_bytes, st), "workspace clear");
    if (!s) s = cuda_check(cudaMemsetAsync(result, 0, sizeof(int64_t) * kResCount, st), "result clear");
    if (s) return s;
    SmallArgs a;
    a.Acp = A->colptr;
    a.ap64 = A->ptr_type == SPG_IDX_I64;
    a.Arow = (const int32_t *)A->rowidx;
    a.Aval = A->vals;
    a.avt = A->val_type;
    a.Bcp = B->colptr;
    a.bp64 = B->ptr_type == SPG_IDX_I64;
    a.Brow = B->rowidx;
    a.bi64 = B->idx_type == SPG_IDX_I64;
    a.Bval = B->vals;
    a.bvt = B->val_type;
    a.m = A->nrows;
    a.k = B->nrows;
    a.n = B->ncols;
    a.P = P;
    a.b = b;
    a.W = (a.k + 31) / 32;
    a.nfb = (a.k + b - 1) / b;
    a.bar = (unsigned *)(ws + L.bar);
    a.H = (uint32_t *)(ws + L.H);
    a.fetch = (uint8_t *)(ws + L.fetch);
    a.cnt = (int64_t *)(ws + L.cnt);
    a.chunk = (long long *)(ws + L.chunk);
    a.Ccp = C_colptr;
    a.Crow = C_rowidx;
    a.Cval = C_vals;
    a.capacity = capacity;
    a.res = (long long *)result;
    a.timeout_ns = timeout_ns;
    if (cls == 0)
        return f64 ? launch_class<8, 32, double>(grid, st, a) : launch_class<8, 32, long long>(grid, st, a);
    return f64 ? launch_class<10, 8, double>(grid, st, a) : launch_class<10, 8, long long>(grid, st, a);
}
