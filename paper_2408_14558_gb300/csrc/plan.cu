// Planning phase of the sparsity-aware 1D SpGEMM: steps 1-4 of Algorithm 1
// for all P column blocks at once, on one GPU.
//   k_nonempty_bits  D, the nonempty columns of A (Algorithm 1, allgather of
//                    nonzero column ids: here A.colptr is local)
//   k_block_eoff     the first entry of B of every column block
//   k_mark_H         H_i, nonzero rows of B_i (Table 1, Algorithm 1), one
//                    thread per entry of B
//   k_popc_HD        popc(H_i & D) per word, then a scan gives each required
//                    column its place in D~ (Algorithm 1, D~ = H_i AND D)
//   k_dtilde         the ascending list D~_i
//   k_fetch          Algorithm 2 with groups of b consecutive column ids
//   k_gather_len / k_gather_shift / k_gather_copy   A~_i = A(:, D~_i) for all
//                    blocks in one entry-balanced copy (on one GPU the chosen
//                    fetch blocks only give the volume Algorithm 2 transfers)
//   k_remap_B        B_i's rows k -> column of A~_i (Algorithm 1's local index)
//   k_col_stats      flops_j (Section 3.2), row window, features, bin id
//   k_split          heavy bins: per A~ column, the first entry of every row slab
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <new>

#include "spg_internal.cuh"

namespace spg {

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

const char *last_error_str() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

spg_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SPG_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return SPG_OUT_OF_MEMORY;
    return SPG_CUDA_ERROR;
}

// --------------------------------------------------------------- workspace

static void *ws_alloc_direct(spg_plan *p, size_t bytes);

// Workspace: requests up to kArenaMax bytes are carved from chunks of
// kArenaChunk bytes, each one allocator call (through the caller's callbacks
// these are calls into Python); larger requests get their own allocation.
// Everything is released by ws_free_all.
constexpr size_t kArenaMax = 1 << 20, kArenaChunk = 4 << 20;

void *ws_alloc(spg_plan *p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes > kArenaMax) return ws_alloc_direct(p, bytes);
    if (!p->arena || p->arena_used + bytes > p->arena_size) {
        p->arena = (char *)ws_alloc_direct(p, kArenaChunk);
        if (!p->arena) {
            p->arena_used = p->arena_size = 0;
            return nullptr;
        }
        p->arena_used = 0;
        p->arena_size = kArenaChunk;
    }
    void *ptr = p->arena + p->arena_used;
    p->arena_used += bytes;
    return ptr;
}

static void *ws_alloc_direct(spg_plan *p, size_t bytes) {
    void *ptr = nullptr;
    if (p->opt.alloc) {
        ptr = p->opt.alloc(bytes, p->opt.alloc_ctx, (void *)p->st);
    } else {
        if (cudaMallocAsync(&ptr, bytes, p->st) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
    }
    if (!ptr) {
        set_error("workspace allocation of %zu bytes failed", bytes);
        return nullptr;
    }
    p->allocs.push_back({ptr, bytes});
    return ptr;
}

void ws_free_all(spg_plan *p) {
    for (auto &a : p->allocs) {
        if (p->opt.free)
            p->opt.free(a.p, a.bytes, p->opt.alloc_ctx, (void *)p->st);
        else if (!p->opt.alloc)
            cudaFreeAsync(a.p, p->st);
    }
    p->allocs.clear();
    p->arena = nullptr;
    p->arena_used = p->arena_size = 0;
}

int grid_for(int64_t work, int per_block, int max_blocks) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

spg_status read_dev_err(spg_plan *p, const char *phase) {
    // the error word lands in the last pinned slot so that other read-backs
    // queued before this call stay intact
    int64_t *slot = p->h_pinned + 63;
    *slot = 0;
    spg_status s = cuda_check(
        cudaMemcpyAsync(slot, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st), phase);
    if (s) return s;
    s = cuda_check(cudaStreamSynchronize(p->st), phase);
    if (s) return s;
    int e = *(int *)slot;
    if (e & kDevErrInput) {
        set_error("%s: input matrix is not canonical CSC (colptr not monotone, or a row id out of range, unsorted or repeated)", phase);
        return SPG_INVALID_INPUT;
    }
    if (e & kDevErrRange) {
        set_error("%s: a size limit was exceeded", phase);
        return SPG_UNSUPPORTED;
    }
    if (e & kDevErrInternal) {
        set_error("%s: internal consistency check failed", phase);
        return SPG_CUDA_ERROR;
    }
    return SPG_OK;
}

// ------------------------------------------------------------------ kernels

// Device counters in plan->d_cnt.
enum {
    kCntSumH = 0,
    kCntProducts = 1,
    kCntFetchChosen = 2,
    kCntVolBlock = 3,
    kCntMaxAcol = 4,
    kCntBin0 = 8,  // kNumBins histogram counters
    kCntHeavyItems = 16,
    kCntNnzBHeavy = 17,
    kCntRemote = 21,
    kCntSlots = 24
};

// Input checks, in two passes that read the matrix once, coalesced.
// Per column: 0 <= colptr[j] <= colptr[j+1] <= nnz, colptr[0] = 0 and
// colptr[ncols] = nnz; the first entry of every non-empty column is marked in
// `starts` (one bit per entry, zeroed by the caller).
__global__ void k_validate_cols(const void *colptr, int p64, int64_t ncols, int64_t nnz, uint32_t *starts,
                                int *err) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (ld_ptr(colptr, p64, 0) != 0 || ld_ptr(colptr, p64, ncols) != nnz)) atomicOr(err, kDevErrInput);
    for (int64_t j = t0; j < ncols; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = ld_ptr(colptr, p64, j), e = ld_ptr(colptr, p64, j + 1);
        if (s > e || s < 0 || e > nnz)
            atomicOr(err, kDevErrInput);
        else if (s < e)
            atomicOr(starts + (s >> 5), 1u << (s & 31));
    }
}

// Per entry: 0 <= row < nrows, and rows strictly increase inside a column: a
// row not above its predecessor is allowed only where a column starts.
__global__ void k_validate_rows(const void *rowidx, int i64, int64_t nnz, int64_t nrows,
                                const uint32_t *__restrict__ starts, int *err) {
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = ld_ptr(rowidx, i64, q);
        if (r < 0 || r >= nrows)
            bad = true;
        else if (q > 0 && ld_ptr(rowidx, i64, q - 1) >= r && !((starts[q >> 5] >> (q & 31)) & 1u))
            bad = true;
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kDevErrInput);
}

__global__ void k_nonempty_bits(const void *colptr, int p64, int64_t k, int64_t W, uint32_t *D) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < W;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        int64_t h0 = w * 32;
        int64_t prev = ld_ptr(colptr, p64, h0);
        for (int bb = 0; bb < 32 && h0 + bb < k; bb++) {
            int64_t nx = ld_ptr(colptr, p64, h0 + bb + 1);
            if (nx > prev) bits |= 1u << bb;
            prev = nx;
        }
        D[w] = bits;
    }
}

// Flop-balanced split: flops of every column of B (Section 3.2 count, from
// A's column lengths), then bound_i = the smallest j with P * pre[j] >= i * F
// (pre = exclusive prefix of the flops, F = pre[n]), bound_0 = 0, bound_P = n.
__global__ void k_split_flops(const void *Bcp, int p64B, const void *Brow, int i64B, const void *Acp, int p64A,
                              int64_t n, int64_t *fl) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t s = ld_ptr(Bcp, p64B, j), e = ld_ptr(Bcp, p64B, j + 1);
        long long f = 0;
        for (int64_t q = s + lane; q < e; q += 32) {
            const int64_t kk = ld_ptr(Brow, i64B, q);
            f += ld_ptr(Acp, p64A, kk + 1) - ld_ptr(Acp, p64A, kk);
        }
        f = warp_sum_ll(f);
        if (lane == 0) fl[j] = f;
    }
}

__global__ void k_split_bounds(const int64_t *pre, int64_t n, int P, int64_t *bounds) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > P) return;
    if (i == 0 || i == P) {
        bounds[i] = i == 0 ? 0 : n;
        return;
    }
    const int64_t F = pre[n];
    int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]; P * pre[n] >= i * F always holds
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((__int128)P * pre[mid] >= (__int128)i * F)
            hi = mid;
        else
            lo = mid + 1;
    }
    bounds[i] = lo;
}

// Per-block flops of the plan's split (warp-aggregated when a warp's columns
// share a block).
__global__ void k_block_flops(const int64_t *flops, int64_t n, int P, const int64_t *bounds, long long *blk_flops) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = base + lane;
        const bool valid = j < n;
        const int i = valid ? block_of_b(j, n, P, bounds) : -1;
        const long long f = valid ? flops[j] : 0;
        const int i0 = __shfl_sync(kFull, i, 0);
        if (__all_sync(kFull, !valid || i == i0)) {
            const long long t = warp_sum_ll(f);
            if (lane == 0 && t) atomicAdd((unsigned long long *)(blk_flops + i0), (unsigned long long)t);
        } else if (valid && f) {
            atomicAdd((unsigned long long *)(blk_flops + i), (unsigned long long)f);
        }
    }
}

// Warp per column j of B: set bit r of H_{block(j)} for every stored row r.
// First entry of every column block of B: eoff[i] = colptr[bound_i], i <= P.
__global__ void k_block_eoff(const void *colptr, int p64, int64_t n, int P, const int64_t *bounds, int64_t *eoff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= P; i += gridDim.x * blockDim.x)
        eoff[i] = ld_ptr(colptr, p64, bounds ? bounds[i] : (int64_t)i * n / P);
}

// The column block of B's entry q: the largest i < P with eoff[i] <= q
// (empty blocks share their offset with the next one).
__device__ __forceinline__ int block_of_entry(int64_t q, const int64_t *__restrict__ eoff, int P) {
    int lo = 0, hi = P;  // eoff[lo] <= q < eoff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(eoff + mid) <= q)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// H_i: one atomicOr per entry of B into its block's bitmap (entry-parallel).
__global__ void k_mark_H(const void *rowidx, int i64, int64_t nnz, int P, int64_t W, uint32_t *H,
                         const int64_t *__restrict__ eoff) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = ld_ptr(rowidx, i64, q);
        const int i = block_of_entry(q, eoff, P);
        atomicOr(H + (int64_t)i * W + (r >> 5), 1u << (r & 31));
    }
}

// cnt[i*W + w] = popc(H_i[w] & D[w]); also sum_i |H_i| for the statistics.
__global__ void k_popc_HD(const uint32_t *H, const uint32_t *D, int64_t W, int64_t total,
                          int32_t *cnt, long long *sumH) {
    long long h = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint32_t hw = H[x];
        cnt[x] = __popc(hw & D[x % W]);
        h += __popc(hw);
    }
    h = warp_sum_ll(h);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd((unsigned long long *)sumH, (unsigned long long)h);
}

// Global index in D~ of the first required column >= x in block i.
__device__ __forceinline__ int64_t rank_at(const uint32_t *H, const uint32_t *D, const int64_t *rankpre,
                                           int64_t W, int i, int64_t x) {
    int64_t w = x >> 5;
    int64_t r = rankpre[(int64_t)i * W + w];
    if (x & 31) r += __popc(H[(int64_t)i * W + w] & D[w] & ((1u << (x & 31)) - 1u));
    return r;
}

__global__ void k_dtilde(const uint32_t *H, const uint32_t *D, const int64_t *rankpre, int64_t W,
                         int64_t total, int32_t *dtilde) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t w = x % W;
        uint32_t bits = H[x] & D[w];
        int64_t base = rankpre[x];
        while (bits) {
            int bb = __ffs(bits) - 1;
            dtilde[base++] = (int32_t)(w * 32 + bb);
            bits &= bits - 1;
        }
    }
}

// Algorithm 2: fetch block t of block i is chosen iff it contains a required column.
__global__ void k_fetch(const uint32_t *H, const uint32_t *D, const int64_t *rankpre, int64_t W,
                        int64_t k, int64_t b, int64_t nfb, int P, const void *Acolptr, int p64,
                        uint8_t *fetch, long long *chosen, long long *volblock) {
    long long c = 0, v = 0;
    int64_t total = nfb * P;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(x / nfb);
        int64_t t = x % nfb;
        int64_t lo = t * b, hi = min(k, lo + b);
        bool f = rank_at(H, D, rankpre, W, i, hi) > rank_at(H, D, rankpre, W, i, lo);
        fetch[x] = f ? 1 : 0;
        if (f) {
            c++;
            v += ld_ptr(Acolptr, p64, hi) - ld_ptr(Acolptr, p64, lo);
        }
    }
    c = warp_sum_ll(c);
    v = warp_sum_ll(v);
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd((unsigned long long *)chosen, (unsigned long long)c);
        if (v) atomicAdd((unsigned long long *)volblock, (unsigned long long)v);
    }
}

// Length of every A~ column, the longest, and the entries whose column lies
// outside the block's own column range [floor(i*k/P), floor((i+1)*k/P)) of A
// (what a distributed run fetches from other owners); dt_base (P + 1) gives
// each block's range of D~ entries.
__global__ void k_gather_len(const int32_t *dtilde, int64_t ndt, const void *Acolptr, int p64,
                             int64_t *len, long long *maxlen, const int64_t *dt_base, int P, int64_t k,
                             long long *remote, long long *blk_gathered, long long *blk_remote) {
    const int lane = threadIdx.x & 31;
    long long mx = 0, rem = 0;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < ndt;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = base + lane;
        const bool valid = g < ndt;
        long long l = 0, lr = 0;
        int lo = -1;
        if (valid) {
            const int64_t h = dtilde[g];
            l = ld_ptr(Acolptr, p64, h + 1) - ld_ptr(Acolptr, p64, h);
            len[g] = l;
            mx = max(mx, l);
            lo = 0;
            int hi = P;  // the block i with dt_base[i] <= g < dt_base[i + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (dt_base[mid] <= g)
                    lo = mid;
                else
                    hi = mid;
            }
            if (h < (int64_t)lo * k / P || h >= (int64_t)(lo + 1) * k / P) lr = l;
            rem += lr;
        }
        // per-block sums, one atomic per warp when its entries share a block
        const int b0 = __shfl_sync(kFull, lo, 0);
        if (__all_sync(kFull, !valid || lo == b0)) {
            const long long tl = warp_sum_ll(l), tr = warp_sum_ll(lr);
            if (lane == 0 && tl) atomicAdd((unsigned long long *)(blk_gathered + b0), (unsigned long long)tl);
            if (lane == 0 && tr) atomicAdd((unsigned long long *)(blk_remote + b0), (unsigned long long)tr);
        } else if (valid) {
            if (l) atomicAdd((unsigned long long *)(blk_gathered + lo), (unsigned long long)l);
            if (lr) atomicAdd((unsigned long long *)(blk_remote + lo), (unsigned long long)lr);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        rem += __shfl_xor_sync(kFull, rem, o);
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax((unsigned long long *)maxlen, (unsigned long long)mx);
    if ((threadIdx.x & 31) == 0 && rem) atomicAdd((unsigned long long *)remote, (unsigned long long)rem);
}

template <typename Acc>
__device__ __forceinline__ Acc load_val(const void *v, int vt, int64_t i);
template <>
__device__ __forceinline__ double load_val<double>(const void *v, int, int64_t i) {
    return __ldg((const double *)v + i);
}
template <>
__device__ __forceinline__ long long load_val<long long>(const void *v, int vt, int64_t i) {
    return vt == SPG_VAL_I32 ? (long long)__ldg((const int *)v + i) : (long long)__ldg((const long long *)v + i);
}

// Per A~ column g: the entry e of A~ sits at position e + shift[g] of A.
__global__ void k_gather_shift(const int32_t *dtilde, int64_t ndt, const void *Acolptr, int p64,
                               const int64_t *At_colptr, int64_t *shift) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ndt; g += (int64_t)gridDim.x * blockDim.x)
        shift[g] = ld_ptr(Acolptr, p64, dtilde[g]) - At_colptr[g];
}

// A~ = A(:, D~) for all blocks at once (rows narrowed to int32, values widened
// to the accumulation type), balanced by entries: warp w copies the entries
// [w * chunk, (w + 1) * chunk) of A~.  It finds the column of its first entry
// by a 32-way search of At_colptr, then walks 32 entries a step; every A~
// column is non-empty (D~ is a subset of D), so the column starts inside a
// step mark distinct positions and one warp OR-reduction gives each lane its
// column.
template <typename Acc>
__global__ void k_gather_copy(const int64_t *__restrict__ At_colptr, const int64_t *__restrict__ shift, int64_t ndt,
                              int64_t nAt, int64_t chunk, const void *Arow, int i64, const void *Aval, int vt,
                              int32_t *__restrict__ At_row, Acc *__restrict__ At_val) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t e0 = w * chunk, e1 = min(nAt, e0 + chunk);
    if (e0 >= e1) return;  // the whole warp
    // largest g with At_colptr[g] <= e0, searched in [lo, hi)
    int64_t lo = 0, hi = ndt;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t idx = lo + lane * step;
        const uint32_t b = __ballot_sync(kFull, idx < hi && At_colptr[idx] <= e0);
        lo += (31 - __clz(b)) * step;  // lane 0 always votes yes
        hi = min(hi, lo + step);
    }
    {
        const int64_t idx = lo + lane;
        const uint32_t b = __ballot_sync(kFull, idx < hi && At_colptr[idx] <= e0);
        lo += 31 - __clz(b);
    }
    int64_t s0 = lo;  // the column holding entry f
    for (int64_t f = e0; f < e1; f += 32) {
        // lane k holds column s0 + k: its start and its shift
        const int64_t sk = s0 + lane;
        const int64_t bk = sk < ndt ? At_colptr[sk] : INT64_MAX;
        const int64_t shk = sk < ndt ? shift[sk] : 0;
        const int64_t pos = bk - f;  // >= 1 for k >= 1
        const uint32_t M = __reduce_or_sync(kFull, (lane > 0 && pos < 32) ? (1u << (int)pos) : 0u);
        const int k = __popc(M & ((2u << lane) - 1u));
        const int64_t sh = __shfl_sync(kFull, shk, k);
        const int64_t e = f + lane;
        if (e < e1) {
            const int64_t src = e + sh;
            At_row[e] = (int32_t)ld_ptr(Arow, i64, src);
            At_val[e] = load_val<Acc>(Aval, vt, src);
        }
        // the column holding f + 32
        int c = __popc(M);
        int64_t nb;
        if (c < 31)
            nb = __shfl_sync(kFull, bk, c + 1);
        else
            nb = s0 + 32 < ndt ? At_colptr[s0 + 32] : INT64_MAX;
        if (nb == f + 32) c++;
        s0 += c;
    }
}

// Every entry of B_i (entry-parallel): its row k becomes its column index in
// A~ (or -1 when A(:, k) is empty), its value the accumulation type.
template <typename Acc>
__global__ void k_remap_B(const void *rowidx, int i64, const void *vals, int vt, int64_t nnz, int P,
                          const uint32_t *__restrict__ H, const uint32_t *__restrict__ D,
                          const int64_t *__restrict__ rankpre, int64_t W, int32_t *Bq, Acc *Bv,
                          const int64_t *__restrict__ eoff) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = ld_ptr(rowidx, i64, q);
        const int i = block_of_entry(q, eoff, P);
        const int64_t w = r >> 5;
        const uint32_t word = H[(int64_t)i * W + w] & D[w];
        const uint32_t sh = (uint32_t)(r & 31);
        int32_t loc = -1;
        if ((word >> sh) & 1u) loc = (int32_t)(rankpre[(int64_t)i * W + w] + __popc(word & ((1u << sh) - 1u)));
        Bq[q] = loc;
        Bv[q] = load_val<Acc>(vals, vt, q);
    }
}

__device__ __forceinline__ int light_bin(long long U, int light_max) {
    if (U <= 0) return kBinEmpty;
    if (U > light_max) return kBinHeavy;
    // table size S = max(64, next power of two >= 2U); bin = log2(S) - 5
    long long S = 64;
    int bin = 1;
    while (S < 2 * U) {
        S <<= 1;
        bin++;
    }
    return bin;
}

// Warp per output column: flops_j, the row window of its products, the MLP
// features and the symbolic bin (bound U = min(flops_j, window)).
__global__ void k_col_stats(const void *Bcolptr, int p64, int64_t n, const int32_t *Bq,
                            const int64_t *At_colptr, const int32_t *At_row, int light_max,
                            int64_t *flops, int32_t *win_lo, int32_t *win_hi, int32_t *nnzb,
                            int32_t *maxa, int8_t *bin_of, long long *bincnt, long long *products) {
    __shared__ int hist[kNumBins];
    __shared__ long long prod_sh;
    if (threadIdx.x < kNumBins) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) prod_sh = 0;
    __syncthreads();
    int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    long long prod_local = 0;
    for (int64_t j = warp; j < n; j += nwarps) {
        int64_t s = ld_ptr(Bcolptr, p64, j), e = ld_ptr(Bcolptr, p64, j + 1);
        long long fl = 0;
        int mx = 0, lo = INT32_MAX, hi = -1;
        // four entries per lane and step, each stage's loads issued together
        // (long columns of B would otherwise be a chain of dependent loads)
        for (int64_t q0 = s + lane; q0 < e; q0 += 32 * 4) {
            int loc[4];
            int64_t a0[4], a1[4];
#pragma unroll
            for (int u = 0; u < 4; u++) loc[u] = q0 + 32 * u < e ? Bq[q0 + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                a0[u] = loc[u] >= 0 ? At_colptr[loc[u]] : 0;
                a1[u] = loc[u] >= 0 ? At_colptr[loc[u] + 1] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int len = (int)(a1[u] - a0[u]);
                fl += len;
                mx = max(mx, len);
                if (len > 0) {
                    lo = min(lo, At_row[a0[u]]);
                    hi = max(hi, At_row[a1[u] - 1]);
                }
            }
        }
        fl = warp_sum_ll(fl);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = max(mx, __shfl_xor_sync(kFull, mx, o));
            lo = min(lo, __shfl_xor_sync(kFull, lo, o));
            hi = max(hi, __shfl_xor_sync(kFull, hi, o));
        }
        if (lane == 0) {
            flops[j] = fl;
            win_lo[j] = fl ? lo : 0;
            win_hi[j] = fl ? hi : -1;
            nnzb[j] = (int32_t)(e - s);
            maxa[j] = mx;
            long long U = fl ? min(fl, (long long)(hi - lo + 1)) : 0;
            int bin = light_bin(U, light_max);
            bin_of[j] = (int8_t)bin;
            atomicAdd(&hist[bin], 1);
            prod_local += fl;
        }
    }
    if (lane == 0 && prod_local) atomicAdd((unsigned long long *)&prod_sh, (unsigned long long)prod_local);
    __syncthreads();
    if (threadIdx.x < kNumBins && hist[threadIdx.x])
        atomicAdd((unsigned long long *)&bincnt[threadIdx.x], (unsigned long long)hist[threadIdx.x]);
    if (threadIdx.x == 0 && prod_sh) atomicAdd((unsigned long long *)products, (unsigned long long)prod_sh);
}

// Stable counting sort of column ids by bin.  Columns are cut into chunks of
// kBinChunk; cnt[bin * nchunks + chunk] counts each chunk's columns per bin, a
// scan of cnt (bin-major) gives every (bin, chunk) its first slot, and the
// scatter keeps column order inside each chunk.  Within a bin the columns are
// therefore ascending, so the heavy items of block i run before those of
// block i + 1 and share A~_i in L2.
constexpr int kBinChunk = 2048;

__global__ void k_bin_chunk_count(const int8_t *bin_of, int64_t n, int64_t nchunks, int32_t *cnt) {
    __shared__ int h[kNumBins];
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (threadIdx.x < kNumBins) h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t j0 = c * kBinChunk;
        for (int i = threadIdx.x; i < kBinChunk; i += blockDim.x) {
            int64_t j = j0 + i;
            if (j < n) atomicAdd(&h[bin_of[j]], 1);
        }
        __syncthreads();
        if (threadIdx.x < kNumBins) cnt[(int64_t)threadIdx.x * nchunks + c] = h[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
    k_bin_chunk_scatter(const int8_t *bin_of, int64_t n, int64_t nchunks, const int64_t *off, int32_t *list) {
    __shared__ int run[kNumBins];
    __shared__ int wcnt[8][kNumBins];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (threadIdx.x < kNumBins) run[threadIdx.x] = 0;
        __syncthreads();
        for (int r = 0; r < kBinChunk; r += blockDim.x) {
            const int64_t j = c * kBinChunk + r + threadIdx.x;
            const int b = j < n ? bin_of[j] : -1;
            int myrank = 0;
#pragma unroll
            for (int bb = 0; bb < kNumBins; bb++) {
                unsigned m = __ballot_sync(kFull, b == bb);
                if (b == bb) myrank = __popc(m & ((1u << lane) - 1u));
                if (lane == 0) wcnt[wid][bb] = __popc(m);
            }
            __syncthreads();
            if (b >= 0) {
                int before = run[b];
                for (int w = 0; w < wid; w++) before += wcnt[w][b];
                list[off[(int64_t)b * nchunks + c] + before + myrank] = (int32_t)j;
            }
            __syncthreads();
            if (threadIdx.x < kNumBins) {
                int tot = 0;
                for (int w = 0; w < nw; w++) tot += wcnt[w][threadIdx.x];
                run[threadIdx.x] += tot;
            }
            __syncthreads();
        }
    }
}

spg_status bin_columns(spg_plan *p, const int8_t *bin_of, int32_t *list, int64_t *off_host) {
    const int64_t n = p->n;
    const int64_t nchunks = (n + kBinChunk - 1) / kBinChunk;
    const int64_t ncnt = nchunks * kNumBins;
    int32_t *cnt = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(ncnt + 1));
    int64_t *off = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(ncnt + 1));
    if (!cnt || !off) return SPG_OUT_OF_MEMORY;
    const int g = grid_for(nchunks, 1, p->sm_count * 8);
    launch(p, k_bin_chunk_count, g, 256, 0, bin_of, n, nchunks, cnt);
    spg_status s = scan_exclusive_i32(p, cnt, off, ncnt);
    if (s) return s;
    for (int b = 0; b <= kNumBins; b++) {
        s = cuda_check(cudaMemcpyAsync(p->h_pinned + b, off + (int64_t)b * nchunks, sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, p->st), "bin readback");
        if (s) return s;
    }
    launch(p, k_bin_chunk_scatter, g, 256, 0, bin_of, n, nchunks, (const int64_t *)off, list);
    s = cuda_check(cudaGetLastError(), "bin scatter");
    if (s) return s;
    s = cuda_check(cudaStreamSynchronize(p->st), "bin readback");
    if (s) return s;
    for (int b = 0; b <= kNumBins; b++) off_host[b] = p->h_pinned[b];
    return SPG_OK;
}

// Heavy bins: slabs [t_lo, t_hi] of every heavy column from its row window.
__global__ void k_heavy_nslab(const int32_t *list, int64_t nheavy, const int32_t *win_lo,
                              const int32_t *win_hi, const int32_t *nnzb, int R, int64_t *nslab,
                              long long *nnzb_heavy) {
    long long sb = 0;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x) {
        int j = list[h];
        nslab[h] = (int64_t)(win_hi[j] / R - win_lo[j] / R + 1);
        sb += nnzb[j];
    }
    sb = warp_sum_ll(sb);
    if ((threadIdx.x & 31) == 0 && sb) atomicAdd((unsigned long long *)nnzb_heavy, (unsigned long long)sb);
}

// Records (column, base slab) of every heavy column, and the number of
// symbolic items (groups of <= smr consecutive records) it needs.
__global__ void k_heavy_records(const int32_t *list, int64_t nheavy, const int32_t *win_lo, int R, int smr,
                                const int64_t *rec_first, int32_t *rec_col, int32_t *rec_slab, int64_t *nsym) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x) {
        int j = list[h];
        int t0 = win_lo[j] / R;
        for (int64_t r = rec_first[h]; r < rec_first[h + 1]; r++) {
            rec_col[r] = j;
            rec_slab[r] = t0 + (int)(r - rec_first[h]);
        }
        nsym[h] = (rec_first[h + 1] - rec_first[h] + smr - 1) / smr;
    }
}

__global__ void k_sym_items(int64_t nheavy, int smr, const int64_t *rec_first, const int64_t *sym_first,
                            int32_t *sym_rec0, int32_t *sym_nrec) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = rec_first[h], e = rec_first[h + 1];
        for (int64_t it = sym_first[h]; it < sym_first[h + 1]; it++) {
            sym_rec0[it] = (int32_t)r;
            sym_nrec[it] = (int32_t)min((int64_t)smr, e - r);
            r += smr;
        }
    }
}

// split[q*(T+1) + t] = offset in A~ column q of its first row >= t*R.
__global__ void k_split(const int64_t *At_colptr, const int32_t *At_row, int64_t nq, int T, int R,
                        int32_t *split) {
    int64_t total = nq * (int64_t)(T + 1);
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = x / (T + 1);
        int t = (int)(x % (T + 1));
        int64_t s = At_colptr[q], e = At_colptr[q + 1];
        long long bound = (long long)t * R;
        int64_t lo = s, hi = e;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((long long)At_row[mid] < bound)
                lo = mid + 1;
            else
                hi = mid;
        }
        split[x] = (int32_t)(lo - s);
    }
}

// ------------------------------------------------------------------ host

// Step 3 and the remap of B: A~ = A(:, D~) (rows and values, entry-balanced)
// and B's entries as (column of A~, value).  Launches only, so that
// spgemm_numeric_refresh can re-run it (new values, same patterns) inside a
// captured graph; its scratch is allocated once.
spg_status copy_operands(spg_plan *p) {
    const spg_csc &A = p->A, &B = p->B;
    const int sm = p->sm_count, P = p->P;
    const int64_t W = p->W;
    const int p64A = A.ptr_type == SPG_IDX_I64, i64A = A.idx_type == SPG_IDX_I64;
    const int i64B = B.idx_type == SPG_IDX_I64;
    if (p->ndt > 0 && p->nAt > 0) {
        if (!p->gshift) p->gshift = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)p->ndt);
        if (!p->gshift) return SPG_OUT_OF_MEMORY;
        // about 2048 entries per warp, at most 32 CTAs of 8 warps per SM
        const int64_t warps = std::max<int64_t>(1, std::min<int64_t>((p->nAt + 2047) / 2048, (int64_t)sm * 32 * 8));
        const int64_t chunk = ((p->nAt + warps - 1) / warps + 31) & ~(int64_t)31;
        const int64_t g = (((p->nAt + chunk - 1) / chunk) + 7) / 8;
        group_begin(p, kKGather);
        launch(p, k_gather_shift, grid_for(p->ndt, 256, sm * 8), 256, 0, p->dtilde, p->ndt, A.colptr, p64A,
               p->At_colptr, p->gshift);
        if (p->acc_f64)
            launch(p, k_gather_copy<double>, (unsigned)g, 256, 0, p->At_colptr, p->gshift, p->ndt, p->nAt, chunk,
                   A.rowidx, i64A, A.vals, A.val_type, p->At_row, (double *)p->At_val);
        else
            launch(p, k_gather_copy<long long>, (unsigned)g, 256, 0, p->At_colptr, p->gshift, p->ndt, p->nAt, chunk,
                   A.rowidx, i64A, A.vals, A.val_type, p->At_row, (long long *)p->At_val);
        group_end(p, kKGather);
        spg_status s = cuda_check(cudaGetLastError(), "gather");
        if (s) return s;
    }
    if (B.nnz > 0) {
        int g = grid_for(B.nnz, 256, sm * 16);
        if (p->acc_f64)
            launch(p, k_remap_B<double>, g, 256, 0, B.rowidx, i64B, B.vals, B.val_type, B.nnz, P, p->Hbits, p->Dbits,
                   p->rankpre, W, p->Bq, (double *)p->Bv, (const int64_t *)p->eoff);
        else
            launch(p, k_remap_B<long long>, g, 256, 0, B.rowidx, i64B, B.vals, B.val_type, B.nnz, P, p->Hbits,
                   p->Dbits, p->rankpre, W, p->Bq, (long long *)p->Bv, (const int64_t *)p->eoff);
        return cuda_check(cudaGetLastError(), "remap B");
    }
    return SPG_OK;
}

static bool valid_type(int32_t v, int maxv) { return v >= 0 && v <= maxv; }

static spg_status check_csc(const spg_csc *M, const char *name) {
    if (!M) {
        set_error("%s is NULL", name);
        return SPG_INVALID_ARGUMENT;
    }
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0 || !valid_type(M->ptr_type, 1) ||
        !valid_type(M->idx_type, 1) || !valid_type(M->val_type, 2)) {
        set_error("%s: negative size or unknown type code", name);
        return SPG_INVALID_ARGUMENT;
    }
    if (!M->colptr || (M->nnz > 0 && (!M->rowidx || !M->vals))) {
        set_error("%s: missing array pointer", name);
        return SPG_INVALID_ARGUMENT;
    }
    if (M->ptr_type == SPG_IDX_I32 && M->nnz > INT32_MAX) {
        set_error("%s: nnz does not fit its int32 column pointers", name);
        return SPG_INVALID_ARGUMENT;
    }
    return SPG_OK;
}

#define TRY(x)                        \
    do {                              \
        spg_status _s = (x);          \
        if (_s != SPG_OK) return _s;  \
    } while (0)
#define LAUNCH_OK(what) TRY(cuda_check(cudaGetLastError(), what))

static spg_status plan_build(spg_plan *p) {
    const spg_csc &A = p->A, &B = p->B;
    cudaStream_t st = p->st;
    const int64_t m = p->m, k = p->k, n = p->n;
    const int P = p->P;
    const int sm = p->sm_count;
    const int p64A = A.ptr_type == SPG_IDX_I64;
    const int p64B = B.ptr_type == SPG_IDX_I64, i64B = B.idx_type == SPG_IDX_I64;
    const size_t accsz = 8;

    p->d_err = (int *)ws_alloc(p, sizeof(int) * 4);
    p->d_cnt = (int64_t *)ws_alloc(p, sizeof(int64_t) * kCntSlots);
    p->d_bincur = (int64_t *)ws_alloc(p, sizeof(int64_t) * kNumBins);
    if (!p->d_err || !p->d_cnt || !p->d_bincur) return SPG_OUT_OF_MEMORY;
    TRY(cuda_check(cudaMemsetAsync(p->d_err, 0, sizeof(int) * 4, st), "memset"));
    TRY(cuda_check(cudaMemsetAsync(p->d_cnt, 0, sizeof(int64_t) * kCntSlots, st), "memset"));
    cudaEventRecord(p->ev[0], st);

    if (p->opt.validate) {
        const int64_t sw = (std::max<int64_t>(A.nnz, B.nnz) + 31) / 32 + 1;
        uint32_t *starts = (uint32_t *)ws_alloc(p, sizeof(uint32_t) * (size_t)sw);
        if (!starts) return SPG_OUT_OF_MEMORY;
        const spg_csc *M[2] = {&A, &B};
        for (int i = 0; i < 2; i++) {
            const int pp = M[i]->ptr_type == SPG_IDX_I64, ii = M[i]->idx_type == SPG_IDX_I64;
            TRY(cuda_check(cudaMemsetAsync(starts, 0, sizeof(uint32_t) * (size_t)sw, st), "memset"));
            launch(p, k_validate_cols, grid_for(M[i]->ncols + 1, 256, sm * 8), 256, 0, M[i]->colptr, pp,
                   M[i]->ncols, M[i]->nnz, starts, p->d_err);
            if (M[i]->nnz > 0)
                launch(p, k_validate_rows, grid_for(M[i]->nnz, 256, sm * 16), 256, 0, M[i]->rowidx, ii, M[i]->nnz,
                       M[i]->nrows, (const uint32_t *)starts, p->d_err);
        }
        LAUNCH_OK("validate");
        TRY(read_dev_err(p, "input validation"));
    }

    // --- column blocks: uniform, or contiguous with balanced flops
    p->blk = (int64_t *)ws_alloc(p, sizeof(int64_t) * 3 * (size_t)P);
    if (!p->blk) return SPG_OUT_OF_MEMORY;
    TRY(cuda_check(cudaMemsetAsync(p->blk, 0, sizeof(int64_t) * 3 * (size_t)P, st), "memset"));
    p->bounds_h.resize(P + 1);
    for (int i = 0; i <= P; i++) p->bounds_h[i] = (int64_t)i * n / P;
    if (p->opt.split == SPG_SPLIT_FLOPS && P > 1 && n > 0) {
        int64_t *fl = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
        int64_t *pre = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
        p->bounds_d = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(P + 1));
        if (!fl || !pre || !p->bounds_d) return SPG_OUT_OF_MEMORY;
        launch(p, k_split_flops, grid_for(n * 32, 256, sm * 16), 256, 0, B.colptr, p64B, B.rowidx, i64B, A.colptr,
               p64A, n, fl);
        TRY(scan_exclusive_i64(p, fl, pre, n));
        launch(p, k_split_bounds, grid_for(P + 1, 256, sm), 256, 0, pre, n, P, p->bounds_d);
        LAUNCH_OK("flop split");
        int64_t *hb = p->h_pinned + 64;
        TRY(cuda_check(cudaMemcpyAsync(hb, p->bounds_d, sizeof(int64_t) * (size_t)(P + 1), cudaMemcpyDeviceToHost, st),
                       "split readback"));
        TRY(cuda_check(cudaStreamSynchronize(st), "split readback"));
        p->bounds_h.assign(hb, hb + P + 1);
    }

    // --- step 1: D and H_i
    p->W = (k + 31) / 32;
    const int64_t W = p->W;
    p->Dbits = (uint32_t *)ws_alloc(p, sizeof(uint32_t) * (size_t)(W + 1));
    p->Hbits = (uint32_t *)ws_alloc(p, sizeof(uint32_t) * (size_t)(P * W + 1));
    p->rankpre = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(P * W + 1));
    int32_t *popc = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(P * W + 1));
    p->nfb = (k + p->b - 1) / p->b;
    p->fetch = (uint8_t *)ws_alloc(p, (size_t)(P * p->nfb + 1));
    if (!p->Dbits || !p->Hbits || !p->rankpre || !popc || !p->fetch) return SPG_OUT_OF_MEMORY;
    p->eoff = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(P + 1));
    if (!p->eoff) return SPG_OUT_OF_MEMORY;
    TRY(cuda_check(cudaMemsetAsync(p->Hbits, 0, sizeof(uint32_t) * (size_t)(P * W + 1), st), "memset H"));
    if (W > 0) launch(p, k_nonempty_bits, grid_for(W, 256, sm * 8), 256, 0, A.colptr, p64A, k, W, p->Dbits);
    launch(p, k_block_eoff, grid_for(P + 1, 256, sm), 256, 0, B.colptr, p64B, n, P, (const int64_t *)p->bounds_d,
           p->eoff);
    if (B.nnz > 0)
        launch(p, k_mark_H, grid_for(B.nnz, 256, sm * 16), 256, 0, B.rowidx, i64B, B.nnz, P, W, p->Hbits,
               (const int64_t *)p->eoff);
    LAUNCH_OK("mark H");

    // --- step 2: D~_i = H_i & D, its ranks and Algorithm 2
    int64_t PW = (int64_t)P * W;
    if (PW > 0)
        launch(p, k_popc_HD, grid_for(PW, 256, sm * 8), 256, 0, p->Hbits, p->Dbits, W, PW, popc,
                                                            (long long *)(p->d_cnt + kCntSumH));
    TRY(scan_exclusive_i32(p, popc, p->rankpre, PW));
    // |D~| in total and per block: read the block boundaries of the scan
    std::vector<int64_t> idx(P + 1);
    for (int i = 0; i <= P; i++) idx[i] = (int64_t)i * W;
    int64_t *hb = p->h_pinned + 64;
    for (int i = 0; i <= P; i++)
        TRY(cuda_check(cudaMemcpyAsync(hb + i, p->rankpre + idx[i], sizeof(int64_t), cudaMemcpyDeviceToHost, st),
                       "rank readback"));
    TRY(cuda_check(cudaStreamSynchronize(st), "rank readback"));
    p->dt_base.assign(hb, hb + P + 1);
    p->ndt = p->dt_base[P];
    if (p->ndt >= INT32_MAX) {
        set_error("sum of |D~_i| (%lld) exceeds int32", (long long)p->ndt);
        return SPG_UNSUPPORTED;
    }
    p->dtilde = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->ndt + 1));
    p->At_colptr = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->ndt + 1));
    int64_t *glen = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->ndt + 1));
    int64_t *d_dt_base = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(P + 1));
    if (!p->dtilde || !p->At_colptr || !glen || !d_dt_base) return SPG_OUT_OF_MEMORY;
    TRY(cuda_check(cudaMemcpyAsync(d_dt_base, hb, sizeof(int64_t) * (size_t)(P + 1), cudaMemcpyHostToDevice, st),
                   "block offsets"));
    if (PW > 0) launch(p, k_dtilde, grid_for(PW, 256, sm * 8), 256, 0, p->Hbits, p->Dbits, p->rankpre, W, PW, p->dtilde);
    if (P * p->nfb > 0)
        launch(p, k_fetch, grid_for(P * p->nfb, 256, sm * 8), 256, 0,
            p->Hbits, p->Dbits, p->rankpre, W, k, p->b, p->nfb, P, A.colptr, p64A, p->fetch,
            (long long *)(p->d_cnt + kCntFetchChosen), (long long *)(p->d_cnt + kCntVolBlock));
    LAUNCH_OK("dtilde / fetch");

    // --- step 3: gather A~
    if (p->ndt > 0)
        launch(p, k_gather_len, grid_for(p->ndt, 256, sm * 8), 256, 0, p->dtilde, p->ndt, A.colptr, p64A, glen,
                                                                  (long long *)(p->d_cnt + kCntMaxAcol), d_dt_base, P, k, (long long *)(p->d_cnt + kCntRemote),
               (long long *)(p->blk + P), (long long *)(p->blk + 2 * P));
    TRY(scan_exclusive_i64(p, glen, p->At_colptr, p->ndt));
    TRY(cuda_check(cudaMemcpyAsync(p->h_pinned, p->At_colptr + p->ndt, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "readback"));
    TRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 1, p->d_cnt + kCntMaxAcol, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "readback"));
    TRY(cuda_check(cudaStreamSynchronize(st), "readback"));
    p->nAt = p->h_pinned[0];
    if (p->h_pinned[1] >= (1LL << 26)) {
        set_error("a column of A holds %lld nonzeros; this build supports < 2^26 per column", (long long)p->h_pinned[1]);
        return SPG_UNSUPPORTED;
    }
    p->At_row = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->nAt + 1));
    p->At_val = ws_alloc(p, accsz * (size_t)(p->nAt + 1));
    p->Bq = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->nnzB + 1));
    p->Bv = ws_alloc(p, accsz * (size_t)(p->nnzB + 1));
    if (!p->At_row || !p->At_val || !p->Bq || !p->Bv) return SPG_OUT_OF_MEMORY;
    TRY(copy_operands(p));

    // --- step 4: flops, windows, bins
    p->flops = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    p->win_lo = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    p->win_hi = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    p->nnzb = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    p->maxa = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    p->bin_of = (int8_t *)ws_alloc(p, (size_t)(n + 1));
    p->binlist = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    p->nnzcol = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    p->Ccolptr = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    if (!p->flops || !p->win_lo || !p->win_hi || !p->nnzb || !p->maxa || !p->bin_of || !p->binlist ||
        !p->nnzcol || !p->Ccolptr)
        return SPG_OUT_OF_MEMORY;
    if (n > 0) {
        launch(p, k_col_stats, grid_for(n * 32, 256, sm * 16), 256, 0,
            B.colptr, p64B, n, p->Bq, p->At_colptr, p->At_row, p->light_max, p->flops, p->win_lo, p->win_hi,
            p->nnzb, p->maxa, p->bin_of, (long long *)(p->d_cnt + kCntBin0), (long long *)(p->d_cnt + kCntProducts));
        launch(p, k_block_flops, grid_for(n, 256, sm * 8), 256, 0, p->flops, n, P, p->bounds_d, (long long *)p->blk);
        LAUNCH_OK("column stats");
        TRY(bin_columns(p, p->bin_of, p->binlist, p->bin_off));
    }
    p->nheavy = p->bin_off[kBinHeavy + 1] - p->bin_off[kBinHeavy];

    // --- heavy bins: slab items and the split index of A~
    p->T = (int)((m + p->R - 1) / p->R);
    if (p->T < 1) p->T = 1;
    if (p->nheavy > 0) {
        const int32_t *hl = p->binlist + p->bin_off[kBinHeavy];
        int64_t *nslab = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        int64_t *nsym = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        int64_t *sym_first = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        p->rec_first = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        if (!nslab || !nsym || !sym_first || !p->rec_first) return SPG_OUT_OF_MEMORY;
        launch(p, k_heavy_nslab, grid_for(p->nheavy, 256, sm * 8), 256, 0, hl, p->nheavy, p->win_lo, p->win_hi,
               p->nnzb, p->R, nslab, (long long *)(p->d_cnt + kCntNnzBHeavy));
        TRY(scan_exclusive_i64(p, nslab, p->rec_first, p->nheavy));
        TRY(cuda_check(cudaMemcpyAsync(p->h_pinned, p->rec_first + p->nheavy, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "records"));
        TRY(cuda_check(cudaStreamSynchronize(st), "records"));
        p->nrec = p->h_pinned[0];
        if (p->nrec >= INT32_MAX) {
            set_error("too many heavy slab records (%lld)", (long long)p->nrec);
            return SPG_UNSUPPORTED;
        }
        p->rec_col = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)p->nrec);
        p->rec_slab = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)p->nrec);
        p->rec_cnt = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)p->nrec);
        p->rec_off = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)p->nrec);
        p->hbits = (uint32_t *)ws_alloc(p, sizeof(uint32_t) * (size_t)p->nrec * (size_t)(p->R / 32));
        p->split = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->ndt + 1) * (size_t)(p->T + 1));
        if (!p->rec_col || !p->rec_slab || !p->rec_cnt || !p->rec_off || !p->hbits || !p->split)
            return SPG_OUT_OF_MEMORY;
        launch(p, k_heavy_records, grid_for(p->nheavy, 256, sm * 8), 256, 0, hl, p->nheavy, p->win_lo, p->R,
               p->sym_max_recs, p->rec_first, p->rec_col, p->rec_slab, nsym);
        TRY(scan_exclusive_i64(p, nsym, sym_first, p->nheavy));
        TRY(cuda_check(cudaMemcpyAsync(p->h_pinned, sym_first + p->nheavy, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "items"));
        TRY(cuda_check(cudaStreamSynchronize(st), "items"));
        p->nsym = p->h_pinned[0];
        p->sym_rec0 = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)p->nsym);
        p->sym_nrec = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)p->nsym);
        if (!p->sym_rec0 || !p->sym_nrec) return SPG_OUT_OF_MEMORY;
        launch(p, k_sym_items, grid_for(p->nheavy, 256, sm * 8), 256, 0, p->nheavy, p->sym_max_recs, p->rec_first,
               sym_first, p->sym_rec0, p->sym_nrec);
        if (p->ndt > 0)
            launch(p, k_split, grid_for(p->ndt * (p->T + 1), 256, sm * 16), 256, 0, p->At_colptr, p->At_row, p->ndt, p->T,
                                                                                 p->R, p->split);
        LAUNCH_OK("heavy items");
    }
    cudaEventRecord(p->ev[1], st);

    // statistics
    TRY(cuda_check(cudaMemcpyAsync(p->h_pinned, p->d_cnt, sizeof(int64_t) * kCntSlots, cudaMemcpyDeviceToHost, st), "stats"));
    TRY(cuda_check(cudaStreamSynchronize(st), "stats"));
    spg_stats &S = p->stats;
    S.m = m; S.k = k; S.n = n; S.nnzA = p->nnzA; S.nnzB = p->nnzB; S.P = P; S.b = p->b;
    S.products = p->h_pinned[kCntProducts];
    S.nnzC = -1;
    S.sum_H = p->h_pinned[kCntSumH];
    S.sum_dtilde = p->ndt;
    S.fetch_blocks_total = (int64_t)P * p->nfb;
    S.fetch_blocks_chosen = p->h_pinned[kCntFetchChosen];
    S.gathered_nnz_exact = p->nAt;
    S.gathered_nnz_block = p->h_pinned[kCntVolBlock];
    S.empty_columns = p->bin_off[kBinEmpty + 1] - p->bin_off[kBinEmpty];
    S.heavy_columns = p->nheavy;
    S.light_columns = n - S.empty_columns - S.heavy_columns;
    S.heavy_items = p->nrec;
    S.nnzB_heavy = p->h_pinned[kCntNnzBHeavy];
    S.gathered_nnz_remote = p->h_pinned[kCntRemote];
    S.nnzC_heavy = -1;
    float ms = 0;
    cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]);
    S.ms_plan = ms;
    if (p->kev_used[kKGather] && cudaEventElapsedTime(&ms, p->kev[0], p->kev[1]) == cudaSuccess) S.ms_gather = ms;
    return read_dev_err(p, "plan");
}

}  // namespace spg

using namespace spg;

extern "C" void spgemm_default_options(spg_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->P = 1;
    opt->b = 1024;
    opt->sizing = SPG_SIZING_EXACT;
    opt->validate = 1;
    opt->learned_slack = 1.25;
}

extern "C" spg_status spgemm_plan(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_plan **out) {
    spg::PhaseRange nvtx_range("spgemm_plan");
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return SPG_INVALID_ARGUMENT;
    }
    *out = nullptr;
    if (!opt) {
        set_error("options are NULL");
        return SPG_INVALID_ARGUMENT;
    }
    TRY(check_csc(A, "A"));
    TRY(check_csc(B, "B"));
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A is %lld x %lld, B is %lld x %lld", (long long)A->nrows, (long long)A->ncols,
                  (long long)B->nrows, (long long)B->ncols);
        return SPG_INVALID_ARGUMENT;
    }
    bool fa = A->val_type == SPG_VAL_F64, fb = B->val_type == SPG_VAL_F64;
    if (fa != fb) {
        set_error("A and B must both hold doubles or both hold integers");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->idx_type != B->idx_type) {
        set_error("A and B must use the same row index type");
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->P < 1 || opt->b < 1) {
        set_error("P and b must be >= 1 (P=%d, b=%lld)", opt->P, (long long)opt->b);
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->sizing != SPG_SIZING_EXACT && opt->sizing != SPG_SIZING_LEARNED) {
        set_error("unknown sizing mode %d", opt->sizing);
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->semiring != SPG_SEMIRING_PLUS_TIMES) {
        set_error("semiring %d: this build computes (+, x) only", opt->semiring);
        return SPG_UNSUPPORTED;
    }
    if (A->nrows >= INT32_MAX || A->ncols >= INT32_MAX || B->ncols >= INT32_MAX) {
        set_error("m, k and n must be < 2^31 - 1");
        return SPG_UNSUPPORTED;
    }
    int lm = opt->light_max ? opt->light_max : 1024;
    if (opt->split != SPG_SPLIT_UNIFORM && opt->split != SPG_SPLIT_FLOPS) {
        set_error("split must be SPG_SPLIT_UNIFORM or SPG_SPLIT_FLOPS (got %d)", opt->split);
        return SPG_INVALID_ARGUMENT;
    }
    int R = opt->slab_rows ? opt->slab_rows : 4096;
    if (lm < 32 || lm > 1024 || (lm & (lm - 1)) || R < 1024 || R > 16384 || (R & (R - 1))) {
        set_error("light_max must be a power of two in [32, 1024] and slab_rows one in [1024, 16384]");
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->mask) {
        if (opt->mask_words < (A->nrows + 31) / 32 || (opt->mask_complement != 0 && opt->mask_complement != 1)) {
            set_error("mask_words must be >= ceil(nrows(A) / 32) = %lld and mask_complement 0 or 1",
                      (long long)((A->nrows + 31) / 32));
            return SPG_INVALID_ARGUMENT;
        }
        if (opt->sizing == SPG_SIZING_LEARNED) {
            set_error("an output mask is not available with learned sizing");
            return SPG_INVALID_ARGUMENT;
        }
    }

    spg_plan *p = new (std::nothrow) spg_plan();
    if (!p) {
        set_error("host allocation failed");
        return SPG_OUT_OF_MEMORY;
    }
    p->A = *A;
    p->B = *B;
    p->opt = *opt;
    if (opt->mask) {
        p->omask.bits = opt->mask;
        p->omask.words = opt->mask_words;
        p->omask.flip = opt->mask_complement ? ~0u : 0u;
    }
    p->st = (cudaStream_t)opt->stream;
    p->m = A->nrows;
    p->k = A->ncols;
    p->n = B->ncols;
    p->nnzA = A->nnz;
    p->nnzB = B->nnz;
    p->P = opt->P;
    p->b = opt->b;
    p->acc_f64 = fa;
    p->out_idx64 = A->idx_type == SPG_IDX_I64;
    p->light_max = lm;
    p->R = R;
    p->num_cap = R > kNumCapMin ? R : kNumCapMin;  // one base slab always fits a numeric item
    p->sym_max_recs = kSymMaxWords / (R / 32);
    p->num_max_recs = kNumMaxWords / (R / 32);
    int dev = 0;
    spg_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (!s) s = cuda_check(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev), "attr");
    // slots 0..63: counters and the error word; 64..64+P: the per-block D~ offsets
    if (!s) s = cuda_check(cudaMallocHost(&p->h_pinned, sizeof(int64_t) * (64 + (size_t)p->P + 1)), "cudaMallocHost");
    for (int i = 0; i < 8 && !s; i++) s = cuda_check(cudaEventCreate(&p->ev[i]), "event");
    for (int i = 0; i < 10 && !s; i++) s = cuda_check(cudaEventCreate(&p->kev[i]), "event");
    if (!s) s = plan_build(p);
    if (s) {
        std::string keep = last_error_str();
        spgemm_plan_destroy(p);
        set_error("%s", keep.c_str());
        return s;
    }
    *out = p;
    return SPG_OK;
}

extern "C" spg_status spgemm_plan_destroy(spg_plan *p) {
    if (!p) return SPG_OK;
    cudaStreamSynchronize(p->st);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    ws_free_all(p);
    cudaStreamSynchronize(p->st);
    for (int i = 0; i < 8; i++)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    for (int i = 0; i < 10; i++)
        if (p->kev[i]) cudaEventDestroy(p->kev[i]);
    if (p->h_pinned) cudaFreeHost(p->h_pinned);
    delete p;
    return SPG_OK;
}
