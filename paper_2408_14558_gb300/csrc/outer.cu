// Outer-product 1D SpGEMM (Algorithm 3) on one GPU: C = sum over the P row
// blocks K_i of B of A(:, K_i) * B(K_i, :).
//   redistribution  B is split by row blocks into B' (k x P*n): column i*n + j
//                   holds the entries of B(:, j) whose row lies in row block
//                   i = [floor(i*k/P), floor((i+1)*k/P))  (k_outer_count, a
//                   scan, k_outer_copy)
//                   B' keeps only its non-empty columns (most (i, j) pairs
//                   are empty), in (i, j) order, with the map back to j
//   local products  C' = A * B' by the column 1D path with P column blocks;
//                   the columns of block i have all their rows in K_i, so
//                   its owner needs only A(:, K_i): the columns it holds
//   merge           C = C' * S with S[c, j(c)] = 1 (k_outer_merge_fill): the
//                   partial columns of every column added up, by the same
//                   column 1D path
// Volumes of a distributed run (process i owning column block i of A, B and C,
// as in Algorithm 1) are counted on the way: B entries that change owner in
// the redistribution and partial nonzeros computed away from their column's
// owner.
#include <algorithm>

#include "spg_internal.cuh"

namespace spg {

const char *last_error_str();
void clear_error();

// Block of index r among the P blocks [floor(i*len/P), floor((i+1)*len/P)):
// the largest i with floor(i*len/P) <= r, that is floor(((r+1)*P - 1) / len).
__device__ __forceinline__ int64_t outer_block(int64_t r, int64_t len, int64_t P) {
    return ((r + 1) * P - 1) / len;
}

// counts[i*n + j] = entries of B(:, j) in row block i; moved = entries whose
// row block differs from the block of their column.  Warp per column.
__global__ void k_outer_count(const void *Bcp, int p64, const void *Brow, int i64, int64_t n, int64_t k, int P,
                              unsigned long long *counts, unsigned long long *moved) {
    const int lane = threadIdx.x & 31;
    unsigned long long mv = 0;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c0 = ld_ptr(Bcp, p64, j), c1 = ld_ptr(Bcp, p64, j + 1);
        const int64_t cb = outer_block(j, n, P);
        for (int64_t e = c0 + lane; e < c1; e += 32) {
            const int64_t blk = outer_block(ld_ptr(Brow, i64, e), k, P);
            atomicAdd(counts + blk * n + j, 1ull);
            mv += blk != cb;
        }
    }
    mv = warp_sum_ll((long long)mv);
    if (lane == 0 && mv) atomicAdd(moved, mv);
}

// B'(:, i*n + j) = the entries of B(:, j) in row block i, rows and values
// copied unchanged (row ids of rb bytes, values of vb bytes).  Warp per
// column; an entry's place inside its block is its distance to the block's
// first entry, found by binary search over the column's sorted rows.
__global__ void k_outer_copy(const void *Bcp, int p64, const void *Brow, int i64, const void *Bval, int vb,
                             int64_t n, int64_t k, int P, const int64_t *__restrict__ Scp, void *Srow, void *Sval) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c0 = ld_ptr(Bcp, p64, j), c1 = ld_ptr(Bcp, p64, j + 1);
        for (int64_t e = c0 + lane; e < c1; e += 32) {
            const int64_t r = ld_ptr(Brow, i64, e);
            const int64_t blk = outer_block(r, k, P);
            const int64_t lo = blk * k / P;
            int64_t a = c0, b = e;  // first entry of the column with row >= lo lies in [c0, e]
            while (a < b) {
                const int64_t mid = (a + b) >> 1;
                if (ld_ptr(Brow, i64, mid) < lo)
                    a = mid + 1;
                else
                    b = mid;
            }
            const int64_t pos = Scp[blk * n + j] + (e - a);
            if (i64)
                ((int64_t *)Srow)[pos] = r;
            else
                ((int32_t *)Srow)[pos] = (int32_t)r;
            if (vb == 8)
                ((uint64_t *)Sval)[pos] = ((const uint64_t *)Bval)[e];
            else
                ((uint32_t *)Sval)[pos] = ((const uint32_t *)Bval)[e];
        }
    }
}

// Flags of the non-empty (i, j) columns, for the scan that numbers them.
__global__ void k_outer_flags(const unsigned long long *counts, int64_t tot, int64_t *flags) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < tot; c += (int64_t)gridDim.x * blockDim.x)
        flags[c] = counts[c] > 0;
}

// The non-empty columns c = i*n + j of B', numbered cid[c]: their column
// pointers (cp2, nc + 1 entries) and their output column j and row block i.
__global__ void k_outer_compact(const unsigned long long *counts, const int64_t *cp, const int64_t *cid,
                                int64_t n, int64_t tot, int64_t *cp2, int32_t *jmap, int32_t *imap) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= tot; c += (int64_t)gridDim.x * blockDim.x) {
        if (c == tot) {
            cp2[cid[tot]] = cp[tot];
        } else if (counts[c]) {
            const int64_t d = cid[c];
            cp2[d] = cp[c];
            jmap[d] = (int32_t)(c % n);
            imap[d] = (int32_t)(c / n);
        }
    }
}

// Entries per column of the merge matrix: the non-empty blocks of column j.
__global__ void k_outer_merge_count(const unsigned long long *counts, int64_t n, int P, int64_t *cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int i = 0; i < P; i++) c += counts[(int64_t)i * n + j] > 0;
        cnt[j] = c;
    }
}

// The merge matrix S (nc x n): column j holds the numbers d of the non-empty
// partial columns of j (ascending, as their blocks ascend), each with value
// one (double or int64).
__global__ void k_outer_merge_fill(const unsigned long long *counts, const int32_t *jmap, const int32_t *imap,
                                   int64_t nc, int64_t n, const int64_t *Scp, void *rows, int i64, void *vals,
                                   int f64) {
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < nc; d += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = jmap[d];
        const int i = imap[d];
        int64_t rank = 0;
        for (int q = 0; q < i; q++) rank += counts[(int64_t)q * n + j] > 0;
        const int64_t t = Scp[j] + rank;
        if (i64)
            ((int64_t *)rows)[t] = d;
        else
            ((int32_t *)rows)[t] = (int32_t)d;
        if (f64)
            ((double *)vals)[t] = 1.0;
        else
            ((int64_t *)vals)[t] = 1;
    }
}

// Partial nonzeros of column j computed by block i != owner(j).
__global__ void k_outer_partial_moved(const int64_t *__restrict__ Cpcp, const int32_t *jmap, const int32_t *imap,
                                      int64_t nc, int64_t n, int P, unsigned long long *moved) {
    unsigned long long mv = 0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < nc; d += (int64_t)gridDim.x * blockDim.x)
        if (imap[d] != outer_block(jmap[d], n, P)) mv += (unsigned long long)(Cpcp[d + 1] - Cpcp[d]);
    mv = warp_sum_ll((long long)mv);
    if ((threadIdx.x & 31) == 0 && mv) atomicAdd(moved, mv);
}

}  // namespace spg

using namespace spg;

static void outer_free(const spg_options *o, void *p, size_t bytes) {
    if (!p) return;
    if (o->free)
        o->free(p, bytes, o->alloc_ctx, o->stream);
    else if (!o->alloc)
        cudaFreeAsync(p, (cudaStream_t)o->stream);
}

static size_t csc_idx_bytes(const spg_csc &M) { return M.idx_type == SPG_IDX_I64 ? 8 : 4; }
static size_t csc_val_bytes(const spg_csc &M) { return M.val_type == SPG_VAL_I32 ? 4 : 8; }

static void free_csc(const spg_options *o, spg_csc &M) {
    outer_free(o, M.colptr, sizeof(int64_t) * (size_t)(M.ncols + 1));
    outer_free(o, M.rowidx, csc_idx_bytes(M) * (size_t)std::max<int64_t>(M.nnz, 1));
    outer_free(o, M.vals, csc_val_bytes(M) * (size_t)std::max<int64_t>(M.nnz, 1));
    M.colptr = M.rowidx = M.vals = nullptr;
}

extern "C" spg_status spgemm_outer_multiply(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C,
                                            spg_outer_stats *stats) {
    spg::PhaseRange nvtx_range("spgemm_outer_multiply");
    clear_error();
    if (!A || !B || !opt || !C) {
        set_error("A, B, options and C must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->ncols != B->nrows || A->nrows < 0 || B->ncols < 0 || opt->P < 1 || !B->colptr) {
        set_error("outer product needs A.ncols == B.nrows and P >= 1 (A %lld x %lld, B %lld x %lld, P %d)",
                  (long long)A->nrows, (long long)A->ncols, (long long)B->nrows, (long long)B->ncols, opt->P);
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->mask) {
        set_error("an output mask is not available with the outer-product form");
        return SPG_INVALID_ARGUMENT;
    }
    const int P = opt->P;
    const int64_t k = B->nrows, n = B->ncols, Pn = (int64_t)P * n;
    const bool a_idx64 = A->idx_type == SPG_IDX_I64;
    cudaStream_t st = (cudaStream_t)opt->stream;
    spg_outer_stats S{};
    S.P = P;

    // a bare plan: workspace, stream and launch counting for the scan
    spg_plan w;
    w.opt = *opt;
    w.st = st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w.sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], st);

    spg_status s = SPG_OK;
    spg_csc Bs{}, Cp{}, M{};
    const size_t bib = csc_idx_bytes(*B), bvb = csc_val_bytes(*B);
    const int p64 = B->ptr_type == SPG_IDX_I64, i64 = B->idx_type == SPG_IDX_I64;
    const int sm = w.sm_count;
    // --- redistribution of B by row blocks
    unsigned long long *counts = (unsigned long long *)ws_alloc(&w, sizeof(unsigned long long) * (size_t)(Pn + 1));
    unsigned long long *moved = (unsigned long long *)ws_alloc(&w, sizeof(unsigned long long) * 2);
    int64_t *cp = (int64_t *)ws_alloc(&w, sizeof(int64_t) * (size_t)(Pn + 1));
    int64_t *flags = (int64_t *)ws_alloc(&w, sizeof(int64_t) * (size_t)(Pn + 1));
    int64_t *cid = (int64_t *)ws_alloc(&w, sizeof(int64_t) * (size_t)(Pn + 1));
    int64_t *hnc = nullptr;
    if (!counts || !moved || !cp || !flags || !cid) s = SPG_OUT_OF_MEMORY;
    if (!s) s = cuda_check(cudaMallocHost(&hnc, sizeof(int64_t)), "cudaMallocHost");
    if (!s) s = cuda_check(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)(Pn + 1), st), "memset");
    if (!s) s = cuda_check(cudaMemsetAsync(moved, 0, sizeof(unsigned long long) * 2, st), "memset");
    if (!s && n > 0) {
        launch(&w, k_outer_count, grid_for(n * 32, 256, sm * 16), 256, 0, B->colptr, p64, B->rowidx, i64, n, k, P,
               counts, moved);
        s = cuda_check(cudaGetLastError(), "outer count");
    }
    if (!s) s = scan_exclusive_i64(&w, (const int64_t *)counts, cp, Pn);
    if (!s && Pn > 0) {
        launch(&w, k_outer_flags, grid_for(Pn, 256, sm * 8), 256, 0, counts, Pn, flags);
        s = cuda_check(cudaGetLastError(), "outer flags");
    }
    if (!s) s = scan_exclusive_i64(&w, flags, cid, Pn);
    if (!s) s = cuda_check(cudaMemcpyAsync(hnc, cid + Pn, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "nc");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "nc");
    const int64_t nc = s ? 0 : *hnc;
    if (!s && !a_idx64 && nc >= INT32_MAX) {
        set_error("%lld non-empty partial columns need int64 row ids in A", (long long)nc);
        s = SPG_UNSUPPORTED;
    }
    int32_t *jmap = nullptr, *imap = nullptr;
    if (!s) {
        jmap = (int32_t *)ws_alloc(&w, sizeof(int32_t) * (size_t)(nc + 1));
        imap = (int32_t *)ws_alloc(&w, sizeof(int32_t) * (size_t)(nc + 1));
        Bs.nrows = k;
        Bs.ncols = nc;
        Bs.nnz = B->nnz;
        Bs.ptr_type = SPG_IDX_I64;
        Bs.idx_type = B->idx_type;
        Bs.val_type = B->val_type;
        Bs.colptr = alloc_user(opt, sizeof(int64_t) * (size_t)(nc + 1));
        Bs.rowidx = alloc_user(opt, bib * (size_t)std::max<int64_t>(B->nnz, 1));
        Bs.vals = alloc_user(opt, bvb * (size_t)std::max<int64_t>(B->nnz, 1));
        if (!jmap || !imap || !Bs.colptr || !Bs.rowidx || !Bs.vals) s = SPG_OUT_OF_MEMORY;
    }
    if (!s) {
        launch(&w, k_outer_compact, grid_for(Pn + 1, 256, sm * 8), 256, 0, counts, cp, cid, n, Pn,
               (int64_t *)Bs.colptr, jmap, imap);
        s = cuda_check(cudaGetLastError(), "outer compact");
    }
    if (!s && n > 0 && B->nnz > 0) {
        launch(&w, k_outer_copy, grid_for(n * 32, 256, sm * 16), 256, 0, B->colptr, p64, B->rowidx, i64, B->vals,
               (int)bvb, n, k, P, (const int64_t *)cp, Bs.rowidx, Bs.vals);
        s = cuda_check(cudaGetLastError(), "outer copy");
    }
    cudaEventRecord(ev[1], st);
    // --- local products C' = A * B' (the columns of row block i are process i's)
    if (!s) {
        spg_options o = *opt;
        s = spgemm_1d_multiply(A, &Bs, &o, &Cp);
        if (s == SPG_OVERFLOW_RECOMPUTED) s = SPG_OK;
        if (!s) {
            spg_stats ls{};
            spgemm_last_multiply_stats(&ls);
            S.products = ls.products;
            S.partial_nnz = Cp.nnz;
        }
    }
    free_csc(opt, Bs);
    if (!s && nc > 0) {
        launch(&w, k_outer_partial_moved, grid_for(nc, 256, sm * 8), 256, 0, (const int64_t *)Cp.colptr, jmap, imap,
               nc, n, P, moved + 1);
        s = cuda_check(cudaGetLastError(), "outer moved");
    }
    cudaEventRecord(ev[2], st);
    // --- merge C = C' * S
    int64_t *scnt = nullptr;
    if (!s) {
        M.nrows = nc;
        M.ncols = n;
        M.nnz = nc;
        M.ptr_type = SPG_IDX_I64;
        M.idx_type = a_idx64 ? SPG_IDX_I64 : SPG_IDX_I32;
        M.val_type = Cp.val_type;
        M.colptr = alloc_user(opt, sizeof(int64_t) * (size_t)(n + 1));
        M.rowidx = alloc_user(opt, csc_idx_bytes(M) * (size_t)std::max<int64_t>(nc, 1));
        M.vals = alloc_user(opt, 8 * (size_t)std::max<int64_t>(nc, 1));
        scnt = (int64_t *)ws_alloc(&w, sizeof(int64_t) * (size_t)(n + 1));
        if (!M.colptr || !M.rowidx || !M.vals || !scnt) s = SPG_OUT_OF_MEMORY;
    }
    if (!s && n > 0) {
        launch(&w, k_outer_merge_count, grid_for(n, 256, sm * 8), 256, 0, counts, n, P, scnt);
        s = cuda_check(cudaGetLastError(), "merge count");
    }
    if (!s) s = scan_exclusive_i64(&w, scnt, (int64_t *)M.colptr, n);
    if (!s && nc > 0) {
        launch(&w, k_outer_merge_fill, grid_for(nc, 256, sm * 8), 256, 0, counts, jmap, imap, nc, n,
               (const int64_t *)M.colptr, M.rowidx, (int)a_idx64, M.vals, (int)(M.val_type == SPG_VAL_F64));
        s = cuda_check(cudaGetLastError(), "merge fill");
    }
    if (!s) {
        spg_options o = *opt;
        s = spgemm_1d_multiply(&Cp, &M, &o, C);
        if (s == SPG_OVERFLOW_RECOMPUTED) s = SPG_OK;
        if (!s) S.nnzC = C->nnz;
    }
    cudaEventRecord(ev[3], st);
    unsigned long long hv[2] = {0, 0};
    if (!s) s = cuda_check(cudaMemcpyAsync(hv, moved, sizeof(hv), cudaMemcpyDeviceToHost, st), "outer stats");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "outer stats");
    if (!s) {
        S.nnzB_moved = (int64_t)hv[0];
        S.partial_moved = (int64_t)hv[1];
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        S.ms_split = ms;
        cudaEventElapsedTime(&ms, ev[1], ev[2]);
        S.ms_local = ms;
        cudaEventElapsedTime(&ms, ev[2], ev[3]);
        S.ms_merge = ms;
        if (stats) *stats = S;
    }
    std::string keep = s ? std::string(last_error_str()) : std::string();
    cudaStreamSynchronize(st);
    free_csc(opt, Cp);
    free_csc(opt, M);
    ws_free_all(&w);
    if (hnc) cudaFreeHost(hnc);
    for (auto &e : ev) cudaEventDestroy(e);
    if (s) set_error("%s", keep.c_str());
    return s;
}
