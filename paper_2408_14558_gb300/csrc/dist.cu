// Kernels of the distributed 1D SpGEMM (Section 3.1, Algorithm 1 run by P
// processes; Algorithm 2 for what each process fetches).  Process i owns
// column block i of A, B and C.  Before its local multiply it needs the
// columns H_i of A (the nonzero rows of its B_i) that are nonempty, fetched in
// blocks of b consecutive column ids from their owners.  These entry points
// are the device steps of that exchange; the transport between processes
// (NCCL or another collective library) sits above them, in the caller:
//   spgemm_dist_fetch_blocks   H_i and the chosen fetch blocks of one process
//   spgemm_dist_pack           an owner's side: copy the requested column
//                              ranges of its A_j into one contiguous buffer
//   spgemm_dist_fetched_colptr the requester's side: column pointers of the
//                              matrix that holds exactly the fetched columns
#include "spg_internal.cuh"

namespace spg {
void clear_error();

namespace {

__device__ __forceinline__ int64_t ld_idx(const void *p, int is64, int64_t i) {
    return is64 ? (int64_t)__ldg((const long long *)p + i) : (int64_t)__ldg((const int *)p + i);
}

// One thread per stored entry of B_i: set bit k of H for its row k.  Rows
// outside [0, k) touch nothing (and are reported).
__global__ void k_dist_mark_H(const void *Brow, int bi64, int64_t nnzB, int64_t k, uint32_t *H, int *bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnzB; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = ld_idx(Brow, bi64, e);
        if ((uint64_t)r >= (uint64_t)k) {
            *bad = 1;
            continue;
        }
        atomicOr(H + (r >> 5), 1u << (r & 31));
    }
}

// One thread per column id: a fetch block is chosen iff one of its columns is
// in H_i and nonempty in A (D~_i = H_i AND D, Algorithm 1; Algorithm 2 with
// groups of b consecutive ids).  fetch[] is zero on entry.
__global__ void k_dist_choose(const uint32_t *H, const int64_t *Acp, int64_t k, int64_t b, uint8_t *fetch) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
        if (((__ldg(H + (c >> 5)) >> (c & 31)) & 1u) && __ldg(Acp + c + 1) > __ldg(Acp + c)) fetch[c / b] = 1;
    }
}

// One thread per packed entry: the entry's range by binary search over the
// ranges' output offsets, then one copy of its row id and value.  Reads stay
// inside the range's column span of A and inside A's arrays.
__global__ void k_dist_pack(const void *Acp, int ap64, const void *Arow, const void *Aval, int idx_bytes,
                            int val_bytes, int64_t ncols, int64_t nnzA, const int64_t *ranges,
                            const int64_t *out_off, int64_t nr, void *rows_out, void *vals_out, int *bad) {
    const int64_t total = out_off[nr];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nr;  // out_off[lo] <= e < out_off[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (out_off[mid] <= e)
                lo = mid;
            else
                hi = mid;
        }
        const int64_t c0 = ranges[2 * lo], c1 = ranges[2 * lo + 1];
        if (c0 < 0 || c1 > ncols || c0 > c1) {
            *bad = 1;
            continue;
        }
        const int64_t s0 = ld_ptr(Acp, ap64, c0), s1 = ld_ptr(Acp, ap64, c1);
        const int64_t src = s0 + (e - out_off[lo]);
        if (src >= s1 || src < 0 || src >= nnzA) {
            *bad = 1;
            continue;
        }
        if (idx_bytes == 8)
            ((long long *)rows_out)[e] = __ldg((const long long *)Arow + src);
        else
            ((int *)rows_out)[e] = __ldg((const int *)Arow + src);
        if (val_bytes == 8)
            ((long long *)vals_out)[e] = __ldg((const long long *)Aval + src);
        else
            ((int *)vals_out)[e] = __ldg((const int *)Aval + src);
    }
}

// Fetched column pointers, phase 1 (one CTA): the entries of every fetch
// block that was chosen, scanned over the blocks; the exclusive prefix of
// block t goes to out[t * b] (the block's first column) and the total to
// out[k].
__global__ void __launch_bounds__(1024)
    k_dist_block_prefix(const int64_t *Acp, const uint8_t *fetch, int64_t k, int64_t b, int64_t nblk, int64_t *out) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < nblk; t0 += blockDim.x) {
        const int64_t t = t0 + tid;
        long long v = 0;
        if (t < nblk && fetch[t]) {
            const int64_t hi = (t + 1) * b < k ? (t + 1) * b : k;
            v = Acp[hi] - Acp[t * b];
        }
        long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += y;
            }
            wsum[lane] = wi - w;  // exclusive prefix of the warp sums
        }
        __syncthreads();
        const long long ex = carry + wsum[wid] + inc - v;
        if (t < nblk) out[t * b] = ex;
        __syncthreads();
        if (tid == (int)blockDim.x - 1) carry = ex + v;
        __syncthreads();
    }
    if (tid == 0) out[k] = carry;
}

// Phase 2: every other column c of block t: prefix of t plus the entries of
// the block's columns before c when the block was chosen.
__global__ void k_dist_colptr(const int64_t *Acp, const uint8_t *fetch, int64_t k, int64_t b, int64_t *out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = c / b, c0 = t * b;
        if (c == c0) continue;
        out[c] = out[c0] + (fetch[t] ? Acp[c] - Acp[c0] : 0);
    }
}

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

bool bad_csc_header(const spg_csc *M) {
    return !M || !M->colptr || (M->nnz > 0 && (!M->rowidx || !M->vals)) || M->ptr_type < 0 || M->ptr_type > 1 ||
           M->idx_type < 0 || M->idx_type > 1 || M->val_type < 0 || M->val_type > 2 || M->nrows < 0 ||
           M->ncols < 0 || M->nnz < 0;
}

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" spg_status spgemm_dist_fetch_blocks(const spg_csc *B, const int64_t *A_colptr, int64_t b, uint32_t *H,
                                               uint8_t *fetch, int *bad, void *stream) {
    clear_error();
    if (bad_csc_header(B) || !A_colptr || b < 1 || (B->nrows > 0 && (!H || !fetch)) || !bad) {
        set_error("spgemm_dist_fetch_blocks: NULL pointer, bad header or b < 1");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t k = B->nrows;
    if (k == 0) return SPG_OK;
    const int64_t nblk = (k + b - 1) / b;
    spg_status s = cuda_check(cudaMemsetAsync(H, 0, sizeof(uint32_t) * (size_t)((k + 31) / 32), st), "memset H");
    if (!s) s = cuda_check(cudaMemsetAsync(fetch, 0, (size_t)nblk, st), "memset fetch");
    if (!s) s = cuda_check(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset flag");
    if (s) return s;
    if (B->nnz > 0)
        k_dist_mark_H<<<grid_of(B->nnz, 256), 256, 0, st>>>(B->rowidx, B->idx_type == SPG_IDX_I64, B->nnz, k, H, bad);
    k_dist_choose<<<grid_of(k, 256), 256, 0, st>>>(H, A_colptr, k, b, fetch);
    return cuda_check(cudaGetLastError(), "spgemm_dist_fetch_blocks launch");
}

extern "C" spg_status spgemm_dist_pack(const spg_csc *A, const int64_t *ranges, const int64_t *out_off, int64_t nr,
                                       int64_t total, void *rows_out, void *vals_out, int *bad, void *stream) {
    clear_error();
    if (bad_csc_header(A) || nr < 0 || total < 0 || (nr > 0 && (!ranges || !out_off)) ||
        (total > 0 && (!rows_out || !vals_out)) || !bad) {
        set_error("spgemm_dist_pack: NULL pointer, bad header or negative size");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    spg_status s = cuda_check(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset flag");
    if (s || nr == 0 || total == 0) return s;
    const int idx_bytes = A->idx_type == SPG_IDX_I64 ? 8 : 4;
    const int val_bytes = A->val_type == SPG_VAL_I32 ? 4 : 8;
    k_dist_pack<<<grid_of(total, 256), 256, 0, st>>>(A->colptr, A->ptr_type == SPG_IDX_I64, A->rowidx, A->vals,
                                                    idx_bytes, val_bytes, A->ncols, A->nnz, ranges, out_off, nr,
                                                    rows_out, vals_out, bad);
    return cuda_check(cudaGetLastError(), "spgemm_dist_pack launch");
}

extern "C" spg_status spgemm_dist_fetched_colptr(const int64_t *A_colptr, const uint8_t *fetch, int64_t k, int64_t b,
                                                 int64_t *colptr_out, void *stream) {
    clear_error();
    if (!A_colptr || !colptr_out || (k > 0 && !fetch) || k < 0 || b < 1) {
        set_error("spgemm_dist_fetched_colptr: NULL pointer, k < 0 or b < 1");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (k == 0) return cuda_check(cudaMemsetAsync(colptr_out, 0, sizeof(int64_t), st), "memset colptr");
    const int64_t nblk = (k + b - 1) / b;
    k_dist_block_prefix<<<1, 1024, 0, st>>>(A_colptr, fetch, k, b, nblk, colptr_out);
    k_dist_colptr<<<grid_of(k, 256), 256, 0, st>>>(A_colptr, fetch, k, b, colptr_out);
    return cuda_check(cudaGetLastError(), "spgemm_dist_fetched_colptr launch");
}
