// spgemm_count_noalloc: nnz(C(:,j)) of C = A * B without allocating memory.
//
// It is a variant of the symbolic count whose scratch (one row bitmap per
// CTA) is not allocated per call but lives in a file-scope device array of
// fixed size, so the call never asks the CUDA runtime, PyTorch or any other
// allocator for memory.  That serves callers that may not allocate device
// memory at all: a process whose device memory is entirely owned by another
// allocator (a framework's caching pool sized to the whole GPU), a service
// that reserves its memory once at start-up and must not grow afterwards, or
// code on a latency path where an allocation call (which can synchronise the
// device) is not acceptable.  The caller passes the inputs and the output.
//
// Costs and limits:
//   * every GPU that loads the library holds kNaScratchBytes (8 MiB) of
//     device memory for the array until the process exits;
//   * A may have at most kNaMaxRows (1,048,576) rows;
//   * all calls share the array: two calls whose kernels overlap on the GPU
//     (different streams, or different host threads on one device) race and
//     give wrong counts; order them on one stream;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture on the device.  The address is cached for the
//     life of the process: a cudaDeviceReset of that device between calls is
//     not supported (the module, and so the array, may move).
#include <mutex>

#include "spg_internal.cuh"

namespace spg {
namespace {

constexpr int kNaCtas = 64;
constexpr int64_t kNaMaxRows = int64_t(1) << 20;
constexpr int64_t kNaWordsPerCta = kNaMaxRows / 32;
constexpr size_t kNaScratchBytes = sizeof(uint32_t) * kNaCtas * kNaWordsPerCta;  // 8 MiB
constexpr int kNaMaxDevices = 64;
static_assert(kNaScratchBytes == (size_t(8) << 20), "the documented scratch size is 8 MiB");

// One bitmap of up to kNaMaxRows bits per CTA.  Host code must not use this
// name as an address: it is a host-side stand-in; the kernel receives the
// device address looked up by na_scratch().
static __device__ __align__(256) uint32_t g_na_scratch[kNaCtas * kNaWordsPerCta];

std::mutex g_na_mutex;
uint32_t *g_na_ptr[kNaMaxDevices] = {nullptr};

// Device address of g_na_scratch on the current device (looked up once).
spg_status na_scratch(uint32_t **out) {
    int dev = 0;
    spg_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s) return s;
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("spgemm_count_noalloc supports device ordinals below %d", kNaMaxDevices);
        return SPG_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        s = cuda_check(cudaGetSymbolAddress(&ptr, g_na_scratch), "cudaGetSymbolAddress");
        if (s) return s;
        g_na_ptr[dev] = (uint32_t *)ptr;
    }
    *out = g_na_ptr[dev];
    return SPG_OK;
}

// CTA per output column (grid-stride).  Each CTA owns one bitmap of `words`
// words; it clears it once, then for every column marks the rows of all its
// products, counts the bits that were newly set, and clears the words it
// touched again so that the bitmap is zero before the next column.
__global__ void __launch_bounds__(256)
    k_count_noalloc(const void *Acp, int ap64, const void *Arow, int ai64, const void *Bcp, int bp64,
                    const void *Brow, int bi64, int64_t n, int64_t *nnz_out, uint32_t *scratch, int64_t words) {
    __shared__ int red[32];
    uint32_t *bits = scratch + (int64_t)blockIdx.x * kNaWordsPerCta;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0;
    __syncthreads();
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const int64_t p0 = ld_ptr(Bcp, bp64, j), p1 = ld_ptr(Bcp, bp64, j + 1);
        int cnt = 0;
        for (int64_t p = p0 + wid; p < p1; p += nw) {
            const int64_t k = ld_ptr(Brow, bi64, p);
            const int64_t s = ld_ptr(Acp, ap64, k), e = ld_ptr(Acp, ap64, k + 1);
            for (int64_t q = s + lane; q < e; q += 32) {
                const int64_t r = ld_ptr(Arow, ai64, q);
                if ((uint64_t)r >= (uint64_t)words * 32) continue;  // row outside A: never touch memory
                const uint32_t bit = 1u << (r & 31);
                const uint32_t old = atomicOr(bits + (r >> 5), bit);
                cnt += (old & bit) ? 0 : 1;
            }
        }
        cnt = warp_sum_i(cnt);
        if (lane == 0) red[wid] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; w++) tot += red[w];
            nnz_out[j] = tot;
        }
        for (int64_t p = p0 + wid; p < p1; p += nw) {
            const int64_t k = ld_ptr(Brow, bi64, p);
            const int64_t s = ld_ptr(Acp, ap64, k), e = ld_ptr(Acp, ap64, k + 1);
            for (int64_t q = s + lane; q < e; q += 32) {
                const int64_t r = ld_ptr(Arow, ai64, q);
                if ((uint64_t)r < (uint64_t)words * 32) bits[r >> 5] = 0;
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" spg_status spgemm_count_noalloc(const spg_csc *A, const spg_csc *B, int64_t *nnz_out, void *stream) {
    if (!A || !B || !A->colptr || !B->colptr) {
        set_error("A, B and their column pointers must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if ((A->nnz > 0 && !A->rowidx) || (B->nnz > 0 && !B->rowidx) || A->ptr_type < 0 || A->ptr_type > 1 ||
        A->idx_type < 0 || A->idx_type > 1 || B->ptr_type < 0 || B->ptr_type > 1 || B->idx_type < 0 ||
        B->idx_type > 1 || A->nrows < 0 || B->ncols < 0) {
        set_error("bad array pointer, size or index type");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A has %lld columns, B has %lld rows", (long long)A->ncols,
                  (long long)B->nrows);
        return SPG_INVALID_ARGUMENT;
    }
    if (A->nrows > kNaMaxRows) {
        set_error("spgemm_count_noalloc supports at most %lld rows of A (A has %lld); use spgemm_symbolic",
                  (long long)kNaMaxRows, (long long)A->nrows);
        return SPG_UNSUPPORTED;
    }
    if (B->ncols == 0) return SPG_OK;
    if (!nnz_out) {
        set_error("nnz_out must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    uint32_t *scratch = nullptr;
    spg_status s = na_scratch(&scratch);
    if (s) return s;
    const int64_t words = (A->nrows + 31) / 32;
    const int grid = (int)(B->ncols < kNaCtas ? B->ncols : kNaCtas);
    k_count_noalloc<<<grid, 256, 0, (cudaStream_t)stream>>>(
        A->colptr, A->ptr_type == SPG_IDX_I64, A->rowidx, A->idx_type == SPG_IDX_I64, B->colptr,
        B->ptr_type == SPG_IDX_I64, B->rowidx, B->idx_type == SPG_IDX_I64, B->ncols, nnz_out, scratch, words);
    return cuda_check(cudaGetLastError(), "spgemm_count_noalloc launch");
}
