// Exclusive prefix sums (reduce-then-scan, three launches, no spin waits).
// Used for the rank of required columns, the gathered column pointers, the
// heavy-slab item lists and the column pointers of C.
#include "spg_internal.cuh"

namespace spg {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename T>
__global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, long long *__restrict__ part) {
    __shared__ long long red[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += (long long)in[idx];
    }
    s = warp_sum_ll(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long v = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
        v = warp_sum_ll(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// One block scans the per-tile partial sums in place (exclusive) and writes
// the grand total to *total.
__global__ void k_scan_partials(long long *part, int64_t ntiles, long long *total) {
    __shared__ long long carry_sh;
    __shared__ long long wsum[32];
    if (threadIdx.x == 0) carry_sh = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        long long v = idx < ntiles ? part[idx] : 0;
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int nw = blockDim.x >> 5;
            long long w = lane < nw ? wsum[lane] : 0;
            long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < nw) wsum[lane] = wi - w;
        }
        __syncthreads();
        long long carry = carry_sh;
        if (idx < ntiles) part[idx] = carry + wsum[wid] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_sh = carry + wsum[wid] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_sh;
}

template <typename T>
__global__ void k_scan_tiles(const T *__restrict__ in, int64_t n, const long long *__restrict__ part,
                             const long long *__restrict__ total, int64_t *__restrict__ out) {
    __shared__ long long wsum[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    // each thread owns kScanPer consecutive elements
    long long v[kScanPer];
    long long run = 0;
    int64_t my = base + (int64_t)threadIdx.x * kScanPer;
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        v[i] = (my + i < n) ? (long long)in[my + i] : 0;
        run += v[i];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < kScanThreads / 32 ? wsum[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanThreads / 32) wsum[lane] = wi - w;
    }
    __syncthreads();
    long long acc = part[blockIdx.x] + wsum[wid] + incl - run;
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        if (my + i < n) out[my + i] = acc;
        acc += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

template <typename T>
static spg_status scan_impl(spg_plan *p, const T *in, int64_t *out, int64_t n) {
    if (n == 0) {
        return cuda_check(cudaMemsetAsync(out, 0, sizeof(int64_t), p->st), "scan memset");
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    long long *part = (long long *)ws_alloc(p, sizeof(long long) * (size_t)(ntiles + 1));
    if (!part) return SPG_OUT_OF_MEMORY;
    launch(p, k_scan_reduce<T>, (unsigned)ntiles, kScanThreads, 0, in, n, part);
    launch(p, k_scan_partials, 1, 1024, 0, part, ntiles, part + ntiles);
    launch(p, k_scan_tiles<T>, (unsigned)ntiles, kScanThreads, 0, in, n, part, part + ntiles, out);
    return cuda_check(cudaGetLastError(), "scan launch");
}

spg_status scan_exclusive_i32(spg_plan *p, const int32_t *in, int64_t *out, int64_t n) {
    return scan_impl<int32_t>(p, in, out, n);
}
spg_status scan_exclusive_i64(spg_plan *p, const int64_t *in, int64_t *out, int64_t n) {
    return scan_impl<int64_t>(p, in, out, n);
}

}  // namespace spg
