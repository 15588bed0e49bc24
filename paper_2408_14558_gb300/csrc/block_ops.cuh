// CTA- and warp-level helpers shared by the numeric and learned kernels.
#pragma once

#include "spg_internal.cuh"

namespace spg {

// Exclusive scan of popc(bits[w]) over the RW words of a slab by the whole CTA.
// Writes pre[0..RW) and returns the total to every thread.
__device__ __forceinline__ int cta_scan_popc(const uint32_t *bits, int *pre, int RW, int *wsum) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (RW + nt - 1) / nt;
    const int w0 = tid * per;
    int local = 0;
    for (int w = w0; w < min(RW, w0 + per); w++) local += __popc(bits[w]);
    const int lane = tid & 31, wid = tid >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int nw = nt >> 5;
        int v = lane < nw ? wsum[lane] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < nw) wsum[lane] = vi - v;
        if (lane == 31) wsum[32] = vi;
    }
    __syncthreads();
    int run = wsum[wid] + incl - local;
    for (int w = w0; w < min(RW, w0 + per); w++) {
        pre[w] = run;
        run += __popc(bits[w]);
    }
    int total = wsum[32];
    __syncthreads();
    return total;
}

// The same scan over packed (word, prefix) pairs: fills bp[w].y.
__device__ __forceinline__ int cta_scan_popc_packed(uint2 *bp, int n, int *wsum) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (n + nt - 1) / nt;
    const int w0 = tid * per;
    int local = 0;
    for (int w = w0; w < min(n, w0 + per); w++) local += __popc(bp[w].x);
    const int lane = tid & 31, wid = tid >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int nw = nt >> 5;
        int v = lane < nw ? wsum[lane] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < nw) wsum[lane] = vi - v;
        if (lane == 31) wsum[32] = vi;
    }
    __syncthreads();
    int run = wsum[wid] + incl - local;
    for (int w = w0; w < min(n, w0 + per); w++) {
        bp[w].y = (uint32_t)run;
        run += __popc(bp[w].x);
    }
    int total = wsum[32];
    __syncthreads();
    return total;
}

// Sort keys[0..npad) ascending (npad a power of two), carrying vals along.
template <typename Acc>
__device__ __forceinline__ void warp_bitonic(int *keys, Acc *vals, int npad, int lane) {
    for (int kk = 2; kk <= npad; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < (npad >> 1); t += 32) {
                int i = 2 * jj * (t / jj) + (t % jj);
                int l = i + jj;
                bool up = (i & kk) == 0;
                int ki = keys[i], kl = keys[l];
                if ((ki > kl) == up) {
                    keys[i] = kl;
                    keys[l] = ki;
                    Acc tv = vals[i];
                    vals[i] = vals[l];
                    vals[l] = tv;
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace spg
