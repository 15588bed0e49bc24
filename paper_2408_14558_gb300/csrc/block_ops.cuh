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

// The same scan with one barrier: pre[] is complete for every thread only
// after the caller's next barrier, and wsum must not be written again before
// that barrier.
__device__ __forceinline__ int cta_scan_popc1(const uint32_t *bits, int *pre, int n, int *wsum) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (n + nt - 1) / nt;
    const int w0 = tid * per;
    int local = 0;
    for (int w = w0; w < min(n, w0 + per); w++) local += __popc(bits[w]);
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    const int wt = lane < nw ? wsum[lane] : 0;
    const int before = __reduce_add_sync(kFull, lane < wid ? wt : 0);
    const int total = __reduce_add_sync(kFull, wt);
    int run = before + incl - local;
    for (int w = w0; w < min(n, w0 + per); w++) {
        pre[w] = run;
        run += __popc(bits[w]);
    }
    return total;
}

// The same scan over packed (word, prefix) pairs: fills bp[w].y and returns
// the total to every thread.  One barrier: every warp then reads all warp
// totals and takes its own offset, so the y fields are complete for every
// thread only after the caller's next barrier, and wsum must not be written
// again before that barrier.
__device__ __forceinline__ int cta_scan_popc_packed(uint2 *bp, int n, int *wsum) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (n + nt - 1) / nt;
    const int w0 = tid * per;
    int local = 0;
    for (int w = w0; w < min(n, w0 + per); w++) local += __popc(bp[w].x);
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    // lane l < nw holds warp l's total; the warps before this one give its offset
    const int wt = lane < nw ? wsum[lane] : 0;
    const int before = __reduce_add_sync(kFull, lane < wid ? wt : 0);
    const int total = __reduce_add_sync(kFull, wt);
    int run = before + incl - local;
    for (int w = w0; w < min(n, w0 + per); w++) {
        bp[w].y = (uint32_t)run;
        run += __popc(bp[w].x);
    }
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

// Sort the pairs (keys[0..n), vals[0..n)) ascending by key with one warp; the
// keys are distinct and non-negative, and keys/vals are the front of a table of
// S slots.  n <= 32: one bitonic network across the lanes' registers.
// n <= S/2: LSD radix sort with 8-bit digits over the bits the largest key
// uses, ping-ponging between the front and the upper half of the table; each
// pass is stable because the entries are scattered 32 at a time in order and
// lanes holding equal digits are ranked by __match_any_sync.  Otherwise the
// in-place bitonic network above.  hist: 256 ints of this warp.
template <typename Acc>
__device__ __forceinline__ void warp_sort_pairs(int *keys, Acc *vals, int n, int S, int *hist, int lane) {
    if (n <= 1) return;
    if (n <= 32) {
        int k = lane < n ? keys[lane] : INT32_MAX;
        Acc v = lane < n ? vals[lane] : Acc(0);
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const int ok = __shfl_xor_sync(kFull, k, stride);
                const Acc ov = __shfl_xor_sync(kFull, v, stride);
                const bool ascending = (lane & size) == 0;
                const bool lower = (lane & stride) == 0;
                // the lower lane of a pair keeps the smaller key in an
                // ascending block, the larger in a descending one
                if (lower == ascending ? ok < k : ok > k) {
                    k = ok;
                    v = ov;
                }
            }
        }
        __syncwarp();
        if (lane < n) {
            keys[lane] = k;
            vals[lane] = v;
        }
        __syncwarp();
        return;
    }
    if (n > (S >> 1)) {
        int npad = 1;
        while (npad < n) npad <<= 1;
        for (int s = n + lane; s < npad; s += 32) keys[s] = INT32_MAX;
        __syncwarp();
        warp_bitonic<Acc>(keys, vals, npad, lane);
        return;
    }
    int kmax = 0;
    for (int s = lane; s < n; s += 32) kmax = max(kmax, keys[s]);
    kmax = __reduce_max_sync(kFull, kmax);
    const int bits = 32 - __clz(kmax);
    int *sk = keys, *dk = keys + (S >> 1);
    Acc *sv = vals, *dv = vals + (S >> 1);
    const unsigned below = (1u << lane) - 1u;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0;
        __syncwarp();
        for (int s = lane; s < n; s += 32) atomicAdd(hist + ((sk[s] >> shift) & 255), 1);
        __syncwarp();
        // exclusive scan of the 256 counts, 8 consecutive per lane
        int c[8], tot = 0;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            c[u] = hist[lane * 8 + u];
            tot += c[u];
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        int run = incl - tot;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            hist[lane * 8 + u] = run;
            run += c[u];
        }
        __syncwarp();
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int s = c0 + lane;
            const bool valid = s < n;
            const int k = valid ? sk[s] : 0;
            const Acc v = valid ? sv[s] : Acc(0);
            const int d = valid ? ((k >> shift) & 255) : 256 + lane;
            const unsigned peers = __match_any_sync(kFull, d);
            const int rank = __popc(peers & below);
            const int pos = valid ? hist[d] + rank : 0;
            __syncwarp();
            if (valid) {
                dk[pos] = k;
                dv[pos] = v;
                if (rank == 0) hist[d] += __popc(peers);
            }
            __syncwarp();
        }
        int *tk = sk;
        sk = dk;
        dk = tk;
        Acc *tv = sv;
        sv = dv;
        dv = tv;
    }
    if (sk != keys) {
        for (int s = lane; s < n; s += 32) {
            keys[s] = sk[s];
            vals[s] = sv[s];
        }
        __syncwarp();
    }
}

// Shared-memory accumulator of a heavy item (slots addressed by rank or by
// row).  Doubles use the native atomic add of a double.  Wrapping int64
// sums are kept as two 32-bit halves in separate arrays: a 64-bit add is a
// 32-bit atomic add on the low half that returns the old low word, from which
// the carry out of the low half follows exactly; the high half then receives
// the value's high word plus that carry (skipped when zero, the common case
// for small non-negative values).  Every update is thus exact modulo 2^64 in
// any order, and 32-bit shared atomics run several times faster than 64-bit
// ones on this GPU.
template <typename Acc>
struct HeavyAcc;
template <>
struct HeavyAcc<double> {
    double *a;
    static constexpr size_t bytes_per_slot = 8;
    __device__ __forceinline__ HeavyAcc(void *base, int) : a((double *)base) {}
    __device__ __forceinline__ void zero(int i) const { a[i] = 0.0; }
    __device__ __forceinline__ void add(int i, double v) const { atomicAdd(a + i, v); }
    __device__ __forceinline__ double get(int i) const { return a[i]; }
    __device__ __forceinline__ int32_t *scratch32() const { return (int32_t *)a; }
};
template <>
struct HeavyAcc<long long> {
    uint32_t *lo, *hi;
    static constexpr size_t bytes_per_slot = 8;
    __device__ __forceinline__ HeavyAcc(void *base, int slots) : lo((uint32_t *)base), hi((uint32_t *)base + slots) {}
    __device__ __forceinline__ void zero(int i) const {
        lo[i] = 0u;
        hi[i] = 0u;
    }
    __device__ __forceinline__ void add(int i, long long v) const {
        const unsigned long long u = (unsigned long long)v;
        const uint32_t vlo = (uint32_t)u, vhi = (uint32_t)(u >> 32);
        const uint32_t old = atomicAdd(lo + i, vlo);
        const uint32_t h = vhi + ((uint32_t)(old + vlo) < old ? 1u : 0u);
        if (h) atomicAdd(hi + i, h);
    }
    __device__ __forceinline__ long long get(int i) const {
        return (long long)(((unsigned long long)hi[i] << 32) | (unsigned long long)lo[i]);
    }
    __device__ __forceinline__ int32_t *scratch32() const { return (int32_t *)lo; }
};

// Load a heavy item's bitmap words into bp[].x and their exclusive popcount
// prefix into bp[].y, returning the total.  Warp w takes 32-word chunks w,
// w + nw, ...: lanes load consecutive words (coalesced, one word per bank
// pair) and scan them with shuffles; a second pass adds the chunk offsets
// (every warp scans the chunk totals itself).  ctot holds one int per chunk
// (nwords <= 32 * 64).  Ends with a barrier.
__device__ __forceinline__ int cta_load_scan_bitmap(const uint32_t *__restrict__ src, uint2 *bp, int nwords,
                                                    int *ctot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = (nwords + 31) >> 5;
    for (int c = wid; c < nch; c += nw) {
        const int w = (c << 5) + lane;
        const uint32_t x = w < nwords ? ld_stream(src + w) : 0u;
        const int pc = __popc(x);
        int inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (w < nwords) bp[w] = make_uint2(x, (uint32_t)(inc - pc));
        if (lane == 31) ctot[c] = inc;
    }
    __syncthreads();
    // exclusive prefix of the chunk totals, each warp for itself (<= 64 chunks)
    const int t0 = lane < nch ? ctot[lane] : 0, t1 = lane + 32 < nch ? ctot[lane + 32] : 0;
    int i0 = t0, i1 = t1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(kFull, i0, o), b = __shfl_up_sync(kFull, i1, o);
        if (lane >= o) {
            i0 += a;
            i1 += b;
        }
    }
    const int half = __shfl_sync(kFull, i0, 31);
    const int total = half + __shfl_sync(kFull, i1, 31);
    for (int c = wid; c < nch; c += nw) {
        // offset of chunk c = exclusive prefix at c
        const int src_lane = c & 31;
        const int e0 = __shfl_sync(kFull, i0 - t0, src_lane), e1 = __shfl_sync(kFull, i1 - t1, src_lane);
        const int off = c < 32 ? e0 : half + e1;
        const int w = (c << 5) + lane;
        if (w < nwords) bp[w].y += (uint32_t)off;
    }
    __syncthreads();
    return total;
}

}  // namespace spg
