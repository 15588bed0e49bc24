// CTA-wide walk over the products of one heavy output column (used by the
// heavy symbolic and numeric kernels).
#pragma once

#include "spg_internal.cuh"

namespace spg {

// Staging area of cta_products for one batch of kBatch B' entries: the
// non-empty A~ segments they multiply.  Long segments (>= kLongSeg entries)
// sit at [0, nl) and are walked in chunks of 32 entries, one chunk per warp
// step; short ones sit at [nl, nl + ns) and are packed one product per lane.
// pref holds the exclusive prefix of the chunk counts (long part) and of the
// product counts (short part).
template <typename Acc>
struct CtaBatch {
    long long start[kBatch];
    int pref[kBatch + 2];
    int len[kBatch];
    Acc bv[kBatch];
    int wsum[4][33];
    int nl, nchunk, ns, nshort;
};

// Exclusive CTA scan of four counters at once; the totals land in tot[0..3].
__device__ __forceinline__ void cta_scan4(const int v[4], int ex[4], int (*wsum)[33], int *tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int in[4];
#pragma unroll
    for (int q = 0; q < 4; q++) in[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int t = __shfl_up_sync(kFull, in[q], o);
            if (lane >= o) in[q] += t;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < 4; q++) wsum[q][wid] = in[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int x = lane < nw ? wsum[q][lane] : 0;
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(kFull, xi, o);
                if (lane >= o) xi += t;
            }
            if (lane < nw) wsum[q][lane] = xi - x;
            if (lane == 31) tot[q] = xi;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) ex[q] = wsum[q][wid] + in[q] - v[q];
}

// Walk every product of the B' entries [p0, p1) of one output column with the
// whole CTA (all threads must call it; blockDim.x == kBatch).
// seg(p, start, len, bv) gives the A~ positions [start, start+len) that B'
// entry p multiplies and its value; body(row, product) runs once per product.
// The chunks of the long segments are shared evenly by the warps (lanes read
// consecutive entries: no search, coalesced); U chunks are in flight per warp
// step so that U loads per lane overlap.  The products of short segments are
// shared evenly too, each lane locating its segment by a binary search over
// a window of at most 64 segments.  One batch must hold < 2^31 products
// (heavy items bound their segments to the item's row range).  Ends with a
// barrier.
template <bool NEED_VAL, int U, typename Acc, typename SegFn, typename Body>
__device__ __forceinline__ void cta_products(int64_t p0, int64_t p1, CtaBatch<Acc> &sb,
                                             const int32_t *__restrict__ At_row, const Acc *__restrict__ At_val,
                                             SegFn seg, Body body) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int64_t b0 = p0; b0 < p1; b0 += kBatch) {
        const int nb = (int)min((int64_t)kBatch, p1 - b0);
        long long st = 0;
        int len = 0;
        Acc bv = Acc(0);
        if (tid < nb) seg(b0 + tid, st, len, bv);
        const bool is_long = len >= kLongSeg;
        const int v[4] = {is_long ? 1 : 0, is_long ? (len + 31) >> 5 : 0, (!is_long && len > 0) ? 1 : 0,
                          is_long ? 0 : len};
        int ex[4];
        cta_scan4(v, ex, sb.wsum, &sb.nl);
        const int nl = sb.nl, nch = sb.nchunk, ns = sb.ns, nsp = sb.nshort;
        if (is_long) {
            sb.start[ex[0]] = st;
            sb.pref[ex[0]] = ex[1];
            sb.len[ex[0]] = len;
            if (NEED_VAL) sb.bv[ex[0]] = bv;
        } else if (len > 0) {
            sb.start[nl + ex[2]] = st;
            sb.pref[nl + ex[2]] = ex[3];
            if (NEED_VAL) sb.bv[nl + ex[2]] = bv;
        }
        __syncthreads();

        // long segments: chunks [c0, c1) of this warp, U per step
        {
            const int per = (nch + nw - 1) / nw;
            const int c0 = wid * per, c1 = min(nch, c0 + per);
            if (c0 < c1) {
                int s = 0;
                for (int stp = kBatch >> 1; stp > 0; stp >>= 1)
                    if (s + stp < nl && sb.pref[s + stp] <= c0) s += stp;
                // segment by segment: the chunks of segment s inside [c0, c1)
                for (int c = c0; c < c1; s++) {
                    const int sp = sb.pref[s];
                    const int cend = min(c1, s + 1 < nl ? sb.pref[s + 1] : nch);
                    const int skip = (c - sp) << 5;
                    const long long st = sb.start[s] + skip + lane;
                    const int rem = sb.len[s] - skip - lane;  // entries left for this lane's first chunk
                    const Acc bvs = NEED_VAL ? sb.bv[s] : Acc(0);
                    const int nck = cend - c;
                    for (int k = 0; k < nck; k += U) {
                        int r[U];
                        Acc a[U];
                        bool ok[U];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            ok[u] = k + u < nck && ((k + u) << 5) < rem;
                            r[u] = 0;
                            a[u] = Acc(0);
                            if (ok[u]) {
                                r[u] = __ldg(At_row + st + ((k + u) << 5));
                                if (NEED_VAL) a[u] = __ldg(At_val + st + ((k + u) << 5));
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (ok[u]) body(r[u], NEED_VAL ? mul_acc<Acc>(a[u], bvs) : Acc(0));
                    }
                    c = cend;
                }
            }
        }
        // short segments: products [f0, f1) of this warp, one per lane
        {
            const int per = (nsp + nw - 1) / nw;
            const int f0 = wid * per, f1 = min(nsp, f0 + per);
            const int *spref = sb.pref + nl;
            const long long *sstart = sb.start + nl;
            const Acc *sbv = sb.bv + nl;
            if (f0 < f1) {
                // s0: the segment holding product f (found once by binary search)
                int s0 = 0;
                for (int stp = kBatch >> 1; stp > 0; stp >>= 1)
                    if (s0 + stp < ns && spref[s0 + stp] <= f0) s0 += stp;
                for (int f = f0; f < f1; f += 32) {
                    // lane k holds segment s0 + k; segments are non-empty, so the
                    // window [f, f+32) meets at most s0 .. s0+31, and segment
                    // s0+k (k >= 1) starts at window position spref - f >= 1
                    const int sk = s0 + lane;
                    const int pk = sk < ns ? spref[sk] : 0x7fffffff;
                    const long long stk = sk < ns ? sstart[sk] : 0;
                    const Acc bvk = (NEED_VAL && sk < ns) ? sbv[sk] : Acc(0);
                    const int pos = pk - f;
                    const uint32_t M = __reduce_or_sync(kFull, (lane > 0 && pos < 32) ? (1u << pos) : 0u);
                    const int k = __popc(M & ((2u << lane) - 1u));  // segment starts at positions <= lane
                    const long long st = __shfl_sync(kFull, stk, k);
                    const int sp = __shfl_sync(kFull, pk, k);
                    const int fi = f + lane;
                    if (NEED_VAL) {
                        const Acc b = __shfl_sync(kFull, bvk, k);
                        if (fi < f1) {
                            const long long e = st + (fi - sp);
                            body(__ldg(At_row + e), mul_acc<Acc>(__ldg(At_val + e), b));
                        }
                    } else if (fi < f1) {
                        body(__ldg(At_row + st + (fi - sp)), Acc(0));
                    }
                    // the segment holding product f + 32
                    int c = __popc(M);
                    if (s0 + c + 1 < ns && spref[s0 + c + 1] == f + 32) c++;
                    s0 += c;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace spg
