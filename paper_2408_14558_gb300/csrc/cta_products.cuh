// CTA-wide walk over the products of one heavy output column (used by the
// heavy symbolic and numeric kernels).
#pragma once

#include <type_traits>

#include "spg_internal.cuh"

namespace spg {

// Staging area of cta_products for one batch of kBatch B' entries: the
// non-empty A~ segments they multiply.  Long segments (>= kLongSeg entries)
// sit at [0, nl), short ones at [nl, nl + ns); each part numbers its products
// consecutively and pref holds a segment's first product in that numbering.
template <typename Acc>
struct CtaBatch {
    long long start[kBatch];
    int pref[kBatch + 2];
    Acc bv[kBatch];
    int wsum[4][33];
};

// Exclusive CTA scan of four counters at once; every thread gets the totals in
// tot[0..3].  One barrier: every warp reads all warp sums and takes its own
// offsets, so wsum must not be written again before the caller's next barrier.
__device__ __forceinline__ void cta_scan4(const int v[4], int ex[4], int (*wsum)[33], int tot[4]) {
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
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int wt = lane < nw ? wsum[q][lane] : 0;
        ex[q] = __reduce_add_sync(kFull, lane < wid ? wt : 0) + in[q] - v[q];
        tot[q] = __reduce_add_sync(kFull, wt);
    }
}

// One thread's B' entry of a batch: its A~ segment and its value.
template <typename Acc>
struct SegReg {
    long long st = 0;
    int len = 0;
    Acc bv = Acc(0);
};

// The segment of this thread's entry in the first batch of [p0, p1); callers
// fetch it early so that its loads overlap their own set-up.
template <typename Acc, typename SegFn>
__device__ __forceinline__ SegReg<Acc> cta_first_seg(int64_t p0, int64_t p1, SegFn seg) {
    SegReg<Acc> r;
    if (p0 + threadIdx.x < p1) seg(p0 + threadIdx.x, r.st, r.len, r.bv);
    return r;
}

// Walk every product of the B' entries [p0, p1) of one output column with the
// whole CTA (all threads must call it; blockDim.x == kBatch); `first` is
// cta_first_seg(p0, p1, seg).
// seg(p, start, len, bv) gives the A~ positions [start, start+len) that B'
// entry p multiplies and its value; body(row, product) runs once per product.
// The segments of the next batch are fetched before the current batch is
// walked.  The products of the long segments are shared evenly by the warps
// (lanes read consecutive entries, coalesced); each warp step takes the next
// 32 x U products of the warp's range, across segment boundaries, so that U
// loads per lane are in flight however the segments fall.  The products of
// short segments are shared evenly too (a warp bitmask locates each lane's
// segment).  One batch must hold < 2^31 products (heavy items bound their
// segments to the item's row range).  Ends with a barrier.
static_assert(kLongSeg >= 32, "a 32-product window must meet at most two long segments");

template <bool NEED_VAL, int U, typename Acc, typename SegFn, typename Body>
__device__ __forceinline__ void cta_products(int64_t p0, int64_t p1, CtaBatch<Acc> &sb,
                                             const int32_t *__restrict__ At_row, const Acc *__restrict__ At_val,
                                             SegReg<Acc> first, SegFn seg, Body body) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    SegReg<Acc> cur = first;
    for (int64_t b0 = p0; b0 < p1; b0 += kBatch) {
        const long long st = cur.st;
        const int len = cur.len;
        const Acc bv = cur.bv;
        const bool is_long = len >= kLongSeg;
        const int v[4] = {is_long ? 1 : 0, is_long ? len : 0, (!is_long && len > 0) ? 1 : 0, is_long ? 0 : len};
        int ex[4], tot[4];
        cta_scan4(v, ex, sb.wsum, tot);
        const int nl = tot[0], nlp = tot[1], ns = tot[2], nsp = tot[3];
        if (is_long) {
            sb.start[ex[0]] = st;
            sb.pref[ex[0]] = ex[1];
            if (NEED_VAL) sb.bv[ex[0]] = bv;
        } else if (len > 0) {
            sb.start[nl + ex[2]] = st;
            sb.pref[nl + ex[2]] = ex[3];
            if (NEED_VAL) sb.bv[nl + ex[2]] = bv;
        }
        __syncthreads();
        if (b0 + kBatch < p1) cur = cta_first_seg<Acc>(b0 + kBatch, p1, seg);

        // long segments: products [f0, f1) of this warp in the long
        // segments' own numbering (no padding between segments), 32 per warp
        // step, U steps in flight.  A long segment holds >= 32 products, so a
        // window of 32 consecutive products meets at most two segments (the
        // current one, A, and the next, B) and crosses at most one boundary
        // per step.  Each segment's start is kept minus its product prefix,
        // so product f of it is entry base + f of A~.
        {
            const int per = (nlp + nw - 1) / nw;
            const int f0 = wid * per, f1 = min(nlp, f0 + per);
            if (f0 < f1) {
                int s = 0;
                for (int stp = kBatch >> 1; stp > 0; stp >>= 1)
                    if (s + stp < nl && sb.pref[s + stp] <= f0) s += stp;
                long long baseA = sb.start[s] - sb.pref[s];
                Acc bvA = NEED_VAL ? sb.bv[s] : Acc(0);
                int nB = s + 1 < nl ? sb.pref[s + 1] : nlp;  // first product of B
                long long baseB = 0;
                Acc bvB = Acc(0);
                if (s + 1 < nl) {
                    baseB = sb.start[s + 1] - nB;
                    if (NEED_VAL) bvB = sb.bv[s + 1];
                }
                // one step: U windows located and loaded, then used; FULL: all
                // 32 x U products lie in the warp's range (every step but the
                // last), so no lane needs a bounds check
                auto step = [&](const int f, auto full) {
                    constexpr bool FULL = decltype(full)::value;
                    int r[U];
                    Acc a[U], bu[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int fb = f + 32 * u;
                        if (fb >= nB) {  // the window starts in B: B becomes A
                            s++;
                            baseA = baseB;
                            bvA = bvB;
                            nB = s + 1 < nl ? sb.pref[s + 1] : nlp;
                            if (s + 1 < nl) {
                                baseB = sb.start[s + 1] - nB;
                                if (NEED_VAL) bvB = sb.bv[s + 1];
                            }
                        }
                        const int fi = fb + lane;
                        const bool inB = fi >= nB;
                        const long long e = (inB ? baseB : baseA) + fi;
                        bu[u] = inB ? bvB : bvA;
                        ok[u] = FULL || fi < f1;
                        r[u] = 0;
                        a[u] = Acc(0);
                        if (ok[u]) {
                            r[u] = __ldg(At_row + e);
                            if (NEED_VAL) a[u] = __ldg(At_val + e);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (ok[u]) body(r[u], NEED_VAL ? mul_acc<Acc>(a[u], bu[u]) : Acc(0));
                };
                int f = f0;
                for (; f + 32 * U <= f1; f += 32 * U) step(f, std::true_type{});
                if (f < f1) step(f, std::false_type{});
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
