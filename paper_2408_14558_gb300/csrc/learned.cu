// Learned nnz sizing: an extension beyond the paper.  A small MLP predicts
// nnz(C(:,j)) from cheap per-column features; the prediction sizes every
// column's output room, so the numeric work runs without the exact symbolic
// pass.  Columns whose product overflows its room are recomputed through the
// exact path (plan, symbolic, numeric on the columns that overflowed), so C is
// the same as the exact path's: identical structure, identical integer values,
// double values within the same accumulation-order bound.
//
//   model: 4 -> 32 -> 32 -> 1, ReLU, float32; features log1p(flops_j),
//          log1p(nnz(B(:,j))), log1p(max nnz(A(:,k))), log1p(mean nnz(A(:,k)));
//          target log1p(nnz(C(:,j))); loss MSE; Adam.
//   kernels: k_mlp_forward (thread per sample), k_mlp_grad (thread per sample,
//          warp-shuffle reduction of every gradient component), k_adam.
//   learned multiply: light columns use warp hash tables sized from the
//          prediction; heavy columns use a fused one-pass kernel (dense row
//          accumulator + row bitmap per 4096-row item) whose counts are exact,
//          in groups of heavy columns, each group placed in C (on a second
//          stream) while the next one computes; overflowed columns are
//          recomputed and C is then assembled after them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "block_ops.cuh"
#include "cta_products.cuh"
#include "spg_internal.cuh"

namespace spg {

constexpr int kH = 32, kF = 4;
constexpr int kW1 = 0, kB1 = kW1 + kH * kF, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
constexpr int kNP = kB3 + 1;  // 1249
static_assert(kNP == 1249, "parameter layout");
#ifndef SPG_FUSED_ROWS
#define SPG_FUSED_ROWS 4096
#endif
constexpr int kFusedRows = SPG_FUSED_ROWS;  // rows of one fused heavy item (dense accumulator in shared memory)

const char *last_error_str();
void clear_error();

}  // namespace spg

struct spg_model {
    float *d_params = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr, *d_loss = nullptr;
    int64_t step = 0;
};

namespace spg {

// ----------------------------------------------------------------- the MLP

__device__ __forceinline__ void mlp_layer1(const float *P, const float x[kF], float h1[kH]) {
#pragma unroll
    for (int j = 0; j < kH; j++) {
        float z = P[kB1 + j];
#pragma unroll
        for (int k = 0; k < kF; k++) z = fmaf(P[kW1 + j * kF + k], x[k], z);
        h1[j] = fmaxf(z, 0.f);
    }
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ params, const float *__restrict__ X,
                                                     int64_t n, float *__restrict__ out) {
    __shared__ float P[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        float x[kF], h1[kH];
#pragma unroll
        for (int k = 0; k < kF; k++) x[k] = X[s * kF + k];
        mlp_layer1(P, x, h1);
        float y = P[kB3];
#pragma unroll 1
        for (int i = 0; i < kH; i++) {
            float z = P[kB2 + i];
#pragma unroll
            for (int j = 0; j < kH; j++) z = fmaf(P[kW2 + i * kH + j], h1[j], z);
            y = fmaf(P[kW3 + i], fmaxf(z, 0.f), y);
        }
        out[s] = y;
    }
}

__device__ __forceinline__ void grad_acc(float *G, int idx, float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(G + idx, v);
}

// Gradient of scale * sum (y - t)^2 over samples [n0, n1) (scale = 1/batch
// gives the mean squared error).  One thread per sample; every gradient
// component is summed over the warp with shuffles, then added to a
// per-CTA buffer, then to `grad`.  loss receives sum (y - t)^2.
__global__ void __launch_bounds__(256) k_mlp_grad(const float *__restrict__ params, const float *__restrict__ X,
                                                  const float *__restrict__ T, int64_t n0, int64_t n1, float scale,
                                                  float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ float P[kNP];
    __shared__ float G[kNP];
    __shared__ float lsum;
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) {
        P[i] = params[i];
        G[i] = 0.f;
    }
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();
    float lacc = 0.f;
    for (int64_t base = n0 + (int64_t)blockIdx.x * blockDim.x; base < n1; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = base + threadIdx.x;
        const bool valid = s < n1;
        float x[kF], h1[kH], z2[kH];
#pragma unroll
        for (int k = 0; k < kF; k++) x[k] = valid ? X[s * kF + k] : 0.f;
        const float t = valid ? T[s] : 0.f;
        mlp_layer1(P, x, h1);
        float y = P[kB3];
#pragma unroll
        for (int i = 0; i < kH; i++) {
            float z = P[kB2 + i];
#pragma unroll
            for (int j = 0; j < kH; j++) z = fmaf(P[kW2 + i * kH + j], h1[j], z);
            z2[i] = z;
            y = fmaf(P[kW3 + i], fmaxf(z, 0.f), y);
        }
        const float e = y - t;
        const float dy = valid ? 2.f * scale * e : 0.f;
        if (valid) lacc += e * e;
#pragma unroll
        for (int i = 0; i < kH; i++) grad_acc(G, kW3 + i, dy * fmaxf(z2[i], 0.f));
        grad_acc(G, kB3, dy);
        float dh1[kH];
#pragma unroll
        for (int j = 0; j < kH; j++) dh1[j] = 0.f;
#pragma unroll
        for (int i = 0; i < kH; i++) {
            const float g2 = z2[i] > 0.f ? dy * P[kW3 + i] : 0.f;
            grad_acc(G, kB2 + i, g2);
#pragma unroll
            for (int j = 0; j < kH; j++) {
                grad_acc(G, kW2 + i * kH + j, g2 * h1[j]);
                dh1[j] = fmaf(g2, P[kW2 + i * kH + j], dh1[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kH; j++) {
            const float g1 = h1[j] > 0.f ? dh1[j] : 0.f;
            grad_acc(G, kB1 + j, g1);
#pragma unroll
            for (int k = 0; k < kF; k++) grad_acc(G, kW1 + j * kF + k, g1 * x[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(kFull, lacc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&lsum, lacc);
    __syncthreads();
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) atomicAdd(grad + i, G[i]);
    if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------ features and labels

__global__ void k_features(int64_t n, const int64_t *flops, const int32_t *nnzb, const int32_t *maxa, float *X) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double f = (double)flops[j], b = (double)nnzb[j];
        X[j * 4 + 0] = log1pf((float)f);
        X[j * 4 + 1] = log1pf((float)b);
        X[j * 4 + 2] = log1pf((float)maxa[j]);
        X[j * 4 + 3] = log1pf(b > 0 ? (float)(f / b) : 0.f);
    }
}

__global__ void k_labels(int64_t n, const int64_t *nnzcol, float *y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        y[j] = log1pf((float)nnzcol[j]);
}

// ------------------------------------------------------- learned multiply

// Capacity of every column: the prediction times the slack, at least 1, at
// most the exact bound U_j = min(flops_j, row window) (which always fits).
__global__ void k_capacity(int64_t n, const float *pred, const int8_t *bin_of, const int64_t *flops,
                           const int32_t *win_lo, const int32_t *win_hi, float slack, int light_max, int64_t *cap,
                           int8_t *lbin) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin_of[j];
        int64_t U = 0;
        if (b != kBinEmpty) U = min((long long)flops[j], (long long)(win_hi[j] - win_lo[j] + 1));
        float pr = pred[j];
        if (!(pr > 0.f)) pr = 0.f;
        if (pr > 40.f) pr = 40.f;
        const double want = ceil((double)slack * (double)expm1f(pr));
        int64_t c = U == 0 ? 0 : (int64_t)fmin((double)U, fmax(want, 1.0));
        cap[j] = c;
        int lb = b;
        if (b != kBinHeavy && b != kBinEmpty) {
            long long S = 64;
            lb = 1;
            while (S < 2 * c) {
                S <<= 1;
                lb++;
            }
        }
        lbin[j] = (int8_t)lb;
    }
}

__device__ __forceinline__ void mark_overflow(int32_t *flag, int j, unsigned long long *nflag) {
    if (atomicExch(flag + j, 1) == 0) atomicAdd(nflag, 1ull);
}

// Light columns: warp hash of 2^LOGS slots sized from the capacity; the
// sorted column goes to its room [capoff_j, capoff_j + cap_j) of the
// predicted layout, or the column is flagged if it holds more than cap_j.
template <int LOGS, int WARPS, typename Acc, typename OutIdx>
__global__ void __launch_bounds__(WARPS * 32)
    k_light_learned(const int32_t *__restrict__ list, int64_t ncols, const void *Bcolptr, int p64,
                    const int32_t *__restrict__ Bq, const Acc *__restrict__ Bv,
                    const int64_t *__restrict__ At_colptr, const int32_t *__restrict__ At_row,
                    const Acc *__restrict__ At_val, const int64_t *__restrict__ capoff,
                    const int64_t *__restrict__ cap, int64_t *__restrict__ nnz, int32_t *flag,
                    unsigned long long *nflag, OutIdx *__restrict__ trow, Acc *__restrict__ tval) {
    constexpr int S = 1 << LOGS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSeg<Acc> *segs = (WarpSeg<Acc> *)smem_raw;
    Acc *vals_all = (Acc *)(segs + WARPS);
    int *keys_all = (int *)(vals_all + WARPS * S);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *keys = keys_all + wid * S;
    Acc *vals = vals_all + wid * S;
    int *hist = keys_all + WARPS * S + wid * 256;
    for (int64_t c = (int64_t)blockIdx.x * WARPS + wid; c < ncols; c += (int64_t)gridDim.x * WARPS) {
        const int j = list[c];
        for (int s = lane; s < S; s += 32) {
            keys[s] = kEmptyKey;
            vals[s] = Acc(0);
        }
        __syncwarp();
        const int64_t p0 = ld_ptr(Bcolptr, p64, j), p1 = ld_ptr(Bcolptr, p64, j + 1);
        bool full = false;
        warp_products<true, Acc>(
            p0, p1, lane, segs[wid], At_row, At_val,
            [&](int64_t p, long long &st, int &len, Acc &bv) {
                int q = Bq[p];
                if (q >= 0) {
                    st = At_colptr[q];
                    len = (int)(At_colptr[q + 1] - st);
                    bv = Bv[p];
                }
            },
            [&](int r, Acc v) {
                bool fresh;
                int slot = hash_insert(keys, LOGS, r, &fresh);
                if (slot < 0)
                    full = true;
                else
                    atomic_add_acc(vals + slot, v);
            });
        __syncwarp();
        int nout = 0;
        for (int c0 = 0; c0 < S; c0 += 32) {
            int kk = keys[c0 + lane];
            Acc vv = vals[c0 + lane];
            bool occ = kk != kEmptyKey;
            unsigned bal = __ballot_sync(kFull, occ);
            __syncwarp();
            if (occ) {
                int pos = nout + __popc(bal & ((1u << lane) - 1u));
                keys[pos] = kk;
                vals[pos] = vv;
            }
            nout += __popc(bal);
            __syncwarp();
        }
        full = __any_sync(kFull, full);
        if (full || nout > cap[j]) {
            if (lane == 0) mark_overflow(flag, j, nflag);
        } else {
            warp_sort_pairs<Acc>(keys, vals, nout, S, hist, lane);
            const int64_t base = capoff[j];
            for (int s = lane; s < nout; s += 32) {
                trow[base + s] = (OutIdx)keys[s];
                tval[base + s] = vals[s];
            }
            if (lane == 0) nnz[j] = nout;
        }
        __syncwarp();
    }
}

// Heavy columns, one pass: CTA per item of <= kFusedRows rows of one column,
// items claimed one at a time from a device counter.  Every product sets its
// row bit and adds into a dense row accumulator; the item's count is then
// exact, its room is reserved inside the column's predicted room (atomically,
// items of a column land in any order), and the item is written there in row
// order, one bitmap word per warp step (the set bits of a word are consecutive
// entries: coalesced).  An item that does not fit flags its column (the count
// still adds to colfill, which ends as the exact nnz).  The accumulator is
// cleared as it is read, so it is zero again for the next item.  One launch
// takes the items [it_begin, it_begin + nitems).
template <typename Acc, typename OutIdx>
__global__ void __launch_bounds__(kBatch)
    k_fused_heavy(int64_t nitems, const int32_t *__restrict__ it_rec0, const int32_t *__restrict__ it_nrec,
                  const int32_t *__restrict__ rec_col, const int32_t *__restrict__ rec_slab, const void *Bcolptr,
                  int p64, const int32_t *__restrict__ Bq, const Acc *__restrict__ Bv,
                  const int64_t *__restrict__ At_colptr, const int32_t *__restrict__ At_row,
                  const Acc *__restrict__ At_val, const int32_t *__restrict__ split, int T, int R,
                  const int64_t *__restrict__ capoff, const int64_t *__restrict__ cap,
                  unsigned long long *__restrict__ colfill, int32_t *flag, unsigned long long *nflag,
                  int32_t *__restrict__ item_cnt, int64_t *__restrict__ item_pos, OutIdx *__restrict__ trow,
                  Acc *__restrict__ tval, unsigned long long *next, int64_t it_begin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaBatch<Acc> &sb = *(CtaBatch<Acc> *)smem_raw;
    unsigned char *acc_raw = smem_raw + ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15);
    const HeavyAcc<Acc> acc(acc_raw, kFusedRows);  // dense: slot = row within the item
    uint32_t *bits = (uint32_t *)(acc_raw + HeavyAcc<Acc>::bytes_per_slot * kFusedRows);
    int *pre = (int *)(bits + kFusedRows / 32);
    __shared__ int wsum[33];
    __shared__ long long pos_sh, claim;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < kFusedRows; i += blockDim.x) acc.zero(i);
    const int RW = R >> 5;
    for (int64_t li = cta_claim(next, &claim); li < nitems; li = cta_claim(next, &claim)) {
        const int64_t it = it_begin + li;
        const int r0 = it_rec0[it], nr = it_nrec[it];
        const int j = rec_col[r0], t0 = rec_slab[r0];
        const int nwords = nr * RW;
        const long long rbase = (long long)t0 * R;
        const int64_t p0 = ld_ptr(Bcolptr, p64, j), p1 = ld_ptr(Bcolptr, p64, j + 1);
        auto seg = [&](int64_t p, long long &st, int &len, Acc &bv) {
            int q = Bq[p];
            if (q >= 0) {
                const int32_t *sp = split + (int64_t)q * (T + 1);
                int a = sp[t0], b = sp[t0 + nr];
                st = At_colptr[q] + a;
                len = b - a;
                bv = Bv[p];
            }
        };
        const SegReg<Acc> first = cta_first_seg<Acc>(p0, p1, seg);
        // (the first barrier of cta_products orders this before every product)
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0;
        cta_products<true, SPG_NUM_UNROLL, Acc>(
            p0, p1, sb, At_row, At_val, first, seg,
            [&](int r, Acc v) {
                const int lr = (int)(r - rbase);
                set_bit_shared(bits + (lr >> 5), 1u << (lr & 31));
                acc.add(lr, v);
            });
        const int cnt = cta_scan_popc1(bits, pre, nwords, wsum);
        if (threadIdx.x == 0) {
            long long pos = (long long)atomicAdd(colfill + j, (unsigned long long)cnt);
            if (pos + cnt > cap[j]) {
                mark_overflow(flag, j, nflag);
                pos = -1;
            }
            pos_sh = pos;
            item_cnt[it] = cnt;
            item_pos[it] = pos;
        }
        __syncthreads();
        const long long pos = pos_sh;
        const int64_t base = pos >= 0 ? capoff[j] + pos : 0;
        for (int w = wid; w < nwords; w += nw) {
            const uint32_t word = bits[w];
            if (((word >> lane) & 1u) == 0) continue;
            const int lr = w * 32 + lane;
            if (pos >= 0) {
                const int64_t o = base + pre[w] + __popc(word & ((1u << lane) - 1u));
                st_stream(trow + o, (OutIdx)(rbase + lr));
                st_stream(tval + o, acc.get(lr));
            }
            acc.zero(lr);
        }
    }
}

__global__ void k_count_groups(int64_t nheavy, const int64_t *rec_first, int per, int64_t *cnt) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x)
        cnt[h] = (rec_first[h + 1] - rec_first[h] + per - 1) / per;
}

// Exact nnz of every column after the learned pass: heavy columns from their
// fill counter, light ones from the kernel; overflowed columns get 0 here and
// their exact count later.
__global__ void k_learned_nnz(int64_t n, const int8_t *bin_of, const unsigned long long *colfill,
                              const int64_t *nnz_light, const int32_t *flag, int64_t *nnz,
                              unsigned long long *heavy_sum) {
    unsigned long long hsum = 0;  // entries of the heavy columns the fused pass completed
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin_of[j];
        int64_t v = 0;
        if (!flag[j]) {
            if (b == kBinHeavy) {
                v = (int64_t)colfill[j];
                hsum += (unsigned long long)v;
            } else if (b != kBinEmpty) {
                v = nnz_light[j];
            }
        }
        nnz[j] = v;
    }
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
    if ((threadIdx.x & 31) == 0 && hsum) atomicAdd(heavy_sum, hsum);
}

// The same for the columns [c0, c1) of one group of the pipelined assembly;
// a flagged column (its count is not known yet) marks the order broken:
// later columns cannot be placed before the recompute.
__global__ void k_learned_nnz_range(int64_t c0, int64_t c1, const int8_t *bin_of,
                                    const unsigned long long *colfill, const int64_t *nnz_light,
                                    const int32_t *flag, int64_t *nnz, unsigned long long *heavy_sum,
                                    int *broken) {
    unsigned long long hsum = 0;
    bool any = false;
    for (int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c1;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin_of[j];
        int64_t v = 0;
        if (flag[j]) {
            any = true;
        } else if (b == kBinHeavy) {
            v = (int64_t)colfill[j];
            hsum += (unsigned long long)v;
        } else if (b != kBinEmpty) {
            v = nnz_light[j];
        }
        nnz[j] = v;
    }
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
    if ((threadIdx.x & 31) == 0 && hsum) atomicAdd(heavy_sum, hsum);
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(broken, 1);
}

// Canonical column pointers of one group: the group's exclusive scan
// local[0..len] plus the entries of all earlier groups (carry[g]); the
// group's end goes to carry[g + 1].
__global__ void k_add_carry(const int64_t *local, int64_t len, const int64_t *carry_in, int64_t *carry_out,
                            int64_t *colptr) {
    const int64_t c = *carry_in;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= len; i += (int64_t)gridDim.x * blockDim.x)
        colptr[i] = c + local[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *carry_out = c + local[len];
}

// Boundaries of the pipelined assembly's groups: for g = 0..G, the first item
// of heavy column hb[g] and the first column of group g (0 for the first
// group, n past the last one, else the id of the group's first heavy column;
// the heavy list is in column order).
__global__ void k_group_bounds(const int64_t *hb, int64_t G, int64_t nheavy, const int32_t *heavy_list,
                               const int64_t *it_first, int64_t n, int64_t *out) {
    for (int64_t g = threadIdx.x; g <= G; g += blockDim.x) {
        const int64_t h = hb[g];
        out[2 * g] = it_first[h];
        out[2 * g + 1] = g == 0 ? 0 : (g == G || h >= nheavy ? n : (int64_t)heavy_list[h]);
    }
}

// Position of every flagged column in the list of flagged columns.
__global__ void k_flag_list(int64_t n, const int32_t *flag, const int64_t *fpos, int32_t *list) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        if (flag[j]) list[fpos[j]] = (int32_t)j;
}

__global__ void k_sub_counts(int64_t nf, const int32_t *list, const void *Bcolptr, int p64, int64_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = list[i];
        cnt[i] = ld_ptr(Bcolptr, p64, j + 1) - ld_ptr(Bcolptr, p64, j);
    }
}

// B_f = B(:, list): warp per column copies rows and values unchanged.
__global__ void k_sub_copy(int64_t nf, const int32_t *list, const void *Bcolptr, int p64, const void *Brow,
                           int rowsz, const void *Bval, int valsz, const int64_t *fcolptr, void *frow, void *fval) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < nf; i += nw) {
        const int j = list[i];
        const int64_t s = ld_ptr(Bcolptr, p64, j), len = fcolptr[i + 1] - fcolptr[i], d = fcolptr[i];
        for (int64_t e = lane; e < len; e += 32) {
            if (rowsz == 8)
                ((long long *)frow)[d + e] = ((const long long *)Brow)[s + e];
            else
                ((int *)frow)[d + e] = ((const int *)Brow)[s + e];
            if (valsz == 8)
                ((long long *)fval)[d + e] = ((const long long *)Bval)[s + e];
            else
                ((int *)fval)[d + e] = ((const int *)Bval)[s + e];
        }
    }
}

__global__ void k_put_flagged_nnz(int64_t nf, const int32_t *list, const int64_t *fcolptr, int64_t *nnz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x)
        nnz[list[i]] = fcolptr[i + 1] - fcolptr[i];
}

// Canonical offset of every fused item inside its column: items of a column
// are generated in row order, so the offset is the sum of earlier counts.
__global__ void k_item_canon(int64_t h0, int64_t h1, const int64_t *it_first, const int32_t *item_cnt,
                             int64_t *canon) {
    for (int64_t h = h0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < h1; h += (int64_t)gridDim.x * blockDim.x) {
        int64_t off = 0;
        for (int64_t it = it_first[h]; it < it_first[h + 1]; it++) {
            canon[it] = off;
            off += item_cnt[it];
        }
    }
}

// Light columns [c0, c1) from the predicted layout to C (nothing when
// `broken` is set: their places in C are not known).
template <typename Acc, typename OutIdx>
__global__ void k_copy_light(int64_t c0, int64_t c1, const int8_t *bin_of, const int32_t *flag,
                             const int64_t *capoff, const int64_t *nnz, const int64_t *Ccolptr, const OutIdx *trow,
                             const Acc *tval, OutIdx *Crow, Acc *Cval, const int *broken) {
    if (broken && *(volatile const int *)broken) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = c0 + warp; j < c1; j += nw) {
        const int b = bin_of[j];
        if (b == kBinHeavy || b == kBinEmpty || flag[j]) continue;
        const int64_t s = capoff[j], d = Ccolptr[j], len = nnz[j];
        for (int64_t e = lane; e < len; e += 32) {
            Crow[d + e] = trow[s + e];
            Cval[d + e] = tval[s + e];
        }
    }
}

// Fused items [i0, i1) from the predicted layout to C (nothing when `broken`
// is set).
template <typename Acc, typename OutIdx>
__global__ void k_copy_items(int64_t i0, int64_t i1, const int32_t *it_rec0, const int32_t *rec_col,
                             const int32_t *flag, const int64_t *capoff, const int32_t *item_cnt,
                             const int64_t *item_pos, const int64_t *canon, const int64_t *Ccolptr,
                             const OutIdx *trow, const Acc *tval, OutIdx *Crow, Acc *Cval, const int *broken) {
    if (broken && *(volatile const int *)broken) return;
    for (int64_t it = i0 + blockIdx.x; it < i1; it += gridDim.x) {
        const int j = rec_col[it_rec0[it]];
        if (flag[j]) continue;
        const int64_t s = capoff[j] + item_pos[it], d = Ccolptr[j] + canon[it];
        for (int e = threadIdx.x; e < item_cnt[it]; e += blockDim.x) {
            Crow[d + e] = trow[s + e];
            Cval[d + e] = tval[s + e];
        }
    }
}

template <typename Acc, typename OutIdx>
__global__ void k_copy_flagged(int64_t nf, const int32_t *list, const int64_t *fcolptr, const OutIdx *frow,
                               const Acc *fval, const int64_t *Ccolptr, OutIdx *Crow, Acc *Cval) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < nf; i += nw) {
        const int64_t s = fcolptr[i], len = fcolptr[i + 1] - s, d = Ccolptr[list[i]];
        for (int64_t e = lane; e < len; e += 32) {
            Crow[d + e] = frow[s + e];
            Cval[d + e] = fval[s + e];
        }
    }
}

}  // namespace spg

using namespace spg;

// ------------------------------------------------------------- model API

static spg_status model_alloc(spg_model *m) {
    spg_status s = cuda_check(cudaMalloc(&m->d_params, sizeof(float) * kNP * 4 + sizeof(float) * 4), "model alloc");
    if (s) return s;
    m->d_m = m->d_params + kNP;
    m->d_v = m->d_m + kNP;
    m->d_grad = m->d_v + kNP;
    m->d_loss = m->d_grad + kNP;
    return cuda_check(cudaMemset(m->d_params, 0, sizeof(float) * kNP * 4 + sizeof(float) * 4), "model memset");
}

static uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Standard normal by the Box-Muller transform of two uniforms in (0, 1].
static double normal01(uint64_t &s) {
    const double u1 = ((double)(splitmix64(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

extern "C" spg_status spgemm_model_create(uint64_t seed, spg_model **out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return SPG_INVALID_ARGUMENT;
    }
    *out = nullptr;
    spg_model *m = new (std::nothrow) spg_model();
    if (!m) return SPG_OUT_OF_MEMORY;
    spg_status s = model_alloc(m);
    if (s) {
        delete m;
        return s;
    }
    // He-normal weights (std sqrt(2 / fan_in)), zero biases
    std::vector<float> h(kNP, 0.f);
    uint64_t st = seed;
    for (int i = 0; i < kH * kF; i++) h[kW1 + i] = (float)(normal01(st) * std::sqrt(2.0 / kF));
    for (int i = 0; i < kH * kH; i++) h[kW2 + i] = (float)(normal01(st) * std::sqrt(2.0 / kH));
    for (int i = 0; i < kH; i++) h[kW3 + i] = (float)(normal01(st) * std::sqrt(2.0 / kH));
    s = cuda_check(cudaMemcpy(m->d_params, h.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice), "model init");
    if (s) {
        cudaFree(m->d_params);
        delete m;
        return s;
    }
    *out = m;
    return SPG_OK;
}

extern "C" spg_status spgemm_model_destroy(spg_model *m) {
    if (!m) return SPG_OK;
    cudaFree(m->d_params);
    delete m;
    return SPG_OK;
}

extern "C" spg_status spgemm_model_set_params(spg_model *m, const float *host, int64_t count) {
    clear_error();
    if (!m || !host || count != kNP) {
        set_error("model parameters: need %d floats", kNP);
        return SPG_INVALID_ARGUMENT;
    }
    m->step = 0;
    spg_status s = cuda_check(cudaMemset(m->d_m, 0, sizeof(float) * kNP * 2), "model reset");
    if (s) return s;
    return cuda_check(cudaMemcpy(m->d_params, host, sizeof(float) * kNP, cudaMemcpyHostToDevice), "set params");
}

extern "C" spg_status spgemm_model_get_params(const spg_model *m, float *host, int64_t count) {
    clear_error();
    if (!m || !host || count != kNP) {
        set_error("model parameters: need %d floats", kNP);
        return SPG_INVALID_ARGUMENT;
    }
    return cuda_check(cudaMemcpy(host, m->d_params, sizeof(float) * kNP, cudaMemcpyDeviceToHost), "get params");
}

static int sm_count_now() {
    int dev = 0, sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    return sm > 0 ? sm : 1;
}

extern "C" spg_status spgemm_model_predict(const spg_model *m, const float *X, int64_t n, float *out, void *stream) {
    clear_error();
    if (!m || (n > 0 && (!X || !out)) || n < 0) {
        set_error("bad model prediction arguments");
        return SPG_INVALID_ARGUMENT;
    }
    if (n == 0) return SPG_OK;
    int g = grid_for(n, 256, sm_count_now() * 8);
    k_mlp_forward<<<g, 256, 0, (cudaStream_t)stream>>>(m->d_params, X, n, out);
    return cuda_check(cudaGetLastError(), "model predict");
}

static spg_status model_grad(spg_model *m, const float *X, const float *y, int64_t n0, int64_t n1, cudaStream_t st) {
    spg_status s = cuda_check(cudaMemsetAsync(m->d_grad, 0, sizeof(float) * (kNP + 1), st), "grad memset");
    if (s) return s;
    int g = grid_for(n1 - n0, 256, sm_count_now() * 4);
    k_mlp_grad<<<g, 256, 0, st>>>(m->d_params, X, y, n0, n1, 1.0f / (float)(n1 - n0), m->d_grad, m->d_loss);
    return cuda_check(cudaGetLastError(), "model gradient");
}

extern "C" spg_status spgemm_model_gradient(spg_model *m, const float *X, const float *y, int64_t n,
                                            float *grad_host, float *loss_host, void *stream) {
    clear_error();
    if (!m || !X || !y || n <= 0) {
        set_error("bad model gradient arguments");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    spg_status s = model_grad(m, X, y, 0, n, st);
    if (s) return s;
    std::vector<float> h(kNP + 1);
    s = cuda_check(cudaMemcpyAsync(h.data(), m->d_grad, sizeof(float) * (kNP + 1), cudaMemcpyDeviceToHost, st), "grad");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "grad");
    if (s) return s;
    if (grad_host) memcpy(grad_host, h.data(), sizeof(float) * kNP);
    if (loss_host) *loss_host = h[kNP] / (float)n;
    return SPG_OK;
}

extern "C" spg_status spgemm_model_train(spg_model *m, const float *X, const float *y, int64_t n, int32_t epochs,
                                         int32_t batch, float lr, void *stream, float *final_loss) {
    clear_error();
    if (!m || !X || !y || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f)) {
        set_error("bad training arguments");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; e++) {
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t b1e = b0 + batch < n ? b0 + batch : n;
            spg_status s = model_grad(m, X, y, b0, b1e, st);
            if (s) return s;
            m->step++;
            const float bc1 = 1.f - (float)std::pow((double)b1, (double)m->step);
            const float bc2 = 1.f - (float)std::pow((double)b2, (double)m->step);
            k_adam<<<(kNP + 255) / 256, 256, 0, st>>>(m->d_params, m->d_grad, m->d_m, m->d_v, kNP, lr, b1, b2, eps, bc1,
                                                      bc2);
            s = cuda_check(cudaGetLastError(), "adam");
            if (s) return s;
        }
    }
    if (final_loss) {
        float g = 0.f;
        spg_status s = spgemm_model_gradient(m, X, y, n, nullptr, &g, stream);
        if (s) return s;
        *final_loss = g;
    }
    return SPG_OK;
}

static const char kMagic[8] = {'S', 'P', 'G', 'M', 'L', 'P', '0', '1'};

extern "C" spg_status spgemm_model_save(const spg_model *m, const char *path) {
    clear_error();
    if (!m || !path) {
        set_error("bad save arguments");
        return SPG_INVALID_ARGUMENT;
    }
    std::vector<float> h(kNP);
    spg_status s = spgemm_model_get_params(m, h.data(), kNP);
    if (s) return s;
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return SPG_INVALID_ARGUMENT;
    }
    int32_t cnt = kNP;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&cnt, sizeof cnt, 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), kNP, f) == (size_t)kNP;
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return SPG_INVALID_ARGUMENT;
    }
    return SPG_OK;
}

extern "C" spg_status spgemm_model_load(const char *path, spg_model **out) {
    clear_error();
    if (!path || !out) {
        set_error("bad load arguments");
        return SPG_INVALID_ARGUMENT;
    }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return SPG_INVALID_ARGUMENT;
    }
    char magic[8];
    int32_t cnt = 0;
    std::vector<float> h(kNP);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&cnt, sizeof cnt, 1, f) == 1 &&
              cnt == kNP && fread(h.data(), sizeof(float), kNP, f) == (size_t)kNP;
    fclose(f);
    if (!ok) {
        set_error("%s is not an nnz-model file of %d parameters", path, kNP);
        return SPG_INVALID_INPUT;
    }
    spg_model *m = nullptr;
    spg_status s = spgemm_model_create(0, &m);
    if (s) return s;
    s = spgemm_model_set_params(m, h.data(), kNP);
    if (s) {
        spgemm_model_destroy(m);
        return s;
    }
    *out = m;
    return SPG_OK;
}

extern "C" spg_status spgemm_plan_features(const spg_plan *pc, float *X) {
    clear_error();
    if (!pc || (pc->n > 0 && !X)) {
        set_error("bad feature arguments");
        return SPG_INVALID_ARGUMENT;
    }
    spg_plan *p = const_cast<spg_plan *>(pc);
    if (p->n == 0) return SPG_OK;
    launch(p, k_features, grid_for(p->n, 256, p->sm_count * 8), 256, 0, p->n, p->flops, p->nnzb, p->maxa, X);
    return cuda_check(cudaGetLastError(), "features");
}

extern "C" spg_status spgemm_plan_labels(const spg_plan *pc, float *y) {
    clear_error();
    if (!pc || (pc->n > 0 && !y)) {
        set_error("bad label arguments");
        return SPG_INVALID_ARGUMENT;
    }
    spg_plan *p = const_cast<spg_plan *>(pc);
    if (!p->symbolic_done) {
        set_error("labels need the symbolic pass (spgemm_symbolic)");
        return SPG_INVALID_ARGUMENT;
    }
    if (p->n == 0) return SPG_OK;
    launch(p, k_labels, grid_for(p->n, 256, p->sm_count * 8), 256, 0, p->n, p->nnzcol, y);
    return cuda_check(cudaGetLastError(), "labels");
}

// --------------------------------------------------- the learned multiply

namespace spg {

template <int LOGS, int WARPS, typename Acc, typename OutIdx>
static spg_status launch_light_learned(spg_plan *p, const int32_t *list, int64_t cnt, const int64_t *capoff,
                                       const int64_t *cap, int64_t *nnz, int32_t *flag, unsigned long long *nflag,
                                       void *trow, void *tval) {
    size_t smem = sizeof(WarpSeg<Acc>) * WARPS + (sizeof(Acc) + sizeof(int)) * (size_t)WARPS * (1 << LOGS) +
                  sizeof(int) * 256 * (size_t)WARPS;
    auto kern = k_light_learned<LOGS, WARPS, Acc, OutIdx>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WARPS * 32, smem);
    if (occ < 1) occ = 1;
    launch(p, kern, grid_for(cnt, WARPS, p->sm_count * occ), WARPS * 32, smem, list, cnt, p->B.colptr,
           p->B.ptr_type == SPG_IDX_I64, p->Bq, (const Acc *)p->Bv, p->At_colptr, p->At_row, (const Acc *)p->At_val,
           capoff, cap, nnz, flag, nflag, (OutIdx *)trow, (Acc *)tval);
    return cuda_check(cudaGetLastError(), "learned light");
}

// Groups of heavy columns in the pipelined assembly (pinned read-back slots
// 24 .. 24 + 2 * (groups + 1) of the plan hold their boundaries).
constexpr int64_t kLearnedGroups = 8;
static_assert(24 + 2 * (kLearnedGroups + 1) <= 63, "pinned slots");

struct LearnedState {
    int64_t *cap = nullptr, *capoff = nullptr, *nnz_light = nullptr, *nnz = nullptr;
    int8_t *lbin = nullptr;
    int32_t *llist = nullptr;
    int64_t loff[kNumBins + 1] = {0};
    int32_t *flag = nullptr;
    unsigned long long *colfill = nullptr, *nflag = nullptr;
    void *trow = nullptr, *tval = nullptr;
    int64_t nitems = 0;
    int64_t *it_first = nullptr, *item_pos = nullptr, *canon = nullptr;
    int32_t *it_rec0 = nullptr, *it_nrec = nullptr, *item_cnt = nullptr;
};

template <typename Acc, typename OutIdx>
static spg_status learned_light(spg_plan *p, LearnedState &L) {
    spg_status s = SPG_OK;
    // timed as the light numeric group
    group_begin(p, kKNumLight);
    for (int bin = 1; bin <= kMaxLightBin && !s; bin++) {
        int64_t cnt = L.loff[bin + 1] - L.loff[bin];
        if (!cnt) continue;
        const int32_t *list = L.llist + L.loff[bin];
        switch (bin) {
            case 1: s = launch_light_learned<6, 8, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
            case 2: s = launch_light_learned<7, 8, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
            case 3: s = launch_light_learned<8, 8, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
            case 4: s = launch_light_learned<9, 8, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
            case 5: s = launch_light_learned<10, 4, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
            default: s = launch_light_learned<11, 4, Acc, OutIdx>(p, list, cnt, L.capoff, L.cap, L.nnz_light, L.flag, L.nflag, L.trow, L.tval); break;
        }
    }
    group_end(p, kKNumLight);
    return s;
}

// The fused heavy pass over items [i0, i1) (one persistent launch on the
// plan's stream, its own item counter).
template <typename Acc, typename OutIdx>
static spg_status learned_fused(spg_plan *p, LearnedState &L, int64_t i0, int64_t i1) {
    if (i1 <= i0) return SPG_OK;
    size_t smem = ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15) + sizeof(Acc) * kFusedRows +
                  sizeof(uint32_t) * (kFusedRows / 32) + sizeof(int) * (kFusedRows / 32 + 1);
    auto kern = k_fused_heavy<Acc, OutIdx>;
    spg_status s0 = cuda_check(cudaMemsetAsync(p->d_cnt + kCntFusedNextSlot, 0, sizeof(int64_t), p->st), "memset");
    if (s0) return s0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatch, smem);
    if (occ < 1) occ = 1;
    launch(p, kern, grid_for(i1 - i0, 1, p->sm_count * occ), kBatch, smem, i1 - i0, L.it_rec0, L.it_nrec, p->rec_col,
           p->rec_slab, p->B.colptr, p->B.ptr_type == SPG_IDX_I64, p->Bq, (const Acc *)p->Bv, p->At_colptr, p->At_row,
           (const Acc *)p->At_val, p->split, p->T, p->R, L.capoff, L.cap, L.colfill, L.flag, L.nflag, L.item_cnt,
           L.item_pos, (OutIdx *)L.trow, (Acc *)L.tval, (unsigned long long *)(p->d_cnt + kCntFusedNextSlot), i0);
    return cuda_check(cudaGetLastError(), "fused heavy");
}

// Launch on a given stream (counted with the plan's launches).
template <typename... KArgs, typename... Args>
static void launch_on(spg_plan *p, cudaStream_t st, void (*kern)(KArgs...), dim3 grid, dim3 block, Args &&...args) {
    p->launches++;
    kern<<<grid, block, 0, st>>>(static_cast<KArgs>(args)...);
}

// Pipelined assembly, group g of G: once the fused items of heavy columns
// [h0, h1) are done (event `done` on the plan's stream), the side stream
// counts the columns [c0, c1), places them after all earlier groups and
// copies their light columns and items into C, while the plan's stream goes
// on with the next group's items.
template <typename Acc, typename OutIdx>
static spg_status learned_place_group(spg_plan *p, LearnedState &L, cudaStream_t side, int g, int64_t c0, int64_t c1,
                                      int64_t h0, int64_t h1, int64_t i0, int64_t i1, int64_t *local, int64_t *carry,
                                      int *broken, spg_csc *C) {
    const int sm = p->sm_count;
    const int64_t len = c1 - c0;
    if (len > 0) {
        launch_on(p, side, k_learned_nnz_range, grid_for(len, 256, sm * 8), 256, c0, c1, (const int8_t *)p->bin_of,
                  (const unsigned long long *)L.colfill, (const int64_t *)L.nnz_light, (const int32_t *)L.flag, L.nnz,
                  (unsigned long long *)(p->d_cnt + kCntNnzCHeavySlot), broken);
        // the group's scan runs on the side stream too
        cudaStream_t keep = p->st;
        p->st = side;
        spg_status s = scan_exclusive_i64(p, L.nnz + c0, local, len);
        p->st = keep;
        if (s) return s;
    } else {
        const spg_status s = cuda_check(cudaMemsetAsync(local, 0, sizeof(int64_t), side), "memset");
        if (s) return s;
    }
    launch_on(p, side, k_add_carry, grid_for(len + 1, 256, sm * 8), 256, (const int64_t *)local, len,
              (const int64_t *)(carry + g), carry + g + 1, p->Ccolptr + c0);
    if (len > 0)
        launch_on(p, side, k_copy_light<Acc, OutIdx>, grid_for(len * 32, 256, sm * 4), 256, c0, c1,
                  (const int8_t *)p->bin_of, (const int32_t *)L.flag, (const int64_t *)L.capoff,
                  (const int64_t *)L.nnz, (const int64_t *)p->Ccolptr, (const OutIdx *)L.trow, (const Acc *)L.tval,
                  (OutIdx *)C->rowidx, (Acc *)C->vals, (const int *)broken);
    if (h1 > h0) {
        launch_on(p, side, k_item_canon, grid_for(h1 - h0, 256, sm * 8), 256, h0, h1, (const int64_t *)L.it_first,
                  (const int32_t *)L.item_cnt, L.canon);
        launch_on(p, side, k_copy_items<Acc, OutIdx>, grid_for(i1 - i0, 1, sm * 4), 256, i0, i1,
                  (const int32_t *)L.it_rec0, (const int32_t *)p->rec_col, (const int32_t *)L.flag,
                  (const int64_t *)L.capoff, (const int32_t *)L.item_cnt, (const int64_t *)L.item_pos,
                  (const int64_t *)L.canon, (const int64_t *)p->Ccolptr, (const OutIdx *)L.trow, (const Acc *)L.tval,
                  (OutIdx *)C->rowidx, (Acc *)C->vals, (const int *)broken);
    }
    return cuda_check(cudaGetLastError(), "learned group");
}

template <typename Acc, typename OutIdx>
static spg_status learned_assemble(spg_plan *p, LearnedState &L, int64_t nf, const int32_t *flist,
                                   const int64_t *fcolptr, const void *frow, const void *fval, spg_csc *C) {
    const int sm = p->sm_count;
    launch(p, k_copy_light<Acc, OutIdx>, grid_for(p->n * 32, 256, sm * 16), 256, 0, (int64_t)0, p->n,
           (const int8_t *)p->bin_of, (const int32_t *)L.flag, (const int64_t *)L.capoff, (const int64_t *)L.nnz,
           (const int64_t *)p->Ccolptr, (const OutIdx *)L.trow, (const Acc *)L.tval, (OutIdx *)C->rowidx,
           (Acc *)C->vals, (const int *)nullptr);
    if (L.nitems > 0) {
        launch(p, k_item_canon, grid_for(p->nheavy, 256, sm * 8), 256, 0, (int64_t)0, p->nheavy,
               (const int64_t *)L.it_first, (const int32_t *)L.item_cnt, L.canon);
        launch(p, k_copy_items<Acc, OutIdx>, grid_for(L.nitems, 1, sm * 8), 256, 0, (int64_t)0, L.nitems,
               (const int32_t *)L.it_rec0, (const int32_t *)p->rec_col, (const int32_t *)L.flag,
               (const int64_t *)L.capoff, (const int32_t *)L.item_cnt, (const int64_t *)L.item_pos,
               (const int64_t *)L.canon, (const int64_t *)p->Ccolptr, (const OutIdx *)L.trow, (const Acc *)L.tval,
               (OutIdx *)C->rowidx, (Acc *)C->vals, (const int *)nullptr);
    }
    if (nf > 0)
        launch(p, k_copy_flagged<Acc, OutIdx>, grid_for(nf * 32, 256, sm * 16), 256, 0, nf, flist, fcolptr,
               (const OutIdx *)frow, (const Acc *)fval, p->Ccolptr, (OutIdx *)C->rowidx, (Acc *)C->vals);
    return cuda_check(cudaGetLastError(), "assemble");
}

static void *alloc_out(const spg_options *opt, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (opt->alloc) return opt->alloc(bytes, opt->alloc_ctx, opt->stream);
    void *q = nullptr;
    if (cudaMallocAsync(&q, bytes, (cudaStream_t)opt->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

static void free_out(const spg_options *opt, void *ptr, size_t bytes) {
    if (!ptr) return;
    if (opt->free)
        opt->free(ptr, bytes, opt->alloc_ctx, opt->stream);
    else if (!opt->alloc)
        cudaFreeAsync(ptr, (cudaStream_t)opt->stream);
}

#define LTRY(x)                        \
    do {                               \
        spg_status _s = (x);           \
        if (_s != SPG_OK) return _s;   \
    } while (0)

static spg_status learned_run(spg_plan *p, const spg_options *opt, spg_csc *C, int64_t *nrecomputed) {
    cudaStream_t st = p->st;
    const int64_t n = p->n;
    const int sm = p->sm_count;
    const spg_model *model = (const spg_model *)opt->model;
    const float slack = opt->learned_slack > 0 ? (float)opt->learned_slack : 1.25f;
    LearnedState L;
    cudaEventRecord(p->ev[4], st);

    // 1. predict nnz per column and turn it into capacities
    float *X = (float *)ws_alloc(p, sizeof(float) * 4 * (size_t)(n + 1));
    float *pred = (float *)ws_alloc(p, sizeof(float) * (size_t)(n + 1));
    L.cap = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    L.capoff = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    L.nnz_light = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    L.nnz = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
    L.lbin = (int8_t *)ws_alloc(p, (size_t)(n + 1));
    L.llist = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    L.flag = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    L.colfill = (unsigned long long *)ws_alloc(p, sizeof(unsigned long long) * (size_t)(n + 1));
    L.nflag = (unsigned long long *)ws_alloc(p, sizeof(unsigned long long));
    if (!X || !pred || !L.cap || !L.capoff || !L.nnz_light || !L.nnz || !L.lbin || !L.llist || !L.flag ||
        !L.colfill || !L.nflag)
        return SPG_OUT_OF_MEMORY;
    LTRY(cuda_check(cudaMemsetAsync(L.flag, 0, sizeof(int32_t) * (size_t)(n + 1), st), "memset"));
    LTRY(cuda_check(cudaMemsetAsync(L.colfill, 0, sizeof(unsigned long long) * (size_t)(n + 1), st), "memset"));
    LTRY(cuda_check(cudaMemsetAsync(L.nflag, 0, sizeof(unsigned long long), st), "memset"));
    LTRY(cuda_check(cudaMemsetAsync(L.nnz_light, 0, sizeof(int64_t) * (size_t)(n + 1), st), "memset"));
    if (n > 0) {
        LTRY(spgemm_plan_features(p, X));
        launch(p, k_mlp_forward, grid_for(n, 256, sm * 8), 256, 0, (const float *)model->d_params, (const float *)X, n,
               pred);
        launch(p, k_capacity, grid_for(n, 256, sm * 8), 256, 0, n, (const float *)pred, p->bin_of, p->flops,
               p->win_lo, p->win_hi, slack, p->light_max, L.cap, L.lbin);
        LTRY(cuda_check(cudaGetLastError(), "capacity"));
    }
    LTRY(scan_exclusive_i64(p, L.cap, L.capoff, n));
    LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 16, L.capoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "cap"));
    LTRY(cuda_check(cudaStreamSynchronize(st), "cap"));
    const int64_t totcap = p->h_pinned[16];
    p->stats.learned_capacity = totcap;
    if (n > 0) LTRY(bin_columns(p, L.lbin, L.llist, L.loff));  // uses pinned slots 0..8
    const size_t idxsz = p->out_idx64 ? 8 : 4;
    L.trow = ws_alloc(p, idxsz * (size_t)(totcap + 1));
    L.tval = ws_alloc(p, 8 * (size_t)(totcap + 1));
    if (!L.trow || !L.tval) return SPG_OUT_OF_MEMORY;

    // 2. fused heavy items: groups of kFusedRows / R consecutive records
    if (p->nrec > 0) {
        const int per = kFusedRows / p->R > 0 ? kFusedRows / p->R : 1;
        int64_t *icnt = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        L.it_first = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
        if (!icnt || !L.it_first) return SPG_OUT_OF_MEMORY;
        launch(p, k_count_groups, grid_for(p->nheavy, 256, sm * 8), 256, 0, p->nheavy, (const int64_t *)p->rec_first,
               per, icnt);
        LTRY(scan_exclusive_i64(p, icnt, L.it_first, p->nheavy));
        LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 17, L.it_first + p->nheavy, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "items"));
        LTRY(cuda_check(cudaStreamSynchronize(st), "items"));
        L.nitems = p->h_pinned[17];
        L.it_rec0 = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(L.nitems + 1));
        L.it_nrec = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(L.nitems + 1));
        L.item_cnt = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(L.nitems + 1));
        L.item_pos = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(L.nitems + 1));
        L.canon = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(L.nitems + 1));
        if (!L.it_rec0 || !L.it_nrec || !L.item_cnt || !L.item_pos || !L.canon) return SPG_OUT_OF_MEMORY;
        launch(p, k_sym_items, grid_for(p->nheavy, 256, sm * 8), 256, 0, p->nheavy, per, (const int64_t *)p->rec_first,
               (const int64_t *)L.it_first, L.it_rec0, L.it_nrec);
    }

    // 3. the learned numeric work: light columns, then the fused items in G
    // groups of heavy columns; as soon as a group's items are done, a side
    // stream counts its columns, places them after the earlier groups and
    // copies them into C (allocated at the predicted capacity) while the next
    // group computes.  A column that overflowed its room stops the placement
    // (its count is known only after the recompute): C is then assembled
    // after the recompute instead, from the predicted layout.
    const size_t cp_bytes = sizeof(int64_t) * (size_t)(n + 1);
    const size_t ri_bytes = idxsz * (size_t)(totcap + 1), va_bytes = 8 * (size_t)(totcap + 1);
    void *cp_opt = alloc_out(opt, cp_bytes);
    void *ri_opt = alloc_out(opt, ri_bytes);
    void *va_opt = alloc_out(opt, va_bytes);
    auto free_opt = [&]() {
        free_out(opt, cp_opt, cp_bytes);
        free_out(opt, ri_opt, ri_bytes);
        free_out(opt, va_opt, va_bytes);
        cp_opt = ri_opt = va_opt = nullptr;
    };
    if (!cp_opt || !ri_opt || !va_opt) {
        free_opt();
        set_error("allocation of C at the predicted capacity (%lld entries) failed", (long long)totcap);
        return SPG_OUT_OF_MEMORY;
    }
    spg_csc Copt{};
    Copt.rowidx = ri_opt;
    Copt.vals = va_opt;
    const int64_t G = p->nrec > 0 ? std::min<int64_t>(kLearnedGroups, p->nheavy) : 0;
    // group boundaries: heavy columns hb[g], items ib[g], columns cb[g]
    std::vector<int64_t> hb(G + 1), ib(G + 1, 0), cb(G + 2, 0);
    int64_t *carry = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(G + 2));
    int64_t *local = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 2));
    int *broken = (int *)ws_alloc(p, sizeof(int));
    int64_t *bnd = (int64_t *)ws_alloc(p, sizeof(int64_t) * 2 * (size_t)(G + 1));
    if (!carry || !local || !broken || !bnd) {
        free_opt();
        return SPG_OUT_OF_MEMORY;
    }
    spg_status s = SPG_OK;
    if (G > 0) {
        for (int64_t g = 0; g <= G; g++) hb[g] = g * p->nheavy / G;
        int64_t *hb_d = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(G + 1));
        if (!hb_d) s = SPG_OUT_OF_MEMORY;
        if (!s) s = cuda_check(cudaMemcpyAsync(hb_d, hb.data(), sizeof(int64_t) * (size_t)(G + 1),
                                               cudaMemcpyHostToDevice, st), "groups");
        if (!s) {
            launch(p, k_group_bounds, 1, 64, 0, (const int64_t *)hb_d, G, p->nheavy,
                   (const int32_t *)(p->binlist + p->bin_off[kBinHeavy]), (const int64_t *)L.it_first, n, bnd);
            s = cuda_check(cudaMemcpyAsync(p->h_pinned + 24, bnd, sizeof(int64_t) * 2 * (size_t)(G + 1),
                                           cudaMemcpyDeviceToHost, st), "groups");
        }
        if (!s) s = cuda_check(cudaStreamSynchronize(st), "groups");
        for (int64_t g = 0; g <= G && !s; g++) {
            ib[g] = p->h_pinned[24 + 2 * g];
            cb[g] = p->h_pinned[24 + 2 * g + 1];
        }
    } else {
        cb[0] = 0;
        cb[1] = n;
    }
    if (!s) s = cuda_check(cudaMemsetAsync(carry, 0, sizeof(int64_t), st), "memset");
    if (!s) s = cuda_check(cudaMemsetAsync(broken, 0, sizeof(int), st), "memset");
    if (!s) s = cuda_check(cudaMemsetAsync(p->d_cnt + kCntNnzCHeavySlot, 0, sizeof(int64_t), st), "memset");
    if (!s) s = p->acc_f64 ? (p->out_idx64 ? learned_light<double, long long>(p, L) : learned_light<double, int>(p, L))
                           : (p->out_idx64 ? learned_light<long long, long long>(p, L)
                                           : learned_light<long long, int>(p, L));
    cudaStream_t side = nullptr;
    cudaEvent_t ev = nullptr;
    if (!s) s = cuda_check(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking), "stream");
    if (!s) s = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    if (!s && G > 0) group_begin(p, kKNumHeavy);
    const int64_t ngroups = G > 0 ? G : 1;
    for (int64_t g = 0; g < ngroups && !s; g++) {
        if (G > 0)
            s = p->acc_f64 ? (p->out_idx64 ? learned_fused<double, long long>(p, L, ib[g], ib[g + 1])
                                           : learned_fused<double, int>(p, L, ib[g], ib[g + 1]))
                           : (p->out_idx64 ? learned_fused<long long, long long>(p, L, ib[g], ib[g + 1])
                                           : learned_fused<long long, int>(p, L, ib[g], ib[g + 1]));
        if (!s) s = cuda_check(cudaEventRecord(ev, st), "event");
        if (!s) s = cuda_check(cudaStreamWaitEvent(side, ev, 0), "event");
        const int64_t h0 = G > 0 ? hb[g] : 0, h1 = G > 0 ? hb[g + 1] : 0;
        const int64_t i0 = G > 0 ? ib[g] : 0, i1 = G > 0 ? ib[g + 1] : 0;
        if (!s)
            s = p->acc_f64
                    ? (p->out_idx64 ? learned_place_group<double, long long>(p, L, side, (int)g, cb[g], cb[g + 1], h0, h1,
                                                                             i0, i1, local, carry, broken, &Copt)
                                    : learned_place_group<double, int>(p, L, side, (int)g, cb[g], cb[g + 1], h0, h1,
                                                                       i0, i1, local, carry, broken, &Copt))
                    : (p->out_idx64 ? learned_place_group<long long, long long>(p, L, side, (int)g, cb[g], cb[g + 1],
                                                                                h0, h1, i0, i1, local, carry, broken,
                                                                                &Copt)
                                    : learned_place_group<long long, int>(p, L, side, (int)g, cb[g], cb[g + 1], h0,
                                                                          h1, i0, i1, local, carry, broken, &Copt));
    }
    if (!s && G > 0) group_end(p, kKNumHeavy);
    // join the side stream (also after an error, before anything is freed)
    if (side) {
        if (ev && cudaEventRecord(ev, side) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
    }
    if (ev) cudaEventDestroy(ev);
    if (s) {
        free_opt();
        return s;
    }
    LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 18, L.nflag, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "nflag"));
    LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 20, carry + ngroups, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
                    "nnz"));
    LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 21, p->d_cnt + kCntNnzCHeavySlot, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st), "nnz"));
    LTRY(cuda_check(cudaStreamSynchronize(st), "nflag"));
    const int64_t nf = p->h_pinned[18];
    *nrecomputed = nf;
    if (nf == 0) {
        // every column was placed: C is the pipelined one (its arrays hold
        // the predicted capacity, of which the first nnz(C) entries are used)
        p->nnzC = p->h_pinned[20];
        p->stats.nnzC = p->nnzC;
        p->stats.nnzC_heavy = p->h_pinned[21];
        s = cuda_check(cudaMemcpyAsync(cp_opt, p->Ccolptr, cp_bytes, cudaMemcpyDeviceToDevice, st), "colptr");
        cudaEventRecord(p->ev[5], st);
        if (!s) s = read_dev_err(p, "learned");
        if (s) {
            free_opt();
            return s;
        }
        spg_csc out{};
        out.nrows = p->m;
        out.ncols = n;
        out.nnz = p->nnzC;
        out.ptr_type = SPG_IDX_I64;
        out.idx_type = p->out_idx64 ? SPG_IDX_I64 : SPG_IDX_I32;
        out.val_type = p->acc_f64 ? SPG_VAL_F64 : SPG_VAL_I64;
        out.colptr = cp_opt;
        out.rowidx = ri_opt;
        out.vals = va_opt;
        *C = out;
        return SPG_OK;
    }
    free_opt();
    LTRY(cuda_check(cudaMemsetAsync(p->d_cnt + kCntNnzCHeavySlot, 0, sizeof(int64_t), st), "memset"));
    if (n > 0)
        launch(p, k_learned_nnz, grid_for(n, 256, sm * 8), 256, 0, n, p->bin_of, (const unsigned long long *)L.colfill,
               (const int64_t *)L.nnz_light, (const int32_t *)L.flag, L.nnz,
               (unsigned long long *)(p->d_cnt + kCntNnzCHeavySlot));

    // 4. recompute the overflowed columns through the exact path
    int32_t *flist = nullptr;
    int64_t *fcolptr = nullptr;
    void *frow = nullptr, *fval = nullptr;
    spg_plan *sub = nullptr;
    if (nf > 0) {
        int64_t *fpos = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(n + 1));
        flist = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(nf + 1));
        int64_t *bcnt = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(nf + 1));
        int64_t *bcolptr = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(nf + 1));
        if (!fpos || !flist || !bcnt || !bcolptr) return SPG_OUT_OF_MEMORY;
        LTRY(scan_exclusive_i32(p, L.flag, fpos, n));
        launch(p, k_flag_list, grid_for(n, 256, sm * 8), 256, 0, n, (const int32_t *)L.flag, (const int64_t *)fpos, flist);
        launch(p, k_sub_counts, grid_for(nf, 256, sm * 8), 256, 0, nf, (const int32_t *)flist, p->B.colptr,
               p->B.ptr_type == SPG_IDX_I64, bcnt);
        LTRY(scan_exclusive_i64(p, bcnt, bcolptr, nf));
        LTRY(cuda_check(cudaMemcpyAsync(p->h_pinned + 19, bcolptr + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "sub"));
        LTRY(cuda_check(cudaStreamSynchronize(st), "sub"));
        const int64_t fnnz = p->h_pinned[19];
        const int rowsz = p->B.idx_type == SPG_IDX_I64 ? 8 : 4;
        const int valsz = p->B.val_type == SPG_VAL_I32 ? 4 : 8;
        void *brow = ws_alloc(p, (size_t)rowsz * (size_t)(fnnz + 1));
        void *bval = ws_alloc(p, (size_t)valsz * (size_t)(fnnz + 1));
        if (!brow || !bval) return SPG_OUT_OF_MEMORY;
        launch(p, k_sub_copy, grid_for(nf * 32, 256, sm * 16), 256, 0, nf, (const int32_t *)flist, p->B.colptr,
               p->B.ptr_type == SPG_IDX_I64, p->B.rowidx, rowsz, p->B.vals, valsz, (const int64_t *)bcolptr, brow, bval);
        LTRY(cuda_check(cudaGetLastError(), "sub copy"));
        spg_csc Bf = p->B;
        Bf.ncols = nf;
        Bf.nnz = fnnz;
        Bf.ptr_type = SPG_IDX_I64;
        Bf.colptr = bcolptr;
        Bf.rowidx = brow;
        Bf.vals = bval;
        spg_options so = *opt;
        so.P = 1;
        so.sizing = SPG_SIZING_EXACT;
        so.validate = 0;
        so.stream = (void *)st;
        LTRY(spgemm_plan(&p->A, &Bf, &so, &sub));
        int64_t fnz = 0;
        s = spgemm_symbolic(sub, nullptr, &fnz);
        if (!s) {
            fcolptr = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(nf + 1));
            frow = ws_alloc(p, idxsz * (size_t)(fnz + 1));
            fval = ws_alloc(p, 8 * (size_t)(fnz + 1));
            if (!fcolptr || !frow || !fval) s = SPG_OUT_OF_MEMORY;
        }
        if (!s) {
            spg_csc Cf{};
            Cf.colptr = fcolptr;
            Cf.rowidx = frow;
            Cf.vals = fval;
            s = spgemm_numeric(sub, &Cf);
        }
        if (!s) s = read_dev_err(sub, "recompute");
        if (s) {
            spgemm_plan_destroy(sub);
            return s;
        }
        launch(p, k_put_flagged_nnz, grid_for(nf, 256, sm * 8), 256, 0, nf, (const int32_t *)flist,
               (const int64_t *)fcolptr, L.nnz);
    }

    // 5. canonical column pointers, then C
    s = scan_exclusive_i64(p, L.nnz, p->Ccolptr, n);
    if (!s) s = cuda_check(cudaMemcpyAsync(p->h_pinned + 20, p->Ccolptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "nnz");
    if (!s) s = cuda_check(cudaMemcpyAsync(p->h_pinned + 21, p->d_cnt + kCntNnzCHeavySlot, sizeof(int64_t),
                                           cudaMemcpyDeviceToHost, st), "nnz");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "nnz");
    if (s) {
        if (sub) spgemm_plan_destroy(sub);
        return s;
    }
    p->nnzC = p->h_pinned[20];
    p->stats.nnzC = p->nnzC;
    p->stats.nnzC_heavy = p->h_pinned[21];
    void *cp = alloc_out(opt, sizeof(int64_t) * (size_t)(n + 1));
    void *ri = alloc_out(opt, idxsz * (size_t)p->nnzC);
    void *va = alloc_out(opt, 8 * (size_t)p->nnzC);
    if (!cp || !ri || !va) {
        free_out(opt, cp, sizeof(int64_t) * (size_t)(n + 1));
        free_out(opt, ri, idxsz * (size_t)p->nnzC);
        free_out(opt, va, 8 * (size_t)p->nnzC);
        if (sub) spgemm_plan_destroy(sub);
        set_error("allocation of C (%lld nonzeros) failed", (long long)p->nnzC);
        return SPG_OUT_OF_MEMORY;
    }
    spg_csc out{};
    out.nrows = p->m;
    out.ncols = n;
    out.nnz = p->nnzC;
    out.ptr_type = SPG_IDX_I64;
    out.idx_type = p->out_idx64 ? SPG_IDX_I64 : SPG_IDX_I32;
    out.val_type = p->acc_f64 ? SPG_VAL_F64 : SPG_VAL_I64;
    out.colptr = cp;
    out.rowidx = ri;
    out.vals = va;
    s = cuda_check(cudaMemcpyAsync(cp, p->Ccolptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, st), "colptr");
    if (!s) {
        if (p->acc_f64)
            s = p->out_idx64 ? learned_assemble<double, long long>(p, L, nf, flist, fcolptr, frow, fval, &out)
                             : learned_assemble<double, int>(p, L, nf, flist, fcolptr, frow, fval, &out);
        else
            s = p->out_idx64 ? learned_assemble<long long, long long>(p, L, nf, flist, fcolptr, frow, fval, &out)
                             : learned_assemble<long long, int>(p, L, nf, flist, fcolptr, frow, fval, &out);
    }
    cudaEventRecord(p->ev[5], st);
    if (!s) s = read_dev_err(p, "learned");
    if (sub) spgemm_plan_destroy(sub);
    if (s) {
        free_out(opt, cp, sizeof(int64_t) * (size_t)(n + 1));
        free_out(opt, ri, idxsz * (size_t)p->nnzC);
        free_out(opt, va, 8 * (size_t)p->nnzC);
        return s;
    }
    *C = out;
    return SPG_OK;
}

spg_status multiply_learned(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C) {
    if (!opt->model) {
        set_error("learned sizing needs options.model (an spg_model)");
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->slab_rows > kFusedRows) {
        set_error("learned sizing needs slab_rows <= %d", kFusedRows);
        return SPG_UNSUPPORTED;
    }
    spg_plan *p = nullptr;
    spg_status s = spgemm_plan(A, B, opt, &p);
    if (s) return s;
    int64_t nrec = 0;
    s = learned_run(p, opt, C, &nrec);
    std::string keep = last_error_str();
    p->stats.recomputed_columns = nrec;
    if (!s) {
        spg_stats st{};
        if (spgemm_plan_stats(p, &st) == SPG_OK) remember_multiply_stats(st);
    }
    spgemm_plan_destroy(p);
    if (s) {
        set_error("%s", keep.c_str());
        return s;
    }
    return nrec > 0 ? SPG_OVERFLOW_RECOMPUTED : SPG_OK;
}

}  // namespace spg
