// Numeric pass: the rows and values of C (Algorithm 1, local multiply
// C_i = A~_i * B_i, Gustavson column by column), written at the column
// pointers produced by the symbolic pass.
//   light bins: one warp per column, shared open-addressing table of
//               (row, value) sized >= 2 x nnz_j; afterwards the occupied slots
//               are compacted in place and sorted by row (warp radix sort)
//   heavy bin:  one CTA per (column, row slab): the symbolic bitmap of the
//               slab gives every present row its rank, products accumulate at
//               acc[rank] in shared memory, and the slab is written out in row
//               order with no sort
#include "block_ops.cuh"
#include "cta_products.cuh"
#include "spg_internal.cuh"

namespace spg {

template <int LOGS, int WARPS, typename Acc, typename OutIdx>
__global__ void __launch_bounds__(WARPS * 32)
    k_num_light(const int32_t *__restrict__ list, int64_t ncols, const void *Bcolptr, int p64,
                const int32_t *__restrict__ Bq, const Acc *__restrict__ Bv, const int64_t *__restrict__ At_colptr,
                const int32_t *__restrict__ At_row, const Acc *__restrict__ At_val,
                const int64_t *__restrict__ Ccolptr, OutIdx *__restrict__ Crow, Acc *__restrict__ Cval, int *err,
                OutMask mask) {
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
                if (mask.bits && !mask_keeps(mask, j, r)) return;
                bool fresh;
                int slot = hash_insert(keys, LOGS, r, &fresh);
                if (slot < 0)
                    full = true;
                else
                    atomic_add_acc(vals + slot, v);
            });
        __syncwarp();
        // compact the occupied slots to the front: a write never reaches a slot
        // of a later, still unread chunk because the count so far is <= c0
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
        const int64_t base = Ccolptr[j];
        if ((int64_t)nout != Ccolptr[j + 1] - base) {
            full = true;
        } else {
            warp_sort_pairs<Acc>(keys, vals, nout, S, hist, lane);
            for (int s = lane; s < nout; s += 32) {
                st_stream(Crow + base + s, (OutIdx)keys[s]);
                st_stream(Cval + base + s, vals[s]);
            }
        }
        if (__any_sync(kFull, full) && lane == 0) atomicOr(err, kDevErrInternal);
        __syncwarp();
    }
}

// Everything a numeric item needs before its first product, in one record.
struct NumItem {
    int32_t j, t0, nr, cnt, r0, pad;
    long long cbase, p0, p1;  // first entry of the item in C; B(:, j) = [p0, p1)
};

__global__ void k_num_headers(int64_t nitems, const int32_t *__restrict__ num_rec0,
                              const int32_t *__restrict__ num_nrec, const int32_t *__restrict__ rec_col,
                              const int32_t *__restrict__ rec_slab, const int32_t *__restrict__ rec_cnt,
                              const int64_t *__restrict__ rec_off, const void *Bcolptr, int p64,
                              const int64_t *__restrict__ Ccolptr, NumItem *__restrict__ items) {
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (int64_t)gridDim.x * blockDim.x) {
        NumItem h;
        h.r0 = num_rec0[it];
        h.nr = num_nrec[it];
        h.j = rec_col[h.r0];
        h.t0 = rec_slab[h.r0];
        int cnt = 0;
        for (int rr = 0; rr < h.nr; rr++) cnt += rec_cnt[h.r0 + rr];
        h.cnt = cnt;
        h.pad = 0;
        h.cbase = Ccolptr[h.j] + rec_off[h.r0];
        h.p0 = ld_ptr(Bcolptr, p64, h.j);
        h.p1 = ld_ptr(Bcolptr, p64, h.j + 1);
        items[it] = h;
    }
}

// One CTA per numeric item: records [r0, r0 + nr) of one heavy column (base
// slabs t0 .. t0 + nr - 1) holding cnt <= cap entries of C.  The symbolic
// bitmaps of the records give every present row its rank (pre[word] + popc of
// the lower bits); products accumulate at acc[rank]; the item is then written
// at its final place in C, values and rows each as one coalesced run.  Thread
// 0 claims the next item when the current one starts and fetches its header
// while the current one is written out.  MASKED: the bitmaps hold only the
// rows an output mask admits, and a product whose row is absent is dropped.
template <typename Acc, typename OutIdx, bool MASKED>
__global__ void __launch_bounds__(kBatch, SPG_NUM_MINB)
    k_num_heavy(int64_t nitems, const NumItem *__restrict__ items, const uint32_t *__restrict__ hbits,
                const int32_t *__restrict__ Bq, const Acc *__restrict__ Bv, const int64_t *__restrict__ At_colptr,
                const int32_t *__restrict__ At_row, const Acc *__restrict__ At_val,
                const int32_t *__restrict__ split, int T, int R, int cap, OutIdx *__restrict__ Crow,
                Acc *__restrict__ Cval, int *err, unsigned long long *next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RW = R >> 5;
    CtaBatch<Acc> &sb = *(CtaBatch<Acc> *)smem_raw;
    unsigned char *acc_raw = smem_raw + ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15);
    const HeavyAcc<Acc> acc(acc_raw, cap + 1);
    uint2 *bp = (uint2 *)(acc_raw + HeavyAcc<Acc>::bytes_per_slot * (size_t)(cap + 1));  // (bitmap word, prefix)
    __shared__ int ctot[kNumMaxWords / 32];
    __shared__ int bad_sh;
    __shared__ long long claim;
    __shared__ NumItem hdr;
    const int tid = threadIdx.x;
    if (tid == 0) {
        bad_sh = 0;
        const long long it = (long long)atomicAdd(next, 1ull);
        claim = it;
        if (it < nitems) hdr = items[it];
    }
    __syncthreads();
    for (;;) {
        const int64_t it = claim;
        if (it >= nitems) break;
        const NumItem h = hdr;
        unsigned long long nxt = 0;
        if (tid == 0) nxt = atomicAdd(next, 1ull);
        const int t0 = h.t0, nr = h.nr;
        const int nwords = nr * RW;
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
        const SegReg<Acc> first = cta_first_seg<Acc>(h.p0, h.p1, seg);
        const uint32_t *src = hbits + (int64_t)h.r0 * RW;
        const int cnt = cta_load_scan_bitmap(src, bp, nwords, ctot);
        NumItem nh;
        if (cnt == h.cnt && cnt <= cap) {
            // (the first barrier of cta_products orders the zeroing before
            // every product)
            for (int i = tid; i < cnt; i += blockDim.x) acc.zero(i);
            const int wbase = t0 * RW;
            bool miss = false;
            cta_products<true, SPG_NUM_UNROLL, Acc>(
                h.p0, h.p1, sb, At_row, At_val, first, seg,
                [&](int r, Acc v) {
                    const uint2 x = bp[(r >> 5) - wbase];
                    const uint32_t sh = r & 31;
#if SPG_CHECK_MEMBERSHIP
                    // a row missing from the symbolic bitmap (never expected) goes
                    // to the dump slot acc[cap] and is reported
                    const bool hit = (x.x >> sh) & 1u;
                    miss |= !hit && !MASKED;  // a masked product is absent by design
                    acc.add(hit ? (int)(x.y + __popc(x.x & ((1u << sh) - 1u))) : cap, v);
#else
                    if constexpr (MASKED) {
                        if ((x.x >> sh) & 1u) acc.add((int)(x.y + __popc(x.x & ((1u << sh) - 1u))), v);
                    } else {
                        // the rank of a present row; an absent one would still
                        // land inside [0, cnt] (never outside the accumulator)
                        acc.add((int)(x.y + __popc(x.x & ((1u << sh) - 1u))), v);
                    }
#endif
                });
            if (miss) bad_sh = 1;
            if (tid == 0 && (long long)nxt < nitems) nh = items[nxt];
            // cta_products ends with a barrier: acc is complete
            for (int i = tid; i < cnt; i += blockDim.x) st_stream(Cval + h.cbase + i, acc.get(i));
            __syncthreads();
            // the row ids go to shared memory by rank first (over the consumed
            // values: cnt ints fit in the first cnt slots), then to C in one
            // coalesced run
            int32_t *srow = acc.scratch32();
            for (int w = tid; w < nwords; w += blockDim.x) {
                uint32_t word = bp[w].x;
                int pos = (int)bp[w].y;
                while (word) {
                    int bb = __ffs(word) - 1;
                    srow[pos++] = w * 32 + bb;
                    word &= word - 1u;
                }
            }
            __syncthreads();
            const int64_t rbase = (int64_t)t0 * R;
            for (int i = tid; i < cnt; i += blockDim.x) st_stream(Crow + h.cbase + i, (OutIdx)(rbase + srow[i]));
        } else {
            // the item's room in C was sized from the record counts: never
            // write past it
            if (tid == 0) {
                bad_sh = 1;
                if ((long long)nxt < nitems) nh = items[nxt];
            }
        }
        if (tid == 0) {
            claim = (long long)nxt;
            if ((long long)nxt < nitems) hdr = nh;
        }
        __syncthreads();
    }
    if (tid == 0 && bad_sh) atomicOr(err, kDevErrInternal);
}

__global__ void k_rebin_numeric(const int8_t *bin_sym, const int64_t *nnzcol, int64_t n, int8_t *bin_num) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int b = bin_sym[j];
        if (b != kBinHeavy && b != kBinEmpty) {
            long long U = nnzcol[j];
            if (U <= 0) {
                b = kBinEmpty;
            } else {
                long long S = 64;
                b = 1;
                while (S < 2 * U) {
                    S <<= 1;
                    b++;
                }
            }
        }
        bin_num[j] = (int8_t)b;
    }
}

template <int LOGS, int WARPS, typename Acc, typename OutIdx>
static spg_status launch_num_light(spg_plan *p, const int32_t *list, int64_t cnt, spg_csc *C) {
    size_t smem = sizeof(WarpSeg<Acc>) * WARPS + (sizeof(Acc) + sizeof(int)) * (size_t)WARPS * (1 << LOGS) +
                  sizeof(int) * 256 * (size_t)WARPS;
    auto kern = k_num_light<LOGS, WARPS, Acc, OutIdx>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WARPS * 32, smem);
    if (occ < 1) occ = 1;
    int g = grid_for(cnt, WARPS, p->sm_count * occ);
    launch(p, kern, g, WARPS * 32, smem, list, cnt, p->B.colptr, p->B.ptr_type == SPG_IDX_I64, p->Bq,
                                         (const Acc *)p->Bv, p->At_colptr, p->At_row, (const Acc *)p->At_val,
                                         p->Ccolptr, (OutIdx *)C->rowidx, (Acc *)C->vals, p->d_err, p->omask);
    return cuda_check(cudaGetLastError(), "numeric light");
}

template <typename Acc, typename OutIdx>
static spg_status numeric_typed(spg_plan *p, spg_csc *C) {
    spg_status s = SPG_OK;
    const bool any_light = p->nbin_off[kMaxLightBin + 1] > p->nbin_off[1];
    if (any_light) group_begin(p, kKNumLight);
    for (int bin = 1; bin <= kMaxLightBin && !s; bin++) {
        int64_t cnt = p->nbin_off[bin + 1] - p->nbin_off[bin];
        if (cnt == 0) continue;
        const int32_t *list = p->nbinlist + p->nbin_off[bin];
        switch (bin) {
            case 1: s = launch_num_light<6, 8, Acc, OutIdx>(p, list, cnt, C); break;
            case 2: s = launch_num_light<7, 8, Acc, OutIdx>(p, list, cnt, C); break;
            case 3: s = launch_num_light<8, 8, Acc, OutIdx>(p, list, cnt, C); break;
            case 4: s = launch_num_light<9, 8, Acc, OutIdx>(p, list, cnt, C); break;
            case 5: s = launch_num_light<10, 4, Acc, OutIdx>(p, list, cnt, C); break;
            default: s = launch_num_light<11, 4, Acc, OutIdx>(p, list, cnt, C); break;
        }
    }
    if (any_light) group_end(p, kKNumLight);
    if (s) return s;
    if (p->nnum > 0) {
        const int threads = kBatch;
        size_t smem = ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15) + sizeof(Acc) * (size_t)(p->num_cap + 1) +
                      sizeof(uint2) * (size_t)kNumMaxWords;
        auto kern = p->omask.bits ? k_num_heavy<Acc, OutIdx, true> : k_num_heavy<Acc, OutIdx, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        if (occ < 1) occ = 1;
        int g = grid_for(p->nnum, 1, p->sm_count * occ);
        if (!p->num_items) p->num_items = ws_alloc(p, sizeof(NumItem) * (size_t)p->nnum);
        NumItem *items = (NumItem *)p->num_items;
        if (!items) return SPG_OUT_OF_MEMORY;
        s = cuda_check(cudaMemsetAsync(p->d_cnt + kCntNumNextSlot, 0, sizeof(int64_t), p->st), "memset");
        if (s) return s;
        group_begin(p, kKNumHeavy);
        launch(p, k_num_headers, grid_for(p->nnum, 256, p->sm_count * 8), 256, 0, p->nnum, p->num_rec0, p->num_nrec,
               p->rec_col, p->rec_slab, p->rec_cnt, p->rec_off, p->B.colptr, p->B.ptr_type == SPG_IDX_I64,
               p->Ccolptr, items);
        launch(p, kern, g, threads, smem, p->nnum, items, p->hbits, p->Bq, (const Acc *)p->Bv, p->At_colptr,
               p->At_row, (const Acc *)p->At_val, p->split, p->T, p->R, p->num_cap, (OutIdx *)C->rowidx,
               (Acc *)C->vals, p->d_err, (unsigned long long *)(p->d_cnt + kCntNumNextSlot));
        group_end(p, kKNumHeavy);
        s = cuda_check(cudaGetLastError(), "numeric heavy");
    }
    return s;
}

// The light columns' numeric bins (by their exact counts), once per plan: the
// only step of the numeric pass that reads back to the host (the bin sizes).
spg_status prepare_numeric(spg_plan *p) {
    const int64_t n = p->n;
    if (p->nbinlist) return SPG_OK;
    int8_t *bn = (int8_t *)ws_alloc(p, (size_t)(n + 1));
    p->nbinlist = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(n + 1));
    if (!bn || !p->nbinlist) return SPG_OUT_OF_MEMORY;
    if (n > 0) {
        launch(p, k_rebin_numeric, grid_for(n, 256, p->sm_count * 8), 256, 0, p->bin_of, p->nnzcol, n, bn);
        spg_status s = cuda_check(cudaGetLastError(), "rebin");
        if (s) return s;
        s = bin_columns(p, bn, p->nbinlist, p->nbin_off);
        if (s) return s;
    }
    return SPG_OK;
}

spg_status run_numeric(spg_plan *p, spg_csc *C) {
    spg::PhaseRange nvtx_range("numeric");
    cudaStream_t st = p->st;
    const int64_t n = p->n;
    spg_status s0 = prepare_numeric(p);
    if (s0) return s0;
    if (C->colptr && C->colptr != (void *)p->Ccolptr) {
        spg_status s = cuda_check(cudaMemcpyAsync(C->colptr, p->Ccolptr, sizeof(int64_t) * (size_t)(n + 1),
                                                  cudaMemcpyDeviceToDevice, st),
                                  "colptr copy");
        if (s) return s;
    }
    cudaEventRecord(p->ev[4], st);
    spg_status s;
    if (p->acc_f64)
        s = p->out_idx64 ? numeric_typed<double, long long>(p, C) : numeric_typed<double, int>(p, C);
    else
        s = p->out_idx64 ? numeric_typed<long long, long long>(p, C) : numeric_typed<long long, int>(p, C);
    cudaEventRecord(p->ev[5], st);
    return s;
}

}  // namespace spg
