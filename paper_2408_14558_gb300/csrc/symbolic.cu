// Symbolic pass: nnz(C(:,j)) for every output column, then the column
// pointers of C (Algorithm 1, local multiply, first of its two passes).
//   light bins: one warp per column, open-addressing table of 2^LOGS row ids
//               in shared memory, sized >= 2 x min(flops_j, row window)
//   heavy bin:  one CTA per item of up to 262,144 rows (base slabs) of a column:
//               a shared bitmap of the item's rows; the per-slab bitmaps are
//               kept for the numeric pass, which uses them to place every
//               product at its final rank without sorting
#include "cta_products.cuh"
#include "spg_internal.cuh"

namespace spg {

template <int LOGS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_sym_light(const int32_t *__restrict__ list, int64_t ncols, const void *Bcolptr, int p64,
                const int32_t *__restrict__ Bq, const int64_t *__restrict__ At_colptr,
                const int32_t *__restrict__ At_row, int64_t *__restrict__ nnzcol, int *err, OutMask mask) {
    constexpr int S = 1 << LOGS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSeg<long long> *segs = (WarpSeg<long long> *)smem_raw;
    int *keys_all = (int *)(segs + WARPS);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *tab = keys_all + wid * S;
    for (int64_t c = (int64_t)blockIdx.x * WARPS + wid; c < ncols; c += (int64_t)gridDim.x * WARPS) {
        const int j = list[c];
        for (int s = lane; s < S; s += 32) tab[s] = kEmptyKey;
        __syncwarp();
        const int64_t p0 = ld_ptr(Bcolptr, p64, j), p1 = ld_ptr(Bcolptr, p64, j + 1);
        int cnt = 0;
        bool full = false;
        warp_products<false, long long>(
            p0, p1, lane, segs[wid], At_row, (const long long *)nullptr,
            [&](int64_t p, long long &st, int &len, long long &) {
                int q = Bq[p];
                if (q >= 0) {
                    st = At_colptr[q];
                    len = (int)(At_colptr[q + 1] - st);
                }
            },
            [&](int r, long long) {
                if (mask.bits && !mask_keeps(mask, j, r)) return;
                bool fresh;
                if (hash_insert(tab, LOGS, r, &fresh) < 0) full = true;
                cnt += fresh ? 1 : 0;
            });
        cnt = warp_sum_i(cnt);
        if (__any_sync(kFull, full) && lane == 0) atomicOr(err, kDevErrInternal);
        if (lane == 0) nnzcol[j] = cnt;
        __syncwarp();
    }
}

// Hub columns of A: the columns with at least `T` entries get a row bitmap
// of their own (Wa words, padded to a multiple of 4), so that the heavy
// symbolic pass ORs a hub's words into an item's bitmap instead of walking
// the hub's entries one product at a time (the bitmap it builds is the same).
// In skewed graphs a few hundred such columns carry most of the products.
__global__ void k_deg_hist(const void *Acp, int ap64, int64_t k, unsigned long long *hist) {
    __shared__ unsigned int h[64];
    if (threadIdx.x < 64) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = ld_ptr(Acp, ap64, c + 1) - ld_ptr(Acp, ap64, c);
        if (d > 0) atomicAdd(h + (63 - __clzll((unsigned long long)d)), 1u);
    }
    __syncthreads();
    if (threadIdx.x < 64 && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

__global__ void k_hub_index(const void *Acp, int ap64, int64_t k, int64_t T, int32_t *hubidx, int *count,
                            int32_t *hubcol) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = ld_ptr(Acp, ap64, c + 1) - ld_ptr(Acp, ap64, c);
        int h = -1;
        if (d >= T) {
            h = atomicAdd(count, 1);
            hubcol[h] = (int32_t)c;
        }
        hubidx[c] = h;
    }
}

// CTA per hub (column hubcol[h] of A): its Wa words built in shared memory
// with one atomicOr per entry (rows outside [0, m) are skipped: validation
// reports them), then stored whole (coalesced).
__global__ void __launch_bounds__(256)
    k_hub_bits(const void *Acp, int ap64, const void *Arow, int ai64, int64_t m, const int32_t *hubcol, int64_t Wa,
               uint32_t *hubbits) {
    extern __shared__ uint32_t hw[];
    const int64_t c = hubcol[blockIdx.x];
    for (int64_t w = threadIdx.x; w < Wa; w += blockDim.x) hw[w] = 0;
    __syncthreads();
    const int64_t e0 = ld_ptr(Acp, ap64, c), e1 = ld_ptr(Acp, ap64, c + 1);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t r = ld_ptr(Arow, ai64, e);
        if ((uint64_t)r < (uint64_t)m && (r >> 5) < Wa) atomicOr(hw + (r >> 5), 1u << (r & 31));
    }
    __syncthreads();
    uint32_t *dst = hubbits + (int64_t)blockIdx.x * Wa;
    for (int64_t w = threadIdx.x; w < Wa; w += blockDim.x) dst[w] = hw[w];
}

// Hub entries one symbolic item may OR instead of walking (the rest walk).
constexpr int kSymMaxHubs = 512;

// One CTA per symbolic item: records [r0, r0 + nr) of one heavy column, i.e.
// base slabs t0 .. t0 + nr - 1.  Every product sets its row's bit; then the
// bitmap of each record and its population count are stored.
__global__ void SPG_SYM_BOUNDS
    k_sym_heavy(int64_t nitems, const int32_t *__restrict__ sym_rec0, const int32_t *__restrict__ sym_nrec,
                const int32_t *__restrict__ rec_col, const int32_t *__restrict__ rec_slab, const void *Bcolptr,
                int p64, const int32_t *__restrict__ Bq, const int64_t *__restrict__ At_colptr,
                const int32_t *__restrict__ At_row, const int32_t *__restrict__ split, int T, int R,
                uint32_t *__restrict__ hbits, int32_t *__restrict__ rec_cnt, unsigned long long *next,
                const int64_t *__restrict__ flops, const int32_t *__restrict__ win_lo,
                const int32_t *__restrict__ win_hi, OutMask mask, int64_t mwords_used,
                const int32_t *__restrict__ dtilde, const int32_t *__restrict__ hubidx,
                const uint4 *__restrict__ hubbits, int64_t Wa4, int hub_min_len) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RW = R >> 5;
    CtaBatch<long long> &sb = *(CtaBatch<long long> *)smem_raw;
    // 16-byte aligned: the hub words are ORed in as uint4
    uint32_t *bits = (uint32_t *)(smem_raw + ((sizeof(CtaBatch<long long>) + 15) & ~(size_t)15));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ long long claim;
    __shared__ int hubs[kSymMaxHubs];
    __shared__ int nhub;
    if (threadIdx.x == 0) nhub = 0;
    for (int64_t it = cta_claim(next, &claim); it < nitems; it = cta_claim(next, &claim)) {
        const int r0 = sym_rec0[it], nr = sym_nrec[it];
        const int j = rec_col[r0], t0 = rec_slab[r0];
        const int nwords = nr * RW;
        const int64_t p0 = ld_ptr(Bcolptr, p64, j), p1 = ld_ptr(Bcolptr, p64, j + 1);
        // a segment of a hub column of A at least hub_min_len long, and
        // long enough that ORing the item's words costs less than walking it
        // (8 x its length >= the item's words), is not walked: the hub's
        // bitmap words are ORed in after the walk
        auto seg = [&](int64_t p, long long &st, int &len, long long &) {
            int q = Bq[p];
            if (q >= 0) {
                const int32_t *sp = split + (int64_t)q * (T + 1);
                int a = sp[t0], b = sp[t0 + nr];
                st = At_colptr[q] + a;
                len = b - a;
                if (hubbits && len >= hub_min_len && 8 * (int64_t)len >= nwords) {
                    const int h = hubidx[dtilde[q]];
                    if (h >= 0) {
                        const int pos = atomicAdd(&nhub, 1);
                        if (pos < kSymMaxHubs) {
                            hubs[pos] = h;
                            len = 0;
                        }
                    }
                }
            }
        };
        const SegReg<long long> first = cta_first_seg<long long>(p0, p1, seg);
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0;
        __syncthreads();
        const int wbase = t0 * RW;
        // many products per row of the column's window: most bits get set
        // again and again, so read before the atomic
        const bool dense = flops[j] > 4 * (int64_t)(win_hi[j] - win_lo[j] + 1);
        cta_products<false, SPG_SYM_UNROLL, long long>(
            p0, p1, sb, At_row, (const long long *)nullptr, first, seg,
            [&](int r, long long) {
                if (dense)
                    set_bit_shared(bits + ((r >> 5) - wbase), 1u << (r & 31));
                else
                    atomicOr(bits + ((r >> 5) - wbase), 1u << (r & 31));
            });
        // cta_products ends with a barrier: the walked products are marked;
        // now the hub segments, each thread ORing the words it owns (the rows
        // of the item are words [t0 * RW, t0 * RW + nwords) of a hub bitmap;
        // both are multiples of 4, so whole uint4 words)
        const int nh = min(nhub, kSymMaxHubs);
        if (nh > 0) {
            uint4 *b4 = (uint4 *)bits;
            const int64_t base4 = (int64_t)t0 * RW / 4;
            for (int w4 = threadIdx.x; w4 < nwords / 4; w4 += blockDim.x) {
                uint4 y = b4[w4];
                for (int hh = 0; hh < nh; hh++) {
                    const uint4 x = __ldg(hubbits + (int64_t)hubs[hh] * Wa4 + base4 + w4);
                    y.x |= x.x;
                    y.y |= x.y;
                    y.z |= x.z;
                    y.w |= x.w;
                }
                b4[w4] = y;
            }
            __syncthreads();
        }
        if (mask.bits) {
            // keep the rows the output mask admits (words past the last row of
            // C hold no products and have no mask words)
            const uint32_t *mw = mask.bits + (int64_t)j * mask.words;
            for (int w = threadIdx.x; w < nwords; w += blockDim.x)
                bits[w] = wbase + w < mwords_used ? bits[w] & (__ldg(mw + wbase + w) ^ mask.flip) : 0u;
            __syncthreads();
        }
        uint32_t *dst = hbits + (int64_t)r0 * RW;
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) st_stream(dst + w, bits[w]);
        for (int rr = wid; rr < nr; rr += nw) {
            int c = 0;
            for (int w = lane; w < RW; w += 32) c += __popc(bits[rr * RW + w]);
            c = warp_sum_i(c);
            if (lane == 0) rec_cnt[r0 + rr] = c;
        }
        __syncthreads();
        // every thread has read nhub; the next claim's barrier publishes the reset
        if (threadIdx.x == 0) nhub = 0;
    }
}

// Per heavy column: offset of each record inside the column, nnz_j, and the
// number of numeric items (greedy groups of consecutive records holding at
// most `cap` entries and at most maxrec records).
__device__ __forceinline__ int num_groups(const int32_t *rec_cnt, int64_t r0, int64_t r1, int cap, int maxrec,
                                          int32_t *g_rec0, int32_t *g_nrec) {
    int groups = 0, cur = 0, nin = 0;
    int64_t start = r0;
    for (int64_t r = r0; r < r1; r++) {
        int c = rec_cnt[r];
        if (nin > 0 && (cur + c > cap || nin == maxrec)) {
            if (g_rec0) {
                g_rec0[groups] = (int32_t)start;
                g_nrec[groups] = nin;
            }
            groups++;
            cur = 0;
            nin = 0;
            start = r;
        }
        cur += c;
        nin++;
    }
    if (nin > 0) {
        if (g_rec0) {
            g_rec0[groups] = (int32_t)start;
            g_nrec[groups] = nin;
        }
        groups++;
    }
    return groups;
}

__global__ void k_heavy_offsets(const int32_t *list, int64_t nheavy, const int64_t *rec_first,
                                const int32_t *rec_cnt, int64_t *rec_off, int64_t *nnzcol, int cap, int maxrec,
                                int64_t *nnum, long long *nnzc_heavy) {
    long long sum = 0;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x) {
        int64_t off = 0;
        for (int64_t r = rec_first[h]; r < rec_first[h + 1]; r++) {
            rec_off[r] = off;
            off += rec_cnt[r];
        }
        nnzcol[list[h]] = off;
        nnum[h] = num_groups(rec_cnt, rec_first[h], rec_first[h + 1], cap, maxrec, nullptr, nullptr);
        sum += off;
    }
    sum = warp_sum_ll(sum);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd((unsigned long long *)nnzc_heavy, (unsigned long long)sum);
}

__global__ void k_num_items(int64_t nheavy, const int64_t *rec_first, const int32_t *rec_cnt, int cap, int maxrec,
                            const int64_t *num_first, int32_t *num_rec0, int32_t *num_nrec) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x)
        num_groups(rec_cnt, rec_first[h], rec_first[h + 1], cap, maxrec, num_rec0 + num_first[h],
                   num_nrec + num_first[h]);
}

template <int LOGS, int WARPS>
static spg_status launch_sym_light(spg_plan *p, const int32_t *list, int64_t cnt) {
    size_t smem = sizeof(WarpSeg<long long>) * WARPS + sizeof(int) * (size_t)WARPS * (1 << LOGS);
    auto kern = k_sym_light<LOGS, WARPS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WARPS * 32, smem);
    if (occ < 1) occ = 1;
    int g = grid_for(cnt, WARPS, p->sm_count * occ);
    launch(p, kern, g, WARPS * 32, smem, list, cnt, p->B.colptr, p->B.ptr_type == SPG_IDX_I64, p->Bq, p->At_colptr,
           p->At_row, p->nnzcol, p->d_err, p->omask);
    return cuda_check(cudaGetLastError(), "symbolic light");
}

// Hub columns of A for the heavy symbolic pass: the threshold is the smallest
// power of two >= kHubMinDeg whose hubs' bitmaps fit kHubBytes (one
// histogram read-back).  No hubs (also when one hub's bitmap, rows / 8
// bytes, exceeds kHubMaxSmem of shared memory): *hubbits stays NULL.
constexpr int64_t kHubMinDeg = 1024;
constexpr size_t kHubBytes = size_t(64) << 20;
constexpr size_t kHubMaxSmem = size_t(192) << 10;  // bitmap words of one hub (rows / 8 bytes) at most

static spg_status build_hubs(spg_plan *p, int32_t **hubidx, uint4 **hubbits, int64_t *Wa4) {
    *hubidx = nullptr;
    *hubbits = nullptr;
    *Wa4 = 0;
    const int64_t k = p->k;
    if (k == 0) return SPG_OK;
    cudaStream_t st = p->st;
    const int ap64 = p->A.ptr_type == SPG_IDX_I64;
    // words of a hub bitmap: every base slab of the heavy items (a multiple of 4)
    const int64_t Wa = (int64_t)p->T * (p->R / 32);
    // a hub's bitmap is built in one CTA's shared memory
    if ((size_t)Wa * sizeof(uint32_t) > kHubMaxSmem) return SPG_OK;
    unsigned long long *hist = (unsigned long long *)ws_alloc(p, sizeof(unsigned long long) * 64);
    int *count = (int *)ws_alloc(p, sizeof(int) * 4);
    if (!hist || !count) return SPG_OUT_OF_MEMORY;
    spg_status s = cuda_check(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 64, st), "memset");
    if (s) return s;
    launch(p, k_deg_hist, grid_for(k, 256, p->sm_count * 4), 256, 0, p->A.colptr, ap64, k, hist);
    s = cuda_check(cudaMemcpyAsync(p->h_pinned + 16, hist, sizeof(int64_t) * 32, cudaMemcpyDeviceToHost, st),
                   "hub histogram");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "hub histogram");
    if (s) return s;
    int lg = 0;
    while ((int64_t(1) << lg) < kHubMinDeg) lg++;
    int64_t nh = 0;
    for (; lg < 32; lg++) {
        nh = 0;
        for (int b = lg; b < 32; b++) nh += p->h_pinned[16 + b];
        if ((size_t)nh * (size_t)Wa * sizeof(uint32_t) <= kHubBytes) break;
    }
    if (nh == 0 || lg >= 32) return SPG_OK;
    int32_t *idx = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)k);
    int32_t *col = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)nh);
    uint32_t *bits = (uint32_t *)ws_alloc(p, sizeof(uint32_t) * (size_t)(nh * Wa));
    if (!idx || !col || !bits) return SPG_OUT_OF_MEMORY;
    s = cuda_check(cudaMemsetAsync(count, 0, sizeof(int), st), "memset");
    if (s) return s;
    launch(p, k_hub_index, grid_for(k, 256, p->sm_count * 4), 256, 0, p->A.colptr, ap64, k, int64_t(1) << lg, idx,
           count, col);
    const size_t smem = sizeof(uint32_t) * (size_t)Wa;
    s = cuda_check(cudaFuncSetAttribute(k_hub_bits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "hub bitmaps");
    if (s) return s;
    launch(p, k_hub_bits, (unsigned)nh, 256, smem, p->A.colptr, ap64, p->A.rowidx, p->A.idx_type == SPG_IDX_I64,
           p->m, (const int32_t *)col, Wa, bits);
    s = cuda_check(cudaGetLastError(), "hub bitmaps");
    if (s) return s;
    *hubidx = idx;
    *hubbits = (uint4 *)bits;
    *Wa4 = Wa / 4;
    return SPG_OK;
}

static spg_status symbolic_heavy(spg_plan *p) {
    spg::PhaseRange nvtx_range("symbolic: heavy columns");
    cudaStream_t st = p->st;
    const int threads = kBatch;
    size_t smem = ((sizeof(CtaBatch<long long>) + 15) & ~(size_t)15) + sizeof(uint32_t) * (size_t)kSymMaxWords;
    cudaFuncSetAttribute(k_sym_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sym_heavy, threads, smem);
    if (occ < 1) occ = 1;
    int g = grid_for(p->nsym, 1, p->sm_count * occ);
    int32_t *hubidx = nullptr;
    uint4 *hubbits = nullptr;
    int64_t Wa4 = 0;
    spg_status s0 = build_hubs(p, &hubidx, &hubbits, &Wa4);
    if (s0) return s0;
    s0 = cuda_check(cudaMemsetAsync(p->d_cnt + kCntSymNextSlot, 0, sizeof(int64_t), st), "memset");
    if (s0) return s0;
    group_begin(p, kKSymHeavy);
    launch(p, k_sym_heavy, g, threads, smem, p->nsym, p->sym_rec0, p->sym_nrec, p->rec_col, p->rec_slab,
           p->B.colptr, p->B.ptr_type == SPG_IDX_I64, p->Bq, p->At_colptr, p->At_row, p->split, p->T, p->R,
           p->hbits, p->rec_cnt, (unsigned long long *)(p->d_cnt + kCntSymNextSlot), p->flops, p->win_lo,
           p->win_hi, p->omask, (int64_t)((p->m + 31) / 32), (const int32_t *)p->dtilde, (const int32_t *)hubidx,
           (const uint4 *)hubbits, Wa4, 0);
    group_end(p, kKSymHeavy);
    int64_t *nnum = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
    int64_t *num_first = (int64_t *)ws_alloc(p, sizeof(int64_t) * (size_t)(p->nheavy + 1));
    if (!nnum || !num_first) return SPG_OUT_OF_MEMORY;
    const int gh = grid_for(p->nheavy, 256, p->sm_count * 8);
    launch(p, k_heavy_offsets, gh, 256, 0, p->binlist + p->bin_off[kBinHeavy], p->nheavy, p->rec_first, p->rec_cnt,
           p->rec_off, p->nnzcol, p->num_cap, p->num_max_recs, nnum, (long long *)(p->d_cnt + kCntNnzCHeavySlot));
    spg_status s = scan_exclusive_i64(p, nnum, num_first, p->nheavy);
    if (s) return s;
    s = cuda_check(cudaMemcpyAsync(p->h_pinned + 2, num_first + p->nheavy, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
                   "numeric items");
    if (s) return s;
    s = cuda_check(cudaStreamSynchronize(st), "numeric items");
    if (s) return s;
    p->nnum = p->h_pinned[2];
    p->num_rec0 = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->nnum + 1));
    p->num_nrec = (int32_t *)ws_alloc(p, sizeof(int32_t) * (size_t)(p->nnum + 1));
    if (!p->num_rec0 || !p->num_nrec) return SPG_OUT_OF_MEMORY;
    launch(p, k_num_items, gh, 256, 0, p->nheavy, p->rec_first, p->rec_cnt, p->num_cap, p->num_max_recs, num_first,
           p->num_rec0,
           p->num_nrec);
    return cuda_check(cudaGetLastError(), "symbolic heavy");
}

spg_status run_symbolic(spg_plan *p) {
    spg::PhaseRange nvtx_range("symbolic");
    cudaStream_t st = p->st;
    const int64_t n = p->n;
    spg_status s = cuda_check(cudaMemsetAsync(p->nnzcol, 0, sizeof(int64_t) * (size_t)(n + 1), st), "memset");
    if (s) return s;
    s = cuda_check(cudaMemsetAsync(p->d_cnt + kCntNnzCHeavySlot, 0, sizeof(int64_t), st), "memset");
    if (s) return s;
    cudaEventRecord(p->ev[2], st);
    if (p->bin_off[kMaxLightBin + 1] > p->bin_off[1]) group_begin(p, kKSymLight);
    for (int bin = 1; bin <= kMaxLightBin && !s; bin++) {
        int64_t cnt = p->bin_off[bin + 1] - p->bin_off[bin];
        if (cnt == 0) continue;
        const int32_t *list = p->binlist + p->bin_off[bin];
        switch (bin) {
            case 1: s = launch_sym_light<6, 8>(p, list, cnt); break;
            case 2: s = launch_sym_light<7, 8>(p, list, cnt); break;
            case 3: s = launch_sym_light<8, 8>(p, list, cnt); break;
            case 4: s = launch_sym_light<9, 8>(p, list, cnt); break;
            case 5: s = launch_sym_light<10, 8>(p, list, cnt); break;
            default: s = launch_sym_light<11, 8>(p, list, cnt); break;
        }
    }
    if (p->bin_off[kMaxLightBin + 1] > p->bin_off[1]) group_end(p, kKSymLight);
    if (s) return s;
    if (p->nrec > 0) {
        s = symbolic_heavy(p);
        if (s) return s;
    }
    s = scan_exclusive_i64(p, p->nnzcol, p->Ccolptr, n);
    if (s) return s;
    cudaEventRecord(p->ev[3], st);
    s = cuda_check(cudaMemcpyAsync(p->h_pinned, p->Ccolptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "nnz readback");
    if (s) return s;
    s = cuda_check(cudaMemcpyAsync(p->h_pinned + 1, p->d_cnt + kCntNnzCHeavySlot, sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, st), "nnz readback");
    if (s) return s;
    s = read_dev_err(p, "symbolic");
    if (s) return s;
    p->nnzC = p->h_pinned[0];
    p->stats.nnzC = p->nnzC;
    p->stats.nnzC_heavy = p->h_pinned[1];
    float ms = 0;
    cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]);
    p->stats.ms_symbolic = ms;
    p->symbolic_done = true;
    return SPG_OK;
}

}  // namespace spg
