// Symbolic pass: nnz(C(:,j)) for every output column, then the column
// pointers of C (Algorithm 1, local multiply, first of its two passes).
//   light bins: one warp per column, open-addressing table of 2^LOGS row ids
//               in shared memory, sized >= 2 x min(flops_j, row window)
//   heavy bin:  one CTA per (column, row slab of R rows): a shared bitmap of
//               the slab; the bitmap is kept for the numeric pass, which uses
//               it to place every product at its final rank without sorting
#include "spg_internal.cuh"

namespace spg {

template <int LOGS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_sym_light(const int32_t *__restrict__ list, int64_t ncols, const void *Bcolptr, int p64,
                const int32_t *__restrict__ Bq, const int64_t *__restrict__ At_colptr,
                const int32_t *__restrict__ At_row, int64_t *__restrict__ nnzcol, int *err) {
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

__global__ void __launch_bounds__(256)
    k_sym_heavy(int64_t nitems, const int32_t *__restrict__ item_col, const int32_t *__restrict__ item_slab,
                const void *Bcolptr, int p64, const int32_t *__restrict__ Bq,
                const int64_t *__restrict__ At_colptr, const int32_t *__restrict__ At_row,
                const int32_t *__restrict__ split, int T, int R, uint32_t *__restrict__ hbits,
                int32_t *__restrict__ item_cnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RW = R >> 5;
    WarpSeg<long long> *segs = (WarpSeg<long long> *)smem_raw;
    uint32_t *bits = (uint32_t *)(segs + (blockDim.x >> 5));
    __shared__ int red[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int j = item_col[it], t = item_slab[it];
        for (int w = threadIdx.x; w < RW; w += blockDim.x) bits[w] = 0;
        __syncthreads();
        const int64_t p0 = ld_ptr(Bcolptr, p64, j), p1 = ld_ptr(Bcolptr, p64, j + 1);
        const int64_t wbase = (int64_t)t * RW;
        for (int64_t c0 = p0 + (int64_t)wid * 32; c0 < p1; c0 += (int64_t)nw * 32) {
            warp_products<false, long long>(
                c0, min(c0 + 32, p1), lane, segs[wid], At_row, (const long long *)nullptr,
                [&](int64_t p, long long &st, int &len, long long &) {
                    int q = Bq[p];
                    if (q >= 0) {
                        const int32_t *sp = split + (int64_t)q * (T + 1) + t;
                        int a = sp[0], b = sp[1];
                        st = At_colptr[q] + a;
                        len = b - a;
                    }
                },
                [&](int r, long long) { atomicOr(bits + ((r >> 5) - wbase), 1u << (r & 31)); });
        }
        __syncthreads();
        int c = 0;
        uint32_t *dst = hbits + it * RW;
        for (int w = threadIdx.x; w < RW; w += blockDim.x) {
            uint32_t x = bits[w];
            dst[w] = x;
            c += __popc(x);
        }
        c = warp_sum_i(c);
        if (lane == 0) red[wid] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < nw; w++) s += red[w];
            item_cnt[it] = s;
        }
        __syncthreads();
    }
}

// Per heavy column: place each slab after the ones above it, total = nnz_j.
__global__ void k_heavy_offsets(const int32_t *list, int64_t nheavy, const int64_t *item_first,
                                const int32_t *item_cnt, int64_t *item_off, int64_t *nnzcol,
                                long long *nnzc_heavy) {
    long long sum = 0;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x) {
        int64_t off = 0;
        for (int64_t it = item_first[h]; it < item_first[h + 1]; it++) {
            item_off[it] = off;
            off += item_cnt[it];
        }
        nnzcol[list[h]] = off;
        sum += off;
    }
    sum = warp_sum_ll(sum);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd((unsigned long long *)nnzc_heavy, (unsigned long long)sum);
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
           p->At_row, p->nnzcol, p->d_err);
    return cuda_check(cudaGetLastError(), "symbolic light");
}

spg_status run_symbolic(spg_plan *p) {
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
    if (p->nitems > 0) {
        const int threads = 256;
        size_t smem = sizeof(WarpSeg<long long>) * (threads / 32) + sizeof(uint32_t) * (size_t)(p->R / 32);
        cudaFuncSetAttribute(k_sym_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sym_heavy, threads, smem);
        if (occ < 1) occ = 1;
        int g = grid_for(p->nitems, 1, p->sm_count * occ);
        group_begin(p, kKSymHeavy);
        launch(p, k_sym_heavy, g, threads, smem, p->nitems, p->item_col, p->item_slab, p->B.colptr,
               p->B.ptr_type == SPG_IDX_I64, p->Bq, p->At_colptr, p->At_row, p->split, p->T, p->R, p->hbits,
               p->item_cnt);
        group_end(p, kKSymHeavy);
        launch(p, k_heavy_offsets, grid_for(p->nheavy, 256, p->sm_count * 8), 256, 0,
               p->binlist + p->bin_off[kBinHeavy], p->nheavy, p->item_first, p->item_cnt, p->item_off, p->nnzcol,
               (long long *)(p->d_cnt + kCntNnzCHeavySlot));
        s = cuda_check(cudaGetLastError(), "symbolic heavy");
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
