// Batched execution of many independent products C_i = A_i * B_i in one
// persistent kernel launch (captured once in a CUDA graph), driven by a device
// work queue.  An extension beyond the paper: its local multiply (Algorithm 1,
// last step, Gustavson column by column) run for hundreds of uneven problems at
// once; each instance is one column block (P = 1), so A_i is read in place
// (gathering the single block would copy A_i whole).
//
// Queue: every instance is cut into tasks of `task_cols` consecutive columns.
// The queue holds all symbolic tasks, then all numeric tasks; a warp takes one
// task at a time (a global atomic counter).
//   symbolic task: per column, a warp hash of row ids gives nnz(C_i(:,j)); the
//     warp that finishes an instance's last symbolic task scans its counts into
//     the instance's column pointers and publishes a ready flag;
//   numeric task: waits (bounded) for the instance's flag, then per column a
//     warp hash of (row, value), compaction, bitonic sort, and the column is
//     written at its place.
// Because all symbolic tasks precede all numeric ones in the queue, a warp
// that waits only waits for warps that already hold their tasks.  The wait is
// bounded: after `timeout_ns` it records SPG_TIMEOUT and the kernel returns.
// Output: one pool for all instances; instance i owns [out_base_i,
// out_base_i + bound_i) where bound_i = sum_j min(flops_j, m_i) (from the
// bounds pass at creation), of which it uses its nnz.
// Heavy columns (bound above the largest warp table, 1024) are CTA tasks of
// two more kernels in the same graph: one before the class kernels counts
// each such column with a shared row bitmap (kept in a global scratch) and
// one after them writes it in row windows of up to kHeavyCap entries, the
// rows' ranks taken from the stored bitmap.  Kernel order in the graph makes
// every wait of theirs already satisfied: the class kernels find the heavy
// counts done, and the heavy numeric kernel finds its instances' column
// pointers published.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "block_ops.cuh"
#include "cta_products.cuh"
#include "spg_internal.cuh"

namespace spg {

const char *last_error_str();
void clear_error();

struct BatchInst {
    const void *Acp, *Bcp, *Aval, *Bval;
    const int32_t *Arow, *Brow;
    int64_t m, k, n;
    int64_t out_base;     // first entry of the output region
    int64_t col_base;     // first column of the instance in the batch-wide column arrays
    int32_t acp64, bcp64;
    int32_t ntask;        // column tasks of the instance
    int32_t vt;           // value type of A and B
};

struct BatchTask {
    int32_t inst, c0, c1, pad;
};

// One heavy column: instance, column, and the first word of its row bitmap in
// the heavy scratch (ceil(m / 32) words).
struct BatchHeavy {
    int32_t inst, col;
    int64_t bits_off;
};
constexpr int kHeavyMaxWords = 8192;   // a heavy column's instance has at most 262,144 rows
constexpr int kHeavyWinWords = 2048;   // rows of one numeric window: <= 65,536
constexpr int kHeavyCap = 4096;        // entries of one numeric window

constexpr int kBatchMaxLogS = 11;  // per-warp tables of up to 2048 slots
// Instances are launched in three classes by the table their largest column
// needs (up to 512, 1024 and 2048 slots), each class by its own persistent
// kernel, so that small tables buy more resident warps; the three kernels are
// parallel branches of the graph.
constexpr int kBatchClasses = 3;
constexpr int kBatchClassLogS[kBatchClasses] = {9, 10, 11};
enum : int { kBatchErrTimeout = 8 };

template <typename Acc>
__device__ __forceinline__ Acc bval_load(const void *v, int vt, int64_t i) {
    if (vt == SPG_VAL_F64) return (Acc)__ldg((const double *)v + i);
    if (vt == SPG_VAL_I32) return (Acc)__ldg((const int *)v + i);
    return (Acc)__ldg((const long long *)v + i);
}
template <>
__device__ __forceinline__ double bval_load<double>(const void *v, int, int64_t i) {
    return __ldg((const double *)v + i);
}
template <>
__device__ __forceinline__ long long bval_load<long long>(const void *v, int vt, int64_t i) {
    return vt == SPG_VAL_I32 ? (long long)__ldg((const int *)v + i) : __ldg((const long long *)v + i);
}

// Per column: flops_j and U_j = min(flops_j, m); per instance: sum of U_j
// (the output bound) and max U_j (the table size).
__global__ void k_batch_bounds(const BatchInst *insts, const BatchTask *tasks, int64_t ntasks,
                               unsigned long long *bound, unsigned int *maxU, unsigned int *colU) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < ntasks; t += nw) {
        const BatchTask tk = tasks[t];
        const BatchInst in = insts[tk.inst];
        unsigned long long sum = 0;
        unsigned int mx = 0;
        for (int j = tk.c0; j < tk.c1; j++) {
            const int64_t p0 = ld_ptr(in.Bcp, in.bcp64, j), p1 = ld_ptr(in.Bcp, in.bcp64, j + 1);
            long long fl = 0;
            for (int64_t p = p0 + lane; p < p1; p += 32) {
                const int k = in.Brow[p];
                fl += ld_ptr(in.Acp, in.acp64, k + 1) - ld_ptr(in.Acp, in.acp64, k);
            }
            fl = warp_sum_ll(fl);
            const long long U = min(fl, (long long)in.m);
            sum += (unsigned long long)U;
            mx = max(mx, (unsigned int)min(U, (long long)UINT32_MAX));
            if (lane == 0) colU[in.col_base + j] = (unsigned int)min(U, (long long)UINT32_MAX);
        }
        if (lane == 0) {
            atomicAdd(bound + tk.inst, sum);
            atomicMax(maxU + tk.inst, mx);
        }
    }
}

// Column pointers of instance `inst` from its per-column counts (one warp),
// then its ready flag.
__device__ __forceinline__ void instance_scan(const BatchInst &in, int inst, const int64_t *nnz, int64_t *colptr,
                                              int *ready, int lane) {
    const int64_t colb = in.col_base;
    __threadfence();
    int64_t run = 0;
    for (int64_t j0 = 0; j0 < in.n; j0 += 32) {
        const int64_t j = j0 + lane;
        const int64_t v = j < in.n ? *(volatile const int64_t *)(nnz + colb + j) : 0;
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t x = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += x;
        }
        if (j < in.n) colptr[colb + inst + j] = run + inc - v;
        run += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) {
        colptr[colb + inst + in.n] = run;
        __threadfence();
        atomicExch(ready + inst, 1);
    }
    __syncwarp();
}

// Bounded wait (one thread) for an instance's ready flag; false on timeout.
__device__ __forceinline__ bool wait_ready(const int *ready, int inst, int stall_inst, long long timeout_ns, int *err) {
    const int *flag = ready + inst;
    int never = 0;
    if (inst == stall_inst) flag = &never;  // failure test: a flag nothing sets
    unsigned long long start = 0, now = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(start));
    while (true) {
        if (*(volatile const int *)flag == 1) {
            __threadfence();
            return true;
        }
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if ((long long)(now - start) > timeout_ns) break;
        __nanosleep(256);
    }
    atomicOr(err, kBatchErrTimeout);
    return false;
}

__device__ __forceinline__ int log_table(long long U) {
    int l = 6;
    while ((1ll << l) < 2 * U) l++;
    return l;
}

template <int LOGS_MAX, typename Acc, typename OutIdx>
__global__ void k_batch_persistent(const BatchInst *__restrict__ insts, const BatchTask *__restrict__ tasks,
                                   int64_t ntasks, unsigned long long *head, int *sym_done, int *ready,
                                   int64_t *nnz, int64_t *colptr, OutIdx *__restrict__ out_row,
                                   Acc *__restrict__ out_val, int *err, long long timeout_ns, int stall_inst,
                                   const uint8_t *__restrict__ heavy_col) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int S_MAX = 1 << LOGS_MAX;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    WarpSeg<Acc> *segs = (WarpSeg<Acc> *)smem_raw;
    Acc *vals_all = (Acc *)(segs + nwarps);
    int *keys_all = (int *)(vals_all + nwarps * S_MAX);
    int *keys = keys_all + wid * S_MAX;
    Acc *vals = vals_all + wid * S_MAX;
    int *hist = keys_all + nwarps * S_MAX + wid * 256;
    WarpSeg<Acc> &ws = segs[wid];
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(head, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= (unsigned long long)(2 * ntasks)) break;
        const bool numeric = t >= (unsigned long long)ntasks;
        const BatchTask tk = tasks[numeric ? t - ntasks : t];
        const BatchInst in = insts[tk.inst];
        const int64_t colb = in.col_base;
        auto seg = [&](int64_t p, long long &st, int &len, Acc &bv) {
            const int k = in.Brow[p];
            st = ld_ptr(in.Acp, in.acp64, k);
            len = (int)(ld_ptr(in.Acp, in.acp64, k + 1) - st);
            bv = bval_load<Acc>(in.Bval, in.vt, p);
        };
        if (!numeric) {
            for (int j = tk.c0; j < tk.c1; j++) {
                if (heavy_col[colb + j]) continue;  // counted by the heavy kernel
                const int64_t p0 = ld_ptr(in.Bcp, in.bcp64, j), p1 = ld_ptr(in.Bcp, in.bcp64, j + 1);
                // twice the class's largest table, in the warp's value area
                // (8 bytes per slot of the numeric table: room for 2 x S_MAX
                // row ids): every column's bound min(flops, m) is <= S_MAX / 2,
                // so the load factor stays <= 1/4 (a table sized from the
                // column's own bound probes more: slower)
                static_assert(sizeof(Acc) == 2 * sizeof(int), "the value area holds 2 x S_MAX row ids");
                const int logS = LOGS_MAX + 1;
                const int S = 1 << logS;
                int *skeys = (int *)vals;
                for (int s = lane; s < S; s += 32) skeys[s] = kEmptyKey;
                __syncwarp();
                int cnt = 0;
                bool full = false;
                warp_products<false, Acc>(
                    p0, p1, lane, ws, in.Arow, (const Acc *)nullptr, seg, [&](int r, Acc) {
                        bool fresh;
                        if (hash_insert(skeys, logS, r, &fresh) < 0) full = true;
                        cnt += fresh ? 1 : 0;
                    });
                cnt = warp_sum_i(cnt);
                if (__any_sync(kFull, full) && lane == 0) atomicOr(err, kDevErrInternal);
                if (lane == 0) nnz[colb + j] = cnt;
                __syncwarp();
            }
            int mine = 0;
            if (lane == 0) {
                __threadfence();
                // the warp finishing the instance's last symbolic task scans it
                mine = atomicAdd(sym_done + tk.inst, 1) + 1 == in.ntask ? 1 : 0;
            }
            mine = __shfl_sync(kFull, mine, 0);
            if (mine) instance_scan(in, tk.inst, nnz, colptr, ready, lane);
        } else {
            // wait, bounded, for the instance's column pointers
            int ok = 0;
            if (lane == 0) ok = wait_ready(ready, tk.inst, stall_inst, timeout_ns, err) ? 1 : 0;
            ok = __shfl_sync(kFull, ok, 0);
            if (!ok) break;
            const int64_t *cp = colptr + colb + tk.inst;
            for (int j = tk.c0; j < tk.c1; j++) {
                if (heavy_col[colb + j]) continue;  // written by the heavy kernel
                const int64_t base = in.out_base + cp[j];
                const int64_t want = cp[j + 1] - cp[j];
                const int64_t p0 = ld_ptr(in.Bcp, in.bcp64, j), p1 = ld_ptr(in.Bcp, in.bcp64, j + 1);
                // >= 4 x the column's count (at most the class's table): a
                // sparser table probes less, which outweighs clearing more
                const int logS = min(LOGS_MAX, log_table(want > 0 ? want : 1) + 1);
                const int S = 1 << logS;
                for (int s = lane; s < S; s += 32) {
                    keys[s] = kEmptyKey;
                    vals[s] = Acc(0);
                }
                __syncwarp();
                bool full = false;
                // A's values may be stored as double, int32 or int64
                warp_products_v<true, 4, Acc>(
                    p0, p1, lane, ws, in.Arow, seg,
                    [&](long long e) { return bval_load<Acc>(in.Aval, in.vt, e); },
                    [&](int r, Acc v) {
                        bool fresh;
                        const int slot = hash_insert(keys, logS, r, &fresh);
                        if (slot < 0)
                            full = true;
                        else
                            atomic_add_acc(vals + slot, v);
                    });
                __syncwarp();
                int nout = 0;
                for (int c0 = 0; c0 < S; c0 += 32) {
                    const int kk = keys[c0 + lane];
                    const Acc vv = vals[c0 + lane];
                    const bool occ = kk != kEmptyKey;
                    const unsigned bal = __ballot_sync(kFull, occ);
                    __syncwarp();
                    if (occ) {
                        const int pos = nout + __popc(bal & ((1u << lane) - 1u));
                        keys[pos] = kk;
                        vals[pos] = vv;
                    }
                    nout += __popc(bal);
                    __syncwarp();
                }
                full = __any_sync(kFull, full);
                if (full || nout != want) {
                    if (lane == 0) atomicOr(err, kDevErrInternal);
                } else {
                    warp_sort_pairs<Acc>(keys, vals, nout, S, hist, lane);
                    for (int s = lane; s < nout; s += 32) {
                        out_row[base + s] = (OutIdx)keys[s];
                        out_val[base + s] = vals[s];
                    }
                }
                __syncwarp();
            }
        }
    }
}

// Heavy columns of the batch, one CTA per column task (claimed from `head`);
// the instance's A is read in place (its values in the accumulation type).
// PHASE 0: every product sets its row's bit in a shared bitmap of the
// instance's rows; the bitmap goes to the scratch, its popcount to nnz, and
// the instance's symbolic-task counter advances (its last task scans).
// PHASE 1: after the instance's ready flag, the column in row windows of at
// most kHeavyWinWords bitmap words and kHeavyCap entries: the window's words
// and their popcount prefix give every row its rank, products of rows in the
// window accumulate at acc[rank], and the window is written in row order.
template <int PHASE, typename Acc, typename OutIdx>
__global__ void __launch_bounds__(kBatch)
    k_batch_heavy(const BatchInst *__restrict__ insts, const BatchHeavy *__restrict__ htasks, int64_t nh,
                  unsigned long long *head, int *sym_done, int *ready, int64_t *nnz, int64_t *colptr,
                  uint32_t *__restrict__ scratch, OutIdx *__restrict__ out_row, Acc *__restrict__ out_val, int *err,
                  long long timeout_ns, int stall_inst) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaBatch<Acc> &sb = *(CtaBatch<Acc> *)smem_raw;
    unsigned char *area = smem_raw + ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15);
    __shared__ long long claim;
    __shared__ int ctot[kHeavyWinWords / 32];
    __shared__ int red[32];
    __shared__ int cut_sh, flag_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int64_t t = cta_claim(head, &claim); t < nh; t = cta_claim(head, &claim)) {
        const BatchHeavy hv = htasks[t];
        const BatchInst in = insts[hv.inst];
        const int j = hv.col;
        const int64_t p0 = ld_ptr(in.Bcp, in.bcp64, j), p1 = ld_ptr(in.Bcp, in.bcp64, j + 1);
        const int nwords = (int)((in.m + 31) / 32);
        auto seg = [&](int64_t p, long long &st, int &len, Acc &bv) {
            const int k = in.Brow[p];
            if ((uint64_t)k < (uint64_t)in.k) {
                st = ld_ptr(in.Acp, in.acp64, k);
                len = (int)(ld_ptr(in.Acp, in.acp64, k + 1) - st);
                if (PHASE == 1) bv = bval_load<Acc>(in.Bval, in.vt, p);
            }
        };
        if (PHASE == 0) {
            uint32_t *bits = (uint32_t *)area;
            const SegReg<Acc> first = cta_first_seg<Acc>(p0, p1, seg);
            for (int w = tid; w < nwords; w += blockDim.x) bits[w] = 0;
            // (the first barrier of cta_products orders the clearing before every product)
            cta_products<false, SPG_SYM_UNROLL, Acc>(p0, p1, sb, in.Arow, (const Acc *)nullptr, first, seg,
                                                     [&](int r, Acc) {
                                                         if ((uint64_t)r < (uint64_t)in.m)
                                                             set_bit_shared(bits + (r >> 5), 1u << (r & 31));
                                                     });
            int c = 0;
            uint32_t *dst = scratch + hv.bits_off;
            for (int w = tid; w < nwords; w += blockDim.x) {
                const uint32_t x = bits[w];
                dst[w] = x;
                c += __popc(x);
            }
            c = warp_sum_i(c);
            if (lane == 0) red[wid] = c;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < nw; w++) tot += red[w];
                nnz[in.col_base + j] = tot;
                __threadfence();
                flag_sh = atomicAdd(sym_done + hv.inst, 1) + 1 == in.ntask ? 1 : 0;
            }
            __syncthreads();
            if (flag_sh && wid == 0) instance_scan(in, hv.inst, nnz, colptr, ready, lane);
        } else {
            if (tid == 0) flag_sh = wait_ready(ready, hv.inst, stall_inst, timeout_ns, err) ? 1 : 0;
            __syncthreads();
            if (!flag_sh) return;  // a timeout is recorded; the CTA stops
            const HeavyAcc<Acc> acc(area, kHeavyCap + 1);
            uint2 *bp = (uint2 *)(area + HeavyAcc<Acc>::bytes_per_slot * (size_t)(kHeavyCap + 1));
            const int64_t cbase = in.out_base + colptr[in.col_base + hv.inst + j];
            const int64_t want = colptr[in.col_base + hv.inst + j + 1] - colptr[in.col_base + hv.inst + j];
            const uint32_t *src = scratch + hv.bits_off;
            int64_t done = 0;
            for (int w0 = 0; w0 < nwords;) {
                const int nwin = min(kHeavyWinWords, nwords - w0);
                const int total = cta_load_scan_bitmap(src + w0, bp, nwin, ctot);
                if (tid == 0) cut_sh = nwin;
                __syncthreads();
                if (total > kHeavyCap) {
                    // the first word that does not fit ends the window
                    for (int w = tid; w < nwin; w += blockDim.x)
                        if ((int)bp[w].y + __popc(bp[w].x) > kHeavyCap) atomicMin(&cut_sh, w);
                    __syncthreads();
                }
                const int wcut = cut_sh;
                const int cnt = wcut < nwin ? (int)bp[wcut].y : total;
                for (int i = tid; i < cnt; i += blockDim.x) acc.zero(i);
                const int rlo = w0 * 32, span = wcut * 32;
                const SegReg<Acc> first = cta_first_seg<Acc>(p0, p1, seg);
                // (the first barrier of cta_products orders the zeroing before every product)
                cta_products<true, SPG_NUM_UNROLL, Acc>(
                    p0, p1, sb, in.Arow, (const Acc *)in.Aval, first, seg, [&](int r, Acc v) {
                        const int lr = r - rlo;
                        if ((unsigned)lr < (unsigned)span) {
                            const uint2 x = bp[lr >> 5];
                            const uint32_t sh = lr & 31;
                            if ((x.x >> sh) & 1u) acc.add((int)(x.y + __popc(x.x & ((1u << sh) - 1u))), v);
                        }
                    });
                if (done + cnt <= want) {
                    for (int i = tid; i < cnt; i += blockDim.x) out_val[cbase + done + i] = acc.get(i);
                    __syncthreads();
                    int32_t *srow = acc.scratch32();
                    for (int w = tid; w < wcut; w += blockDim.x) {
                        uint32_t word = bp[w].x;
                        int pos = (int)bp[w].y;
                        while (word) {
                            srow[pos++] = rlo + w * 32 + __ffs(word) - 1;
                            word &= word - 1u;
                        }
                    }
                    __syncthreads();
                    for (int i = tid; i < cnt; i += blockDim.x) out_row[cbase + done + i] = (OutIdx)srow[i];
                } else if (tid == 0) {
                    atomicOr(err, kDevErrInternal);  // never write past the column's room
                }
                __syncthreads();
                done += cnt;
                w0 += wcut;
            }
            if (tid == 0 && done != want) atomicOr(err, kDevErrInternal);
        }
    }
}

}  // namespace spg

struct spg_batch {
    int count = 0;
    int64_t total_cols = 0, ntasks = 0, pool = 0;
    bool f64 = true;
    spg_batch_options opt{};
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side[spg::kBatchClasses] = {};  // branches of the captured graph (class c > 0)
    cudaEvent_t fork = nullptr, join[spg::kBatchClasses] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<spg::BatchInst> hinst;
    std::vector<void *> allocs;
    spg::BatchInst *insts = nullptr;
    spg::BatchTask *tasks = nullptr;
    unsigned long long *head = nullptr;
    int *sym_done = nullptr, *ready = nullptr, *err = nullptr;
    int64_t *nnz = nullptr, *colptr = nullptr;
    void *out_row = nullptr, *out_val = nullptr;
    int grid = 0, warps = 8;
    size_t smem = 0;
    int64_t class_off[spg::kBatchClasses + 1] = {};  // tasks of class c: [class_off[c], class_off[c + 1])
    int sm_count = 0;
    // heavy columns (CTA tasks)
    int64_t nheavy = 0;
    spg::BatchHeavy *htasks = nullptr;
    uint8_t *heavy_col = nullptr;   // per batch column: 1 = handled by the heavy kernels
    uint32_t *hscratch = nullptr;   // the heavy columns' row bitmaps
};

using namespace spg;

static void *batch_alloc(spg_batch *b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch allocation of %zu bytes failed", bytes);
        return nullptr;
    }
    b->allocs.push_back(p);
    return p;
}

extern "C" void spgemm_batch_default_options(spg_batch_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->task_cols = 64;
    o->warps_per_cta = 8;
    o->timeout_ns = 2000000000ll;
    o->stall_instance = -1;
}

extern "C" spg_status spgemm_batch_destroy(spg_batch *b) {
    if (!b) return SPG_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int c = 0; c < kBatchClasses; c++) {
        if (b->side[c]) cudaStreamDestroy(b->side[c]);
        if (b->join[c]) cudaEventDestroy(b->join[c]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaDeviceSynchronize();
    for (void *p : b->allocs) cudaFree(p);
    delete b;
    return SPG_OK;
}

template <int LOGS_MAX, typename Acc, typename OutIdx>
static spg_status batch_launch_class(spg_batch *b, int c, cudaStream_t st) {
    const int64_t t0 = b->class_off[c], nt = b->class_off[c + 1] - t0;
    if (nt == 0) return SPG_OK;
    auto kern = k_batch_persistent<LOGS_MAX, Acc, OutIdx>;
    const size_t smem = sizeof(WarpSeg<double>) * (size_t)b->warps +
                        (8 + sizeof(int)) * (size_t)b->warps * (1u << LOGS_MAX) + sizeof(int) * 256 * (size_t)b->warps;
    spg_status s = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              "batch smem");
    if (s) return s;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, b->warps * 32, smem);
    if (occ < 1) {
        set_error("batch kernel does not fit on an SM with %d warps", b->warps);
        return SPG_UNSUPPORTED;
    }
    const int grid = b->sm_count * occ;
    b->grid = std::max(b->grid, grid);
    b->smem = std::max(b->smem, smem);
    kern<<<grid, b->warps * 32, smem, st>>>(
        b->insts, b->tasks + t0, nt, b->head + c, b->sym_done, b->ready, b->nnz, b->colptr, (OutIdx *)b->out_row,
        (Acc *)b->out_val, b->err, b->opt.timeout_ns, b->opt.stall_instance, b->heavy_col);
    return cuda_check(cudaGetLastError(), "batch kernel launch");
}

// The heavy columns' kernel of one phase (0: counts, 1: values), CTAs claim
// column tasks from their own counter.
template <int PHASE, typename Acc, typename OutIdx>
static spg_status batch_launch_heavy(spg_batch *b) {
    if (b->nheavy == 0) return SPG_OK;
    auto kern = k_batch_heavy<PHASE, Acc, OutIdx>;
    const size_t area = std::max(sizeof(uint32_t) * (size_t)kHeavyMaxWords,
                                 sizeof(Acc) * (size_t)(kHeavyCap + 1) + sizeof(uint2) * (size_t)kHeavyWinWords);
    const size_t smem = ((sizeof(CtaBatch<Acc>) + 15) & ~(size_t)15) + area;
    spg_status s = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              "batch heavy smem");
    if (s) return s;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatch, smem);
    if (occ < 1) occ = 1;
    const int grid = (int)std::min<int64_t>((int64_t)b->sm_count * occ, b->nheavy);
    kern<<<grid, kBatch, smem, b->cap_stream>>>(b->insts, b->htasks, b->nheavy, b->head + kBatchClasses + PHASE,
                                               b->sym_done, b->ready, b->nnz, b->colptr, b->hscratch,
                                               (OutIdx *)b->out_row, (Acc *)b->out_val, b->err, b->opt.timeout_ns,
                                               b->opt.stall_instance);
    return cuda_check(cudaGetLastError(), "batch heavy kernel launch");
}

// One graph: clear the counters and flags, the heavy columns' counts, the
// three class kernels side by side, then the heavy columns' values.
template <typename Acc, typename OutIdx>
static spg_status batch_capture(spg_batch *b) {
    spg_status s = cuda_check(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
    if (s) return s;
    cudaMemsetAsync(b->head, 0, sizeof(unsigned long long) * (kBatchClasses + 2), b->cap_stream);
    cudaMemsetAsync(b->sym_done, 0, sizeof(int) * (size_t)b->count * 2 + sizeof(int) * 4, b->cap_stream);
    static_assert(kBatchClasses == 3, "one launch per class below");
    // heavy counts first: the class kernels' last symbolic task of an instance
    // then scans counts that are all there; heavy values last: their
    // instances' column pointers are published by then
    s = batch_launch_heavy<0, Acc, OutIdx>(b);
    // the class kernels as parallel branches of the graph: a class's CTAs take
    // the SMs that another class's CTAs leave as its queue drains (each
    // kernel's waits are on its own warps' tasks only)
    cudaStream_t cst[kBatchClasses] = {b->cap_stream, b->side[1], b->side[2]};
    if (!s) s = cuda_check(cudaEventRecord(b->fork, b->cap_stream), "fork");
    for (int c = 1; c < kBatchClasses && !s; c++) s = cuda_check(cudaStreamWaitEvent(cst[c], b->fork, 0), "fork");
    if (!s) s = batch_launch_class<kBatchClassLogS[0], Acc, OutIdx>(b, 0, cst[0]);
    if (!s) s = batch_launch_class<kBatchClassLogS[1], Acc, OutIdx>(b, 1, cst[1]);
    if (!s) s = batch_launch_class<kBatchClassLogS[2], Acc, OutIdx>(b, 2, cst[2]);
    for (int c = 1; c < kBatchClasses; c++) {
        // joined even after an error, so that the capture can end
        cudaEventRecord(b->join[c], cst[c]);
        cudaStreamWaitEvent(b->cap_stream, b->join[c], 0);
    }
    if (!s) s = batch_launch_heavy<1, Acc, OutIdx>(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    b->graph = g;
    if (s) return s;
    s = cuda_check(e, "end capture");
    if (s) return s;
    return cuda_check(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
}

extern "C" spg_status spgemm_batch_create(int32_t count, const spg_csc *A, const spg_csc *B,
                                          const spg_batch_options *opt, spg_batch **out) {
    clear_error();
    if (!out || count < 1 || !A || !B) {
        set_error("batch needs count >= 1, A, B and out");
        return SPG_INVALID_ARGUMENT;
    }
    *out = nullptr;
    spg_batch_options o;
    spgemm_batch_default_options(&o);
    if (opt) o = *opt;
    if (o.task_cols < 1 || (o.warps_per_cta != 4 && o.warps_per_cta != 8) || o.timeout_ns <= 0) {
        set_error("task_cols >= 1, warps_per_cta 4 or 8, timeout_ns > 0");
        return SPG_INVALID_ARGUMENT;
    }
    const bool f64 = A[0].val_type == SPG_VAL_F64;
    for (int i = 0; i < count; i++) {
        const spg_csc &a = A[i], &bb = B[i];
        if (a.ncols != bb.nrows || a.idx_type != SPG_IDX_I32 || bb.idx_type != SPG_IDX_I32 || a.val_type != bb.val_type ||
            (a.val_type == SPG_VAL_F64) != f64 || (bb.val_type == SPG_VAL_F64) != f64 || !a.colptr || !bb.colptr ||
            a.nrows >= INT32_MAX || bb.ncols >= INT32_MAX || a.nrows < 0 || bb.ncols < 0) {
            set_error("instance %d: dimensions, int32 row ids and one value kind (double or integer) for all", i);
            return SPG_INVALID_ARGUMENT;
        }
    }
    spg_batch *b = new (std::nothrow) spg_batch();
    if (!b) return SPG_OUT_OF_MEMORY;
    b->count = count;
    b->opt = o;
    b->f64 = f64;
    b->warps = o.warps_per_cta;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    spg_status s = cuda_check(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
    for (int c = 1; c < kBatchClasses && !s; c++) {
        s = cuda_check(cudaStreamCreateWithFlags(&b->side[c], cudaStreamNonBlocking), "stream");
        if (!s) s = cuda_check(cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming), "event");
    }
    if (!s) s = cuda_check(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
    // instances and tasks
    std::vector<BatchTask> htask;
    b->hinst.resize(count);
    int64_t col = 0;
    for (int i = 0; i < count && !s; i++) {
        BatchInst &in = b->hinst[i];
        in.Acp = A[i].colptr;
        in.Bcp = B[i].colptr;
        in.Aval = A[i].vals;
        in.Bval = B[i].vals;
        in.Arow = (const int32_t *)A[i].rowidx;
        in.Brow = (const int32_t *)B[i].rowidx;
        in.m = A[i].nrows;
        in.k = A[i].ncols;
        in.n = B[i].ncols;
        in.acp64 = A[i].ptr_type == SPG_IDX_I64;
        in.bcp64 = B[i].ptr_type == SPG_IDX_I64;
        in.vt = A[i].val_type;
        in.col_base = col;
        int nt = 0;
        for (int64_t c0 = 0; c0 < in.n; c0 += o.task_cols) {
            htask.push_back({i, (int32_t)c0, (int32_t)std::min<int64_t>(in.n, c0 + o.task_cols), 0});
            nt++;
        }
        if (nt == 0) htask.push_back({i, 0, 0, 0}), nt = 1;  // empty instance: one empty task
        in.ntask = nt;
        col += in.n;
    }
    b->total_cols = col;
    b->ntasks = (int64_t)htask.size();
    if (!s) {
        b->insts = (BatchInst *)batch_alloc(b, sizeof(BatchInst) * (size_t)count);
        b->tasks = (BatchTask *)batch_alloc(b, sizeof(BatchTask) * (size_t)b->ntasks);
        b->head = (unsigned long long *)batch_alloc(b, sizeof(unsigned long long) * (kBatchClasses + 2));
        b->sym_done = (int *)batch_alloc(b, sizeof(int) * (size_t)count * 2 + sizeof(int) * 4);
        b->nnz = (int64_t *)batch_alloc(b, sizeof(int64_t) * (size_t)(col + 1));
        b->colptr = (int64_t *)batch_alloc(b, sizeof(int64_t) * (size_t)(col + count + 1));
        if (!b->insts || !b->tasks || !b->head || !b->sym_done || !b->nnz || !b->colptr) s = SPG_OUT_OF_MEMORY;
    }
    if (!s) {
        b->ready = b->sym_done + count;
        b->err = b->ready + count;
        s = cuda_check(cudaMemcpy(b->insts, b->hinst.data(), sizeof(BatchInst) * (size_t)count, cudaMemcpyHostToDevice), "insts");
    }
    if (!s) s = cuda_check(cudaMemcpy(b->tasks, htask.data(), sizeof(BatchTask) * htask.size(), cudaMemcpyHostToDevice), "tasks");
    // bounds pass: output room, table sizes and every column's bound
    std::vector<unsigned long long> bound(count);
    std::vector<unsigned int> maxU(count, 0u), colU((size_t)std::max<int64_t>(col, 1));
    if (!s) {
        unsigned long long *db = (unsigned long long *)batch_alloc(b, sizeof(unsigned long long) * (size_t)count);
        unsigned int *dm = (unsigned int *)batch_alloc(b, sizeof(unsigned int) * (size_t)count);
        unsigned int *du = (unsigned int *)batch_alloc(b, sizeof(unsigned int) * (size_t)std::max<int64_t>(col, 1));
        if (!db || !dm || !du) s = SPG_OUT_OF_MEMORY;
        if (!s) {
            cudaMemset(db, 0, sizeof(unsigned long long) * (size_t)count);
            cudaMemset(dm, 0, sizeof(unsigned int) * (size_t)count);
            k_batch_bounds<<<grid_for(b->ntasks * 32, 256, b->sm_count * 16), 256>>>(b->insts, b->tasks, b->ntasks, db,
                                                                                  dm, du);
            s = cuda_check(cudaGetLastError(), "bounds");
        }
        if (!s) s = cuda_check(cudaMemcpy(bound.data(), db, sizeof(unsigned long long) * (size_t)count, cudaMemcpyDeviceToHost), "bounds");
        if (!s && col > 0)
            s = cuda_check(cudaMemcpy(colU.data(), du, sizeof(unsigned int) * (size_t)col, cudaMemcpyDeviceToHost), "bounds");
    }
    // heavy columns: bound above the largest warp table; the rest sets the
    // instance's table class
    std::vector<BatchHeavy> hheavy;
    std::vector<uint8_t> hflag((size_t)std::max<int64_t>(col, 1), 0);
    int64_t hwords = 0;
    if (!s) {
        const unsigned int lim = 1u << (kBatchMaxLogS - 1);
        for (int i = 0; i < count && !s; i++) {
            const BatchInst &in = b->hinst[i];
            for (int64_t j = 0; j < in.n; j++) {
                const unsigned int U = colU[in.col_base + j];
                if (U <= lim) {
                    maxU[i] = std::max(maxU[i], U);
                    continue;
                }
                if (in.m > (int64_t)kHeavyMaxWords * 32 || (in.vt == SPG_VAL_I32)) {
                    set_error("instance %d has a column of up to %u entries: heavy columns need at most %d rows and "
                              "double or int64 values (use spgemm_1d_multiply for such products)", i, U,
                              kHeavyMaxWords * 32);
                    s = SPG_UNSUPPORTED;
                    break;
                }
                hflag[in.col_base + j] = 1;
                hheavy.push_back({i, (int32_t)j, hwords});
                hwords += (in.m + 31) / 32;
                b->hinst[i].ntask++;
            }
        }
    }
    if (!s) {
        b->nheavy = (int64_t)hheavy.size();
        b->heavy_col = (uint8_t *)batch_alloc(b, (size_t)std::max<int64_t>(col, 1));
        b->htasks = (BatchHeavy *)batch_alloc(b, sizeof(BatchHeavy) * (size_t)std::max<int64_t>(b->nheavy, 1));
        b->hscratch = (uint32_t *)batch_alloc(b, sizeof(uint32_t) * (size_t)std::max<int64_t>(hwords, 1));
        if (!b->heavy_col || !b->htasks || !b->hscratch) s = SPG_OUT_OF_MEMORY;
        if (!s) s = cuda_check(cudaMemcpy(b->heavy_col, hflag.data(), (size_t)std::max<int64_t>(col, 1),
                                          cudaMemcpyHostToDevice), "heavy flags");
        if (!s && b->nheavy)
            s = cuda_check(cudaMemcpy(b->htasks, hheavy.data(), sizeof(BatchHeavy) * hheavy.size(),
                                      cudaMemcpyHostToDevice), "heavy tasks");
    }
    if (!s) {
        // the tasks of each class together, instance order kept inside a class
        std::vector<int> cls(count);
        for (int i = 0; i < count; i++) {
            int c = 0;
            while (c < kBatchClasses - 1 && maxU[i] > (1u << (kBatchClassLogS[c] - 1))) c++;
            cls[i] = c;
        }
        std::vector<BatchTask> sorted;
        sorted.reserve(htask.size());
        for (int c = 0; c < kBatchClasses; c++) {
            b->class_off[c] = (int64_t)sorted.size();
            for (const BatchTask &t : htask)
                if (cls[t.inst] == c) sorted.push_back(t);
        }
        b->class_off[kBatchClasses] = (int64_t)sorted.size();
        s = cuda_check(cudaMemcpy(b->tasks, sorted.data(), sizeof(BatchTask) * sorted.size(), cudaMemcpyHostToDevice),
                       "tasks");
    }
    if (!s) {
        int64_t off = 0;
        for (int i = 0; i < count; i++) {
            b->hinst[i].out_base = off;
            off += (int64_t)bound[i];
        }
        b->pool = off;
        s = cuda_check(cudaMemcpy(b->insts, b->hinst.data(), sizeof(BatchInst) * (size_t)count, cudaMemcpyHostToDevice), "insts");
        if (!s) {
            b->out_row = batch_alloc(b, sizeof(int32_t) * (size_t)(off + 1));
            b->out_val = batch_alloc(b, 8 * (size_t)(off + 1));
            if (!b->out_row || !b->out_val) s = SPG_OUT_OF_MEMORY;
        }
    }
    if (!s) s = f64 ? batch_capture<double, int>(b) : batch_capture<long long, int>(b);
    if (s) {
        std::string keep = last_error_str();
        spgemm_batch_destroy(b);
        set_error("%s", keep.c_str());
        return s;
    }
    *out = b;
    return SPG_OK;
}

extern "C" spg_status spgemm_batch_execute(spg_batch *b, void *stream) {
    spg::PhaseRange nvtx_range("spgemm_batch_execute");
    clear_error();
    if (!b) {
        set_error("batch is NULL");
        return SPG_INVALID_ARGUMENT;
    }
    return cuda_check(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "batch graph launch");
}

extern "C" spg_status spgemm_batch_status(spg_batch *b, void *stream) {
    clear_error();
    if (!b) {
        set_error("batch is NULL");
        return SPG_INVALID_ARGUMENT;
    }
    int e = 0;
    spg_status s = cuda_check(cudaMemcpyAsync(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "status");
    if (!s) s = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "status");
    if (s) return s;
    if (e & kBatchErrTimeout) {
        set_error("a batched task waited longer than %lld ns for its instance's column pointers",
                  (long long)b->opt.timeout_ns);
        return SPG_TIMEOUT;
    }
    if (e) {
        set_error("batched kernel consistency check failed");
        return SPG_CUDA_ERROR;
    }
    return SPG_OK;
}

extern "C" spg_status spgemm_batch_result(const spg_batch *b, int32_t i, spg_csc *C) {
    clear_error();
    if (!b || !C || i < 0 || i >= b->count) {
        set_error("bad batch result arguments");
        return SPG_INVALID_ARGUMENT;
    }
    const BatchInst &in = b->hinst[i];
    int64_t nnz = 0;
    spg_status s = cuda_check(cudaMemcpy(&nnz, b->colptr + in.col_base + i + in.n, sizeof(int64_t),
                                         cudaMemcpyDeviceToHost), "result");
    if (s) return s;
    C->nrows = in.m;
    C->ncols = in.n;
    C->nnz = nnz;
    C->ptr_type = SPG_IDX_I64;
    C->idx_type = SPG_IDX_I32;
    C->val_type = b->f64 ? SPG_VAL_F64 : SPG_VAL_I64;
    C->colptr = b->colptr + in.col_base + i;
    C->rowidx = (int32_t *)b->out_row + in.out_base;
    C->vals = (char *)b->out_val + 8 * in.out_base;
    return SPG_OK;
}

extern "C" spg_status spgemm_batch_copy_result(const spg_batch *b, int32_t i, void *colptr, void *rowidx, void *vals,
                                               void *stream) {
    spg_csc C{};
    spg_status s = spgemm_batch_result(b, i, &C);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (colptr)
        s = cuda_check(cudaMemcpyAsync(colptr, C.colptr, sizeof(int64_t) * (size_t)(C.ncols + 1), cudaMemcpyDeviceToDevice, st), "copy");
    if (!s && rowidx && C.nnz)
        s = cuda_check(cudaMemcpyAsync(rowidx, C.rowidx, sizeof(int32_t) * (size_t)C.nnz, cudaMemcpyDeviceToDevice, st), "copy");
    if (!s && vals && C.nnz)
        s = cuda_check(cudaMemcpyAsync(vals, C.vals, 8 * (size_t)C.nnz, cudaMemcpyDeviceToDevice, st), "copy");
    return s;
}

extern "C" spg_status spgemm_batch_info(const spg_batch *b, int64_t *ntasks, int64_t *pool_entries, int32_t *grid) {
    if (!b) return SPG_INVALID_ARGUMENT;
    if (ntasks) *ntasks = b->ntasks;
    if (pool_entries) *pool_entries = b->pool;
    if (grid) *grid = b->grid;
    return SPG_OK;
}
