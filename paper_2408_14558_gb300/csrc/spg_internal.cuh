// Internal declarations of the GB300 sparsity-aware 1D SpGEMM library.
//
// Layout in HBM (all per plan, all P column blocks processed together):
//   Dbits     ceil(k/32) u32          nonempty columns of A (the set D of Algorithm 1)
//   Hbits     P * W u32               H_i, nonzero rows of B_i (Table 1), W = ceil(k/32)
//   rankpre   P * W + 1 i64           exclusive prefix of popc(H_i & D) over (block, word):
//                                     the global index of the first required column of a word
//   dtilde    sum|D~_i| i32           required column ids, block after block, ascending
//   fetch     P * ceil(k/b) u8        chosen fetch blocks (Algorithm 2)
//   At_*      CSC of all A~_i         colptr i64 (sum|D~_i| + 1), rows i32, values Acc
//   Bq, Bv    nnz(B) i32 / Acc        B with each row k replaced by its column of A~_i (-1 if
//                                     column k of A is empty), values widened to Acc
//   flops, win_lo/hi, nnzb, maxa      per output column statistics (Section 3.2 flop count)
//   binlist   n i32                   column ids grouped by bin
//   split     sum|D~_i| * (T+1) i32   heavy bins only: offset of the first row >= t*R in each
//                                     A~ column (R rows per base slab, T = ceil(m/R))
//   hbits     records * R/32 u32      heavy bins only: symbolic row bitmap of each
//                                     (column, base slab) record
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "spgemm1d.h"

namespace spg {

// A named NVTX range for the lifetime of the object: every entry point and
// every phase of a multiply shows up by name in a profiler's timeline (the
// calls do nothing unless a tool is attached).
struct PhaseRange {
    explicit PhaseRange(const char *name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
    PhaseRange(const PhaseRange &) = delete;
    PhaseRange &operator=(const PhaseRange &) = delete;
};

constexpr unsigned kFull = 0xffffffffu;
constexpr int kEmptyKey = -1;

// Per-column bins.  0: no products.  1..6: warp hash with table size 32 << bin.
// 7: dense row slabs (heavy).
constexpr int kBinEmpty = 0;
constexpr int kBinHeavy = 7;
constexpr int kNumBins = 8;
constexpr int kMaxLightBin = 6;

// Device error bits (OR-ed into plan->d_err).
enum : int {
    kDevErrInput = 1,      // input not canonical
    kDevErrInternal = 2,   // a kernel found an inconsistency (hash full, count mismatch)
    kDevErrRange = 4,      // a size limit of this build was exceeded
};

struct Alloc {
    void *p;
    size_t bytes;
};

}  // namespace spg

// Optional output mask of a plan: column j of C keeps row r iff bit r of
// column j's words, XOR flip, is set (flip = ~0 for a complemented mask).
struct OutMask {
    const uint32_t *bits = nullptr;  // nullptr: every row is kept
    int64_t words = 0;               // words per column
    uint32_t flip = 0;
};
__device__ __forceinline__ bool mask_keeps(const OutMask &m, int64_t j, int r) {
    return ((__ldg(m.bits + j * m.words + (r >> 5)) ^ m.flip) >> (r & 31)) & 1u;
}

struct spg_plan {
    spg_csc A{}, B{};
    spg_options opt{};
    OutMask omask;
    cudaStream_t st = nullptr;
    int64_t m = 0, k = 0, n = 0, nnzA = 0, nnzB = 0;
    int P = 1;
    int64_t b = 1;
    bool acc_f64 = true;     // double accumulation, else int64 wrapping
    bool out_idx64 = false;  // C row ids int64
    int64_t W = 0;           // u32 words per H_i bitmap
    int64_t nfb = 0;         // fetch blocks per column block
    int light_max = 1024;
    int R = 8192, T = 1;     // heavy slab rows and slab count
    int sm_count = 0;

    std::vector<spg::Alloc> allocs;
    // small workspace buffers are carved from shared chunks (one allocator call per chunk)
    char *arena = nullptr;
    size_t arena_used = 0, arena_size = 0;
    int *d_err = nullptr;
    int64_t *d_cnt = nullptr;      // small device counters (see kCnt* in plan.cu)
    int64_t *h_pinned = nullptr;   // pinned host mirror for read-backs

    uint32_t *Dbits = nullptr, *Hbits = nullptr;
    int64_t *rankpre = nullptr;
    int32_t *dtilde = nullptr;
    int64_t ndt = 0;
    std::vector<int64_t> dt_base;  // host: first global D~ index of each block (P + 1)
    uint8_t *fetch = nullptr;
    int64_t *At_colptr = nullptr;
    int32_t *At_row = nullptr;
    void *At_val = nullptr;
    int64_t nAt = 0;
    int32_t *Bq = nullptr;
    void *Bv = nullptr;
    int64_t *flops = nullptr;
    int32_t *win_lo = nullptr, *win_hi = nullptr, *nnzb = nullptr, *maxa = nullptr;
    int8_t *bin_of = nullptr;
    int32_t *binlist = nullptr;
    int64_t bin_off[spg::kNumBins + 1] = {0};
    int64_t *d_bincur = nullptr;

    // heavy bins.  A record is one (heavy column, base slab of R rows) inside
    // the column's row window; the records of a column are consecutive.
    int64_t nheavy = 0, nrec = 0;
    int32_t *split = nullptr;
    int64_t *rec_first = nullptr;  // per heavy column: first record (nheavy + 1)
    int32_t *rec_col = nullptr, *rec_slab = nullptr;
    int32_t *rec_cnt = nullptr;    // nnz of C inside the record
    int64_t *rec_off = nullptr;    // offset of the record inside its column of C
    uint32_t *hbits = nullptr;     // R/32 words per record
    // symbolic items: <= sym_max_recs consecutive records of one column
    int64_t nsym = 0;
    int32_t *sym_rec0 = nullptr, *sym_nrec = nullptr;
    int sym_max_recs = 64;
    // numeric items: <= num_max_recs consecutive records of one column holding
    // <= num_cap entries of C
    int64_t nnum = 0;
    int32_t *num_rec0 = nullptr, *num_nrec = nullptr;
    int num_cap = 4096, num_max_recs = 32;

    // symbolic / numeric
    int64_t *nnzcol = nullptr;
    int64_t *Ccolptr = nullptr;  // plan-owned copy of C's column pointers
    int64_t nnzC = -1;
    bool symbolic_done = false;
    int32_t *nbinlist = nullptr;
    void *num_items = nullptr;  // one header per numeric item (k_num_heavy)
    int64_t *bounds_d = nullptr;     // column block bounds (P + 1) of a non-uniform split, else null
    int64_t *eoff = nullptr;         // first entry of B of every column block (P + 1)
    std::vector<int64_t> bounds_h;   // the bounds in effect (P + 1), host
    int64_t *blk = nullptr;          // per block: flops, gathered A~ nonzeros, of them fetched (3 x P)
    int64_t *gshift = nullptr;       // per A~ column: its entries' offset into A (gather)
    bool numeric_done = false;       // a numeric pass ran: the light lists and item headers exist
    cudaGraph_t graph = nullptr;     // captured refresh + numeric (spgemm_plan_capture)
    cudaGraphExec_t graph_exec = nullptr;
    int64_t nbin_off[spg::kNumBins + 1] = {0};

    spg_stats stats{};
    // ev[0..1] plan, ev[2..3] symbolic, ev[4..5] numeric; kev[2g], kev[2g+1]
    // bracket kernel group g (see KernelGroup)
    cudaEvent_t ev[8] = {nullptr};
    cudaEvent_t kev[10] = {nullptr};
    bool kev_used[5] = {false, false, false, false, false};
    int64_t launches = 0;
};

namespace spg {

// Every kernel of the library is launched through here, on the plan's
// stream, so that the plan can report how many kernels it ran.
template <typename... KArgs, typename... Args>
inline void launch(spg_plan *p, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args &&...args) {
    p->launches++;
    kern<<<grid, block, smem, p->st>>>(static_cast<KArgs>(args)...);
}

// Slot of plan->d_cnt that collects nnz(C) of the heavy columns (the other
// slots are used by the planning kernels).
constexpr int kCntNnzCHeavySlot = 18;
// Slots of plan->d_cnt holding the next unclaimed heavy item of the symbolic
// and numeric heavy kernels (CTAs claim items one at a time, in column order).
constexpr int kCntSymNextSlot = 19;
constexpr int kCntNumNextSlot = 20;
constexpr int kCntFusedNextSlot = 22;  // next item of the learned path's fused heavy kernel

// Claim the next item for the whole CTA; every thread must call it, and the
// CTA must have passed a barrier since the previous claim was read.
__device__ __forceinline__ int64_t cta_claim(unsigned long long *next, long long *slot) {
    if (threadIdx.x == 0) *slot = (long long)atomicAdd(next, 1ull);
    __syncthreads();
    return *slot;
}

// Kernel groups timed with their own event pair.
enum KernelGroup { kKGather = 0, kKSymLight = 1, kKSymHeavy = 2, kKNumLight = 3, kKNumHeavy = 4 };
inline void group_begin(spg_plan *p, int g) {
    cudaEventRecord(p->kev[2 * g], p->st);
    p->kev_used[g] = true;
}
inline void group_end(spg_plan *p, int g) { cudaEventRecord(p->kev[2 * g + 1], p->st); }

// ---- host helpers (plan.cu)
void set_error(const char *fmt, ...);
spg_status cuda_check(cudaError_t e, const char *what);
void *ws_alloc(spg_plan *p, size_t bytes);
void ws_free_all(spg_plan *p);
spg_status copy_operands(spg_plan *p);
spg_status prepare_numeric(spg_plan *p);
// Memory handed to the caller (C's arrays): through opt->alloc, else cudaMallocAsync.
void *alloc_user(const spg_options *opt, size_t bytes);
spg_status read_dev_err(spg_plan *p, const char *phase);
int grid_for(int64_t work, int per_block, int max_blocks);

// ---- scans (scan.cu): out[0..n] = exclusive prefix of in[0..n), out[n] = total.
spg_status scan_exclusive_i32(spg_plan *p, const int32_t *in, int64_t *out, int64_t n);
spg_status scan_exclusive_i64(spg_plan *p, const int64_t *in, int64_t *out, int64_t n);

// ---- binning (plan.cu): group the columns whose bin id is in bin_of into binlist.
spg_status bin_columns(spg_plan *p, const int8_t *bin_of, int32_t *list, int64_t *off_host);

// ---- phases
spg_status run_symbolic(spg_plan *p);
spg_status run_numeric(spg_plan *p, spg_csc *C);
spg_status multiply_learned(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C);
void remember_multiply_stats(const spg_stats &st);  // api.cu: spgemm_last_multiply_stats

// ---- shared kernels (plan.cu): groups of <= smr consecutive records of every
// heavy column, listed as (first record, count) starting at sym_first[h].
__global__ void k_sym_items(int64_t nheavy, int smr, const int64_t *rec_first, const int64_t *sym_first,
                            int32_t *sym_rec0, int32_t *sym_nrec);

// ---- device helpers
__device__ __forceinline__ int64_t ld_ptr(const void *p, int is64, int64_t i) {
    return is64 ? (int64_t)__ldg((const long long *)p + i) : (int64_t)__ldg((const int *)p + i);
}

// Column block of output column j: block i holds [floor(i*n/P), floor((i+1)*n/P)).
__device__ __forceinline__ int block_of(int64_t j, int64_t n, int P) {
    return (int)(((j + 1) * (int64_t)P - 1) / n);
}

// The same with explicit bounds (P + 1 ascending column ids from 0 to n, empty
// blocks allowed) when the plan has them: the largest i with bounds[i] <= j.
__device__ __forceinline__ int block_of_b(int64_t j, int64_t n, int P, const int64_t *bounds) {
    if (!bounds) return block_of(j, n, P);
    int lo = 0, hi = P;  // bounds[lo] <= j < bounds[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bounds[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <typename Acc>
__device__ __forceinline__ Acc mul_acc(Acc a, Acc b);
template <>
__device__ __forceinline__ double mul_acc<double>(double a, double b) { return a * b; }
template <>
__device__ __forceinline__ long long mul_acc<long long>(long long a, long long b) {
    return (long long)((unsigned long long)a * (unsigned long long)b);
}

__device__ __forceinline__ void atomic_add_acc(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_acc(long long *p, long long v) {
    atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// Per-warp scratch for walking the products of one output column.
template <typename Acc>
struct WarpSeg {
    int pref[33];
    long long start[32];
    Acc bv[32];
};

// Walk every product of the B' entries [p0, p1) of one output column with a
// whole warp.  seg(p, start, len, bv) gives the A~ positions [start, start+len)
// that B' entry p multiplies and its value; aval(e) loads A~'s value e.  The
// lengths of 32 consecutive entries are prefix-summed so that all 32 lanes stay
// busy however short the segments are; each step locates and loads U windows
// of 32 products before any of them is used, so that U loads per lane are in
// flight.  body(row, product) is called once per product.
template <bool NEED_VAL, int U, typename Acc, typename SegFn, typename ValFn, typename Body>
__device__ __forceinline__ void warp_products_v(int64_t p0, int64_t p1, int lane, WarpSeg<Acc> &ws,
                                                const int32_t *__restrict__ At_row, SegFn seg, ValFn aval,
                                                Body body) {
    for (int64_t base = p0; base < p1; base += 32) {
        int64_t p = base + lane;
        long long st = 0;
        int len = 0;
        Acc bv = Acc(0);
        if (p < p1) seg(p, st, len, bv);
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        int total = __shfl_sync(kFull, incl, 31);
        ws.pref[lane] = incl - len;
        ws.start[lane] = st;
        if (NEED_VAL) ws.bv[lane] = bv;
        __syncwarp();
        for (int f0 = 0; f0 < total; f0 += 32 * U) {
            int r[U];
            Acc a[U], b[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int fi = f0 + 32 * u + lane;
                ok[u] = fi < total;
                r[u] = 0;
                a[u] = Acc(0);
                b[u] = Acc(0);
                if (ok[u]) {
                    int s = 0;
#pragma unroll
                    for (int stp = 16; stp > 0; stp >>= 1)
                        if (ws.pref[s + stp] <= fi) s += stp;
                    const long long e = ws.start[s] + (fi - ws.pref[s]);
                    r[u] = __ldg(At_row + e);
                    if (NEED_VAL) {
                        a[u] = aval(e);
                        b[u] = ws.bv[s];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (ok[u]) body(r[u], NEED_VAL ? mul_acc<Acc>(a[u], b[u]) : Acc(0));
        }
        __syncwarp();
    }
}

// The same walk over A~ values stored in the accumulation type.
template <bool NEED_VAL, typename Acc, typename SegFn, typename Body>
__device__ __forceinline__ void warp_products(int64_t p0, int64_t p1, int lane, WarpSeg<Acc> &ws,
                                              const int32_t *__restrict__ At_row,
                                              const Acc *__restrict__ At_val, SegFn seg, Body body) {
    warp_products_v<NEED_VAL, 4, Acc>(
        p0, p1, lane, ws, At_row, seg, [&](long long e) { return __ldg(At_val + e); }, body);
}

// Heavy items: the rows of a symbolic item have their bitmap in shared memory
// (at most kSymMaxWords words = 262,144 rows), those of a numeric item their
// packed (bitmap word, prefix) pairs (at most kNumMaxWords words = 65,536
// rows by default: a small table lets four numeric CTAs share an SM).
#ifndef SPG_SYM_MAX_WORDS
#define SPG_SYM_MAX_WORDS 8192
#endif
constexpr int kSymMaxWords = SPG_SYM_MAX_WORDS;
// Launch bound of k_sym_heavy: 0 gives the compiler only the CTA size.
#ifndef SPG_SYM_MINB
#define SPG_SYM_MINB 0
#endif
#if SPG_SYM_MINB > 0
#define SPG_SYM_BOUNDS __launch_bounds__(kBatch, SPG_SYM_MINB)
#else
#define SPG_SYM_BOUNDS __launch_bounds__(kBatch)
#endif
#ifndef SPG_NUM_MAX_WORDS
#define SPG_NUM_MAX_WORDS 2048
#endif
constexpr int kNumMaxWords = SPG_NUM_MAX_WORDS;
// Smallest entry capacity of a numeric item (the capacity is max(this, R) so
// that one base slab always fits).
#ifndef SPG_NUM_CAP_MIN
#define SPG_NUM_CAP_MIN 4096
#endif
constexpr int kNumCapMin = SPG_NUM_CAP_MIN;
// C and the heavy bitmaps pass through L2 once; storing (and reading the
// bitmaps) with the evict-first hint keeps A~, which the products re-read,
// resident instead.
#ifndef SPG_STREAM_HINTS
#define SPG_STREAM_HINTS 1
#endif
template <typename T>
__device__ __forceinline__ void st_stream(T *p, T v) {
#if SPG_STREAM_HINTS
    __stcs(p, v);
#else
    *p = v;
#endif
}
template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) {
#if SPG_STREAM_HINTS
    return __ldcs(p);
#else
    return *p;
#endif
}

// Set bit b of a shared bitmap word; with SPG_TEST_FIRST the word is read
// first and the atomic skipped when the bit is already set (bits are only ever
// set during a pass, so a stale read can only cause a redundant atomic).
#ifndef SPG_TEST_FIRST
#define SPG_TEST_FIRST 1
#endif
__device__ __forceinline__ void set_bit_shared(uint32_t *word, uint32_t mask) {
#if SPG_TEST_FIRST
    if ((*(volatile uint32_t *)word & mask) == 0) atomicOr(word, mask);
#else
    atomicOr(word, mask);
#endif
}

// k_num_heavy checks that every product's row is in the symbolic bitmap (1)
// or relies on the two passes enumerating the same products (0: they walk the
// same segments with the same code, and every row lies in exactly one record
// whose bitmap the item loads; the item's entry count is still checked).
#ifndef SPG_CHECK_MEMBERSHIP
#define SPG_CHECK_MEMBERSHIP 0
#endif

// Minimum resident CTAs per SM asked of the compiler for k_num_heavy: four
// (60 registers a thread) fill the register file and the shared memory of an
// SM with the default table; more CTAs hide more of the kernel's latency.
#ifndef SPG_NUM_MINB
#define SPG_NUM_MINB 4
#endif
// Chunks of 32 products each warp keeps in flight in the heavy kernels
// (compile-time tuning knobs).
#ifndef SPG_NUM_UNROLL
#define SPG_NUM_UNROLL 4
#endif
#ifndef SPG_SYM_UNROLL
#define SPG_SYM_UNROLL 8
#endif
#ifndef SPG_HEAVY_THREADS
#define SPG_HEAVY_THREADS 256
#endif
// threads of a heavy-bin CTA = B' entries staged per round by cta_products
constexpr int kBatch = SPG_HEAVY_THREADS;
constexpr int kLongSeg = 32;  // segments this long are walked 32 entries per warp step

__device__ __forceinline__ unsigned hash_row(int r, int shift) {
    return ((unsigned)r * 0x9E3779B1u) >> shift;
}

// Insert row r into an open-addressing table of 2^logS int keys (linear
// probing).  Returns the slot, and sets *fresh when this call created it.
// The table is sized >= 2x its final occupancy, so a free slot is always
// reached; the probe count is still bounded (-1 = table full).
__device__ __forceinline__ int hash_insert(int *keys, int logS, int r, bool *fresh) {
    const int mask = (1 << logS) - 1;
    unsigned h = hash_row(r, 32 - logS);
    volatile int *vk = keys;
    for (int probe = 0; probe <= mask; probe++) {
        int cur = vk[h];
        if (cur == r) {
            *fresh = false;
            return (int)h;
        }
        if (cur == kEmptyKey) {
            int old = atomicCAS(keys + h, kEmptyKey, r);
            if (old == kEmptyKey) {
                *fresh = true;
                return (int)h;
            }
            if (old == r) {
                *fresh = false;
                return (int)h;
            }
        }
        h = (h + 1) & mask;
    }
    *fresh = false;
    return -1;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

}  // namespace spg
