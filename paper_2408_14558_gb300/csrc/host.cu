// C = A * B for matrices in host memory: the column 1D multiply (Algorithm 1)
// with the host-device copies inside the call.  B's columns are cut into
// `chunks` groups of consecutive column blocks; every group is planned and
// counted first (so that C's total size is known and its host arrays can be
// requested once), then the groups' numeric passes run in order while the
// part of C computed by the previous group is copied to the host on a second
// stream.
#include <algorithm>
#include <string>
#include <vector>

#include "spg_internal.cuh"

namespace spg {
const char *last_error_str();
void clear_error();
void remember_multiply_stats(const spg_stats &st);
}  // namespace spg

using namespace spg;

namespace {

size_t idx_bytes(int32_t t) { return t == SPG_IDX_I64 ? 8 : 4; }
size_t val_bytes(int32_t t) { return t == SPG_VAL_I32 ? 4 : 8; }

int64_t host_ptr(const void *colptr, int32_t type, int64_t j) {
    return type == SPG_IDX_I64 ? ((const int64_t *)colptr)[j] : (int64_t)((const int32_t *)colptr)[j];
}

bool host_csc_ok(const spg_csc *M) {
    if (!M || M->nrows < 0 || M->ncols < 0 || M->nnz < 0 || !M->colptr) return false;
    if (M->ptr_type < 0 || M->ptr_type > 1 || M->idx_type < 0 || M->idx_type > 1 || M->val_type < 0 ||
        M->val_type > 2)
        return false;
    if (M->nnz > 0 && (!M->rowidx || !M->vals)) return false;
    return host_ptr(M->colptr, M->ptr_type, 0) == 0 && host_ptr(M->colptr, M->ptr_type, M->ncols) == M->nnz;
}

void free_dev(const spg_options *opt, void *p, size_t bytes) {
    if (!p) return;
    if (opt->free)
        opt->free(p, bytes, opt->alloc_ctx, opt->stream);
    else if (!opt->alloc)
        cudaFreeAsync(p, (cudaStream_t)opt->stream);
}

// Everything the call owns, released in one place.
struct HostRun {
    const spg_options *opt = nullptr;
    std::vector<std::pair<void *, size_t>> dev;  // device buffers from the option's allocator
    std::vector<spg_plan *> plans;
    cudaStream_t copy = nullptr;
    std::vector<cudaEvent_t> events;
    void *dev_alloc(size_t bytes) {
        void *p = alloc_user(opt, bytes ? bytes : 16);
        if (p) dev.push_back({p, bytes ? bytes : 16});
        return p;
    }
    ~HostRun() {
        cudaStreamSynchronize((cudaStream_t)opt->stream);
        if (copy) cudaStreamSynchronize(copy);
        for (spg_plan *p : plans) spgemm_plan_destroy(p);
        for (auto &d : dev) free_dev(opt, d.first, d.second);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        if (copy) cudaStreamDestroy(copy);
    }
};

// A device copy of a host CSC matrix (same types).
spg_status to_device(HostRun &run, const spg_csc &H, spg_csc *D, cudaStream_t st) {
    *D = H;
    const size_t pb = idx_bytes(H.ptr_type) * (size_t)(H.ncols + 1);
    const size_t ib = idx_bytes(H.idx_type) * (size_t)H.nnz, vb = val_bytes(H.val_type) * (size_t)H.nnz;
    D->colptr = run.dev_alloc(pb);
    D->rowidx = run.dev_alloc(ib);
    D->vals = run.dev_alloc(vb);
    if (!D->colptr || !D->rowidx || !D->vals) {
        set_error("device copy of a %lld-nonzero input failed", (long long)H.nnz);
        return SPG_OUT_OF_MEMORY;
    }
    spg_status s = cuda_check(cudaMemcpyAsync(D->colptr, H.colptr, pb, cudaMemcpyHostToDevice, st), "input copy");
    if (!s && ib) s = cuda_check(cudaMemcpyAsync(D->rowidx, H.rowidx, ib, cudaMemcpyHostToDevice, st), "input copy");
    if (!s && vb) s = cuda_check(cudaMemcpyAsync(D->vals, H.vals, vb, cudaMemcpyHostToDevice, st), "input copy");
    return s;
}

// A device-to-host copy issued in pieces: the small read-backs of the later
// groups' passes queue on the same copy engine and wait for at most one piece
// instead of the whole transfer.
// True when the GPU can store into [p, p + bytes) through the same pointer:
// page-locked (registered or allocated by CUDA) host memory on a device that
// uses host pointers for registered memory (Grace and other coherent
// systems).  Pageable memory is never written by a kernel here.
bool device_writable_host(const void *p, size_t bytes) {
    if (!p || bytes == 0) return false;
    int dev = 0, can = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&can, cudaDevAttrCanUseHostPointerForRegisteredMem, dev) != cudaSuccess || !can) {
        cudaGetLastError();
        return false;
    }
    for (const char *q : {(const char *)p, (const char *)p + bytes - 1}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer != (const void *)q) return false;
    }
    return true;
}

spg_status copy_back(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    constexpr size_t kPiece = (size_t)128 << 20;
    for (size_t o = 0; o < bytes; o += kPiece) {
        const spg_status s = cuda_check(cudaMemcpyAsync((char *)dst + o, (const char *)src + o,
                                                        std::min(kPiece, bytes - o), cudaMemcpyDeviceToHost, st),
                                        "C read-back");
        if (s) return s;
    }
    return SPG_OK;
}

void add_stats(spg_stats &S, const spg_stats &t) {
    S.products += t.products;
    S.nnzC += t.nnzC;
    S.sum_H += t.sum_H;
    S.sum_dtilde += t.sum_dtilde;
    S.fetch_blocks_total += t.fetch_blocks_total;
    S.fetch_blocks_chosen += t.fetch_blocks_chosen;
    S.gathered_nnz_exact += t.gathered_nnz_exact;
    S.gathered_nnz_block += t.gathered_nnz_block;
    S.gathered_nnz_remote += t.gathered_nnz_remote;
    S.light_columns += t.light_columns;
    S.heavy_columns += t.heavy_columns;
    S.heavy_items += t.heavy_items;
    S.empty_columns += t.empty_columns;
    S.nnzB_heavy += t.nnzB_heavy;
    S.nnzC_heavy += t.nnzC_heavy;
    S.kernel_launches += t.kernel_launches;
    S.ms_plan += t.ms_plan;
    S.ms_symbolic += t.ms_symbolic;
    S.ms_numeric += t.ms_numeric;
    S.ms_gather += t.ms_gather;
    S.ms_sym_light += t.ms_sym_light;
    S.ms_sym_heavy += t.ms_sym_heavy;
    S.ms_num_light += t.ms_num_light;
    S.ms_num_heavy += t.ms_num_heavy;
}

}  // namespace

extern "C" spg_status spgemm_1d_multiply_host(const spg_csc *A, const spg_csc *B, const spg_options *opt,
                                              int32_t chunks, spg_host_alloc_fn host_alloc,
                                              spg_host_free_fn host_free, void *host_ctx, spg_csc *C) {
    spg::PhaseRange nvtx_range("spgemm_1d_multiply_host");
    clear_error();
    if (!opt || !C || !host_alloc || chunks < 1) {
        set_error("options, C and host_alloc must not be NULL; chunks >= 1");
        return SPG_INVALID_ARGUMENT;
    }
    if (!host_csc_ok(A) || !host_csc_ok(B)) {
        set_error("A and B must be host CSC matrices with colptr[0] = 0 and colptr[ncols] = nnz");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A is %lld x %lld, B is %lld x %lld", (long long)A->nrows, (long long)A->ncols,
                  (long long)B->nrows, (long long)B->ncols);
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->sizing != SPG_SIZING_EXACT || opt->P < 1) {
        set_error("the host-buffer multiply runs exact sizing with P >= 1");
        return SPG_INVALID_ARGUMENT;
    }
    cudaStream_t st = (cudaStream_t)opt->stream;
    const int64_t n = B->ncols;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)chunks, (int64_t)opt->P, std::max<int64_t>(n, 1)}));
    HostRun run;
    run.opt = opt;
    spg_status s = cuda_check(cudaStreamCreateWithFlags(&run.copy, cudaStreamNonBlocking), "copy stream");
    if (s) return s;
    // inputs on the device (B is A when both name the same host arrays)
    spg_csc dA{}, dB{};
    s = to_device(run, *A, &dA, st);
    if (s) return s;
    if (B->colptr == A->colptr && B->rowidx == A->rowidx && B->vals == A->vals && B->ptr_type == A->ptr_type &&
        B->idx_type == A->idx_type && B->val_type == A->val_type && B->nrows == A->nrows && B->ncols == A->ncols)
        dB = dA;
    else if ((s = to_device(run, *B, &dB, st)))
        return s;
    // groups of consecutive column blocks: columns [c[g], c[g + 1]), P_g blocks each
    std::vector<int64_t> c(G + 1), e(G + 1);
    std::vector<int> Pg(G);
    for (int g = 0; g <= G; g++) {
        const int64_t blk = (int64_t)g * opt->P / G;
        c[g] = blk * n / opt->P;
        e[g] = host_ptr(B->colptr, B->ptr_type, c[g]);
    }
    for (int g = 0; g < G; g++) Pg[g] = (int)((int64_t)(g + 1) * opt->P / G - (int64_t)g * opt->P / G);
    // the groups' column pointers, rebased to their first entry (int64)
    std::vector<int64_t> cp_h(n + G);
    for (int64_t g = 0, o = 0; g < G; g++) {
        for (int64_t j = c[g]; j <= c[g + 1]; j++) cp_h[o + (j - c[g])] = host_ptr(B->colptr, B->ptr_type, j) - e[g];
        o += c[g + 1] - c[g] + 1;
    }
    int64_t *cp_d = (int64_t *)run.dev_alloc(sizeof(int64_t) * cp_h.size());
    if (!cp_d) {
        set_error("device allocation failed");
        return SPG_OUT_OF_MEMORY;
    }
    s = cuda_check(cudaMemcpyAsync(cp_d, cp_h.data(), sizeof(int64_t) * cp_h.size(), cudaMemcpyHostToDevice, st),
                   "colptr copy");
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "colptr copy");  // cp_h is pageable and goes out of scope
    if (s) return s;
    // plan and count every group
    std::vector<int64_t> nnz(G), off(G + 1, 0);
    std::vector<spg_csc> Bg(G);
    for (int64_t g = 0, o = 0; g < G && !s; g++) {
        spg_csc &M = Bg[g];
        M = dB;
        M.ncols = c[g + 1] - c[g];
        M.nnz = e[g + 1] - e[g];
        M.ptr_type = SPG_IDX_I64;
        M.colptr = cp_d + o;
        M.rowidx = (char *)dB.rowidx + idx_bytes(dB.idx_type) * (size_t)e[g];
        M.vals = (char *)dB.vals + val_bytes(dB.val_type) * (size_t)e[g];
        o += M.ncols + 1;
        spg_options og = *opt;
        og.P = Pg[g];
        if (opt->mask) og.mask = opt->mask + c[g] * opt->mask_words;
        spg_plan *p = nullptr;
        s = spgemm_plan(&dA, &M, &og, &p);
        if (s) break;
        run.plans.push_back(p);
        s = spgemm_symbolic(p, nullptr, &nnz[g]);
        off[g + 1] = off[g] + nnz[g];
    }
    if (s) return s;
    // C's host arrays, then the numeric passes with the copies behind them
    const int64_t total = off[G];
    const size_t ib = A->idx_type == SPG_IDX_I64 ? 8 : 4;
    const bool f64 = A->val_type == SPG_VAL_F64;
    int64_t *hcp = (int64_t *)host_alloc(sizeof(int64_t) * (size_t)(n + 1), host_ctx);
    void *hri = host_alloc(ib * (size_t)std::max<int64_t>(total, 1), host_ctx);
    void *hva = host_alloc(8 * (size_t)std::max<int64_t>(total, 1), host_ctx);
    auto give_back = [&]() {
        if (!host_free) return;
        if (hcp) host_free(hcp, sizeof(int64_t) * (size_t)(n + 1), host_ctx);
        if (hri) host_free(hri, ib * (size_t)std::max<int64_t>(total, 1), host_ctx);
        if (hva) host_free(hva, 8 * (size_t)std::max<int64_t>(total, 1), host_ctx);
    };
    if (!hcp || !hri || !hva) {
        give_back();
        set_error("host allocation of C (%lld nonzeros) failed", (long long)total);
        return SPG_OUT_OF_MEMORY;
    }
    spg_stats S{};
    S.m = A->nrows;
    S.k = A->ncols;
    S.n = n;
    S.nnzA = A->nnz;
    S.nnzB = B->nnz;
    S.P = opt->P;
    S.b = opt->b;
    // every group's numeric set-up (it reads bin sizes back: done before any
    // copy of C occupies the copy engine) and every group's C first
    for (int g = 0; g < G && !s; g++) s = prepare_numeric(run.plans[g]);
    // direct: the numeric kernels store C's rows and values straight into the
    // host arrays (page-locked memory the GPU addresses with the same
    // pointers), with no device copy of C and no copy engine; otherwise each
    // group's part of C is computed on the device and copied back behind it
    const bool direct = total > 0 && device_writable_host(hri, ib * (size_t)total) &&
                        device_writable_host(hva, 8 * (size_t)total);
    std::vector<spg_csc> Cg(G);
    for (int g = 0; g < G && !s; g++) {
        Cg[g].colptr = run.plans[g]->Ccolptr;
        if (direct) {
            Cg[g].rowidx = (char *)hri + ib * (size_t)off[g];
            Cg[g].vals = (char *)hva + 8 * (size_t)off[g];
            continue;
        }
        Cg[g].rowidx = run.dev_alloc(ib * (size_t)nnz[g]);
        Cg[g].vals = run.dev_alloc(8 * (size_t)nnz[g]);
        if (!Cg[g].rowidx || !Cg[g].vals) {
            set_error("device allocation of C's group %d failed", g);
            s = SPG_OUT_OF_MEMORY;
        }
    }
    // the numeric passes back to back on opt->stream; group g's copies wait
    // only for its own pass, so they run while the later groups compute
    for (int g = 0; g < G && !s; g++) {
        s = spgemm_numeric(run.plans[g], &Cg[g]);
        if (direct) continue;
        cudaEvent_t ev = nullptr;
        if (!s) s = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        if (ev) run.events.push_back(ev);
        if (!s) s = cuda_check(cudaEventRecord(ev, st), "event");
        if (!s) s = cuda_check(cudaStreamWaitEvent(run.copy, ev, 0), "event");
        if (!s) s = copy_back((char *)hri + ib * (size_t)off[g], Cg[g].rowidx, ib * (size_t)nnz[g], run.copy);
        if (!s) s = copy_back((char *)hva + 8 * (size_t)off[g], Cg[g].vals, 8 * (size_t)nnz[g], run.copy);
    }
    for (int g = 0; g < G && !s; g++) {
        s = read_dev_err(run.plans[g], "numeric");
        spg_stats t{};
        if (!s && spgemm_plan_stats(run.plans[g], &t) == SPG_OK) add_stats(S, t);
    }
    if (!s) s = cuda_check(cudaStreamSynchronize(run.copy), "C read-back");
    if (!s && direct) s = cuda_check(cudaStreamSynchronize(st), "C stores");
    // the groups' own column pointers (small), rebased into C's
    std::vector<int64_t> lcp(n + G);
    for (int64_t g = 0, o = 0; g < G && !s; g++) {
        s = cuda_check(cudaMemcpy(lcp.data() + o, run.plans[g]->Ccolptr,
                                  sizeof(int64_t) * (size_t)(c[g + 1] - c[g] + 1), cudaMemcpyDeviceToHost),
                       "colptr read-back");
        o += c[g + 1] - c[g] + 1;
    }
    if (s) {
        std::string keep = last_error_str();
        // copies already queued may still be writing into C's host arrays
        cudaStreamSynchronize(run.copy);
        cudaStreamSynchronize(st);
        give_back();
        set_error("%s", keep.c_str());
        return s;
    }
    for (int64_t g = 0, o = 0; g < G; g++) {
        for (int64_t j = c[g]; j <= c[g + 1]; j++) hcp[j] = off[g] + lcp[o + (j - c[g])];
        o += c[g + 1] - c[g] + 1;
    }
    if (n == 0) hcp[0] = 0;
    C->nrows = A->nrows;
    C->ncols = n;
    C->nnz = total;
    C->ptr_type = SPG_IDX_I64;
    C->idx_type = A->idx_type;
    C->val_type = f64 ? SPG_VAL_F64 : SPG_VAL_I64;
    C->reserved = 0;
    C->colptr = hcp;
    C->rowidx = hri;
    C->vals = hva;
    remember_multiply_stats(S);
    return SPG_OK;
}

extern "C" int32_t spgemm_host_writable(const void *ptr, size_t bytes) {
    return device_writable_host(ptr, bytes) ? 1 : 0;
}
