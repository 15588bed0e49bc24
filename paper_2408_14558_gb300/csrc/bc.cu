// Batched Brandes betweenness centrality (Section 3.2) with the column 1D
// SpGEMM inside both phases, for one batch of s sources on an unweighted
// graph A (n x n; column v lists the neighbours of v, values ignored).
//   forward search  F_0 holds one entry per source (its own vertex, sigma 1);
//                   F_{d+1} = A * F_d masked by the complement of the visited
//                   bitmap (s x n bits): its values are the shortest-path
//                   counts sigma of the newly reached (vertex, source) pairs;
//                   k_bc_mark then adds them to the visited bitmap
//   backward sweep  W_d = (1 + delta_d) / sigma_d on F_d's pattern,
//                   T = A * W_d masked by F_{d-1}'s pattern (a bitmap built by
//                   k_bc_mark), delta_{d-1} = T times sigma_{d-1} on F_{d-1}'s
//                   entries (k_bc_weights, k_bc_delta), added into bc for
//                   d - 1 >= 1
// Both masks are applied inside the SpGEMM (symbolic and numeric passes), so
// no product outside them is counted or stored.
// A frontier column j belongs to source j; row v of it is vertex v.
#include <algorithm>
#include <vector>

#include "spg_internal.cuh"

namespace spg {

const char *last_error_str();
void clear_error();

__global__ void k_bc_ones(double *v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 1.0;
}

// F_0 and the visited bits of the sources.
__global__ void k_bc_init(const int32_t *src, int s, int64_t W, int64_t *colptr, void *rows, int i64, double *vals,
                          uint32_t *V, int *err, int64_t n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= s; i += gridDim.x * blockDim.x) {
        colptr[i] = i;
        if (i == s) break;
        const int64_t v = src[i];
        if (v < 0 || v >= n) {
            atomicOr(err, 1);
            continue;
        }
        if (i64)
            ((int64_t *)rows)[i] = v;
        else
            ((int32_t *)rows)[i] = (int32_t)v;
        vals[i] = 1.0;
        atomicOr(V + (int64_t)i * W + (v >> 5), 1u << (v & 31));
    }
}

__global__ void k_bc_mark(const int64_t *Fcp, const void *Frow, int i64, int64_t s, uint32_t *V, int64_t W) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < s;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5)
        for (int64_t e = Fcp[j] + lane; e < Fcp[j + 1]; e += 32) {
            const int64_t r = ld_ptr(Frow, i64, e);
            atomicOr(V + j * W + (r >> 5), 1u << (r & 31));
        }
}

__global__ void k_bc_weights(const double *sigma, const double *delta, int64_t nnz, double *w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (1.0 + (delta ? delta[i] : 0.0)) / sigma[i];
}

// delta(v, j) = T(v, j) * sigma(v, j) over F(:, j)'s entries (T's column,
// whose rows are a subset of F's, is searched for row v); added into bc[v]
// when `add`.
__global__ void k_bc_delta(const int64_t *Fcp, const void *Frow, const double *Fsig, const int64_t *Tcp,
                           const void *Trow, const double *Tval, int i64, int64_t s, double *delta, double *bc,
                           int add) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < s;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t t0 = Tcp[j], t1 = Tcp[j + 1];
        for (int64_t e = Fcp[j] + lane; e < Fcp[j + 1]; e += 32) {
            const int64_t r = ld_ptr(Frow, i64, e);
            int64_t lo = t0, hi = t1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ld_ptr(Trow, i64, mid) < r)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const double t = (lo < t1 && ld_ptr(Trow, i64, lo) == r) ? Tval[lo] : 0.0;
            const double d = t * Fsig[e];
            delta[e] = d;
            if (add && d != 0.0) atomicAdd(bc + r, d);
        }
    }
}

}  // namespace spg

using namespace spg;

namespace {

struct BcRun {
    const spg_options *opt;
    spg_plan w;  // workspace, stream and launch counting
    std::vector<spg_csc> F;           // frontiers (values sigma)
    std::vector<double *> delta;      // per level, aligned with F's entries

    void free_ptr(void *p, size_t bytes) {
        if (!p) return;
        if (opt->free)
            opt->free(p, bytes, opt->alloc_ctx, opt->stream);
        else if (!opt->alloc)
            cudaFreeAsync(p, (cudaStream_t)opt->stream);
    }
    void free_csc(spg_csc &M) {
        const size_t ib = M.idx_type == SPG_IDX_I64 ? 8 : 4;
        free_ptr(M.colptr, sizeof(int64_t) * (size_t)(M.ncols + 1));
        free_ptr(M.rowidx, ib * (size_t)std::max<int64_t>(M.nnz, 1));
        free_ptr(M.vals, 8 * (size_t)std::max<int64_t>(M.nnz, 1));
        M.colptr = M.rowidx = M.vals = nullptr;
    }
    ~BcRun() {
        for (auto &M : F) free_csc(M);
        for (size_t d = 0; d < delta.size(); d++)
            free_ptr(delta[d], 8 * (size_t)std::max<int64_t>(d < F.size() ? F[d].nnz : 1, 1));
        ws_free_all(&w);
    }
};

spg_status multiply_f64(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C, int64_t *products,
                        spg_bc_stats *S) {
    spg_options o = *opt;
    spg_status s = spgemm_1d_multiply(A, B, &o, C);
    if (s == SPG_OVERFLOW_RECOMPUTED) s = SPG_OK;
    if (!s) {
        spg_stats st{};
        spgemm_last_multiply_stats(&st);
        *products += st.products;
        S->ms_plan += st.ms_plan;
        S->ms_sym_light += st.ms_sym_light;
        S->ms_sym_heavy += st.ms_sym_heavy;
        S->ms_num_light += st.ms_num_light;
        S->ms_num_heavy += st.ms_num_heavy;
        S->ms_gather += st.ms_gather;
        S->multiplies++;
        S->nnzC_total += st.nnzC;
    }
    return s;
}

}  // namespace

extern "C" spg_status spgemm_bc_batch(const spg_csc *A, const int32_t *sources, int32_t s, const spg_options *opt,
                                      double *bc, int64_t *level_nnz, int32_t level_cap, spg_bc_stats *stats) {
    spg::PhaseRange nvtx_range("spgemm_bc_batch");
    clear_error();
    if (!A || !opt || !bc || (s > 0 && !sources) || s < 0 || level_cap < 0) {
        set_error("A, options, bc and (for s > 0) sources must not be NULL; s >= 0");
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->mask) {
        set_error("betweenness masks its own products: pass options without a mask");
        return SPG_INVALID_ARGUMENT;
    }
    if (A->nrows != A->ncols || !A->colptr) {
        set_error("betweenness needs a square adjacency matrix (got %lld x %lld)", (long long)A->nrows,
                  (long long)A->ncols);
        return SPG_INVALID_ARGUMENT;
    }
    spg_bc_stats S{};
    if (s == 0) {
        if (stats) *stats = S;
        return SPG_OK;
    }
    const int64_t n = A->ncols, W = (n + 31) / 32;
    const int i64 = A->idx_type == SPG_IDX_I64;
    const size_t ib = i64 ? 8 : 4;
    cudaStream_t st = (cudaStream_t)opt->stream;
    BcRun run;
    run.opt = opt;
    run.w.opt = *opt;
    run.w.st = st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&run.w.sm_count, cudaDevAttrMultiProcessorCount, dev);
    const int sm = run.w.sm_count;
    spg_plan *w = &run.w;
    cudaEvent_t ev[3];
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], st);
    spg_status rc = SPG_OK;
#define BC_TRY(x)                 \
    do {                          \
        rc = (x);                 \
        if (rc) goto done;        \
    } while (0)
    {
        // the graph with values one, and the first frontier
        spg_csc G = *A;
        G.val_type = SPG_VAL_F64;
        G.vals = ws_alloc(w, sizeof(double) * (size_t)std::max<int64_t>(A->nnz, 1));
        uint32_t *V = (uint32_t *)ws_alloc(w, sizeof(uint32_t) * (size_t)(s * W + 1));
        uint32_t *Mb = (uint32_t *)ws_alloc(w, sizeof(uint32_t) * (size_t)(s * W + 1));
        int *derr = (int *)ws_alloc(w, sizeof(int));
        int64_t *hn = nullptr;
        if (!G.vals || !V || !Mb || !derr) BC_TRY(SPG_OUT_OF_MEMORY);
        BC_TRY(cuda_check(cudaMallocHost(&hn, sizeof(int64_t) * 2), "cudaMallocHost"));
        BC_TRY(cuda_check(cudaMemsetAsync(V, 0, sizeof(uint32_t) * (size_t)(s * W + 1), st), "memset"));
        BC_TRY(cuda_check(cudaMemsetAsync(derr, 0, sizeof(int), st), "memset"));
        if (A->nnz > 0) launch(w, k_bc_ones, grid_for(A->nnz, 256, sm * 8), 256, 0, (double *)G.vals, A->nnz);
        {
            spg_csc F0{};
            F0.nrows = n;
            F0.ncols = s;
            F0.nnz = s;
            F0.ptr_type = SPG_IDX_I64;
            F0.idx_type = A->idx_type;
            F0.val_type = SPG_VAL_F64;
            F0.colptr = alloc_user(opt, sizeof(int64_t) * (size_t)(s + 1));
            F0.rowidx = alloc_user(opt, ib * (size_t)s);
            F0.vals = alloc_user(opt, 8 * (size_t)s);
            run.F.push_back(F0);
            if (!F0.colptr || !F0.rowidx || !F0.vals) BC_TRY(SPG_OUT_OF_MEMORY);
            launch(w, k_bc_init, grid_for(s + 1, 256, sm * 8), 256, 0, sources, (int)s, W, (int64_t *)F0.colptr,
                   F0.rowidx, i64, (double *)F0.vals, V, derr, n);
            BC_TRY(cuda_check(cudaMemcpyAsync(hn, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "sources"));
            BC_TRY(cuda_check(cudaStreamSynchronize(st), "sources"));
            if (*(int *)hn) {
                set_error("a source vertex is outside [0, %lld)", (long long)n);
                BC_TRY(SPG_INVALID_ARGUMENT);
            }
        }
        S.frontier_nnz = s;
        // forward search
        {
            spg_options fo = *opt;
            fo.mask = V;
            fo.mask_words = W;
            fo.mask_complement = 1;
            while (true) {
                spg_csc T{};
                BC_TRY(multiply_f64(&G, &run.F.back(), &fo, &T, &S.products_forward, &S));
                if (T.nnz == 0) {
                    run.free_csc(T);
                    break;
                }
                launch(w, k_bc_mark, grid_for(s * 32, 256, sm * 16), 256, 0, (const int64_t *)T.colptr, T.rowidx,
                       i64, (int64_t)s, V, W);
                run.F.push_back(T);
                BC_TRY(cuda_check(cudaGetLastError(), "frontier kernels"));
                S.frontier_nnz += T.nnz;
            }
        }
        cudaEventRecord(ev[1], st);
        S.levels = (int64_t)run.F.size();
        // backward sweep
        run.delta.assign(run.F.size(), nullptr);
        for (int64_t d = (int64_t)run.F.size() - 1; d >= 1; d--) {
            spg_csc Wd = run.F[d];
            Wd.vals = ws_alloc(w, 8 * (size_t)std::max<int64_t>(Wd.nnz, 1));
            if (!Wd.vals) BC_TRY(SPG_OUT_OF_MEMORY);
            launch(w, k_bc_weights, grid_for(Wd.nnz, 256, sm * 8), 256, 0, (const double *)run.F[d].vals,
                   (const double *)run.delta[d], Wd.nnz, (double *)Wd.vals);
            const spg_csc &Fp = run.F[d - 1];
            BC_TRY(cuda_check(cudaMemsetAsync(Mb, 0, sizeof(uint32_t) * (size_t)(s * W + 1), st), "memset"));
            launch(w, k_bc_mark, grid_for(s * 32, 256, sm * 16), 256, 0, (const int64_t *)Fp.colptr, Fp.rowidx, i64,
                   (int64_t)s, Mb, W);
            spg_options bo = *opt;
            bo.mask = Mb;
            bo.mask_words = W;
            bo.mask_complement = 0;
            spg_csc T{};
            BC_TRY(multiply_f64(&G, &Wd, &bo, &T, &S.products_backward, &S));
            run.delta[d - 1] = (double *)alloc_user(opt, 8 * (size_t)std::max<int64_t>(Fp.nnz, 1));
            if (!run.delta[d - 1]) {
                run.free_csc(T);
                BC_TRY(SPG_OUT_OF_MEMORY);
            }
            launch(w, k_bc_delta, grid_for(s * 32, 256, sm * 16), 256, 0, (const int64_t *)Fp.colptr, Fp.rowidx,
                   (const double *)Fp.vals, (const int64_t *)T.colptr, T.rowidx, (const double *)T.vals, i64,
                   (int64_t)s, run.delta[d - 1], bc, (int)(d - 1 >= 1));
            rc = cuda_check(cudaGetLastError(), "backward kernels");
            run.free_csc(T);
            if (rc) goto done;
        }
        cudaEventRecord(ev[2], st);
        BC_TRY(cuda_check(cudaStreamSynchronize(st), "bc"));
        {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            S.ms_forward = ms;
            cudaEventElapsedTime(&ms, ev[1], ev[2]);
            S.ms_backward = ms;
        }
        if (level_nnz)
            for (int64_t d = 0; d < std::min<int64_t>(S.levels, level_cap); d++) level_nnz[d] = run.F[d].nnz;
        if (stats) *stats = S;
    done:
        if (hn) cudaFreeHost(hn);
    }
#undef BC_TRY
    {
        std::string keep = rc ? std::string(last_error_str()) : std::string();
        cudaStreamSynchronize(st);
        for (auto &e : ev) cudaEventDestroy(e);
        if (rc) set_error("%s", keep.c_str());
    }
    return rc;
}
