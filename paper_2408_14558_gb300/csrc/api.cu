// C ABI entry points that sit on top of the plan: symbolic, numeric, the
// one-call multiply, statistics and phase inspection.
#include <algorithm>
#include <cstring>

#include "spg_internal.cuh"

namespace spg {
const char *last_error_str();
void clear_error();
}  // namespace spg

using namespace spg;

extern "C" const char *spgemm_last_error(void) { return last_error_str(); }

static thread_local spg_stats g_last_stats;
static thread_local bool g_have_last_stats = false;

namespace spg {
void remember_multiply_stats(const spg_stats &st) {
    g_last_stats = st;
    g_have_last_stats = true;
}
}  // namespace spg

extern "C" spg_status spgemm_last_multiply_stats(spg_stats *st) {
    if (!st || !g_have_last_stats) {
        set_error("no spgemm_1d_multiply has completed on this thread");
        return SPG_INVALID_ARGUMENT;
    }
    *st = g_last_stats;
    return SPG_OK;
}

extern "C" spg_status spgemm_symbolic(spg_plan *p, void *C_colptr, int64_t *nnzC) {
    spg::PhaseRange nvtx_range("spgemm_symbolic");
    clear_error();
    if (!p || !nnzC) {
        set_error("plan and nnzC must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (!p->symbolic_done) {
        spg_status s = run_symbolic(p);
        if (s) return s;
    }
    if (C_colptr) {
        spg_status s = cuda_check(cudaMemcpyAsync(C_colptr, p->Ccolptr, sizeof(int64_t) * (size_t)(p->n + 1),
                                                  cudaMemcpyDeviceToDevice, p->st),
                                  "colptr copy");
        if (s) return s;
    }
    *nnzC = p->nnzC;
    return SPG_OK;
}

extern "C" spg_status spgemm_numeric(spg_plan *p, spg_csc *C) {
    spg::PhaseRange nvtx_range("spgemm_numeric");
    clear_error();
    if (!p || !C) {
        set_error("plan and C must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (!p->symbolic_done) {
        set_error("spgemm_symbolic must run before spgemm_numeric");
        return SPG_INVALID_ARGUMENT;
    }
    if (!C->colptr || (p->nnzC > 0 && (!C->rowidx || !C->vals))) {
        set_error("C arrays must be allocated (nnzC = %lld)", (long long)p->nnzC);
        return SPG_INVALID_ARGUMENT;
    }
    C->nrows = p->m;
    C->ncols = p->n;
    C->nnz = p->nnzC;
    C->ptr_type = SPG_IDX_I64;
    C->idx_type = p->out_idx64 ? SPG_IDX_I64 : SPG_IDX_I32;
    C->val_type = p->acc_f64 ? SPG_VAL_F64 : SPG_VAL_I64;
    spg_status s = run_numeric(p, C);
    if (!s) p->numeric_done = true;
    return s;
}

extern "C" spg_status spgemm_numeric_refresh(spg_plan *p, spg_csc *C) {
    clear_error();
    if (!p || !C) {
        set_error("plan and C must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (!p->numeric_done) {
        set_error("spgemm_numeric must have run once on this plan before a refresh");
        return SPG_INVALID_ARGUMENT;
    }
    spg_status s = copy_operands(p);
    if (!s) s = spgemm_numeric(p, C);
    return s;
}

extern "C" spg_status spgemm_plan_capture(spg_plan *p, spg_csc *C) {
    clear_error();
    if (!p || !C) {
        set_error("plan and C must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (!p->numeric_done) {
        set_error("spgemm_numeric must have run once on this plan before a capture");
        return SPG_INVALID_ARGUMENT;
    }
    spg_status s = cuda_check(cudaStreamSynchronize(p->st), "capture");
    if (s) return s;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    s = cuda_check(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal), "capture (the plan's stream must not be the legacy default stream)");
    if (s) return s;
    spg_status sr = spgemm_numeric_refresh(p, C);
    cudaGraph_t g = nullptr;
    s = cuda_check(cudaStreamEndCapture(p->st, &g), "end capture");
    if (sr) {
        if (g) cudaGraphDestroy(g);
        return sr;
    }
    if (s) return s;
    p->graph = g;
    return cuda_check(cudaGraphInstantiate(&p->graph_exec, g, 0), "graph instantiate");
}

extern "C" spg_status spgemm_plan_replay(spg_plan *p) {
    spg::PhaseRange nvtx_range("spgemm_plan_replay");
    clear_error();
    if (!p || !p->graph_exec) {
        set_error("no captured graph on this plan (spgemm_plan_capture)");
        return SPG_INVALID_ARGUMENT;
    }
    return cuda_check(cudaGraphLaunch(p->graph_exec, p->st), "graph launch");
}

extern "C" spg_status spgemm_plan_stats(const spg_plan *pc, spg_stats *st) {
    clear_error();
    if (!pc || !st) {
        set_error("plan and stats must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    spg_plan *p = const_cast<spg_plan *>(pc);
    spg_status s = cuda_check(cudaStreamSynchronize(p->st), "stats sync");
    if (s) return s;
    if (p->symbolic_done) {
        float ms = 0;
        if (cudaEventQuery(p->ev[5]) == cudaSuccess && cudaEventElapsedTime(&ms, p->ev[4], p->ev[5]) == cudaSuccess)
            p->stats.ms_numeric = ms;
        cudaGetLastError();
    }
    double *group_ms[5] = {&p->stats.ms_gather, &p->stats.ms_sym_light, &p->stats.ms_sym_heavy,
                           &p->stats.ms_num_light, &p->stats.ms_num_heavy};
    for (int g = 0; g < 5; g++) {
        float ms = 0;
        if (p->kev_used[g] && cudaEventElapsedTime(&ms, p->kev[2 * g], p->kev[2 * g + 1]) == cudaSuccess)
            *group_ms[g] = ms;
        cudaGetLastError();
    }
    p->stats.kernel_launches = p->launches;
    *st = p->stats;
    return read_dev_err(p, "stats");
}

static void free_user(const spg_options *opt, void *ptr, size_t bytes) {
    if (!ptr) return;
    if (opt->free)
        opt->free(ptr, bytes, opt->alloc_ctx, opt->stream);
    else if (!opt->alloc)
        cudaFreeAsync(ptr, (cudaStream_t)opt->stream);
}

void *spg::alloc_user(const spg_options *opt, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (opt->alloc) return opt->alloc(bytes, opt->alloc_ctx, opt->stream);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, (cudaStream_t)opt->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

extern "C" spg_status spgemm_1d_multiply(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C) {
    spg::PhaseRange nvtx_range("spgemm_1d_multiply");
    clear_error();
    if (!C || !opt) {
        set_error("C and options must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    if (opt->sizing == SPG_SIZING_LEARNED) return multiply_learned(A, B, opt, C);
    spg_plan *p = nullptr;
    spg_status s = spgemm_plan(A, B, opt, &p);
    if (s) return s;
    int64_t nnz = 0;
    s = spgemm_symbolic(p, nullptr, &nnz);
    void *cp = nullptr, *ri = nullptr, *va = nullptr;
    size_t idxsz = A->idx_type == SPG_IDX_I64 ? 8 : 4;
    if (!s) {
        cp = alloc_user(opt, sizeof(int64_t) * (size_t)(p->n + 1));
        ri = alloc_user(opt, idxsz * (size_t)nnz);
        va = alloc_user(opt, 8 * (size_t)nnz);
        if (!cp || !ri || !va) {
            set_error("allocation of C (%lld nonzeros) failed", (long long)nnz);
            s = SPG_OUT_OF_MEMORY;
        }
    }
    if (!s) {
        spg_csc out{};
        out.colptr = cp;
        out.rowidx = ri;
        out.vals = va;
        s = spgemm_numeric(p, &out);
        if (!s) s = read_dev_err(p, "numeric");
        if (!s) *C = out;
    }
    if (s) {
        std::string keep = last_error_str();
        free_user(opt, cp, sizeof(int64_t) * (size_t)(p ? p->n + 1 : 1));
        free_user(opt, ri, idxsz * (size_t)nnz);
        free_user(opt, va, 8 * (size_t)nnz);
        spgemm_plan_destroy(p);
        set_error("%s", keep.c_str());
        return s;
    }
    spg_stats st{};
    if (spgemm_plan_stats(p, &st) == SPG_OK) remember_multiply_stats(st);
    spgemm_plan_destroy(p);
    return SPG_OK;
}

extern "C" spg_status spgemm_plan_export(const spg_plan *pc, int32_t block, void *H_bits, void *dtilde,
                                         int64_t *n_dtilde, void *fetch, void *At_colptr, void *At_rowidx,
                                         void *At_vals, void *flops) {
    clear_error();
    if (!pc || block < 0 || block >= pc->P) {
        set_error("bad plan or block index");
        return SPG_INVALID_ARGUMENT;
    }
    spg_plan *p = const_cast<spg_plan *>(pc);
    cudaStream_t st = p->st;
    const int64_t g0 = p->dt_base[block], g1 = p->dt_base[block + 1];
    spg_status s = SPG_OK;
    if (n_dtilde) *n_dtilde = g1 - g0;
    if (H_bits && p->W > 0)
        s = cuda_check(cudaMemcpyAsync(H_bits, p->Hbits + (int64_t)block * p->W, sizeof(uint32_t) * (size_t)p->W,
                                       cudaMemcpyDeviceToDevice, st), "export H");
    if (!s && dtilde && g1 > g0)
        s = cuda_check(cudaMemcpyAsync(dtilde, p->dtilde + g0, sizeof(int32_t) * (size_t)(g1 - g0),
                                       cudaMemcpyDeviceToDevice, st), "export dtilde");
    if (!s && fetch && p->nfb > 0)
        s = cuda_check(cudaMemcpyAsync(fetch, p->fetch + (int64_t)block * p->nfb, (size_t)p->nfb,
                                       cudaMemcpyDeviceToDevice, st), "export fetch");
    if (!s && (At_colptr || At_rowidx || At_vals)) {
        int64_t hb[2];
        s = cuda_check(cudaMemcpyAsync(p->h_pinned, p->At_colptr + g0, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "e");
        if (!s) s = cuda_check(cudaMemcpyAsync(p->h_pinned + 1, p->At_colptr + g1, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "e");
        if (!s) s = cuda_check(cudaStreamSynchronize(st), "export");
        hb[0] = p->h_pinned[0];
        hb[1] = p->h_pinned[1];
        if (!s && At_colptr)
            s = cuda_check(cudaMemcpyAsync(At_colptr, p->At_colptr + g0, sizeof(int64_t) * (size_t)(g1 - g0 + 1),
                                           cudaMemcpyDeviceToDevice, st), "export At colptr");
        if (!s && At_rowidx && hb[1] > hb[0])
            s = cuda_check(cudaMemcpyAsync(At_rowidx, p->At_row + hb[0], sizeof(int32_t) * (size_t)(hb[1] - hb[0]),
                                           cudaMemcpyDeviceToDevice, st), "export At rows");
        if (!s && At_vals && hb[1] > hb[0])
            s = cuda_check(cudaMemcpyAsync(At_vals, (char *)p->At_val + 8 * hb[0], 8 * (size_t)(hb[1] - hb[0]),
                                           cudaMemcpyDeviceToDevice, st), "export At vals");
    }
    if (!s && flops) {
        const int64_t c0 = p->bounds_h[block], c1 = p->bounds_h[block + 1];
        if (c1 > c0)
            s = cuda_check(cudaMemcpyAsync(flops, p->flops + c0, sizeof(int64_t) * (size_t)(c1 - c0),
                                           cudaMemcpyDeviceToDevice, st), "export flops");
    }
    if (!s) s = cuda_check(cudaStreamSynchronize(st), "export");
    return s;
}

extern "C" spg_status spgemm_plan_blocks(const spg_plan *pc, int64_t *bounds, int64_t *flops, int64_t *gathered,
                                         int64_t *remote) {
    clear_error();
    if (!pc) {
        set_error("plan must not be NULL");
        return SPG_INVALID_ARGUMENT;
    }
    spg_plan *p = const_cast<spg_plan *>(pc);
    const int P = p->P;
    if (bounds) std::copy(p->bounds_h.begin(), p->bounds_h.end(), bounds);
    spg_status s = SPG_OK;
    int64_t *dst[3] = {flops, gathered, remote};
    for (int q = 0; q < 3 && !s; q++)
        if (dst[q])
            s = cuda_check(cudaMemcpyAsync(dst[q], p->blk + (int64_t)q * P, sizeof(int64_t) * (size_t)P,
                                           cudaMemcpyDeviceToHost, p->st), "block counters");
    if (!s) s = cuda_check(cudaStreamSynchronize(p->st), "block counters");
    return s;
}
