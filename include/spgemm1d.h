/*
 * spgemm1d.h -- C ABI of the GB300 sparsity-aware 1D SpGEMM, C = A * B.
 *
 * The operation (Section 2, problem statement; Section 3.1, Algorithm 1):
 * A is m x k, B is k x n, C is m x n, all in compressed sparse column (CSC)
 * form.  B and C are split into P column blocks; block i holds columns
 * [floor(i*n/P), floor((i+1)*n/P)) (Algorithm 1 only asks that the n_i sum
 * to n).  For every block the library
 *   1. marks H_i, the nonzero rows of B_i (Table 1; Algorithm 1, step on H_i),
 *   2. forms the required column ids D~_i = H_i AND D, D = nonempty columns of
 *      A (Algorithm 1, step on D~), and chooses fetch blocks of b consecutive
 *      column ids, a block being chosen iff it holds a required column
 *      (Algorithm 2 with fixed-width groups),
 *   3. gathers A~_i = A(:, D~_i), reading A one chosen fetch block per work
 *      unit (Algorithm 1, one-sided fetch and "new sparse matrix" steps),
 *   4. counts per output column the sparse flops (Section 3.2) and bins the
 *      columns,
 *   5. runs a symbolic pass giving nnz(C(:,j)) and the column pointers of C,
 *   6. runs a numeric pass giving the sorted rows and values of C
 *      (Algorithm 1, local multiply C_i = A~_i * B_i, Gustavson form).
 *
 * Result contract: a position (r, j) of C is present iff at least one product
 * a_rk * b_kj exists (sums that cancel to zero stay stored); rows within a
 * column strictly increase; integer values use the (+, x) semiring on 64-bit
 * two's-complement words (wrapping); double values are sums in an unspecified
 * order (each entry within 1e-12 * sum |a_rk * b_kj| of the exact sum).
 *
 * Conventions shared by every entry point:
 *   - Matrix arrays are DEVICE pointers owned by the caller.  Inputs must be
 *     canonical: colptr[0] = 0, non-decreasing, colptr[ncols] = nnz, row ids
 *     in [0, nrows) and strictly increasing within each column.  With
 *     spg_options.validate = 1 (the default of spgemm_default_options) the
 *     plan checks this and returns SPG_INVALID_INPUT otherwise.
 *   - All work is ordered on spg_options.stream (a cudaStream_t; NULL is the
 *     legacy default stream).  Only the calls documented as synchronising wait
 *     on the host.
 *   - Errors are returned as spg_status; spgemm_last_error() gives a message
 *     for the calling thread.  No C++ exception crosses this boundary.
 *   - A, B and C may not alias.  A plan keeps pointers to A and B: they must
 *     stay valid and unchanged until spgemm_plan_destroy.
 */
#ifndef SPGEMM1D_H
#define SPGEMM1D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPG_OK = 0,
    SPG_INVALID_ARGUMENT = 1,   /* null pointer, bad enum, dimension mismatch (A.ncols != B.nrows) */
    SPG_INVALID_INPUT = 2,      /* input not canonical: colptr not monotone, row out of range / unsorted / repeated */
    SPG_OUT_OF_MEMORY = 3,      /* a workspace or output allocation failed */
    SPG_CUDA_ERROR = 4,         /* a CUDA runtime call or kernel launch failed */
    SPG_TIMEOUT = 5,            /* a bounded device-side wait gave up (batched executor) */
    SPG_UNSUPPORTED = 6,        /* sizes beyond this build's limits (e.g. m >= 2^31) */
    SPG_OVERFLOW_RECOMPUTED = 7 /* informational: learned sizing under-predicted some columns, they were recomputed exactly */
} spg_status;

typedef enum { SPG_IDX_I32 = 0, SPG_IDX_I64 = 1 } spg_index_type;
typedef enum { SPG_VAL_F64 = 0, SPG_VAL_I32 = 1, SPG_VAL_I64 = 2 } spg_value_type;
typedef enum { SPG_SIZING_EXACT = 0, SPG_SIZING_LEARNED = 1 } spg_sizing;
/* How B's columns are cut into the P blocks: uniformly, [floor(i*n/P),
 * floor((i+1)*n/P)) (Algorithm 1), or contiguously with balanced flops
 * (Section 3.2 count as the weight: bound_i is the smallest j whose preceding
 * columns hold at least i/P of all flops). */
typedef enum { SPG_SPLIT_UNIFORM = 0, SPG_SPLIT_FLOPS = 1 } spg_split;
/* The (add, multiply) pair of the product.  This build computes the ordinary
 * (+, x): doubles, or wrapping 64-bit integers (see the result contract). */
typedef enum { SPG_SEMIRING_PLUS_TIMES = 0 } spg_semiring;

/* One CSC matrix.  colptr has ncols + 1 entries of ptr_type; rowidx has nnz
 * entries of idx_type; vals has nnz entries of val_type.  All device memory,
 * owned by the caller.  For an output C the library fills ptr_type = I64,
 * idx_type = the inputs' idx_type and val_type = F64 (double inputs) or I64
 * (integer inputs; I32 inputs are widened before multiplying). */
typedef struct {
    int64_t nrows, ncols, nnz;
    int32_t ptr_type;   /* spg_index_type */
    int32_t idx_type;   /* spg_index_type */
    int32_t val_type;   /* spg_value_type */
    int32_t reserved;
    void *colptr, *rowidx, *vals;
} spg_csc;

/* Device-memory callbacks.  alloc returns a device pointer of at least `bytes`
 * usable in stream order on `stream` (NULL on failure); free releases it.
 * When both are NULL the library uses cudaMallocAsync / cudaFreeAsync. */
typedef void *(*spg_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*spg_free_fn)(void *ptr, size_t bytes, void *ctx, void *stream);

typedef struct {
    int32_t P;              /* number of column blocks, >= 1 */
    int32_t sizing;         /* spg_sizing */
    int64_t b;              /* fetch-block width in column ids of A, >= 1 */
    int32_t validate;       /* 1: check that A and B are canonical */
    int32_t light_max;      /* largest per-column bound handled by the warp hash bins (power of two, 32..1024; 0 = 1024) */
    int32_t slab_rows;      /* rows per base slab of the heavy bins (power of two, 1024..16384; 0 = 4096) */
    int32_t split;          /* spg_split (0 = uniform) */
    void *stream;           /* cudaStream_t */
    spg_alloc_fn alloc;
    spg_free_fn free;
    void *alloc_ctx;
    const void *model;      /* spg_model* for SPG_SIZING_LEARNED, else NULL */
    double learned_slack;   /* capacity = ceil(slack * predicted nnz) for learned sizing (0 = 1.25) */
    /* Optional structural output mask (the masked product C<M> = A*B that the
     * batched betweenness search of Section 3.2 multiplies with; NULL = none).
     * Column j of C keeps row r iff bit (r & 31) of mask[j * mask_words +
     * (r >> 5)] is set, inverted when mask_complement = 1.  An entry of A*B
     * outside the mask is neither counted nor stored; entries inside it are
     * exactly those of A*B.  Device memory of n * mask_words words owned by the
     * caller; the symbolic and numeric passes (and a refresh or graph replay of
     * the plan) read it, so it must stay valid and unchanged until the plan is
     * destroyed.  Not available with learned sizing, spgemm_outer_multiply or
     * spgemm_bc_batch (which masks its own products): those return
     * SPG_INVALID_ARGUMENT. */
    const uint32_t *mask;
    int64_t mask_words;     /* words per column of mask, >= ceil(nrows(A) / 32) */
    int32_t mask_complement; /* 0: keep rows whose bit is set; 1: keep rows whose bit is clear */
    int32_t semiring;       /* spg_semiring (0 = PLUS_TIMES, the only one; others give SPG_UNSUPPORTED) */
} spg_options;

/* Counters of one plan (filled progressively by plan, symbolic and numeric). */
typedef struct {
    int64_t m, k, n, nnzA, nnzB, P, b;
    int64_t products;            /* sum_j flops_j = <colnnz(A), rownnz(B)> (Section 3.2) */
    int64_t nnzC;                /* -1 until the symbolic pass ran */
    int64_t sum_H;               /* sum_i |H_i| */
    int64_t sum_dtilde;          /* sum_i |D~_i| */
    int64_t fetch_blocks_total;  /* P * ceil(k / b) */
    int64_t fetch_blocks_chosen; /* sum_i M_i of Algorithm 2 */
    int64_t gathered_nnz_exact;  /* nonzeros copied into all A~_i */
    int64_t gathered_nnz_block;  /* nonzeros inside the chosen fetch blocks (block-granular volume) */
    int64_t light_columns, heavy_columns, heavy_items, empty_columns;
    int64_t recomputed_columns;  /* learned sizing: columns that overflowed their predicted capacity */
    int64_t nnzB_heavy;          /* nonzeros of B in the heavy (dense-slab) columns */
    int64_t nnzC_heavy;          /* nonzeros of C in the heavy columns (-1 before symbolic) */
    int64_t kernel_launches;     /* kernels this plan launched so far */
    int64_t learned_capacity;    /* learned sizing: sum of the predicted column capacities (0 otherwise) */
    double ms_plan, ms_symbolic, ms_numeric; /* device time of each phase (CUDA events) */
    /* device time of kernel groups (CUDA events on the plan's stream):
     * gather = A~ copy; sym/num light = all warp-hash bins; sym/num heavy = dense slabs */
    double ms_gather, ms_sym_light, ms_sym_heavy, ms_num_light, ms_num_heavy;
    int64_t gathered_nnz_remote; /* of gathered_nnz_exact, the entries whose column lies outside the block's own
                                    column block of A (what a distributed run fetches from other owners) */
} spg_stats;

typedef struct spg_plan spg_plan;

/* Fill *opt with defaults: P = 1, b = 1024, exact sizing, validate = 1,
 * default stream, library allocator. */
void spgemm_default_options(spg_options *opt);

/*
 * Steps 1-4 above for all P blocks (Algorithm 1 up to the local multiply,
 * Algorithm 2).  Reads A and B, allocates and owns the plan's workspace.
 * Synchronises the stream a few times (to size the workspace).
 * Errors: SPG_INVALID_ARGUMENT (null, P < 1, b < 1, A.ncols != B.nrows,
 * bad type codes, mismatched A/B value types, an output mask with fewer than
 * ceil(nrows(A) / 32) words per column, mask_complement not 0 or 1, or a mask
 * with learned sizing), SPG_INVALID_INPUT,
 * SPG_UNSUPPORTED (a semiring other than SPG_SEMIRING_PLUS_TIMES),
 * SPG_UNSUPPORTED (m, k, n or the gathered column count >= 2^31),
 * SPG_OUT_OF_MEMORY, SPG_CUDA_ERROR.  On error *out is NULL.
 */
spg_status spgemm_plan(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_plan **out);

/*
 * Step 5: exact nnz per column of C.  Writes the n + 1 int64 column pointers
 * of C into C_colptr (device, caller-allocated, may be NULL to skip) and the
 * total into *nnzC (host).  Synchronises the stream once (the total is read
 * back so that the caller can allocate C).
 */
spg_status spgemm_symbolic(spg_plan *plan, void *C_colptr, int64_t *nnzC);

/*
 * Step 6: fill C.  C->colptr must hold the column pointers written by
 * spgemm_symbolic (int64, n + 1), C->rowidx room for nnzC entries of the
 * inputs' idx_type and C->vals room for nnzC doubles (double inputs) or int64
 * (integer inputs).  C's size fields and type codes are set by this call.
 * The first call for a plan synchronises the stream once (the sizes of the
 * light columns' bins are read back); otherwise stream-ordered.
 */
spg_status spgemm_numeric(spg_plan *plan, spg_csc *C);

/*
 * plan + symbolic + numeric + destroy in one call.  C's three arrays are
 * allocated through opt->alloc (or cudaMallocAsync) and belong to the caller
 * afterwards (release them with the matching free).  With opt->sizing =
 * SPG_SIZING_LEARNED the symbolic pass is replaced by the model's prediction
 * and an exact recompute of the columns that overflow; the result is
 * identical and the call returns SPG_OVERFLOW_RECOMPUTED when any column was
 * recomputed.
 */
spg_status spgemm_1d_multiply(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C);

/*
 * Repeated products with fixed patterns (an extension beyond the paper):
 * after one spgemm_numeric on the plan, new values in A's and B's value
 * arrays (same pointers, same patterns) are taken up by
 * spgemm_numeric_refresh, which re-gathers A~'s values, re-maps B's and runs
 * the numeric pass into C (C->colptr as for spgemm_numeric).  It only
 * launches kernels, so spgemm_plan_capture can record it once as a CUDA graph
 * (on the plan's stream, which must not be the legacy default stream; C's
 * arrays are captured by address) and spgemm_plan_replay launches that graph.
 * Errors: SPG_INVALID_ARGUMENT (NULL pointers, no numeric pass yet, nothing
 * captured), SPG_CUDA_ERROR.
 */
spg_status spgemm_numeric_refresh(spg_plan *plan, spg_csc *C);
spg_status spgemm_plan_capture(spg_plan *plan, spg_csc *C);
spg_status spgemm_plan_replay(spg_plan *plan);

/* Copy the plan's counters into *st (host).  Synchronises the stream. */
spg_status spgemm_plan_stats(const spg_plan *plan, spg_stats *st);

/* Counters of the last successful spgemm_1d_multiply on the calling thread
 * (its plan is gone by then; this keeps a copy).  SPG_INVALID_ARGUMENT if
 * there was none. */
spg_status spgemm_last_multiply_stats(spg_stats *st);

/* Per-block diagnostics of a plan (host arrays, any may be NULL): bounds
 * (P + 1 column ids of B's blocks), flops (P, Section 3.2 count per block),
 * gathered (P, nonzeros of A~_i) and remote (P, those of A~_i whose column lies
 * outside the block's own column block of A: the communication volume of a
 * distributed run; the Discussion's CV/memA is their mean over nnz(A)).
 * Synchronises the stream.  SPG_INVALID_ARGUMENT for a NULL plan. */
spg_status spgemm_plan_blocks(const spg_plan *plan, int64_t *bounds, int64_t *flops, int64_t *gathered,
                              int64_t *remote);

/* Release the plan and its workspace (stream-ordered).  NULL is a no-op. */
spg_status spgemm_plan_destroy(spg_plan *plan);

/* Message describing the last error on the calling thread ("" if none). */
const char *spgemm_last_error(void);

/*
 * Phase inspection for tests: copy planning quantities of block `block` into
 * caller device buffers (any pointer may be NULL to skip it).
 *   H_bits      : ceil(k/32) uint32 words, bit h set iff row h of B_i is nonzero
 *   dtilde      : |D~_i| int32 required column ids, ascending      (*n_dtilde receives |D~_i|)
 *   fetch       : ceil(k/b) uint8 flags of the chosen fetch blocks
 *   At_colptr   : |D~_i| + 1 int64 column pointers of A~_i into the plan's
 *                 gathered arrays (subtract the first entry to index At_rowidx)
 *   At_rowidx   : int32 rows of A~_i;  At_vals: double or int64 values of A~_i
 *   flops       : n_i int64 sparse flops of the block's output columns
 * Synchronises the stream.
 */
spg_status spgemm_plan_export(const spg_plan *plan, int32_t block, void *H_bits, void *dtilde,
                              int64_t *n_dtilde, void *fetch, void *At_colptr, void *At_rowidx,
                              void *At_vals, void *flops);

/* ---------------------------------------------------------------------------
 * Batched execution (an extension beyond the paper): many independent
 * products C_i = A_i * B_i, each one column block (P = 1), computed by one
 * persistent kernel captured once in a CUDA graph and fed by a device work
 * queue (symbolic tasks of every instance first, then numeric tasks; a
 * numeric task waits, bounded by timeout_ns, for its instance's column
 * pointers).  Limits: int32 row ids; every column of every C_i with at most
 * 1024 products-bound entries (min(flops_j, m_i) <= 1024, SPG_UNSUPPORTED
 * otherwise: use spgemm_1d_multiply); one value kind for all instances.
 * The output of all instances lives in one pool owned by the batch, sized
 * from per-instance bounds sum_j min(flops_j, m_i); the inputs must stay
 * valid and unchanged while the batch exists.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t task_cols;      /* columns per queue task (>= 1; default 64) */
    int32_t warps_per_cta;  /* 4 or 8 (default 8) */
    int64_t timeout_ns;     /* bound of a numeric task's wait (default 2 s) */
    int32_t stall_instance; /* failure test: numeric tasks of this instance wait on a flag nothing sets (-1 = off) */
    int32_t reserved;
} spg_batch_options;

typedef struct spg_batch spg_batch;

void spgemm_batch_default_options(spg_batch_options *opt);
/* Plan the batch: task table, output bounds (one synchronising bounds pass),
 * pools, and the captured graph.  A and B are arrays of `count` matrices. */
spg_status spgemm_batch_create(int32_t count, const spg_csc *A, const spg_csc *B, const spg_batch_options *opt,
                               spg_batch **out);
/* Launch the batch's graph on `stream` (asynchronous). */
spg_status spgemm_batch_execute(spg_batch *batch, void *stream);
/* Synchronise `stream` and report the last execution: SPG_OK, SPG_TIMEOUT
 * (a wait gave up) or SPG_CUDA_ERROR (a consistency check failed). */
spg_status spgemm_batch_status(spg_batch *batch, void *stream);
/* View of instance i's C inside the batch's pools (int64 colptr, int32 rows;
 * device pointers owned by the batch).  Synchronous (reads nnz). */
spg_status spgemm_batch_result(const spg_batch *batch, int32_t i, spg_csc *C);
/* Copy instance i's C (colptr n+1 int64, rows int32, values 8 bytes) into
 * caller device buffers, ordered on `stream`.  Any pointer may be NULL. */
spg_status spgemm_batch_copy_result(const spg_batch *batch, int32_t i, void *colptr, void *rowidx, void *vals,
                                    void *stream);
/* Queue tasks (symbolic and numeric each), pool entries and persistent grid size. */
spg_status spgemm_batch_info(const spg_batch *batch, int64_t *ntasks, int64_t *pool_entries, int32_t *grid);
spg_status spgemm_batch_destroy(spg_batch *batch);

/* ---------------------------------------------------------------------------
 * Autotuner (an extension beyond the paper): times candidate configurations
 * on the given inputs and returns the fastest; with cache_path (a JSON file,
 * created or updated) the result is stored under the device name and a
 * signature of the workload and reused without timing next time.
 *   spgemm_batch_autotune: task_cols in {16, 64, 256} x warps_per_cta in
 *     {4, 8}, timed on the first `sample` instances (0 = all).
 *   spgemm_autotune: light_max in {256, 512, 1024} x slab_rows in
 *     {2048, 4096, 8192} for the plain path (other fields from `base`).
 * Both synchronise; best_ms (may be NULL) receives the winner's time.
 * ------------------------------------------------------------------------ */
spg_status spgemm_batch_autotune(int32_t count, const spg_csc *A, const spg_csc *B, int32_t sample,
                                 const char *cache_path, spg_batch_options *best, double *best_ms);
spg_status spgemm_autotune(const spg_csc *A, const spg_csc *B, const spg_options *base, const char *cache_path,
                           spg_options *best, double *best_ms);

/* ---------------------------------------------------------------------------
 * Learned nnz sizing (an extension beyond the paper).  A small float32 MLP
 * (4 inputs, two hidden layers of 32 ReLU units, one output) predicts
 * log1p(nnz(C(:,j))) from log1p of four features of column j: flops_j,
 * nnz(B(:,j)), and the largest and mean nnz(A(:,k)) over the k of B(:,j).
 * With spg_options.sizing = SPG_SIZING_LEARNED and .model set,
 * spgemm_1d_multiply sizes every column's output room from the prediction
 * (times learned_slack, at most the exact bound min(flops_j, row window)),
 * runs the numeric work without the symbolic pass and recomputes the columns
 * that overflow through the exact path; C is the exact path's C.  The heavy
 * columns run in groups; each finished group is placed in C while the next
 * one computes, so C's row and value arrays are allocated at the predicted
 * capacity (spg_stats.learned_capacity entries, of which the first nnz(C)
 * hold C).  When a column overflows, C is instead assembled after the
 * recompute, at its exact size.  Learned sizing needs slab_rows <= 4096.
 * Parameters: one flat float vector of SPG_MODEL_NPARAMS entries, laid out
 * W1 (32 x 4, row-major by hidden unit) | b1 (32) | W2 (32 x 32) | b2 (32) |
 * w3 (32) | b3 (1).  X arrays are n x 4 row-major device floats; y, out are
 * n device floats.  All device work runs on `stream`.
 * ------------------------------------------------------------------------ */
#define SPG_MODEL_NPARAMS 1249
typedef struct spg_model spg_model;

/* He-normal weights from `seed` (splitmix64 + Box-Muller), zero biases. */
spg_status spgemm_model_create(uint64_t seed, spg_model **out);
spg_status spgemm_model_destroy(spg_model *model);
/* Host copies of the parameters; set also resets the Adam state. */
spg_status spgemm_model_set_params(spg_model *model, const float *params, int64_t count);
spg_status spgemm_model_get_params(const spg_model *model, float *params, int64_t count);
/* epochs over the n samples in mini-batches of `batch` (in order), one Adam
 * step (beta 0.9 / 0.999, eps 1e-8) per batch; *final_loss (host, may be NULL)
 * receives the mean squared error over all samples afterwards.  Synchronises. */
spg_status spgemm_model_train(spg_model *model, const float *X, const float *y, int64_t n, int32_t epochs,
                              int32_t batch, float lr, void *stream, float *final_loss);
spg_status spgemm_model_predict(const spg_model *model, const float *X, int64_t n, float *out, void *stream);
/* Gradient of the mean squared error over the n samples (host, NPARAMS
 * floats) and the loss; no parameter changes.  Synchronises. */
spg_status spgemm_model_gradient(spg_model *model, const float *X, const float *y, int64_t n, float *grad,
                                 float *loss, void *stream);
/* Binary file: "SPGMLP01", int32 count, count float32 parameters. */
spg_status spgemm_model_save(const spg_model *model, const char *path);
spg_status spgemm_model_load(const char *path, spg_model **out);
/* Training data from a plan: features X (n x 4) of every output column, and
 * after spgemm_symbolic the labels y = log1p(nnz(C(:,j))). */
spg_status spgemm_plan_features(const spg_plan *plan, float *X);
spg_status spgemm_plan_labels(const spg_plan *plan, float *y);

/*
 * nnz(C(:,j)) for every column j of C = A * B, written to nnz_out (device,
 * B.ncols int64 entries, caller-allocated), without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory at all -- a process whose GPU memory is owned
 * entirely by another allocator, a service that reserves its memory once at
 * start-up, or a latency path where an allocation call (which can synchronise
 * the device) is not acceptable.  Its scratch is one fixed array inside the
 * library (8 MiB, held on every GPU that loads the library until the process
 * exits), so:
 *   - A may have at most 1,048,576 rows (SPG_UNSUPPORTED otherwise);
 *   - calls whose kernels overlap on the GPU share that array and race:
 *     order them on one stream;
 *   - the first call on a device looks up the array's address with that
 *     device current (cudaGetSymbolAddress); make that first call before any
 *     stream capture on the device.  The address is kept for the life of the
 *     process, so a cudaDeviceReset of that device between calls is not
 *     supported.
 * Inputs must be canonical (no validation pass: that would need memory for a
 * flag).  Asynchronous on `stream` (a cudaStream_t; NULL = legacy stream).
 * Errors: SPG_INVALID_ARGUMENT, SPG_UNSUPPORTED, SPG_CUDA_ERROR.
 */
spg_status spgemm_count_noalloc(const spg_csc *A, const spg_csc *B, int64_t *nnz_out, void *stream);

/* ---------------------------------------------------------------------------
 * Outer-product 1D SpGEMM (the paper's Algorithm 3, used there for the right
 * multiplication of the Galerkin product): C = sum over the opt->P row blocks
 * K_i = [floor(i*k/P), floor((i+1)*k/P)) of B of A(:, K_i) * B(K_i, :).
 * Steps: B is redistributed by row blocks (B' holds, for every non-empty
 * pair (i, j) in (i, j) order, the entries of B(:, j) in K_i); C' = A * B' by
 * the column 1D path with P column blocks, the columns of row block i reading
 * only A(:, K_i); C = C' * S with S[c, j(c)] = 1 (the merge of the partial
 * results), again by the column 1D path.  The result equals A * B (doubles within the usual
 * rounding bound, integers exactly).
 * A, B: device CSC as for spgemm_1d_multiply; opt: as for spgemm_1d_multiply
 * (P = number of row blocks, b = fetch-block width of both products; learned
 * sizing is ignored).  C: receives int64 column pointers, row ids of A's
 * idx_type and double or int64 values, allocated through opt->alloc (or
 * cudaMallocAsync) and owned by the caller.  B', C' and S are released before
 * the call returns.  stats (host, may be NULL): the volumes a distributed run
 * with process i owning column block i of A, B and C would move.  Synchronises
 * the stream.  Errors: SPG_INVALID_ARGUMENT (NULL pointers, A.ncols != B.nrows,
 * P < 1, options carrying a mask), SPG_UNSUPPORTED (int32 row ids of A with 2^31 or more non-empty
 * (i, j) pairs), and those of spgemm_1d_multiply.
 */
/* ---------------------------------------------------------------------------
 * Batched betweenness centrality (Section 3.2: Brandes' algorithm for a batch
 * of sources, multi-source BFS forward search and backward sweep, each level
 * one masked column 1D SpGEMM: the forward product keeps the (vertex, source)
 * pairs not yet visited, the backward product the pairs of the level above).
 * A: n x n device CSC of an unweighted graph, column v
 * listing the neighbours of v (values ignored; symmetric for an undirected
 * graph).  sources: s device int32 vertex ids (one frontier column each).
 * opt: as for spgemm_1d_multiply (P, b, stream, allocator).  bc: n device
 * doubles to which the batch adds sum over its sources of the Brandes
 * dependency delta_s(v) (zero it before the first batch).  level_nnz (host,
 * may be NULL): the (vertex, source) pairs reached at each BFS level, up to
 * level_cap levels.  stats (host, may be NULL).  Intermediate frontiers live
 * in memory from opt->alloc and are released before the call returns.
 * Synchronises the stream.  Errors: SPG_INVALID_ARGUMENT (NULL pointers,
 * non-square A, s < 0, a source outside [0, n), options carrying a mask), and
 * those of spgemm_1d_multiply.
 */
typedef struct {
    int64_t levels;            /* BFS levels, the sources' own level included */
    int64_t frontier_nnz;      /* (vertex, source) pairs reached over all levels */
    int64_t products_forward;  /* sparse flops of the forward-search products */
    int64_t products_backward; /* sparse flops of the backward-sweep products */
    double ms_forward, ms_backward;
    /* sums over all the batch's SpGEMMs of their spg_stats device times */
    double ms_plan, ms_sym_light, ms_sym_heavy, ms_num_light, ms_num_heavy, ms_gather;
    int64_t multiplies;        /* SpGEMMs the batch ran */
    int64_t nnzC_total;        /* sum of their output nonzeros (all inside the masks) */
} spg_bc_stats;

spg_status spgemm_bc_batch(const spg_csc *A, const int32_t *sources, int32_t s, const spg_options *opt, double *bc,
                           int64_t *level_nnz, int32_t level_cap, spg_bc_stats *stats);

typedef struct {
    int64_t P;
    int64_t products;      /* sum_j flops_j of A * B */
    int64_t nnzB_moved;    /* entries of B whose row block differs from their column block */
    int64_t partial_nnz;   /* nnz(C'): the nonzeros of the P partial products together */
    int64_t partial_moved; /* partial nonzeros of column j computed by a block other than j's owner */
    int64_t nnzC;
    double ms_split, ms_local, ms_merge; /* device time of the three steps (CUDA events) */
} spg_outer_stats;

spg_status spgemm_outer_multiply(const spg_csc *A, const spg_csc *B, const spg_options *opt, spg_csc *C,
                                 spg_outer_stats *stats);

/*
 * C = A * B (Algorithm 1, exact sizing) for matrices in HOST memory, the
 * host-device copies inside the call.  A and B are spg_csc with host pointers
 * (pinned memory for full copy speed; any types spgemm_plan accepts); when B
 * names the same host arrays as A they are copied once.  B's columns are cut
 * into min(chunks, P, n) groups of consecutive column blocks (group g holds
 * blocks [g*P/G, (g+1)*P/G) of the uniform split and multiplies them as a
 * plan of its own); all groups are planned and counted, C's three host
 * arrays are requested from host_alloc (column pointers int64 n + 1, rows of
 * A's idx_type, values double or int64; NULL from it gives SPG_OUT_OF_MEMORY),
 * then each group's numeric pass runs on opt->stream while the previous
 * group's part of C is copied to the host on a stream of the call's own.
 * When C's row and value arrays are page-locked memory that the GPU
 * addresses through the same pointers (spgemm_host_writable), the numeric
 * kernels store C into them directly instead (over the CPU-GPU link, no
 * device copy of C, no copy engine).  The groups also bound the host range
 * the kernels write at once: on a GB300 with Grace host memory, one group
 * writing 35 GB at once ran 2-4x slower than four groups of about 9 GB.
 * Device workspace and device copies come from opt->alloc / opt->free (or
 * cudaMallocAsync) and are released before returning; opt->mask, if set,
 * applies as in spgemm_plan (its columns are C's columns).  Blocks until C is
 * on the host; on success C describes the host arrays, which belong to the
 * caller; on failure any array host_alloc returned is handed to host_free
 * (which may be NULL) and C is untouched.  spgemm_last_multiply_stats then
 * holds the counters and device times summed over the groups.  Errors:
 * SPG_INVALID_ARGUMENT for NULL options / C / host_alloc, chunks < 1, learned
 * sizing, a dimension mismatch or a host colptr whose first entry is not 0 or
 * whose last is not nnz; otherwise as spgemm_plan, spgemm_symbolic and
 * spgemm_numeric.
 */
typedef void *(*spg_host_alloc_fn)(size_t bytes, void *ctx);
/* 1 if kernels can store into the host range [ptr, ptr + bytes) through ptr
 * itself: page-locked memory (cudaHostRegister or cudaMallocHost) on a
 * device with cudaDevAttrCanUseHostPointerForRegisteredMem; 0 otherwise
 * (pageable memory, NULL, bytes = 0). */
int32_t spgemm_host_writable(const void *ptr, size_t bytes);
typedef void (*spg_host_free_fn)(void *ptr, size_t bytes, void *ctx);
spg_status spgemm_1d_multiply_host(const spg_csc *A, const spg_csc *B, const spg_options *opt, int32_t chunks,
                                   spg_host_alloc_fn host_alloc, spg_host_free_fn host_free, void *host_ctx,
                                   spg_csc *C);

/* ---------------------------------------------------------------------------
 * One-launch multiply for small products: C = A * B with B and C cut into P
 * column blocks (Section 3.1, Algorithm 1: per block H_i, D~_i and the chosen
 * fetch blocks of b column ids (Algorithm 2), then the symbolic and numeric
 * passes of the local multiply), every step in ONE cooperative persistent
 * kernel with grid-wide barriers.  The gather of A~_i is fused into the
 * product loads (each required column of A is read in place), so C is that of
 * the column 1D path.  Nothing is read back to the host and nothing is
 * allocated: the call is two clears and one kernel on `stream`, and can be
 * captured in a CUDA graph and replayed.
 *
 * Table classes (table_log): 8 gives every warp 256 slots and runs 32 warps
 * per SM, for products whose column bounds min(flops_j, m) are all <= 128; 10
 * gives 1024 slots and 8 warps per SM, for bounds <= 512.
 *
 * spgemm_small_bound: bound[0] = max_j min(flops_j, m), bound[1] = sum_j
 * min(flops_j, m) (an upper bound of nnz(C), usable as C's capacity), written
 * to `bound` (device, 2 int64) on `stream`; the caller reads them once to
 * choose the table class and allocate C.
 *
 * spgemm_small_workspace: bytes of device workspace the call needs for these
 * shapes, P, b and table class (depends on the sizes only, and on the GPU's
 * SM count).
 *
 * spgemm_small_multiply:
 *   A, B:      device CSC as for spgemm_plan; A's row ids must be int32; A and
 *              B both doubles, or both integers (int32 widened, int64 wrapping).
 *   workspace: device, >= spgemm_small_workspace bytes, caller-owned; its
 *              contents need not be preserved between calls.
 *   C_colptr:  device, n + 1 int64 (written even when C does not fit);
 *   C_rowidx, C_vals: device, `capacity` int32 row ids and `capacity` values
 *              (double, or int64 for integer inputs).
 *   result:    device, 8 int64 written by the kernel: [0] nnz(C), [1] status
 *              (0, or the spg_status of the first failure: SPG_OUT_OF_MEMORY
 *              when nnz(C) > capacity (no rows written), SPG_UNSUPPORTED when a
 *              column's bound min(flops_j, m) exceeds the table class's
 *              limit (128 or 512), SPG_INVALID_INPUT
 *              for a row id of B outside A's columns, SPG_TIMEOUT when a grid
 *              barrier wait exceeded timeout_ns, SPG_CUDA_ERROR for an
 *              internal inconsistency), [2] products, [3] sum of |H_i|,
 *              [4] sum of |D~_i|, [5] nonzeros of the A~_i, [6] nonzeros of
 *              the chosen fetch blocks, [7] chosen fetch blocks.
 *   timeout_ns: limit of each grid-barrier wait (the CTAs of a cooperative
 *              launch are co-resident, so it only guards against faults).
 * Host-side errors (returned): SPG_INVALID_ARGUMENT (NULL pointers, bad
 * header, P < 1, b < 1, dimension mismatch, mixed value kinds, workspace too
 * small, table_log not 8 or 10), SPG_UNSUPPORTED (int64 row ids of A),
 * SPG_CUDA_ERROR (launch).
 * Inputs are not validated beyond the row ids of B.
 */
spg_status spgemm_small_bound(const spg_csc *A, const spg_csc *B, int64_t *bound, void *stream);
spg_status spgemm_small_workspace(const spg_csc *A, const spg_csc *B, int32_t P, int64_t b, int32_t table_log,
                                  size_t *bytes);
spg_status spgemm_small_multiply(const spg_csc *A, const spg_csc *B, int32_t P, int64_t b, int32_t table_log,
                                 void *workspace, size_t workspace_bytes, int64_t *C_colptr, int32_t *C_rowidx,
                                 void *C_vals, int64_t capacity, int64_t *result, int64_t timeout_ns, void *stream);

/* ---------------------------------------------------------------------------
 * Distributed 1D SpGEMM: the device steps of Algorithm 1 (Section 3.1) when P
 * processes each own column block i of A, B and C, with Algorithm 2 choosing
 * what each process fetches.  The transport between processes (NCCL, gloo,
 * or anything else that moves device buffers) belongs to the caller; the
 * Python binding's dist1d module drives these calls around collectives.
 * All three are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 * stream), allocate nothing and take only caller-owned device memory.
 *
 * spgemm_dist_fetch_blocks: process i's H_i (the nonzero rows of its B_i,
 * Table 1) and its chosen fetch blocks: block t = column ids
 * [t*b, min((t+1)*b, k)) is chosen iff it holds a column c with bit c of H_i
 * set and A_colptr[c+1] > A_colptr[c] (D~_i = H_i AND D, Algorithm 1;
 * Algorithm 2 with fixed-width groups).
 *   B:        process i's local block (k x n_i, rows = global column ids of A);
 *             only its row ids are read.
 *   A_colptr: k + 1 int64, the GLOBAL column pointers of A (the per-owner
 *             column counts after an allgather, scanned).
 *   H:        workspace and output, ceil(k/32) uint32 words (bit c = row c).
 *   fetch:    output, ceil(k/b) bytes, 1 = chosen.
 *   bad:      one device int, set to 1 if a row id of B lies outside [0, k)
 *             (such ids are skipped, never used as an address).
 * Errors: SPG_INVALID_ARGUMENT (NULL pointers, bad header, b < 1),
 * SPG_CUDA_ERROR.
 */
spg_status spgemm_dist_fetch_blocks(const spg_csc *B, const int64_t *A_colptr, int64_t b, uint32_t *H,
                                    uint8_t *fetch, int *bad, void *stream);
/* spgemm_dist_pack: an owner's reply to one requester (the one-sided fetch of
 * Algorithm 1, here a send buffer): the entries of local columns
 * [ranges[2r], ranges[2r+1]) of A, range after range, copied to rows_out /
 * vals_out starting at out_off[r].
 *   A:        the owner's local columns (its colptr starts at 0), any index
 *             and value types; the outputs take A's row id and value types.
 *   ranges:   device, 2*nr int64 (local column ids, lo <= hi <= A.ncols).
 *   out_off:  device, nr + 1 int64, out_off[r+1] - out_off[r] = the entries of
 *             range r, out_off[nr] = total.
 *   bad:      one device int, set to 1 if a range lies outside A or its size
 *             disagrees with out_off (offending entries are not copied).
 * Errors: SPG_INVALID_ARGUMENT, SPG_CUDA_ERROR.
 */
spg_status spgemm_dist_pack(const spg_csc *A, const int64_t *ranges, const int64_t *out_off, int64_t nr,
                            int64_t total, void *rows_out, void *vals_out, int *bad, void *stream);
/* spgemm_dist_fetched_colptr: the requester's side.  The fetched pieces,
 * received in ascending column order, form the m x k matrix A_f whose column
 * c equals A(:, c) when c's fetch block was chosen and is empty otherwise;
 * A_f * B_i = A * B_i because every column of D~_i lies in a chosen block.
 * This writes A_f's k + 1 int64 column pointers to colptr_out (device) from
 * the global A_colptr (device, k + 1) and fetch (device, ceil(k/b) bytes).
 * Errors: SPG_INVALID_ARGUMENT, SPG_CUDA_ERROR.
 */
spg_status spgemm_dist_fetched_colptr(const int64_t *A_colptr, const uint8_t *fetch, int64_t k, int64_t b,
                                      int64_t *colptr_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPGEMM1D_H */
