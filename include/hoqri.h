/*
 * hoqri.h: C ABI of the GB300 HOQRI hot path.
 *
 * HOQRI (higher-order QR iteration, arXiv 2510.16930) computes a low
 * multilinear rank (Tucker) approximation X ~ G x {U} of a sparse N-way tensor
 * X (prob. (tucker), Sec. 2.2) with orthonormal factors U_n (I_n x K_n) and the
 * optimal core G = X x {U^T} (Sec. 2.2).  Its hot path (Alg. 2) repeats, for
 * n = 1..N:
 *     A_n <- TTMcTC(X, {U}, n) = Y_(n) G_(n)^T,  Y = X x_{-n} {U^T}   (Eq. ttmctc)
 *     U_n <- an orthonormal basis of A_n via QR                          (Alg. 2)
 * with G recomputed from the current factors before every TTMcTC (Alg. 3,
 * first step).
 *
 * Layouts (all row-major, 0-based):
 *   - COO input: idx[m] is an array of nnz int32 mode-m indices, vals an array
 *     of nnz values.  A coordinate listed more than once denotes ONE entry
 *     whose value is the sum of the listed values.
 *   - U_n: I_n x K_n, element (i, k) at i*K_n + k.
 *   - G: K_1 x ... x K_N with the LAST index fastest, so the columns of the
 *     unfolding G_(n) follow the Kronecker order B^(1) (x) ... (x) B^(N) of
 *     Eq. (2) with mode n skipped.
 *   - A_n: I_n x K_n; rows of X_(n) without nonzeros give zero rows.
 * Element type ("real" below): double for HOQRI_FP64, float otherwise.
 *
 * Pointers: every array argument may point to host memory or to device
 * memory of the context's device; the library tells them apart with
 * cudaPointerGetAttributes.  Inputs are copied: the caller keeps ownership of
 * everything it passes.  Output buffers are allocated by the caller.  Work is
 * ordered on the stream given to hoqri_create; a call that writes a host
 * buffer returns after the data is there, a call that writes only device
 * buffers returns once the work is queued.
 *
 * Errors: every call returns a hoqri_status and never aborts or throws;
 * hoqri_last_error() gives a message for the calling thread's last failure.
 * After HOQRI_ERR_CUDA the context should be destroyed.
 */
#ifndef HOQRI_H
#define HOQRI_H

#include <stdint.h>

#if defined(__GNUC__)
#define HOQRI_API __attribute__((visibility("default")))
#else
#define HOQRI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hoqri_ctx hoqri_ctx; /* opaque; owns all device state of one tensor */

typedef enum {
    HOQRI_OK = 0,
    HOQRI_ERR_INVALID = 1,      /* bad argument, NULL pointer, index out of range */
    HOQRI_ERR_OOM = 2,          /* a device allocation failed */
    HOQRI_ERR_CUDA = 3,         /* a CUDA runtime call or kernel failed */
    HOQRI_ERR_QR_BREAKDOWN = 4, /* Cholesky breakdown with the fallback disabled */
    HOQRI_ERR_RANK = 5,         /* K_n > I_n or K_n > prod_{m != n} K_m */
    HOQRI_ERR_TIMEOUT = 6,      /* a bounded device wait ran out */
    HOQRI_ERR_UNSUPPORTED = 7   /* shape or precision outside the library's kernels */
} hoqri_status;

typedef enum {
    HOQRI_FP64 = 0,  /* values, factors, core and A_n in double */
    HOQRI_FP32 = 1,  /* float on the nonzero streams; Gram, Cholesky and fit in double */
    HOQRI_BF16X3 = 2 /* FP32 storage; Kronecker-times-core products on the tensor
                        cores in split BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate */
} hoqri_precision;

typedef struct {
    int32_t prec;       /* hoqri_precision */
    int32_t qr_kind;    /* 0: CholeskyQR2 in FP64 (shifted CholeskyQR3 when the first
                           pivot is not clearly positive), Householder when that breaks
                           down too; 1: Householder only; 2: as 0, but a breakdown
                           is an error (HOQRI_ERR_QR_BREAKDOWN) */
    int32_t chunk_nnz;  /* nonzeros per warp task; 0 = chosen by the library */
    int32_t autotune;   /* 1: at create, time candidate layouts of the nonzero-stream
                           pass per mode (long-row threshold, work-item size) and keep
                           the fastest; cached per problem kind, and in the file named by
                           the environment variable HOQRI_TUNE_CACHE if set */
    int32_t use_graphs; /* 1: hoqri_iterate replays one sweep as a CUDA graph */
    int32_t one_stream; /* 0/1: FP32 modes with a register-tile plan stream their nonzeros
                           once per block update and keep Y_(n) (R_n x P_{-n} floats) for
                           the core G = U_n^T Y_(n) (sliced pass); 2: the paper's O(IK)
                           memory form (separate core pass, no Y); 3: as 0, through the
                           fiber-factored pass where the shape has one (order 3 or 4,
                           other ranks powers of two >= 4, P_{-n} <= 1024) */
    uint64_t seed;      /* seed of the initial factors when U0 is NULL */
    double tol;         /* hoqri_run: stop after the first sweep whose residual differs
                           from the previous one by less than tol (0: never) */
    int32_t tile_rows;  /* FP32 sliced pass: accumulators per lane along the Kronecker
                           prefix (8 or 4) and along the last mode (tile_cols, 8 or 4),
                           for every mode whose plan allows it; 0, 0: the plan's tile
                           (8 x 8 where the ranks allow), or the autotuner's choice */
    int32_t tile_cols;
} hoqri_options;

/* Fills *opt with the defaults (FP32, CholeskyQR2 + fallback, library-chosen
 * chunk, no autotune, graphs on, seed 0, tol 0, the plan's lane tile). */
HOQRI_API void hoqri_default_options(hoqri_options *opt);

/*
 * Builds the device state for one sparse tensor (Sec. 6: COO storage) and the
 * initial factors (Alg. 2, first step).
 *   N        order, 2 <= N <= 8
 *   dims     N mode sizes, 1 <= I_n < 2^31
 *   ranks    N multilinear ranks K_n, 1 <= K_n <= 64 and K_n <= I_n and
 *            K_n <= prod_{m != n} K_m (else HOQRI_ERR_RANK: A_n would be rank
 *            deficient by construction; the paper is silent on this case)
 *   nnz      number of listed entries (repeats allowed; they are summed), >= 0
 *   idx      N pointers to nnz int32 indices each, 0 <= idx[m][z] < dims[m]
 *   vals     nnz reals
 *   opt      options (NULL: defaults)
 *   U0       NULL, or N pointers to I_n x K_n reals with orthonormal columns
 *            (not checked); NULL draws a seeded Gaussian and orthonormalises it
 *   stream   cudaStream_t to order all work on (NULL: the legacy default stream;
 *            on a created stream the context's device memory is allocated
 *            stream-ordered from the library's pool, see hoqri_trim_memory)
 * Duplicates are summed, then one mode-sorted copy of the nonzeros per mode is
 * built with its permutation and row (slice) descriptors; the raw input is
 * released before returning.  On failure *out is NULL.
 */
HOQRI_API hoqri_status hoqri_create(hoqri_ctx **out, int32_t N, const int64_t *dims, const int32_t *ranks,
                          int64_t nnz, const int32_t *const *idx, const void *vals,
                          const hoqri_options *opt, const void *const *U0, void *stream);

/* G = X x_1 U_1^T ... x_N U_N^T with the current factors (Sec. 2.2; Alg. 2
 * last step).  G_out: prod K_n reals, layout above. */
HOQRI_API hoqri_status hoqri_core(hoqri_ctx *ctx, void *G_out);

/* A_n = TTMcTC(X, {U}, n) with the current factors (Eq. ttmctc; Alg. 3: the core
 * is recomputed first).  mode is 0-based; A_out: I_n x K_n reals.  The factors
 * are not changed. */
HOQRI_API hoqri_status hoqri_ttmctc(hoqri_ctx *ctx, int32_t mode, void *A_out);

/* U_out = orthonormal basis of the columns of A_in (Alg. 2, the QR step): thin QR
 * with diag(R) > 0 by CholeskyQR2 in FP64 (shifted CholeskyQR3 for an
 * ill-conditioned A_in, Householder on breakdown, per qr_kind).  A_in: I_mode x K_mode reals; U_out may equal A_in.  The factors of
 * the context are not changed. */
HOQRI_API hoqri_status hoqri_orthonormalize(hoqri_ctx *ctx, int32_t mode, const void *A_in, void *U_out);

/*
 * Runs `iters` HOQRI iterations (Alg. 2; one iteration = one sweep n = 1..N of
 * core, TTMcTC and QR), then the final core.  resid_hist (host, NULL or iters
 * doubles) receives after each sweep the relative residual
 *   r = sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||,
 * which equals ||X - G x {U}|| / ||X|| for orthonormal U and optimal G (Sec. 2.2).
 */
HOQRI_API hoqri_status hoqri_iterate(hoqri_ctx *ctx, int32_t iters, double *resid_hist);

/*
 * Runs sweeps of Alg. 2 as hoqri_iterate does, at most max_iters of them, and
 * stops after the first sweep t whose residual satisfies |r_t - r_{t-1}| < tol
 * (options.tol; r_0 is the residual of the core before the first sweep): the
 * stopping rule of Sec. 6.1.  With tol = 0 every sweep runs.  Each sweep then
 * ends with a device-to-host read of its residual (the stream is synchronised
 * once per sweep).  resid_hist (host, NULL or max_iters doubles) receives
 * r_1 .. r_done; iters_done (host, NULL allowed) the number of sweeps run.  The
 * results of the sweeps that ran are identical to those of hoqri_iterate with
 * that count.  Errors: HOQRI_ERR_INVALID for max_iters < 0 or tol < 0, else as
 * hoqri_iterate.
 */
HOQRI_API hoqri_status hoqri_run(hoqri_ctx *ctx, int32_t max_iters, double *resid_hist, int32_t *iters_done);

/*
 * ||grad f||^2 at the current factors, f = ||X x {U^T}||^2 on the product of
 * Stiefel manifolds (Sec. 5, Eq. tucker_grad and Eq. grad2):
 * sum_n ||2 A_n - 2 U_n G_(n) G_(n)^T||_F^2 with A_n = TTMcTC(X, {U}, n) and G
 * the core of the current factors; zero exactly at a stationary point
 * (Def. stationary).  Each mode's term is formed row by row and summed in FP64
 * in a fixed order.  Costs one core pass and one TTMcTC pass per mode; the
 * factors are not changed (the context's core is left at that of the last
 * mode).  out: host double.  Errors: HOQRI_ERR_INVALID for a NULL out.
 */
HOQRI_API hoqri_status hoqri_grad_norm2(hoqri_ctx *ctx, double *out);

/*
 * Replaces every factor U_n by an orthonormal basis of the leading K_n left
 * singular subspace of the unfolding X_(n), the HOSVD initialisation that
 * Alg. 2 allows: orthogonal iteration on X_(n) X_(n)^T (power_iters steps,
 * from the seeded Gaussian start of options.seed), each step
 * Y = X_(n) (X_(n)^T V) from the nonzeros followed by the QR of the sweep.
 * The subspace error after q steps falls like (sigma_{K+1} / sigma_K)^(2q).
 * Temporary device memory: about 32 bytes per nonzero plus one K_n-vector per
 * distinct column of X_(n), freed before the call returns (the call waits for
 * its stream).  Errors: HOQRI_ERR_INVALID for power_iters < 1, HOQRI_ERR_OOM.
 */
HOQRI_API hoqri_status hoqri_init_hosvd(hoqri_ctx *ctx, int32_t power_iters);

/* Copies the current factor U_mode (I_mode x K_mode reals) to U_out. */
HOQRI_API hoqri_status hoqri_get_factor(hoqri_ctx *ctx, int32_t mode, void *U_out);

/* Replaces the current factor U_mode with U_in (I_mode x K_mode reals, assumed
 * orthonormal). */
HOQRI_API hoqri_status hoqri_set_factor(hoqri_ctx *ctx, int32_t mode, const void *U_in);

/* Residual of the last core computed (by hoqri_core, hoqri_ttmctc,
 * hoqri_iterate, hoqri_run or hoqri_grad_norm2; not by hoqri_set_factor or
 * hoqri_init_hosvd, which change the factors only): resid as in hoqri_iterate,
 * ||X||^2 and ||G||^2 in FP64.  Any output pointer may be NULL (host
 * pointers). */
HOQRI_API hoqri_status hoqri_fit(hoqri_ctx *ctx, double *resid, double *normX2, double *normG2);

/* Sizes after set-up (host pointers, each may be NULL): nnz after summing
 * repeats; rows[N] = number of non-empty mode-n slices; device bytes held. */
HOQRI_API hoqri_status hoqri_info(hoqri_ctx *ctx, int64_t *nnz, int64_t *rows, int64_t *device_bytes);

/* The nonzero-stream layout mode `mode` runs with (host, NULL allowed, 4 values):
 * the row length above which a row is streamed contiguously, the work-item size
 * (nonzeros), and the rows and columns of the FP32 lane tile; all -1 when the
 * mode does not use the sliced pass (two-pass kernels or the fiber pass).  Not
 * in the paper (a property of this implementation's gather layout; the
 * autotuner's choices are read here). */
HOQRI_API hoqri_status hoqri_layout(hoqri_ctx *ctx, int32_t mode, int64_t *out4);

/* Tracing: enable = 1 clears the totals and starts recording a CUDA event pair
 * around every core pass, TTMcTC pass, QR and nonzero-stream kernel on the
 * context's stream; enable = 0 stops recording.  Cheap enough to leave on
 * during timing. */
HOQRI_API hoqri_status hoqri_profile_enable(hoqri_ctx *ctx, int32_t enable);

/* Totals since the last hoqri_profile_enable(ctx, 1) (synchronises the stream).
 * out (host, NULL or 8 doubles): core-pass ms, core-pass count, TTMcTC-pass ms,
 * TTMcTC-pass count, QR ms, QR count, ms and count of the kernel that streams
 * the nonzeros of a mode into Y_(n) (one launch inside each core or TTMcTC pass
 * of a mode stored in the sliced layout; 0 for the other modes).
 * kernel_launches (host, may be NULL): the number of kernels the library has
 * launched since hoqri_create. */
HOQRI_API hoqri_status hoqri_profile_read(hoqri_ctx *ctx, double *out, int64_t *kernel_launches);

/* Blocks until all work queued on the context's stream has finished. */
HOQRI_API hoqri_status hoqri_synchronize(hoqri_ctx *ctx);

/* Allocation-free orthonormalisation (no counterpart in the paper, which has no
 * memory-management interface; the arithmetic is the QR step of Alg. 2).
 *
 * U_out = Q of the thin QR of A_in with diag(R) > 0, by CholeskyQR2 in FP64,
 * with no context and no device allocation: no cudaMalloc or cudaFree, no
 * allocating library call.  It serves callers that cannot allocate device
 * memory at the point of the call: code running under a fixed device-memory
 * budget (a server that has partitioned HBM among requests, where an
 * allocation can fail or evict), or code between the allocation-free
 * launches of a pre-planned sequence.  hoqri_orthonormalize needs a context,
 * whose creation allocates, and may allocate a staging buffer per call.
 *
 *   prec    HOQRI_FP64 or HOQRI_FP32 (element type of A_in and U_out)
 *   I, K    A_in is I x K, row-major; 1 <= K <= HOQRI_NOALLOC_MAXK, I >= K
 *   A_in    device buffer, read only (unless U_out == A_in)
 *   U_out   device buffer of I x K; equal to A_in (in place) or not
 *           overlapping it
 *   stream  cudaStream_t all work is ordered on (NULL: legacy default stream)
 * Scratch: one file-scope device array of HOQRI_NOALLOC_SCRATCH_BYTES per
 * device (Gram partials of at most 160 blocks, R^{-1} and four flags).  Every
 * call sets its flags to zero itself (cudaMemsetAsync on the stream);
 * the partials and R^{-1} are fully written before they are read, so nothing
 * needs to start at zero.  Its address is looked up with cudaGetSymbolAddress
 * on every call, on the device current at the call.  Under lazy module
 * loading the first call on a device loads the library's device code, which
 * reserves the array (and the module's other memory) at that point: make one
 * call during set-up if later calls must not reserve anything.  Calls whose
 * work overlaps in time (different streams, or different host threads) share
 * the one scratch array and race: order them on one stream.
 * The call copies the breakdown flag to the host and waits for the stream,
 * so it may not be called while its stream, or any stream under global
 * capture, is being captured into a CUDA graph.
 * Errors: HOQRI_ERR_INVALID for a precision other than the two above, K out of
 * range (the message names the limit), I < K, host or overlapping buffers;
 * HOQRI_ERR_QR_BREAKDOWN when a Cholesky pivot is not clearly positive after
 * the shifted first pass (A_in rank deficient; there is no Householder
 * fallback here, U_out is then unspecified); HOQRI_ERR_CUDA on a CUDA failure. */
#define HOQRI_NOALLOC_MAXK 32
#define HOQRI_NOALLOC_SCRATCH_BYTES (160 * 528 * 8 + 32 * 32 * 8 + 256)
HOQRI_API hoqri_status hoqri_orthonormalize_noalloc(int32_t prec, int64_t I, int32_t K, const void *A_in,
                                                    void *U_out, void *stream);

/* ---- Serving: many decompositions resident on one GPU (continuous batching).
 * Not in the paper, which runs one decomposition at a time; the per-request
 * arithmetic is exactly that of hoqri_create + hoqri_iterate (Alg. 2).
 *
 * A request is queued by hoqri_server_submit.  hoqri_server_step (called in
 * the caller's loop, never blocks on the GPU) marks running requests whose
 * sweeps have finished as done, then admits queued requests in submission
 * order while the device-memory budget and the slot limit allow: an admitted
 * request gets its own CUDA stream and context (sorted COO, factors, core
 * resident on the device), and all of its sweeps are queued at once, each a
 * replay of the context's captured sweep graph; requests on different streams
 * overlap on the device.  A done request holds its memory until
 * hoqri_server_take copies its results out and frees it.  Its results are
 * those of the same request run alone (same kernels, same order).
 * Ownership: the index and value buffers of a request (host or device) must
 * stay valid until the request is admitted (state RUNNING or later).  Errors:
 * the calls return a status; a request that fails at admission is reported
 * FAILED by hoqri_server_poll / hoqri_server_take with its own status. */
typedef struct hoqri_server hoqri_server;

typedef struct {
    int32_t N;                   /* order, 2..8 */
    const int64_t *dims;         /* N mode sizes */
    const int32_t *ranks;        /* N ranks (rules of hoqri_create) */
    int64_t nnz;                 /* listed entries (repeats summed) */
    const int32_t *const *idx;   /* N arrays of nnz 0-based indices (host or device) */
    const void *vals;            /* nnz reals of the request's precision */
    int32_t iters;               /* sweeps to run */
    int32_t prec;                /* hoqri_precision */
    uint64_t seed;               /* seeded Gaussian initial factors (orthonormalised) */
} hoqri_request;

enum { HOQRI_REQ_QUEUED = 0, HOQRI_REQ_RUNNING = 1, HOQRI_REQ_DONE = 2, HOQRI_REQ_FAILED = 3 };

/* budget_bytes: device bytes the admitted requests may hold together (each is
 * charged an estimate at admission, then its actual bytes); max_active: most
 * requests running at once. */
HOQRI_API hoqri_status hoqri_server_create(hoqri_server **out, int64_t budget_bytes, int32_t max_active);
/* Queues a request; *id identifies it.  HOQRI_ERR_OOM if it alone exceeds the budget. */
HOQRI_API hoqri_status hoqri_server_submit(hoqri_server *srv, const hoqri_request *req, int64_t *id);
/* One scheduling round (see above); optional counts of running and queued requests. */
HOQRI_API hoqri_status hoqri_server_step(hoqri_server *srv, int32_t *n_running, int32_t *n_queued);
/* state (HOQRI_REQ_*), times[3] = submit, admission, completion (seconds on the
 * server's steady clock; 0 if not reached), device bytes held (while QUEUED:
 * the estimate admission will charge).  Each may be NULL. */
HOQRI_API hoqri_status hoqri_server_poll(hoqri_server *srv, int64_t id, int32_t *state, double *times,
                                         int64_t *device_bytes);
/* Results of a DONE request into caller buffers (each may be NULL; host or
 * device): U_out = N factor pointers, G_out = core, resid = fit after the last
 * sweep.  Frees the request's device memory and forgets the id. */
HOQRI_API hoqri_status hoqri_server_take(hoqri_server *srv, int64_t id, void *const *U_out, void *G_out,
                                         double *resid);
/* Frees every request and the server; NULL is a no-op. */
HOQRI_API void hoqri_server_destroy(hoqri_server *srv);

/*
 * Contexts created on a stream (not the legacy default stream) allocate from a
 * memory pool per device owned by the library, which keeps the memory of
 * destroyed contexts reserved for the next ones (no mapping and unmapping per
 * context).  This call releases the reserved memory of every such pool to the
 * device; memory of live contexts stays allocated.  Thread safe; always
 * HOQRI_OK.
 */
HOQRI_API hoqri_status hoqri_trim_memory(void);

/* Message for the calling thread's last failed call ("" if none). */
HOQRI_API const char *hoqri_last_error(void);

/* Frees all device state; NULL is a no-op. */
HOQRI_API void hoqri_destroy(hoqri_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HOQRI_H */
