// Internal declarations shared by the translation units of libhoqri.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hoqri.h"

#define HOQRI_MAXN 8
#define HOQRI_MAXK 64
// most blocks of the hybrid pass kernel per SM (8 warps each); the work
// ranges of its long rows are cut for hyb_blocks_per_sm() * 8 warps per SM
#define HY_BLOCKS_PER_SM 2

namespace hoqri {

// ---------------------------------------------------------------- errors

void set_error(const std::string &msg);

struct Status {
    hoqri_status code = HOQRI_OK;
    bool ok() const { return code == HOQRI_OK; }
};

#define HQ_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::hoqri::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));     \
            return e_ == cudaErrorMemoryAllocation ? HOQRI_ERR_OOM : HOQRI_ERR_CUDA;     \
        }                                                                               \
    } while (0)

#define HQ_TRY(expr)                         \
    do {                                     \
        hoqri_status s_ = (expr);            \
        if (s_ != HOQRI_OK) return s_;       \
    } while (0)

// ------------------------------------------------------- per-mode storage

// kernel and shape of the fiber-factored pass of one mode (fiber.cu)
struct FibShapeSel {
    int nm1 = 0, KA = 0, KB = 1, KL = 0, PP = 0;
    const void *fn = nullptr;  // k_fib<nm1, PP, KL>
    int warp_floats = 0;       // its shared memory per warp (4-byte words)
};

// Nonzeros sorted by their mode-n index (stable from the coalesced,
// lexicographic order), stored as structure of arrays.
struct ModeStore {
    int32_t *oidx[HOQRI_MAXN - 1] = {};  // indices of the other modes (ascending m != n)
    void *vals = nullptr;                // real[nnz]
    int32_t *perm = nullptr;             // sorted position -> coalesced entry id
    int64_t R = 0;                       // non-empty rows (slices)
    int32_t *row_id = nullptr;           // [R] mode-n index of each non-empty row
    int64_t *row_ptr = nullptr;          // [R+1] first sorted position of each row
    // Partition into warp tasks ("chunks") of at most C consecutive nonzeros:
    // whole rows are packed together; a row longer than C is cut into pieces
    // that are chunks of their own ("big" rows).
    int32_t C = 0;
    int64_t nchunks = 0;
    int64_t *chunk_start = nullptr;      // [nchunks+1] first sorted position of each chunk
    int32_t *chunk_row = nullptr;        // [nchunks] first row (index into row_id) of each chunk
    int64_t nbig = 0;
    int32_t *big = nullptr;              // [3*nbig] (row, first chunk, last chunk) of each big row

    // Hybrid copy of the same nonzeros for the register-tiled FP32 kernels:
    // rows longer than Lshort stay contiguous (row order) at the front; the
    // other rows are sorted by length and stored as slices of 8 rows, element
    // (step s, row g) of slice j at sbase[j] + 8*s + g, shorter rows padded with
    // (index 0, value 0) entries.  Work items: long tasks (contiguous ranges of
    // the long part, cut every ~T nonzeros at multiples of 8) then slice tasks
    // (runs of consecutive slices).
    bool hyb = false;
    int64_t htotal = 0;                  // stored elements (with padding)
    int32_t *hidx[HOQRI_MAXN - 1] = {};
    void *hvals = nullptr;
    int64_t nlong = 0;                   // rows in the long part
    int64_t *lrp = nullptr;              // [nlong+1] offsets of the long rows
    int32_t *lrow = nullptr;             // [nlong] compact row index r (into row_id)
    int64_t nslice = 0;
    int64_t *sbase = nullptr;            // [nslice+1]
    int32_t *srow = nullptr;             // [8*nslice] compact row index, -1 for padding rows
    int64_t nitem = 0, nitem_long = 0;
    int64_t *item_s = nullptr, *item_e = nullptr;  // [nitem] element ranges
    int32_t *item_aux = nullptr;         // long: first long row; slice task: first slice
    int64_t ipw = 1, nrange = 0;         // warp w processes items [w*ipw, (w+1)*ipw)
    int64_t nspan = 0;
    int32_t *span = nullptr;             // [3*nspan] (long row j, first range, last range) of rows cut by ranges
    int64_t tune_Lshort = 0, tune_T = 0; // the layout parameters it was built with
    int tune_TL = 0, tune_TV = 0;        // lane tile of the FP32 pass (0: the plan's own)
    int64_t long_elems = 0;              // nonzeros in the long part
    int64_t hyb_bytes = 0;               // device bytes of the hybrid arrays

    // Fiber-factored layout (fiber.cu) over the sorted stream above: pieces of at
    // most FB_LP nonzeros of one fiber (run of equal prefix indices in a row), in
    // stream order; contiguous piece ranges per warp.
    bool fib = false;
    FibShapeSel fb_sel;
    int64_t fb_np = 0;                   // pieces
    int32_t *fb_pstart = nullptr;        // [np] first sorted position
    uint32_t *fb_plenf = nullptr;        // [np] length | first-piece-of-row bit
    int32_t *fb_pa = nullptr, *fb_pb = nullptr;  // [np] prefix indices
    int fb_W = 0, fb_grid = 0;           // ranges (one per warp) and CTAs
    size_t fb_smem = 0;
    int32_t *fb_prange = nullptr;        // [W+1]
    int32_t *fb_rrow0 = nullptr;         // [W] compact row of each range's first piece
    int64_t fb_nspan = 0;
    int32_t *fb_span = nullptr;          // [3*nspan] (row, first range, last range) of cut rows
    int64_t fb_bytes = 0;
};

struct Workspace;  // defined in the pass unit

}  // namespace hoqri

struct hoqri_ctx {
    int N = 0;
    int64_t dims[HOQRI_MAXN] = {};
    int32_t K[HOQRI_MAXN] = {};
    int64_t P = 1;                      // prod K
    hoqri_options opt{};
    int prec = HOQRI_FP32;
    size_t rsize = 4;                   // sizeof(real)
    bool mix = false;                   // HOQRI_BF16X3: FP32 storage, split-BF16 tensor-core long rows
    void *usplit = nullptr;             // BF16 (hi | lo) rows of one factor (tensor-core B operand)
    unsigned long long *claim = nullptr;  // work counter of the slice launch of the hybrid pass
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int64_t nnz = 0;                    // after summing repeats
    hoqri::ModeStore ms[HOQRI_MAXN];
    void *U[HOQRI_MAXN] = {};           // factors, real[I_n*K_n]
    float *Upad[HOQRI_MAXN] = {};       // zero-padded copies I_n x padded_rank(K_n) for the sliced
                                        // pass of modes whose other ranks are not powers of two >= 4
    void *G = nullptr;                  // real[P]
    void *A = nullptr;                  // real[max I_n*K_n], TTMcTC output of the sweep
    // FP64 scalars on the device: [0] ||X||^2, [1] ||G||^2 of the last core,
    // [2 ...] ||G||^2 history of hoqri_iterate (one slot per core pass)
    double *dnorm = nullptr;
    int64_t dnorm_slots = 0;
    int32_t *dflag = nullptr;           // [0] QR state of the current QR, [1] breakdown count,
                                        // [2] device wait ran out (error), [3] the current
                                        // QR's first pass was shifted
    // scratch of the passes (partials); see passes.cu
    void *core_part = nullptr;          // per-CTA core partials
    int64_t core_part_bytes = 0;
    void *a_part = nullptr;             // per-chunk TTMcTC partial rows
    int64_t a_part_bytes = 0;
    double *qr_part = nullptr;          // Gram partials
    int64_t qr_part_bytes = 0;
    double *qr_small = nullptr;         // K x K FP64 workspace (Rinv) and norms
    double *qr_work = nullptr;          // Householder fallback workspace (max I*K doubles)
    double *gnorm_part = nullptr;       // block partials of ||G||^2
    float *Y = nullptr;                 // rows y_i of Y_(n) for the modes using the hybrid kernels
    int64_t Y_bytes = 0;
    float *ypart = nullptr;             // [nitem_long][2][P_{-n}] pieces of rows cut by long tasks
    int64_t ypart_bytes = 0;
    float *fpart = nullptr;             // [W][2][P_{-n}] rows cut by the fiber pass's ranges
    int64_t fpart_bytes = 0;
    int core_grid = 0;                  // CTAs of the core pass (fixed per context)
    int core_mode = -1;                 // stream the two-pass core is computed from (cheapest)
    int pass_grid = 0;
    int core_grid_fast = 0;             // the same for the register-tiled FP32 kernels
    int pass_grid_fast = 0;
    int64_t device_bytes = 0;
    // CUDA graph of one sweep
    cudaGraphExec_t sweep_exec = nullptr;  // one captured sweep (use_graphs)
    int64_t sweep_launches = 0;             // kernels in the captured sweep
    bool sweep_graph_off = false;           // capture failed once: plain launches from then on
    double *gslot = nullptr;                // ||G||^2 after each block update of the captured sweep
    int32_t *gcount = nullptr;              // sweeps replayed since the history base
    int graph_slot_base = -1;
    double host_norm[2] = {0, 0};
    // tracing
    int64_t nlaunch = 0;                // kernels launched by the library
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct EvRec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<EvRec> ev_recs;
    double prof[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // (ms, count) per trace kind 0..3
};

namespace hoqri {

// device memory helpers (track bytes)
// Device memory of a context.  A context on a created stream allocates and
// frees in stream order (cudaMallocAsync / cudaFreeAsync), so creating and
// destroying contexts does not wait for work on other streams; on the legacy
// default stream plain cudaMalloc / cudaFree are used.
cudaError_t raw_alloc(void **p, size_t bytes, cudaStream_t st);
void raw_free(void *p, cudaStream_t st);
hoqri_status dalloc(hoqri_ctx *c, void **p, size_t bytes);
void dfree(void *p, cudaStream_t st = nullptr);
// Lets a kernel take `bytes` of dynamic shared memory on the current device by
// setting its limit to the most it may have (an error if `bytes` exceeds that).
// Contexts are built on several host threads at once (the request server):
// with the limit set to each launch's own need, a limit lowered by one thread
// between another thread's setting and its launch would fail that launch.
cudaError_t smem_limit_raw(const void *fn, size_t bytes);
template <typename F>
cudaError_t smem_limit(F *fn, size_t bytes) {
    return smem_limit_raw(reinterpret_cast<const void *>(fn), bytes);
}

// setup (setup.cu)
hoqri_status build_storage(hoqri_ctx *c, const int32_t *const *idx_dev, const void *vals_dev, int64_t nnz_raw);
hoqri_status build_partition(hoqri_ctx *c, int n, int32_t C);
hoqri_status build_hybrid(hoqri_ctx *c, int n, int64_t Lshort, int64_t T, int SW);
void free_hybrid(hoqri_ctx *c, int n);             // releases what build_hybrid allocated
hoqri_status autotune_hybrid(hoqri_ctx *c);        // tune.cu: layout per mode by timing

// register-tile plan of the FP32 kernels for mode n (passes.cu)
struct FastTile {
    bool ok = false;
    int nm1 = 0, TL = 0, TV = 0, GL = 0, GV = 0, lpn = 0;
    int Ka = 0, Kb = 0, Kl = 0, Pm = 0;
    // sliced pass only: ranks of the other modes rounded up to powers of two >= 4
    // (the factors are gathered from zero-padded copies; Ka, Kb, Kl, Pm are padded)
    bool pad = false;
};
// rank of mode m's factor as the sliced pass gathers it (a power of two >= 4)
int padded_rank(int K);
bool fast_tile(const hoqri_ctx *c, int n, FastTile *out);
// tile of the hybrid (sliced) pass for mode n: the plan above with at most 32
// FP32 accumulators per lane where the shape allows (three blocks per SM)
bool hyb_tile(const hoqri_ctx *c, int n, FastTile *out);
int hyb_blocks_per_sm(const FastTile &p);

// passes (passes.cu)
hoqri_status core_reduce(hoqri_ctx *c, int n, int nblk, void *G_out, double *normG2_slot);
hoqri_status unfold_core(hoqri_ctx *c, int n, const void *G, void *Gn);

// one-stream FP32 passes on the hybrid layout (hybrid.cu)
bool hyb_mode(const hoqri_ctx *c, int n);
hoqri_status hyb_pass(hoqri_ctx *c, int n);
hoqri_status hyb_a_from_y(hoqri_ctx *c, int n, const float *Gn, float *A_out);
hoqri_status hyb_core_partials(hoqri_ctx *c, int n, int *nblk);
size_t hyb_smem_need(const hoqri_ctx *c, int n);
size_t hyb_smem_cap();
// fiber-factored pass (fiber.cu): supported shape, layout, cut-row buffer size, pass
bool fib_shape(const hoqri_ctx *c, int n, FibShapeSel *sel);
hoqri_status build_fiber(hoqri_ctx *c, int n);
void free_fiber(hoqri_ctx *c, int n);
int64_t fib_part_bytes(const hoqri_ctx *c, int n);
hoqri_status fib_pass(hoqri_ctx *c, int n);
hoqri_status passes_init(hoqri_ctx *c);
hoqri_status core_pass(hoqri_ctx *c, int n, void *G_out, double *normG2_slot);
hoqri_status ttmctc_pass(hoqri_ctx *c, int n, const void *G, void *A_out);

// QR (qr.cu)
hoqri_status qr_init(hoqri_ctx *c);
// CholeskyQR2 with scratch in a static device array (no allocation); prec is
// HOQRI_FP64 or HOQRI_FP32, 1 <= K <= HOQRI_NOALLOC_MAXK, I >= K (checked by the caller)
hoqri_status orthonormalize_noalloc(int prec, int64_t I, int K, const void *A, void *U, cudaStream_t st);
hoqri_status orthonormalize(hoqri_ctx *c, int n, void *A_inout, void *U_out);
// ||A_n - U_n G_(n) G_(n)^T||_F^2 in FP64 into *slot (device), G the context's core (grad.cu)
hoqri_status grad_term(hoqri_ctx *c, int n, const void *A, double *slot);
hoqri_status init_factors_seeded(hoqri_ctx *c);

int64_t ceil_div(int64_t a, int64_t b);

// tracing: kinds 0 = core pass, 1 = TTMcTC pass, 2 = QR, 3 = nonzero-stream kernel (k_hyb)
hoqri_status prof_begin(hoqri_ctx *c, int kind, cudaEvent_t *a);
hoqri_status prof_end(hoqri_ctx *c, int kind, cudaEvent_t a);

}  // namespace hoqri
