/*
 * aci.h - C ABI of the GB300 library for alternating cross interpolation (ACI).
 *
 * ACI (arXiv:2604.00037, Sec. 2 and Algorithm 1) computes a tensor train (TT) y with
 * y[sigma] ~ f(x^1[sigma], ..., x^N[sigma]) for an elementwise function f of N <= 4 input
 * TTs, in O(chi^3) per bond instead of the O(chi^4) of a Kronecker-delta contraction.
 * Every step of the sweep runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *  - A TT has L sites; core s has shape rank[s] x d[s] x rank[s+1], stored row-major and
 *    contiguous ([alpha][sigma][beta], sigma in the middle), rank[0] = rank[L] = 1 (Sec. 2.1).
 *    Site 0 is the most significant quantics bit (Eq. (quanticsrep)).
 *  - All calls are ordered on the context's CUDA stream. Input pointers are borrowed and
 *    only read. Device pointers must belong to the context's device.
 *  - No C++ exception crosses this interface. A negative status leaves outputs untouched
 *    and sets a message readable with aci_last_error().
 *  - Not thread-safe per context: one call at a time on a given aci_ctx.
 */
#ifndef ACI_H
#define ACI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aci_ctx aci_ctx;

/* Status codes. > 0: warning, the output is valid. < 0: error, the output is untouched. */
typedef enum {
    ACI_OK = 0,
    ACI_W_NOT_CONVERGED = 1, /* max_sweeps reached before the stop test of Algorithm 1 held */
    ACI_E_ARG = -1,          /* null pointer, bad enum, tol < 0, max_rank < 1, ...          */
    ACI_E_SHAPE = -2,        /* inputs differ in L or d, rank[0] or rank[L] != 1, d < 1     */
    ACI_E_DTYPE = -3,        /* unsupported dtype, mixed dtypes, complex coefficients on reals */
    ACI_E_ALLOC = -4,        /* the allocator returned NULL                                 */
    ACI_E_CUDA = -5,         /* a CUDA runtime call failed (message has the CUDA error)      */
    ACI_E_TIMEOUT = -6,      /* a device-side wait exceeded its iteration limit             */
    ACI_E_NUMERIC = -7       /* a non-finite value reached a pivot                         */
} aci_status;

/* Element types of the input cores (a and b have the same dtype). The method runs in FP64 /
 * complex128: FP32 and complex64 inputs are widened to FP64 / complex128 on load (exactly, in the
 * library's kernels), and their outputs are FP64 / complex128. A warm-start TT may be FP32 or FP64
 * of the inputs' kind (real or complex). */
typedef enum { ACI_R64 = 0, ACI_C128 = 1, ACI_R32 = 2, ACI_C64 = 3 } aci_dtype;
typedef enum { ACI_MEM_DEVICE = 0, ACI_MEM_HOST = 1 } aci_memory;

/* Elementwise functions f (Sec. 2.1). N = 2 except ABS2_MUL (N = 1, b ignored).
 * AFFINE: f = c0 + c1 a + c2 b + c3 a b, complex coefficients c[i] = {re, im};
 * for real dtypes every imaginary part must be 0. For real dtypes MUL_CONJ equals MUL. */
typedef enum { ACI_OP_MUL = 0, ACI_OP_MUL_CONJ = 1, ACI_OP_ABS2_MUL = 2, ACI_OP_AFFINE = 3 } aci_op_kind;
typedef struct {
    int32_t kind;     /* aci_op_kind */
    int32_t _pad;
    double c[4][2];   /* AFFINE coefficients, ignored otherwise */
} aci_op;

typedef enum { ACI_TOL_REL = 0, ACI_TOL_ABS = 1 } aci_tol_kind;
/* Pivot search of Algorithm 2.
 *  ACI_PIVOT_FULL  argmax over the whole Schur complement at every step (the paper's prrLU).
 *  ACI_PIVOT_ROOK  rook search (not in the paper; its O(d chi'^3) cost per update in App. A fits a
 *                  partial search): residual columns and rows R = M - L D U are formed one at a
 *                  time; from a start column (step 0: the column of max|M|; later the largest
 *                  residual of the previous pivot row) a row argmax and a column argmax alternate
 *                  until a fixed point or the fourth hop. O((m + n) p) work per step instead of
 *                  O(m n); the error estimate is the rejected rook pivot's magnitude. Requires
 *                  min(m, n, max_rank) <= 4096 (real) / 2048 (complex) per bond. */
/*  ACI_PIVOT_PROPOSED  (not in the paper) the learned proposer of aci_set_proposer restricts the
 *                  left-to-right sweeps: per bond it scores the candidate rows and columns of the
 *                  Pi block from cheap features (environment norms, local index, parent pivot
 *                  position, bond, previous membership), keeps the ceil(keep * k_prev) + 8 best
 *                  of each, forms Pi on them only and runs the full search there. Right-to-left
 *                  sweeps stay the full search: they produce the output and the error estimates
 *                  of the stop test, so plain ACI remains the arbiter and the fallback. */
typedef enum { ACI_PIVOT_FULL = 0, ACI_PIVOT_ROOK = 1, ACI_PIVOT_PROPOSED = 2 } aci_pivot_mode;
/* Arithmetic of the contractions (the frame half-products of Algorithm 5 and the Pi blocks of
 * Eq. (pifromframes)). The pivot search (Algorithm 2), its Schur updates and error estimates and
 * the output assembly Y = T P^-1 run in FP64 / complex128 in every mode.
 *  ACI_PREC_FP64       FP64 / complex128 multiply-adds (default).
 *  ACI_PREC_BF16X2..8  s = 2..8 exact BF16 digit planes per operand on the tensor cores: row r of
 *                      A and column c of B are scaled by powers of two 2^e_r > max|A[r,:]|,
 *                      2^f_c > max|B[:,c]| and truncated to s signed digits of b <= 7 bits
 *                      (b the largest with s K (2^b - 1)^2 < 2^24, K doubled for complex); digit
 *                      products of order i + j < s are summed exactly in FP32 and recombined in
 *                      FP64. Per entry |err| <= K 2^(e_r + f_c) 2^(-b s) (s + 3.1). */
typedef enum {
    ACI_PREC_FP64 = 0,
    ACI_PREC_BF16X2 = 2,
    ACI_PREC_BF16X3 = 3,
    ACI_PREC_BF16X4 = 4,
    ACI_PREC_BF16X5 = 5,
    ACI_PREC_BF16X6 = 6,
    ACI_PREC_BF16X7 = 7,
    ACI_PREC_BF16X8 = 8
} aci_precision;

/* A tensor train. For inputs every field is set by the caller. For outputs the library
 * fills it: d, rank and core are library-owned until aci_tt_release(). */
typedef struct {
    int32_t L;             /* number of sites, >= 1                                       */
    int32_t dtype;         /* aci_dtype                                                    */
    int32_t memory;        /* aci_memory: where core[s] points                             */
    int32_t _pad;
    const int32_t *d;      /* host array [L], local dimensions d[s] >= 1                    */
    const int64_t *rank;   /* host array [L+1], rank[0] = rank[L] = 1                       */
    void *const *core;     /* host array [L] of pointers to cores rank[s] x d[s] x rank[s+1] */
} aci_tt;

/* Optional controls of aci_elementwise_ex (aci_opts_default() fills the defaults). */
typedef struct {
    int32_t tol_kind;      /* ACI_TOL_REL (default): tau = tol * max|Pi| seen so far in the call;
                              ACI_TOL_ABS: tau = tol, the absolute tolerance of Algorithm 1     */
    int32_t max_sweeps;    /* maxiter of Algorithm 1 (default 20)                          */
    int32_t pivot_mode;    /* aci_pivot_mode                                               */
    int32_t precision;     /* aci_precision                                                */
    uint64_t seed;         /* seed of the counter-based SplitMix64 initial guess            */
    const aci_tt *init;    /* optional initial guess Y^init (warm start); NULL = random      */
    int32_t out_memory;    /* aci_memory of the output cores (default device)              */
    int32_t profile;       /* 1: time every kernel with CUDA events on the context stream and
                              count its algorithmic flops (aci_stats.kernel_*); 0: off        */
    int32_t batch_streams; /* aci_elementwise_batch: products in flight at once; 0 = autotuned:
                              per batch-size class (floor(log2 n)) the context tries 1, 2 and 3
                              products per 16 SMs (the width of one pivot-search cluster) on
                              successive calls, timing each, then keeps the fastest          */
    int32_t sweep_overlap; /* aci_overlap: schedule of the sweeps (results agree to rounding)    */
    int32_t autotune;      /* 1: before its sweeps, a call times its contractions' launch shape on
                              every shape class it will launch (capacity buckets of M, N, K;
                              products; Pi or frame form; precision) that the context has not tuned
                              yet, and keeps the fastest in the context for this and later calls:
                              for FP64 the split-K granularity (1, 2, 4 or 8 work units per SM), for
                              digit planes the output tile width (128 x 32 or 128 x 64 where tensor
                              memory allows). Results are unchanged except for the summation order
                              of the FP64 contractions. 0 (default): 4 per SM; 64 wide up to 4
                              digits, else 32                                                  */
    int32_t _pad2;
} aci_opts;

/* Schedule of the sweeps (aci_opts.sweep_overlap). The frame half-products and the Pi block of a
 * bond depend on the previous bond's pivots only through a row (left-to-right) or column (right-
 * to-left) selection. The overlapped schedule computes them for every candidate row or column on
 * a second stream while the previous bond's pivot search runs, then gathers the selected ones:
 * d_b times the contraction work, taken off the critical path of the sweep. Results differ from
 * the plain schedule only by the rounding of the contractions (their K splits differ).
 *  ACI_OVERLAP_AUTO  overlapped when every local dimension is 2 and the call is not one product
 *                    of aci_elementwise_batch (whose products already fill the GPU); plain
 *                    otherwise
 *  ACI_OVERLAP_OFF   plain: every step on the context stream, in order
 *  ACI_OVERLAP_ON    overlapped wherever it applies (L >= 3)
 * With ACI_PIVOT_PROPOSED only the right-to-left sweep (the full one) is overlapped; the learned
 * left-to-right sweep keeps the plain order.                                                   */
typedef enum { ACI_OVERLAP_AUTO = 0, ACI_OVERLAP_OFF = 1, ACI_OVERLAP_ON = 2 } aci_overlap;

/* Kernel classes of aci_stats.kernel_* (profile = 1). Flops are real-equivalent (a complex
 * multiply-add counts 8) and algorithmic: what the step needs, not what the kernel issues. */
typedef enum {
    ACI_KCLASS_FRAME = 0,  /* frame half-products L X and X R (Algorithm 5, Eq. (framesrecursive)) */
    ACI_KCLASS_PI = 1,     /* Pi block with f (Eq. (pifromframes), Eq. (localupdate))              */
    ACI_KCLASS_PIVOT = 2,  /* rank-revealing LU (Algorithm 2); flops = Schur-update multiply-adds  */
    ACI_KCLASS_OTHER = 3,  /* initial guess, stop test, output assembly                            */
    ACI_KCLASS_N = 4
} aci_kernel_class;

/* Optional diagnostics. Host arrays may be NULL; when given they must hold the sizes noted. */
typedef struct {
    int32_t iterations;    /* sweeps (left-to-right + right-to-left) performed              */
    int32_t converged;     /* 1 if the stop test of Algorithm 1 held                       */
    int32_t fixed_point;   /* 1 if an iteration reproduced every J set of the previous one  */
    int32_t L;
    double max_eps;        /* max over bonds of the last iteration's error estimates        */
    double scale;          /* S = max |Pi| over the call                                    */
    double tau;            /* final absolute tolerance                                      */
    double device_ms;      /* device time of the call (CUDA events), 0 if not measured       */
    int64_t kernel_launches; /* kernels the call launched                                     */
    int64_t *ranks;        /* [L+1] output ranks                                            */
    double *eps;           /* [L-1] per-bond error estimate of the last iteration (max of the two half-sweeps) */
    int32_t *pivot_rows;   /* [(L-1) * max_rank]: bond b's final pivot rows (positions in its Pi matrix) */
    int32_t *pivot_cols;   /* [(L-1) * max_rank]: bond b's final pivot columns                            */
    double kernel_ms[4];   /* profile = 1: summed device time per aci_kernel_class              */
    int64_t kernel_count[4];   /* launches per class (always filled)                           */
    double kernel_flops[4];    /* profile = 1: algorithmic flops per class                      */
    double tensor_flops[4];    /* profile = 1: BF16 tensor-core flops issued per class (digit-plane
                                  precisions; 0 for ACI_PREC_FP64)                               */
    /* Pivot history (optional: all three NULL = not recorded; recording adds one small launch per
     * local update). Local updates are numbered u = 0 for the CI-canonicalisation of the initial
     * guess (its update of site s is stored at bond s - 1), then u = 1 + 2 (i - 1) + h for sweep
     * iteration i = 1..max_sweeps, h = 0 left to right, h = 1 right to left. With
     * U = 1 + 2 max_sweeps and B = L - 1:
     *  hist_rank  [U * B]             rank of update u at bond b, at u * B + b (-1: did not run)
     *  hist_rows  [U * B * max_rank]  its pivot rows (positions in the factorised matrix) in pivot
     *                                 order, at (u * B + b) * max_rank + q
     *  hist_cols  [U * B * max_rank]  its pivot columns, likewise                            */
    int32_t *hist_rank;
    int32_t *hist_rows;
    int32_t *hist_cols;
} aci_stats;

/* Device memory hooks. alloc returns a device pointer of at least `bytes` bytes aligned to
 * 256 bytes, or NULL; free releases it. Both NULL: cudaMallocAsync / cudaFreeAsync on the
 * context stream. */
typedef void *(*aci_alloc_fn)(size_t bytes, void *user);
typedef void (*aci_free_fn)(void *ptr, void *user);

/* Create a context on `device`, ordered on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream). The context owns reusable scratch sized for the largest call so far.
 * Returns ACI_OK, ACI_E_ARG (ctx NULL, exactly one hook NULL) or ACI_E_CUDA. */
aci_status aci_create(aci_ctx **ctx, int device, void *cuda_stream,
                      aci_alloc_fn alloc, aci_free_fn free_fn, void *user);

/* Release the context and its scratch. Outputs not yet released stay valid only if they
 * were allocated by the caller's hooks and the caller keeps the memory. NULL is a no-op. */
void aci_destroy(aci_ctx *ctx);

/* Message of the last error on this context ("" if none). Valid until the next call. */
const char *aci_last_error(const aci_ctx *ctx);

/* Fill `opts` with defaults: relative tol, 20 sweeps, full pivot search, FP64, seed 0,
 * random initial guess, device output. */
void aci_opts_default(aci_opts *opts);

/* y ~ f(a, b) by ACI (Algorithm 1 with Algorithms 2-5, Sec. 2.6): CI-canonicalise the
 * initial guess right to left, then alternate left-to-right and right-to-left sweeps of
 * local updates at bonds (l, l+1). Each update forms Pi^n = L^n X^n_l X^n_{l+1} R^n
 * (Eq. (pifromframes)), applies f entrywise, factorises Pi by the rank-revealing LU of
 * Algorithm 2 with tolerance tau and rank cap max_rank, and updates the frames
 * (Algorithm 5). Stops when no bond grew and the largest error estimate is <= tau, or
 * when an iteration is a fixed point of the index sets, or after max_sweeps.
 *  a, b      inputs (b may be NULL for ACI_OP_ABS2_MUL); same L, d and dtype.
 *  tol       >= 0; relative to max|Pi| by default (see aci_opts.tol_kind).
 *  max_rank  >= 1; the output ranks stay <= max_rank.
 *  out       filled on success; the cores are library-owned until aci_tt_release().
 * The call returns after the result is complete (one host sync per sweep). */
aci_status aci_elementwise(aci_ctx *ctx, const aci_tt *a, const aci_tt *b, aci_op op,
                           double tol, int32_t max_rank, aci_tt *out);

/* As aci_elementwise, with explicit options (opts may be NULL for defaults) and optional
 * diagnostics (stats may be NULL). */
aci_status aci_elementwise_ex(aci_ctx *ctx, const aci_tt *a, const aci_tt *b, aci_op op,
                              double tol, int32_t max_rank, const aci_opts *opts,
                              aci_tt *out, aci_stats *stats);

/* y ~ f(x^1, ..., x^n) for n = 1..4 inputs (Sec. 2.1: the method takes N input TTs): the call of
 * aci_elementwise_ex with the input list as an array. n = 1 takes ACI_OP_ABS2_MUL, n = 2 any op
 * (inputs[0] = a, inputs[1] = b), n = 3 or 4 the product of all inputs, ACI_OP_MUL
 * (f = x^1 x^2 ... x^n, multiplied left to right). Each input has its own frames and Pi block
 * (Eq. (pifromframes)); f combines the n blocks entrywise. The inputs share L, d, dtype and
 * memory kind. For n > 2 the contractions run in FP64 (ACI_PREC_FP64) and ACI_PIVOT_PROPOSED is
 * not available (ACI_E_ARG). Outputs, options and diagnostics are those of aci_elementwise_ex. */
aci_status aci_elementwise_n(aci_ctx *ctx, int32_t n, const aci_tt *inputs, aci_op op, double tol,
                             int32_t max_rank, const aci_opts *opts, aci_tt *out, aci_stats *stats);

/* Independent products in one call (no counterpart in the paper: a throughput form of
 * aci_elementwise_ex for many pairs of uneven length and rank). Product i is
 * f(a[i], b[i]) with op[i], tol[i], max_rank[i] and the shared opts (opts->init must be NULL),
 * exactly as aci_elementwise_ex would compute it with the schedule the batch uses: same kernels,
 * same results bit for bit. In a batch ACI_OVERLAP_AUTO is the plain schedule (ACI_OVERLAP_OFF).
 * Up to opts->batch_streams products run at once, each on a worker stream of the context with its
 * own scratch and CUDA graphs, driven by a host thread; workers take the next product as they
 * finish, so uneven products balance. The pivot search of one product keeps at most one thread-
 * block cluster (16 SMs) busy, so concurrent products fill the GPU.
 *  a, out        arrays of n; b an array of n (NULL if every op is ACI_OP_ABS2_MUL);
 *  op, tol, max_rank  arrays of n; stats (array of n) and status (array of n) may be NULL.
 * Outputs are owned as for aci_elementwise_ex: release each with aci_tt_release(ctx, &out[i]).
 * The work is ordered after the context stream's earlier work, and the context stream waits for
 * it; the call returns when every product is done. Returns ACI_OK, else the first error (its
 * message in aci_last_error) or a warning; status[i] holds each product's own status. */
aci_status aci_elementwise_batch(aci_ctx *ctx, int32_t n, const aci_tt *a, const aci_tt *b,
                                 const aci_op *op, const double *tol, const int32_t *max_rank,
                                 const aci_opts *opts, aci_tt *out, aci_stats *stats,
                                 aci_status *status);

/* The learned proposer of ACI_PIVOT_PROPOSED: `params` is a device FP32 parameter vector of the
 * network of aci_k_mlp_forward (include/aci_kernels.h) with nfeatures = 7, kept by the caller
 * while the context uses it (NULL clears it); keep >= 1 sets the kept count ceil(keep * k_prev) + 8
 * per side and bond. Inference rounds the weights to FP16. */
aci_status aci_set_proposer(aci_ctx *ctx, const float *params, int32_t nfeatures, float keep);

/* Training data for the proposer: while set, every full left-to-right local update appends one
 * record per candidate row and column, the 7 features then 1 if it became a pivot else 0
 * (8 floats), to the device buffer `buf` (capacity records); *count (device, zeroed by the
 * caller) counts the records requested, of which the first `capacity` are stored. NULL stops. */
aci_status aci_set_proposer_record(aci_ctx *ctx, float *buf, int64_t capacity, uint64_t *count);

/* Free the library-owned parts of an output TT and zero the struct. */
aci_status aci_tt_release(aci_ctx *ctx, aci_tt *out);

#ifdef __cplusplus
}
#endif
#endif /* ACI_H */
