/*
 * aci_kernels.h - step-level entry points of the ACI library.
 *
 * Each call runs one step of the ACI hot path on device buffers the caller owns, in the
 * same kernels aci_elementwise() uses, so that every step can be checked on its own.
 * All matrices are row-major and contiguous unless noted; all pointers are device
 * pointers on the context's device unless noted "host". Calls are ordered on the
 * context stream and return after the stream has synchronised (results are ready).
 * Status codes and error reporting are those of aci.h.
 */
#ifndef ACI_KERNELS_H
#define ACI_KERNELS_H

#include "aci.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Frame half-product (Algorithm 5 before truncation; Sec. 2.5, Eq. (framesrecursive)):
 *   C[i, j] = sum_k A[arows[i], k] * B[k, bcols[j]],  i < M, j < N, k < K.
 * A has leading dimension lda (>= K), B has leading dimension ldb. arows (length M) and
 * bcols (length N) are optional device int32 gathers; NULL means the identity.
 * Truncating rows to I (left frame) or columns to J (right frame) is this gather applied
 * by the consumer. dtype is ACI_R64 or ACI_C128. C is M x N, ldc = N. */
aci_status aci_k_frame_gemm(aci_ctx *ctx, int32_t dtype, const void *A, const int32_t *arows,
                            int32_t M, int32_t K, int32_t lda, const void *B,
                            const int32_t *bcols, int32_t N, int32_t ldb, void *C);

/* Pi-block evaluation (Eq. (pifromframes) and Eq. (localupdate), Algorithm 1):
 *   Pi = f(A^0 B^0, ..., A^{nprod-1} B^{nprod-1})  entrywise, Pi is M x N.
 * A^n is M x K[n] (lda = K[n]), B^n is K[n] x N (ldb = N). nprod is 1 or 2 (2 unless
 * op.kind == ACI_OP_ABS2_MUL). K is a host array. *maxabs (host, may be NULL) receives
 * max |Pi| (|z| = sqrt(re^2 + im^2) for complex). */
aci_status aci_k_pi_block(aci_ctx *ctx, int32_t dtype, int32_t nprod, const void *const *A,
                          const void *const *B, int32_t M, int32_t N, const int32_t *K,
                          aci_op op, void *Pi, double *maxabs);

/* aci_k_frame_gemm and aci_k_pi_block in the arithmetic `precision` selects (aci_precision):
 * ACI_PREC_FP64 runs the FP64 kernels of the two calls above; ACI_PREC_BF16X2..8 runs the
 * tensor-core digit-plane contraction aci_elementwise_ex uses at that precision (error bound in
 * aci.h). Other values give ACI_E_ARG. Arguments and results are otherwise those of the two calls. */
aci_status aci_k_frame_gemm_prec(aci_ctx *ctx, int32_t dtype, int32_t precision, const void *A,
                                 const int32_t *arows, int32_t M, int32_t K, int32_t lda,
                                 const void *B, const int32_t *bcols, int32_t N, int32_t ldb,
                                 void *C);
aci_status aci_k_pi_block_prec(aci_ctx *ctx, int32_t dtype, int32_t precision, int32_t nprod,
                               const void *const *A, const void *const *B, int32_t M, int32_t N,
                               const int32_t *K, aci_op op, void *Pi, double *maxabs);

/* Rank-revealing LU with full pivot search (Algorithm 2, its garbles read as: the second
 * swap exchanges J_j; the loop stops before accepting a pivot; L and U are unit
 * triangular): greedy argmax |S| over the unused rows and columns, ties to the lowest
 * row * n + col, |z|^2 = re*re + im*im for complex (no fused multiply-add),
 * Schur-complement update, stop before a pivot with |pivot| <= tau or after chimax
 * pivots (at least one pivot is always taken).
 *  Min       m x n row-major input, not modified.
 *  piv_rows, piv_cols  [min(m,n,chimax)] int32 pivot positions in pivot order.
 *  D         [min(m,n,chimax)] pivots.
 *  L         m x kcap column-major (column p contiguous, kcap = min(m,n,chimax)), unit lower
 *            triangular in pivot order: L[r,p] = S_p[r,j_p] / D[p], 0 on rows pivoted before p.
 *  U         kcap x n row-major, unit upper triangular in pivot order.
 *  k_out, eps_out  host: rank and error estimate (magnitude of the first rejected pivot,
 *            0 when every row or column was used). L and U may be NULL. */
aci_status aci_k_prrlu(aci_ctx *ctx, int32_t dtype, const void *Min, int32_t m, int32_t n,
                       double tau, int32_t chimax, int32_t *piv_rows, int32_t *piv_cols,
                       void *D, void *L, void *U, int32_t *k_out, double *eps_out);

/* aci_k_prrlu with the rook search of ACI_PIVOT_ROOK (aci.h): the same arguments, layouts and
 * results (the error estimate is the rejected rook pivot's magnitude). L and U may be NULL (the
 * call then uses scratch for the residual factors). min(m, n, chimax) <= 4096 real / 2048 complex,
 * else ACI_E_SHAPE. */
aci_status aci_k_prrlu_rook(aci_ctx *ctx, int32_t dtype, const void *Min, int32_t m, int32_t n,
                            double tau, int32_t chimax, int32_t *piv_rows, int32_t *piv_cols,
                            void *D, void *L, void *U, int32_t *k_out, double *eps_out);

/* The pivot-proposer network (not in the paper): a perceptron with two hidden layers of 128
 * ReLU units and one logit, scoring candidate rows and columns of a Pi block. Parameters are one
 * FP32 device vector for F inputs (1 <= F <= 16): W1 (128 x F), b1 (128), W2 (128 x 128), b2 (128),
 * W3 (128), b3 (1), row-major; aci_k_mlp_param_count gives its length.
 *  aci_k_mlp_forward  z[s] = W3 . relu(W2 relu(W1 X[s] + b1) + b2) + b3 for the n rows of X (n x F,
 *                     row-major FP32, device); fp16_weights = 1 rounds every weight to FP16 first
 *                     (the inference form), 0 uses FP32.
 *  aci_k_mlp_grad     grad = d loss / d params (device, same layout) and *loss (host) of the mean
 *                     weighted logistic loss over the n samples with labels y (0/1, device):
 *                     weight pos_weight on y = 1, 1 otherwise. FP32 arithmetic, sums over samples
 *                     by atomics (order-dependent rounding).
 *  aci_k_mlp_adam     one Adam step (Kingma and Ba, 2015) at step t >= 1 on `count` parameters,
 *                     updating params and the moment vectors m, v (device, zero before t = 1). */
int64_t aci_k_mlp_param_count(int32_t F);
aci_status aci_k_mlp_forward(aci_ctx *ctx, int32_t n, int32_t F, const float *X, const float *params,
                             int32_t fp16_weights, float *z);
aci_status aci_k_mlp_grad(aci_ctx *ctx, int32_t n, int32_t F, const float *X, const float *y,
                          float pos_weight, const float *params, float *grad, double *loss);
aci_status aci_k_mlp_adam(aci_ctx *ctx, int32_t count, float *params, const float *grad, float *m,
                          float *v, int32_t t, float lr, float beta1, float beta2, float eps);

/* Random initial guess Y^init (Algorithm 1 input; Sec. 2.6): fills cores[s]
 * (rank[s] x d[s] x rank[s+1]) with SplitMix64 uniforms in [-1, 1): real entry e of the
 * concatenated cores uses counter e, complex entry e uses 2e (re) and 2e+1 (im).
 * d, rank and cores are host arrays; the cores are device buffers. */
aci_status aci_k_tt_random(aci_ctx *ctx, int32_t dtype, uint64_t seed, int32_t L,
                           const int32_t *d, const int64_t *rank, void *const *cores);

/* Output assembly of one site (CI-canonical form, Eq. (ycicanonical) with
 * Y_l = T_l P_l^-1, Sec. 2.5): Y = T P^-1 with P = L_I D U_J given by its unit lower
 * factor LI (k x k, row-major), pivots D (k) and unit upper factor UJ (k x k, row-major).
 * T and Y are R x k row-major; D[p] == 0 is read as D^-1 = 0. */
aci_status aci_k_apply_pinv(aci_ctx *ctx, int32_t dtype, const void *T, int32_t R, int32_t k,
                            const void *LI, const void *D, const void *UJ, void *Y);

/* The reciprocal 1/x the pivot search uses for its multipliers (Algorithm 2's Schur step
 * divides by the pivot): the hardware's approximate FP64 reciprocal refined by two Newton-Raphson
 * steps in FP64, within two units in the last place of 1/x for |x| in (1e-30, 1e30) and the
 * correctly rounded 1/x outside.
 * x and y are device arrays of n doubles. */
aci_status aci_k_reciprocal(aci_ctx *ctx, const double *x, int32_t n, double *y);

/* Limits of the library's device-side waits for the context's later calls (no counterpart in the
 * paper: a diagnostic of its failure detection). Every wait of a kernel on another CTA or on the
 * tensor-core pipeline is bounded; when the bound is reached the kernel records a timeout, leaves
 * its copies in flight to finish (their own wait keeps the default bound), returns, and the call
 * returns ACI_E_TIMEOUT with its outputs untouched. exchange_polls > 0 bounds the pivot search's
 * inter-CTA exchange waits to that many polls (the cooperative grid variant's tagged words; the 2D
 * register variant's candidate and pushed row / column mbarriers, as non-blocking tests);
 * pipeline_polls > 0 bounds the tensor-core contraction's copy and multiply waits likewise; 0
 * restores the defaults (2^24 polls; 1 s for the 2D variant's waits, 2 s for the tensor-core
 * pipeline's). Small values make an ordinary call run its waits out. Negative values give
 * ACI_E_ARG. */
aci_status aci_set_wait_limits(aci_ctx *ctx, int64_t exchange_polls, int64_t pipeline_polls);

/* Throughput of the FP64 pipe (no counterpart in the paper: the denominator of the FP64
 * rooflines the library's measurements quote). Runs `blocks` CTAs of 512 threads, each thread
 * `iters` rounds of 8 independent FP64 fused multiply-adds, twice, and times the second run with
 * CUDA events on the context stream. *tflops (host) = 2 x multiply-adds / seconds / 1e12.
 * blocks in [1, 65535], iters in [1, 2^24], else ACI_E_ARG. */
aci_status aci_k_fp64_peak(aci_ctx *ctx, int32_t blocks, int32_t iters, double *tflops);

/* The pivot search of aci_k_prrlu for callers that cannot allocate device memory; the paper
 * has no counterpart (it concerns how this library obtains scratch memory, not the method).
 * Such callers include code inside a host application that owns all device memory and forbids
 * libraries from allocating behind its back, code with a fixed memory budget, and code that
 * must not enter a device allocator (which can block on the device or take locks).
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine. Its
 * scratch is one 8 MiB file-scope device array that every GPU loading the library holds until
 * the process exits. Arguments and results are those of aci_k_prrlu, except:
 *  cuda_stream  the cudaStream_t to run on (NULL = legacy default stream), on the current device;
 *  limits       m <= 4096, n <= 4096, m * n <= 262144, else ACI_E_SHAPE and nothing runs. Every
 *               shape within them runs: when the block takes the cooperative grid variant (m n >
 *               2^18 real, > 2^16 complex), its grid is capped to what the array holds, so such a
 *               call may use fewer CTAs than aci_k_prrlu (the results do not depend on it).
 * No aci_ctx is involved, so there is no aci_last_error() message: the status says what failed.
 * The first call on each device (with that device current) looks up the array's address; make
 * that first call before any stream capture. All calls on a device share the array: calls that
 * overlap on the GPU race and must be serialised by the caller. The call returns after the
 * stream has synchronised. */
aci_status aci_k_prrlu_static(void *cuda_stream, int32_t dtype, const void *Min, int32_t m, int32_t n,
                              double tau, int32_t chimax, int32_t *piv_rows, int32_t *piv_cols,
                              void *D, void *L, void *U, int32_t *k_out, double *eps_out);

#ifdef __cplusplus
}
#endif
#endif /* ACI_KERNELS_H */
