/*
 * vne.h -- C ABI of the GB300 (sm_103a) randomized von Neumann entropy library.
 *
 * The library estimates H(R) = -tr(R ln R) of a real symmetric positive
 * (semi)definite density matrix R with unit trace (Section 1.1, eqs. earlyR,
 * R, R1, VN of Kontopoulou et al., "Randomized linear algebra approaches to
 * estimate the von Neumann entropy of density matrices", arXiv:1801.01072) by
 *   - Algorithm 1a (Section 2): Taylor series of ln(u^-1 R) with a Gaussian /
 *     Rademacher trace estimator (Lemma thm:trace),
 *   - Algorithm 1b (Section 3): Chebyshev expansion f_m of h(x) = x ln x on
 *     [0, u] (Lemma lem:prior) with the same trace estimator,
 * where u = min{1, c * p1~} comes from the power method of Appendix A
 * (Algorithm alg:power).  Every arithmetic step runs in CUDA kernels of this
 * library; the host code only validates, sequences launches and copies the
 * final scalars back.
 *
 * Conventions for every call below
 *   - Ownership: the caller owns R, the probes and every output buffer.  The
 *     handle owns a device workspace that grows on demand (cudaMalloc) and is
 *     released by vne_destroy.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  All work is enqueued on it; calls that return host
 *     outputs synchronise that stream before returning.
 *   - Errors: every call returns a vne_status and never aborts or throws.
 *     VNE_ERR_CUDA keeps the CUDA error code, readable by vne_last_cuda_error.
 *     A handle is not thread safe: use one handle per host thread.
 *   - Memory: matrix data is DEVICE memory unless vne_matrix.memory is
 *     VNE_MEM_HOST, in which case the call copies it to the device itself
 *     (pinned host memory gives the fastest copy).
 */
#ifndef VNE_H
#define VNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vne_status {
    VNE_OK = 0,
    VNE_ERR_INVALID_ARG = 1,    /* NULL pointer, n < 1, m < 1, s < 1, bad enum, ld < n ... */
    VNE_ERR_NOT_UNIT_TRACE = 2, /* check_trace set and |tr R - 1| > 1e-6 (Section 1.1)     */
    VNE_ERR_BAD_INTERVAL = 3,   /* u <= 0, u > 1 or non-finite (Algorithms 1a/1b, step 3) */
    VNE_ERR_OOM = 4,            /* workspace allocation failed                             */
    VNE_ERR_CUDA = 5,           /* a CUDA runtime call failed; see vne_last_cuda_error     */
    VNE_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up                      */
    VNE_ERR_NONFINITE = 7,      /* a moment or the estimate is NaN / Inf                   */
    VNE_ERR_UNSUPPORTED = 8     /* valid but not implemented combination                   */
} vne_status;

/* vne_matrix.layout */
enum { VNE_DENSE = 0, VNE_DIA = 1, VNE_DENSE_UPPER = 2 };
/* vne_matrix.dtype: storage type of the matrix entries.  The complex types
 * hold a Hermitian R (Section 4) as interleaved (real, imaginary) pairs, dense
 * layout only; ld counts complex entries. */
enum { VNE_F64 = 0, VNE_F32 = 1, VNE_C128 = 2, VNE_C64 = 3 };
/* vne_params.precision: arithmetic of the R.Y products of the recurrence
 *   F64     : FP64 operands, FP64 accumulation (dense and banded)
 *   F32     : FP32 operands, FP32 accumulation (dense and banded)
 *   BF16    : R and Y rounded to bf16, FP32 accumulation on the tensor cores
 *   BF16X3  : R = R_0 + R_1, Y = Y_0 + Y_1 in bf16 (piece k = bf16 of the
 *             residual of the earlier pieces), products R_0 Y_0 + R_0 Y_1 +
 *             R_1 Y_0 accumulated in FP32 (dense only)
 *   BF16X6  : three bf16 pieces of R and of Y, the six products R_a Y_b with
 *             a + b <= 2 accumulated in FP32: about FP32 operand precision
 *             (dense only)
 * The three-term update keeps an FP32 (or FP64) master copy of Y; moments,
 * coefficients and the final combination are always FP64.  The power method
 * (the interval u) runs in bf16 for BF16, and in the input's precision (FP64
 * for an FP64 R) for the split modes BF16X3 and BF16X6. */
enum {
    VNE_PREC_F64 = 0,
    VNE_PREC_F32 = 1,
    VNE_PREC_BF16 = 2,
    VNE_PREC_BF16X3 = 3,
    VNE_PREC_BF16X6 = 4
};
/* vne_params.probe: law of the trace-estimator probe vectors g_j */
enum { VNE_RADEMACHER = 0, VNE_GAUSSIAN = 1 };
/* vne_matrix.memory */
enum { VNE_MEM_DEVICE = 0, VNE_MEM_HOST = 1 };
/* vne_suggest_m.method */
enum { VNE_METHOD_TAYLOR = 0, VNE_METHOD_CHEBYSHEV = 1, VNE_METHOD_BOTH = 2 };

/* The density matrix R (eq. R1).
 *   n        : order of R (n >= 1).
 *   layout   : VNE_DENSE -- row-major, entry (i, k) at data[i*ld + k], ld >= n.
 *                           Only symmetric R is meaningful; the full square is read.
 *              VNE_DENSE_UPPER -- the same storage, but only the upper triangle
 *                           (k >= i) is used; the strictly lower entries may hold
 *                           anything.  R is taken as exactly symmetric: the call
 *                           mirrors the upper triangle into a full copy on the
 *                           device first (a HOST matrix is copied whole, then
 *                           mirrored in place).  Real dtypes only; the
 *                           estimators, vne_lambda_max and the sequence and
 *                           batched calls accept it; the projection, learned,
 *                           autotuner and allocation-free calls do not
 *                           (VNE_ERR_UNSUPPORTED or VNE_ERR_INVALID_ARG).
 *              VNE_DIA   -- symmetric banded: n_diags stored diagonals with offsets
 *                           0..n_diags-1, entry R[i, i+d] at data[d*ld + i] for
 *                           i < n-d (the rest of each row is ignored); the lower
 *                           triangle is implied by symmetry.  ld >= n.
 *   dtype    : VNE_F64 or VNE_F32; VNE_C128 / VNE_C64 for a complex Hermitian R
 *              (dense).  A Hermitian R = B + iC runs Algorithms alg1a_complex /
 *              alg1b_complex (Section 4): real probes g_j, estimates of
 *              g^T Re[f(R)] g, and u = 1 (the printed bound) unless u_override
 *              is given; the products act on the real 2n x 2n embedding
 *              [[B, -C], [C, B]] with probes [g_j; 0], which gives the same
 *              quadratic forms.  check_trace tests sum_i Re R_ii.
 *   data     : pointer to the entries (device, or host if memory == VNE_MEM_HOST).
 *   memory   : VNE_MEM_DEVICE or VNE_MEM_HOST. */
typedef struct vne_matrix {
    int64_t n;
    int32_t layout;
    int32_t dtype;
    const void* data;
    int64_t ld;
    int32_t n_diags;
    int32_t memory;
} vne_matrix;

/* Estimator parameters (Algorithms 1a / 1b and alg:power).
 *   m            : polynomial degree (Chebyshev) / number of Taylor terms, m >= 1.
 *   s            : number of probe vectors, s >= 1.
 *   probe        : VNE_RADEMACHER or VNE_GAUSSIAN.
 *   precision    : VNE_PREC_*.
 *   seed         : seeds the SplitMix64 counter generator of the probes (entry
 *                  (i, j) of the n x s probe block uses counter j*n + i; Gaussian
 *                  entries use counters 2e, 2e+1 and Box-Muller) and of the
 *                  power method's start vectors (seed ^ 0x5851F42D4C957F2D).
 *   power_iters  : t of Algorithm alg:power (t >= 1).
 *   power_trials : q of Algorithm alg:power (q >= 1).
 *   u_scale      : c in u = min{1, c * p1~}; the algorithms print c = 6, the
 *                  experiments of Section 6 use c = 1 and c = 6.  0 means 1.
 *   u_override   : > 0 skips the power method and uses this u.
 *   check_trace  : nonzero: reject R with |tr R - 1| > 1e-6 (VNE_ERR_NOT_UNIT_TRACE).
 *   probe_offset : j0 >= 0, the first probe of the call in the seed's stream:
 *                  the call draws probes j0 .. j0+s-1 (entry (i, j) uses
 *                  counter (j0+j)*n + i) and its moments_out column j belongs
 *                  to probe j0+j.  The estimate is a mean of per-probe
 *                  quadratic forms (Lemma thm:trace), so an s-probe estimate
 *                  can be split across calls or GPUs by probe range and
 *                  recombined with vne_combine_moments; the power method does
 *                  not depend on j0.  0 for a single call. */
typedef struct vne_params {
    int32_t m;
    int32_t s;
    int32_t probe;
    int32_t precision;
    uint64_t seed;
    int32_t power_iters;
    int32_t power_trials;
    double u_scale;
    double u_override;
    int32_t check_trace;
    int32_t reserved;
    int64_t probe_offset;
} vne_params;

typedef struct vne_handle vne_handle;

/* Create a handle bound to CUDA device `device`.  No workspace is allocated
 * until the first estimator call. */
vne_status vne_create(vne_handle** h, int device);
/* Free the handle and its workspace (synchronises the device). NULL is a no-op. */
void vne_destroy(vne_handle* h);

/* Algorithm 1b (Section 3): H~ = -(1/s) sum_j g_j^T f_m(R) g_j with f_m the
 * degree-m Chebyshev expansion of x ln x on [0, u] (Lemma lem:prior).
 * The moments mu[k, j] = g_j^T T_k((2/u)R - I) g_j, k = 0..m, are produced by
 * the forward three-term recurrence Y_k = 2((2/u)R - I)Y_{k-1} - Y_{k-2}
 * (equivalent to the Clenshaw form of Appendix C) and combined in FP64.
 *   H_out       : host, 1 double (required).
 *   moments_out : host, (m+1)*s doubles, row k = moment k of every probe, or NULL.
 *   u_out       : host, 1 double (the interval end u actually used), or NULL. */
vne_status vne_entropy_chebyshev(vne_handle* h, const vne_matrix* R, const vne_params* p,
                                 double* H_out, double* moments_out, double* u_out,
                                 void* stream);

/* Algorithm 1a (Section 2): H~ = ln u^-1 + (1/s) sum_j sum_{k=1}^m
 * g_j^T R (I - R/u)^k g_j / k.  moments_out (if not NULL) receives
 * tau[k, j] = g_j^T R (I - R/u)^k g_j for k = 0..m ((m+1)*s doubles). */
vne_status vne_entropy_taylor(vne_handle* h, const vne_matrix* R, const vne_params* p,
                              double* H_out, double* moments_out, double* u_out,
                              void* stream);

/* The work queue of the batched recurrence's persistent launch (host logic
 * only, no GPU call; the paper has no batched form).  For `count` dense
 * matrices of orders n[i] (host array), degree m, s probes and `method`
 * (VNE_METHOD_*), the queue holds one item per (matrix i, step t, 128-row tile)
 * with t = 1..m (1..m+1 with a Taylor estimator), in launch order: rounds of
 * one step of every active matrix, matrices admitted in the given order while
 * their bf16 R (2 * round_up(n, 128) * round_up(n, 64) bytes) fit l2_mb MiB
 * or a round has fewer than min_tiles tiles.  Every item's dependencies (all
 * tiles of the previous step of its matrix) come earlier in the queue.
 *   items_out : host, 4 int32 per item (i, t, tile, 0), or NULL to count.
 * Returns the item count, or -1 on invalid arguments. */
int64_t vne_batch_queue(const int64_t* n, int32_t count, int32_t m, int32_t s, int32_t method,
                        double l2_mb, int32_t min_tiles, int32_t* items_out);

/* Algorithms 1b and 1a on probes the caller gives, instead of the seed's
 * stream (Lemma thm:trace holds for any probe law with E[g g^T] = I; a single
 * probe g gives the quadratic form g^T f(R) g of Section 3 / Section 2, which
 * is how edge cases such as a unit vector or an eigenvector are checked).
 *   G : device, s probe vectors as an n x s row-major block (G[i*s + j] =
 *       g_j[i]), FP64 when p->precision is VNE_PREC_F64, else FP32 (the
 *       type of the path's probe block); n is R's order (for a complex R, its
 *       complex order).  Caller-owned, read during the call only.
 * Everything else as in vne_entropy_chebyshev / vne_entropy_taylor: p->probe
 * and p->probe_offset are ignored, p->seed still seeds the power method.
 * G == NULL returns VNE_ERR_INVALID_ARG. */
vne_status vne_entropy_chebyshev_probes(vne_handle* h, const vne_matrix* R, const void* G,
                                        const vne_params* p, double* H_out, double* moments_out,
                                        double* u_out, void* stream);
vne_status vne_entropy_taylor_probes(vne_handle* h, const vne_matrix* R, const void* G,
                                     const vne_params* p, double* H_out, double* moments_out,
                                     double* u_out, void* stream);

/* Both estimators on the same R, probes and u: one power method, and the two
 * recurrences share every pass over R (their probe blocks are placed side by
 * side, 2s columns).  Outputs as in the two calls above (moment buffers may be
 * NULL). */
vne_status vne_entropy_both(vne_handle* h, const vne_matrix* R, const vne_params* p,
                            double* H_cheb, double* H_taylor,
                            double* moments_cheb, double* moments_taylor,
                            double* u_out, void* stream);

/* The final combination of Algorithms 1b and 1a from per-probe moments:
 * H_cheb = -(1/s) sum_j sum_k alpha_k mu[k, j] (Lemma lem:prior coefficients
 * on [0, u]) and H_taylor = ln(1/u) + (1/s) sum_j sum_{k=1}^m tau[k, j] / k,
 * with the same device kernel and summation order as a single estimator
 * call.  For an estimate split by probe range (vne_params.probe_offset)
 * across calls or GPUs: gather the calls' moments_out in probe order, and the
 * result equals the single call's whenever the per-probe moments do.
 *   m, s          : degree and total number of probes (>= 1).
 *   u             : the interval end the moments were taken at (0 < u <= 1).
 *   moments_cheb  : host, (m+1)*s doubles, row k = moment k of every probe, or NULL.
 *   moments_taylor: host, the same for Algorithm 1a, or NULL (not both NULL).
 *   H_cheb, H_taylor: host outputs for the arrays given (the other may be NULL).
 * Errors: VNE_ERR_INVALID_ARG (sizes, NULLs), VNE_ERR_BAD_INTERVAL (u),
 * VNE_ERR_NONFINITE.  Synchronises `stream`. */
vne_status vne_combine_moments(vne_handle* h, int32_t m, int32_t s, double u,
                               const double* moments_cheb, const double* moments_taylor,
                               double* H_cheb, double* H_taylor, void* stream);

/* Many density matrices of uneven sizes in one call (Algorithms 1a/1b with
 * alg:power, applied to each).  Rs[i] (DEVICE memory, any layout and dtype a
 * single call accepts) is estimated with the same parameters p; method is
 * VNE_METHOD_CHEBYSHEV, VNE_METHOD_TAYLOR or VNE_METHOD_BOTH.  The matrices
 * run concurrently on the handle's streams (32, or VNE_BATCH_STREAMS in 1..64,
 * read once per process), each with its own slice of a
 * batch workspace.  use_graph != 0 captures the whole batch once as a CUDA
 * graph and replays it while the matrices (pointers, sizes, layouts), p and
 * method stay the same -- one graph launch per batch; a change recaptures.
 * H_cheb / H_taylor / u_out: host arrays of count doubles (those of the
 * estimators not run may be NULL; u_out may be NULL).  Returns the first
 * failing status; a matrix that failed gets NaN.  Results equal the single
 * calls' exactly.  Synchronises `stream`. */
vne_status vne_entropy_batched(vne_handle* h, const vne_matrix* Rs, int32_t count,
                               const vne_params* p, int32_t method, int32_t use_graph,
                               double* H_cheb, double* H_taylor, double* u_out, void* stream);

/* A sequence of density matrices estimated one after another (Algorithms
 * 1a/1b with alg:power, applied to each), with the transfers of HOST-resident
 * matrices hidden behind the estimates.  Rs[i] (HOST or DEVICE memory, any
 * layout and dtype a single call accepts) is estimated on `stream` by the
 * single call's kernels with the same parameters p; method is
 * VNE_METHOD_CHEBYSHEV, VNE_METHOD_TAYLOR or VNE_METHOD_BOTH.  Each host
 * matrix is copied into one of two device slots held by the handle (each the
 * size of the largest host matrix of the call) on the handle's own copy
 * stream, one matrix ahead: the copy of host matrix j + 1 runs while matrix j
 * is estimated.  Host memory that is pinned (cudaHostAlloc,
 * cudaHostRegister) overlaps; pageable memory is copied correctly but the
 * runtime stages it without overlap.
 * H_cheb / H_taylor / u_out: host arrays of count doubles (those of the
 * estimators not run may be NULL; u_out may be NULL).  Every matrix is
 * validated before the first transfer.  Returns the first failing status;
 * the matrix that failed and the ones after it get NaN.  Results equal the
 * single calls' exactly.  No transfer from the caller's memory is in flight
 * when the call returns.  Synchronises `stream`. */
vne_status vne_entropy_sequence(vne_handle* h, const vne_matrix* Rs, int32_t count,
                                const vne_params* p, int32_t method, double* H_cheb,
                                double* H_taylor, double* u_out, void* stream);

/* Autotuner of the tensor-core step (BF16 / BF16X3 dense paths; not in the
 * paper).  Times every candidate tile shape -- BN probe columns per CTA (the
 * widest MMA, half of it, 128), each with and without the K split over a CTA
 * pair -- on full estimator calls of R with p and method
 * (CUDA events around the tensor-core steps), and keeps the fastest for the
 * size bucket of R (ceil log2 of its 128-row tiles) and of the step's column
 * count.  The choice is process-wide and applies to later calls (single and
 * batched) whose sizes fall in the same buckets; the environment variable
 * VNE_TC_TILE="BN,1,1[,ksplit]" still overrides it.
 *   shape_out: host, 4 ints (BN, CM, CN, ksplit) or NULL; CM = CN = 1 always
 *              (every CTA loads its own operand tiles);
 *   us_out:    host, the chosen shape's microseconds per step, or NULL. */
vne_status vne_tc_autotune(vne_handle* h, const vne_matrix* R, const vne_params* p,
                           int32_t method, int32_t* shape_out, double* us_out, void* stream);

/* The tile shape the tensor-core step takes for n rows and ncols step columns
 * (2s for the fused Chebyshev + Taylor steps, s otherwise) on sm_count SMs,
 * without the autotuner's or VNE_TC_TILE's choice: the widest tile (BN up to
 * 256), with the K split over a CTA pair (ksplit = 2) when the row tiles leave
 * most SMs idle and the doubled grid still fits in one wave.  Host logic only:
 * no CUDA call, no handle.
 *   shape_out: host, 4 ints (BN, CM, CN, ksplit).
 * Errors: VNE_ERR_INVALID_ARG for n, ncols or sm_count < 1 or a NULL shape_out.
 * An autotuned shape for the same size bucket, or VNE_TC_TILE, replaces this
 * default inside the estimators. */
vne_status vne_tc_shape(int64_t n, int32_t ncols, int32_t sm_count, int32_t* shape_out);

/* Algorithm alg:power: p1~ = max_j x_t^T R x_t / x_t^T x_t over q = power_trials
 * start vectors in {+1,-1}^n after t = power_iters products (each iterate is
 * divided by its 2-norm, which leaves the Rayleigh quotient unchanged).  The
 * products use the arithmetic of p->precision (BF16 modes use bf16 R with FP32
 * accumulation; BF16X3 / BF16X6 use R in its input precision); the Rayleigh
 * quotient is accumulated in FP64.
 *   lam_out : host, 1 double. */
vne_status vne_lambda_max(vne_handle* h, const vne_matrix* R, const vne_params* p,
                          double* lam_out, void* stream);

/* Allocation-free variant of vne_lambda_max, for callers that cannot
 * allocate device memory when they need the estimate: code running under an
 * allocator that forbids new allocations, plug-ins inside applications that
 * own the device memory budget, or loops that cannot afford cudaMalloc's
 * implicit synchronisation.  The paper has no counterpart: it is a
 * deployment convenience of this library.
 *
 * It runs the same power-method kernels as vne_lambda_max but keeps all of
 * its scratch in one fixed device array inside the library
 * (VNE_STATIC_SCRATCH_BYTES on every GPU that loads the library, held until
 * the process exits), needs no handle, and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The caller still passes R and receives lam_out.
 *   - Device: the calling thread's current device.  The first call on a
 *     device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture.  The address is kept
 *     with the device's context: a call from a thread with no current
 *     context yet, or after a device reset (a new primary context), looks
 *     it up again.
 *   - Results: the same power-method kernels with the same block counts as
 *     vne_lambda_max, so the same lam_out for the same R and p.
 *   - Limits: R must be device memory stored in the computed precision
 *     (F64 with VNE_PREC_F64, F32 with VNE_PREC_F32); n * power_trials
 *     must not exceed VNE_STATIC_MAX_VECTOR_ELEMS.  Anything else returns
 *     VNE_ERR_UNSUPPORTED; bad arguments (including n_diags < 1 for a
 *     banded R) return VNE_ERR_INVALID_ARG.  Device-side failures map as in
 *     vne_lambda_max: VNE_ERR_TIMEOUT, VNE_ERR_BAD_INTERVAL, VNE_ERR_NONFINITE.
 *   - Sharing: every call on a device uses the same array, which keeps the
 *     previous call's contents (the call clears what must start at zero).
 *     Calls that overlap on the GPU (other streams or host threads) race on
 *     it and must be serialised by the caller.
 *   - Synchronises `stream` before returning. */
#define VNE_STATIC_MAX_VECTOR_ELEMS 131072
#define VNE_STATIC_SCRATCH_BYTES 2621440
vne_status vne_lambda_max_static(const vne_matrix* R, const vne_params* p, double* lam_out,
                                 void* stream);

/* vne_entropy_projection.sketch: the random projection Pi of Algorithm alg:EN */
enum { VNE_SKETCH_GAUSSIAN = 0, VNE_SKETCH_SRHT = 1, VNE_SKETCH_COUNT = 2 };

/* Algorithm alg:EN (Section 5): for R of rank at most k, the k largest
 * singular values p~_i of R~ = R Pi (Pi n x s) and H~ = sum_i p~_i ln(1/p~_i).
 *   k            : 1 <= k <= s.
 *   s            : sketch width, 1 <= s <= 512.
 *   sketch       : VNE_SKETCH_GAUSSIAN -- i.i.d. N(0,1)/sqrt(s) entries, entry
 *                  (i, c) from counter c*n + i as for the Gaussian probes;
 *                  VNE_SKETCH_SRHT -- Algorithm alg:SHD scaled by sqrt(N/s):
 *                  Pi[i, c] = D_i (-1)^popcount(i & t_c) / sqrt(s) with N the
 *                  next power of two >= n (R read as zero-padded to N), D_i the
 *                  top bit of SplitMix64 output i of seed ^ 0xA0761D6478BD642F,
 *                  t_c = floor(u N), u = (output c of seed ^ 0xE7037ED1A0B428DB
 *                  >> 11) / 2^53;
 *                  VNE_SKETCH_COUNT -- Algorithm alg:IS: Pi[i, h(i)] = D_i with
 *                  h(i) = floor(u s), u from output i of the same index stream.
 *   krylov_iters : 0 -- Algorithm alg:EN as printed (1 <= k <= s).
 *                  q >= 1 -- the block-Krylov extension (not in the paper): the
 *                  block size is b = s (<= 64, q*b <= 512, k <= q*b); V_0 = R Pi,
 *                  V_j = R Q_(j-1); each V_j is orthogonalised against the
 *                  earlier blocks (two passes of block Gram-Schmidt) and made
 *                  orthonormal through the eigendecomposition of its Gram
 *                  matrix (Jacobi), dropping directions with Gram eigenvalue
 *                  below 1e-12 (FP64) / 1e-6 (FP32) of the first block's
 *                  largest; the k largest eigenvalues theta of T = K^T R K
 *                  (K = [Q_0 .. Q_(q-1)]) give H~ = sum theta ln(1/theta)
 *                  plus the tail t ln((n-k)/t), t = 1 - sum theta (the rest
 *                  of the unit trace spread evenly); p_out gets theta.
 *   precision    : VNE_PREC_F64 or VNE_PREC_F32: arithmetic of Pi and of the
 *                  product R Pi on the CUDA cores.  VNE_PREC_BF16X3 /
 *                  VNE_PREC_BF16X6: Pi in FP32, the products R Pi (and R Q_j)
 *                  on the tensor cores with R and Pi split into two / three
 *                  bf16 pieces and FP32 accumulation (the recurrence's split
 *                  modes), FP32 results.  VNE_PREC_BF16 is unsupported (its
 *                  rounding would cost the p~ accuracy).  The Gram matrix
 *                  R~^T R~ (compensated FP32 sums for FP32 results), its
 *                  eigenvalues (Householder tridiagonalisation + bisection) and
 *                  H~ are FP64.
 *   R            : VNE_DENSE only.
 *   H_out        : host, 1 double.   p_out : host, k doubles (descending), or NULL.
 * Singular values come from the eigenvalues of R~^T R~: the top-k values have
 * full relative accuracy; those below ~1e-8 p~_1 only absolute accuracy. */
vne_status vne_entropy_projection(vne_handle* h, const vne_matrix* R, int32_t k, int32_t s,
                                  int32_t sketch, int32_t krylov_iters, int32_t precision,
                                  uint64_t seed, double* H_out, double* p_out, void* stream);

/* ---------------------------------------------------------------------------
 * Learned moment correction (an extension of Algorithm 1b; the paper has no
 * learned component).  The Chebyshev estimate of degree m = 16 carries the
 * truncation error of f_16 (Lemma lem:prior).  A network maps 19 features of
 * the estimate -- tot_k / (s n) for k = 0..15 with tot_k = sum_j mu_{k,j} the
 * probe totals of the moments, ln(n)/10, ln(lambda~)/10 and ln(u)/10 -- to
 * c = 100 (H - H_16) / (n u), and the corrected estimate is H_16 + c n u / 100.
 * (With p = u y the truncation error of f_m is u e_m(y), e_m that of y ln y
 * on [0, 1], so c is a mean over the spectral distribution of y.)
 * Network: 19 -> 128 -> 128 -> 128 -> 1, GELU(x) = x Phi(x) on the hidden
 * layers, linear output, FP32.  Parameters are one flat device array of
 * VNE_MLP_N_PARAMS floats: [W1 (128 x 19, row-major), b1 (128), W2 (128 x 128),
 * b2, W3 (128 x 128), b3, W4 (1 x 128), b4 (1)].  Feature rows are
 * VNE_MLP_N_IN floats.  All pointers below are DEVICE pointers unless marked
 * host.
 * ------------------------------------------------------------------------- */
#define VNE_MLP_N_IN 19
#define VNE_MLP_N_MOMENTS 16
#define VNE_MLP_N_HIDDEN 128
#define VNE_MLP_N_PARAMS 35713
#define VNE_MLP_DEGREE 16

/* Training data without forming R: for `count` spectra p (index b), with
 *   kind[b] 0: p_i ~ exp(-(i-1)/a[b]); 1: p_i ~ i^-a[b] for i <= ktop[b],
 *   floor[b] beyond (i = 1..n[b], unit trace, n[b] >= 2),
 * u = c[b] * p_1 and lambda~ = p_1, draws the probe totals of Algorithm 1b for
 * R = Psi diag(p) Psi^T with Haar Psi and s Gaussian probes -- sum_j mu_{k,j}
 * = sum_i w_i T_k(2 p_i / u - 1), w_i = sum_j z_ij^2, z_ij the Gaussian probe
 * value (i, j) of seeds[b] -- for k = 0..m (15 <= m <= 64), and writes
 * features[b] (19 floats), target[b] = 100 (H(p) - H_m) / (n u) (float), the exact
 * entropy H_exact[b], the estimate H_low[b] = H_m and, if totals != NULL,
 * totals[b*(m+1) + k].  Arithmetic: FP32 draws and polynomials, FP64 sums. */
vne_status vne_spectral_samples(vne_handle* h, int32_t count, const int32_t* kind,
                                const int32_t* n, const float* a, const int32_t* ktop,
                                const float* floor, const float* c, const uint64_t* seeds,
                                int32_t m, int32_t s, float* features, float* target,
                                double* H_exact, double* H_low, double* totals, void* stream);

/* y[b] = net(X[b]) for b < batch (X: batch x 19 floats, y: batch floats). */
vne_status vne_mlp_forward(vne_handle* h, const float* params, const float* X, int32_t batch,
                           float* y, void* stream);

/* Mean squared error of net(X) against target (batch rows) and its gradient
 * (grad: VNE_MLP_N_PARAMS floats, same layout as params); loss_out is host. */
vne_status vne_mlp_gradient(vne_handle* h, const float* params, const float* X,
                            const float* target, int32_t batch, float* grad, double* loss_out,
                            void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step counts from 1) on
 * the batch of rows idx_i = (a * ((first + i) mod rows) + c) mod rows, i < batch,
 * of X / target (rows rows), where a (coprime to rows) and c come from
 * perm_seed: `first` = e * rows + (offset in epoch e) walks a fixed
 * permutation.  params, adam_m, adam_v: VNE_MLP_N_PARAMS floats each (Adam
 * moments start at zero).  loss_out: host, or NULL (then the call does not
 * synchronise the stream). */
vne_status vne_mlp_train_step(vne_handle* h, float* params, float* adam_m, float* adam_v,
                              int32_t step, float lr, const float* X, const float* target,
                              int64_t rows, int32_t batch, int64_t first, uint64_t perm_seed,
                              double* loss_out, void* stream);

/* Algorithm 1b with Gaussian probes at degree p->m (VNE_MLP_DEGREE, the
 * degree the network is trained for; >= 15 required) followed by the learned
 * correction: H_out = H_m + (n u / 100) net(features).  H_plain_out (host, or
 * NULL) receives H_m itself -- the uncorrected estimate, which is also the
 * fallback when no trained network is at hand.  Other arguments as for
 * vne_entropy_chebyshev; params is the trained network (device). */
vne_status vne_entropy_chebyshev_learned(vne_handle* h, const vne_matrix* R, const vne_params* p,
                                         const float* params, double* H_out,
                                         double* H_plain_out, double* u_out, void* stream);

/* The random projection of vne_entropy_projection: out[c*n + i] = Pi[i, c]
 * (FP64, device, n*s doubles, caller-owned). */
vne_status vne_sketch_block(vne_handle* h, int64_t n, int32_t s, int32_t sketch, uint64_t seed,
                            double* out, void* stream);

/* The probe block the estimators draw: out[j*n + i] = g_j[i] (FP64, device,
 * n*s doubles, caller-owned).  Lets callers check the generator. */
vne_status vne_probe_block(vne_handle* h, int64_t n, int32_t s, int32_t probe, uint64_t seed,
                           double* out, void* stream);

/* Per-kernel timing: when enabled, the handle records CUDA events on the call's
 * stream around the launches of kernel class `kind` (0 = dense tensor-core
 * steps, 1 = dense SIMT steps, 2 = banded steps, 3 = power-method products):
 * around each launch for classes 1 and 2, and around the whole run of
 * consecutive launches of a call for classes 0 and 3 (the tensor-core steps and
 * the power-method products overlap each other's start-up, which an event
 * between them would prevent).  vne_profile_read
 * returns the total time (ms) and the number of launches since the last reset. */
vne_status vne_profile_enable(vne_handle* h, int32_t on);
vne_status vne_profile_read(vne_handle* h, int32_t kind, double* total_ms, int64_t* launches);
vne_status vne_profile_reset(vne_handle* h);

/* Number of the library's own kernel launches enqueued by this handle so far. */
int64_t vne_launch_count(const vne_handle* h);

/* Check of the library's failure path for lost arrivals (no counterpart in
 * the paper): launches a kernel whose mbarrier wait has no arrival, so its
 * bounded wait gives up after the library's deadline (2 s), flags the
 * timeout and returns.  Expected result: VNE_ERR_TIMEOUT, with the context
 * still usable for the next call.  Synchronises `stream`. */
vne_status vne_selftest_timeout(vne_handle* h, void* stream);

/* Human-readable name of a status code (static string). */
const char* vne_status_string(vne_status s);
/* cudaError_t behind the last VNE_ERR_CUDA of this handle (0 if none). */
int32_t vne_last_cuda_error(const vne_handle* h);
/* Degree suggested by Theorem thm:taylor (m = ceil((u/l) ln(1/eps))) or
 * Theorem thm:cheb (m = sqrt(u / (2 eps l ln(1/(1-l)))), rounded up);
 * returns -1 for invalid arguments. */
int32_t vne_suggest_m(int32_t method, double u, double ell, double eps);

#ifdef __cplusplus
}
#endif
#endif /* VNE_H */
