// Internal launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace vne {

// Moment partial sums: slot 0 holds ntiles0 x S partials of g^T Y_0 terms
// (written by the init kernels), slot t >= 1 holds ntiles x S partials
// written by recurrence step t.  Column c of a step belongs to probe c % s.
struct Partials {
    double* base;
    int ntiles0;
    int ntiles;
    int S;
    __host__ __device__ double* slot(int t) const {
        return t == 0 ? base : base + (size_t)ntiles0 * S + (size_t)(t - 1) * ntiles * S;
    }
};

// Epilogue kinds of one recurrence step t (Z = R Y_{t-1}):
//   CHEB1 : Y_1 = a Z - G              (a = 2/u), moment g^T Y_1
//   CHEB  : Y_t = 2(a Z - Y_{t-1}) - Y_{t-2},      moment g^T Y_t
//   TAYLOR: Y_t = Y_{t-1} - Z / u,                 moment g^T Z  (= tau_{t-1})
//   PLAIN : Y_t = Z (the plain product, tensor-core step only; no moments)
enum EpiKind { EPI_NONE = 0, EPI_CHEB1 = 1, EPI_CHEB = 2, EPI_TAYLOR = 3, EPI_PLAIN = 4 };

struct StepCols {
    // columns [c0, c0+ncheb) are Chebyshev, [t0, t0+ntay) are Taylor
    int cheb_c0, ncheb, tay_c0, ntay;
    int cheb_kind;  // EPI_CHEB1, EPI_CHEB or EPI_NONE for this step
};

// ---- probes / initial blocks (vne_probe.cu) --------------------------------
cudaError_t launch_probe_block_f64(double* out, int64_t n, int s, int kind, uint64_t seed,
                                   cudaStream_t st);
// Dense layout [column][row] with row stride n (master) / ldk (bf16 shadows).
// Rows i < probe_n draw counter j*probe_n + i; rows probe_n <= i < n are zero
// (the lower half of the probes [g; 0] of a Hermitian embedding).
// Ysh[k], k < pieces (pieces 0: none): the bf16 pieces of Y0 (see launch_tc_step).
// Probe j of the call is probe j0 + j of the seed's stream; kind PROBE_GIVEN
// copies the caller's probes Gin (probe_n x s, row-major, the path's type).
constexpr int PROBE_GIVEN = 2;
template <typename T>
cudaError_t launch_dense_init(T* G, T* Y0, __nv_bfloat16* const* Ysh, int pieces, int64_t ldk,
                              int64_t n, int S, int s, int kind, uint64_t seed, Partials P,
                              int rows_per_tile, cudaStream_t st, int64_t probe_n, int64_t j0,
                              const T* Gin);
// Banded layout [row][column] (row stride S).  Rademacher probes are packed
// as bits (bit j%64 of word j/64 of row i set when g_j[i] = -1; W words per
// row); Gaussian probes are stored as values G[i*s + j].
template <typename T>
cudaError_t launch_dia_init(T* G, uint64_t* bits, int W, T* Y0, int64_t n, int S, int s, int kind,
                            uint64_t seed, Partials P, int rows_per_tile, cudaStream_t st,
                            int64_t j0, const T* Gin);

// ---- conversions / checks (vne_prep.cu) --------------------------------------
cudaError_t launch_dense_convert_f64(const void* src, int src_dtype, int64_t n, int64_t ld,
                                     double* dst, cudaStream_t st);
cudaError_t launch_dense_convert_f32(const void* src, int src_dtype, int64_t n, int64_t ld,
                                     float* dst, cudaStream_t st);
// bf16 split, zero padded to rows_pad x ldk (ldk >= n): piece 0 = bf16(R), piece k
// = bf16(R - pieces 0..k-1), residuals in FP64; out[k] for k < pieces (1..3)
cudaError_t launch_dense_convert_bf16(const void* src, int src_dtype, int64_t n, int64_t ld,
                                      __nv_bfloat16* const* out, int pieces, int64_t rows_pad,
                                      int64_t ldk, cudaStream_t st);
// The same split of a rectangular block: rows x cols entries src[i*ld + k],
// zero padded to rows_pad x ldk.
cudaError_t launch_convert_bf16_rect(const void* src, int src_dtype, int64_t rows, int64_t cols,
                                     int64_t ld, __nv_bfloat16* const* out, int pieces,
                                     int64_t rows_pad, int64_t ldk, cudaStream_t st);
cudaError_t launch_dia_convert(const void* src, int src_dtype, int64_t n, int64_t ld, int D,
                               void* dst, int dst_dtype, cudaStream_t st);
// [[B, -C], [C, B]] of the Hermitian R = B + iC (complex dtype 2 or 3, n x n,
// ld complex elements) into dst (2n x 2n, ld 2n, FP64 if dst_dtype 0 else FP32)
cudaError_t launch_hermitian_embed(const void* src, int cdtype, int64_t n, int64_t ld, void* dst,
                                   int dst_dtype, cudaStream_t st);
// A full symmetric copy of a dense R whose upper triangle is authoritative
// (dtype 0 = FP64, 1 = FP32; in place when dst == src, then lds == ldd).
cudaError_t launch_dense_symmetrize(const void* src, int64_t lds, void* dst, int64_t ldd,
                                    int64_t n, int dtype, cudaStream_t st);
cudaError_t launch_trace(const void* R, int layout, int dtype, int64_t n, int64_t ld,
                         double* partial, unsigned int* counter, double* sc, cudaStream_t st);
cudaError_t launch_set_u(double* sc, double u, cudaStream_t st);

// ---- L2 residency of the bf16 R (vne_power.cu) ---------------------------------
// Rows [0, l2_keep_rows) of a matrix whose rows take row_bytes are loaded with
// an evict-last L2 policy by the power-method and tensor-core kernels, so that
// they stay in L2 from one pass over R to the next; the rest streams with
// evict-first.  Budget: VNE_L2_KEEP_MB (MB of the 129 MB L2; default 0, off).
int64_t l2_keep_rows(int64_t rows, int64_t row_bytes);

// ---- power method (vne_power.cu) ---------------------------------------------
// x vectors are stored [trial][row] in float (bf16/FP32 paths) or double (FP64).
template <typename TX>
cudaError_t launch_power_init(TX* x0, int64_t n, int q, uint64_t seed, double* sc,
                              cudaStream_t st);
// One product y = R (x / ||x||).  `final_step` computes the Rayleigh quotients,
// p1~ (SC_LAM) and u (SC_U) = min(1, u_scale * p1~).
cudaError_t launch_power_step_dense(const void* R, int rdtype /*0 f64,1 f32,2 bf16*/, int64_t n,
                                    int64_t ld, const void* x, void* y, int xdouble, int q,
                                    double* sc, double* partial, unsigned int* counter,
                                    int final_step, double u_scale, int nblocks_cap,
                                    cudaStream_t st);
// All t+1 products of the power method, R the sum of `pieces` (1 or 2) bf16
// pieces R[k] (rows_pad x ldk, symmetric; only the upper-triangle 128 x 128
// tiles are read), one trial, x0 the start vector; writes SC_LAM, SC_U and
// SC_NORM as the per-product kernels do.  One cooperative launch of `grid`
// CTAs, or (phased) 2t + 3 plain launches, one per phase, with the same
// result bits for any grid.  scratch: power_sym_scratch_bytes(rows_pad).
int64_t power_sym_scratch_bytes(int64_t rows_pad);
bool power_sym_fits(int64_t rows_pad, int grid);  // size limits of launch_power_sym
cudaError_t launch_power_sym(const __nv_bfloat16* const* R, int pieces, int64_t n,
                             int64_t rows_pad, int64_t ldk, const float* x0, int t, double* sc,
                             void* scratch, double u_scale, int grid, bool phased,
                             cudaStream_t st);
cudaError_t launch_power_step_dia(const void* vals, int rdtype /*0 f64,1 f32*/, int64_t n,
                                  int64_t ld, int D, const void* x, void* y, int q, double* sc,
                                  double* partial, unsigned int* counter, int final_step,
                                  double u_scale, int nblocks, cudaStream_t st);

// ---- dense SIMT recurrence (vne_dense_simt.cu) ---------------------------------
template <typename T>
cudaError_t launch_dense_simt_step(const T* R, int64_t ld, int64_t n, const T* Yprev, T* Zpart,
                                   int S, int col0, int ncols, int splitk, cudaStream_t st);
template <typename T>
cudaError_t launch_dense_simt_epilogue(const T* Zpart, int splitk, const T* G, const T* Yprev,
                                       const T* Yprev2, T* Ynew, int64_t n, int S, int s,
                                       StepCols cols, const double* sc, Partials P, int t,
                                       cudaStream_t st);
int dense_simt_splitk(int64_t n, int ncols, int sm_count, int elt_bytes);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel, device and
// size (a process-wide table; later calls with a size already set are no-ops).
cudaError_t set_max_dynamic_smem(const void* kernel, int bytes);

// ---- banded recurrence (vne_dia.cu) --------------------------------------------
template <typename T>
cudaError_t launch_dia_step(const T* vals, int64_t ld, int D, int64_t n, const T* Yprev,
                            const T* Yprev2, T* Ynew, const T* G, const uint64_t* bits, int W,
                            int S, int s, StepCols cols, const double* sc, Partials P, int t,
                            int nblocks, cudaStream_t st, int band_aligned);
int dia_supported_halfbw(int D);  // the compiled window >= D-1, or -1
// Grid of the banded step; band_aligned: the operand band starts on a 16-byte
// boundary with ld a multiple of 4 (FP32), which selects the bulk-copy kernel
// for S in {32, 64, 128}.  launch_dia_step takes the same flag.
int dia_step_grid(int is_double, int D, int64_t n, int ncols, int s, int sm_count,
                  int band_aligned);
// The bulk-copy FP32 step (vne_dia_tma.cu): where it applies, its grid, and
// its launch (Y [n][S], S in {32, 64, 128}; the arguments of launch_dia_step).
bool dia_tma_ok(int is_double, int D, int64_t n, int S, int s, int band_aligned);
int dia_tma_grid(int D, int64_t n, int S, int sm_count);
cudaError_t launch_dia_step_tma(const float* vals, int64_t ld, int D, int64_t n, const float* Yprev,
                                const float* Yprev2, float* Ynew, const float* G,
                                const uint64_t* bits, int Wd, int S, int s, StepCols cols,
                                const double* sc, Partials P, int t, int nblocks, cudaStream_t st);

// ---- dense tensor-core recurrence (vne_tc.cu) -------------------------------------
// R and Y are each a sum of `pieces` bf16 matrices (1: BF16; 2: bf16x3; 3:
// bf16x6): piece k holds the rounding residual of pieces 0..k-1.  The step
// accumulates the products R_a Y_b with a + b < pieces in FP32 (1, 3 or 6).
constexpr int kMaxPieces = 3;
struct TcStep {
    const __nv_bfloat16* R[kMaxPieces];  // [rows_pad][ldk]; pieces >= `pieces` unused
    const __nv_bfloat16* Y[kMaxPieces];  // shadows of Y_{t-1}, [S_pad][ldk]
    __nv_bfloat16* Y_out[kMaxPieces];    // shadows of Y_t
    int pieces;
    const float* G;             // [s][n]
    const float* Yprev;         // FP32 master Y_{t-1} [S][n]
    const float* Yprev2;        // FP32 master Y_{t-2}
    float* Ynew;                // FP32 master Y_t
    int64_t n, rows_pad, ldk;
    int S, s, split;
    StepCols cols;
    const double* sc;
    Partials P;
    int t;
};
cudaError_t launch_tc_step(const TcStep& a, int sm_count, cudaStream_t st);
// A 2-D tensor map of a bf16 matrix (inner x rows, row stride in elements)
// with box box_inner x box_rows and no swizzle (rows land in shared memory as
// stored); false if the driver refuses it.
bool tma_map_bf16_plain(void* map, const void* base, int64_t inner, int64_t rows,
                        int64_t row_stride_elems, int box_inner, int box_rows);
// The operand map of the tensor-core steps: bf16 rows of `inner` elements,
// box 64 (128-byte rows, 128-byte swizzle) x box_rows.
bool tma_map_bf16_operand(void* map, const void* base, int64_t inner, int64_t rows,
                          int64_t row_stride_elems, int box_rows);

// ---- batched recurrence, one persistent launch (vne_tc_batch.cu) ---------------
// One matrix of a batch after its prologue (bf16 R, power method, probe block):
// the buffers of the single-call BF16 path, whose layout the steps keep.
struct TcBatchMat {
    const __nv_bfloat16* R;   // [rows_pad][ldk]
    __nv_bfloat16* sh[2];     // bf16 probe blocks [S_pad][ldk]; Y_0 in sh[0]
    const float* G;           // [s][n]
    float* Y[3];              // FP32 masters [S][n]; Y_0 in Y[0]
    const double* sc;         // scalar block (u)
    double* flags;            // &sc[SC_FLAGS], raised on a timeout
    Partials P;               // moment partials, ntiles = rows_pad / 128
    int64_t n, rows_pad, ldk;
    int S, s, m, T, tiles, has_cheb, has_tay;
    // power method in the batch's persistent launch (NULL x[0]: u is given)
    float* x[2];              // iterates [n]; x_0 in x[0]
    double* ppart;            // per-tile norm partials [2][tiles][3]
};
// Work items of the queue in launch order, (matrix, step, row tile), built so
// that every item's dependencies (all tiles of the previous step of its
// matrix) come earlier: rounds over an active set of matrices, admitted in the
// given order while their bf16 R fit `budget_bytes` or the round has fewer
// than `min_tiles` tiles.  Returns the item count; items may be NULL.
int64_t tc_batch_schedule(const TcBatchMat* mats, int count, double budget_bytes, int min_tiles,
                          int* items);
// Bytes of the launch's device table (maps, matrices, items, counters).
size_t tc_batch_table_bytes(const TcBatchMat* mats, int count, int64_t n_items);
// Fills the table in host memory `host` (pinned, tc_batch_table_bytes) for the
// device copy `dev`, copies it, clears the counters and launches the kernel
// on `st` (grid: 2 CTAs per SM).
// dep_extra > 0 raises every dependency's required count beyond what can
// arrive (a test of the bounded waits: the launch times out, FLAG_TIMEOUT).
cudaError_t launch_tc_batch(const TcBatchMat* mats, int count, const int* items, int64_t n_items,
                            void* host, void* dev, int sm_count, cudaStream_t st,
                            int dep_extra = 0);
// The power method (Algorithm alg:power, one trial, t + 1 products with the
// bf16 R) of every matrix with x[0] set, in one persistent launch: items
// (matrix, product k, 128-row tile) from `items` (the schedule of
// tc_batch_schedule with T = t + 1); the last product writes p1~, u =
// min(1, u_scale p1~) and the norm sums to each matrix's scalar block.  The
// table (host, dev) is laid out as for launch_tc_batch.
cudaError_t launch_power_batch(const TcBatchMat* mats, int count, const int* items,
                               int64_t n_items, int power_iters, double u_scale, void* host,
                               void* dev, int sm_count, cudaStream_t st, int dep_extra = 0);

// autotuner: set (BN = 0 clears) the shape of n x ncols steps; candidates
int tc_set_tuned(int64_t n, int ncols, int BN, int CM, int CN, int ksplit);
int tc_candidates(int64_t n, int ncols, int (*out)[4], int max);
// The shape launch_tc_step would use for n rows and ncols step columns on
// sm_count SMs: out = {BN, CM, CN, ksplit}; 0, or -1 on bad arguments.
int tc_plan(int64_t n, int ncols, int sm_count, int* out);
int tc_tile_m();
int tc_tile_k();

// ---- random projection (vne_proj.cu) ------------------------------------------------
// Pi stored [s][n]; kind 0 Gaussian, 1 SRHT, 2 input-sparsity (vne.h VNE_SKETCH_*).
template <typename T>
cudaError_t launch_sketch(T* Pi, int64_t n, int s, int kind, uint64_t seed, int sm_count,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_split_sum(const T* Zpart, int splitk, int64_t len, T* Z, int sm_count,
                             cudaStream_t st);
int gram_chunks(int64_t n, int s, int sm_count);
// C (s x s, FP64, exactly symmetric) = Z^T Z for Z stored [s][n]; part holds chunks*s*s.
template <typename T>
cudaError_t launch_gram(const T* Z, int64_t n, int s, int chunks, double* part, double* C,
                        cudaStream_t st);
// The `top` largest eigenvalues (descending, evals[0..top)) of a symmetric
// N x N FP64 matrix, N <= 512; Wg is N*N scratch, d and e N each.
cudaError_t launch_sym_eigvals(const double* A, int N, int top, double* Wg, double* d, double* e,
                               double* evals, cudaStream_t st);
// out[0] = H~, out[1..k] = p~ from the k largest Gram eigenvalues.
cudaError_t launch_proj_combine(const double* evals, int k, double* out, cudaStream_t st);
// block Krylov pieces
template <typename T>
cudaError_t launch_xgram(const T* A, int ra, const T* B, int rb, int64_t n, int chunks,
                         double* part, double* C, cudaStream_t st);
template <typename T>
cudaError_t launch_ts_mm(const T* A, int ra, const double* M, int rc, double scale, const T* In,
                         T* Out, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_jacobi(const double* G, int b, double* lam, double* U, cudaStream_t st);
cudaError_t launch_basis_coeffs(const double* lam, const double* U, int b, double* lam_ref,
                                int first, double drop, double* M, cudaStream_t st);
cudaError_t launch_symmetrize(double* T, int N, cudaStream_t st);
cudaError_t launch_krylov_combine(const double* ev, int k, int64_t n, double* out,
                                  cudaStream_t st);

// ---- learned correction (vne_mlp.cu) ------------------------------------------------
cudaError_t launch_spectral_sample(int count, const int* kind, const int* n, const float* a,
                                   const int* ktop, const float* floor, const float* c,
                                   const uint64_t* seeds, int m, int s, float* feat, float* target,
                                   double* H_exact, double* H_low, double* totals,
                                   cudaStream_t st);
size_t mlp_workspace_floats(int B);
cudaError_t mlp_forward(const float* th, const float* X, int B, float* y, float* ws, int* launches,
                        cudaStream_t st);
cudaError_t mlp_loss_grad(const float* th, const float* X, const float* t, const int* idx, int B,
                          float* grad, double* loss, float* ws, int* launches, cudaStream_t st);
cudaError_t mlp_train_step(float* th, float* am, float* av, int step, float lr, const float* X,
                           const float* t, int64_t rows, int B, int64_t first, uint64_t perm_seed,
                           int* idx, float* grad, double* loss, float* ws, int* launches,
                           cudaStream_t st);
// ws: 64 + mlp_workspace_floats(1) floats
cudaError_t launch_learned(const double* mom, int m, int s, int64_t n, double* sc,
                           const float* params, float* ws, int* launches, cudaStream_t st);

// ---- bounded-wait check (vne_selftest.cu) ----------------------------------------
cudaError_t launch_wait_never(double* sc, cudaStream_t st);

// ---- combine (vne_combine.cu) ----------------------------------------------------
// moments[k][j] for k = 0..m of the Chebyshev columns / Taylor columns, then
// the FP64 estimates into sc.
cudaError_t launch_combine(Partials P, int s, int m, int cheb_c0, int tay_c0, double* mom_cheb,
                           double* mom_taylor, double* sc, cudaStream_t st);
// Only the final stage: the estimates from per-probe moments already in
// mom_cheb / mom_taylor (either may be NULL) and u in sc.
cudaError_t launch_combine_final(int s, int m, const double* mom_cheb, const double* mom_taylor,
                                 double* sc, cudaStream_t st);

}  // namespace vne
