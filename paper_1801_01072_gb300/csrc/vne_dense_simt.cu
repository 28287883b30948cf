// Dense recurrence on the CUDA cores (FP64 or FP32): Z = R Y_{t-1}, then the
// three-term (Chebyshev, Section 3) or Taylor (Section 2) update and the
// per-probe moment partials.  This is the plain-precision path: FP64 is the
// reference the mixed-precision tensor-core path is measured against.
//
// Layout: R row-major (ld), Y column blocks [S][n] (probe c contiguous).
// FP64 step kernel: 32 x 32 output tile, K split into `splitk` slices so that
// small problems still fill the GPU; partial products go to Zpart[split][S][n]
// and the epilogue kernel sums them in split order (deterministic).
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

constexpr int SB_M = 32, SB_N = 32, SB_K = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_simt_step(const T* __restrict__ R, int64_t ld, int64_t n,
                                                   const T* __restrict__ Y, T* __restrict__ Zpart,
                                                   int S, int col0, int ncols, int64_t kchunk) {
    __shared__ T As[SB_K][SB_M + 1];
    __shared__ T Bs[SB_K][SB_N + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * SB_M;
    const int c0 = col0 + blockIdx.y * SB_N;
    const int cend = col0 + ncols;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    int64_t ke = kb + kchunk;
    if (ke > n) ke = n;
    T acc[2][2] = {{(T)0, (T)0}, {(T)0, (T)0}};
    for (int64_t k0 = kb; k0 < ke; k0 += SB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int r = e >> 5, kk = e & 31;
            const int64_t i = i0 + r, k = k0 + kk;
            As[kk][r] = (i < n && k < ke) ? R[i * ld + k] : (T)0;
            const int c = c0 + r;
            Bs[kk][r] = (c < cend && k < ke) ? Y[(int64_t)c * n + k] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < SB_K; ++kk) {
            const T a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
            const T b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            acc[0][0] = Math<T>::fma(a0, b0, acc[0][0]);
            acc[0][1] = Math<T>::fma(a0, b1, acc[0][1]);
            acc[1][0] = Math<T>::fma(a1, b0, acc[1][0]);
            acc[1][1] = Math<T>::fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t i = i0 + ty * 2 + a;
            const int c = c0 + tx * 2 + b;
            if (i < n && c < cend) Zpart[((int64_t)blockIdx.z * S + c) * n + i] = acc[a][b];
        }
}

// FP32 step: 128 x 64 output tile, 8 x 4 outputs per thread from a
// register tile (two float4 loads of R's column slice and one of Y's per k),
// K staged 16 at a time.  blockIdx.x runs over the column tiles, so the CTAs
// that share a 128-row block of R are launched together and R is fetched from
// HBM about once (the other column tiles hit in L2).
constexpr int FB_M = 128, FB_N = 64, FB_K = 16;

__global__ void __launch_bounds__(256) k_simt_step_f32(const float* __restrict__ R, int64_t ld,
                                                       int64_t n, const float* __restrict__ Y,
                                                       float* __restrict__ Zpart, int S, int col0,
                                                       int ncols, int64_t kchunk, int vec) {
    __shared__ __align__(16) float As[FB_K][FB_M + 4];
    __shared__ __align__(16) float Bs[FB_K][FB_N + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int c0 = col0 + blockIdx.x * FB_N;
    const int64_t i0 = (int64_t)blockIdx.y * FB_M;
    const int cend = col0 + ncols;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    int64_t ke = kb + kchunk;
    if (ke > n) ke = n;
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int ar = tid >> 1, ak = (tid & 1) * 8;   // A: row, first k of 8
    const int bc = tid >> 2, bk = (tid & 3) * 4;   // B: column, first k of 4
    const int64_t arow = i0 + ar;
    const int bcol = c0 + bc;
    for (int64_t k0 = kb; k0 < ke; k0 += FB_K) {
        float a[8], bv[4];
        if (vec && arow < n && k0 + ak + 8 <= ke) {
            const float4 x = *reinterpret_cast<const float4*>(R + arow * ld + k0 + ak);
            const float4 y = *reinterpret_cast<const float4*>(R + arow * ld + k0 + ak + 4);
            a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
            a[4] = y.x; a[5] = y.y; a[6] = y.z; a[7] = y.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t k = k0 + ak + q;
                a[q] = (arow < n && k < ke) ? R[arow * ld + k] : 0.f;
            }
        }
        if (vec && bcol < cend && k0 + bk + 4 <= ke) {
            const float4 y = *reinterpret_cast<const float4*>(Y + (int64_t)bcol * n + k0 + bk);
            bv[0] = y.x; bv[1] = y.y; bv[2] = y.z; bv[3] = y.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t k = k0 + bk + q;
                bv[q] = (bcol < cend && k < ke) ? Y[(int64_t)bcol * n + k] : 0.f;
            }
        }
        __syncthreads();  // the previous slice has been consumed
#pragma unroll
        for (int q = 0; q < 8; ++q) As[ak + q][ar] = a[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) Bs[bk + q][bc] = bv[q];
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < FB_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bw[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bw[c], acc[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (i >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = c0 + tx * 4 + c;
            if (col < cend) Zpart[((int64_t)blockIdx.z * S + col) * n + i] = acc[r][c];
        }
    }
}

int dense_simt_splitk(int64_t n, int ncols, int sm_count, int elt_bytes) {
    const int64_t tm = elt_bytes == 4 ? FB_M : SB_M, tn = elt_bytes == 4 ? FB_N : SB_N;
    const int64_t tiles = ((n + tm - 1) / tm) * ((ncols + tn - 1) / tn);
    const int64_t kblocks = (n + SB_K - 1) / SB_K;
    int64_t split = 1;
    while (tiles * split < 2 * (int64_t)sm_count && split * 2 <= kblocks && split < 16) split *= 2;
    return (int)split;
}

template <typename T>
cudaError_t launch_dense_simt_step(const T* R, int64_t ld, int64_t n, const T* Yprev, T* Zpart,
                                   int S, int col0, int ncols, int splitk, cudaStream_t st) {
    const int64_t kblocks = (n + SB_K - 1) / SB_K;
    const int64_t kchunk = ((kblocks + splitk - 1) / splitk) * SB_K;
    if (sizeof(T) == 4) {
        const int vec = (ld % 4 == 0) && (n % 4 == 0) &&
                        (reinterpret_cast<uintptr_t>(R) % 16 == 0) &&
                        (reinterpret_cast<uintptr_t>(Yprev) % 16 == 0);
        dim3 grid((unsigned)((ncols + FB_N - 1) / FB_N), (unsigned)((n + FB_M - 1) / FB_M),
                  (unsigned)splitk);
        k_simt_step_f32<<<grid, 256, 0, st>>>((const float*)R, ld, n, (const float*)Yprev,
                                              (float*)Zpart, S, col0, ncols, kchunk, vec);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((n + SB_M - 1) / SB_M), (unsigned)((ncols + SB_N - 1) / SB_N),
              (unsigned)splitk);
    k_simt_step<T><<<grid, 256, 0, st>>>(R, ld, n, Yprev, Zpart, S, col0, ncols, kchunk);
    return cudaGetLastError();
}
template cudaError_t launch_dense_simt_step<double>(const double*, int64_t, int64_t, const double*,
                                                    double*, int, int, int, int, cudaStream_t);
template cudaError_t launch_dense_simt_step<float>(const float*, int64_t, int64_t, const float*,
                                                   float*, int, int, int, int, cudaStream_t);

// One thread per row, blockIdx.y = active column index; rows_per_tile = 256.
template <typename T>
__global__ void __launch_bounds__(256) k_simt_epilogue(const T* __restrict__ Zpart, int splitk,
                                                       const T* __restrict__ G,
                                                       const T* __restrict__ Yprev,
                                                       const T* __restrict__ Yprev2,
                                                       T* __restrict__ Ynew, int64_t n, int S,
                                                       int s, StepCols cols, const double* sc,
                                                       Partials P, int t) {
    __shared__ double sh[32];
    const int ci = blockIdx.y;
    const bool is_cheb = ci < cols.ncheb;
    const int c = is_cheb ? cols.cheb_c0 + ci : cols.tay_c0 + (ci - cols.ncheb);
    const int j = c % s;
    const double u = sc[SC_U];
    const T a = (T)(2.0 / u), invu = (T)(1.0 / u);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double mom = 0.0;
    if (i < n) {
        T z = (T)0;
        for (int q = 0; q < splitk; ++q) z += Zpart[((int64_t)q * S + c) * n + i];
        const T g = G[(int64_t)j * n + i];
        const int64_t idx = (int64_t)c * n + i;
        if (is_cheb) {
            T y;
            if (cols.cheb_kind == EPI_CHEB1) y = a * z - g;
            else y = (T)2 * (a * z - Yprev[idx]) - Yprev2[idx];
            Ynew[idx] = y;
            mom = (double)g * (double)y;
        } else {
            mom = (double)g * (double)z;
            Ynew[idx] = Yprev[idx] - z * invu;
        }
    }
    const double tot = block_sum(mom, sh);
    if (threadIdx.x == 0) P.slot(t)[(size_t)blockIdx.x * S + c] = tot;
}

template <typename T>
cudaError_t launch_dense_simt_epilogue(const T* Zpart, int splitk, const T* G, const T* Yprev,
                                       const T* Yprev2, T* Ynew, int64_t n, int S, int s,
                                       StepCols cols, const double* sc, Partials P, int t,
                                       cudaStream_t st) {
    const int nact = cols.ncheb + cols.ntay;
    if (nact <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)nact);
    k_simt_epilogue<T><<<grid, 256, 0, st>>>(Zpart, splitk, G, Yprev, Yprev2, Ynew, n, S, s, cols,
                                             sc, P, t);
    return cudaGetLastError();
}
template cudaError_t launch_dense_simt_epilogue<double>(const double*, int, const double*,
                                                        const double*, const double*, double*,
                                                        int64_t, int, int, StepCols, const double*,
                                                        Partials, int, cudaStream_t);
template cudaError_t launch_dense_simt_epilogue<float>(const float*, int, const float*,
                                                       const float*, const float*, float*, int64_t,
                                                       int, int, StepCols, const double*, Partials,
                                                       int, cudaStream_t);

}  // namespace vne
