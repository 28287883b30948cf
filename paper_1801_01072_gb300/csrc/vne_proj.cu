// Random-projection estimator (Algorithm alg:EN, Section 5) on the GPU:
//   1. the random projection Pi (n x s): Gaussian, subsampled randomized
//      Hadamard (Algorithm alg:SHD) or input-sparsity (Algorithm alg:IS),
//      generated from counters, stored [s][n];
//   2. R~ = R Pi on the dense SIMT product kernel (vne_dense_simt.cu);
//   3. the s x s Gram matrix R~^T R~ accumulated in FP64;
//   4. its eigenvalues (Householder reduction to tridiagonal form, then
//      Sturm-sequence bisection), i.e. the squared singular values of R~;
//   5. p~_i = sqrt(lambda_i) for the k largest and H~ = sum p~_i ln(1/p~_i).
// The Gram route squares the singular values: the top-k p~_i keep full
// relative accuracy, values below ~1e-8 p~_1 (FP64) only absolute accuracy,
// and they enter H~ as p ln(1/p), i.e. at the 1e-15 level.
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

constexpr uint64_t kSketchSignXor = 0xA0761D6478BD642Full;
constexpr uint64_t kSketchIndexXor = 0xE7037ED1A0B428DBull;

// floor(u * m) with u = (out >> 11) / 2^53 in [0, 1), as an FP64 product
// (exact for m a power of two, and the same IEEE product otherwise).
__device__ __forceinline__ int64_t uniform_index(uint64_t seed, uint64_t t, int64_t m) {
    const double u = (double)(splitmix_out(seed ^ kSketchIndexXor, t) >> 11) * 0x1.0p-53;
    int64_t v = (int64_t)floor(u * (double)m);
    return v < m - 1 ? v : m - 1;
}

__device__ __forceinline__ double sketch_sign(uint64_t seed, uint64_t i) {
    return (splitmix_out(seed ^ kSketchSignXor, i) >> 63) ? -1.0 : 1.0;
}

template <typename T> __device__ __forceinline__ T gauss_t(uint64_t seed, uint64_t e);
template <> __device__ __forceinline__ double gauss_t<double>(uint64_t seed, uint64_t e) {
    return gaussian(seed, e);
}
template <> __device__ __forceinline__ float gauss_t<float>(uint64_t seed, uint64_t e) {
    return gaussian_f32(seed, e);
}

// Pi[c*n + i] for i < n, c < s.  kind 0 Gaussian / sqrt(s); kind 1 SRHT:
// D_i (-1)^popcount(i & idx_c) / sqrt(s) with idx_c uniform in [0, N), N the
// next power of two >= n (R read as zero-padded to N); kind 2 input-sparsity:
// D_i where h(i) = c, else 0.
template <typename T>
__global__ void k_sketch(T* __restrict__ Pi, int64_t n, int s, int kind, uint64_t seed, int64_t N) {
    const int64_t total = n * (int64_t)s;
    const double inv_sqrt_s = 1.0 / sqrt((double)s);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        T v;
        if (kind == 0) {
            v = (T)((double)gauss_t<T>(seed, (uint64_t)e) * inv_sqrt_s);
        } else if (kind == 1) {
            const uint64_t idx = (uint64_t)uniform_index(seed, (uint64_t)c, N);
            const int par = __popcll((unsigned long long)((uint64_t)i & idx)) & 1;
            v = (T)(sketch_sign(seed, (uint64_t)i) * (par ? -inv_sqrt_s : inv_sqrt_s));
        } else {
            v = (uniform_index(seed, (uint64_t)i, s) == c) ? (T)sketch_sign(seed, (uint64_t)i) : (T)0;
        }
        Pi[e] = v;
    }
}

template <typename T>
cudaError_t launch_sketch(T* Pi, int64_t n, int s, int kind, uint64_t seed, int sm_count,
                          cudaStream_t st) {
    int64_t N = 1;
    while (N < n) N <<= 1;
    const int64_t total = n * (int64_t)s;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8 * (int64_t)sm_count) blocks = 8 * (int64_t)sm_count;
    k_sketch<T><<<(unsigned)blocks, 256, 0, st>>>(Pi, n, s, kind, seed, N);
    return cudaGetLastError();
}

// Z = sum over the K splits of Zpart[split][s][n] (in split order).
template <typename T>
__global__ void k_split_sum(const T* __restrict__ Zpart, int splitk, int64_t len, T* __restrict__ Z) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        T acc = Zpart[e];
        for (int k = 1; k < splitk; ++k) acc += Zpart[(int64_t)k * len + e];
        Z[e] = acc;
    }
}

template <typename T>
cudaError_t launch_split_sum(const T* Zpart, int splitk, int64_t len, T* Z, int sm_count,
                             cudaStream_t st) {
    int64_t blocks = (len + 255) / 256;
    if (blocks > 8 * (int64_t)sm_count) blocks = 8 * (int64_t)sm_count;
    k_split_sum<T><<<(unsigned)blocks, 256, 0, st>>>(Zpart, splitk, len, Z);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gram matrix C = Z^T Z of Z stored [s][n]: 32 x 32 output tiles, the rows
// split into `chunks` slices whose FP64 partials are summed in slice order.
// Entry (a, b) and (b, a) take the same products in the same order, so C is
// exactly symmetric.
// ---------------------------------------------------------------------------
constexpr int GR_T = 32, GR_K = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ Z, int64_t n, int s,
                                              int64_t rows_per_chunk, double* __restrict__ part) {
    __shared__ double As[GR_K][GR_T + 1];
    __shared__ double Bs[GR_K][GR_T + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.y * GR_T, b0 = blockIdx.x * GR_T;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk;
    int64_t r1 = r0 + rows_per_chunk;
    if (r1 > n) r1 = n;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t k0 = r0; k0 < r1; k0 += GR_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int col = e >> 5, kk = e & 31;
            const int64_t r = k0 + kk;
            const int ca = a0 + col, cb = b0 + col;
            As[kk][col] = (ca < s && r < r1) ? (double)Z[(int64_t)ca * n + r] : 0.0;
            Bs[kk][col] = (cb < s && r < r1) ? (double)Z[(int64_t)cb * n + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GR_K; ++kk) {
            const double x0 = As[kk][ty * 2], x1 = As[kk][ty * 2 + 1];
            const double y0 = Bs[kk][tx * 2], y1 = Bs[kk][tx * 2 + 1];
            acc[0][0] = fma(x0, y0, acc[0][0]);
            acc[0][1] = fma(x0, y1, acc[0][1]);
            acc[1][0] = fma(x1, y0, acc[1][0]);
            acc[1][1] = fma(x1, y1, acc[1][1]);
        }
        __syncthreads();
    }
    double* out = part + (int64_t)blockIdx.z * s * s;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int a = a0 + ty * 2 + i, b = b0 + tx * 2 + j;
            if (a < s && b < s) out[(int64_t)a * s + b] = acc[i][j];
        }
}

__global__ void k_sum_chunks(const double* __restrict__ part, int chunks, int64_t len,
                             double* __restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = part[e];
        for (int k = 1; k < chunks; ++k) acc += part[(int64_t)k * len + e];
        C[e] = acc;
    }
}

int gram_chunks(int64_t n, int s, int sm_count) {
    const int64_t tiles = (int64_t)((s + GR_T - 1) / GR_T) * ((s + GR_T - 1) / GR_T);
    int64_t chunks = (2 * (int64_t)sm_count + tiles - 1) / tiles;
    const int64_t max_chunks = (n + 255) / 256;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks > 64) chunks = 64;
    if (chunks < 1) chunks = 1;
    return (int)chunks;
}

template <typename T>
cudaError_t launch_gram(const T* Z, int64_t n, int s, int chunks, double* part, double* C,
                        cudaStream_t st) {
    int64_t rows = (n + chunks - 1) / chunks;
    rows = (rows + GR_K - 1) / GR_K * GR_K;
    dim3 grid((unsigned)((s + GR_T - 1) / GR_T), (unsigned)((s + GR_T - 1) / GR_T), (unsigned)chunks);
    k_gram<T><<<grid, 256, 0, st>>>(Z, n, s, rows, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t len = (int64_t)s * s;
    k_sum_chunks<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, chunks, len, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Symmetric eigenvalues, N <= kEigMaxN, one block.
// Householder reduction (Golub & Van Loan, Algorithm 8.3.1): for column k,
// x = A[k+1:, k], alpha = -sign(x_0) ||x||, v = (x - alpha e_1) / ||.||,
// p = A_sub v, w = p - (v^T p) v, A_sub -= 2 (v w^T + w v^T); the diagonal
// and alpha form the tridiagonal (d, e).  A is worked on in place in W (shared
// memory when it fits, otherwise the caller's global scratch).
// ---------------------------------------------------------------------------
constexpr int kEigMaxN = 512;
constexpr int kEigThreads = 512;

__device__ __forceinline__ double block_sum_bcast(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

__global__ void __launch_bounds__(kEigThreads) k_tridiag(const double* __restrict__ A, int N,
                                                         double* __restrict__ Wg, int use_smem,
                                                         double* __restrict__ d_out,
                                                         double* __restrict__ e_out) {
    extern __shared__ double dyn[];
    __shared__ double v[kEigMaxN], p[kEigMaxN], red[32];
    double* W = use_smem ? dyn : Wg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int64_t e = tid; e < (int64_t)N * N; e += blockDim.x) W[e] = A[e];
    __syncthreads();
    for (int k = 0; k + 2 < N; ++k) {
        const int m = N - k - 1;
        const int o = k + 1;
        double part_tail = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            const double x = W[(int64_t)(o + i) * N + k];
            v[i] = x;
            if (i > 0) part_tail += x * x;
        }
        const double tail = block_sum_bcast(part_tail, red);  // ends with a barrier
        const double x0 = v[0];
        if (tail == 0.0) {
            if (tid == 0) {
                d_out[k] = W[(int64_t)k * N + k];
                e_out[k] = x0;
            }
            __syncthreads();
            continue;
        }
        const double xx = tail + x0 * x0;
        const double alpha = x0 >= 0.0 ? -sqrt(xx) : sqrt(xx);
        const double v0 = x0 - alpha;
        const double scale = 1.0 / sqrt(tail + v0 * v0);
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) v[i] = (i == 0 ? v0 : v[i]) * scale;
        __syncthreads();
        // p = A_sub v, one warp per row
        for (int r = warp; r < m; r += nwarps) {
            const double* row = W + (int64_t)(o + r) * N + o;
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc = fma(row[j], v[j], acc);
            acc = warp_sum(acc);
            if (lane == 0) p[r] = acc;
        }
        __syncthreads();
        double part_k = 0.0;
        for (int i = tid; i < m; i += blockDim.x) part_k += v[i] * p[i];
        const double K = block_sum_bcast(part_k, red);
        for (int i = tid; i < m; i += blockDim.x) p[i] -= K * v[i];
        __syncthreads();
        for (int r = warp; r < m; r += nwarps) {
            double* row = W + (int64_t)(o + r) * N + o;
            const double vr = v[r], wr = p[r];
            for (int j = lane; j < m; j += 32) row[j] -= 2.0 * (vr * p[j] + wr * v[j]);
        }
        if (tid == 0) {
            d_out[k] = W[(int64_t)k * N + k];
            e_out[k] = alpha;
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (N >= 2) {
            d_out[N - 2] = W[(int64_t)(N - 2) * N + (N - 2)];
            e_out[N - 2] = W[(int64_t)(N - 1) * N + (N - 2)];
        }
        d_out[N - 1] = W[(int64_t)(N - 1) * N + (N - 1)];
        e_out[N - 1] = 0.0;
    }
}

// Number of eigenvalues of the tridiagonal (d, e) below x (Sturm sequence of
// the LDL^T pivots; a pivot of magnitude <= pivmin is replaced by -pivmin).
__device__ __forceinline__ int sturm_count(const double* d, const double* e, int N, double x,
                                           double pivmin) {
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) <= pivmin) q = -pivmin;
    if (q < 0.0) ++c;
    for (int i = 1; i < N; ++i) {
        q = d[i] - x - (e[i - 1] * e[i - 1]) / q;
        if (fabs(q) <= pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

// Bisection: thread j finds the j-th smallest eigenvalue and stores it at
// evals[N-1-j] (descending order).
__global__ void k_bisect(const double* __restrict__ d_in, const double* __restrict__ e_in, int N,
                         double* __restrict__ evals) {
    __shared__ double d[kEigMaxN], e[kEigMaxN];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        d[i] = d_in[i];
        e[i] = e_in[i];
    }
    __syncthreads();
    double lo = d[0], hi = d[0], emax2 = 0.0;
    for (int i = 0; i < N; ++i) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < N ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < N) emax2 = fmax(emax2, e[i] * e[i]);
    }
    const double pivmin = 0x1.0p-1022 * fmax(1.0, emax2);
    const double pad = 2.2204460492503131e-16 * fmax(fabs(lo), fabs(hi)) + pivmin;
    lo -= pad;
    hi += pad;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double a = lo, b = hi;
    for (int it = 0; it < 256; ++it) {
        const double mid = 0.5 * (a + b);
        if (!(mid > a && mid < b)) break;
        if (sturm_count(d, e, N, mid, pivmin) >= j + 1) b = mid;
        else a = mid;
    }
    evals[N - 1 - j] = 0.5 * (a + b);
}

cudaError_t launch_sym_eigvals(const double* A, int N, double* Wg, double* d, double* e,
                               double* evals, cudaStream_t st) {
    if (N < 1 || N > kEigMaxN) return cudaErrorInvalidValue;
    const size_t smem = (size_t)N * N * sizeof(double);
    const int use_smem = smem <= 160 * 1024;
    if (use_smem) {
        cudaError_t r = cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r != cudaSuccess) return r;
    }
    k_tridiag<<<1, kEigThreads, use_smem ? smem : 0, st>>>(A, N, Wg, use_smem, d, e);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    k_bisect<<<(N + 31) / 32, 32, 0, st>>>(d, e, N, evals);
    return cudaGetLastError();
}

// out[0] = H~ = sum_{i<k, p~_i>0} p~_i ln(1/p~_i); out[1+i] = p~_i = sqrt(max(lambda_i, 0)).
__global__ void k_proj_combine(const double* __restrict__ evals, int k, double* __restrict__ out) {
    __shared__ double red[32];
    double h = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double p = sqrt(fmax(evals[i], 0.0));
        out[1 + i] = p;
        if (p > 0.0) h -= p * log(p);
    }
    const double H = block_sum(h, red);
    if (threadIdx.x == 0) out[0] = H;
}

cudaError_t launch_proj_combine(const double* evals, int k, double* out, cudaStream_t st) {
    k_proj_combine<<<1, 256, 0, st>>>(evals, k, out);
    return cudaGetLastError();
}

template cudaError_t launch_sketch<double>(double*, int64_t, int, int, uint64_t, int, cudaStream_t);
template cudaError_t launch_sketch<float>(float*, int64_t, int, int, uint64_t, int, cudaStream_t);
template cudaError_t launch_split_sum<double>(const double*, int, int64_t, double*, int, cudaStream_t);
template cudaError_t launch_split_sum<float>(const float*, int, int64_t, float*, int, cudaStream_t);
template cudaError_t launch_gram<double>(const double*, int64_t, int, int, double*, double*,
                                         cudaStream_t);
template cudaError_t launch_gram<float>(const float*, int64_t, int, int, double*, double*,
                                        cudaStream_t);

}  // namespace vne
