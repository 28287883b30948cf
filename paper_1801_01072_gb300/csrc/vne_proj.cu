// Random-projection estimator (Algorithm alg:EN, Section 5) on the GPU:
//   1. the random projection Pi (n x s): Gaussian, subsampled randomized
//      Hadamard (Algorithm alg:SHD) or input-sparsity (Algorithm alg:IS),
//      generated from counters, stored [s][n];
//   2. R~ = R Pi on the dense SIMT product kernel (vne_dense_simt.cu);
//   3. the s x s Gram matrix R~^T R~ (FP64, or compensated FP32 sums);
//   4. its eigenvalues (Householder reduction to tridiagonal form, then
//      Sturm-sequence bisection), i.e. the squared singular values of R~;
//   5. p~_i = sqrt(lambda_i) for the k largest and H~ = sum p~_i ln(1/p~_i).
// The Gram route squares the singular values: the top-k p~_i keep full
// relative accuracy, values below ~1e-8 p~_1 (FP64) only absolute accuracy,
// and they enter H~ as p ln(1/p), i.e. at the 1e-15 level.
#include <cstdlib>

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
// Gram matrix C = Z^T Z of Z stored [s][n]: 32 x 32 output tiles of the lower
// triangle (mirrored on store), the rows split into `chunks` slices whose
// partials are summed in slice order.  Entries (a, b) and (b, a) of a diagonal
// tile take the same products in the same order, so C is exactly symmetric.
// FP64 Z: FP64 fused multiply-adds.  FP32 Z: each product is split exactly
// into p + e (p = fl(xy), e = fma(x, y, -p)) and summed with Knuth's TwoSum
// into an FP32 (sum, correction) pair -- the compensated dot product of
// Ogita, Rump and Oishi (2005) -- which is as accurate as FP64 accumulation
// while running on the FP32 pipes; the pair is added in FP64 at the end.
// ---------------------------------------------------------------------------
constexpr int GR_T = 32, GR_K = 32;

template <typename T> struct GramAcc;
template <> struct GramAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct GramAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x, float y) {
        const float p = __fmul_rn(x, y);
        const float e = __fmaf_rn(x, y, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fadd_rn(t, -s);
        const float err = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ Z, int64_t n, int s,
                                              int64_t rows_per_chunk, double* __restrict__ part) {
    __shared__ T As[GR_K][GR_T + 1];
    __shared__ T Bs[GR_K][GR_T + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // blockIdx.x enumerates the lower-triangle tiles (ta >= tb)
    int ta = 0, rem = (int)blockIdx.x;
    while (rem > ta) {
        rem -= ta + 1;
        ++ta;
    }
    const int tb = rem;
    const int a0 = ta * GR_T, b0 = tb * GR_T;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    int64_t r1 = r0 + rows_per_chunk;
    if (r1 > n) r1 = n;
    GramAcc<T> acc[2][2];
    for (int64_t k0 = r0; k0 < r1; k0 += GR_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int col = e >> 5, kk = e & 31;
            const int64_t r = k0 + kk;
            const int ca = a0 + col, cb = b0 + col;
            As[kk][col] = (ca < s && r < r1) ? Z[(int64_t)ca * n + r] : (T)0;
            Bs[kk][col] = (cb < s && r < r1) ? Z[(int64_t)cb * n + r] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GR_K; ++kk) {
            const T x0 = As[kk][ty * 2], x1 = As[kk][ty * 2 + 1];
            const T y0 = Bs[kk][tx * 2], y1 = Bs[kk][tx * 2 + 1];
            acc[0][0].add(x0, y0);
            acc[0][1].add(x0, y1);
            acc[1][0].add(x1, y0);
            acc[1][1].add(x1, y1);
        }
        __syncthreads();
    }
    double* out = part + (int64_t)blockIdx.y * s * s;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int a = a0 + ty * 2 + i, b = b0 + tx * 2 + j;
            if (a < s && b < s) {
                const double v = acc[i][j].value();
                out[(int64_t)a * s + b] = v;
                if (ta != tb) out[(int64_t)b * s + a] = v;
            }
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
    const int64_t nt = (s + GR_T - 1) / GR_T;
    const int64_t tiles = nt * (nt + 1) / 2;
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
    const unsigned nt = (unsigned)((s + GR_T - 1) / GR_T);
    dim3 grid(nt * (nt + 1) / 2, (unsigned)chunks);
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

// ---------------------------------------------------------------------------
// The same reduction on a thread-block cluster of C CTAs, the matrix held in
// distributed shared memory: row r lives in CTA r % C (local row r / C).  Per
// column k every CTA
//   1. sends its entries of x = A[k+1:, k] and its part of ||x||^2 to all CTAs;
//   2. forms v locally, computes p = A_sub v for its own rows and sends p and
//      its part of v^T p to all CTAs;
//   3. updates its own rows with w = p - (v^T p) v.
// Gathered vectors and partial sums are double-buffered by column parity, so
// the two cluster barriers of a column separate every write from the reads it
// could overwrite.  Partial sums are added in CTA order, so every CTA takes the
// same branch and the same scalars.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ uint32_t proj_smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void proj_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
__device__ __forceinline__ uint32_t proj_cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t proj_cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Store v at the address of *local_ptr in the shared memory of CTA `rank`.
__device__ __forceinline__ void st_peer_f64(const double* local_ptr, uint32_t rank, double v) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(proj_smem_u32(local_ptr)), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}
}  // namespace

constexpr int kClusterMax = 16;
constexpr int kEigWarps = kEigThreads / 32;

__global__ void __launch_bounds__(kEigThreads) k_tridiag_cluster(const double* __restrict__ A, int N,
                                                                 double* __restrict__ d_out,
                                                                 double* __restrict__ e_out) {
    extern __shared__ double Wl[];
    __shared__ double xb[2][kEigMaxN], pb[2][kEigMaxN], vb[kEigMaxN], wb[kEigMaxN];
    __shared__ double part[2][2][kClusterMax];
    __shared__ double wsum[2][kEigWarps];
    __shared__ double scal[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)proj_cluster_rank(), C = (int)proj_cluster_size();
    const int rows_local = (N - rank + C - 1) / C;
    // local row lr belongs to warp lr % kEigWarps in every phase, so a warp
    // only ever reads the rows it wrote itself
    for (int lr = warp; lr < rows_local; lr += kEigWarps) {
        const int r = rank + lr * C;
        for (int j = lane; j < N; j += 32) Wl[(int64_t)lr * N + j] = A[(int64_t)r * N + j];
    }
    proj_cluster_sync();
    for (int k = 0; k + 2 < N; ++k) {
        const int b = k & 1, m = N - k - 1, o = k + 1;
        // 1. gather x = A[o:, k] and ||x[1:]||^2
        double tpart = 0.0;
        for (int lr = warp; lr < rows_local; lr += kEigWarps) {
            const int r = rank + lr * C;
            if (r < o) continue;
            const double x = Wl[(int64_t)lr * N + k];
            if (r > o) tpart += x * x;
            if (lane < C) st_peer_f64(&xb[b][r - o], (uint32_t)lane, x);
        }
        if (lane == 0) wsum[0][warp] = tpart;
        __syncthreads();
        if (warp == 0) {
            double t = lane < kEigWarps ? wsum[0][lane] : 0.0;
            t = warp_sum(t);
            if (lane < C) st_peer_f64(&part[b][0][rank], (uint32_t)lane, t);
        }
        proj_cluster_sync();
        // the scalars of the column, once per CTA (FP64 instructions are
        // expensive on this part: one thread computes, the block reads)
        if (tid == 0) {
            double tail = 0.0;
            for (int c = 0; c < C; ++c) tail += part[b][0][c];
            const double x0 = xb[b][0];
            if (k % C == rank) d_out[k] = Wl[(int64_t)(k / C) * N + k];
            double alpha = x0, v0 = 0.0, scale = 0.0;
            if (tail != 0.0) {
                const double xx = tail + x0 * x0;
                alpha = x0 >= 0.0 ? -sqrt(xx) : sqrt(xx);
                v0 = x0 - alpha;
                scale = 1.0 / sqrt(tail + v0 * v0);
            }
            if (rank == 0) e_out[k] = alpha;
            scal[0] = tail;
            scal[1] = v0 * scale;
            scal[2] = scale;
        }
        __syncthreads();
        if (scal[0] == 0.0) continue;  // column already reduced: same branch in every CTA
        // v once per column (every CTA keeps the whole vector)
        {
            const double scale = scal[2], v0s = scal[1];
            for (int j = tid; j < m; j += blockDim.x) vb[j] = j ? xb[b][j] * scale : v0s;
        }
        __syncthreads();
        // 2. p = A_sub v on own rows, v^T p
        double kpart = 0.0;
        for (int lr = warp; lr < rows_local; lr += kEigWarps) {
            const int r = rank + lr * C;
            if (r < o) continue;
            const double* row = Wl + (int64_t)lr * N + o;
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc = fma(row[j], vb[j], acc);
            acc = warp_sum(acc);
            if (lane < C) st_peer_f64(&pb[b][r - o], (uint32_t)lane, acc);
            kpart += vb[r - o] * acc;
        }
        if (lane == 0) wsum[1][warp] = kpart;
        __syncthreads();
        if (warp == 0) {
            double t = lane < kEigWarps ? wsum[1][lane] : 0.0;
            t = warp_sum(t);
            if (lane < C) st_peer_f64(&part[b][1][rank], (uint32_t)lane, t);
        }
        proj_cluster_sync();
        if (tid == 0) {
            double K = 0.0;
            for (int c = 0; c < C; ++c) K += part[b][1][c];
            scal[3] = -K;
        }
        __syncthreads();
        // w = p - K v, stored scaled by -2 so the update is two fused multiply-adds
        {
            const double mK = scal[3];
            for (int j = tid; j < m; j += blockDim.x) wb[j] = -2.0 * fma(mK, vb[j], pb[b][j]);
        }
        __syncthreads();
        // 3. own rows -= 2 (v w^T + w v^T)
        for (int lr = warp; lr < rows_local; lr += kEigWarps) {
            const int r = rank + lr * C;
            if (r < o) continue;
            double* row = Wl + (int64_t)lr * N + o;
            const int i = r - o;
            const double vr = vb[i], wr2 = wb[i];
            for (int j = lane; j < m; j += 32) row[j] = fma(vr, wb[j], fma(wr2, vb[j], row[j]));
        }
        __syncwarp();  // next column's x is read by all lanes of the owning warp
    }
    __syncthreads();
    if (tid == 0) {
        if (N >= 2) {
            if ((N - 2) % C == rank) d_out[N - 2] = Wl[(int64_t)((N - 2) / C) * N + (N - 2)];
            if ((N - 1) % C == rank) e_out[N - 2] = Wl[(int64_t)((N - 1) / C) * N + (N - 2)];
        }
        if ((N - 1) % C == rank) {
            d_out[N - 1] = Wl[(int64_t)((N - 1) / C) * N + (N - 1)];
            e_out[N - 1] = 0.0;
        }
    }
    proj_cluster_sync();
}

// Number of eigenvalues of the tridiagonal (d, e) below x: sign changes of
// the leading principal minors p_i = det(T_i - x I), p_0 = 1,
//   p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2}
// (Sturm's theorem), without divisions: FP64 division is many times the cost
// of a fused multiply-add on this part.  The pair (p_{i-1}, p_i) is rescaled by
// a power of two (exact) whenever |p_i| leaves [2^-400, 2^400]; a minor that
// comes out exactly zero is replaced by -2^-60 p_{i-1}, i.e. a tiny negative
// pivot, the usual convention of the pivot form of the count.
// e2 holds the squared off-diagonal entries.
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int N, double x) {
    int c = 0;
    double pm2 = 0.0, pm1 = 1.0;
    for (int i = 0; i < N; ++i) {
        double p = (d[i] - x) * pm1;
        if (i > 0) p = fma(-e2[i - 1], pm2, p);
        long long bits = __double_as_longlong(p);
        if ((bits << 1) == 0) {  // exact zero
            p = -pm1 * 0x1.0p-60;
            bits = __double_as_longlong(p);
        }
        c += (int)(((unsigned long long)bits >> 63) ^ ((unsigned long long)__double_as_longlong(pm1) >> 63));
        const int ex = (int)((bits >> 52) & 0x7FF) - 1023;
        if (ex > 400 || ex < -400) {
            const double sc = __longlong_as_double((long long)(1023 - ex) << 52);  // 2^-ex
            p *= sc;
            pm1 *= sc;
        }
        pm2 = pm1;
        pm1 = p;
    }
    return c;
}

// The same count in FP32 (rescaling outside [2^-60, 2^60]): cheap, and
// exact away from the eigenvalues; used only to narrow the bracket before the
// FP64 rounds, which re-check it.
__device__ __forceinline__ int sturm_count_f32(const float* d, const float* e2, int N, float x) {
    int c = 0;
    float pm2 = 0.f, pm1 = 1.f;
    for (int i = 0; i < N; ++i) {
        float p = (d[i] - x) * pm1;
        if (i > 0) p = fmaf(-e2[i - 1], pm2, p);
        int bits = __float_as_int(p);
        if ((bits << 1) == 0) {
            p = -pm1 * 0x1.0p-30f;
            bits = __float_as_int(p);
        }
        c += (int)(((unsigned)bits >> 31) ^ ((unsigned)__float_as_int(pm1) >> 31));
        const int ex = ((bits >> 23) & 0xFF) - 127;
        if (ex > 60 || ex < -60) {
            const float sc = __int_as_float((127 - ex) << 23);  // 2^-ex
            p *= sc;
            pm1 *= sc;
        }
        pm2 = pm1;
        pm1 = p;
    }
    return c;
}

// Multisection: each group of kMsLanes lanes owns one eigenvalue (ascending
// rank j >= j0) and splits its bracket [a, b] (count(a) <= j < count(b)) at kMsLanes interior points
// per round, keeping the sub-interval where the count passes j.  It stops
// when the bracket is within 16 ulps of the spectrum's scale and stores the
// midpoint at evals[N-1-j] (descending order).
constexpr int kMsLanes = 32;

__global__ void __launch_bounds__(32) k_bisect_multi(const double* __restrict__ d_in,
                                                     const double* __restrict__ e_in, int N,
                                                     int j0, double* __restrict__ evals) {
    __shared__ double d[kEigMaxN], e[kEigMaxN], e2[kEigMaxN];
    __shared__ float df[kEigMaxN], e2f[kEigMaxN];
    const int lane = threadIdx.x;
    for (int i = lane; i < N; i += 32) {
        d[i] = d_in[i];
        e[i] = e_in[i];
        e2[i] = e_in[i] * e_in[i];
        df[i] = (float)d[i];
        e2f[i] = (float)e2[i];
    }
    __syncwarp();
    double lo = 1e308, hi = -1e308, emax2 = 0.0;
    for (int i = lane; i < N; i += 32) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < N ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < N) emax2 = fmax(emax2, e[i] * e[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
    }
    const double pivmin = 0x1.0p-1022 * fmax(1.0, emax2);
    const double scale = fmax(fabs(lo), fabs(hi));
    const double pad = 2.2204460492503131e-16 * scale + pivmin;
    const double tol = 16.0 * 2.2204460492503131e-16 * scale + 2.0 * pivmin;
    const int g = lane / kMsLanes, l = lane % kMsLanes;
    const int j = j0 + blockIdx.x * (32 / kMsLanes) + g;
    const bool live = j < N;
    const unsigned gmask =
        kMsLanes == 32 ? 0xFFFFFFFFu : (((1u << (kMsLanes & 31)) - 1u) << (g * kMsLanes));
    double a = lo - pad, b = hi + pad;
    // FP32 rounds down to ~64 FP32 ulps of the scale, then an FP64 check of the
    // bracket (count(a) <= j < count(b)); a bracket that fails it restarts
    // from the Gershgorin bounds
    const double tol32 = 64.0 * 1.1920928955078125e-07 * scale;
    for (int round = 0; round < 16; ++round) {
        if (!(b - a > tol32)) break;
        const double x = a + (b - a) * ((double)(l + 1) / (double)(kMsLanes + 1));
        const bool up = live ? sturm_count_f32(df, e2f, N, (float)x) >= j + 1 : true;
        const unsigned bal = (__ballot_sync(gmask, up) & gmask) >> (g * kMsLanes);
        const int L = bal ? __ffs(bal) - 1 : kMsLanes;
        const double xl = __shfl_sync(gmask, x, g * kMsLanes + (L > 0 ? L - 1 : 0));
        const double xr = __shfl_sync(gmask, x, g * kMsLanes + (L < kMsLanes ? L : kMsLanes - 1));
        const double na = L > 0 ? xl : a;
        const double nb = L < kMsLanes ? xr : b;
        if (!(na >= a && nb <= b && na < nb)) break;
        a = na;
        b = nb;
    }
    {
        const double xe = l == 0 ? a : b;
        const int ce = (live && l < 2) ? sturm_count(d, e2, N, xe) : 0;
        const int ca = __shfl_sync(gmask, ce, g * kMsLanes);
        const int cb = __shfl_sync(gmask, ce, g * kMsLanes + 1);
        if (live && !(ca <= j && cb >= j + 1)) {
            a = lo - pad;
            b = hi + pad;
        }
    }
    for (int round = 0; round < 64; ++round) {
        if (!(b - a > tol)) break;  // uniform within the lane group
        const double x = a + (b - a) * ((double)(l + 1) / (double)(kMsLanes + 1));
        const bool up = live ? sturm_count(d, e2, N, x) >= j + 1 : true;
        const unsigned bal = (__ballot_sync(gmask, up) & gmask) >> (g * kMsLanes);
        const int L = bal ? __ffs(bal) - 1 : kMsLanes;  // first point with count > j
        const double xl = __shfl_sync(gmask, x, g * kMsLanes + (L > 0 ? L - 1 : 0));
        const double xr = __shfl_sync(gmask, x, g * kMsLanes + (L < kMsLanes ? L : kMsLanes - 1));
        const double na = L > 0 ? xl : a;
        const double nb = L < kMsLanes ? xr : b;
        if (!(na >= a && nb <= b && na < nb)) break;  // no progress at this scale
        a = na;
        b = nb;
    }
    if (live && l == 0) evals[N - 1 - j] = 0.5 * (a + b);
}

// CTAs of the reduction: about 16 rows each (FP64 work spread over SMs), at
// most 16 CTAs and 160 KB of rows per CTA.
int eig_cluster_size(int N) {
    int C = 1;
    while (C < kClusterMax && C * 16 < N) C *= 2;
    static int force = -1;
    if (force < 0) {
        force = 0;
        if (const char* e = getenv("VNE_EIG_CLUSTER")) force = atoi(e);
    }
    if (force == 1 || force == 2 || force == 4 || force == 8 || force == 16) C = force;
    if ((int64_t)((N + C - 1) / C) * N * 8 > 160 * 1024) return -1;
    return C;
}

cudaError_t launch_sym_eigvals(const double* A, int N, int top, double* Wg, double* d, double* e,
                               double* evals, cudaStream_t st) {
    if (N < 1 || N > kEigMaxN || top < 1 || top > N) return cudaErrorInvalidValue;
    int C = eig_cluster_size(N);
    cudaError_t r = cudaSuccess;
    bool done = false;
    if (C >= 1) {
        const size_t smem = (size_t)((N + C - 1) / C) * N * sizeof(double);
        r = cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (r == cudaSuccess && C > 8)
            r = cudaFuncSetAttribute(k_tridiag_cluster,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kEigThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (r == cudaSuccess)
            r = cudaOccupancyMaxActiveClusters(&clusters, k_tridiag_cluster, &cfg);
        if (r == cudaSuccess && clusters == 0 && C > 8) {
            // 16-CTA clusters not schedulable here: 8 CTAs if their rows fit
            const int C8 = 8;
            const size_t smem8 = (size_t)((N + C8 - 1) / C8) * N * sizeof(double);
            if (smem8 <= 160 * 1024) {
                attr[0].val.clusterDim.x = C8;
                cfg.gridDim = dim3(C8);
                cfg.dynamicSmemBytes = smem8;
                r = cudaFuncSetAttribute(k_tridiag_cluster,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8);
                if (r == cudaSuccess)
                    r = cudaOccupancyMaxActiveClusters(&clusters, k_tridiag_cluster, &cfg);
            }
        }
        if (r == cudaSuccess && clusters > 0) {
            r = cudaLaunchKernelEx(&cfg, k_tridiag_cluster, A, N, d, e);
            if (r != cudaSuccess) return r;
            done = true;
        } else {
            cudaGetLastError();  // fall back to the one-CTA kernel
        }
    }
    if (!done) {
        const size_t smem = (size_t)N * N * sizeof(double);
        const int use_smem = smem <= 160 * 1024;
        if (use_smem) {
            r = cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (r != cudaSuccess) return r;
        }
        k_tridiag<<<1, kEigThreads, use_smem ? smem : 0, st>>>(A, N, Wg, use_smem, d, e);
        r = cudaGetLastError();
        if (r != cudaSuccess) return r;
    }
    // only the `top` largest eigenvalues: ascending ranks N-top .. N-1
    k_bisect_multi<<<(top + 32 / kMsLanes - 1) / (32 / kMsLanes), 32, 0, st>>>(d, e, N, N - top,
                                                                             evals);
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

// ---------------------------------------------------------------------------
// Block Krylov extension (the batched workload's projection path; not in the
// paper): V_0 = R Pi, V_j = R Q_{j-1}; each V_j is orthogonalised against the
// earlier blocks (two passes of block Gram-Schmidt) and made orthonormal through
// the eigendecomposition of its Gram matrix, dropping the directions below
// drop * (largest Gram eigenvalue of the first block); the Ritz values of R on
// K = [Q_0 .. Q_{q-1}] are the eigenvalues of T = K^T (R K).
// ---------------------------------------------------------------------------

// C (ra x rb, FP64) = A^T B for A stored [ra][n], B [rb][n]: all 32 x 32 tiles,
// rows split into `chunks` slices summed in order by k_sum_chunks.
template <typename T>
__global__ void __launch_bounds__(256) k_xgram(const T* __restrict__ A, int ra,
                                               const T* __restrict__ B, int rb, int64_t n,
                                               int64_t rows_per_chunk, double* __restrict__ part) {
    __shared__ T As[GR_K][GR_T + 1];
    __shared__ T Bs[GR_K][GR_T + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.y * GR_T, b0 = blockIdx.x * GR_T;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk;
    int64_t r1 = r0 + rows_per_chunk;
    if (r1 > n) r1 = n;
    GramAcc<T> acc[2][2];
    for (int64_t k0 = r0; k0 < r1; k0 += GR_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int col = e >> 5, kk = e & 31;
            const int64_t r = k0 + kk;
            const int ca = a0 + col, cb = b0 + col;
            As[kk][col] = (ca < ra && r < r1) ? A[(int64_t)ca * n + r] : (T)0;
            Bs[kk][col] = (cb < rb && r < r1) ? B[(int64_t)cb * n + r] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GR_K; ++kk) {
            const T x0 = As[kk][ty * 2], x1 = As[kk][ty * 2 + 1];
            const T y0 = Bs[kk][tx * 2], y1 = Bs[kk][tx * 2 + 1];
            acc[0][0].add(x0, y0);
            acc[0][1].add(x0, y1);
            acc[1][0].add(x1, y0);
            acc[1][1].add(x1, y1);
        }
        __syncthreads();
    }
    double* out = part + (int64_t)blockIdx.z * ra * rb;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int a = a0 + ty * 2 + i, b = b0 + tx * 2 + j;
            if (a < ra && b < rb) out[(int64_t)a * rb + b] = acc[i][j].value();
        }
}

template <typename T>
cudaError_t launch_xgram(const T* A, int ra, const T* B, int rb, int64_t n, int chunks,
                         double* part, double* C, cudaStream_t st) {
    int64_t rows = (n + chunks - 1) / chunks;
    rows = (rows + GR_K - 1) / GR_K * GR_K;
    dim3 grid((unsigned)((rb + GR_T - 1) / GR_T), (unsigned)((ra + GR_T - 1) / GR_T),
              (unsigned)chunks);
    k_xgram<T><<<grid, 256, 0, st>>>(A, ra, B, rb, n, rows, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t len = (int64_t)ra * rb;
    k_sum_chunks<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, chunks, len, C);
    return cudaGetLastError();
}

// Out[c][i] = In[c][i] (or 0) + scale * sum_r A[r][i] M[r][c] for i < n, c < rc;
// A stored [ra][n], M (ra x rc) FP64 row-major.  One thread per row, 16
// columns per block; M's 16 columns staged in shared memory in T.
constexpr int TS_COLS = 16;

template <typename T>
__global__ void __launch_bounds__(128) k_ts_mm(const T* __restrict__ A, int ra,
                                               const double* __restrict__ M, int rc, double scale,
                                               const T* In, T* Out, int64_t n) {
    extern __shared__ unsigned char ts_raw[];
    T* Ms = reinterpret_cast<T*>(ts_raw);  // [ra][TS_COLS]
    const int c0 = blockIdx.y * TS_COLS;
    for (int e = threadIdx.x; e < ra * TS_COLS; e += blockDim.x) {
        const int r = e / TS_COLS, c = c0 + e % TS_COLS;
        Ms[e] = c < rc ? (T)(scale * M[(int64_t)r * rc + c]) : (T)0;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[TS_COLS];
#pragma unroll
    for (int c = 0; c < TS_COLS; ++c) acc[c] = (T)0;
    for (int r = 0; r < ra; ++r) {
        const T a = A[(int64_t)r * n + i];
#pragma unroll
        for (int c = 0; c < TS_COLS; ++c) acc[c] = Math<T>::fma(a, Ms[r * TS_COLS + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < TS_COLS; ++c) {
        const int col = c0 + c;
        if (col < rc) {
            const int64_t idx = (int64_t)col * n + i;
            Out[idx] = (In ? In[idx] : (T)0) + acc[c];
        }
    }
}

template <typename T>
cudaError_t launch_ts_mm(const T* A, int ra, const double* M, int rc, double scale, const T* In,
                         T* Out, int64_t n, cudaStream_t st) {
    const size_t smem = (size_t)ra * TS_COLS * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t r = cudaFuncSetAttribute(k_ts_mm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r != cudaSuccess) return r;
    }
    dim3 grid((unsigned)((n + 127) / 128), (unsigned)((rc + TS_COLS - 1) / TS_COLS));
    k_ts_mm<T><<<grid, 128, smem, st>>>(A, ra, M, rc, scale, In, Out, n);
    return cudaGetLastError();
}

// Cyclic Jacobi (parallel ordering: every round rotates b/2 disjoint pairs of
// the circle schedule) on the b x b symmetric G, b <= 64, in arithmetic T:
// eigenvalues lam and eigenvectors U (columns), both written in FP64.
constexpr int kJacobiMaxB = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_jacobi(const double* __restrict__ G, int b,
                                                double* __restrict__ lam, double* __restrict__ Uout) {
    // A and U with row stride b + 1: the column updates (lanes along a column)
    // then fall in distinct shared-memory banks
    extern __shared__ unsigned char jac_raw[];
    const int ld = b + 1;
    T* A = reinterpret_cast<T*>(jac_raw);
    T* U = A + b * ld;
    __shared__ T rc[kJacobiMaxB / 2 + 1][2];
    __shared__ int rp[kJacobiMaxB / 2 + 1][2];
    __shared__ double red[8];
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = warp; i < b; i += nwarps)
        for (int j = lane; j < b; j += 32) {
            A[i * ld + j] = (T)G[i * b + j];
            U[i * ld + j] = (i == j) ? (T)1 : (T)0;
        }
    const int B = b + (b & 1), np = B / 2;
    // stop when the off-diagonal mass is negligible, or (after 4 sweeps) when
    // a sweep no longer halves it: convergence is quadratic until the rounding
    // level of T, where the mass stays put
    const double eps2 = sizeof(T) == 8 ? 1e-30 : 1e-16;
    double off_prev = 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = warp; i < b; i += nwarps)
            for (int j = lane; j < b; j += 32) {
                const double v = (double)A[i * ld + j];
                if (i > j) off += v * v;
                else if (i == j) dia += v * v;
            }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if (lane == 0) red[warp] = off;
        __syncthreads();
        if (tid == 0) {
            double o = 0.0;
            for (int w = 0; w < nwarps; ++w) o += red[w];
            red[0] = o;
        }
        __syncthreads();
        const double offt = red[0];
        __syncthreads();
        if (lane == 0) red[warp] = dia;
        __syncthreads();
        if (tid == 0) {
            double d = 0.0;
            for (int w = 0; w < nwarps; ++w) d += red[w];
            stop = !(offt > eps2 * d) || (sweep >= 4 && offt > 0.5 * off_prev);
        }
        off_prev = offt;
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < B - 1; ++r) {
            if (tid < np) {
                int p, q;
                if (tid == 0) {
                    p = r;
                    q = B - 1;
                } else {
                    p = (r + tid) % (B - 1);
                    q = (r - tid + (B - 1)) % (B - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                T c = (T)1, sn = (T)0;
                if (q < b) {
                    const T apq = A[p * ld + q];
                    if (apq != (T)0) {
                        const T th = (A[q * ld + q] - A[p * ld + p]) / ((T)2 * apq);
                        const T t = th != (T)0 ? (th > (T)0 ? (T)1 : (T)-1) /
                                                     (fabs(th) + sqrt(th * th + (T)1))
                                               : (T)1;
                        c = (T)1 / sqrt(t * t + (T)1);
                        sn = t * c;
                    }
                }
                rc[tid][0] = c;
                rc[tid][1] = sn;
                rp[tid][0] = p;
                rp[tid][1] = q;
            }
            __syncthreads();
            for (int k = warp; k < np; k += nwarps) {  // rows: A <- J^T A
                const int p = rp[k][0], q = rp[k][1];
                if (q >= b) continue;
                const T c = rc[k][0], sn = rc[k][1];
                for (int j = lane; j < b; j += 32) {
                    const T ap = A[p * ld + j], aq = A[q * ld + j];
                    A[p * ld + j] = c * ap - sn * aq;
                    A[q * ld + j] = sn * ap + c * aq;
                }
            }
            __syncthreads();
            for (int k = warp; k < np; k += nwarps) {  // columns: A <- A J, U <- U J
                const int p = rp[k][0], q = rp[k][1];
                if (q >= b) continue;
                const T c = rc[k][0], sn = rc[k][1];
                for (int i = lane; i < b; i += 32) {
                    const T ap = A[i * ld + p], aq = A[i * ld + q];
                    A[i * ld + p] = c * ap - sn * aq;
                    A[i * ld + q] = sn * ap + c * aq;
                    const T up = U[i * ld + p], uq = U[i * ld + q];
                    U[i * ld + p] = c * up - sn * uq;
                    U[i * ld + q] = sn * up + c * uq;
                }
            }
            __syncthreads();
        }
    }
    for (int i = warp; i < b; i += nwarps)
        for (int j = lane; j < b; j += 32) Uout[i * b + j] = (double)U[i * ld + j];
    for (int i = tid; i < b; i += blockDim.x) lam[i] = (double)A[i * ld + i];
}

template <typename T>
cudaError_t launch_jacobi(const double* G, int b, double* lam, double* U, cudaStream_t st) {
    if (b < 1 || b > kJacobiMaxB) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * b * (b + 1) * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t r = cudaFuncSetAttribute(k_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r != cudaSuccess) return r;
    }
    k_jacobi<T><<<1, 256, smem, st>>>(G, b, lam, U);
    return cudaGetLastError();
}

// M[:, c] = U[:, c] / sqrt(lam_c) where lam_c > drop * lam_ref, else 0.  The
// first block (first != 0) sets lam_ref = max lam.
__global__ void k_basis_coeffs(const double* __restrict__ lam, const double* __restrict__ U, int b,
                               double* __restrict__ lam_ref, int first, double drop,
                               double* __restrict__ M) {
    __shared__ double ref;
    if (threadIdx.x == 0) {
        if (first) {
            double mx = lam[0];
            for (int i = 1; i < b; ++i) mx = fmax(mx, lam[i]);
            *lam_ref = mx;
        }
        ref = *lam_ref;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int c = e % b;
        const double l = lam[c];
        M[e] = (l > drop * ref && l > 0.0) ? U[e] / sqrt(l) : 0.0;
    }
}

__global__ void k_symmetrize(double* T, int N) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
        const int i = e / N, j = e % N;
        if (i < j) {
            const double v = 0.5 * (T[(int64_t)i * N + j] + T[(int64_t)j * N + i]);
            T[(int64_t)i * N + j] = v;
            T[(int64_t)j * N + i] = v;
        }
    }
}

// out[0] = sum_{i<k, theta_i>0} theta_i ln(1/theta_i) + tail, out[1+i] = theta_i;
// tail: the rest of the unit trace, 1 - sum theta_i, spread evenly over n - k.
__global__ void k_krylov_combine(const double* __restrict__ ev, int k, int64_t n,
                                 double* __restrict__ out) {
    __shared__ double red[32];
    double h = 0.0, sum = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double t = ev[i];
        out[1 + i] = t;
        sum += t;
        if (t > 0.0) h -= t * log(t);
    }
    const double H = block_sum(h, red);
    __syncthreads();
    const double S = block_sum(sum, red);
    if (threadIdx.x == 0) {
        double tot = H;
        const double rest = 1.0 - S;
        if (rest > 0.0 && n > k) tot += rest * log((double)(n - k) / rest);
        out[0] = tot;
    }
}

cudaError_t launch_basis_coeffs(const double* lam, const double* U, int b, double* lam_ref,
                                int first, double drop, double* M, cudaStream_t st) {
    k_basis_coeffs<<<1, 256, 0, st>>>(lam, U, b, lam_ref, first, drop, M);
    return cudaGetLastError();
}
cudaError_t launch_symmetrize(double* T, int N, cudaStream_t st) {
    k_symmetrize<<<(N * N + 255) / 256, 256, 0, st>>>(T, N);
    return cudaGetLastError();
}
cudaError_t launch_krylov_combine(const double* ev, int k, int64_t n, double* out,
                                  cudaStream_t st) {
    k_krylov_combine<<<1, 256, 0, st>>>(ev, k, n, out);
    return cudaGetLastError();
}

template cudaError_t launch_xgram<double>(const double*, int, const double*, int, int64_t, int,
                                          double*, double*, cudaStream_t);
template cudaError_t launch_xgram<float>(const float*, int, const float*, int, int64_t, int,
                                         double*, double*, cudaStream_t);
template cudaError_t launch_ts_mm<double>(const double*, int, const double*, int, double,
                                          const double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_ts_mm<float>(const float*, int, const double*, int, double,
                                         const float*, float*, int64_t, cudaStream_t);
template cudaError_t launch_jacobi<double>(const double*, int, double*, double*, cudaStream_t);
template cudaError_t launch_jacobi<float>(const double*, int, double*, double*, cudaStream_t);

template cudaError_t launch_sketch<double>(double*, int64_t, int, int, uint64_t, int, cudaStream_t);
template cudaError_t launch_sketch<float>(float*, int64_t, int, int, uint64_t, int, cudaStream_t);
template cudaError_t launch_split_sum<double>(const double*, int, int64_t, double*, int, cudaStream_t);
template cudaError_t launch_split_sum<float>(const float*, int, int64_t, float*, int, cudaStream_t);
template cudaError_t launch_gram<double>(const double*, int64_t, int, int, double*, double*,
                                         cudaStream_t);
template cudaError_t launch_gram<float>(const float*, int64_t, int, int, double*, double*,
                                        cudaStream_t);

}  // namespace vne
