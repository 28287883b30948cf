// Probe generation and the initial recurrence blocks Y_0 = G.
//
// The trace estimator of Lemma thm:trace (used by Algorithms 1a and 1b)
// draws s i.i.d. probe vectors g_j.  They come from the SplitMix64 counter
// generator of vne_common.cuh, entry (i, j) at counter j*n + i.
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

__global__ void k_probe_block_f64(double* out, int64_t n, int s, int kind, uint64_t seed) {
    const int64_t total = n * (int64_t)s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = probe_value(kind, seed, (uint64_t)e);
}

cudaError_t launch_probe_block_f64(double* out, int64_t n, int s, int kind, uint64_t seed,
                                   cudaStream_t st) {
    const int64_t total = n * (int64_t)s;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_probe_block_f64<<<blocks, 256, 0, st>>>(out, n, s, kind, seed);
    return cudaGetLastError();
}

// Dense layout: one thread per row of a row tile (blockDim.x = rows_per_tile),
// blockIdx.y = probe j.  Writes G[j][i], Y0[c][i] for every column c = j + r*s
// (r < S/s), the bf16 pieces of Y0 if requested (piece k = bf16 of the
// residual of pieces 0..k-1, exact in FP32), and the slot-0 partials
// sum_i g_j[i]^2 of each row tile.  kind PROBE_GIVEN takes g_j[i] from the
// caller's block Gin[i*s + j] (probe_n x s, row-major) instead of the stream.
struct Pieces {
    __nv_bfloat16* p[kMaxPieces];
};
template <typename T>
__global__ void k_dense_init(T* G, T* Y0, Pieces Ysh, int pieces, int64_t ldk, int64_t n, int S,
                             int s, int kind, uint64_t seed, Partials P, int64_t probe_n,
                             int64_t j0, const T* __restrict__ Gin) {
    __shared__ double sh[32];
    const int j = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double g = 0.0;
    if (i < n) {
        if (i < probe_n) {
            const uint64_t e = (uint64_t)(j0 + j) * (uint64_t)probe_n + (uint64_t)i;
            if (kind == PROBE_GIVEN) g = (double)Gin[i * s + j];
            else if (sizeof(T) == 4 && kind == 1) g = (double)gaussian_f32(seed, e);
            else g = probe_value(kind, seed, e);
        }
        const T gt = (T)g;
        G[(int64_t)j * n + i] = gt;
        for (int c = j; c < S; c += s) {
            Y0[(int64_t)c * n + i] = gt;
            float r = (float)gt;
            for (int k = 0; k < pieces; ++k) {
                const __nv_bfloat16 b = __float2bfloat16_rn(r);
                Ysh.p[k][(int64_t)c * ldk + i] = b;
                r -= __bfloat162float(b);
            }
        }
    }
    // g^2 summed in the path's precision within each warp, FP64 across warps
    const T gw = warp_sum((T)(g * g));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)gw;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        for (int c = j; c < S; c += s) P.slot(0)[(size_t)blockIdx.x * S + c] = tot;
    }
}

template <typename T>
cudaError_t launch_dense_init(T* G, T* Y0, __nv_bfloat16* const* Ysh, int pieces, int64_t ldk,
                              int64_t n, int S, int s, int kind, uint64_t seed, Partials P,
                              int rows_per_tile, cudaStream_t st, int64_t probe_n, int64_t j0,
                              const T* Gin) {
    if (pieces < 0 || pieces > kMaxPieces || (pieces > 0 && !Ysh)) return cudaErrorInvalidValue;
    if (kind == PROBE_GIVEN && !Gin) return cudaErrorInvalidValue;
    Pieces ps{};
    for (int k = 0; k < pieces; ++k) {
        if (!Ysh[k]) return cudaErrorInvalidValue;
        ps.p[k] = Ysh[k];
    }
    dim3 grid((unsigned)((n + rows_per_tile - 1) / rows_per_tile), (unsigned)s);
    k_dense_init<T><<<grid, rows_per_tile, 0, st>>>(G, Y0, ps, pieces, ldk, n, S, s, kind, seed, P,
                                                    probe_n, j0, Gin);
    return cudaGetLastError();
}
template cudaError_t launch_dense_init<double>(double*, double*, __nv_bfloat16* const*, int,
                                               int64_t, int64_t, int, int, int, uint64_t, Partials,
                                               int, cudaStream_t, int64_t, int64_t, const double*);
template cudaError_t launch_dense_init<float>(float*, float*, __nv_bfloat16* const*, int,
                                              int64_t, int64_t, int, int, int, uint64_t, Partials,
                                              int, cudaStream_t, int64_t, int64_t, const float*);

// Banded layout: a block of 8 warps owns a tile of rows_per_tile rows; each
// warp walks rows w, w+8, ... of the tile and lane l covers probes l, l+32, ...
// kind PROBE_GIVEN reads the caller's block Gin[i*s + j].
template <typename T>
__global__ void k_dia_init(T* G, uint64_t* bits, int W, T* Y0, int64_t n, int S, int s, int kind,
                           uint64_t seed, Partials P, int rows_per_tile, int64_t j0,
                           const T* __restrict__ Gin) {
    __shared__ double sh[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nchunk = (s + 31) >> 5;  // <= 8
    T acc[8];  // per-lane sums of g^2 in the path's precision
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = (T)0;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_tile;
    int64_t r1 = r0 + rows_per_tile;
    if (r1 > n) r1 = n;
    for (int64_t i = r0 + w; i < r1; i += 8) {
        uint32_t words[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            words[q] = 0u;
            if (q < nchunk) {
                const int j = q * 32 + lane;
                // Rademacher signs straight from the hash bit (no FP64 on this path)
                T gt = (T)0;
                if (j < s) {
                    const uint64_t e = (uint64_t)(j0 + j) * (uint64_t)n + (uint64_t)i;
                    if (kind == PROBE_GIVEN) gt = Gin[i * s + j];
                    else if (kind == 0) gt = (splitmix_out(seed, e) >> 63) ? (T)-1 : (T)1;
                    else gt = (T)gaussian(seed, e);
                }
                words[q] = __ballot_sync(0xffffffffu, gt < (T)0);
                if (j < s) {
                    if (G) G[i * s + j] = gt;
                    if (Y0)  // the Rademacher path reads Y_0 from the bits instead
                        for (int c = j; c < S; c += s) Y0[i * S + c] = gt;
                    acc[q] += gt * gt;
                }
            }
        }
        if (bits && lane < W) {
            const uint64_t lo = words[2 * lane], hi = words[2 * lane + 1];
            bits[i * W + lane] = lo | (hi << 32);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (q < nchunk) sh[w][q * 32 + lane] = (double)acc[q];
    __syncthreads();
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        double t = 0.0;
        for (int ww = 0; ww < 8; ++ww) t += sh[ww][j];
        for (int c = j; c < S; c += s) P.slot(0)[(size_t)blockIdx.x * S + c] = t;
    }
}

template <typename T>
cudaError_t launch_dia_init(T* G, uint64_t* bits, int W, T* Y0, int64_t n, int S, int s, int kind,
                            uint64_t seed, Partials P, int rows_per_tile, cudaStream_t st,
                            int64_t j0, const T* Gin) {
    if (s > 256 || W > 4) return cudaErrorInvalidValue;
    if (kind == PROBE_GIVEN && (!Gin || bits)) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((n + rows_per_tile - 1) / rows_per_tile);
    k_dia_init<T><<<grid, 256, 0, st>>>(G, bits, W, Y0, n, S, s, kind, seed, P, rows_per_tile, j0,
                                        Gin);
    return cudaGetLastError();
}
template cudaError_t launch_dia_init<double>(double*, uint64_t*, int, double*, int64_t, int, int,
                                             int, uint64_t, Partials, int, cudaStream_t, int64_t,
                                             const double*);
template cudaError_t launch_dia_init<float>(float*, uint64_t*, int, float*, int64_t, int, int, int,
                                            uint64_t, Partials, int, cudaStream_t, int64_t,
                                            const float*);

}  // namespace vne
