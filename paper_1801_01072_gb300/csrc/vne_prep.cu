// Operand preparation: storage-type conversion of R, the bf16 hi/lo split
// of the tensor-core path, the unit-trace check of Section 1.1, and u.
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

// dtype 0 FP64, 1 FP32, 2 complex FP64, 3 complex FP32 (interleaved): the
// real part of entry idx.
__device__ __forceinline__ double load_entry(const void* src, int dtype, int64_t idx) {
    switch (dtype) {
        case 0: return ((const double*)src)[idx];
        case 1: return (double)((const float*)src)[idx];
        case 2: return ((const double*)src)[2 * idx];
        default: return (double)((const float*)src)[2 * idx];
    }
}

// Real symmetric embedding of a Hermitian R = B + iC (Section 4): the 2n x 2n
// matrix [[B, -C], [C, B]] (row-major, ld 2n).  For real g,
// [g; 0]^T f([[B, -C], [C, B]]) [g; 0] = g^T Re[f(R)] g for every polynomial f.
template <typename TO>
__global__ void k_hermitian_embed(const void* src, int cdtype, int64_t n, int64_t ld, TO* dst) {
    const int64_t total = n * n;
    const int64_t n2 = 2 * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, k = e - i * n;
        const int64_t idx = i * ld + k;
        double b, c;
        if (cdtype == 2) {
            b = ((const double*)src)[2 * idx];
            c = ((const double*)src)[2 * idx + 1];
        } else {
            b = (double)((const float*)src)[2 * idx];
            c = (double)((const float*)src)[2 * idx + 1];
        }
        dst[i * n2 + k] = (TO)b;
        dst[i * n2 + n + k] = (TO)(-c);
        dst[(n + i) * n2 + k] = (TO)c;
        dst[(n + i) * n2 + n + k] = (TO)b;
    }
}

template <typename TO>
__global__ void k_dense_convert(const void* src, int dtype, int64_t n, int64_t ld, TO* dst) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, k = e - i * n;
        dst[e] = (TO)load_entry(src, dtype, i * ld + k);
    }
}

static int grid_for(int64_t total) {
    int64_t b = (total + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_hermitian_embed(const void* src, int cdtype, int64_t n, int64_t ld, void* dst,
                                   int dst_dtype, cudaStream_t st) {
    if (dst_dtype == 0)
        k_hermitian_embed<double><<<grid_for(n * n), 256, 0, st>>>(src, cdtype, n, ld, (double*)dst);
    else
        k_hermitian_embed<float><<<grid_for(n * n), 256, 0, st>>>(src, cdtype, n, ld, (float*)dst);
    return cudaGetLastError();
}

cudaError_t launch_dense_convert_f64(const void* src, int src_dtype, int64_t n, int64_t ld,
                                     double* dst, cudaStream_t st) {
    k_dense_convert<double><<<grid_for(n * n), 256, 0, st>>>(src, src_dtype, n, ld, dst);
    return cudaGetLastError();
}
cudaError_t launch_dense_convert_f32(const void* src, int src_dtype, int64_t n, int64_t ld,
                                     float* dst, cudaStream_t st) {
    k_dense_convert<float><<<grid_for(n * n), 256, 0, st>>>(src, src_dtype, n, ld, dst);
    return cudaGetLastError();
}

// Piece 0 = bf16(R), piece k = bf16(R - pieces 0..k-1), zero padding outside
// the n x n block.  One or two pieces split R rounded to FP32 (the residual of
// a float and its bf16 rounding is exact in FP32); three pieces take the
// residuals in FP64, since they resolve R beyond FP32's 24 bits.  Each thread
// converts 8 consecutive columns.
struct BfPieces {
    __nv_bfloat16* p[kMaxPieces];
};
template <int PIECES>
__global__ void k_dense_convert_bf16(const void* src, int dtype, int64_t nrows, int64_t ncols,
                                     int64_t ld, BfPieces out, int64_t rows_pad, int64_t ldk) {
    const int64_t groups = ldk / 8;
    const int64_t total = rows_pad * groups;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / groups, k0 = (e - i * groups) * 8;
        __align__(16) __nv_bfloat16 b8[PIECES][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t k = k0 + q;
            const bool in = i < nrows && k < ncols;
            if (PIECES < 3) {
                const float v = in ? (float)load_entry(src, dtype, i * ld + k) : 0.f;
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                b8[0][q] = h;
                if (PIECES == 2) b8[PIECES - 1][q] = __float2bfloat16_rn(v - __bfloat162float(h));
            } else {
                double r = in ? load_entry(src, dtype, i * ld + k) : 0.0;
#pragma unroll
                for (int c = 0; c < PIECES; ++c) {
                    // bf16 of the FP64 residual through FP32 (the FP32 rounding
                    // moves it by far less than the bf16 spacing)
                    const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
                    b8[c][q] = b;
                    r -= (double)__bfloat162float(b);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < PIECES; ++c) *(uint4*)(out.p[c] + i * ldk + k0) = *(const uint4*)b8[c];
    }
}

cudaError_t launch_convert_bf16_rect(const void* src, int src_dtype, int64_t rows, int64_t cols,
                                     int64_t ld, __nv_bfloat16* const* out, int pieces,
                                     int64_t rows_pad, int64_t ldk, cudaStream_t st) {
    if (ldk % 8 != 0 || pieces < 1 || pieces > kMaxPieces || !out || rows > rows_pad || cols > ldk)
        return cudaErrorInvalidValue;
    BfPieces ps{};
    for (int c = 0; c < pieces; ++c) {
        if (!out[c]) return cudaErrorInvalidValue;
        ps.p[c] = out[c];
    }
    const unsigned g = grid_for(rows_pad * (ldk / 8));
    if (pieces == 1)
        k_dense_convert_bf16<1><<<g, 256, 0, st>>>(src, src_dtype, rows, cols, ld, ps, rows_pad, ldk);
    else if (pieces == 2)
        k_dense_convert_bf16<2><<<g, 256, 0, st>>>(src, src_dtype, rows, cols, ld, ps, rows_pad, ldk);
    else
        k_dense_convert_bf16<3><<<g, 256, 0, st>>>(src, src_dtype, rows, cols, ld, ps, rows_pad, ldk);
    return cudaGetLastError();
}

cudaError_t launch_dense_convert_bf16(const void* src, int src_dtype, int64_t n, int64_t ld,
                                      __nv_bfloat16* const* out, int pieces, int64_t rows_pad,
                                      int64_t ldk, cudaStream_t st) {
    return launch_convert_bf16_rect(src, src_dtype, n, n, ld, out, pieces, rows_pad, ldk, st);
}

// A full symmetric copy of R from its upper triangle (layout VNE_DENSE_UPPER),
// in the storage type T.  Output tile (I, J) of 32 x 32: strictly upper tiles
// are copied (skipped when dst == src: they are already there), strictly
// lower ones are the transposes of the upper tiles (J, I), staged through
// shared memory so that both the reads and the writes are row-contiguous, and
// diagonal tiles take every entry (i, k) from (min(i, k), max(i, k)).  In place,
// no tile is both read by one block and written by another: lower tiles read
// only strictly upper tiles, which nobody writes, and a diagonal tile is read
// and rewritten by its own block alone.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_symmetrize(const T* src, int64_t lds, T* dst,
                                                          int64_t ldd, int64_t n, int in_place) {
    __shared__ T sm[32][33];
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (I < J && in_place) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (I < J) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t r = I * 32 + ty + 8 * k, c = J * 32 + tx;
            if (r < n && c < n) dst[r * ldd + c] = src[r * lds + c];
        }
        return;
    }
    // the source tile: (J, I) for a lower tile, (I, I) for a diagonal one
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t r = J * 32 + ty + 8 * k, c = I * 32 + tx;
        if (r < n && c < n) sm[ty + 8 * k][tx] = src[r * lds + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int y = ty + 8 * k;
        const int64_t r = I * 32 + y, c = J * 32 + tx;
        if (r >= n || c >= n) continue;
        // lower tile: dst(r, c) = src(c, r) = sm[tx][y]; diagonal: upper
        // entries (tx >= y) from sm[y][tx], lower ones mirrored
        dst[r * ldd + c] = (I > J || tx < y) ? sm[tx][y] : sm[y][tx];
    }
}

cudaError_t launch_dense_symmetrize(const void* src, int64_t lds, void* dst, int64_t ldd,
                                    int64_t n, int dtype, cudaStream_t st) {
    if (n < 1 || lds < n || ldd < n || (dtype != 0 && dtype != 1)) return cudaErrorInvalidValue;
    const int64_t tiles = (n + 31) / 32;
    if (tiles > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)tiles, (unsigned)tiles), block(32, 8);
    const int in_place = src == dst ? 1 : 0;
    if (in_place && lds != ldd) return cudaErrorInvalidValue;
    if (dtype == 0)
        k_dense_symmetrize<double><<<grid, block, 0, st>>>((const double*)src, lds, (double*)dst,
                                                           ldd, n, in_place);
    else
        k_dense_symmetrize<float><<<grid, block, 0, st>>>((const float*)src, lds, (float*)dst, ldd,
                                                          n, in_place);
    return cudaGetLastError();
}

__global__ void k_dia_convert(const void* src, int sdt, int64_t n, int64_t ld, int D, void* dst,
                              int ddt) {
    const int64_t total = (int64_t)D * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = e / n, i = e - d * n;
        const double v = (i < n - d) ? load_entry(src, sdt, d * ld + i) : 0.0;
        if (ddt == 0) ((double*)dst)[e] = v;
        else ((float*)dst)[e] = (float)v;
    }
}

cudaError_t launch_dia_convert(const void* src, int src_dtype, int64_t n, int64_t ld, int D,
                               void* dst, int dst_dtype, cudaStream_t st) {
    k_dia_convert<<<grid_for((int64_t)D * n), 256, 0, st>>>(src, src_dtype, n, ld, D, dst,
                                                            dst_dtype);
    return cudaGetLastError();
}

// tr R in FP64: per-block partials, the last block to finish sums them in
// block order (deterministic) and resets the counter.
__global__ void k_trace(const void* R, int layout, int dtype, int64_t n, int64_t ld,
                        double* partial, unsigned int* counter, double* sc) {
    __shared__ double sh[32];
    __shared__ bool last;
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v += load_entry(R, dtype, layout == 0 ? i * ld + i : i);
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = t;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t2 = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t2 += ((volatile double*)partial)[b];
    const double tot = block_sum(t2, sh);
    if (threadIdx.x == 0) {
        sc[SC_TRACE] = tot;
        *counter = 0u;
    }
}

cudaError_t launch_trace(const void* R, int layout, int dtype, int64_t n, int64_t ld,
                         double* partial, unsigned int* counter, double* sc, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 256) blocks = 256;
    k_trace<<<blocks, 256, 0, st>>>(R, layout, dtype, n, ld, partial, counter, sc);
    return cudaGetLastError();
}

__global__ void k_set_u(double* sc, double u) {
    sc[SC_U] = u;
    sc[SC_LAM] = 0.0;
    if (!(u > 0.0 && u <= 1.0)) {
        unsigned long long* f = (unsigned long long*)&sc[SC_FLAGS];
        *f |= FLAG_BAD_INTERVAL;
    }
}

cudaError_t launch_set_u(double* sc, double u, cudaStream_t st) {
    k_set_u<<<1, 1, 0, st>>>(sc, u);
    return cudaGetLastError();
}

}  // namespace vne
