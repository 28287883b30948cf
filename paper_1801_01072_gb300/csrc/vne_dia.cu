// Banded (symmetric DIA) recurrence: one step Z = R Y_{t-1} fused with the
// Chebyshev three-term update (Section 3) or the Taylor update (Section 2)
// and the per-probe moment partials.  The work is HBM-bound: per step it
// streams Y_{t-1}, Y_{t-2} (Chebyshev), the band, and writes Y_t.
//
// Layout: Y is row-major [n][S] (the S probe columns of a row contiguous),
// so a warp's 32 lanes (32 consecutive columns) read and write 128-byte
// rows.  The band is stored vals[d*ld + i] = R[i, i+d], d = 0..D-1.
//
// Work split: a CTA owns chunks of CH consecutive rows (persistent grid).
// It stages the chunk's band (rows r0-W .. r0+CH-1, W = HB+1) transposed in
// shared memory, [row][d], so that a row's W band values are one broadcast
// vector load.  Each warp then sweeps the rows of the chunk for its 32
// columns with register windows:
//   gather  z_p     += sum_{d=0..HB} R[p,p+d] y_{p+d}
//   scatter z_{p+d} += R[p,p+d] y_p           (d >= 1, the lower triangle)
// so every band value and every y value is loaded once per chunk.  Rows are
// handled in blocks of W with static register indices (the unrolled row
// loop); y rows are prefetched two blocks ahead.
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static constexpr int kPad = 4;
};
template <> struct Vec4<double> {
    static constexpr int kPad = 2;
};

template <typename T, int HB> struct DiaCfg {
    static constexpr int W = HB + 1;
    static constexpr int NB = (256 + W - 1) / W;  // row blocks per chunk
    static constexpr int CH = NB * W;             // rows per chunk
    static constexpr int BP = (W + Vec4<T>::kPad - 1) / Vec4<T>::kPad * Vec4<T>::kPad;
    static constexpr int NR = CH + W;             // staged band rows
};

template <int N, typename T>
__device__ __forceinline__ void load_row(T (&v)[N], const T* p) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 q = *reinterpret_cast<const float4*>(p + 4 * k);
            v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
        }
#pragma unroll
        for (int k = (N / 4) * 4; k < N; ++k) v[k] = p[k];
    } else {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const double2 q = *reinterpret_cast<const double2*>(p + 2 * k);
            v[2 * k] = q.x; v[2 * k + 1] = q.y;
        }
#pragma unroll
        for (int k = (N / 2) * 2; k < N; ++k) v[k] = p[k];
    }
}

template <typename T, int HB>
__global__ void __launch_bounds__(256) k_dia_step(
    const T* __restrict__ vals, int64_t ld, int D, int64_t n, const T* __restrict__ Yprev,
    const T* __restrict__ Yprev2, T* __restrict__ Ynew, const T* __restrict__ G,
    const uint64_t* __restrict__ bits, int Wd, int S, int s, StepCols cols, int col_lo,
    int col_hi, const double* __restrict__ sc, Partials P, int t, int64_t nchunks) {
    using C = DiaCfg<T, HB>;
    constexpr int W = C::W, NB = C::NB, CH = C::CH, BP = C::BP, NR = C::NR;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sb = reinterpret_cast<T*>(smraw);                       // [NR][BP]
    uint64_t* sbits = reinterpret_cast<uint64_t*>(sb + NR * BP);  // [CH][Wd]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = col_lo + warp * 32 + lane;
    const bool active = c < col_hi;
    const int j = active ? c % s : 0;
    const bool is_cheb = active && c >= cols.cheb_c0 && c < cols.cheb_c0 + cols.ncheb;
    const bool is_tay = active && !is_cheb && c >= cols.tay_c0 && c < cols.tay_c0 + cols.ntay;
    const bool need_y2 = is_cheb && cols.cheb_kind == EPI_CHEB;
    const bool rad = (bits != nullptr);
    const double u = sc[SC_U];
    const T a = (T)(2.0 / u), invu = (T)(1.0 / u);
    const int cc = active ? c : col_lo;  // safe column for address arithmetic

    double mom_total = 0.0;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t r0 = ch * CH;
        const int64_t rlim = r0 + CH + W;  // rows beyond this are never needed
        __syncthreads();
        // stage the band: sb[row][d] = R[p, p+d], p = r0 - W + row
        for (int e = threadIdx.x; e < NR * W; e += blockDim.x) {
            const int d = e / NR, row = e - d * NR;
            const int64_t p = r0 - W + row;
            T v = (T)0;
            if (d < D && p >= 0 && p < n - d) v = vals[(int64_t)d * ld + p];
            sb[row * BP + d] = v;
        }
        if (rad)
            for (int e = threadIdx.x; e < CH * Wd; e += blockDim.x) {
                const int64_t p = r0 + e / Wd;
                sbits[e] = p < n ? bits[p * Wd + (e % Wd)] : 0ull;
            }
        __syncthreads();

        T y[W], pf[W], pf2[W], z[W], zn[W], q2c[W], q2n[W];
        const int64_t pb = r0 - W;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int64_t p0 = pb + k, p1 = pb + W + k, p2 = pb + 2 * W + k;
            y[k] = (active && p0 >= 0 && p0 < n) ? Yprev[p0 * S + cc] : (T)0;
            pf[k] = (active && p1 >= 0 && p1 < n) ? Yprev[p1 * S + cc] : (T)0;
            pf2[k] = (active && p2 >= 0 && p2 < n && p2 < rlim) ? Yprev[p2 * S + cc] : (T)0;
            z[k] = (T)0;
            zn[k] = (T)0;
            q2n[k] = (need_y2 && r0 + k < n) ? Yprev2[(r0 + k) * S + cc] : (T)0;
            q2c[k] = (T)0;
        }
        T macc = (T)0;  // moment of this chunk (per-block sums folded in)
        for (int b = 0; b <= NB; ++b) {
            const int64_t pbb = pb + (int64_t)b * W;
            const bool out_block = b >= 1;
            if (out_block) {
#pragma unroll
                for (int k = 0; k < W; ++k) q2c[k] = q2n[k];
                if (b < NB) {
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        const int64_t p = pbb + W + k;
                        q2n[k] = (need_y2 && p < n) ? Yprev2[p * S + cc] : (T)0;
                    }
                }
            }
            T bacc = (T)0;
#pragma unroll
            for (int uu = 0; uu < W; ++uu) {
                T v[BP];
                load_row<BP>(v, sb + (b * W + uu) * BP);
                T zz = z[uu];
#pragma unroll
                for (int d = 0; d < W; ++d)
                    zz = Math<T>::fma(v[d], (uu + d < W) ? y[uu + d] : pf[uu + d - W], zz);
#pragma unroll
                for (int d = 1; d < W; ++d) {
                    if (uu + d < W) z[uu + d] = Math<T>::fma(v[d], y[uu], z[uu + d]);
                    else zn[uu + d - W] = Math<T>::fma(v[d], y[uu], zn[uu + d - W]);
                }
                const int64_t p = pbb + uu;
                if (out_block && active && p < n) {
                    T g;
                    if (rad) {
                        const uint64_t wv = sbits[(p - r0) * Wd + (j >> 6)];
                        g = ((wv >> (j & 63)) & 1ull) ? (T)-1 : (T)1;
                    } else {
                        g = G[p * s + j];
                    }
                    T yo;
                    if (is_cheb) {
                        if (cols.cheb_kind == EPI_CHEB1) yo = a * zz - g;
                        else yo = (T)2 * (a * zz - y[uu]) - q2c[uu];
                        bacc = Math<T>::fma(g, yo, bacc);
                    } else {
                        yo = y[uu] - zz * invu;
                        bacc = Math<T>::fma(g, zz, bacc);
                    }
                    Ynew[p * S + c] = yo;
                }
            }
            macc += bacc;
            // rotate the windows by one block
#pragma unroll
            for (int k = 0; k < W; ++k) {
                y[k] = pf[k];
                pf[k] = pf2[k];
                const int64_t p = pbb + 3 * W + k;
                pf2[k] = (active && p < n && p < rlim) ? Yprev[p * S + cc] : (T)0;
                z[k] = zn[k];
                zn[k] = (T)0;
            }
        }
        mom_total += (double)macc;
    }
    if (active && (is_cheb || is_tay)) P.slot(t)[(size_t)blockIdx.x * S + c] = mom_total;
}

int dia_supported_halfbw(int D) {
    const int hb = D - 1;
    if (hb <= 1) return 1;
    if (hb <= 2) return 2;
    if (hb <= 4) return 4;
    if (hb <= 8) return 8;
    if (hb <= 16) return 16;
    return -1;
}

template <typename T, int HB>
static cudaError_t launch_hb(const T* vals, int64_t ld, int D, int64_t n, const T* Yprev,
                             const T* Yprev2, T* Ynew, const T* G, const uint64_t* bits, int Wd,
                             int S, int s, StepCols cols, const double* sc, Partials P, int t,
                             int nblocks, cudaStream_t st) {
    using C = DiaCfg<T, HB>;
    int col_lo, col_hi;
    if (cols.ncheb > 0 && cols.ntay > 0) {
        col_lo = cols.cheb_c0 < cols.tay_c0 ? cols.cheb_c0 : cols.tay_c0;
        const int e1 = cols.cheb_c0 + cols.ncheb, e2 = cols.tay_c0 + cols.ntay;
        col_hi = e1 > e2 ? e1 : e2;
    } else if (cols.ncheb > 0) {
        col_lo = cols.cheb_c0;
        col_hi = cols.cheb_c0 + cols.ncheb;
    } else {
        col_lo = cols.tay_c0;
        col_hi = cols.tay_c0 + cols.ntay;
    }
    const int nw = (col_hi - col_lo + 31) / 32;
    if (nw > 8) return cudaErrorInvalidValue;
    const int64_t nchunks = (n + C::CH - 1) / C::CH;
    const size_t smem = (size_t)C::NR * C::BP * sizeof(T) + (size_t)C::CH * (bits ? Wd : 0) * 8;
    auto kern = k_dia_step<T, HB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int grid = nblocks;
    if (grid < 1) return cudaErrorInvalidValue;
    if ((int64_t)grid > nchunks) grid = (int)nchunks;
    kern<<<grid, nw * 32, smem, st>>>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols,
                                      col_lo, col_hi, sc, P, t, nchunks);
    return cudaGetLastError();
}

template <typename T, int HB>
static int grid_hb(int64_t n, int ncols, int sm_count) {
    using C = DiaCfg<T, HB>;
    const int nw = (ncols + 31) / 32;
    const size_t smem = (size_t)C::NR * C::BP * sizeof(T) + (size_t)C::CH * 4 * 8;
    auto kern = k_dia_step<T, HB>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nw * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t nchunks = (n + C::CH - 1) / C::CH;
    int64_t g = (int64_t)sm_count * per_sm;
    if (g > nchunks) g = nchunks;
    return (int)(g < 1 ? 1 : g);
}

// Persistent grid of the banded step (resident CTAs x SMs, capped by the
// number of row chunks); the caller sizes the moment partials with it.
int dia_step_grid(int is_double, int D, int64_t n, int ncols, int sm_count) {
    const int hb = dia_supported_halfbw(D);
    if (is_double) {
        switch (hb) {
            case 1: return grid_hb<double, 1>(n, ncols, sm_count);
            case 2: return grid_hb<double, 2>(n, ncols, sm_count);
            case 4: return grid_hb<double, 4>(n, ncols, sm_count);
            case 8: return grid_hb<double, 8>(n, ncols, sm_count);
            case 16: return grid_hb<double, 16>(n, ncols, sm_count);
        }
    } else {
        switch (hb) {
            case 1: return grid_hb<float, 1>(n, ncols, sm_count);
            case 2: return grid_hb<float, 2>(n, ncols, sm_count);
            case 4: return grid_hb<float, 4>(n, ncols, sm_count);
            case 8: return grid_hb<float, 8>(n, ncols, sm_count);
            case 16: return grid_hb<float, 16>(n, ncols, sm_count);
        }
    }
    return -1;
}

template <typename T>
cudaError_t launch_dia_step(const T* vals, int64_t ld, int D, int64_t n, const T* Yprev,
                            const T* Yprev2, T* Ynew, const T* G, const uint64_t* bits, int Wd,
                            int S, int s, StepCols cols, const double* sc, Partials P, int t,
                            int nblocks, cudaStream_t st) {
    switch (dia_supported_halfbw(D)) {
        case 1: return launch_hb<T, 1>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols, sc, P, t, nblocks, st);
        case 2: return launch_hb<T, 2>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols, sc, P, t, nblocks, st);
        case 4: return launch_hb<T, 4>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols, sc, P, t, nblocks, st);
        case 8: return launch_hb<T, 8>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols, sc, P, t, nblocks, st);
        case 16: return launch_hb<T, 16>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols, sc, P, t, nblocks, st);
        default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_dia_step<float>(const float*, int64_t, int, int64_t, const float*,
                                            const float*, float*, const float*, const uint64_t*,
                                            int, int, int, StepCols, const double*, Partials, int,
                                            int, cudaStream_t);
template cudaError_t launch_dia_step<double>(const double*, int64_t, int, int64_t, const double*,
                                             const double*, double*, const double*,
                                             const uint64_t*, int, int, int, StepCols,
                                             const double*, Partials, int, int, cudaStream_t);

}  // namespace vne
