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
// loop); the y rows of the next block are loaded while the current block
// computes.
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

// One chunk of CH rows for this lane's column.
//   CHECK = false: interior fast path, every row the windows touch lies in
//                  [0, n), so no per-row bounds checks are needed.
//   MODE 1       : step 1, the input block Y_0 = G (Rademacher) is read from
//                  the staged sign bits instead of memory;
//   MODE 2       : step 2, the same for Y_{t-2} = Y_0 (Chebyshev columns);
//   SC > 0       : the row stride S of Y is the compile-time constant SC, so
//                  every window address is a fixed offset from a chunk base.
template <typename T, int HB, bool CHECK, int MODE, int SC>
__device__ __forceinline__ T dia_chunk(const T* __restrict__ sb, const uint64_t* __restrict__ sbits,
                                       int Wd, int64_t r0, int64_t n, const T* __restrict__ Yprev,
                                       const T* __restrict__ Yprev2, T* __restrict__ Ynew,
                                       const T* __restrict__ G, int S_rt, int s, int cc, int c, int j,
                                       bool active, bool is_cheb, int cheb_kind, bool rad, T a,
                                       T invu) {
    using C = DiaCfg<T, HB>;
    constexpr int W = C::W, NB = C::NB, CH = C::CH, BP = C::BP;
    const int S = SC > 0 ? SC : S_rt;
    const bool need_y2 = is_cheb && cheb_kind == EPI_CHEB;
    const int64_t pb = r0 - W;
    const int64_t rlim = r0 + CH + W;  // rows beyond this are never needed
    // chunk-relative bases: row k of the window (k = p - pb) sits at k * S
    const T* ybase = Yprev + pb * S + cc;
    const T* y2base = Yprev2 + r0 * S + cc;
    T* obase = Ynew + r0 * S + c;
    const int jw = j >> 6, jb = j & 63;
    // sbits covers rows pb .. pb + CH + 2W - 1
    auto ld_y = [&](int k) -> T {  // k = p - pb
        if (MODE == 1) return ((sbits[k * Wd + jw] >> jb) & 1ull) ? (T)-1 : (T)1;
        if (CHECK) {
            const int64_t p = pb + k;
            return (active && p >= 0 && p < n && p < rlim) ? __ldg(ybase + (int64_t)k * S) : (T)0;
        }
        return __ldg(ybase + k * S);
    };
    auto ld_y2 = [&](int k) -> T {  // k = p - r0
        if (!need_y2) return (T)0;
        if (MODE == 2) return ((sbits[(k + W) * Wd + jw] >> jb) & 1ull) ? (T)-1 : (T)1;
        if (CHECK) return (r0 + k < n) ? __ldg(y2base + (int64_t)k * S) : (T)0;
        return __ldg(y2base + k * S);
    };
    T y[W], pf[W], z[W], zn[W], q2c[W], q2n[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        y[k] = ld_y(k);
        pf[k] = ld_y(W + k);
        z[k] = (T)0;
        zn[k] = (T)0;
        q2n[k] = ld_y2(k);
        q2c[k] = (T)0;
    }
    T macc = (T)0;
    for (int b = 0; b <= NB; ++b) {
        const bool out_block = b >= 1;
        if (out_block) {
#pragma unroll
            for (int k = 0; k < W; ++k) q2c[k] = q2n[k];
            if (b < NB) {
#pragma unroll
                for (int k = 0; k < W; ++k) q2n[k] = ld_y2(b * W + k);
            }
        }
        T bacc = (T)0;
#pragma unroll
        for (int uu = 0; uu < W; ++uu) {
            T v[BP];
            load_row<BP>(v, sb + (b * W + uu) * BP);
            // gather in two interleaved chains (shorter dependency chains)
            T za = z[uu], zb = (T)0;
#pragma unroll
            for (int d = 0; d < W; ++d) {
                const T yv = (uu + d < W) ? y[uu + d] : pf[uu + d - W];
                if (d & 1) zb = Math<T>::fma(v[d], yv, zb);
                else za = Math<T>::fma(v[d], yv, za);
            }
            const T zz = za + zb;
#pragma unroll
            for (int d = 1; d < W; ++d) {
                if (uu + d < W) z[uu + d] = Math<T>::fma(v[d], y[uu], z[uu + d]);
                else zn[uu + d - W] = Math<T>::fma(v[d], y[uu], zn[uu + d - W]);
            }
            const int kr = (b - 1) * W + uu;  // row p - r0 of this output
            if (out_block && active && (!CHECK || r0 + kr < n)) {
                T g;
                if (rad) g = ((sbits[(kr + W) * Wd + jw] >> jb) & 1ull) ? (T)-1 : (T)1;
                else g = __ldg(G + (r0 + kr) * s + j);
                T yo;
                if (is_cheb) {
                    if (cheb_kind == EPI_CHEB1) yo = a * zz - g;
                    else yo = (T)2 * (a * zz - y[uu]) - q2c[uu];
                    bacc = Math<T>::fma(g, yo, bacc);
                } else {
                    yo = y[uu] - zz * invu;
                    bacc = Math<T>::fma(g, zz, bacc);
                }
                obase[(int64_t)kr * S] = yo;
            }
        }
        macc += bacc;
        // rotate the windows by one block
#pragma unroll
        for (int k = 0; k < W; ++k) {
            y[k] = pf[k];
            // the block after the last one is never read: no load (the staged
            // sign bits and the interior bound end exactly at row CH + 2W)
            pf[k] = (b < NB) ? ld_y((b + 2) * W + k) : (T)0;
            z[k] = zn[k];
            zn[k] = (T)0;
        }
    }
    return macc;
}

template <typename T, int HB, int SC>
__global__ void __launch_bounds__(256, 2) k_dia_step(
    const T* __restrict__ vals, int64_t ld, int D, int64_t n, const T* __restrict__ Yprev,
    const T* __restrict__ Yprev2, T* __restrict__ Ynew, const T* __restrict__ G,
    const uint64_t* __restrict__ bits, int Wd, int S, int s, StepCols cols, int col_lo,
    int col_hi, const double* __restrict__ sc, Partials P, int t, int64_t nchunks) {
    using C = DiaCfg<T, HB>;
    constexpr int W = C::W, CH = C::CH, BP = C::BP, NR = C::NR;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sb = reinterpret_cast<T*>(smraw);                          // [NR][BP]
    uint64_t* sbits = reinterpret_cast<uint64_t*>(sb + NR * BP);  // [CH + 2W][Wd]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = col_lo + warp * 32 + lane;
    const bool active = c < col_hi;
    const int j = active ? c % s : 0;
    const bool is_cheb = active && c >= cols.cheb_c0 && c < cols.cheb_c0 + cols.ncheb;
    const bool is_tay = active && !is_cheb && c >= cols.tay_c0 && c < cols.tay_c0 + cols.ntay;
    const bool rad = (bits != nullptr);
    // Y_0 = G is never read from memory on the Rademacher path: steps 1 and 2
    // take it from the staged sign bits
    const int mode = rad ? (t == 1 ? 1 : (t == 2 ? 2 : 0)) : 0;
    const T uT = (T)sc[SC_U];  // the path's own precision (FP64 only on the FP64 path)
    const T a = (T)2 / uT, invu = (T)1 / uT;
    const int cc = active ? c : col_lo;  // safe column for address arithmetic

    double mom_total = 0.0;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t r0 = ch * CH;
        __syncthreads();
        // stage the band: sb[row][d] = R[p, p+d], p = r0 - W + row
        for (int row = threadIdx.x; row < NR; row += blockDim.x) {
            const int64_t p = r0 - W + row;
            T v[W];
#pragma unroll
            for (int d = 0; d < W; ++d)
                v[d] = (d < D && p >= 0 && p < n - d) ? __ldg(vals + (int64_t)d * ld + p) : (T)0;
#pragma unroll
            for (int d = 0; d < W; ++d) sb[row * BP + d] = v[d];
        }
        if (rad)  // sign bits of rows r0 - W .. r0 + CH + W - 1 (zero outside [0, n))
            for (int row = threadIdx.x; row < CH + 2 * W; row += blockDim.x) {
                const int64_t p = r0 - W + row;
                for (int w = 0; w < Wd; ++w)
                    sbits[row * Wd + w] = (p >= 0 && p < n) ? __ldg(bits + p * Wd + w) : 0ull;
            }
        __syncthreads();
        const bool interior = (r0 - W >= 0) && (r0 + CH + 2 * W <= n);
        T macc;
#define VNE_DIA_CHUNK(CHK, MD)                                                                    \
    dia_chunk<T, HB, CHK, MD, SC>(sb, sbits, Wd, r0, n, Yprev, Yprev2, Ynew, G, S, s, cc, c, j,   \
                                   active, is_cheb, cols.cheb_kind, rad, a, invu)
        if (mode == 1) macc = interior ? VNE_DIA_CHUNK(false, 1) : VNE_DIA_CHUNK(true, 1);
        else if (mode == 2) macc = interior ? VNE_DIA_CHUNK(false, 2) : VNE_DIA_CHUNK(true, 2);
        else macc = interior ? VNE_DIA_CHUNK(false, 0) : VNE_DIA_CHUNK(true, 0);
#undef VNE_DIA_CHUNK
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
    const size_t smem =
        (size_t)C::NR * C::BP * sizeof(T) + (size_t)(C::CH + 2 * C::W) * (bits ? Wd : 0) * 8;
    auto kern = (sizeof(T) == 4 && S == 64) ? k_dia_step<T, HB, 64> : k_dia_step<T, HB, 0>;
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
    // the sign bits take ceil(s / 64) words per row, s <= ncols
    const size_t smem = (size_t)C::NR * C::BP * sizeof(T) +
                        (size_t)(C::CH + 2 * C::W) * ((ncols + 63) / 64) * 8;
    auto kern = (sizeof(T) == 4 && ncols == 64) ? k_dia_step<T, HB, 64> : k_dia_step<T, HB, 0>;
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
int dia_step_grid(int is_double, int D, int64_t n, int ncols, int s, int sm_count,
                  int band_aligned) {
    if (dia_tma_ok(is_double, D, n, ncols, s, band_aligned)) return dia_tma_grid(D, n, ncols, sm_count);
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
                            int nblocks, cudaStream_t st, int band_aligned) {
    if constexpr (sizeof(T) == 4) {
        if (dia_tma_ok(0, D, n, S, s, band_aligned))
            return launch_dia_step_tma(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, S, s, cols,
                                       sc, P, t, nblocks, st);
    }
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
                                            int, cudaStream_t, int);
template cudaError_t launch_dia_step<double>(const double*, int64_t, int, int64_t, const double*,
                                             const double*, double*, const double*,
                                             const uint64_t*, int, int, int, StepCols,
                                             const double*, Partials, int, int, cudaStream_t, int);

}  // namespace vne
