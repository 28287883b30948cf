// Banded (symmetric DIA) recurrence step in FP32, fed by bulk copies: one
// step Z = R Y_{t-1} fused with the Chebyshev three-term update (Section 3)
// or the Taylor update (Section 2) and the per-probe moment partials, for
// row strides S of 32, 64 or 128 columns.  The FP64 path and other shapes use
// the register-window kernel of vne_dia.cu.
#include <algorithm>
#include <cstdlib>

#include "vne_common.cuh"
#include "vne_internal.h"
#include "vne_ptx.cuh"

namespace vne {

// ---------------------------------------------------------------------------
// FP32 step fed by bulk copies, for S = 32, 64 or 128 columns (the FP32
// workloads: s = 64 Chebyshev, s = 32 Chebyshev + Taylor, ...).
//
// A persistent CTA (384 threads, one per SM) walks a contiguous range of row
// chunks of CH rows (CH = 8 rows x the CTA's row blocks: 192 at S = 64).  For each chunk one thread issues 1-D bulk copies into
// a ring of NS shared-memory stages, NS-1 chunks ahead of the compute:
//   the Y_{t-1} rows r0-HBA .. r0+CH+HBA-1 (contiguous in the [n][S] layout),
//   the D stored diagonals at positions r0-HBA .. r0+CH-1 (vals[d][.]),
//   the probe sign bits of the Y_{t-1} rows (Rademacher probes).
// HBA = HB rounded up to 4, so every copy starts on a 16-byte boundary.
// Y_{t-2} (Chebyshev steps t >= 2) is read once per element: each thread
// loads its rows from global memory at the start of the chunk, and uses
// them in the epilogue.
// Chunks whose rows reach outside [0, n) are filled by the threads with
// bounds-checked loads instead (zeros outside), so no copy leaves a buffer.
//
// Thread (cg, rb) computes rows p0 = r0 + 8 rb .. p0 + 7 of the 4 columns
// 4 cg .. 4 cg + 3: z_p = sum_{d=-HB..HB} R[p, p+d] y_{p+d}.  For each d the
// 8 coefficients R[p0+i, p0+i+d] are two or three vector loads of one staged
// diagonal (R[p, p-e] = vals[e][p-e] for the lower triangle), and the y rows
// p0+d .. p0+d+7 are a register window that advances by one row per d: one
// 16-byte shared load feeds 32 FMAs, one coefficient feeds 4.  The FMAs are
// packed two columns at a time (fma.rn on each half, the rounding of fmaf),
// and the next offset's loads are issued ahead of the current FMAs.
// ---------------------------------------------------------------------------
template <int HB, int SC, int NT_, int RB_> struct DiaTma {
    static constexpr int W = HB + 1;                // stored diagonals
    static constexpr int HBA = (HB + 3) / 4 * 4;    // halo rows, 16-byte aligned copies
    static constexpr int RB = RB_;                  // rows per thread (4 or 8)
    static constexpr int NT = NT_;                  // threads per CTA
    static constexpr int CG = SC / 4;               // threads per row block
    static constexpr int NRB = NT / CG;             // row blocks per chunk
    static constexpr int CH = NRB * RB;             // rows per chunk
    static constexpr int YR = CH + 2 * HBA;         // staged Y_{t-1} rows
    static constexpr int BTP = CH + HBA;            // staged positions per diagonal
    static constexpr int WDMAX = (SC + 63) / 64;    // sign-bit words per row
    static constexpr uint32_t Y_OFF = 0;
    static constexpr uint32_t Y_BYTES = (uint32_t)YR * SC * 4;
    static constexpr uint32_t B_OFF = Y_OFF + Y_BYTES;
    static constexpr uint32_t B_BYTES = (uint32_t)W * BTP * 4;
    static constexpr uint32_t S_OFF = B_OFF + B_BYTES;
    static constexpr uint32_t S_BYTES = (uint32_t)YR * WDMAX * 8;
    static constexpr uint32_t STAGE = (S_OFF + S_BYTES + 127) / 128 * 128;
    static constexpr int NSF = (int)((232448u - 64u) / STAGE);  // stages that fit
    static constexpr int NS = NSF > 4 ? 4 : NSF;                 // ring stages
    static constexpr uint32_t BAR_OFF = NS * STAGE;
    static constexpr uint32_t SMEM = BAR_OFF + 64;  // + NS mbarriers and the abort flag
    static_assert(RB == 4 || RB == 8, "rows per thread");
    static_assert(NT % CG == 0 && NS >= 2, "shape");
    static_assert(Y_BYTES % 16 == 0 && B_BYTES % 16 == 0, "copy sizes");
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert((size_t)NRB * SC * 8 <= STAGE, "moment reduction fits one stage");
};

// Default shape of the kernel: 384 threads, 8 rows of 4 columns per thread
// (measured at n = 1e7, S = 64, 33 diagonals: 1629 us per step; 256 x 8
// 1747 us, 512 x 4 1755 us, 256 x 4 2165 us).
constexpr int kDiaNT = 384, kDiaRB = 8;

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// +-1 of the 4 probes j0 .. j0+3 (bit set = -1), j0 % 4 == 0
__device__ __forceinline__ float4 signs4(uint64_t word, int jb) {
    const uint32_t w = (uint32_t)(word >> jb);
    return make_float4((w & 1u) ? -1.f : 1.f, (w & 2u) ? -1.f : 1.f, (w & 4u) ? -1.f : 1.f,
                       (w & 8u) ? -1.f : 1.f);
}

// Coefficients R[p0+i, p0+i+d], i = 0..RB-1, of diagonal offset d (a
// compile-time value once the loop over d is unrolled) from the staged
// diagonals; o is the staged position of row p0 (a multiple of 4).
template <int RB, int BTP>
__device__ __forceinline__ void band_coeffs(const float* bt, int o, int d, float (&v)[RB]) {
    if (d >= 0) {  // R[p, p+d] = vals[d][p]
        const float* q = bt + d * BTP + o;
#pragma unroll
        for (int k = 0; k < RB / 4; ++k) {
            const float4 x = lds4(q + 4 * k);
            v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
        }
    } else {  // R[p, p-e] = vals[e][p-e]: positions o-e .. o-e+RB-1
        const int e = -d, up = (e + 3) & ~3, sh = up - e;
        const float* q = bt + e * BTP + o - up;
        float L[RB + 4];
#pragma unroll
        for (int k = 0; k < RB / 4; ++k) {
            const float4 x = lds4(q + 4 * k);
            L[4 * k] = x.x; L[4 * k + 1] = x.y; L[4 * k + 2] = x.z; L[4 * k + 3] = x.w;
        }
        if (sh > 0) {
            const float4 x = lds4(q + RB);
            L[RB] = x.x; L[RB + 1] = x.y; L[RB + 2] = x.z; L[RB + 3] = x.w;
        } else {
            L[RB] = L[RB + 1] = L[RB + 2] = L[RB + 3] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) v[i] = L[sh + i];
    }
}

template <int HB, int SC, bool Y0BITS, int NT_, int RB_>
__global__ void __launch_bounds__(NT_, 1) k_dia_step_tma(
    const float* __restrict__ vals, int64_t ld, int D, int64_t n, const float* __restrict__ Yprev,
    const float* __restrict__ Yprev2, float* __restrict__ Ynew, const float* __restrict__ G,
    const uint64_t* __restrict__ bits, int Wd, int s, StepCols cols, double* __restrict__ sc,
    Partials P, int t, int64_t nchunks) {
    using C = DiaTma<HB, SC, NT_, RB_>;
    constexpr int RB = C::RB, SC4 = SC / 4;
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int NS = C::NS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + C::BAR_OFF);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + NS);
    const int tid = threadIdx.x;
    const int cg = tid % C::CG, rb = tid / C::CG;
    const int c0 = 4 * cg;
    // the kind of the thread's 4 columns (one kind: s is a multiple of 4)
    int kind = EPI_NONE, j0 = 0;
    if (c0 >= cols.cheb_c0 && c0 < cols.cheb_c0 + cols.ncheb) {
        kind = cols.cheb_kind;
        j0 = c0 - cols.cheb_c0;
    } else if (c0 >= cols.tay_c0 && c0 < cols.tay_c0 + cols.ntay) {
        kind = EPI_TAYLOR;
        j0 = c0 - cols.tay_c0;
    }
    const bool rad = bits != nullptr;
    const bool y2bits = rad && t == 2;  // Y_{t-2} = Y_0 = G from the sign bits
    const int jw = j0 >> 6, jb = j0 & 63;
    const float uT = (float)sc[SC_U];
    const float a = 2.f / uT, invu = 1.f / uT;

    // contiguous chunk range of this CTA
    const int64_t per = nchunks / gridDim.x, rem = nchunks % gridDim.x;
    const int64_t cbeg = (int64_t)blockIdx.x * per + (blockIdx.x < rem ? blockIdx.x : rem);
    const int64_t nk = per + (blockIdx.x < rem ? 1 : 0);

    if (tid == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&bar[st], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // diagonals D .. HB are never copied: zero in every stage, once
    for (int st = 0; st < NS; ++st) {
        float* bt = reinterpret_cast<float*>(smraw + st * C::STAGE + C::B_OFF);
        for (int k = D * C::BTP + tid; k < C::W * C::BTP; k += C::NT) bt[k] = 0.f;
    }
    fence_proxy_async_smem();
    __syncthreads();

    auto interior = [&](int64_t ch) {
        const int64_t r0 = ch * C::CH;
        return r0 - C::HBA >= 0 && r0 + C::CH + C::HBA <= n;
    };
    auto issue = [&](int64_t ch, int st) {
        unsigned char* sb = smraw + st * C::STAGE;
        const int64_t r0 = ch * C::CH, pb = r0 - C::HBA;
        uint32_t bytes = (uint32_t)D * C::BTP * 4;
        if (!Y0BITS) bytes += C::Y_BYTES;
        if (rad) bytes += (uint32_t)C::YR * Wd * 8;
        mbar_expect_tx(&bar[st], bytes);
        if (!Y0BITS) bulk_load(sb + C::Y_OFF, Yprev + pb * SC, C::Y_BYTES, &bar[st]);
        for (int d = 0; d < D; ++d)
            bulk_load(sb + C::B_OFF + (uint32_t)d * C::BTP * 4, vals + d * ld + pb, C::BTP * 4,
                      &bar[st]);
        if (rad) bulk_load(sb + C::S_OFF, bits + pb * Wd, (uint32_t)C::YR * Wd * 8, &bar[st]);
    };
    auto fill = [&](int64_t ch, int st) {  // edge chunk: bounds-checked loads, zeros outside
        unsigned char* sb = smraw + st * C::STAGE;
        const int64_t r0 = ch * C::CH, pb = r0 - C::HBA;
        if (!Y0BITS) {
            float4* y = reinterpret_cast<float4*>(sb + C::Y_OFF);
            for (int k = tid; k < C::YR * SC4; k += C::NT) {
                const int64_t p = pb + k / SC4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p >= 0 && p < n) v = *reinterpret_cast<const float4*>(Yprev + p * SC + 4 * (k % SC4));
                y[k] = v;
            }
        }
        float* bt = reinterpret_cast<float*>(sb + C::B_OFF);
        for (int k = tid; k < D * C::BTP; k += C::NT) {
            const int d = k / C::BTP;
            const int64_t p = pb + (k - d * C::BTP);
            bt[k] = (p >= 0 && p < n - d) ? vals[d * ld + p] : 0.f;
        }
        if (rad) {
            uint64_t* bs = reinterpret_cast<uint64_t*>(sb + C::S_OFF);
            for (int k = tid; k < C::YR * Wd; k += C::NT) {
                const int64_t p = pb + k / Wd;
                bs[k] = (p >= 0 && p < n) ? bits[p * Wd + (k % Wd)] : 0ull;
            }
        }
        fence_proxy_async_smem();  // before a later bulk copy into this stage
        __syncthreads();
    };

    float mhi[4] = {0.f, 0.f, 0.f, 0.f}, mlo[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t ph = 0u, pend = 0u;  // bit st: parity of stage st / a copy into it in flight
    if (tid == 0)
        for (int k = 0; k < NS - 1 && k < nk; ++k)
            if (interior(cbeg + k)) {
                issue(cbeg + k, k);
                pend |= 1u << k;
            }
    bool aborted = false;
    int st = 0;
    for (int64_t k = 0; k < nk; ++k, st = (st + 1 == NS) ? 0 : st + 1) {
        const int64_t ch = cbeg + k;
        // the stage of chunk k + NS - 1 was released at the end of chunk k - 1
        const int sn = st == 0 ? NS - 1 : st - 1;
        if (tid == 0 && k + NS - 1 < nk && interior(ch + NS - 1)) {
            issue(ch + NS - 1, sn);
            pend |= 1u << sn;
        }
        const int64_t p0 = ch * C::CH + RB * rb;
        // Y_{t-2} of this thread's rows, used in the epilogue
        float4 y2r[RB];
        if (kind == EPI_CHEB && !y2bits) {
#pragma unroll
            for (int i = 0; i < RB; ++i)
                y2r[i] = (p0 + i < n) ? __ldcs(reinterpret_cast<const float4*>(Yprev2 + (p0 + i) * SC + c0))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (interior(ch)) {
            if (!mbar_wait(&bar[st], (ph >> st) & 1u, abort_flag)) *abort_flag = 1;
            ph ^= 1u << st;
            pend &= ~(1u << st);
        } else {
            fill(ch, st);
        }
        const unsigned char* sb = smraw + st * C::STAGE;
        const float* yt = reinterpret_cast<const float*>(sb + C::Y_OFF);
        const float* bt = reinterpret_cast<const float*>(sb + C::B_OFF);
        const uint64_t* bs = reinterpret_cast<const uint64_t*>(sb + C::S_OFF);
        const int o = RB * rb + C::HBA;  // tile row and diagonal position of row p0
        const float* yb = yt + o * SC + c0;
        auto ld_y = [&](int r) -> float4 {  // Y_{t-1} row p0 + r, -HB <= r <= 7 + HB
            if (Y0BITS) return signs4(bs[(o + r) * Wd + jw], jb);
            return lds4(yb + r * SC);
        };
        // accumulators as column pairs: one packed FMA (fma.rn on each half,
        // the same rounding as fmaf) covers two columns
        float2 acc[RB][2];
#pragma unroll
        for (int i = 0; i < RB; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
        float4 win[RB], y1[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) win[i] = ld_y(i - HB);
        float v[RB];
        band_coeffs<RB, C::BTP>(bt, o, -HB, v);
#pragma unroll
        for (int d = -HB; d <= HB; ++d) {
            // the next offset's coefficients and window row, ahead of the FMAs
            float vn[RB];
            float4 wn = make_float4(0.f, 0.f, 0.f, 0.f);
            if (d < HB) {
                band_coeffs<RB, C::BTP>(bt, o, d + 1, vn);
                wn = ld_y(d + RB);
            }
            if (d == 0) {
#pragma unroll
                for (int i = 0; i < RB; ++i) y1[i] = win[i];
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const float2 vv = make_float2(v[i], v[i]);
                acc[i][0] = __ffma2_rn(vv, make_float2(win[i].x, win[i].y), acc[i][0]);
                acc[i][1] = __ffma2_rn(vv, make_float2(win[i].z, win[i].w), acc[i][1]);
            }
            if (d < HB) {
#pragma unroll
                for (int i = 0; i < RB - 1; ++i) win[i] = win[i + 1];
                win[RB - 1] = wn;
#pragma unroll
                for (int i = 0; i < RB; ++i) v[i] = vn[i];
            }
        }
        // epilogue: the update of each row, its moment terms and the store
        float ms[4] = {0.f, 0.f, 0.f, 0.f};
        if (kind != EPI_NONE) {
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int64_t p = p0 + i;
                if (p < n) {
                    const float4 g = rad ? signs4(bs[(o + i) * Wd + jw], jb)
                                         : *reinterpret_cast<const float4*>(G + p * s + j0);
                    const float z[4] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y};
                    const float gv[4] = {g.x, g.y, g.z, g.w};
                    const float yv[4] = {y1[i].x, y1[i].y, y1[i].z, y1[i].w};
                    float yo[4];
                    if (kind == EPI_CHEB1) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            yo[c] = a * z[c] - gv[c];
                            ms[c] = fmaf(gv[c], yo[c], ms[c]);
                        }
                    } else if (kind == EPI_CHEB) {
                        const float4 q2 = y2bits ? g : y2r[i];
                        const float y2v[4] = {q2.x, q2.y, q2.z, q2.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            yo[c] = 2.f * (a * z[c] - yv[c]) - y2v[c];
                            ms[c] = fmaf(gv[c], yo[c], ms[c]);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            yo[c] = yv[c] - z[c] * invu;
                            ms[c] = fmaf(gv[c], z[c], ms[c]);
                        }
                    }
                    *reinterpret_cast<float4*>(Ynew + p * SC + c0) = make_float4(yo[0], yo[1], yo[2], yo[3]);
                }
            }
        }
        // compensated running sum of the chunk sums (Kahan)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float yk = ms[c] - mlo[c];
            const float tk = mhi[c] + yk;
            mlo[c] = (tk - mhi[c]) - yk;
            mhi[c] = tk;
        }
        __syncthreads();  // the stage is free for the next copy
        if (*abort_flag) {
            aborted = true;
            break;
        }
    }
    if (aborted) {
        if (tid == 0) {
            // wait (bounded) for the copies still in flight before the CTA exits
            for (int b = 0; b < NS; ++b) {
                if (!((pend >> b) & 1u)) continue;
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&bar[b], (ph >> b) & 1u) && globaltimer() - t0 < kWaitNs) {
                }
            }
            atomicOr(reinterpret_cast<unsigned long long*>(sc + SC_FLAGS),
                     (unsigned long long)FLAG_TIMEOUT);
        }
        return;
    }
    // per-CTA moment partials, summed over the row blocks in a fixed order
    double* red = reinterpret_cast<double*>(smraw);
#pragma unroll
    for (int c = 0; c < 4; ++c) red[rb * SC + c0 + c] = (double)mhi[c] - (double)mlo[c];
    __syncthreads();
    if (tid < SC) {
        const bool on = (tid >= cols.cheb_c0 && tid < cols.cheb_c0 + cols.ncheb) ||
                        (tid >= cols.tay_c0 && tid < cols.tay_c0 + cols.ntay);
        if (on) {
            double tot = 0.0;
            for (int r = 0; r < C::NRB; ++r) tot += red[r * SC + tid];
            P.slot(t)[(size_t)blockIdx.x * SC + tid] = tot;
        }
    }
}

// VNE_DIA_TMA=0 selects the register-window kernel for every shape (read at
// each call, so that tests can compare the two kernels in one process).
static bool dia_tma_enabled() {
    const char* e = getenv("VNE_DIA_TMA");
    return !(e && e[0] == '0');
}

// The bulk-copy step applies to FP32 with S in {32, 64, 128} columns (s a
// multiple of 4) and a band whose diagonals start on 16-byte boundaries.
bool dia_tma_ok(int is_double, int D, int64_t n, int S, int s, int band_aligned) {
    return !is_double && band_aligned && (S == 32 || S == 64 || S == 128) && s % 4 == 0 &&
           dia_supported_halfbw(D) > 0 && n > 0 && dia_tma_enabled();
}

template <int SC> static int dia_tma_rows(int hb) {
    switch (hb) {
        case 1: return DiaTma<1, SC, kDiaNT, kDiaRB>::CH;
        case 2: return DiaTma<2, SC, kDiaNT, kDiaRB>::CH;
        case 4: return DiaTma<4, SC, kDiaNT, kDiaRB>::CH;
        case 8: return DiaTma<8, SC, kDiaNT, kDiaRB>::CH;
        default: return DiaTma<16, SC, kDiaNT, kDiaRB>::CH;
    }
}

int dia_tma_grid(int D, int64_t n, int S, int sm_count) {
    const int hb = dia_supported_halfbw(D);
    const int ch = S == 32 ? dia_tma_rows<32>(hb) : S == 64 ? dia_tma_rows<64>(hb) : dia_tma_rows<128>(hb);
    const int64_t nchunks = (n + ch - 1) / ch;
    return (int)std::min<int64_t>(sm_count, nchunks);
}

template <int HB, int SC>
static cudaError_t launch_tma_hb(const float* vals, int64_t ld, int D, int64_t n, const float* Yprev,
                                 const float* Yprev2, float* Ynew, const float* G,
                                 const uint64_t* bits, int Wd, int s, StepCols cols,
                                 const double* sc, Partials P, int t, int nblocks, cudaStream_t st) {
    using C = DiaTma<HB, SC, kDiaNT, kDiaRB>;
    const int64_t nchunks = (n + C::CH - 1) / C::CH;
    if (nblocks < 1 || (int64_t)nblocks > nchunks) return cudaErrorInvalidValue;
    if (bits && Wd > C::WDMAX) return cudaErrorInvalidValue;
    auto kern = (bits && t == 1) ? k_dia_step_tma<HB, SC, true, kDiaNT, kDiaRB>
                                 : k_dia_step_tma<HB, SC, false, kDiaNT, kDiaRB>;
    cudaError_t e = set_max_dynamic_smem((const void*)kern, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, C::NT, C::SMEM, st>>>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols,
                                         const_cast<double*>(sc), P, t, nchunks);
    return cudaGetLastError();
}

template <int SC>
static cudaError_t launch_tma_sc(const float* vals, int64_t ld, int D, int64_t n, const float* Yprev,
                                 const float* Yprev2, float* Ynew, const float* G,
                                 const uint64_t* bits, int Wd, int s, StepCols cols,
                                 const double* sc, Partials P, int t, int nblocks, cudaStream_t st) {
    switch (dia_supported_halfbw(D)) {
        case 1: return launch_tma_hb<1, SC>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
        case 2: return launch_tma_hb<2, SC>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
        case 4: return launch_tma_hb<4, SC>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
        case 8: return launch_tma_hb<8, SC>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
        case 16: return launch_tma_hb<16, SC>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
        default: return cudaErrorInvalidValue;
    }
}


cudaError_t launch_dia_step_tma(const float* vals, int64_t ld, int D, int64_t n, const float* Yprev,
                                const float* Yprev2, float* Ynew, const float* G,
                                const uint64_t* bits, int Wd, int S, int s, StepCols cols,
                                const double* sc, Partials P, int t, int nblocks, cudaStream_t st) {
    if (((uintptr_t)vals & 15) || (ld & 3) || ((uintptr_t)Yprev & 15) || ((uintptr_t)Yprev2 & 15) ||
        ((uintptr_t)Ynew & 15) || ((uintptr_t)G & 15) || ((uintptr_t)bits & 15))
        return cudaErrorInvalidValue;
    if (S == 32) return launch_tma_sc<32>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
    if (S == 64) return launch_tma_sc<64>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
    if (S == 128) return launch_tma_sc<128>(vals, ld, D, n, Yprev, Yprev2, Ynew, G, bits, Wd, s, cols, sc, P, t, nblocks, st);
    return cudaErrorInvalidValue;
}

}  // namespace vne
