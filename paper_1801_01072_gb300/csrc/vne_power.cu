// Power method of Appendix A (Algorithm alg:power), q trials side by side.
//
// Each launch forms y = R x_hat for every trial, x_hat = x / ||x|| (the
// printed algorithm does not normalise; dividing each iterate by its norm
// leaves the Rayleigh quotient unchanged and keeps t in the tens finite).
// The norms ||y||^2 (and, after the last product, x_hat^T y and x_hat^T x_hat)
// are reduced per block and then across blocks in FP64: the last block to
// finish sums the block partials in a fixed order and writes the running sums
// to the scalar block.  Per-thread arithmetic uses the accumulation type of
// the path (FP64 on the FP64 path, FP32 otherwise): FP64 throughput on this
// part is a small fraction of FP32, so FP64 stays off the per-element path.
#include <algorithm>
#include <cstdlib>

#include "vne_common.cuh"
#include "vne_internal.h"
#include "vne_ptx.cuh"

namespace vne {

constexpr int kMaxTrials = 8;

template <typename TX>
__global__ void k_power_init(TX* x0, int64_t n, int q, uint64_t seed, double* sc) {
    const int64_t total = n * (int64_t)q;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        x0[e] = (TX)((splitmix_out(seed ^ kPowerSeedXor, (uint64_t)e) >> 63) ? -1 : 1);
    if (blockIdx.x == 0 && threadIdx.x < q) {
        sc[SC_NORM + 3 * threadIdx.x + 0] = (double)n;  // ||x_0||^2 = n
        sc[SC_NORM + 3 * threadIdx.x + 1] = 0.0;
        sc[SC_NORM + 3 * threadIdx.x + 2] = 0.0;
    }
}

template <typename TX>
cudaError_t launch_power_init(TX* x0, int64_t n, int q, uint64_t seed, double* sc,
                              cudaStream_t st) {
    if (q < 1 || q > kMaxTrials) return cudaErrorInvalidValue;
    int blocks = (int)((n * q + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_power_init<TX><<<blocks, 256, 0, st>>>(x0, n, q, seed, sc);
    return cudaGetLastError();
}
template cudaError_t launch_power_init<float>(float*, int64_t, int, uint64_t, double*, cudaStream_t);
template cudaError_t launch_power_init<double>(double*, int64_t, int, uint64_t, double*,
                                               cudaStream_t);

// 1/||x_j|| of the current iterates, computed once per block (FP64) and
// broadcast through shared memory.
template <typename TA>
__device__ __forceinline__ void load_inv_norms(const double* sc, int q, TA* inv_sh) {
    if (threadIdx.x < q) inv_sh[threadIdx.x] = (TA)(1.0 / sqrt(sc[SC_NORM + 3 * threadIdx.x]));
    __syncthreads();
}

// Block partials -> last block -> sc.  acc[3*j + {0,1,2}] holds this
// thread's (y.y, xh.y, xh.xh) of trial j in the path's accumulation type.
template <typename TA>
__device__ void power_finish(const TA* acc, int q, double* partial, unsigned int* counter,
                             double* sc, int final_step, double u_scale) {
    __shared__ double wsum[8][3 * kMaxTrials];
    __shared__ double sh[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nv = 3 * q;
    for (int v = 0; v < nv; ++v) {
        const TA t = warp_sum(acc[v]);
        if (lane == 0) wsum[w][v] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double t = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += wsum[ww][threadIdx.x];
        partial[(size_t)blockIdx.x * 3 * q + threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // each of the 3q sums over gridDim.x partials: every thread takes a fixed
    // strided subset, then a fixed-order block reduction (deterministic)
    const volatile double* vp = partial;
    for (int v = 0; v < nv; ++v) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += vp[(size_t)b * 3 * q + v];
        const double tot = block_sum(t, sh);
        if (threadIdx.x == 0) sc[SC_NORM + v] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *counter = 0u;
        if (final_step) {
            double lam = -1.0;
            bool ok = true;
            for (int j = 0; j < q; ++j) {
                const double r = sc[SC_NORM + 3 * j + 1] / sc[SC_NORM + 3 * j + 2];
                if (!isfinite(r)) ok = false;
                lam = fmax(lam, r);
            }
            double u = fmin(1.0, u_scale * lam);
            sc[SC_LAM] = lam;
            sc[SC_U] = u;
            if (!ok || !(u > 0.0) || !isfinite(u)) {
                unsigned long long* f = (unsigned long long*)&sc[SC_FLAGS];
                *f |= FLAG_BAD_INTERVAL;
            }
        }
    }
}

template <typename TR> struct Ld;
template <> struct Ld<double> {
    static __device__ __forceinline__ double get(const double* p) { return __ldg(p); }
};
template <> struct Ld<float> {
    static __device__ __forceinline__ float get(const float* p) { return __ldg(p); }
};

// Dense, any q: one warp per row, lanes stride over the columns.
template <typename TR, typename TX, typename TA>
__global__ void __launch_bounds__(256) k_power_dense(const TR* R, int64_t n, int64_t ld,
                                                     const TX* x, TX* y, int q, double* sc,
                                                     double* partial, unsigned int* counter,
                                                     int final_step, double u_scale) {
    __shared__ TA inv[kMaxTrials];
    load_inv_norms<TA>(sc, q, inv);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TA acc[3 * kMaxTrials];
    for (int v = 0; v < 3 * q; ++v) acc[v] = (TA)0;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
        TA a[kMaxTrials];
        for (int j = 0; j < q; ++j) a[j] = (TA)0;
        const TR* row = R + i * ld;
        for (int64_t k = lane; k < n; k += 32) {
            const TA r = (TA)Ld<TR>::get(row + k);
            for (int j = 0; j < q; ++j) a[j] += r * (TA)x[(int64_t)j * n + k];
        }
        for (int j = 0; j < q; ++j) {
            const TA yv = warp_sum(a[j]) * inv[j];
            if (lane == 0) {
                y[(int64_t)j * n + i] = (TX)yv;
                acc[3 * j + 0] += yv * yv;
                if (final_step) {
                    const TA xh = (TA)x[(int64_t)j * n + i] * inv[j];
                    acc[3 * j + 1] += xh * yv;
                    acc[3 * j + 2] += xh * xh;
                }
            }
        }
    }
    power_finish<TA>(acc, q, partial, counter, sc, final_step, u_scale);
}

// bf16 rows (16-byte aligned, ld % 8 == 0), any q: 8 entries per lane per load.
__global__ void __launch_bounds__(256) k_power_dense_bf16(const __nv_bfloat16* R, int64_t n,
                                                          int64_t ld, const float* x, float* y,
                                                          int q, double* sc, double* partial,
                                                          unsigned int* counter, int final_step,
                                                          double u_scale) {
    __shared__ float inv[kMaxTrials];
    load_inv_norms<float>(sc, q, inv);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[3 * kMaxTrials];
    for (int v = 0; v < 3 * q; ++v) acc[v] = 0.f;
    const int64_t nvec = n / 8;  // full 8-wide groups
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
        float a[kMaxTrials];
        for (int j = 0; j < q; ++j) a[j] = 0.f;
        const __nv_bfloat16* row = R + i * ld;
        for (int64_t g = lane; g < nvec; g += 32) {
            const uint4 raw = __ldg((const uint4*)(row + g * 8));
            const __nv_bfloat162* h2 = (const __nv_bfloat162*)&raw;
            float r[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h2[e]);
                r[2 * e] = f.x;
                r[2 * e + 1] = f.y;
            }
            for (int j = 0; j < q; ++j) {
                const float4* xv = (const float4*)(x + (int64_t)j * n + g * 8);
                const float4 x0 = xv[0], x1 = xv[1];
                a[j] += r[0] * x0.x + r[1] * x0.y + r[2] * x0.z + r[3] * x0.w + r[4] * x1.x +
                        r[5] * x1.y + r[6] * x1.z + r[7] * x1.w;
            }
        }
        for (int64_t k = nvec * 8 + lane; k < n; k += 32) {
            const float r = __bfloat162float(row[k]);
            for (int j = 0; j < q; ++j) a[j] += r * x[(int64_t)j * n + k];
        }
        for (int j = 0; j < q; ++j) {
            const float yv = warp_sum(a[j]) * inv[j];
            if (lane == 0) {
                y[(int64_t)j * n + i] = yv;
                acc[3 * j + 0] += yv * yv;
                if (final_step) {
                    const float xh = x[(int64_t)j * n + i] * inv[j];
                    acc[3 * j + 1] += xh * yv;
                    acc[3 * j + 2] += xh * xh;
                }
            }
        }
    }
    power_finish<float>(acc, q, partial, counter, sc, final_step, u_scale);
}

// bf16 rows, one trial: U independent 16-byte loads per lane in flight.
// (Sharing x loads across two rows per warp was measured slower.)
template <int U>
__global__ void __launch_bounds__(256) k_power_dense_bf16_q1(
    const __nv_bfloat16* __restrict__ R, int64_t n, int64_t ld, const float* __restrict__ x,
    float* __restrict__ y, double* sc, double* partial, unsigned int* counter, int final_step,
    double u_scale) {
    __shared__ float inv_sh[1];
    load_inv_norms<float>(sc, 1, inv_sh);
    const float inv = inv_sh[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[3] = {0.f, 0.f, 0.f};
    const int64_t nvec = n / 8;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
        const __nv_bfloat16* row = R + i * ld;
        float a = 0.f;
        for (int64_t g0 = lane; g0 < nvec; g0 += 32 * U) {
            uint4 raw[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = g0 + 32 * u;
                raw[u] = g < nvec ? __ldg(reinterpret_cast<const uint4*>(row + g * 8))
                                  : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = g0 + 32 * u;
                if (g < nvec) {
                    const float4 x0 = __ldg(reinterpret_cast<const float4*>(x + g * 8));
                    const float4 x1 = __ldg(reinterpret_cast<const float4*>(x + g * 8 + 4));
                    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&raw[u]);
                    const float2 r0 = __bfloat1622float2(h2[0]), r1 = __bfloat1622float2(h2[1]);
                    const float2 r2 = __bfloat1622float2(h2[2]), r3 = __bfloat1622float2(h2[3]);
                    a = fmaf(r0.x, x0.x, a); a = fmaf(r0.y, x0.y, a);
                    a = fmaf(r1.x, x0.z, a); a = fmaf(r1.y, x0.w, a);
                    a = fmaf(r2.x, x1.x, a); a = fmaf(r2.y, x1.y, a);
                    a = fmaf(r3.x, x1.z, a); a = fmaf(r3.y, x1.w, a);
                }
            }
        }
        for (int64_t k = nvec * 8 + lane; k < n; k += 32) a += __bfloat162float(row[k]) * x[k];
        const float yv = warp_sum(a) * inv;
        if (lane == 0) {
            y[i] = yv;
            acc[0] += yv * yv;
            if (final_step) {
                const float xh = x[i] * inv;
                acc[1] += xh * yv;
                acc[2] += xh * xh;
            }
        }
    }
    power_finish<float>(acc, 1, partial, counter, sc, final_step, u_scale);
}

// bf16 rows, one trial, streamed.  A persistent CTA owns a contiguous range of
// rows and streams them through shared memory with 1-D bulk copies (a ring of
// kStreamStages stages of kStreamRB rows, one mbarrier each), so the HBM
// stream costs a handful of instructions per 16 KB row.  The CTA's two halves
// (128 threads each) consume alternate stages, so one half's reduction and
// barrier overlap the other half's arithmetic.  Each thread keeps the x values
// of its NG column groups (8 columns each) in registers for the whole launch.
constexpr int kStreamRB = 3;      // rows per stage
constexpr int kStreamStages = 4;  // ring depth

// all `nthreads` threads of named barrier `id` arrive; true iff v held for all
__device__ __forceinline__ bool group_all(bool v, int id, int nthreads) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

int64_t l2_keep_rows(int64_t rows, int64_t row_bytes) {
    static int64_t budget = -1;
    if (budget < 0) {
        budget = 0;  // measured: no gain at n = 8192 (the evict-last rows slowed the steps)
        if (const char* e = getenv("VNE_L2_KEEP_MB")) {
            const long v = atol(e);
            if (v >= 0 && v <= 128) budget = (int64_t)v << 20;
        }
    }
    if (row_bytes <= 0) return 0;
    const int64_t k = budget / row_bytes;
    return k < rows ? k : rows;
}

__device__ __forceinline__ uint64_t l2_policy(bool keep) {
    uint64_t p;
    if (keep)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

template <int NG>
__global__ void __launch_bounds__(256, 1) k_power_dense_bf16_stream(
    const __nv_bfloat16* __restrict__ R, int64_t n, int64_t ld, const float* __restrict__ x,
    float* __restrict__ y, double* sc, double* partial, unsigned int* counter, int final_step,
    double u_scale, int keep_per_cta) {
    extern __shared__ __align__(128) uint8_t sraw[];
    __shared__ uint64_t full[kStreamStages];
    __shared__ float red[2][4][kStreamRB];
    __shared__ float inv_sh[1];
    __shared__ int timeout;
    const int tid = threadIdx.x, lane = tid & 31;
    const int grp = tid >> 7, gt = tid & 127, gw = gt >> 5;  // half, thread and warp in half
    const uint32_t row_bytes = (uint32_t)(ld * 2);
    const int nvec = (int)(ld / 8);  // 8-column groups of a padded row
    // rows of this CTA
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per;
    int64_t r1 = r0 + per;
    if (r1 > n) r1 = n;
    const int nblk = r0 < r1 ? (int)((r1 - r0 + kStreamRB - 1) / kStreamRB) : 0;
    if (tid == 0) {
        for (int st = 0; st < kStreamStages; ++st) mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        timeout = 0;
    }
    __syncthreads();
    auto issue = [&](int blk) {
        const int st = blk % kStreamStages;
        const int64_t rb = r0 + (int64_t)blk * kStreamRB;
        const int nr = (int)((r1 - rb) < kStreamRB ? (r1 - rb) : kStreamRB);
        mbar_expect_tx(&full[st], (uint32_t)nr * row_bytes);
        for (int r = 0; r < nr; ++r)
            bulk_load_hint(sraw + ((size_t)st * kStreamRB + r) * row_bytes, R + (rb + r) * ld,
                           row_bytes, &full[st], l2_policy(rb + r - r0 < keep_per_cta));
    };
    // R does not change between products: its first stages are requested
    // before waiting for the previous product (programmatic dependent launch)
    if (tid == 0)
        for (int blk = 0; blk < nblk && blk < kStreamStages; ++blk) issue(blk);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    load_inv_norms<float>(sc, 1, inv_sh);  // includes __syncthreads
    const float inv = inv_sh[0];
    // x of this thread's column groups (g = gt + 128 i), already divided by ||x||
    float xr[NG][8];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int g = gt + 128 * i;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t k = (int64_t)g * 8 + e;
            xr[i][e] = (g < nvec && k < n) ? x[k] * inv : 0.f;
        }
    }
    float acc[3] = {0.f, 0.f, 0.f};
    const int bar_id = 1 + grp;
    for (int blk = grp; blk < nblk; blk += 2) {
        const int st = blk % kStreamStages;
        // bounded wait, then a vote across this half so that all its threads
        // leave the loop together
        const bool got = mbar_wait(&full[st], (uint32_t)(blk / kStreamStages) & 1u, &timeout);
        if (!group_all(got, bar_id, 128)) {
            if (gt == 0) timeout = 1;
            break;
        }
        const int64_t rb = r0 + (int64_t)blk * kStreamRB;
        float part[kStreamRB];
#pragma unroll
        for (int r = 0; r < kStreamRB; ++r) {
            const uint4* row = reinterpret_cast<const uint4*>(sraw + ((size_t)st * kStreamRB + r) * row_bytes);
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int g = gt + 128 * i;
                if (g < nvec) {
                    const uint4 raw = row[g];
                    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
                    const float2 f0 = __bfloat1622float2(h2[0]), f1 = __bfloat1622float2(h2[1]);
                    const float2 f2 = __bfloat1622float2(h2[2]), f3 = __bfloat1622float2(h2[3]);
                    a = fmaf(f0.x, xr[i][0], a); a = fmaf(f0.y, xr[i][1], a);
                    a = fmaf(f1.x, xr[i][2], a); a = fmaf(f1.y, xr[i][3], a);
                    a = fmaf(f2.x, xr[i][4], a); a = fmaf(f2.y, xr[i][5], a);
                    a = fmaf(f3.x, xr[i][6], a); a = fmaf(f3.y, xr[i][7], a);
                }
            }
            part[r] = warp_sum(a);
        }
        if (lane == 0)
#pragma unroll
            for (int r = 0; r < kStreamRB; ++r) red[grp][gw][r] = part[r];
        group_sync(bar_id, 128);  // stage st fully read by this half; partials visible
        if (gt == 0 && blk + kStreamStages < nblk) issue(blk + kStreamStages);
        if (gt < kStreamRB && rb + gt < r1) {
            const float yv = red[grp][0][gt] + red[grp][1][gt] + red[grp][2][gt] + red[grp][3][gt];
            const int64_t i = rb + gt;
            y[i] = yv;
            acc[0] += yv * yv;
            if (final_step) {
                const float xh = x[i] * inv;
                acc[1] += xh * yv;
                acc[2] += xh * xh;
            }
        }
        group_sync(bar_id, 128);  // red[grp] reused by this half's next block
    }
    __syncthreads();
    // the next product may start its prologue and its first R loads now
    if (tid == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0 && timeout) {
        // let every copy already issued land before the block exits
        volatile int never = 0;
        for (int b2 = 0; b2 < nblk && b2 < kStreamStages; ++b2) {
            const int last = ((nblk - 1 - b2) / kStreamStages) * kStreamStages + b2;
            mbar_wait(&full[b2], (uint32_t)(last / kStreamStages) & 1u, &never);
        }
        unsigned long long* f = (unsigned long long*)&sc[SC_FLAGS];
        atomicOr(f, (unsigned long long)FLAG_TIMEOUT);
    }
    power_finish<float>(acc, 1, partial, counter, sc, final_step, u_scale);
}

// ---------------------------------------------------------------------------
// All t+1 products of the power method in one persistent launch (bf16 R, one
// trial), reading only the upper triangle of the symmetric R.
//
// The products y = R x_hat differ only in x, and each launch of the per-
// product kernels above pays a fixed ramp and tail (measured ~13-16 us per
// product at n = 5792 and 8192, whether R came from L2 or HBM).  Here one
// cooperative launch runs every product: R is cut into 128 x 128 tiles (I, K)
// with I <= K, which the CTAs take round-robin; tile (I, K) adds R_IK x_K to
// y_I (row part) and, off the diagonal, R_IK^T x_I to y_K (column part, by
// symmetry R_KI = R_IK^T).  The upper triangle is half of R (67 MB of bf16 at
// n = 8192, which fits in L2 with an evict-last hint), and the TMA ring runs
// on across products, since R does not change.  A product is:
//   x_hat into shared memory (the whole vector, scaled by 1/||x||);
//   the CTA's tiles, each writing its two partial vectors;
//   grid barrier; CTA c sums blocks c, c+G, ... from their nb partials in a
//   fixed order (deterministic) and writes y_b and the block's y.y (and,
//   after the last product, x_hat.y and x_hat.x_hat) in FP64;
//   grid barrier; every CTA forms 1/||y|| from the block sums.
// The same kernel also runs phase by phase (SymArgs::phase >= 0), one launch
// per phase and no grid barrier, for calls that share the GPU with others
// (batched calls): phase 2p = the tiles of product p, 2p + 1 = its block
// sums, 2t + 2 = the Rayleigh quotient.  Every value is computed by the same
// code in the same order in both modes and whatever the grid size, so the
// two give the same bits.
// Every wait is bounded (kWaitNs): on expiry the CTA sets FLAG_TIMEOUT, waits
// (bounded) for its copies in flight and returns.
// ---------------------------------------------------------------------------
constexpr int kSymT = 128;                        // tile edge
constexpr int kSymMaxStages = 4;                  // ring depth (deeper measured no faster)
constexpr int kSymThreads = 256;                  // 8 warps, 16 tile rows each (16 warps: slower)
constexpr int kSymWarps = kSymThreads / 32;
constexpr uint32_t kSymTileBytes = kSymT * kSymT * 2;
constexpr int kSymMaxTiles = 512;                 // tiles per CTA (tile list in smem)
constexpr int64_t kSymMaxRows = 16384;            // x_hat in shared memory (64 KB)

struct SymArgs {
    int pieces;      // 1: R = piece 0; 2: R = piece 0 + piece 1 (the sum is exact in FP32)
    int64_t n;
    int nb;          // 128-row blocks of the padded matrix
    int ntile;       // nb (nb + 1) / 2
    int t;           // products 0..t (the last one gives the Rayleigh quotient)
    int stages;      // ring depth (<= kSymMaxStages)
    const float* x0; // start vector, n entries
    float* ybuf;     // 2 x nb*128 iterates, by product parity
    float* part;     // ntile x 2 x 128 partial vectors (row part, column part)
    unsigned* bar;   // grid barrier counter (zero at launch)
    double* normb;   // nb x 3 block sums (y.y, x_hat.y, x_hat.x_hat)
    double* sc;
    double u_scale;
    int phase;       // -1: every phase in one cooperative launch; else the one phase to run
};

__device__ __forceinline__ int sym_row_start(int I, int nb) { return I * nb - (I * (I - 1)) / 2; }

__device__ __forceinline__ void sym_tma_tile(void* dst, const CUtensorMap* map, uint64_t* bar,
                                             int x, int y, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
        : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier (all CTAs resident: cooperative launch); false on
// timeout, with flag_sh set.
__device__ __forceinline__ bool sym_grid_sync(unsigned* bar, unsigned want, int* flag_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const uint64_t t0 = globaltimer();
        for (uint32_t it = 0;; ++it) {
            if (ld_acquire_u32(bar) >= want) break;
            if ((it & 63u) == 63u && globaltimer() - t0 > kWaitNs) {
                *flag_sh = 1;
                break;
            }
        }
    }
    __syncthreads();
    return *flag_sh == 0;
}

// sum over the CTA of one value per thread, fixed order (result in every thread)
__device__ __forceinline__ double sym_block_sum(double v, double* red) {
    v = block_sum(v, red);  // valid in thread 0
    __syncthreads();
    if (threadIdx.x == 0) red[0] = v;
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

struct SymMaps {
    CUtensorMap R[2];
};

__global__ void __launch_bounds__(kSymThreads, 1) k_power_sym(const __grid_constant__ SymMaps maps,
                                                      const SymArgs a) {
    extern __shared__ __align__(1024) uint8_t sraw[];
    uint8_t* ring = sraw + ((1024u - (smem_u32(sraw) & 1023u)) & 1023u);
    const int NS = a.stages;
    const int NP = a.pieces;
    const uint32_t stage_bytes = (uint32_t)NP * kSymTileBytes;  // the pieces' tiles, one after the other
    float* xsm = reinterpret_cast<float*>(ring + (size_t)NS * stage_bytes);  // nb*128
    __shared__ uint64_t full[kSymMaxStages];
    // 16-byte aligned for its float4 accesses, whatever precedes it
    __shared__ __align__(16) float colsm[2][kSymWarps][kSymT];  // per-warp column partials (two tiles); group sums
    __shared__ int flag_sh;
    __shared__ double red_sh[kSymWarps];
    __shared__ uint32_t tl[kSymMaxTiles];  // this CTA's tiles: (I << 16) | K

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int G = gridDim.x, c = blockIdx.x;
    const int nb = a.nb;
    const int rows = nb * kSymT;
    const bool coop = a.phase < 0;
    const int p_lo = coop ? 0 : a.phase >> 1;
    const int p_hi = coop ? a.t : min(a.phase >> 1, a.t);
    const bool tiles_on = (coop || (a.phase & 1) == 0) && p_lo <= p_hi;
    const bool sums_on = coop || (a.phase & 1) == 1;
    const int mine = tiles_on && c < a.ntile ? (a.ntile - c + G - 1) / G : 0;
    for (int j = tid; j < mine; j += blockDim.x) {
        const int tau = c + j * G;
        int lo = 0, hi = nb - 1;  // the row I whose tiles hold tau
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sym_row_start(mid, nb) <= tau) lo = mid;
            else hi = mid - 1;
        }
        tl[j] = ((uint32_t)lo << 16) | (uint32_t)(lo + (tau - sym_row_start(lo, nb)));
    }
    if (tid == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.R[0])) : "memory");
        flag_sh = 0;
    }
    __syncthreads();
    // 1/||x|| of product p_lo's input, stored by its tile phase for its sum phase
    float* inv_slot = reinterpret_cast<float*>(a.bar + 1);
    const int total = tiles_on && p_hi >= p_lo ? (p_hi - p_lo + 1) * mine : 0;
    uint64_t pol = 0;
    if (tid == 0) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    auto issue = [&](int item) {
        const int st = item % NS;
        const uint32_t tk = tl[item % mine];
        mbar_expect_tx(&full[st], stage_bytes);
        for (int pc = 0; pc < NP; ++pc)
            sym_tma_tile(ring + (size_t)st * stage_bytes + (size_t)pc * kSymTileBytes, &maps.R[pc],
                         &full[st], (int)(tk & 0xFFFFu) * kSymT, (int)(tk >> 16) * kSymT, pol);
    };
    int issued = 0;
    if (tid == 0)
        for (; issued < NS && issued < total; ++issued) issue(issued);

    float inv = (float)(1.0 / sqrt((double)a.n));  // ||x_0||^2 = n
    if (!coop && p_lo > 0 && p_lo <= a.t) {
        if (tiles_on) {  // from the block sums of product p_lo - 1, as below
            double part = 0.0;
            for (int b = tid; b < nb; b += blockDim.x) part += __ldcg(a.normb + (size_t)b * 3);
            inv = (float)(1.0 / sqrt(sym_block_sum(part, red_sh)));
            if (c == 0 && tid == 0) *inv_slot = inv;
        } else {
            inv = __ldcg(inv_slot);
        }
    }
    bool ok = true;
    int consumed = 0;
    for (int p = p_lo; p <= p_hi && ok; ++p) {
        const float* xsrc = p == 0 ? a.x0 : a.ybuf + (size_t)((p - 1) & 1) * rows;
        float* ydst = a.ybuf + (size_t)(p & 1) * rows;
        // x_hat of this product, whole vector, in shared memory (the sums use
        // it only after the last product)
        if (!tiles_on && p != a.t) {
        } else if (p == 0) {
            for (int i = tid; i < rows; i += blockDim.x) xsm[i] = i < a.n ? a.x0[i] * inv : 0.f;
        } else {
            const float4* s4 = reinterpret_cast<const float4*>(xsrc);
            float4* d4 = reinterpret_cast<float4*>(xsm);
            for (int i = tid; i < rows / 4; i += blockDim.x) {
                float4 v = __ldcg(s4 + i);
                v.x *= inv; v.y *= inv; v.z *= inv; v.w *= inv;
                d4[i] = v;
            }
        }
        __syncthreads();
        for (int j = 0; j < mine && tiles_on; ++j) {
            const int item = (p - p_lo) * mine + j;
            const int st = item % NS;
            const uint32_t tk = tl[j];
            const int I = (int)(tk >> 16), K = (int)(tk & 0xFFFFu);
            if (!mbar_wait(&full[st], (uint32_t)(item / NS) & 1u, &flag_sh)) flag_sh = 1;
            const __nv_bfloat16* tile =
                reinterpret_cast<const __nv_bfloat16*>(ring + (size_t)st * stage_bytes);
            const __nv_bfloat16* tile2 = tile + kSymT * kSymT;  // piece 1 (NP == 2)
            const float4 xk = *reinterpret_cast<const float4*>(xsm + K * kSymT + 4 * lane);
            const float* xi_row = xsm + I * kSymT + 16 * w;
            float rp[16];
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int row = 16 * w + r;
                const uint2 raw = *reinterpret_cast<const uint2*>(tile + row * kSymT + 4 * lane);
                float2 f01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
                float2 f23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
                if (NP == 2) {
                    const uint2 r2 = *reinterpret_cast<const uint2*>(tile2 + row * kSymT + 4 * lane);
                    const float2 g01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r2.x));
                    const float2 g23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r2.y));
                    f01.x += g01.x;
                    f01.y += g01.y;
                    f23.x += g23.x;
                    f23.y += g23.y;
                }
                float v = f01.x * xk.x;
                v = fmaf(f01.y, xk.y, v);
                v = fmaf(f23.x, xk.z, v);
                rp[r] = fmaf(f23.y, xk.w, v);
                const float xi = xi_row[r];
                c0 = fmaf(f01.x, xi, c0);
                c1 = fmaf(f01.y, xi, c1);
                c2 = fmaf(f23.x, xi, c2);
                c3 = fmaf(f23.y, xi, c3);
            }
            // row sums over the 32 lanes: fold lane bit 4, then a transpose-
            // reduce over bits 3..0, after which lane l holds row 16w + (l & 15)
#pragma unroll
            for (int r = 0; r < 16; ++r) rp[r] += __shfl_xor_sync(0xffffffffu, rp[r], 16);
#pragma unroll
            for (int o = 8; o >= 1; o >>= 1) {
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int k = 0; k < o; ++k) {
                    const float send = upper ? rp[k] : rp[k + o];
                    const float keep = upper ? rp[k + o] : rp[k];
                    rp[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            const bool diag = I == K;
            // column partials of this tile in colsm[j & 1]: the tile after the
            // next writes that buffer again only after its own barrier below,
            // which every thread passes after this tile's sums
            float (*cs)[kSymT] = colsm[j & 1];
            if (!diag) *reinterpret_cast<float4*>(&cs[w][4 * lane]) = make_float4(c0, c1, c2, c3);
            __syncthreads();  // stage st read by every warp; column partials in smem
            if (flag_sh) {  // a wait gave up (uniform after the barrier)
                ok = false;
                break;
            }
            ++consumed;
            if (tid == 0 && issued < total) issue(issued++);
            float* pr = a.part + (size_t)(c + j * G) * 2 * kSymT;
            if (lane < 16) pr[16 * w + lane] = rp[0];
            if (!diag && tid < kSymT) {
                float sum = 0.f;
#pragma unroll
                for (int ww = 0; ww < kSymWarps; ++ww) sum += cs[ww][tid];
                pr[kSymT + tid] = sum;
            }
        }
        if (!ok) break;
        if (!sums_on) break;
        // every partial of product p is written
        if (coop && !sym_grid_sync(a.bar, (unsigned)(2 * p + 1) * (unsigned)G, &flag_sh)) {
            ok = false;
            break;
        }
        // blocks b = c, c + G, ...: the nb contributions (row parts of tiles
        // (b, b..nb-1), then column parts of tiles (0..b-1, b)); group g (warp
        // g) sums contributions g, g+8, ... with float4 loads, then the eight
        // group sums are added in group order
        for (int b = c; b < nb; b += G) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int e0 = w; e0 < nb; e0 += 8 * kSymWarps) {
                float4 v[8];  // eight loads in flight, summed in order e0, e0 + 16, ...
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + kSymWarps * u;
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < nb) {
                        const float* src = e < nb - b
                            ? a.part + (size_t)(sym_row_start(b, nb) + e) * 2 * kSymT
                            : a.part + (size_t)(sym_row_start(e - (nb - b), nb) + (nb - e)) * 2 * kSymT +
                                  kSymT;
                        v[u] = __ldcg(reinterpret_cast<const float4*>(src) + lane);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    acc.x += v[u].x; acc.y += v[u].y; acc.z += v[u].z; acc.w += v[u].w;
                }
            }
            *reinterpret_cast<float4*>(&colsm[0][w][4 * lane]) = acc;
            __syncthreads();
            double yy = 0.0, xy = 0.0, xx = 0.0;
            if (tid < kSymT) {
                float v = 0.f;
#pragma unroll
                for (int g = 0; g < kSymWarps; ++g) v += colsm[0][g][tid];
                const int gi = b * kSymT + tid;
                ydst[gi] = v;
                yy = (double)v * (double)v;
                const double xh = (double)xsm[gi];
                xy = xh * (double)v;
                xx = xh * xh;
            }
            yy = sym_block_sum(yy, red_sh);
            if (p == a.t) {
                xy = sym_block_sum(xy, red_sh);
                xx = sym_block_sum(xx, red_sh);
            }
            if (tid == 0) {
                a.normb[(size_t)b * 3 + 0] = yy;
                a.normb[(size_t)b * 3 + 1] = xy;
                a.normb[(size_t)b * 3 + 2] = xx;
            }
            __syncthreads();  // colsm reused
        }
        if (!coop) break;
        // every block of product p is final
        if (!sym_grid_sync(a.bar, (unsigned)(2 * p + 2) * (unsigned)G, &flag_sh)) {
            ok = false;
            break;
        }
        if (p < a.t) {
            double part = 0.0;  // ||y||^2 from the block sums (fixed order)
            for (int b = tid; b < nb; b += blockDim.x) part += __ldcg(a.normb + (size_t)b * 3);
            inv = (float)(1.0 / sqrt(sym_block_sum(part, red_sh)));
        }
    }
    if (!ok) {
        // drain: the copies issued and not consumed, each on its own stage
        if (tid == 0) {
            volatile int never = 0;
            for (int item = consumed; item < issued; ++item)
                mbar_wait(&full[item % NS], (uint32_t)(item / NS) & 1u, &never);
            atomicOr(reinterpret_cast<unsigned long long*>(&a.sc[SC_FLAGS]),
                     (unsigned long long)FLAG_TIMEOUT);
        }
        return;
    }
    if (c == 0 && (coop || a.phase == 2 * a.t + 2)) {
        // Rayleigh quotient of the last iterate (Algorithm alg:power)
        double yy = 0.0, xy = 0.0, xx = 0.0;
        for (int b = tid; b < nb; b += blockDim.x) {
            yy += __ldcg(a.normb + (size_t)b * 3 + 0);
            xy += __ldcg(a.normb + (size_t)b * 3 + 1);
            xx += __ldcg(a.normb + (size_t)b * 3 + 2);
        }
        yy = sym_block_sum(yy, red_sh);
        xy = sym_block_sum(xy, red_sh);
        xx = sym_block_sum(xx, red_sh);
        if (tid == 0) {
            a.sc[SC_NORM + 0] = yy;
            a.sc[SC_NORM + 1] = xy;
            a.sc[SC_NORM + 2] = xx;
            const double lam = xy / xx;
            const double u = fmin(1.0, a.u_scale * lam);
            a.sc[SC_LAM] = lam;
            a.sc[SC_U] = u;
            if (!isfinite(lam) || !(u > 0.0) || !isfinite(u))
                *reinterpret_cast<unsigned long long*>(&a.sc[SC_FLAGS]) |= FLAG_BAD_INTERVAL;
        }
    }
}

int64_t power_sym_scratch_bytes(int64_t rows_pad) {
    const int64_t nb = rows_pad / kSymT;
    const int64_t ntile = nb * (nb + 1) / 2;
    return ntile * 2 * kSymT * 4 + 2 * rows_pad * 4 + nb * 3 * 8 + 4 * 256;
}

bool power_sym_fits(int64_t rows_pad, int grid) {
    if (rows_pad % kSymT != 0 || rows_pad > kSymMaxRows || grid < 1) return false;
    const int64_t nb = rows_pad / kSymT, ntile = nb * (nb + 1) / 2;
    const int64_t G = ntile < grid ? ntile : grid;
    return (ntile + G - 1) / G <= kSymMaxTiles;
}

cudaError_t launch_power_sym(const __nv_bfloat16* const* R, int pieces, int64_t n,
                             int64_t rows_pad, int64_t ldk, const float* x0, int t, double* sc,
                             void* scratch, double u_scale, int grid, bool phased,
                             cudaStream_t st) {
    if (!power_sym_fits(rows_pad, grid) || (ldk % 8) != 0 || t < 0 || pieces < 1 || pieces > 2)
        return cudaErrorInvalidValue;
    const int nb = (int)(rows_pad / kSymT);
    const int ntile = nb * (nb + 1) / 2;
    const int G = ntile < grid ? ntile : grid;
    SymMaps maps;
    for (int pc = 0; pc < 2; ++pc)
        if (!tma_map_bf16_plain(&maps.R[pc], R[pc < pieces ? pc : 0], ldk, rows_pad, ldk, kSymT, kSymT))
            return cudaErrorInvalidValue;
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    SymArgs a;
    a.pieces = pieces;
    a.n = n;
    a.nb = nb;
    a.ntile = ntile;
    a.t = t;
    a.x0 = x0;
    a.part = reinterpret_cast<float*>(take((size_t)ntile * 2 * kSymT * 4));
    a.ybuf = reinterpret_cast<float*>(take((size_t)2 * rows_pad * 4));
    a.bar = reinterpret_cast<unsigned*>(take(256));
    a.normb = reinterpret_cast<double*>(take((size_t)nb * 3 * 8));
    a.sc = sc;
    a.u_scale = u_scale;
    a.phase = -1;
    cudaError_t e = phased ? cudaSuccess : cudaMemsetAsync(a.bar, 0, 4, st);
    if (e != cudaSuccess) return e;
    static int static_smem = -1;
    if (static_smem < 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_power_sym);
        if (e != cudaSuccess) return e;
        static_smem = (int)fa.sharedSizeBytes;
    }
    const int64_t room = 227 * 1024 - 1024 - static_smem - rows_pad * 4;
    int stages = (int)(room / ((int64_t)pieces * kSymTileBytes));
    if (stages > kSymMaxStages) stages = kSymMaxStages;
    if (stages < 2) return cudaErrorInvalidValue;
    a.stages = stages;
    const size_t smem = 1024 + (size_t)stages * pieces * kSymTileBytes + (size_t)rows_pad * 4;
    static size_t attr = 0;
    if (smem > attr) {
        e = cudaFuncSetAttribute(k_power_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kSymThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    if (phased) {  // one plain launch per phase: tiles (ring), block sums, Rayleigh quotient
        for (int ph = 0; ph <= 2 * t + 2 && e == cudaSuccess; ++ph) {
            const bool tiles = (ph & 1) == 0 && ph <= 2 * t;
            a.phase = ph;
            a.stages = tiles ? stages : 0;
            cfg.gridDim = dim3(ph == 2 * t + 2 ? 1u : (unsigned)G);
            cfg.dynamicSmemBytes = tiles ? smem : 1024 + (size_t)rows_pad * 4;
            e = cudaLaunchKernelEx(&cfg, k_power_sym, maps, a);
        }
        return e;
    }
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barrier needs it
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_power_sym, maps, a);
}

cudaError_t launch_power_step_dense(const void* R, int rdtype, int64_t n, int64_t ld,
                                    const void* x, void* y, int xdouble, int q, double* sc,
                                    double* partial, unsigned int* counter, int final_step,
                                    double u_scale, int nblocks_cap, cudaStream_t st) {
    if (q < 1 || q > kMaxTrials) return cudaErrorInvalidValue;
    int blocks = (int)((n + 7) / 8);
    if (blocks > nblocks_cap) blocks = nblocks_cap;
    if (rdtype == 0) {
        if (!xdouble) return cudaErrorInvalidValue;
        k_power_dense<double, double, double><<<blocks, 256, 0, st>>>(
            (const double*)R, n, ld, (const double*)x, (double*)y, q, sc, partial, counter,
            final_step, u_scale);
    } else if (rdtype == 1) {
        if (xdouble) return cudaErrorInvalidValue;
        k_power_dense<float, float, float><<<blocks, 256, 0, st>>>(
            (const float*)R, n, ld, (const float*)x, (float*)y, q, sc, partial, counter,
            final_step, u_scale);
    } else {
        if (xdouble || (ld % 8) != 0) return cudaErrorInvalidValue;
        const int nvec = (int)(ld / 8);
        if (q == 1 && nvec <= 128 * 8 && (ld * 2) % 16 == 0) {
            // streamed: one persistent CTA per SM
            static int sms = 0;
            if (!sms) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            }
            int g = sms;
            if (g > blocks) g = blocks;
            if (g < 1) g = 1;
            const size_t smem = (size_t)kStreamStages * kStreamRB * (size_t)ld * 2;
            const int ng = (nvec + 127) / 128;
            // rows kept in L2 across products: the same fraction of every CTA's range
            const int64_t per = (n + g - 1) / g;
            const int64_t keep = l2_keep_rows(n, ld * 2);
            const int keep_per_cta = (int)(keep >= n ? per : (per * keep) / n);
            cudaError_t e = cudaSuccess;
#define VNE_STREAM(NGV)                                                                        \
    do {                                                                                       \
        auto kern = k_power_dense_bf16_stream<NGV>;                                            \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess) {                                                                \
            cudaLaunchConfig_t cfg = {};                                                       \
            cudaLaunchAttribute at[1];                                                         \
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                     \
            at[0].val.programmaticStreamSerializationAllowed = 1;                              \
            cfg.gridDim = dim3(g);                                                             \
            cfg.blockDim = dim3(256);                                                          \
            cfg.dynamicSmemBytes = smem;                                                       \
            cfg.stream = st;                                                                   \
            cfg.attrs = at;                                                                    \
            cfg.numAttrs = 1;                                                                  \
            e = cudaLaunchKernelEx(&cfg, kern, (const __nv_bfloat16*)R, n, ld,                 \
                                   (const float*)x, (float*)y, sc, partial, counter,           \
                                   final_step, u_scale, keep_per_cta);                        \
        }                                                                                      \
    } while (0)
            if (smem <= 200 * 1024) {
                if (ng <= 1) VNE_STREAM(1);
                else if (ng <= 2) VNE_STREAM(2);
                else if (ng <= 4) VNE_STREAM(4);
                else VNE_STREAM(8);
#undef VNE_STREAM
                if (e != cudaSuccess) return e;
                return cudaGetLastError();
            }
        }
        if (q == 1) {
            // one wave of resident blocks (grid-stride over rows): a partial
            // second wave would leave most of the memory system idle
            static int per_sm = 0, sms = 0;
            if (!per_sm) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_power_dense_bf16_q1<16>,
                                                                  256, 0) != cudaSuccess ||
                    per_sm < 1)
                    per_sm = 1;
            }
            int b1 = per_sm * sms;
            if (b1 > blocks) b1 = blocks;
            k_power_dense_bf16_q1<16><<<b1, 256, 0, st>>>(
                (const __nv_bfloat16*)R, n, ld, (const float*)x, (float*)y, sc, partial, counter,
                final_step, u_scale);
            return cudaGetLastError();
        }
        k_power_dense_bf16<<<blocks, 256, 0, st>>>((const __nv_bfloat16*)R, n, ld,
                                                   (const float*)x, (float*)y, q, sc, partial,
                                                   counter, final_step, u_scale);
    }
    return cudaGetLastError();
}

// Banded: one thread per row,
// y_i = sum_d R[i,i+d] x_{i+d} + sum_{d>0} R[i-d,i] x_{i-d}.
template <typename T>
__global__ void __launch_bounds__(256) k_power_dia(const T* __restrict__ vals, int64_t n,
                                                   int64_t ld, int D, const T* __restrict__ x,
                                                   T* __restrict__ y, int q, double* sc,
                                                   double* partial, unsigned int* counter,
                                                   int final_step, double u_scale) {
    __shared__ T inv[kMaxTrials];
    load_inv_norms<T>(sc, q, inv);
    T acc[3 * kMaxTrials];
    for (int v = 0; v < 3 * q; ++v) acc[v] = (T)0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < q; ++j) {
            const T* xj = x + (int64_t)j * n;
            T a = vals[i] * xj[i];
            for (int d = 1; d < D; ++d) {
                if (i + d < n) a += vals[(int64_t)d * ld + i] * xj[i + d];
                if (i - d >= 0) a += vals[(int64_t)d * ld + i - d] * xj[i - d];
            }
            const T yv = a * inv[j];
            y[(int64_t)j * n + i] = yv;
            acc[3 * j + 0] += yv * yv;
            if (final_step) {
                const T xh = xj[i] * inv[j];
                acc[3 * j + 1] += xh * yv;
                acc[3 * j + 2] += xh * xh;
            }
        }
    }
    power_finish<T>(acc, q, partial, counter, sc, final_step, u_scale);
}

// Banded, one trial, compile-time window: every band and x load of a row is
// independent and unrolled; interior rows skip the bounds checks.
template <typename T, int HB>
__global__ void __launch_bounds__(256) k_power_dia_q1(const T* __restrict__ vals, int64_t n,
                                                      int64_t ld, int D, const T* __restrict__ x,
                                                      T* __restrict__ y, double* sc,
                                                      double* partial, unsigned int* counter,
                                                      int final_step, double u_scale) {
    __shared__ T inv_sh[1];
    load_inv_norms<T>(sc, 1, inv_sh);
    const T inv = inv_sh[0];
    T acc[3] = {(T)0, (T)0, (T)0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T a = __ldg(vals + i) * __ldg(x + i);
        if (i >= HB && i + HB < n && D == HB + 1) {
#pragma unroll
            for (int d = 1; d <= HB; ++d) {
                a = Math<T>::fma(__ldg(vals + (int64_t)d * ld + i), __ldg(x + i + d), a);
                a = Math<T>::fma(__ldg(vals + (int64_t)d * ld + i - d), __ldg(x + i - d), a);
            }
        } else {
#pragma unroll
            for (int d = 1; d <= HB; ++d) {
                if (d < D && i + d < n) a += __ldg(vals + (int64_t)d * ld + i) * __ldg(x + i + d);
                if (d < D && i - d >= 0) a += __ldg(vals + (int64_t)d * ld + i - d) * __ldg(x + i - d);
            }
        }
        const T yv = a * inv;
        y[i] = yv;
        acc[0] += yv * yv;
        if (final_step) {
            const T xh = __ldg(x + i) * inv;
            acc[1] += xh * yv;
            acc[2] += xh * xh;
        }
    }
    power_finish<T>(acc, 1, partial, counter, sc, final_step, u_scale);
}

template <typename T>
static void launch_power_dia_q1(int hb, int blocks, cudaStream_t st, const T* vals, int64_t n,
                                int64_t ld, int D, const T* x, T* y, double* sc, double* partial,
                                unsigned int* counter, int final_step, double u_scale) {
    switch (hb) {
        case 1: k_power_dia_q1<T, 1><<<blocks, 256, 0, st>>>(vals, n, ld, D, x, y, sc, partial, counter, final_step, u_scale); break;
        case 2: k_power_dia_q1<T, 2><<<blocks, 256, 0, st>>>(vals, n, ld, D, x, y, sc, partial, counter, final_step, u_scale); break;
        case 4: k_power_dia_q1<T, 4><<<blocks, 256, 0, st>>>(vals, n, ld, D, x, y, sc, partial, counter, final_step, u_scale); break;
        case 8: k_power_dia_q1<T, 8><<<blocks, 256, 0, st>>>(vals, n, ld, D, x, y, sc, partial, counter, final_step, u_scale); break;
        default: k_power_dia_q1<T, 16><<<blocks, 256, 0, st>>>(vals, n, ld, D, x, y, sc, partial, counter, final_step, u_scale); break;
    }
}

// Banded FP32, one trial, fed by bulk copies: a persistent CTA (256 threads,
// one per SM) walks a contiguous run of chunks of CH = 768 rows; one thread
// copies each chunk's D stored diagonals (positions r0-HBA .. r0+CH-1, so that
// both R[p, p+d] = vals[d][p] and R[p, p-e] = vals[e][p-e] are staged) and the
// x rows r0-HBA .. r0+CH+HBA-1 into a ring of shared-memory stages, up to
// NS-1 chunks ahead.  Each thread computes rows r0 + tid + k*256, k < 3, from
// shared memory (consecutive lanes read consecutive words).  Chunks reaching
// outside [0, n) are filled with bounds-checked loads.  Output and norm sums
// as k_power_dia_q1.
template <int HB> struct PowDiaTma {
    static constexpr int W = HB + 1, HBA = (HB + 3) / 4 * 4;
    static constexpr int NT = 256, RPT = 3, CH = NT * RPT;
    static constexpr int BTP = CH + HBA, XR = CH + 2 * HBA;
    static constexpr uint32_t B_BYTES = (uint32_t)W * BTP * 4, X_OFF = B_BYTES;
    static constexpr uint32_t X_BYTES = (uint32_t)XR * 4;
    static constexpr uint32_t STAGE = (X_OFF + X_BYTES + 127) / 128 * 128;
    static constexpr int NSF = (int)((232448u - 64u - 2048u) / STAGE);
    static constexpr int NS = NSF > 4 ? 4 : NSF;
    static constexpr uint32_t BAR_OFF = NS * STAGE, SMEM = BAR_OFF + 64;
    static_assert(NS >= 2 && B_BYTES % 16 == 0 && X_BYTES % 16 == 0, "stage layout");
};

template <int HB>
__global__ void __launch_bounds__(256, 1) k_power_dia_tma(
    const float* __restrict__ vals, int64_t n, int64_t ld, int D, const float* __restrict__ x,
    float* __restrict__ y, double* sc, double* partial, unsigned int* counter, int final_step,
    double u_scale, int64_t nchunks) {
    using C = PowDiaTma<HB>;
    constexpr int NS = C::NS;
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + C::BAR_OFF);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + NS);
    __shared__ float inv_sh[1];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&bar[b], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int b = 0; b < NS; ++b) {  // diagonals D .. HB are never copied
        float* bt = reinterpret_cast<float*>(smraw + b * C::STAGE);
        for (int k = D * C::BTP + tid; k < C::W * C::BTP; k += C::NT) bt[k] = 0.f;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    load_inv_norms<float>(sc, 1, inv_sh);  // ends with __syncthreads
    const float inv = inv_sh[0];

    const int64_t per = nchunks / gridDim.x, rem = nchunks % gridDim.x;
    const int64_t cbeg = (int64_t)blockIdx.x * per + (blockIdx.x < rem ? blockIdx.x : rem);
    const int64_t nk = per + (blockIdx.x < rem ? 1 : 0);
    auto interior = [&](int64_t ch) {
        const int64_t r0 = ch * C::CH;
        return r0 - C::HBA >= 0 && r0 + C::CH + C::HBA <= n;
    };
    auto issue = [&](int64_t ch, int st) {
        unsigned char* sb = smraw + st * C::STAGE;
        const int64_t pb = ch * C::CH - C::HBA;
        mbar_expect_tx(&bar[st], (uint32_t)D * C::BTP * 4 + C::X_BYTES);
        for (int d = 0; d < D; ++d)
            bulk_load(sb + (uint32_t)d * C::BTP * 4, vals + d * ld + pb, C::BTP * 4, &bar[st]);
        bulk_load(sb + C::X_OFF, x + pb, C::X_BYTES, &bar[st]);
    };
    auto fill = [&](int64_t ch, int st) {
        unsigned char* sb = smraw + st * C::STAGE;
        const int64_t pb = ch * C::CH - C::HBA;
        float* bt = reinterpret_cast<float*>(sb);
        for (int k = tid; k < D * C::BTP; k += C::NT) {
            const int d = k / C::BTP;
            const int64_t p = pb + (k - d * C::BTP);
            bt[k] = (p >= 0 && p < n - d) ? vals[d * ld + p] : 0.f;
        }
        float* xt = reinterpret_cast<float*>(sb + C::X_OFF);
        for (int k = tid; k < C::XR; k += C::NT) {
            const int64_t p = pb + k;
            xt[k] = (p >= 0 && p < n) ? x[p] : 0.f;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    };
    uint32_t ph = 0u, pend = 0u;
    if (tid == 0)
        for (int k = 0; k < NS - 1 && k < nk; ++k)
            if (interior(cbeg + k)) {
                issue(cbeg + k, k);
                pend |= 1u << k;
            }
    float acc[3] = {0.f, 0.f, 0.f};
    bool aborted = false;
    int st = 0;
    for (int64_t k = 0; k < nk; ++k, st = (st + 1 == NS) ? 0 : st + 1) {
        const int64_t ch = cbeg + k;
        const int sn = st == 0 ? NS - 1 : st - 1;
        if (tid == 0 && k + NS - 1 < nk && interior(ch + NS - 1)) {
            issue(ch + NS - 1, sn);
            pend |= 1u << sn;
        }
        if (interior(ch)) {
            if (!mbar_wait(&bar[st], (ph >> st) & 1u, abort_flag)) *abort_flag = 1;
            ph ^= 1u << st;
            pend &= ~(1u << st);
        } else {
            fill(ch, st);
        }
        const float* bt = reinterpret_cast<const float*>(smraw + st * C::STAGE);
        const float* xt = reinterpret_cast<const float*>(smraw + st * C::STAGE + C::X_OFF);
#pragma unroll
        for (int r = 0; r < C::RPT; ++r) {
            const int li = tid + r * C::NT;     // row within the chunk
            const int o = li + C::HBA;          // its staged position
            const int64_t p = ch * C::CH + li;
            float a = bt[o] * xt[o];
            float b = 0.f;
#pragma unroll
            for (int d = 1; d <= HB; ++d) {
                a = fmaf(bt[d * C::BTP + o], xt[o + d], a);
                b = fmaf(bt[d * C::BTP + o - d], xt[o - d], b);
            }
            if (p < n) {
                const float yv = (a + b) * inv;
                y[p] = yv;
                acc[0] = fmaf(yv, yv, acc[0]);
                if (final_step) {
                    const float xh = xt[o] * inv;
                    acc[1] = fmaf(xh, yv, acc[1]);
                    acc[2] = fmaf(xh, xh, acc[2]);
                }
            }
        }
        __syncthreads();
        if (*abort_flag) {
            aborted = true;
            break;
        }
    }
    if (aborted) {
        if (tid == 0) {
            for (int b = 0; b < NS; ++b) {
                if (!((pend >> b) & 1u)) continue;
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&bar[b], (ph >> b) & 1u) && globaltimer() - t0 < kWaitNs) {
                }
            }
            atomicOr(reinterpret_cast<unsigned long long*>(sc + SC_FLAGS),
                     (unsigned long long)FLAG_TIMEOUT);
        }
        // the other blocks still count on this one in the final reduction
    }
    power_finish<float>(acc, 1, partial, counter, sc, final_step, u_scale);
}

// The bulk-copy product where it applies (FP32 band on 16-byte boundaries,
// one trial); cudaErrorNotSupported otherwise.
static cudaError_t launch_power_dia_tma(int hb, const float* vals, int64_t n, int64_t ld, int D,
                                        const float* x, float* y, double* sc, double* partial,
                                        unsigned int* counter, int final_step, double u_scale,
                                        int nblocks, cudaStream_t st) {
    if (((uintptr_t)vals & 15) || (ld & 3) || ((uintptr_t)x & 15) || nblocks < 1)
        return cudaErrorNotSupported;
    const char* e = getenv("VNE_DIA_TMA");
    if (e && e[0] == '0') return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorNotSupported;
#define VNE_POW_TMA(HBV)                                                                         \
    {                                                                                            \
        using C = PowDiaTma<HBV>;                                                                \
        const int64_t nchunks = (n + C::CH - 1) / C::CH;                                         \
        const int grid = (int)std::min<int64_t>(std::min(sms, nblocks), nchunks);               \
        cudaError_t err = set_max_dynamic_smem((const void*)k_power_dia_tma<HBV>,                \
                                               (int)C::SMEM);                                    \
        if (err != cudaSuccess) return err;                                                      \
        k_power_dia_tma<HBV><<<grid, C::NT, C::SMEM, st>>>(vals, n, ld, D, x, y, sc, partial,    \
                                                            counter, final_step, u_scale,       \
                                                            nchunks);                            \
        return cudaGetLastError();                                                               \
    }
    switch (hb) {
        case 1: VNE_POW_TMA(1)
        case 2: VNE_POW_TMA(2)
        case 4: VNE_POW_TMA(4)
        case 8: VNE_POW_TMA(8)
        case 16: VNE_POW_TMA(16)
        default: return cudaErrorNotSupported;
    }
#undef VNE_POW_TMA
}

cudaError_t launch_power_step_dia(const void* vals, int rdtype, int64_t n, int64_t ld, int D,
                                  const void* x, void* y, int q, double* sc, double* partial,
                                  unsigned int* counter, int final_step, double u_scale,
                                  int nblocks, cudaStream_t st) {
    if (q < 1 || q > kMaxTrials) return cudaErrorInvalidValue;
    int64_t want = (n + 255) / 256;
    int blocks = (int)(want < nblocks ? want : nblocks);
    if (blocks < 1) blocks = 1;
    const int hb = dia_supported_halfbw(D);
    if (q == 1 && hb > 0) {
        if (rdtype == 0)
            launch_power_dia_q1<double>(hb, blocks, st, (const double*)vals, n, ld, D,
                                        (const double*)x, (double*)y, sc, partial, counter,
                                        final_step, u_scale);
        else {
            const cudaError_t e = launch_power_dia_tma(hb, (const float*)vals, n, ld, D,
                                                       (const float*)x, (float*)y, sc, partial,
                                                       counter, final_step, u_scale, nblocks, st);
            if (e != cudaErrorNotSupported) return e;
            launch_power_dia_q1<float>(hb, blocks, st, (const float*)vals, n, ld, D,
                                       (const float*)x, (float*)y, sc, partial, counter,
                                       final_step, u_scale);
        }
        return cudaGetLastError();
    }
    if (rdtype == 0)
        k_power_dia<double><<<blocks, 256, 0, st>>>((const double*)vals, n, ld, D,
                                                    (const double*)x, (double*)y, q, sc, partial,
                                                    counter, final_step, u_scale);
    else
        k_power_dia<float><<<blocks, 256, 0, st>>>((const float*)vals, n, ld, D,
                                                   (const float*)x, (float*)y, q, sc, partial,
                                                   counter, final_step, u_scale);
    return cudaGetLastError();
}

}  // namespace vne
