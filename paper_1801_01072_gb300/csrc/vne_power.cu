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
        else
            launch_power_dia_q1<float>(hb, blocks, st, (const float*)vals, n, ld, D,
                                       (const float*)x, (float*)y, sc, partial, counter,
                                       final_step, u_scale);
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
