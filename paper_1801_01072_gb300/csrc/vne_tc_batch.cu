// Batched dense recurrence in one persistent launch: the Chebyshev / Taylor
// steps (Sections 2 and 3) of many density matrices of uneven n, BF16 tensor-
// core products with FP32 accumulation, on the buffers each matrix's prologue
// (bf16 R, power method, probe block) left in its workspace.
//
// Work items are (matrix j, step t, 128-row tile i) in a queue ordered so that
// an item's dependencies (every tile of step t-1 of matrix j) come earlier.
// CTAs (two per SM, 192 threads) take items in queue order from one atomic
// counter; before loading an item a CTA waits (bounded) until the counter of
// step t-1 of its matrix reaches the matrix's tile count.  Every item an item
// waits on was taken earlier by a CTA that does not wait on anything later,
// so the queue always advances, resident or not.  The queue visits a bounded
// set of matrices at a time (rounds of one step of each active matrix), so
// each R is re-read from L2 from one step to the next.
//
// Roles:
//   warp 0 lane 0 : scheduler and TMA producer: takes an item, waits on its
//                   dependency, publishes it in one of two item slots, then
//                   streams the item's R tile rows and the probe block's bf16
//                   copy through a 4-stage ring;
//   warp 1        : TMEM allocation (two accumulators of up to 64 columns);
//                   lane 0 issues tcgen05.mma (M = 128, N = S padded to 32 or
//                   64, K = 16) into the item's accumulator;
//   warps 2-5     : epilogue: one row per thread (TMEM lane quarter warp % 4),
//                   the update of the single-call path (Chebyshev three-term or
//                   first step, Taylor), the FP32 master and its bf16 copy, the
//                   per-tile moment partials in FP64, then the step counter.
// Every wait is bounded (2 s); a timeout raises FLAG_TIMEOUT in the scalar
// block of every matrix and stops the queue.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "vne_common.cuh"
#include "vne_internal.h"
#include "vne_ptx.cuh"
#include "vne_tc_ptx.cuh"

namespace vne {

constexpr int TB_THREADS = 192;
constexpr int TB_STAGES = 4;
constexpr int TB_BM = 128, TB_BK = 64, TB_BNMAX = 64;
constexpr uint32_t TB_A_BYTES = TB_BM * TB_BK * 2;     // 16 KB
constexpr uint32_t TB_B_BYTES = TB_BNMAX * TB_BK * 2;  // 8 KB
constexpr uint32_t TB_STAGE = TB_A_BYTES + TB_B_BYTES;  // 24 KB, a multiple of 1024
constexpr uint32_t TB_TMEM_COLS = 2 * TB_BNMAX;

struct TbSlot {
    int j, t, i, valid;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Named barrier `id` over `count` threads that also ANDs a flag over them, so
// that the epilogue warps leave their loop together.
__device__ __forceinline__ bool named_bar_and(uint32_t id, uint32_t count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
        " bar.red.and.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// every matrix of the batch gets FLAG_TIMEOUT, and the queue stops
__device__ void tb_abort(const TcBatchMat* mats, int count, int* abort_g) {
    atomicExch(abort_g, 1);
    for (int j = 0; j < count; ++j)
        atomicOr(reinterpret_cast<unsigned long long*>(mats[j].flags),
                 (unsigned long long)FLAG_TIMEOUT);
}

__global__ void __launch_bounds__(TB_THREADS, 2)
    k_tc_batch(const CUtensorMap* __restrict__ maps, const TcBatchMat* __restrict__ mats,
               const int4* __restrict__ items, int n_items, int count, int* done, int tstride,
               int* head, int* abort_g, int dep_extra) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* tail = smem + TB_STAGES * TB_STAGE;
    uint64_t* full_bar = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty_bar = full_bar + TB_STAGES;
    uint64_t* slot_full = empty_bar + TB_STAGES;  // [2]
    uint64_t* slot_empty = slot_full + 2;         // [2], 5 arrivals: MMA + 4 epilogue warps
    uint64_t* acc_full = slot_empty + 2;          // [2]
    uint64_t* acc_empty = acc_full + 2;           // [2]
    TbSlot* slots = reinterpret_cast<TbSlot*>(acc_empty + 2);  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(slots + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* kt_issued = reinterpret_cast<int*>(tmem_slot + 2);    // ring loads issued
    int* kt_consumed = reinterpret_cast<int*>(tmem_slot + 3);  // ring stages consumed by MMAs
    float* red = reinterpret_cast<float*>(tmem_slot + 4);  // [4][TB_BNMAX]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TB_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&slot_full[b], 1);
            mbar_init(&slot_empty[b], 5);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 1);
        }
        *abort_flag = 0;
        *kt_issued = 0;
        *kt_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TB_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- scheduler + TMA producer ----------------
            const uint64_t pol_R = policy_evict_last();
            int kt = 0;  // ring position, continued across items
            for (int q = 0;; ++q) {
                const int s = q & 1;
                bool stop = false;
                if (!mbar_wait(&slot_empty[s], ((uint32_t)(q >> 1) & 1u) ^ 1u, abort_flag)) {
                    tb_abort(mats, count, abort_g);
                    stop = true;
                }
                int it = stop ? n_items : atomicAdd(head, 1);
                if (ld_acquire_gpu(abort_g)) it = n_items;
                int4 w = make_int4(0, 0, 0, 0);
                if (it < n_items) {
                    w = items[it];
                    if (w.y >= 2) {  // every tile of step t-1 of matrix j
                        const int need = mats[w.x].tiles + dep_extra;
                        const int* cnt = done + (size_t)w.x * tstride + (w.y - 1);
                        const uint64_t t0 = globaltimer();
                        for (uint32_t spin = 0; ld_acquire_gpu(cnt) < need; ++spin) {
                            if ((spin & 63u) == 63u) {
                                if (ld_acquire_gpu(abort_g)) {
                                    it = n_items;
                                    break;
                                }
                                if (globaltimer() - t0 > kWaitNs) {
                                    tb_abort(mats, count, abort_g);
                                    it = n_items;
                                    break;
                                }
                            }
                        }
                    }
                    // the other CTAs' generic stores, released through the
                    // counter, are read below by the async (TMA) proxy
                    fence_proxy_async_global();
                }
                const bool valid = it < n_items;
                slots[s] = TbSlot{w.x, w.y, w.z, valid ? 1 : 0};
                mbar_arrive_local(&slot_full[s]);
                if (!valid) break;
                const TcBatchMat& M = mats[w.x];
                const CUtensorMap* mR = maps + 3 * w.x;
                const CUtensorMap* mY = maps + 3 * w.x + 1 + ((w.y - 1) & 1);
                const int npad = (M.S + 31) & ~31;
                const uint32_t bytes = TB_A_BYTES + (uint32_t)npad * TB_BK * 2;
                const int nkb = (int)(M.ldk / TB_BK);
                for (int kb = 0; kb < nkb; ++kb, ++kt) {
                    const int st = kt % TB_STAGES;
                    const uint32_t ph = (uint32_t)(kt / TB_STAGES) & 1u;
                    if (!mbar_wait(&empty_bar[st], ph ^ 1u, abort_flag)) {
                        tb_abort(mats, count, abort_g);
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t* sA = smem + (size_t)st * TB_STAGE;
                    mbar_expect_tx(&full_bar[st], bytes);
                    tma_load_2d_hint(sA, mR, &full_bar[st], kb * TB_BK, w.z * TB_BM, pol_R);
                    tma_load_2d_hint(sA + TB_A_BYTES, mY, &full_bar[st], kb * TB_BK, 0, pol_R);
                    *kt_issued = kt + 1;
                }
                if (*abort_flag) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int kt = 0;
            for (int q = 0;; ++q) {
                const int s = q & 1, a = q & 1;
                if (!mbar_wait(&slot_full[s], (uint32_t)(q >> 1) & 1u, abort_flag)) {
                    tb_abort(mats, count, abort_g);
                    *abort_flag = 1;
                    break;
                }
                const TbSlot sl = slots[s];
                mbar_arrive_local(&slot_empty[s]);
                if (!sl.valid) break;
                const TcBatchMat& M = mats[sl.j];
                const int npad = (M.S + 31) & ~31;
                const uint32_t idesc = idesc_bf16(TB_BM, npad);
                const int nkb = (int)(M.ldk / TB_BK);
                if (!mbar_wait(&acc_empty[a], ((uint32_t)(q >> 1) & 1u) ^ 1u, abort_flag)) {
                    tb_abort(mats, count, abort_g);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * TB_BNMAX);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++kt) {
                    const int st = kt % TB_STAGES;
                    const uint32_t ph = (uint32_t)(kt / TB_STAGES) & 1u;
                    if (!mbar_wait(&full_bar[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aA = smem_u32(smem + (size_t)st * TB_STAGE);
                    issue_stage<1, TB_BK / 16, false>(d_tmem, aA, TB_A_BYTES, aA + TB_A_BYTES,
                                                      (uint32_t)npad * TB_BK * 2, TB_BK, idesc,
                                                      kb > 0 ? 1u : 0u);
                    tc_commit(&empty_bar[st]);
                    *kt_consumed = kt + 1;
                }
                if (!ok) {
                    tb_abort(mats, count, abort_g);
                    *abort_flag = 1;
                    break;
                }
                tc_commit(&acc_full[a]);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5, 128 threads) ----------------
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const int et = threadIdx.x - 64;
        for (int q = 0;; ++q) {
            const int s = q & 1, a = q & 1;
            bool ok = mbar_wait(&slot_full[s], (uint32_t)(q >> 1) & 1u, abort_flag);
            TbSlot sl = slots[s];
            if (!ok) sl.valid = 0;
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive_local(&slot_empty[s]);
            if (ok && sl.valid) ok = mbar_wait(&acc_full[a], (uint32_t)(q >> 1) & 1u, abort_flag);
            // every epilogue thread leaves together: a wait that timed out in
            // one warp stops all four
            if (!named_bar_and(1, 128, ok)) {
                if (et == 0) tb_abort(mats, count, abort_g);
                *abort_flag = 1;
                break;
            }
            if (!sl.valid) break;
            const TcBatchMat& M = mats[sl.j];
            const int t = sl.t, S = M.S, sp = M.s;
            const int64_t n = M.n, ldk = M.ldk;
            const int64_t row = (int64_t)sl.i * TB_BM + quarter * 32 + lane;
            const bool row_ok = row < n;
            const bool cheb_on = M.has_cheb && t <= M.m;
            const int tay0 = M.has_cheb ? sp : 0;
            const float u = (float)M.sc[SC_U];
            const float fa = 2.f / u, finvu = 1.f / u;
            const float* Yp = M.Y[(t - 1) % 3];
            const float* Yp2 = M.Y[(t + 1) % 3];
            float* Yn = M.Y[t % 3];
            __nv_bfloat16* sh_out = M.sh[t & 1];
            tc_fence_after();
            const int npad = (S + 31) & ~31;
            uint32_t r0[32], r1[32];
            const uint32_t taddr = tmem_base + (uint32_t)(a * TB_BNMAX) + ((uint32_t)(quarter * 32) << 16);
            TMEM_LD32(taddr, r0);
            if (npad > 32) TMEM_LD32(taddr + 32, r1);
            tmem_wait_ld();
            tc_fence_before();
            named_bar_sync(1, 128);
            if (et == 0) mbar_arrive_local(&acc_empty[a]);  // the accumulator is free
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                if (hh * 32 >= S) break;
                // loads predicated per column (no branches), so that a chunk's
                // operand loads can all be in flight together
                float v[32];
#pragma unroll
                for (int qq = 0; qq < 32; ++qq) {
                    const int c = hh * 32 + qq;
                    const bool is_cheb = c < S && cheb_on && c < sp;
                    const bool is_tay = c < S && M.has_tay && c >= tay0 && c < tay0 + sp;
                    const bool on = row_ok && (is_cheb || is_tay);
                    const int gc = c >= sp ? c - sp : c;  // the column's probe
                    const float z = __uint_as_float(hh == 0 ? r0[qq] : r1[qq]);
                    const float g = on ? M.G[(size_t)gc * n + row] : 0.f;
                    const bool need1 = on && (is_tay || t > 1);
                    const float y1 = need1 ? Yp[(size_t)c * n + row] : 0.f;
                    const float y2 = (on && is_cheb && t > 1) ? Yp2[(size_t)c * n + row] : 0.f;
                    float y, vv;
                    if (is_cheb) {
                        y = t == 1 ? fmaf(fa, z, -g) : 2.f * fmaf(fa, z, -y1) - y2;
                        vv = g * y;
                    } else {
                        y = fmaf(-z, finvu, y1);
                        vv = g * z;
                    }
                    v[qq] = on ? vv : 0.f;
                    if (on) {
                        Yn[(size_t)c * n + row] = y;
                        sh_out[(size_t)c * ldk + row] = __float2bfloat16_rn(y);
                    }
                }
                transpose_reduce32(v);  // lane l: the 32-row sum of column hh*32 + l
                red[quarter * TB_BNMAX + hh * 32 + lane] = v[0];
            }
            // the shadows are read by later items through the async proxy
            fence_proxy_async_global();
            named_bar_sync(1, 128);
            if (et < S) {
                const bool on = (cheb_on && et < sp) || (M.has_tay && et >= tay0 && et < tay0 + sp);
                if (on) {
                    double tot = 0.0;
                    for (int w4 = 0; w4 < 4; ++w4) tot += (double)red[w4 * TB_BNMAX + et];
                    M.P.slot(t)[(size_t)sl.i * S + et] = tot;
                }
            }
            named_bar_sync(1, 128);  // partials written, red free for the next item
            if (et == 0) {
                __threadfence();
                atomicAdd(done + (size_t)sl.j * tstride + t, 1);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        // copies issued but never consumed: wait (bounded) until they land
        for (int k = *kt_consumed; k < *kt_issued; ++k) {
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait(&full_bar[k % TB_STAGES], (uint32_t)(k / TB_STAGES) & 1u) &&
                   globaltimer() - t0 < kWaitNs) {
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TB_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// The power method of a batch (Appendix A, Algorithm alg:power, one trial) in
// one persistent launch.  Items (matrix j, product k = 0..t, 128-row tile i)
// come in dependency order from the same kind of queue; a CTA (256 threads)
// takes one item at a time.  Product k forms y = R x_hat_k, x_hat_k =
// x_k / ||x_k||, for its 128 rows with the bf16 R (FP32 accumulation, one warp
// per row, a warp's 8 rows in flight together, 16-byte loads); ||x_k||^2 is n for the Rademacher start vector,
// else the sum, in tile order, of the per-tile FP64 partials of product k-1.
// The tile's partials of ||y||^2 (and, for the last product, x_hat.y and
// x_hat.x_hat) go to ppart[k & 1][tile]; the CTA that completes the last
// product of a matrix sums them in tile order into the scalar block and sets
// p1~ = x_hat.y / x_hat.x_hat and u = min(1, u_scale p1~).
// ---------------------------------------------------------------------------
// rows of a warp in flight together (the power method of the 256-matrix
// benchmark batch: 8 rows 8.3 ms, 4 rows 9.3 ms, 16 rows 8.9 ms)
constexpr int TB_PW_ROWS = 8;

__global__ void __launch_bounds__(256) k_power_batch(const TcBatchMat* __restrict__ mats,
                                                     const int4* __restrict__ items, int n_items,
                                                     int count, int* done, int tstride, int* head,
                                                     int* abort_g, int power_iters,
                                                     double u_scale, int dep_extra) {
    __shared__ int4 sh_item;
    __shared__ float sh_inv;
    __shared__ float wsum[8][3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (;;) {
        if (tid == 0) {
            int it = atomicAdd(head, 1);
            if (it >= n_items || ld_acquire_gpu(abort_g)) it = -1;
            int4 w = make_int4(-1, 0, 0, 0);
            if (it >= 0) {
                w = items[it];
                if (w.y >= 2) {  // every tile of product k-1 of matrix j
                    const int need = mats[w.x].tiles + dep_extra;
                    const int* cnt = done + (size_t)w.x * tstride + (w.y - 1);
                    const uint64_t t0 = globaltimer();
                    for (uint32_t spin = 0; ld_acquire_gpu(cnt) < need; ++spin) {
                        if ((spin & 63u) == 63u) {
                            if (ld_acquire_gpu(abort_g)) {
                                w.x = -1;
                                break;
                            }
                            if (globaltimer() - t0 > kWaitNs) {
                                tb_abort(mats, count, abort_g);
                                w.x = -1;
                                break;
                            }
                        }
                    }
                }
            }
            if (w.x >= 0) {
                const TcBatchMat& M = mats[w.x];
                const int k = w.y - 1;
                double nrm = (double)M.n;  // ||x_0||^2 of the +-1 start vector
                if (k > 0) {
                    nrm = 0.0;
                    const volatile double* pp = M.ppart + (size_t)((k - 1) & 1) * M.tiles * 3;
                    for (int i = 0; i < M.tiles; ++i) nrm += pp[3 * i];
                }
                sh_inv = (float)(1.0 / sqrt(nrm));
            }
            sh_item = w;
        }
        __syncthreads();
        const int4 w = sh_item;
        if (w.x < 0) break;
        const TcBatchMat& M = mats[w.x];
        const int k = w.y - 1, tile = w.z;
        const bool fin = k == power_iters;
        const float inv = sh_inv;
        const float* __restrict__ x = M.x[k & 1];
        float* __restrict__ y = M.x[(k + 1) & 1];
        const int64_t n = M.n, ldk = M.ldk, n8 = n & ~(int64_t)7;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;  // this lane's share of the tile's sums
        for (int rg = 0; rg < 16; rg += TB_PW_ROWS) {
            const int64_t r0 = (int64_t)tile * 128 + warp * 16 + rg;
            float acc[TB_PW_ROWS];
#pragma unroll
            for (int rr = 0; rr < TB_PW_ROWS; ++rr) acc[rr] = 0.f;
            for (int64_t c = (int64_t)lane * 8; c < n8; c += 256) {
                const float4 xa = __ldg(reinterpret_cast<const float4*>(x + c));
                const float4 xb = __ldg(reinterpret_cast<const float4*>(x + c + 4));
#pragma unroll
                for (int rr = 0; rr < TB_PW_ROWS; ++rr) {
                    const uint4 q = __ldcs(reinterpret_cast<const uint4*>(M.R + (r0 + rr) * ldk + c));
                    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
                    const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
                    const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
                    float v = acc[rr];
                    v = fmaf(f0.x, xa.x, v);
                    v = fmaf(f0.y, xa.y, v);
                    v = fmaf(f1.x, xa.z, v);
                    v = fmaf(f1.y, xa.w, v);
                    v = fmaf(f2.x, xb.x, v);
                    v = fmaf(f2.y, xb.y, v);
                    v = fmaf(f3.x, xb.z, v);
                    v = fmaf(f3.y, xb.w, v);
                    acc[rr] = v;
                }
            }
            for (int64_t c = n8 + lane; c < n; c += 32) {  // ragged end of the rows
                const float xv = x[c];
#pragma unroll
                for (int rr = 0; rr < TB_PW_ROWS; ++rr)
                    acc[rr] = fmaf(__bfloat162float(M.R[(r0 + rr) * ldk + c]), xv, acc[rr]);
            }
#pragma unroll
            for (int rr = 0; rr < TB_PW_ROWS; ++rr) {
                const float dot = warp_sum(acc[rr]);
                const int64_t r = r0 + rr;
                if (lane == rr && r < n) {
                    const float yv = dot * inv;
                    y[r] = yv;
                    a0 = fmaf(yv, yv, a0);
                    if (fin) {
                        const float xh = x[r] * inv;
                        a1 = fmaf(xh, yv, a1);
                        a2 = fmaf(xh, xh, a2);
                    }
                }
            }
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
        if (lane == 0) {
            wsum[warp][0] = a0;
            wsum[warp][1] = a1;
            wsum[warp][2] = a2;
        }
        __syncthreads();
        if (tid == 0) {
            double t3[3] = {0.0, 0.0, 0.0};
            for (int ww = 0; ww < 8; ++ww)
                for (int v = 0; v < 3; ++v) t3[v] += (double)wsum[ww][v];
            double* pp = M.ppart + ((size_t)(k & 1) * M.tiles + tile) * 3;
            pp[0] = t3[0];
            pp[1] = t3[1];
            pp[2] = t3[2];
            __threadfence();
            const int old = atomicAdd(done + (size_t)w.x * tstride + w.y, 1);
            if (fin && old == M.tiles - 1) {  // the matrix's last tile: p1~ and u
                __threadfence();
                const volatile double* vp = M.ppart + (size_t)(k & 1) * M.tiles * 3;
                double s3[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < M.tiles; ++i)
                    for (int v = 0; v < 3; ++v) s3[v] += vp[3 * i + v];
                double* sc = const_cast<double*>(M.sc);
                for (int v = 0; v < 3; ++v) sc[SC_NORM + v] = s3[v];
                const double lam = s3[1] / s3[2];
                const double u = fmin(1.0, u_scale * lam);
                sc[SC_LAM] = lam;
                sc[SC_U] = u;
                if (!isfinite(lam) || !(u > 0.0) || !isfinite(u))
                    atomicOr(reinterpret_cast<unsigned long long*>(M.flags),
                             (unsigned long long)FLAG_BAD_INTERVAL);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side: the queue order, the device table and the launch.
// ---------------------------------------------------------------------------

int64_t tc_batch_schedule(const TcBatchMat* mats, int count, double budget_bytes, int min_tiles,
                          int* items) {
    if (!mats || count < 1) return 0;
    std::vector<int> step((size_t)count, 0);  // next step of each active matrix, 0 = not admitted
    std::vector<int> active;
    int next = 0;
    double bytes = 0.0;
    int tiles = 0;
    int64_t k = 0;
    auto rbytes = [&](int j) { return 2.0 * (double)mats[j].rows_pad * (double)mats[j].ldk; };
    while (next < count || !active.empty()) {
        // admit in the given order while the active bf16 R fit the budget, or
        // while a round would have fewer than min_tiles tiles
        while (next < count && (active.empty() || bytes + rbytes(next) <= budget_bytes ||
                                tiles < min_tiles)) {
            active.push_back(next);
            step[next] = 1;
            bytes += rbytes(next);
            tiles += mats[next].tiles;
            ++next;
        }
        // one round: the next step of every active matrix, all its tiles
        std::vector<int> keep;
        for (int j : active) {
            for (int i = 0; i < mats[j].tiles; ++i, ++k)
                if (items) {
                    items[4 * k] = j;
                    items[4 * k + 1] = step[j];
                    items[4 * k + 2] = i;
                    items[4 * k + 3] = 0;
                }
            if (++step[j] <= mats[j].T) {
                keep.push_back(j);
            } else {
                bytes -= rbytes(j);
                tiles -= mats[j].tiles;
            }
        }
        active.swap(keep);
    }
    return k;
}

namespace {
// device table: [maps: 3 per matrix][matrices][items][counters: count x tstride][head, abort]
struct TbLayout {
    size_t maps, mats, items, done, head, total;
    int tstride;
};
TbLayout tb_layout(const TcBatchMat* mats, int count, int64_t n_items) {
    TbLayout L{};
    int tmax = 0;
    for (int j = 0; j < count; ++j) tmax = std::max(tmax, mats[j].T);
    L.tstride = tmax + 1;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    L.maps = 0;
    L.mats = up(L.maps + (size_t)3 * count * sizeof(CUtensorMap));
    L.items = up(L.mats + (size_t)count * sizeof(TcBatchMat));
    L.done = up(L.items + (size_t)n_items * sizeof(int4));
    L.head = up(L.done + (size_t)count * L.tstride * sizeof(int));
    L.total = up(L.head + 2 * sizeof(int));
    return L;
}
}  // namespace

size_t tc_batch_table_bytes(const TcBatchMat* mats, int count, int64_t n_items) {
    return tb_layout(mats, count, n_items).total;
}

cudaError_t launch_tc_batch(const TcBatchMat* mats, int count, const int* items, int64_t n_items,
                            void* host, void* dev, int sm_count, cudaStream_t st, int dep_extra) {
    if (!mats || count < 1 || !items || n_items < 1 || !host || !dev) return cudaErrorInvalidValue;
    const TbLayout L = tb_layout(mats, count, n_items);
    char* hb = static_cast<char*>(host);
    std::memset(hb, 0, L.total);
    CUtensorMap* hmaps = reinterpret_cast<CUtensorMap*>(hb + L.maps);
    for (int j = 0; j < count; ++j) {
        const TcBatchMat& M = mats[j];
        const int npad = (M.S + 31) & ~31;
        if (M.S < 1 || npad > TB_BNMAX || M.ldk % TB_BK || M.rows_pad % TB_BM) return cudaErrorInvalidValue;
        if (!tma_map_bf16_operand(&hmaps[3 * j], M.R, M.ldk, M.rows_pad, M.ldk, TB_BM) ||
            !tma_map_bf16_operand(&hmaps[3 * j + 1], M.sh[0], M.ldk, npad, M.ldk, npad) ||
            !tma_map_bf16_operand(&hmaps[3 * j + 2], M.sh[1], M.ldk, npad, M.ldk, npad))
            return cudaErrorInvalidValue;
    }
    std::memcpy(hb + L.mats, mats, (size_t)count * sizeof(TcBatchMat));
    std::memcpy(hb + L.items, items, (size_t)n_items * sizeof(int4));
    cudaError_t e = cudaMemcpyAsync(dev, host, L.total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    char* db = static_cast<char*>(dev);
    const uint32_t smem = TB_STAGES * TB_STAGE + 2048 + 1024;
    e = set_max_dynamic_smem((const void*)k_tc_batch, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>((int64_t)2 * sm_count, n_items);
    k_tc_batch<<<grid, TB_THREADS, smem, st>>>(
        reinterpret_cast<const CUtensorMap*>(db + L.maps),
        reinterpret_cast<const TcBatchMat*>(db + L.mats), reinterpret_cast<const int4*>(db + L.items),
        (int)n_items, count, reinterpret_cast<int*>(db + L.done), L.tstride,
        reinterpret_cast<int*>(db + L.head), reinterpret_cast<int*>(db + L.head) + 1, dep_extra);
    return cudaGetLastError();
}

cudaError_t launch_power_batch(const TcBatchMat* mats, int count, const int* items,
                               int64_t n_items, int power_iters, double u_scale, void* host,
                               void* dev, int sm_count, cudaStream_t st, int dep_extra) {
    if (!mats || count < 1 || !items || n_items < 1 || !host || !dev || power_iters < 0)
        return cudaErrorInvalidValue;
    const TbLayout L = tb_layout(mats, count, n_items);
    char* hb = static_cast<char*>(host);
    std::memset(hb, 0, L.total);
    for (int j = 0; j < count; ++j)
        if (!mats[j].x[0] || !mats[j].x[1] || !mats[j].ppart || mats[j].T != power_iters + 1)
            return cudaErrorInvalidValue;
    std::memcpy(hb + L.mats, mats, (size_t)count * sizeof(TcBatchMat));
    std::memcpy(hb + L.items, items, (size_t)n_items * sizeof(int4));
    cudaError_t e = cudaMemcpyAsync(dev, host, L.total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    char* db = static_cast<char*>(dev);
    const int grid = (int)std::min<int64_t>((int64_t)4 * sm_count, n_items);
    k_power_batch<<<grid, 256, 0, st>>>(
        reinterpret_cast<const TcBatchMat*>(db + L.mats), reinterpret_cast<const int4*>(db + L.items),
        (int)n_items, count, reinterpret_cast<int*>(db + L.done), L.tstride,
        reinterpret_cast<int*>(db + L.head), reinterpret_cast<int*>(db + L.head) + 1, power_iters,
        u_scale, dep_extra);
    return cudaGetLastError();
}

}  // namespace vne
