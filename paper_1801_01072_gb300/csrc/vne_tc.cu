// Dense recurrence step on the 5th-generation tensor cores (tcgen05, TMEM,
// TMA), BF16 operands with FP32 accumulation, optionally split precision:
// R and Y are each held as P bf16 pieces (piece k = bf16 of the residual of
// pieces 0..k-1) and the step accumulates the products R_a Y_b with a + b < P:
// P = 1 BF16, P = 2 bf16x3 (R_0 Y_0 + R_0 Y_1 + R_1 Y_0), P = 3 bf16x6 (every
// product down to the 2^-16 level: about the precision of FP32 operands).
//
// One CTA computes a 128 x BN tile of Z = R Y_{t-1} (rows of R x probe
// columns) and applies the fused epilogue of the step:
//   Chebyshev (Section 3, forward form of the Clenshaw recurrence of
//   Appendix C): Y_t = 2((2/u) Z - Y_{t-1}) - Y_{t-2}  (Y_1 = (2/u) Z - G),
//   moment partial g^T Y_t;
//   Taylor (Section 2, Algorithm 1a): moment partial g^T Z (= g^T R C^{t-1} g),
//   Y_t = Y_{t-1} - Z/u;
// and writes the bf16 hi/lo shadows of Y_t that are the next step's B operand.
//
// Operands: the R pieces [rows_pad][ldk] and the Y shadows [S_pad][ldk], both
// K-major bf16, loaded by TMA into swizzled shared memory tiles (BK = 64
// elements = 128-byte rows with the 128-byte swizzle, or BK = 32 = 64-byte rows
// with the 64-byte swizzle, which keeps a 3-deep ring for P = 3).  Roles (256
// threads, 8 warps):
//   warp 0 lane 0 : TMA producer over a ring of `stages` buffers
//   warp 1        : TMEM allocation; lane 0 issues tcgen05.mma (M=128, N=BN,
//                   K=16 per instruction) and commits to the ring's "empty"
//                   barriers, finally to the "accumulator full" barrier and
//                   (split K) to the peer's "ring idle" barrier
//   all 8 warps   : epilogue; warp w reads TMEM lanes 32*(w%4).. (its 32 rows)
//                   and the column chunks of parity w/4.
// Every wait on an mbarrier is bounded by a %globaltimer deadline; on
// timeout the CTA raises FLAG_TIMEOUT, drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <algorithm>

#include "vne_common.cuh"
#include "vne_internal.h"
#include "vne_ptx.cuh"
#include "vne_tc_ptx.cuh"

namespace vne {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr int TC_THREADS = 256;

int tc_tile_m() { return TC_BM; }
int tc_tile_k() { return TC_BK; }

// ---------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------

// One full 32-column chunk whose columns are all of one kind, at this thread's
// row: branch-free, so the shared-memory reads, updates and stores of the 32
// columns can be scheduled together.  KIND 0: Taylor, Y_t = Y_{t-1} - Z/u,
// moment g Z; 1: first Chebyshev step, Y_1 = (2/u) Z - G; 2: three-term
// Chebyshev step, Y_t = 2((2/u) Z - Y_{t-1}) - Y_{t-2}; moment g Y_t for both;
// 3: the plain product, Y_t = Z (no moment, no bf16 pieces).
// ob: Y_{t-1} of the chunk in smem ([32 cols][128 rows], Y_{t-2} 32*128 floats
// later); yn / ysh[k]: this row's entry of the chunk's first column in Y_t and
// in its bf16 pieces k < pieces.
struct ShPtr {
    __nv_bfloat16* p[kMaxPieces];
};
__device__ __forceinline__ void store_pieces(float y, const ShPtr& ysh, int pieces, int64_t off) {
    __nv_bfloat16 b = __float2bfloat16_rn(y);
    ysh.p[0][off] = b;
    if (pieces > 1) {
        y -= __bfloat162float(b);  // exact: y minus its own rounding
        b = __float2bfloat16_rn(y);
        ysh.p[1][off] = b;
        if (pieces > 2) ysh.p[2][off] = __float2bfloat16_rn(y - __bfloat162float(b));
    }
}
template <int KIND>
__device__ __forceinline__ void epi_chunk_uniform(const uint32_t* r, const float* g,
                                                  const float* ob, float* yn, const ShPtr& ysh,
                                                  int pieces, int64_t n, int64_t ldk, float fa,
                                                  float finvu, bool row_ok, float* v) {
    float y[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const float z = __uint_as_float(r[q]);
        if (KIND == 0) {
            y[q] = fmaf(-z, finvu, ob[q * TC_BM]);
            v[q] = g[q] * z;
        } else if (KIND == 1) {
            y[q] = fmaf(fa, z, -g[q]);
            v[q] = g[q] * y[q];
        } else if (KIND == 3) {
            y[q] = z;
            v[q] = 0.f;
        } else {
            y[q] = 2.f * fmaf(fa, z, -ob[q * TC_BM]) - ob[(32 + q) * TC_BM];
            v[q] = g[q] * y[q];
        }
    }
    if (row_ok) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            yn[q * n] = y[q];
            if (KIND != 3) store_pieces(y[q], ysh, pieces, q * ldk);
        }
    }
}
struct TcArgs {
    const float* G;
    const float* Yprev;
    const float* Yprev2;
    float* Ynew;
    ShPtr Yout;  // bf16 pieces of Y_t, [S_pad][ldk] each
    int64_t n, ldk;
    int S, s;
    int col0, col_end;  // active columns [col0, col_end)
    int BN, stages, nkb;
    int gst;     // 1: warps 4 and 5 stage the first G chunk of warps 0 and 1 in smem
    int ksplit;  // 2: a CTA pair (cluster along z) splits K and swaps half accumulators
    int64_t keep_rows;  // row tiles starting below this load R evict-last (kept in L2)
    int epi_tma;       // 1: Y_{t-1}, Y_{t-2} of the CTA's own chunks arrive by TMA into smem
    uint32_t ops_off;  // byte offset of that operand area in the 1024-aligned smem
    uint32_t body;     // bytes before the barrier tail: max(operand ring, operand area end)
    uint32_t tmem_cols;
    StepCols cols;
    const double* sc;
    Partials P;
    int t;
};

// Tensor maps of one step: the R pieces, the Y pieces (B operand), and the
// FP32 masters Y_{t-1}, Y_{t-2} read by the epilogue.
struct TcMaps {
    CUtensorMap R[kMaxPieces];
    CUtensorMap Y[kMaxPieces];
    CUtensorMap Yp, Yp2;
};

// P: bf16 pieces of R and Y (1, 2 or 3), a template parameter so that each
// precision's issue loop and epilogue are straight-line code.  P < 3 uses BK =
// 64.  P = 3 uses BK = 32 and chunked accumulation: the tensor cores' FP32
// accumulation truncates toward zero, a bias that grows with the number of
// MMAs summed into one accumulator (measured: -8e-6 relative in R Y at
// n = 8192 with six products into one accumulator).  So each ring stage is
// accumulated afresh in one of two TMEM buffers (columns [0, BN) and [BN,
// 2BN)), its small correction products first while the accumulator is small,
// and warps 4-7 add it with round-to-nearest FP32 adds into a running sum in
// columns [2BN, 3BN), which the epilogue reads (bias then ~4e-8).
// PLAIN: the plain product Y_t = Z (cols.cheb_kind == EPI_PLAIN), compiled
// separately so that the recurrence instances keep their register budget.
template <int P, bool PLAIN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_step(const __grid_constant__ TcMaps maps, const TcArgs a) {
    constexpr int BK = P == 3 ? 32 : 64;
    constexpr bool FLUSH = P == 3;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned carve-out: [stages][A_0 .. A_{P-1} | B_0 .. B_{P-1}] then barriers
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    const uint32_t bytesA = TC_BM * (uint32_t)BK * 2;
    const uint32_t bytesB = (uint32_t)a.BN * (uint32_t)BK * 2;
    const uint32_t stage_bytes = (uint32_t)P * (bytesA + bytesB);
    uint8_t* tail = smem + a.body;  // barriers etc. after both the ring and the operand area
    uint64_t* full_bar = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty_bar = full_bar + a.stages;
    uint64_t* accum_bar = empty_bar + a.stages;
    uint64_t* epi_bar = accum_bar + 1;  // epilogue operands landed
    uint64_t* idle_bar = epi_bar + 1;   // split K: the peer's receive area is idle (1 arrival)
    uint64_t* recv_bar = idle_bar + 1;  // split K: the peer's half has landed (1 per warp)
    uint64_t* accf_bar = recv_bar + 1;  // flush: TMEM buffer b holds a finished chunk [2]
    uint64_t* acce_bar = accf_bar + 2;  // flush: buffer b has been added to the sum [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce_bar + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* red = reinterpret_cast<float*>(tmem_slot + 4);  // [4][BN]
    float* gstash = red + 4 * a.BN;  // [2 chunks][2 warps][32 cols][32 lanes]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM;
    const int n0 = a.col0 + blockIdx.y * a.BN;
    // The only cluster is the split-K CTA pair (along z): each CTA loads its
    // own operand tiles, and the pair meets only in the accumulator exchange.
    const bool in_cluster = a.ksplit > 1;
    int kz = 0;
    bool rank_ok = true;
    if (in_cluster) {
        kz = (int)cluster_ctaid_z();
        rank_ok = (int)cluster_ctarank() == kz;
    }
    // K range of this CTA (the whole K unless the pair splits it)
    const int kb_begin = a.ksplit > 1 ? kz * (a.nkb / 2) : 0;
    const int kb_end = a.ksplit > 1 ? (kz == 0 ? a.nkb / 2 : a.nkb) : a.nkb;
    const int nkb_local = kb_end - kb_begin;
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < a.stages; ++s2) {
            mbar_init(&full_bar[s2], 1);
            mbar_init(&empty_bar[s2], 1);
        }
        mbar_init(accum_bar, 1);
        mbar_init(epi_bar, 1);
        mbar_init(idle_bar, 1);
        mbar_init(recv_bar, TC_THREADS / 32);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 4);  // one arrival per summing warp
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.R[0])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.Y[0])) : "memory");
        // the epilogue's maps too: an unfetched map costs its first copy ~1 us
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.Yp)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.Yp2)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (in_cluster) cluster_sync_all();  // the peer's barriers are initialised before any signal
    tc_fence_after();
    // R: the rows kept in L2 from pass to pass (power method and earlier steps)
    // load evict-last, the rest streams evict-first; the Y shadows are re-read
    // by every row tile (evict last).
    const bool producer = warp == 0 && lane == 0;
    const uint64_t pol_R =
        producer ? ((int64_t)m0 < a.keep_rows ? policy_evict_last() : policy_evict_first()) : 0ull;
    auto load_A = [&](int i) {
        const int st = i % a.stages;
        uint8_t* sA = smem + (size_t)st * stage_bytes;
        const int kb = kb_begin + i;
        mbar_expect_tx(&full_bar[st], stage_bytes);  // whole tiles (A and B) arrive here
#pragma unroll
        for (int p = 0; p < P; ++p)
            tma_load_2d_hint(sA + p * bytesA, &maps.R[p], &full_bar[st], kb * BK, m0, pol_R);
    };
    // R is written before the steps start and never by a step, so the A tiles
    // of the first ring round are requested before waiting on the previous
    // step (their slots are fresh: no empty-barrier wait is needed).
    const int pre = rank_ok ? (nkb_local < a.stages ? nkb_local : a.stages) : 0;
    if (producer)
        for (int i = 0; i < pre; ++i) load_A(i);
    // Launched as a programmatic dependent of the previous step: everything
    // above (barriers, TMEM, tensor-map prefetch, the first R tiles) overlapped
    // that step's tail; from here on this step reads what the previous one wrote.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t tmem_base = *tmem_slot;
    if (!rank_ok && threadIdx.x == 0) *abort_flag = 1;

    bool timed_out = false;
    if (producer) {
        // ---------------- TMA producer ----------------
        const uint64_t pol_Y = policy_evict_last();
        int issued_kb = 0;
        for (int i = 0; i < nkb_local && rank_ok; ++i) {
            const int kb = kb_begin + i;
            const int st = i % a.stages;
            const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
            if (i >= pre) {
                if (!mbar_wait(&empty_bar[st], ph ^ 1u, abort_flag)) {
                    timed_out = true;
                    break;
                }
                load_A(i);
            }
            uint8_t* sB = smem + (size_t)st * stage_bytes + P * bytesA;
#pragma unroll
            for (int p = 0; p < P; ++p)
                tma_load_2d_hint(sB + p * bytesB, &maps.Y[p], &full_bar[st], kb * BK, n0, pol_Y);
            issued_kb = i + 1;
        }
        if (timed_out) {
            *abort_flag = 1;
            // drain: wait (bounded) for the loads of the last `stages` issued blocks
            int first = issued_kb - a.stages;
            if (first < 0) first = 0;
            volatile int never = 0;
            for (int i = first; i < issued_kb; ++i)
                mbar_wait(&full_bar[i % a.stages], (uint32_t)(i / a.stages) & 1u, &never);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_bf16(TC_BM, a.BN);
        for (int i = 0; i < nkb_local && rank_ok; ++i) {
            const int st = i % a.stages;
            const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
            if (!mbar_wait(&full_bar[st], ph, abort_flag)) {
                timed_out = true;
                break;
            }
            tc_fence_after();
            const uint32_t aA = smem_u32(smem + (size_t)st * stage_bytes);
            const uint32_t aB = aA + (uint32_t)P * bytesA;
            if (FLUSH) {
                // this stage is one chunk, accumulated afresh in buffer i & 1
                // once the summing warps have taken its previous contents
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(&acce_bar[b], (uint32_t)((i >> 1) - 1) & 1u, abort_flag)) {
                    timed_out = true;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = tmem_base + (uint32_t)(b * a.BN);
                // the small products first, while the accumulator is small
                issue_stage<P, BK / 16, true>(dcol, aA, bytesA, aB, bytesB, BK, idesc, 0u);
                tc_commit(&accf_bar[b]);
                tc_commit(&empty_bar[st]);
                continue;
            }
            issue_stage<P, BK / 16, false>(tmem_base, aA, bytesA, aB, bytesB, BK, idesc,
                                           i != 0 ? 1u : 0u);
            // frees the ring slot once these MMAs finish
            tc_commit(&empty_bar[st]);
        }
        if (timed_out) *abort_flag = 1;
        tc_commit(accum_bar);  // all issued MMAs (possibly none) complete -> arrive
        if (a.ksplit > 1) {
            // Split K: the peer writes its half of the accumulator into this
            // ring once these MMAs are done; the commit's arrival in the
            // peer's barrier says so as soon as they are (a thread's arrive
            // after the accumulator wait was measured 0.45 us slower).  A CTA
            // that stopped early signals with a plain arrive instead.
            const uint32_t rb = mapa_peer(smem_u32(idle_bar), (uint32_t)(1 - kz));
            if (!timed_out && rank_ok) tc_commit_remote(rb);
            else mbar_remote_arrive(rb);
        }
    } else if (FLUSH && warp >= 4 && rank_ok) {
        // ---------------- chunk sums (flush) ----------------
        // warp 4 + g reads TMEM lanes 32g..32g+31: the rows of lane group g
        const uint32_t lrow = (uint32_t)((warp & 3) * 32) << 16;
        const uint32_t run = tmem_base + lrow + (uint32_t)(2 * a.BN);
        for (int c = 0; c < nkb_local; ++c) {
            const int b = c & 1;
            if (!mbar_wait(&accf_bar[b], (uint32_t)(c >> 1) & 1u, abort_flag)) {
                timed_out = true;
                break;
            }
            tc_fence_after();
            const uint32_t buf = tmem_base + lrow + (uint32_t)(b * a.BN);
            for (int cb = 0; cb < a.BN / 32; ++cb) {
                uint32_t r[32];
                TMEM_LD32(buf + (uint32_t)(cb * 32), r);
                if (c > 0) {
                    uint32_t q[32];
                    TMEM_LD32(run + (uint32_t)(cb * 32), q);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        r[e] = __float_as_uint(__uint_as_float(r[e]) + __uint_as_float(q[e]));
                } else {
                    tmem_wait_ld();
                }
                TMEM_ST32(run + (uint32_t)(cb * 32), r);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_local(&acce_bar[b]);
        }
        if (timed_out) *abort_flag = 1;
    }
    __syncwarp();

    const int rg = warp & 3, chalf = warp >> 2;
    const int row = m0 + rg * 32 + lane;
    const bool row_ok = row < a.n;
    const float uf = (float)a.sc[SC_U];  // FP32 from here on (FP64 is slow on this part)
    const float fa = 2.0f / uf, finvu = 1.0f / uf;
    const int nchunks = a.BN / 32;
    // Split K: the pair swaps halves of their partial accumulators through
    // distributed shared memory (the operand ring is free by now); CTA kz
    // then finishes the chunks [kz*nchunks/2, (kz+1)*nchunks/2).
    const int half = nchunks / 2;
    const int ck_lo = a.ksplit > 1 ? kz * half : 0;
    const int ck_hi = a.ksplit > 1 ? ck_lo + half : nchunks;
    const int ck_first = ck_lo + chalf;
    const int cb0 = a.cols.cheb_c0, cb1 = a.cols.cheb_c0 + a.cols.ncheb;
    const bool three_term = a.cols.cheb_kind == EPI_CHEB;
    constexpr bool plain = PLAIN;  // Y_t = Z: no G, no Y_{t-1}, no moments
    // G of the 32 columns of chunk ck at this thread's row (0 outside the
    // active columns); the columns map to consecutive probes unless the chunk
    // wraps past s.
    auto load_g = [&](int ck, float* g) {
        const int cbase = n0 + ck * 32;
        const int j0 = cbase % a.s;
        const bool nowrap = j0 + 32 <= a.s;
        const float* gcol = a.G + (int64_t)j0 * a.n + row;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int c = cbase + q;
            g[q] = 0.f;
            if (!plain && c < a.col_end && row_ok)
                g[q] = nowrap ? __ldg(gcol + (int64_t)q * a.n)
                              : __ldg(a.G + (int64_t)(c % a.s) * a.n + row);
        }
    };
    // G does not depend on this step: the values of a warp's first two chunks
    // are requested now, so their latency hides behind the mainloop (measured:
    // 0.7 us per launch for the second chunk's).  Warps 0 and 1 come here only
    // at the mainloop's end (their lane 0 produces and issues), so warps 4 and
    // 5, which own the same rows, stage those warps' two chunks in shared
    // memory; loads still in flight in warps 0 and 1 would hold up their next
    // shared-memory access and the cluster barrier behind it.  (Without room
    // for that stash, gst = 0, warps 0 and 1 load their own.)
    float gv[32];
    if ((warp >= 2 || !a.gst) && ck_first < ck_hi) load_g(ck_first, gv);
    float g2[32];
    const bool early2 = (warp >= 2 || a.gst) && ck_first + 2 < ck_hi;
    if (early2 && warp >= 2) load_g(ck_first + 2, g2);
    if (a.gst && (warp == 4 || warp == 5)) {
        // ck_lo < ck_hi: every CTA owns at least one chunk
        for (int j = 0; j < 2 && ck_lo + 2 * j < ck_hi; ++j) {
            float gs[32];
            load_g(ck_lo + 2 * j, gs);
            float* dst = gstash + (j * 2 + warp - 4) * 32 * 32 + lane;
#pragma unroll
            for (int q = 0; q < 32; ++q) dst[q * 32] = gs[q];
        }
        named_bar_arrive(1, 128);
    }

    // the next step may start its prologue on free SMs now
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // ---------------- epilogue (all warps) ----------------
    bool have_acc = mbar_wait(accum_bar, 0u, abort_flag);
    if (!have_acc) {
        // the accumulator barrier may still arrive: wait for it before TMEM is freed
        volatile int never = 0;
        if (threadIdx.x == 0) mbar_wait(accum_bar, 0u, &never);
    }
    // flush: the summing warps have finished (their TMEM stores are complete)
    if (FLUSH) named_bar_sync(2, TC_THREADS);
    bool aborted = (*abort_flag != 0) || !have_acc;
    tc_fence_after();
    __syncwarp();
    const uint32_t peer = (uint32_t)(1 - kz);
    const uint32_t zcol = FLUSH ? (uint32_t)(2 * a.BN) : 0u;  // columns holding Z

    // Y_{t-1} and Y_{t-2} of this CTA's own chunks, [chunk][2][32 cols][128 rows]
    // FP32 in smem, by TMA: the operand ring is idle now, and the copies overlap
    // the accumulator exchange below.  A chunk loads only what its columns use:
    // Y_{t-1} for Taylor and three-term Chebyshev columns, Y_{t-2} for the latter.
    float* ops = reinterpret_cast<float*>(smem + a.ops_off);
    const int nown = ck_hi - ck_lo;
    auto chunk_needs = [&](int ck, bool& n1, bool& n2) {
        const int c0 = n0 + ck * 32;
        const int c1 = c0 + 32 < a.col_end ? c0 + 32 : a.col_end;
        const int o0 = c0 > cb0 ? c0 : cb0, o1 = c1 < cb1 ? c1 : cb1;
        const int ncheb = o1 > o0 ? o1 - o0 : 0;
        const int nall = c1 > c0 ? c1 - c0 : 0;
        n1 = !plain && ((nall > ncheb) || (ncheb > 0 && three_term));
        n2 = !plain && ncheb > 0 && three_term;
    };
    if (a.epi_tma && !aborted && threadIdx.x == 0) {
        uint32_t bytes = 0;
        for (int oc = 0; oc < nown; ++oc) {
            bool n1, n2;
            chunk_needs(ck_lo + oc, n1, n2);
            bytes += (n1 ? 1u : 0u) + (n2 ? 1u : 0u);
        }
        mbar_expect_tx(epi_bar, bytes * 32u * TC_BM * 4u);
        for (int oc = 0; oc < nown; ++oc) {
            bool n1, n2;
            chunk_needs(ck_lo + oc, n1, n2);
            const int c0 = n0 + (ck_lo + oc) * 32;
            if (n1) tma_load_2d(ops + (size_t)(oc * 2 + 0) * 32 * TC_BM, &maps.Yp, epi_bar, m0, c0);
            if (n2) tma_load_2d(ops + (size_t)(oc * 2 + 1) * 32 * TC_BM, &maps.Yp2, epi_bar, m0, c0);
        }
    }

    // Receive buffer of the split-K exchange: float4 slot (chunk*8 + q)*128 + r
    // holds columns 4q..4q+3 of row r, so a warp's 16-byte stores and loads
    // cover 512 contiguous bytes.
    // The pair signals through mbarriers in each other's shared memory: the
    // MMA issuer's commit says that the receive area is idle; every warp says
    // when its part of the half has been written (a release arrive after its
    // stores).  Both signals are sent also by a CTA that aborted, and every
    // CTA waits for the peer's writes before it leaves, so no wait depends on
    // the other CTA's state.
    const float4* recv = reinterpret_cast<const float4*>(smem);
    if (a.ksplit > 1) {
        // the first chunk for the peer is read from TMEM while its signal is awaited
        const int ck0 = (int)peer * half + chalf, ck_end = (int)peer * half + half;
        uint32_t r[32];
        if (!aborted && ck0 < ck_end) {
            TMEM_LD32(tmem_base + ((uint32_t)(rg * 32) << 16) + zcol + (uint32_t)(ck0 * 32), r);
            tmem_wait_ld();
        }
        const bool peer_idle = mbar_wait_cluster(idle_bar, 0u);
        if (!aborted && peer_idle) {
            const uint32_t rbase = mapa_peer(smem_u32(smem), peer);
            for (int ck = ck0; ck < ck_end; ck += 2) {
                if (ck != ck0) {
                    TMEM_LD32(tmem_base + ((uint32_t)(rg * 32) << 16) + zcol + (uint32_t)(ck * 32), r);
                    tmem_wait_ld();
                }
                const uint32_t dst =
                    rbase + (uint32_t)(((ck - (int)peer * half) * 8 * TC_BM + rg * 32 + lane) * 16);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    st_cluster_v4(dst + (uint32_t)(q * TC_BM * 16), r[4 * q], r[4 * q + 1],
                                  r[4 * q + 2], r[4 * q + 3]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_remote_arrive(mapa_peer(smem_u32(recv_bar), peer));
        // the peer's half has landed here
        if (!mbar_wait_cluster(recv_bar, 0u) || !peer_idle) aborted = true;
    }
    const bool ops_ready = a.epi_tma && !aborted && mbar_wait(epi_bar, 0u, abort_flag);

    // One 32-column chunk: Z from TMEM (plus the peer's half), the step's
    // update, Y_t and its bf16 shadows, then the moment partial of each column
    // (transpose-reduce: afterwards lane l holds the 32-row sum of column l).
    // ypf(q) / yp2f(q) return Y_{t-1} / Y_{t-2} of column q; read only where used.
    auto finish_chunk = [&](int ck, uint32_t* r, const float* g, bool uniform_ok, auto ypf,
                            auto yp2f) {
        const int cbase = n0 + ck * 32;
        if (a.ksplit > 1) {
            const float4* rp = recv + (ck - ck_lo) * 8 * TC_BM + rg * 32 + lane;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 p4 = rp[q * TC_BM];
                r[4 * q] = __float_as_uint(__uint_as_float(r[4 * q]) + p4.x);
                r[4 * q + 1] = __float_as_uint(__uint_as_float(r[4 * q + 1]) + p4.y);
                r[4 * q + 2] = __float_as_uint(__uint_as_float(r[4 * q + 2]) + p4.z);
                r[4 * q + 3] = __float_as_uint(__uint_as_float(r[4 * q + 3]) + p4.w);
            }
        }
        float v[32];
        // a full chunk of one kind with its operands in smem takes the
        // branch-free path (G is 0 on rows past n, so their moments vanish)
        const bool full = cbase + 32 <= a.col_end;
        const bool all_cheb = cbase >= cb0 && cbase + 32 <= cb1;
        const bool all_tay = cbase >= cb1 || cbase + 32 <= cb0;
        if (uniform_ok && full && (all_cheb || all_tay)) {
            const float* ob = ops + (size_t)((ck - ck_lo) * 2) * 32 * TC_BM + rg * 32 + lane;
            float* yn = a.Ynew + (int64_t)cbase * a.n + row;
            ShPtr ysh;
            const int64_t o0 = (int64_t)cbase * a.ldk + row;
#pragma unroll
            for (int k = 0; k < kMaxPieces; ++k)
                ysh.p[k] = k < P ? a.Yout.p[k] + o0 : nullptr;
            if (plain)
                epi_chunk_uniform<3>(r, g, ob, yn, ysh, P, a.n, a.ldk, fa, finvu, row_ok, v);
            else if (all_tay)
                epi_chunk_uniform<0>(r, g, ob, yn, ysh, P, a.n, a.ldk, fa, finvu, row_ok, v);
            else if (!three_term)
                epi_chunk_uniform<1>(r, g, ob, yn, ysh, P, a.n, a.ldk, fa, finvu, row_ok, v);
            else
                epi_chunk_uniform<2>(r, g, ob, yn, ysh, P, a.n, a.ldk, fa, finvu, row_ok, v);
        } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int c = cbase + q;
            v[q] = 0.f;
            if (c >= a.col_end || !row_ok) continue;
            const float z = __uint_as_float(r[q]);
            const int64_t idx = (int64_t)c * a.n + row;
            const bool cheb = c >= cb0 && c < cb1;
            float y;
            if (cheb) {
                if (!three_term) y = fmaf(fa, z, -g[q]);
                else y = 2.f * fmaf(fa, z, -ypf(q)) - yp2f(q);
                v[q] = g[q] * y;
            } else if (plain) {
                y = z;
            } else {
                v[q] = g[q] * z;
                y = fmaf(-z, finvu, ypf(q));
            }
            a.Ynew[idx] = y;
            if (!plain) store_pieces(y, a.Yout, P, (int64_t)c * a.ldk + row);
        }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < o; ++k) {
                const float send = upper ? v[k] : v[k + o];
                const float keep = upper ? v[k + o] : v[k];
                v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        red[rg * a.BN + ck * 32 + lane] = v[0];
    };
    if (a.gst && warp < 2) {
        named_bar_sync(1, 128);  // warps 4 and 5 have staged this warp's G chunks
        const float* src = gstash + warp * 32 * 32 + lane;
#pragma unroll
        for (int q = 0; q < 32; ++q) gv[q] = src[q * 32];
        if (early2) {
#pragma unroll
            for (int q = 0; q < 32; ++q) g2[q] = src[2 * 32 * 32 + q * 32];
        }
    }
    if (!aborted && ops_ready) {
        // operands in smem; the next chunk's G is requested while this one runs
        for (int ck = ck_first; ck < ck_hi; ck += 2) {
            uint32_t r[32];
            TMEM_LD32(tmem_base + ((uint32_t)(rg * 32) << 16) + zcol + (uint32_t)(ck * 32), r);
            const bool more = ck + 2 < ck_hi;
            const bool have_early = early2 && ck == ck_first;
            float gn[32];
            if (more && !have_early) load_g(ck + 2, gn);
            const float* ob = ops + (size_t)((ck - ck_lo) * 2) * 32 * TC_BM + rg * 32 + lane;
            tmem_wait_ld();
            finish_chunk(
                ck, r, gv, true, [&](int q) { return ob[q * TC_BM]; },
                [&](int q) { return ob[32 * TC_BM + q * TC_BM]; });
            if (more) {
#pragma unroll
                for (int q = 0; q < 32; ++q) gv[q] = have_early ? g2[q] : gn[q];
            }
        }
    } else if (!aborted) {
        // operands from global memory (rows not 16-byte aligned for TMA):
        // every load of a chunk is issued before any store, which could
        // otherwise alias them and serialise the chunk
        for (int ck = ck_first; ck < ck_hi; ck += 2) {
            uint32_t r[32];
            TMEM_LD32(tmem_base + ((uint32_t)(rg * 32) << 16) + zcol + (uint32_t)(ck * 32), r);
            if (ck != ck_first) load_g(ck, gv);
            float yp[32], yp2[32];
            const int cbase = n0 + ck * 32;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int c = cbase + q;  // warp-uniform
                yp[q] = 0.f;
                yp2[q] = 0.f;
                if (c >= a.col_end || !row_ok) continue;
                const bool cheb = c >= cb0 && c < cb1;
                const int64_t idx = (int64_t)c * a.n + row;
                if (!plain && (!cheb || three_term)) yp[q] = __ldg(a.Yprev + idx);
                if (!plain && cheb && three_term) yp2[q] = __ldg(a.Yprev2 + idx);
            }
            tmem_wait_ld();
            finish_chunk(
                ck, r, gv, false, [&](int q) { return yp[q]; }, [&](int q) { return yp2[q]; });
        }
    }
    tc_fence_before();
    __syncthreads();
    if (!aborted) {
        for (int cl = ck_lo * 32 + threadIdx.x; cl < ck_hi * 32; cl += blockDim.x) {
            const int c = n0 + cl;
            if (c >= a.col_end) continue;
            const double tot = (double)red[cl] + (double)red[a.BN + cl] +
                               (double)red[2 * a.BN + cl] + (double)red[3 * a.BN + cl];
            a.P.slot(a.t)[(size_t)blockIdx.x * a.S + c] = tot;
        }
    }
    // (a split-K pair has already waited for all of its peer's signals, so
    // neither CTA can still be written or signalled by the other here)
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(a.tmem_cols)
                     : "memory");
    }
    if (threadIdx.x == 0 && aborted) {
        unsigned long long* f = (unsigned long long*)&a.sc[SC_FLAGS];
        atomicOr(f, (unsigned long long)FLAG_TIMEOUT);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static bool make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t rows,
                     int64_t row_stride_elems, int box_inner, int box_rows, bool fp32 = false,
                     bool no_swizzle = false) {
    // small cache: consecutive steps reuse the same few operand buffers
    struct Entry {
        const void* base;
        int64_t inner, rows, stride;
        int bi, br;
        bool fp32, nosw;
        CUtensorMap map;
    };
    static Entry cache[16];
    static int next = 0;
    for (const Entry& e : cache)
        if (e.base == base && e.inner == inner && e.rows == rows && e.stride == row_stride_elems &&
            e.bi == box_inner && e.br == box_rows && e.fp32 == fp32 && e.nosw == no_swizzle) {
            *map = e.map;
            return true;
        }
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_stride_elems * (fp32 ? 4 : 2)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    // bf16 operand tiles: the swizzle matches the row length (box_inner * 2 bytes)
    const CUtensorMapSwizzle sw = (fp32 || no_swizzle) ? CU_TENSOR_MAP_SWIZZLE_NONE
                                  : box_inner * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : box_inner * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                         : CU_TENSOR_MAP_SWIZZLE_NONE;
    if (!fp32 && !no_swizzle && sw == CU_TENSOR_MAP_SWIZZLE_NONE) return false;
    CUresult r = enc(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     2, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    Entry& e = cache[next];
    next = (next + 1) % 16;
    e = Entry{base, inner, rows, row_stride_elems, box_inner, box_rows, fp32, no_swizzle, *map};
    return true;
}

bool tma_map_bf16_operand(void* map_out, const void* base, int64_t inner, int64_t rows,
                          int64_t row_stride_elems, int box_rows) {
    return make_map(static_cast<CUtensorMap*>(map_out), base, inner, rows, row_stride_elems,
                    TC_BK, box_rows);
}

bool tma_map_bf16_plain(void* map_out, const void* base, int64_t inner, int64_t rows,
                        int64_t row_stride_elems, int box_inner, int box_rows) {
    return make_map(static_cast<CUtensorMap*>(map_out), base, inner, rows, row_stride_elems,
                    box_inner, box_rows, false, true);
}

// Tile shape of one step.  BN: probe columns per CTA (multiple of 32, <= 256);
// ksplit 2: a CTA pair (cluster along z) splits K.  CM and CN (CTAs along M and
// N sharing operand tiles) are always 1: every CTA loads its own operand
// tiles.  VNE_TC_TILE="BN,1,1[,ksplit]" overrides the default
// (used to sweep shapes); invalid overrides are ignored.
struct TcShape {
    int BN, ntn, CM, CN, ksplit;
};

static bool shape_ok(const TcShape& t, int ncols, int mtiles, int nkb) {
    (void)ncols;
    (void)mtiles;
    if (!(t.BN >= 32 && t.BN <= 256 && t.BN % 32 == 0 && t.CM == 1 && t.CN == 1)) return false;
    return t.ksplit == 1 || (t.ksplit == 2 && t.BN % 64 == 0 && nkb >= 2);
}

// Shapes chosen by the autotuner, per bucket of row tiles (ceil log2) and of
// step columns (<= 32, 64, 128, 256, 512, more); process-wide.
struct TunedShape {
    int valid;
    TcShape sh;
};
static TunedShape g_tuned[16][6];

static int rows_bucket(int mtiles) {
    int b = 0;
    while ((1 << b) < mtiles && b < 15) ++b;
    return b;
}
static int cols_bucket(int ncols) {
    return ncols <= 32 ? 0 : ncols <= 64 ? 1 : ncols <= 128 ? 2 : ncols <= 256 ? 3
                                                            : ncols <= 512 ? 4 : 5;
}

int tc_set_tuned(int64_t n, int ncols, int BN, int CM, int CN, int ksplit) {
    const int mtiles = (int)((n + TC_BM - 1) / TC_BM);
    TunedShape& e = g_tuned[rows_bucket(mtiles)][cols_bucket(ncols)];
    if (BN == 0) {
        e.valid = 0;
        return 0;
    }
    TcShape t{BN, (ncols + BN - 1) / BN, CM, CN, ksplit};
    const int nkb = (int)((n + TC_BK - 1) / TC_BK);
    if (!shape_ok(t, ncols, mtiles, nkb)) return -1;
    e.sh = t;
    e.valid = 1;
    return 0;
}

// Candidate shapes for n x ncols steps: column tiles of one or two MMAs'
// width or 128, each with and without the K split over a CTA pair.
int tc_candidates(int64_t n, int ncols, int (*out)[4], int max) {
    const int mtiles = (int)((n + TC_BM - 1) / TC_BM);
    const int nkb = (int)((n + TC_BK - 1) / TC_BK);
    const int wide = std::min(256, (ncols + 31) / 32 * 32);
    const int bns[3] = {wide, std::max(32, (wide / 2 + 31) / 32 * 32), 128};
    const int cl[2][3] = {{1, 1, 1}, {1, 1, 2}};
    int cnt = 0;
    for (int bi = 0; bi < 3; ++bi) {
        if (bi > 0 && bns[bi] == bns[0]) continue;
        if (bi == 2 && bns[2] == bns[1]) continue;
        for (int ci = 0; ci < 2 && cnt < max; ++ci) {
            TcShape t{bns[bi], (ncols + bns[bi] - 1) / bns[bi], cl[ci][0], cl[ci][1], cl[ci][2]};
            if (!shape_ok(t, ncols, mtiles, nkb)) continue;
            out[cnt][0] = t.BN;
            out[cnt][1] = t.CM;
            out[cnt][2] = t.CN;
            out[cnt][3] = t.ksplit;
            ++cnt;
        }
    }
    return cnt;
}

// Default: the widest tile (BN up to 256 columns, the largest N of one MMA);
// when that leaves most SMs idle and the doubled grid still fits in one wave
// (one CTA per SM), a CTA pair splits K (ksplit = 2): a second wave would cost
// more than the idle SMs.  A shape set by the autotuner for this bucket comes
// first; VNE_TC_TILE overrides both.
static TcShape choose_shape(int ncols, int mtiles, int nkb, int sm_count) {
    TcShape sh;
    const int ntn = (ncols + 255) / 256;
    sh.BN = ((ncols + ntn - 1) / ntn + 31) / 32 * 32;
    sh.ntn = (ncols + sh.BN - 1) / sh.BN;
    sh.CM = sh.CN = 1;
    sh.ksplit = 1;
    if ((int64_t)mtiles * sh.ntn * 4 < (int64_t)sm_count * 3 &&
        (int64_t)mtiles * sh.ntn * 2 <= (int64_t)sm_count && sh.BN % 64 == 0 && nkb >= 2)
        sh.ksplit = 2;
    static int o_bn = -1, o_cm = 0, o_cn = 0, o_ks = 1;
    if (o_bn < 0) {
        o_bn = 0;
        if (const char* e = getenv("VNE_TC_TILE")) {
            const int got = sscanf(e, "%d,%d,%d,%d", &o_bn, &o_cm, &o_cn, &o_ks);
            if (got < 3) o_bn = 0;
            if (got < 4) o_ks = 1;
        }
    }
    const TunedShape& tu = g_tuned[rows_bucket(mtiles)][cols_bucket(ncols)];
    if (tu.valid) {
        TcShape t = tu.sh;
        t.ntn = (ncols + t.BN - 1) / t.BN;
        if (shape_ok(t, ncols, mtiles, nkb)) sh = t;
    }
    if (o_bn > 0) {
        TcShape t{o_bn, (ncols + o_bn - 1) / o_bn, o_cm, o_cn, o_ks};
        if (shape_ok(t, ncols, mtiles, nkb)) sh = t;
    }
    return sh;
}

int tc_plan(int64_t n, int ncols, int sm_count, int* out) {
    if (n < 1 || ncols < 1 || sm_count < 1 || !out) return -1;
    const int64_t rows_pad = (n + TC_BM - 1) / TC_BM * TC_BM;
    const int64_t ldk = (n + TC_BK - 1) / TC_BK * TC_BK;
    const TcShape sh = choose_shape(ncols, (int)(rows_pad / TC_BM), (int)(ldk / TC_BK), sm_count);
    out[0] = sh.BN;
    out[1] = sh.CM;
    out[2] = sh.CN;
    out[3] = sh.ksplit;
    return 0;
}

cudaError_t launch_tc_step(const TcStep& s, int sm_count, cudaStream_t st) {
    int col0, col_end;
    if (s.cols.ncheb > 0) {
        col0 = s.cols.cheb_c0;
        col_end = s.cols.ntay > 0 ? s.cols.tay_c0 + s.cols.ntay : s.cols.cheb_c0 + s.cols.ncheb;
    } else {
        col0 = s.cols.tay_c0;
        col_end = s.cols.tay_c0 + s.cols.ntay;
    }
    const int ncols = col_end - col0;
    if (ncols <= 0) return cudaSuccess;
    if ((s.ldk % TC_BK) != 0 || (s.rows_pad % TC_BM) != 0) return cudaErrorInvalidValue;
    const int mtiles = (int)(s.rows_pad / TC_BM);
    TcShape sh = choose_shape(ncols, mtiles, (int)(s.ldk / TC_BK), sm_count);
    const int P = s.pieces;
    if (P < 1 || P > kMaxPieces) return cudaErrorInvalidValue;
    // three pieces: chunked accumulation (k_tc_step<3>), which needs three
    // BN-column TMEM regions (BN <= 128 of the 512 columns) and no K split
    const bool flush = P == 3;
    if (flush && (sh.BN > 128 || sh.ksplit > 1)) {
        sh.ntn = (ncols + 127) / 128;
        sh.BN = ((ncols + sh.ntn - 1) / sh.ntn + 31) / 32 * 32;
        sh.ksplit = 1;
    }
    const int BN = sh.BN;
    const int S_pad = (s.S + 31) / 32 * 32;
    for (int p = 0; p < P; ++p)
        if (!s.R[p] || !s.Y[p] || !s.Y_out[p]) return cudaErrorInvalidValue;
    // K per ring stage: 64 (128-byte rows); with three pieces 32 (64-byte
    // rows), which keeps three stages of the widest tile in shared memory
    const int bk = P == 3 ? 32 : TC_BK;

    TcMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int p = 0; p < P; ++p) {
        if (!make_map(&maps.R[p], s.R[p], s.ldk, s.rows_pad, s.ldk, bk, TC_BM))
            return cudaErrorInvalidValue;
        if (!make_map(&maps.Y[p], s.Y[p], s.ldk, S_pad, s.ldk, bk, BN)) return cudaErrorInvalidValue;
    }
    for (int p = P; p < kMaxPieces; ++p) {
        maps.R[p] = maps.R[0];
        maps.Y[p] = maps.Y[0];
    }
    const uint32_t stage_bytes = (uint32_t)(TC_BM * bk * 2 + BN * bk * 2) * (uint32_t)P;
    // barriers, slot, flag and red; then (gst) the staged G of two warps
    const size_t tail_min = 2 * 8 * 16 + 16 + 16 + 4 * 256 * 4;
    const size_t stash = 2 * 2 * 32 * 32 * 4;  // [2 chunks][2 warps][32 cols][32 lanes]
    const size_t max_smem = 227 * 1024;
    int gst = 1;
    int stages = (int)((max_smem - 1024 - tail_min - stash) / stage_bytes);
    const int stages_nogst = (int)((max_smem - 1024 - tail_min) / stage_bytes);
    if (stages < 3 && stages_nogst > stages) {  // a deeper ring is worth more than the stash
        gst = 0;
        stages = stages_nogst;
    }
    const size_t tail = tail_min + (gst ? stash : 0);
    if (stages > 8) stages = 8;
    if (stages < 2) return cudaErrorInvalidValue;
    // epilogue operand area (after the split-K receive buffer, if any)
    const int nch = BN / 32;
    const int nown = sh.ksplit > 1 ? nch / 2 : nch;
    const size_t recv_bytes = sh.ksplit > 1 ? (size_t)(nch / 2) * 8 * TC_BM * 16 : 0;
    const size_t ops_off = (recv_bytes + 1023) / 1024 * 1024;
    const size_t ops_end = ops_off + (size_t)nown * 2 * 32 * TC_BM * 4;
    size_t body = (size_t)stages * stage_bytes;
    bool epi_tma = (s.n % 4 == 0) && (1024 + ops_end + tail <= max_smem);
    if (epi_tma && ops_end > body) body = ops_end;
    const size_t smem = 1024 + body + tail;

    TcArgs a{};
    a.G = s.G;
    a.Yprev = s.Yprev;
    a.Yprev2 = s.Yprev2;
    a.Ynew = s.Ynew;
    for (int p = 0; p < kMaxPieces; ++p) a.Yout.p[p] = p < P ? s.Y_out[p] : nullptr;
    a.n = s.n;
    a.ldk = s.ldk;
    a.S = s.S;
    a.s = s.s;
    a.col0 = col0;
    a.col_end = col_end;
    a.BN = BN;
    a.stages = stages;
    a.nkb = (int)(s.ldk / bk);
    a.gst = gst;
    a.ksplit = sh.ksplit;
    // L2 residency: the rows the power method keeps (same budget; split modes stream every piece)
    a.keep_rows = l2_keep_rows(s.rows_pad, s.ldk * 2 * P);
    if (epi_tma) {
        epi_tma = make_map(&maps.Yp, s.Yprev, s.n, s.S, s.n, TC_BM, 32, true) &&
                  make_map(&maps.Yp2, s.Yprev2, s.n, s.S, s.n, TC_BM, 32, true);
    }
    if (!epi_tma) {
        maps.Yp = maps.R[0];
        maps.Yp2 = maps.R[0];
    }
    a.epi_tma = epi_tma ? 1 : 0;
    a.ops_off = (uint32_t)ops_off;
    a.body = (uint32_t)body;
    a.tmem_cols = flush ? 512u : BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
    a.cols = s.cols;
    a.sc = s.sc;
    a.P = s.P;
    a.t = s.t;

    const bool plain = s.cols.cheb_kind == EPI_PLAIN;
    if (plain && P == 1) return cudaErrorInvalidValue;  // plain products use the split modes
    void (*kern)(TcMaps, TcArgs) =
        plain ? (P == 2 ? k_tc_step<2, true> : k_tc_step<3, true>)
              : (P == 1 ? k_tc_step<1, false> : P == 2 ? k_tc_step<2, false> : k_tc_step<3, false>);
    const int ki = plain ? 3 + P : P;
    static size_t smem_set[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // raised as needed, never lowered
    if (smem > smem_set[ki]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        smem_set[ki] = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)mtiles, (unsigned)sh.ntn, (unsigned)sh.ksplit);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = (unsigned)sh.ksplit;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, maps, a);
}

}  // namespace vne
