// Device helpers of the tensor-core kernels (tcgen05, TMEM, TMA with cache
// hints, cluster signalling): inline PTX shared by vne_tc.cu and
// vne_tc_batch.cu.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "vne_ptx.cuh"

namespace vne {

// Tiled 2-D TMA load into this CTA's shared memory with an L2 cache-policy hint.
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int x, int y, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_ctaid_z() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctaid.z;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa_peer(uint32_t local_addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                              uint32_t d) {
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b),
                 "r"(c), "r"(d)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
// Commit whose arrival goes to the mbarrier at a shared::cluster address (a
// peer CTA's, from mapa) once this thread's MMAs are done.
__device__ __forceinline__ void tc_commit_remote(uint32_t cluster_addr) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            cluster_addr)
        : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// K-major operand tile with rows of bk bf16: bk = 64 -> 128-byte rows, 128-byte
// swizzle, 8-row groups 1024 B apart; bk = 32 -> 64-byte rows, 64-byte swizzle,
// 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr, int bk) {
    const uint32_t row_bytes = (uint32_t)bk * 2u;
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused here)
    d |= (uint64_t)((8u * row_bytes) >> 4) << 32;  // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)(bk == 64 ? 2 : 4) << 61;    // 128-byte / 64-byte swizzle
    return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// The MMAs of one ring stage: products R_a Y_b with a + b < P over the stage's
// NKS K=16 slices (+32 bytes along K per slice, descriptor units of 16 B),
// descriptors computed once per stage (the issuing thread must keep ahead of
// the tensor pipe).  Larger terms first, except with SMALL_FIRST (chunked
// accumulation), where the small products go first while the fresh
// accumulator is still small.  acc: accumulate flag of the first MMA.
template <int P, int NKS, bool SMALL_FIRST>
__device__ __forceinline__ void issue_stage(uint32_t d_tmem, uint32_t aA, uint32_t bytesA,
                                            uint32_t aB, uint32_t bytesB, int bk, uint32_t idesc,
                                            uint32_t acc) {
    uint64_t dA[P], dB[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        dA[p] = desc_sw(aA + (uint32_t)p * bytesA, bk);
        dB[p] = desc_sw(aB + (uint32_t)p * bytesB, bk);
    }
    if (SMALL_FIRST) {
#pragma unroll
        for (int oo = 0; oo < P; ++oo) {
            const int o = P - 1 - oo;
#pragma unroll
            for (int k = 0; k < NKS; ++k)
#pragma unroll
                for (int pa = 0; pa <= o; ++pa) {
                    umma_bf16(d_tmem, dA[pa] + 2 * k, dB[o - pa] + 2 * k, idesc, acc);
                    acc = 1u;
                }
        }
    } else {
#pragma unroll
        for (int k = 0; k < NKS; ++k)
#pragma unroll
            for (int o = 0; o < P; ++o)
#pragma unroll
                for (int pa = 0; pa <= o; ++pa) {
                    umma_bf16(d_tmem, dA[pa] + 2 * k, dB[o - pa] + 2 * k, idesc, acc);
                    acc = 1u;
                }
    }
}

#define TMEM_LD32(taddr, r)                                                                     \
    asm volatile(                                                                               \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"      \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),   \
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),           \
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),        \
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),        \
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),        \
          "=r"(r[31])                                                                           \
        : "r"(taddr))

#define TMEM_ST32(taddr, r)                                                                     \
    asm volatile(                                                                               \
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12," \
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"    \
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]),          \
        "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]),          \
        "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]),      \
        "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]),      \
        "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])                              \
        : "memory")

// Named barrier 1 (barrier 0 is __syncthreads): `count` threads of whole warps.
__device__ __forceinline__ void named_bar_arrive(uint32_t id, uint32_t count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Arrive (release, cluster scope) on the mbarrier at this shared::cluster
// address, typically one in the peer CTA (from mapa).
__device__ __forceinline__ void mbar_remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
// Bounded wait with cluster-scope acquire: what the arriving peer wrote
// before its release-arrive is visible afterwards.  False on timeout.
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Plain arrive (count 1) on a barrier of this CTA.
__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Sums over a warp's 32 lanes of 32 values at once: afterwards v[0] of lane l
// holds the sum over the lanes of the values v[l] had (31 shuffles, a
// butterfly that halves the live values at each level).
__device__ __forceinline__ void transpose_reduce32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
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
}

}  // namespace vne
