// Final FP64 combination of the per-probe moments.
//
//   Chebyshev (Algorithm 1b): H = -(1/s) sum_j sum_{k=0}^m alpha_k mu[k, j],
//     alpha_0 = (u/2)(ln(u/4) + 1), alpha_1 = (u/4)(2 ln(u/4) + 3),
//     alpha_k = (-1)^k u / (k^3 - k), k >= 2          (Lemma lem:prior)
//   Taylor (Algorithm 1a):    H = ln(1/u) + (1/s) sum_j sum_{k=1}^m tau[k, j] / k
//
// The moment sums over row tiles are taken in tile order (deterministic).
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

__global__ void k_combine_moments(Partials P, int s, int m, int cheb_c0, int tay_c0,
                                  double* mom_cheb, double* mom_taylor) {
    const int per = (m + 1) * s;
    const int total = (cheb_c0 >= 0 ? per : 0) + (tay_c0 >= 0 ? per : 0);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const bool cheb = (cheb_c0 >= 0) && e < per;
        const int r = cheb ? e : (cheb_c0 >= 0 ? e - per : e);
        const int k = r / s, j = r - k * s;
        const int slot = cheb ? k : k + 1;
        const int col = (cheb ? cheb_c0 : tay_c0) + j;
        const int nt = slot == 0 ? P.ntiles0 : P.ntiles;
        const double* base = P.slot(slot);
        double acc = 0.0;
        for (int tile = 0; tile < nt; ++tile) acc += base[(size_t)tile * P.S + col];
        (cheb ? mom_cheb : mom_taylor)[r] = acc;
    }
}

__device__ double cheb_alpha(int k, double u) {
    if (k == 0) return (u / 2.0) * (log(u / 4.0) + 1.0);
    if (k == 1) return (u / 4.0) * (2.0 * log(u / 4.0) + 3.0);
    const double kk = (double)k;
    return ((k & 1) ? -u : u) / (kk * kk * kk - kk);
}

// One warp per moment index k (k = warp, warp + nwarps, ...): lanes sum the
// s probes, lane 0 folds alpha_k (or 1/k) in; warps are then summed in order.
__global__ void k_combine_final(int s, int m, int cheb, int taylor, const double* mom_cheb,
                                const double* mom_taylor, double* sc) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double u = sc[SC_U];
    if (cheb) {
        double acc = 0.0;
        for (int k = w; k <= m; k += nw) {
            double sk = 0.0;
            for (int j = lane; j < s; j += 32) sk += mom_cheb[(size_t)k * s + j];
            sk = warp_sum(sk);
            if (lane == 0) acc += cheb_alpha(k, u) * sk;
        }
        const double tot = block_sum(lane == 0 ? acc : 0.0, sh);
        if (threadIdx.x == 0) sc[SC_H_CHEB] = -tot / (double)s;
    }
    if (taylor) {
        double acc = 0.0;
        for (int k = 1 + w; k <= m; k += nw) {
            double sk = 0.0;
            for (int j = lane; j < s; j += 32) sk += mom_taylor[(size_t)k * s + j];
            sk = warp_sum(sk);
            if (lane == 0) acc += sk / (double)k;
        }
        const double tot = block_sum(lane == 0 ? acc : 0.0, sh);
        if (threadIdx.x == 0) sc[SC_H_TAYLOR] = log(1.0 / u) + tot / (double)s;
    }
    if (threadIdx.x == 0) {
        bool bad = false;
        if (cheb && !isfinite(sc[SC_H_CHEB])) bad = true;
        if (taylor && !isfinite(sc[SC_H_TAYLOR])) bad = true;
        if (bad) {
            unsigned long long* f = (unsigned long long*)&sc[SC_FLAGS];
            *f |= FLAG_NONFINITE;
        }
    }
}

cudaError_t launch_combine_final(int s, int m, const double* mom_cheb, const double* mom_taylor,
                                 double* sc, cudaStream_t st) {
    k_combine_final<<<1, 256, 0, st>>>(s, m, mom_cheb != nullptr, mom_taylor != nullptr, mom_cheb,
                                       mom_taylor, sc);
    return cudaGetLastError();
}

cudaError_t launch_combine(Partials P, int s, int m, int cheb_c0, int tay_c0, double* mom_cheb,
                           double* mom_taylor, double* sc, cudaStream_t st) {
    const int per = (m + 1) * s;
    const int total = (cheb_c0 >= 0 ? per : 0) + (tay_c0 >= 0 ? per : 0);
    int blocks = (total + 255) / 256;
    if (blocks < 1) blocks = 1;
    k_combine_moments<<<blocks, 256, 0, st>>>(P, s, m, cheb_c0, tay_c0, mom_cheb, mom_taylor);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_combine_final<<<1, 256, 0, st>>>(s, m, cheb_c0 >= 0, tay_c0 >= 0, mom_cheb, mom_taylor, sc);
    return cudaGetLastError();
}

}  // namespace vne
