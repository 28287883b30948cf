// Learned moment correction of the low-degree Chebyshev estimator
// (Algorithm 1b, Section 3, extended by this library; the paper has none):
//   * a spectral sampler that draws the probe totals of Algorithm 1b for
//     R = Psi diag(p) Psi^T, Haar Psi and Gaussian probes g_j = Psi z_j:
//     sum_j g_j^T T_k(A) g_j = sum_i w_i T_k(x_i), w_i = sum_j z_ij^2,
//     x_i = 2 p_i / u - 1 -- training data labelled by the exact entropy of p;
//   * the network 19 -> 128 -> 128 -> 128 -> 1 (GELU hidden layers, linear
//     output), FP32: forward, backward, mean squared error and Adam, all on
//     one strided SIMT GEMM kernel plus element-wise kernels;
//   * the features of a live estimate (from the device moments) and the
//     corrected estimate H_16 + (n u / 100) net(features).
#include <cmath>
#include <utility>

#include "../../include/vne.h"
#include "vne_common.cuh"
#include "vne_internal.h"

namespace vne {

// ---------------------------------------------------------------------------
// spectral sampler: one block per spectrum
// ---------------------------------------------------------------------------
constexpr int kSampleThreads = 256;
// The network's output is c = 100 (H - H_16) / (n u): with p = u y the
// truncation error of f_m is u e_m(y), e_m that of y ln y on [0, 1], so the
// correction over n u is a mean over the distribution of y (n-independent).
constexpr double kTargetScale = 100.0;
constexpr int kSampleMaxM = 64;

__device__ __forceinline__ double block_sum_all(double v, double* red) {
    // sum over the block, returned to every thread (red: blockDim/32 doubles)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

__device__ __forceinline__ double cheb_alpha(int k, double u) {
    const double l = log(u / 4.0);
    if (k == 0) return (u / 2.0) * (l + 1.0);
    if (k == 1) return (u / 4.0) * (2.0 * l + 3.0);
    const double kk = (double)k;
    return ((k & 1) ? -u : u) / (kk * kk * kk - kk);
}

__global__ void __launch_bounds__(kSampleThreads)
k_spectral_sample(const int* __restrict__ kind, const int* __restrict__ n_arr,
                  const float* __restrict__ a_arr, const int* __restrict__ ktop_arr,
                  const float* __restrict__ floor_arr, const float* __restrict__ c_arr,
                  const uint64_t* __restrict__ seeds, int m, int s, float* __restrict__ feat,
                  float* __restrict__ target, double* __restrict__ H_exact,
                  double* __restrict__ H_low, double* __restrict__ totals) {
    __shared__ double red[kSampleThreads / 32];
    __shared__ double tot_sh[kSampleMaxM + 1][kSampleThreads / 32];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = n_arr[b], knd = kind[b], ktop = ktop_arr[b];
    const float a = a_arr[b], fl = floor_arr[b];
    const uint64_t seed = seeds[b];
    auto q = [&](int i) -> float {
        if (knd == 0) return expf(-(float)i / a);
        return (i + 1 <= ktop) ? powf((float)(i + 1), -a) : fl;
    };
    // normalisation and the exact entropy
    float part = 0.f;
    for (int i = tid; i < n; i += blockDim.x) part += q(i);
    const double S = block_sum_all((double)part, red);
    const float inv_S = (float)(1.0 / S);
    float hpart = 0.f;
    for (int i = tid; i < n; i += blockDim.x) {
        const float p = q(i) * inv_S;
        if (p > 0.f) hpart -= p * logf(p);
    }
    const double H = block_sum_all((double)hpart, red);
    const double pmax = (double)q(0) / S;
    const double u = (double)c_arr[b] * pmax;
    // probe totals sum_i w_i T_k(x_i)
    float acc[kSampleMaxM + 1];
#pragma unroll
    for (int k = 0; k <= kSampleMaxM; ++k) acc[k] = 0.f;
    const float two_over_u = (float)(2.0 / u);
    for (int i = tid; i < n; i += blockDim.x) {
        float w = 0.f;
        for (int j = 0; j < s; ++j) {
            const float z = gaussian_f32(seed, (uint64_t)j * (uint64_t)n + (uint64_t)i);
            w = fmaf(z, z, w);
        }
        const float x = fmaf(q(i) * inv_S, two_over_u, -1.f);
        float t0 = 1.f, t1 = x;
        acc[0] += w;
        if (m >= 1) acc[1] = fmaf(w, x, acc[1]);
#pragma unroll
        for (int k = 2; k <= kSampleMaxM; ++k) {
            if (k <= m) {
                const float t2 = fmaf(2.f * x, t1, -t0);
                acc[k] = fmaf(w, t2, acc[k]);
                t0 = t1;
                t1 = t2;
            }
        }
    }
#pragma unroll
    for (int k = 0; k <= kSampleMaxM; ++k) {
        if (k <= m) {
            const double v = warp_sum((double)acc[k]);
            if (lane == 0) tot_sh[k][warp] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        double hl = 0.0;
        double tot[kSampleMaxM + 1];
        for (int k = 0; k <= m; ++k) {
            double t = 0.0;
            for (int w = 0; w < kSampleThreads / 32; ++w) t += tot_sh[k][w];
            tot[k] = t;
            hl -= cheb_alpha(k, u) * t;
            if (totals) totals[(int64_t)b * (m + 1) + k] = t;
        }
        hl /= (double)s;
        const double ln_n = log((double)n);
        float* f = feat + (int64_t)b * VNE_MLP_N_IN;
        for (int k = 0; k < VNE_MLP_N_MOMENTS; ++k)
            f[k] = k <= m ? (float)(tot[k] / ((double)s * (double)n)) : 0.f;
        f[VNE_MLP_N_MOMENTS] = (float)(ln_n / 10.0);
        f[VNE_MLP_N_MOMENTS + 1] = (float)(log(pmax) / 10.0);
        f[VNE_MLP_N_MOMENTS + 2] = (float)(log(u) / 10.0);
        target[b] = (float)(kTargetScale * (H - hl) / ((double)n * u));
        H_exact[b] = H;
        H_low[b] = hl;
    }
}

cudaError_t launch_spectral_sample(int count, const int* kind, const int* n, const float* a,
                                   const int* ktop, const float* floor, const float* c,
                                   const uint64_t* seeds, int m, int s, float* feat, float* target,
                                   double* H_exact, double* H_low, double* totals,
                                   cudaStream_t st) {
    if (m < VNE_MLP_N_MOMENTS - 1 || m > kSampleMaxM) return cudaErrorInvalidValue;
    k_spectral_sample<<<count, kSampleThreads, 0, st>>>(kind, n, a, ktop, floor, c, seeds, m, s,
                                                        feat, target, H_exact, H_low, totals);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Strided FP32 GEMM: C[r][c] = act(sum_k A(r, k) B(k, c) + bias[c]) with
// A(r, k) = A[ra(r) * sam + k * sak], B(k, c) = B[rb(k) * sbk + c * sbn], where
// ra / rb are optional row gathers.  32 x 32 tiles, 256 threads, 2 x 2
// outputs per thread, the K loop in order (deterministic, no atomics).
// act: 0 identity, 1 GELU (then Z receives the pre-activation).
// ---------------------------------------------------------------------------
struct Gemm {
    const float* A;
    int64_t sam, sak;
    const int* ga;
    const float* B;
    int64_t sbk, sbn;
    const int* gb;
    float* C;
    float* Z;
    int64_t ldc;
    int M, N, K;
    const float* bias;
    int act;
};

__device__ __forceinline__ float gelu_f(float x) {
    return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) +
           x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__global__ void __launch_bounds__(256) k_gemm(Gemm g) {
    __shared__ float As[32][33];
    __shared__ float Bs[32][33];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < g.K; k0 += 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int i = e >> 5, kk = e & 31;  // A: row i, column kk
            const int r = r0 + i, k = k0 + kk;
            float va = 0.f;
            if (r < g.M && k < g.K) {
                const int64_t rr = g.ga ? g.ga[r] : r;
                va = g.A[rr * g.sam + (int64_t)k * g.sak];
            }
            As[kk][i] = va;
            const int kb = k0 + i, c = c0 + kk;  // B: row kb, column c
            float vb = 0.f;
            if (kb < g.K && c < g.N) {
                const int64_t kr = g.gb ? g.gb[kb] : kb;
                vb = g.B[kr * g.sbk + (int64_t)c * g.sbn];
            }
            Bs[i][kk] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
            const float b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + ty * 2 + i, c = c0 + tx * 2 + j;
            if (r < g.M && c < g.N) {
                float v = acc[i][j] + (g.bias ? g.bias[c] : 0.f);
                if (g.act == 1) {
                    g.Z[(int64_t)r * g.ldc + c] = v;
                    v = gelu_f(v);
                }
                g.C[(int64_t)r * g.ldc + c] = v;
            }
        }
}

static cudaError_t gemm(const Gemm& g, cudaStream_t st) {
    dim3 grid((unsigned)((g.N + 31) / 32), (unsigned)((g.M + 31) / 32));
    k_gemm<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
}

// dZ = dA * act'(Z) (GELU layers)
__global__ void k_gelu_bwd(const float* __restrict__ dA, const float* __restrict__ Z,
                           float* __restrict__ dZ, int64_t len) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x)
        dZ[e] = dA[e] * gelu_grad_f(Z[e]);
}

// db[c] = sum_r dZ[r][c] (rows in order, one thread per column)
__global__ void k_colsum(const float* __restrict__ dZ, int rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float t = 0.f;
    for (int r = 0; r < rows; ++r) t += dZ[(int64_t)r * cols + c];
    db[c] = t;
}

// loss = mean (y - t)^2 (FP64 sum), dy = 2 (y - t) / B; targets gathered by idx.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t,
                      const int* __restrict__ idx, int B, float* __restrict__ dy,
                      double* __restrict__ loss) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const float d = y[i] - t[idx ? idx[i] : i];
        dy[i] = 2.f * d / (float)B;
        acc += (double)d * (double)d;
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) *loss = tot / (double)B;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int len, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    th[e] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// rows of the batch: idx[i] = (a * (first + i) + c) mod rows (a coprime to rows)
__global__ void k_batch_rows(int* __restrict__ idx, int B, int64_t first, int64_t rows, int64_t a,
                             int64_t c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int64_t k = (first + i) % rows;
    idx[i] = (int)((a % rows * k + c) % rows);
}

// ---------------------------------------------------------------------------
// network passes
// ---------------------------------------------------------------------------
static const int kIn[4] = {VNE_MLP_N_IN, VNE_MLP_N_HIDDEN, VNE_MLP_N_HIDDEN, VNE_MLP_N_HIDDEN};
static const int kOut[4] = {VNE_MLP_N_HIDDEN, VNE_MLP_N_HIDDEN, VNE_MLP_N_HIDDEN, 1};

static int64_t w_off(int l) {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)kIn[i] * kOut[i] + kOut[i];
    return o;
}

size_t mlp_workspace_floats(int B) {
    // Z and A of the 4 layers, two B x 128 backward buffers
    return (size_t)B * (3 * 2 * VNE_MLP_N_HIDDEN + 2) + (size_t)2 * B * VNE_MLP_N_HIDDEN + 64;
}

struct MlpBuffers {
    float* Z[4];
    float* A[4];
    float* d0;
    float* d1;
};

static MlpBuffers carve(float* ws, int B) {
    MlpBuffers m;
    float* p = ws;
    for (int l = 0; l < 4; ++l) {
        m.Z[l] = p;
        p += (size_t)B * kOut[l];
        m.A[l] = p;
        p += (size_t)B * kOut[l];
    }
    m.d0 = p;
    p += (size_t)B * VNE_MLP_N_HIDDEN;
    m.d1 = p;
    return m;
}

static cudaError_t mlp_fwd(const float* th, const float* X, int64_t ldx, const int* rows, int B,
                           MlpBuffers& mb, int* launches, cudaStream_t st) {
    const float* in = X;
    int64_t ldi = ldx;
    const int* gi = rows;
    for (int l = 0; l < 4; ++l) {
        Gemm g{};
        g.A = in;
        g.sam = ldi;
        g.sak = 1;
        g.ga = gi;
        g.B = th + w_off(l);
        g.sbk = 1;
        g.sbn = kIn[l];
        g.C = mb.A[l];
        g.Z = mb.Z[l];
        g.ldc = kOut[l];
        g.M = B;
        g.N = kOut[l];
        g.K = kIn[l];
        g.bias = th + w_off(l) + (int64_t)kIn[l] * kOut[l];
        g.act = l < 3 ? 1 : 0;
        cudaError_t e = gemm(g, st);
        ++*launches;
        if (e != cudaSuccess) return e;
        in = mb.A[l];
        ldi = kOut[l];
        gi = nullptr;
    }
    return cudaSuccess;
}

cudaError_t mlp_forward(const float* th, const float* X, int B, float* y, float* ws, int* launches,
                        cudaStream_t st) {
    MlpBuffers mb = carve(ws, B);
    cudaError_t e = mlp_fwd(th, X, VNE_MLP_N_IN, nullptr, B, mb, launches, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(y, mb.A[3], (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, st);
}

// Loss and gradient (grad: VNE_MLP_N_PARAMS floats) of a batch whose rows of
// X / targets are idx[0..B) (or 0..B-1 when idx is NULL).
cudaError_t mlp_loss_grad(const float* th, const float* X, const float* t, const int* idx, int B,
                          float* grad, double* loss, float* ws, int* launches, cudaStream_t st) {
    MlpBuffers mb = carve(ws, B);
    cudaError_t e = mlp_fwd(th, X, VNE_MLP_N_IN, idx, B, mb, launches, st);
    if (e != cudaSuccess) return e;
    float* dA = mb.d0;  // gradient w.r.t. the current layer's output
    float* dZ = mb.d1;
    k_mse<<<1, 256, 0, st>>>(mb.A[3], t, idx, B, dA, loss);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = 3; l >= 0; --l) {
        const int I = kIn[l], O = kOut[l];
        const float* dz = dA;
        if (l < 3) {
            const int64_t len = (int64_t)B * O;
            k_gelu_bwd<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(dA, mb.Z[l], dZ, len);
            ++*launches;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            dz = dZ;
        }
        const float* in = l == 0 ? X : mb.A[l - 1];
        const int64_t ldi = l == 0 ? VNE_MLP_N_IN : kIn[l];
        const int* gi = l == 0 ? idx : nullptr;
        // dW = dz^T in  (O x I, reduction over the batch)
        Gemm gw{};
        gw.A = dz;
        gw.sam = 1;
        gw.sak = O;
        gw.B = in;
        gw.sbk = ldi;
        gw.sbn = 1;
        gw.gb = gi;
        gw.C = grad + w_off(l);
        gw.ldc = I;
        gw.M = O;
        gw.N = I;
        gw.K = B;
        if ((e = gemm(gw, st)) != cudaSuccess) return e;
        ++*launches;
        k_colsum<<<(O + 127) / 128, 128, 0, st>>>(dz, B, O, grad + w_off(l) + (int64_t)I * O);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l > 0) {
            // dA_prev = dz W  (B x I)
            Gemm gx{};
            gx.A = dz;
            gx.sam = O;
            gx.sak = 1;
            gx.B = th + w_off(l);
            gx.sbk = I;
            gx.sbn = 1;
            gx.C = (dz == dA) ? dZ : dA;
            gx.ldc = I;
            gx.M = B;
            gx.N = I;
            gx.K = O;
            if ((e = gemm(gx, st)) != cudaSuccess) return e;
            ++*launches;
            if (gx.C == dZ) std::swap(dA, dZ);  // dA now holds the new gradient
        }
    }
    return cudaSuccess;
}

cudaError_t mlp_train_step(float* th, float* am, float* av, int step, float lr, const float* X,
                           const float* t, int64_t rows, int B, int64_t first, uint64_t perm_seed,
                           int* idx, float* grad, double* loss, float* ws, int* launches,
                           cudaStream_t st) {
    // a multiplier coprime to `rows` drawn from the seed
    int64_t a = (int64_t)(splitmix_out(perm_seed, 0) % (uint64_t)rows) | 1;
    auto gcd = [](int64_t x, int64_t y) {
        while (y) {
            const int64_t r = x % y;
            x = y;
            y = r;
        }
        return x;
    };
    while (gcd(a, rows) != 1) a = (a + 2) % rows ? (a + 2) % rows : 1;
    const int64_t c = (int64_t)(splitmix_out(perm_seed, 1) % (uint64_t)rows);
    k_batch_rows<<<(B + 255) / 256, 256, 0, st>>>(idx, B, first, rows, a, c);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = mlp_loss_grad(th, X, t, idx, B, grad, loss, ws, launches, st)) != cudaSuccess) return e;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, step)));
    k_adam<<<(VNE_MLP_N_PARAMS + 255) / 256, 256, 0, st>>>(th, grad, am, av, VNE_MLP_N_PARAMS, lr,
                                                           b1, b2, 1e-8f, c1, c2);
    ++*launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// live estimate: features from the device moments, corrected estimate
// ---------------------------------------------------------------------------
// mom: (m+1) x s per-probe moments [k][j]; sc: the call's scalar block.
__global__ void k_learned_features(const double* __restrict__ mom, int m, int s, int64_t n,
                                   const double* __restrict__ sc, float* __restrict__ f) {
    const int k = threadIdx.x;
    if (k < VNE_MLP_N_MOMENTS) {
        double t = 0.0;
        if (k <= m)
            for (int j = 0; j < s; ++j) t += mom[(int64_t)k * s + j];
        f[k] = (float)(t / ((double)s * (double)n));
    }
    if (k == 0) {
        const double u = sc[SC_U];
        const double lam = sc[SC_LAM] > 0.0 ? sc[SC_LAM] : u;
        f[VNE_MLP_N_MOMENTS] = (float)(log((double)n) / 10.0);
        f[VNE_MLP_N_MOMENTS + 1] = (float)(log(lam) / 10.0);
        f[VNE_MLP_N_MOMENTS + 2] = (float)(log(u) / 10.0);
    }
}

__global__ void k_learned_finish(const float* __restrict__ y, int64_t n, double* __restrict__ sc) {
    const double H = sc[SC_H_CHEB] + (double)y[0] * (double)n * sc[SC_U] / kTargetScale;
    sc[SC_H_LEARNED] = H;
    if (!isfinite(H)) {
        unsigned long long* fl = reinterpret_cast<unsigned long long*>(sc + SC_FLAGS);
        *fl |= FLAG_NONFINITE;
    }
}

cudaError_t launch_learned(const double* mom, int m, int s, int64_t n, double* sc,
                           const float* params, float* ws, int* launches, cudaStream_t st) {
    float* f = ws;
    float* y = ws + 32;
    float* mws = ws + 64;
    k_learned_features<<<1, 32, 0, st>>>(mom, m, s, n, sc, f);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = mlp_forward(params, f, 1, y, mws, launches, st)) != cudaSuccess) return e;
    k_learned_finish<<<1, 1, 0, st>>>(y, n, sc);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace vne
