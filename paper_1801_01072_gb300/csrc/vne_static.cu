// Allocation-free power method: vne_lambda_max_static.
//
// Some callers cannot allocate device memory at the point where they need
// the largest eigenvalue: code that runs while a custom allocator forbids
// new allocations, plug-ins of host applications that own the whole device
// memory budget, or real-time loops where cudaMalloc's implicit device
// synchronisation is not acceptable.  This entry point serves them: it runs
// the same power-method kernels as vne_lambda_max, but its scratch memory
// (iterates, block partials, the reduction counter and the scalar block) is
// a fixed file-scope device array, so it calls no cudaMalloc, cudaFree or
// allocating library routine, and needs no handle.
//
// The array costs every GPU that loads the library VNE_STATIC_SCRATCH_BYTES
// of device memory until the process exits.  All calls on one device share
// it and it keeps the last call's contents; the call clears what must start
// at zero.  Calls whose work overlaps on the GPU (other streams, other host
// threads) race on the array: serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/vne.h"
#include "vne_common.cuh"
#include "vne_internal.h"

namespace {

constexpr int kMaxBlocks = 2048;        // power-method blocks (partials rows): >= 8 per SM
constexpr int kMaxTrials = 8;           // q
constexpr int64_t kSc = vne::SC_COUNT;  // doubles
constexpr int64_t kCounter = 32;        // doubles (64 unsigned counters)
constexpr int64_t kPartials = (int64_t)kMaxBlocks * 3 * kMaxTrials;
constexpr int64_t kVec = VNE_STATIC_MAX_VECTOR_ELEMS;
constexpr int64_t kTotal = kSc + kCounter + kPartials + 2 * kVec;  // doubles

static_assert(kTotal * 8 <= VNE_STATIC_SCRATCH_BYTES, "scratch size");

// The scratch itself.  In host code `g_scratch` is only a stand-in symbol,
// not a device address: its address must come from cudaGetSymbolAddress.
static __device__ __align__(256) double g_scratch[VNE_STATIC_SCRATCH_BYTES / 8];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};
void* g_ctx[kMaxDevices] = {};  // the context the address belongs to
int g_sms[kMaxDevices] = {};

// The calling thread's current driver context (cuCtxGetCurrent, reached
// through the runtime's entry-point query, so no driver library is linked).
void* current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
        looked = true;
    }
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Once per device, with that device current: the device address of the array.
// The address belongs to the device's context, so it is cached with that
// context; a thread with no current context yet, or a context that is not
// the cached one (after a device reset the primary context is a new one),
// runs the look-up again (cudaGetSymbolAddress also makes the device's
// primary context current).
vne_status setup(int dev, double** base, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return VNE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    void* ctx = current_context();
    if (!g_ptr[dev] || !ctx || ctx != g_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return VNE_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return VNE_ERR_CUDA;
        }
        g_ptr[dev] = p;
        g_ctx[dev] = current_context();
        g_sms[dev] = n;
    }
    *base = static_cast<double*>(g_ptr[dev]);
    *sms = g_sms[dev];
    return VNE_OK;
}

}  // namespace

extern "C" vne_status vne_lambda_max_static(const vne_matrix* R, const vne_params* p,
                                            double* lam_out, void* stream) {
    if (!R || !p || !lam_out) return VNE_ERR_INVALID_ARG;
    if (R->n < 1 || !R->data || R->ld < R->n) return VNE_ERR_INVALID_ARG;
    if (R->layout != VNE_DENSE && R->layout != VNE_DIA) return VNE_ERR_INVALID_ARG;
    if (R->dtype != VNE_F64 && R->dtype != VNE_F32) return VNE_ERR_INVALID_ARG;
    if (p->power_iters < 1 || p->power_trials < 1 || p->power_trials > kMaxTrials)
        return VNE_ERR_INVALID_ARG;
    // no staging copies here: R must be on the device and stored in the
    // precision that is computed in (F64 with FP64, F32 with FP32)
    if (R->memory != VNE_MEM_DEVICE) return VNE_ERR_UNSUPPORTED;
    if (p->precision != VNE_PREC_F64 && p->precision != VNE_PREC_F32) return VNE_ERR_UNSUPPORTED;
    const bool f64 = p->precision == VNE_PREC_F64;
    if ((R->dtype == VNE_F64) != f64) return VNE_ERR_UNSUPPORTED;
    if (R->layout == VNE_DIA && R->n_diags < 1) return VNE_ERR_INVALID_ARG;
    if (R->layout == VNE_DIA && vne::dia_supported_halfbw(R->n_diags) < 0)
        return VNE_ERR_UNSUPPORTED;
    const int q = p->power_trials;
    if (R->n * (int64_t)q > kVec) return VNE_ERR_UNSUPPORTED;  // beyond the fixed scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VNE_ERR_CUDA;
    }
    double* base = nullptr;
    int sms = 0;
    vne_status vs = setup(dev, &base, &sms);
    if (vs != VNE_OK) return vs;

    cudaStream_t st = (cudaStream_t)stream;
    double* sc = base;
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + kSc);
    double* partial = base + kSc + kCounter;
    double* x0 = partial + kPartials;
    double* x1 = x0 + kVec;
    const int64_t n = R->n;
    const bool dense = R->layout == VNE_DENSE;
    // the block counts of vne_lambda_max, so both sum the same partials in the same order
    int blocks = dense ? (int)std::min<int64_t>((n + 7) / 8, 8 * (int64_t)sms) : 4 * sms;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    const double u_scale = p->u_scale > 0.0 ? p->u_scale : 1.0;

    // what must start at zero: the scalar block and the reduction counter
    cudaError_t e = cudaMemsetAsync(sc, 0, (size_t)(kSc + kCounter) * sizeof(double), st);
    if (e == cudaSuccess)
        e = f64 ? vne::launch_power_init<double>(x0, n, q, p->seed, sc, st)
                : vne::launch_power_init<float>(reinterpret_cast<float*>(x0), n, q, p->seed, sc, st);
    void* xa = x0;
    void* xb = x1;
    for (int it = 0; it <= p->power_iters && e == cudaSuccess; ++it) {
        const int fin = it == p->power_iters;
        if (dense)
            e = vne::launch_power_step_dense(R->data, f64 ? 0 : 1, n, R->ld, xa, xb, f64, q, sc,
                                             partial, counter, fin, u_scale, blocks, st);
        else
            e = vne::launch_power_step_dia(R->data, f64 ? 0 : 1, n, R->ld, R->n_diags, xa, xb, q,
                                           sc, partial, counter, fin, u_scale, blocks, st);
        void* tmp = xa;
        xa = xb;
        xb = tmp;
    }
    double out[vne::SC_FLAGS + 1];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, sc, sizeof(out), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? VNE_ERR_OOM : VNE_ERR_CUDA;
    }
    unsigned long long flags;
    memcpy(&flags, &out[vne::SC_FLAGS], sizeof(flags));
    // the statuses of vne_lambda_max, in its order
    if (flags & vne::FLAG_TIMEOUT) return VNE_ERR_TIMEOUT;
    if (flags & vne::FLAG_BAD_INTERVAL) return VNE_ERR_BAD_INTERVAL;
    if (flags & vne::FLAG_NONFINITE) return VNE_ERR_NONFINITE;
    if (!std::isfinite(out[vne::SC_LAM])) return VNE_ERR_NONFINITE;
    *lam_out = out[vne::SC_LAM];
    return VNE_OK;
}
