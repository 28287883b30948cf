// Host runtime behind the C ABI of include/vne.h: argument checks, the
// workspace, and the launch sequence of one estimator call
//   [H2D copy] -> [trace] -> operand prep -> power method (Appendix A) ->
//   probes -> m (or m+1) recurrence steps -> FP64 combine -> D2H of scalars.
// Every arithmetic step is a kernel of this library; the host only sequences.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <mutex>
#include <vector>

#include "../../include/vne.h"
#include "vne_common.cuh"
#include "vne_internal.h"

using namespace vne;

struct ProfEvent {
    int kind;
    int count;  // launches between the two events
    cudaEvent_t a, b;
};

struct vne_handle {
    int device = 0;
    int sm_count = 0;
    int32_t last_err = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    double* host_sc = nullptr;  // pinned
    int prof_on = 0;
    double prof_ms[4] = {0, 0, 0, 0};
    int64_t prof_n[4] = {0, 0, 0, 0};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfEvent> pending;
    int64_t launches = 0;
    // batched calls
    char* bws = nullptr;
    size_t bws_bytes = 0;
    double* bhost = nullptr;
    size_t bhost_count = 0;
    std::vector<cudaStream_t> bstreams;
    std::vector<cudaEvent_t> bevents;  // [0] fork, [1] done, [2 + k] join of stream k
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_key = 0;
    // the persistent recurrence of a batch: its table, pinned and on the device
    char* btab_dev = nullptr;
    char* btab_host = nullptr;
    size_t btab_bytes = 0;
    // sequences of host-resident matrices: two device slots, one filled by
    // the copy stream while the matrix in the other is estimated
    char* stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    cudaStream_t cstream = nullptr;
    cudaEvent_t cev[2] = {nullptr, nullptr};
};

namespace {

enum Mode { MODE_CHEB = 1, MODE_TAYLOR = 2, MODE_BOTH = 3, MODE_POWER = 4 };

struct Outputs {
    double* H_cheb = nullptr;
    double* H_taylor = nullptr;
    double* mom_cheb = nullptr;
    double* mom_taylor = nullptr;
    double* u = nullptr;
    double* lam = nullptr;
    const float* mlp = nullptr;      // trained correction network (device), or NULL
    double* H_learned = nullptr;
    // batched calls: measure the workspace only, or enqueue into a given
    // workspace and pinned host slot without synchronising
    int measure = 0;
    // batched persistent recurrence: phase 1 enqueues the prologue (operands,
    // power method, probe block) and records the step buffers in *bmat;
    // phase 2 enqueues the combine on the same workspace after the steps ran
    int phase = 0;
    TcBatchMat* bmat = nullptr;
    int batch_power = 0;  // phase 1: leave the power products to the batch's launch
    size_t* measured = nullptr;
    char* ws = nullptr;
    double* host_slot = nullptr;
    // explicit probes (device, n x s row-major, FP64 for F64 precision, else
    // FP32), replacing the seed's stream
    const void* probes = nullptr;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Two-pass bump allocator: pass 1 (base == nullptr) only measures.
struct Bump {
    char* base;
    size_t off = 0;
    explicit Bump(char* b) : base(b) {}
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T) + 16;
        return p;
    }
};

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

struct Call {
    vne_handle* h;
    cudaStream_t st;
    cudaError_t err = cudaSuccess;
    bool ok() const { return err == cudaSuccess; }
    void chk(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    void launched(cudaError_t e) {
        h->launches++;
        chk(e);
    }
    // profiling bracket around one launch of kernel class `kind`
    cudaEvent_t ev() {
        if (h->ev_used == h->ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            h->ev_pool.push_back(e);
        }
        return h->ev_pool[h->ev_used++];
    }
    cudaEvent_t pa = nullptr;
    void prof_begin() {
        pa = nullptr;
        if (!h->prof_on) return;
        pa = ev();
        if (pa) cudaEventRecord(pa, st);
    }
    void prof_end(int kind, int count = 1) {
        if (!h->prof_on || !pa) return;
        cudaEvent_t b = ev();
        if (!b) return;
        cudaEventRecord(b, st);
        h->pending.push_back({kind, count, pa, b});
    }
};

}  // namespace

cudaError_t vne::set_max_dynamic_smem(const void* kernel, int bytes) {
    struct Entry {
        const void* fn;
        int dev, bytes;
    };
    static std::mutex mu;
    static std::vector<Entry> table;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& x : table)
        if (x.fn == kernel && x.dev == dev && x.bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) table.push_back({kernel, dev, bytes});
    return e;
}

namespace {

vne_status map_err(vne_handle* h, cudaError_t e) {
    if (e == cudaSuccess) return VNE_OK;
    h->last_err = (int32_t)e;
    if (e == cudaErrorMemoryAllocation) return VNE_ERR_OOM;
    return VNE_ERR_CUDA;
}

vne_status ensure_ws(vne_handle* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return VNE_OK;
    if (h->ws) {
        cudaDeviceSynchronize();
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc((void**)&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        e = cudaMalloc((void**)&h->ws, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->ws = nullptr;
            h->last_err = (int32_t)e;
            return VNE_ERR_OOM;
        }
        want = bytes;
    }
    h->ws_bytes = want;
    return VNE_OK;
}

size_t elt_size(int dtype) {
    return dtype == VNE_C128 ? 16 : (dtype == VNE_F64 || dtype == VNE_C64) ? 8 : 4;
}
bool is_complex(int dtype) { return dtype == VNE_C128 || dtype == VNE_C64; }

// Adds the event pairs recorded during a finished call to the per-kind totals.
void collect_profile(vne_handle* h) {
    for (const ProfEvent& pe : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            h->prof_ms[pe.kind] += ms;
            h->prof_n[pe.kind] += pe.count;
        }
    }
    h->pending.clear();
}

// Status of a finished call from its scalar block (copied to the host).
vne_status slot_status(const double* hs, int check_trace) {
    uint64_t flags;
    std::memcpy(&flags, &hs[SC_FLAGS], sizeof(flags));
    if (check_trace && !(std::fabs(hs[SC_TRACE] - 1.0) <= 1e-6)) return VNE_ERR_NOT_UNIT_TRACE;
    if (flags & FLAG_TIMEOUT) return VNE_ERR_TIMEOUT;
    if (flags & FLAG_BAD_INTERVAL) return VNE_ERR_BAD_INTERVAL;
    if (flags & FLAG_NONFINITE) return VNE_ERR_NONFINITE;
    return VNE_OK;
}

// The persistent power method (VNE_POWER_SYM=0: one launch per product).
bool power_sym_enabled() {
    static int env = -1;
    if (env < 0) {
        const char* e = getenv("VNE_POWER_SYM");
        env = (e && e[0] == '0') ? 0 : 1;
    }
    return env != 0;
}

// Its single-launch form needs cooperative launches (every CTA resident).
bool coop_launch_ok(const vne_handle* h) {
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return coop != 0;
}

vne_status validate(const vne_matrix* R, const vne_params* p, int mode) {
    if (!R || !p) return VNE_ERR_INVALID_ARG;
    if (R->n < 1 || !R->data) return VNE_ERR_INVALID_ARG;
    if (R->layout != VNE_DENSE && R->layout != VNE_DIA && R->layout != VNE_DENSE_UPPER)
        return VNE_ERR_INVALID_ARG;
    if (R->dtype != VNE_F64 && R->dtype != VNE_F32 && !is_complex(R->dtype))
        return VNE_ERR_INVALID_ARG;
    if (R->memory != VNE_MEM_DEVICE && R->memory != VNE_MEM_HOST) return VNE_ERR_INVALID_ARG;
    if (R->ld < R->n) return VNE_ERR_INVALID_ARG;
    if (is_complex(R->dtype) && R->layout != VNE_DENSE) return VNE_ERR_UNSUPPORTED;
    if (R->layout == VNE_DIA) {
        if (R->n_diags < 1) return VNE_ERR_INVALID_ARG;
        if (dia_supported_halfbw(R->n_diags) < 0) return VNE_ERR_UNSUPPORTED;
    }
    if (p->precision < VNE_PREC_F64 || p->precision > VNE_PREC_BF16X6) return VNE_ERR_INVALID_ARG;
    if (p->probe != VNE_RADEMACHER && p->probe != VNE_GAUSSIAN) return VNE_ERR_INVALID_ARG;
    // u_override > 0 replaces the power method; u must lie in (0, 1] (Algorithms 1a/1b step 3)
    if (std::isnan(p->u_override) || std::isinf(p->u_override) || p->u_override > 1.0)
        return VNE_ERR_BAD_INTERVAL;
    if (!(p->u_scale >= 0.0) || std::isinf(p->u_scale)) return VNE_ERR_INVALID_ARG;
    if (p->u_override <= 0.0) {
        if (p->power_iters < 1 || p->power_trials < 1 || p->power_trials > 8)
            return VNE_ERR_INVALID_ARG;
    }
    if (mode != MODE_POWER) {
        if (p->m < 1 || p->s < 1) return VNE_ERR_INVALID_ARG;
        // probe counters (j0 + j) n + i, doubled for the Gaussian pairs, stay below 2^63
        if (p->probe_offset < 0 || p->probe_offset > ((int64_t)1 << 40) ||
            (double)(p->probe_offset + p->s) * (double)R->n * 2.0 > 9.0e18)
            return VNE_ERR_INVALID_ARG;
        if (p->m > 100000) return VNE_ERR_INVALID_ARG;
        const int S = (mode == MODE_BOTH) ? 2 * p->s : p->s;
        if (R->layout == VNE_DIA) {
            if (p->precision > VNE_PREC_F32) return VNE_ERR_UNSUPPORTED;
            if (p->s > 256 || S > 256) return VNE_ERR_UNSUPPORTED;
        } else if (p->precision >= VNE_PREC_BF16) {
            if (S > 512) return VNE_ERR_UNSUPPORTED;
        }
        if ((int64_t)S * R->n > ((int64_t)1 << 40)) return VNE_ERR_UNSUPPORTED;
    } else {
        if (R->layout == VNE_DIA && p->precision > VNE_PREC_F32) return VNE_ERR_UNSUPPORTED;
    }
    return VNE_OK;
}

// ---------------------------------------------------------------------------
// One estimator call.
// ---------------------------------------------------------------------------
vne_status run(vne_handle* h, const vne_matrix* Rin, const vne_params* p, int mode, Outputs out,
               void* stream) {
    if (!h) return VNE_ERR_INVALID_ARG;
    vne_status vs = validate(Rin, p, mode);
    if (vs != VNE_OK) return vs;
    DeviceGuard guard(h->device);
    Call c{h, (cudaStream_t)stream};

    const vne_matrix R = *Rin;
    // A Hermitian R (complex dtype, Section 4) runs as its real 2n x 2n
    // embedding [[B, -C], [C, B]] with probes [g; 0] and u = 1 unless given.
    const bool cplx = is_complex(R.dtype);
    const int64_t n = cplx ? 2 * R.n : R.n;
    // VNE_DENSE_UPPER runs as VNE_DENSE on a full copy mirrored from its upper triangle
    const bool upper = R.layout == VNE_DENSE_UPPER;
    const bool dense = R.layout != VNE_DIA;
    const int prec = p->precision;
    const bool tc = dense && prec >= VNE_PREC_BF16;
    // bf16 pieces of R and Y on the tensor-core path: 1 (BF16), 2 (bf16x3), 3 (bf16x6)
    const int pieces = !tc ? 0 : prec == VNE_PREC_BF16 ? 1 : prec == VNE_PREC_BF16X3 ? 2 : 3;
    const bool f64 = prec == VNE_PREC_F64;
    const bool has_cheb = mode == MODE_CHEB || mode == MODE_BOTH;
    const bool has_tay = mode == MODE_TAYLOR || mode == MODE_BOTH;
    const int s = mode == MODE_POWER ? 1 : p->s;
    const int m = mode == MODE_POWER ? 0 : p->m;
    const int S = mode == MODE_BOTH ? 2 * s : s;
    const int q = p->power_trials < 1 ? 1 : p->power_trials;
    const bool do_power = !(p->u_override > 0.0) && (!cplx || mode == MODE_POWER);
    const double u_scale = p->u_scale > 0.0 ? p->u_scale : 1.0;
    const int T_steps = mode == MODE_POWER ? 0 : (has_tay ? m + 1 : m);
    const int D = dense ? 0 : R.n_diags;
    // probes drawn from the seed's stream, or the caller's block
    const int pkind = out.probes ? PROBE_GIVEN : p->probe;

    // geometry of each path
    const int64_t rows_pad = tc ? round_up(n, tc_tile_m()) : n;
    const int64_t ldk = tc ? round_up(n, tc_tile_k()) : n;
    const int S_pad = (int)round_up(S, 32);
    int splitk = 1, ntiles = 1, ntiles0 = 1, dia_grid = 0;
    // The banded operand is the caller's band when its type is the computed
    // one (or the device copy of a host band, whose rows keep the caller's
    // ld), else a converted copy with ld = n; the bulk-copy step needs each
    // diagonal to start on a 16-byte boundary.
    int dia_band_aligned = 0;
    if (!dense) {
        const bool same_type = R.dtype == (f64 ? VNE_F64 : VNE_F32);
        const int64_t ld_op = same_type ? R.ld : n;
        const bool base_ok = !same_type || R.memory == VNE_MEM_HOST ||
                             ((uintptr_t)R.data & 15) == 0;
        dia_band_aligned = (base_ok && (ld_op * (f64 ? 8 : 4)) % 16 == 0) ? 1 : 0;
    }
    int rows_per_tile0 = 256;
    if (mode != MODE_POWER) {
        if (dense && !tc) {
            splitk = dense_simt_splitk(n, S, h->sm_count, f64 ? 8 : 4);
            ntiles = ntiles0 = (int)((n + 255) / 256);
        } else if (tc) {
            rows_per_tile0 = tc_tile_m();
            ntiles = ntiles0 = (int)(rows_pad / tc_tile_m());
        } else {
            dia_grid = dia_step_grid(f64, D, n, S, s, h->sm_count, dia_band_aligned);
            if (dia_grid < 1) return VNE_ERR_UNSUPPORTED;
            ntiles = dia_grid;
            rows_per_tile0 = 4096;
            ntiles0 = (int)((n + rows_per_tile0 - 1) / rows_per_tile0);
        }
    }
    const int power_blocks = dense ? (int)std::min<int64_t>((n + 7) / 8, 8 * h->sm_count)
                                   : 4 * h->sm_count;
    // Arithmetic of the power-method products (dense): the FP64/FP32 paths use
    // their own; BF16 uses bf16 R.  The split modes (bf16x3, bf16x6) use
    // R_0 + R_1 (16 significant bits, exact FP32 sums) in the persistent
    // kernel, else R in its input precision (FP64 for an FP64 R; the FP32
    // embedding of a complex R), so that u does not carry bf16 rounding.
    int pw_rdt;  // 0 FP64 R, 1 FP32 R, 2 bf16 pieces
    if (!tc) pw_rdt = f64 ? 0 : 1;
    else if (pieces == 1) pw_rdt = 2;
    else pw_rdt = (!cplx && R.dtype == VNE_F64) ? 0 : 1;
    // bf16 pieces, one trial: the products over the upper triangle, in one
    // persistent launch for a single call, phase by phase (plain launches on a
    // quarter of the SMs, the same bits) in a batched call, which shares the
    // GPU with the calls on its other streams
    const bool sym_phased = out.ws != nullptr || out.measure || !coop_launch_ok(h);
    const int sym_grid = sym_phased ? std::max(1, h->sm_count / 4) : h->sm_count;
    const bool use_sym = do_power && dense && tc && q == 1 && n >= 2048 &&
                         power_sym_fits(rows_pad, sym_grid) && power_sym_enabled();
    const int sym_pieces = pieces >= 2 ? 2 : 1;
    if (use_sym) pw_rdt = 2;
    const int pw_xdouble = dense ? (pw_rdt == 0 ? 1 : 0) : (f64 ? 1 : 0);

    // ---- workspace plan (two passes) ----
    const size_t vt = f64 ? 8 : 4;  // master / operand element size of SIMT & DIA paths
    auto plan = [&](Bump& b, void** Rcopy, void** Rop, __nv_bfloat16** Rpc,
                    double** sc, double** ppart, unsigned int** counter, void** x0, void** x1,
                    void** G, uint64_t** bits, void** Yb0, void** Yb1, void** Yb2, void** Zpart,
                    __nv_bfloat16** Sh, double** part, double** mom_c, double** mom_t,
                    float** mws, void** symws) {
        *sc = b.take<double>(SC_COUNT);
        *mws = out.mlp ? b.take<float>(64 + mlp_workspace_floats(1)) : nullptr;
        *counter = b.take<unsigned int>(64);
        *ppart = b.take<double>((size_t)std::max(power_blocks, 256) * 3 * q);
        *Rcopy = nullptr;
        if (R.memory == VNE_MEM_HOST || upper)
            *Rcopy = b.take<char>((size_t)(dense ? R.n : D) * R.ld * elt_size(R.dtype));
        *Rop = nullptr;
        for (int k = 0; k < kMaxPieces; ++k) Rpc[k] = nullptr;
        if (tc) {
            for (int k = 0; k < pieces; ++k) Rpc[k] = b.take<__nv_bfloat16>((size_t)rows_pad * ldk);
        } else {
            const int want = f64 ? VNE_F64 : VNE_F32;
            if (R.dtype != want) *Rop = b.take<char>((size_t)(dense ? n * n : (int64_t)D * n) * vt);
        }
        if (tc && cplx) {  // the embedding, FP32, before the bf16 split
            *Rop = b.take<char>((size_t)n * n * 4);
        }
        const size_t xs = pw_xdouble ? 8 : 4;
        *x0 = b.take<char>((size_t)n * q * xs);
        *x1 = b.take<char>((size_t)n * q * xs);
        *symws = use_sym ? b.take<char>((size_t)power_sym_scratch_bytes(rows_pad)) : nullptr;
        *G = *Yb0 = *Yb1 = *Yb2 = *Zpart = nullptr;
        *bits = nullptr;
        *Sh = nullptr;
        *part = *mom_c = *mom_t = nullptr;
        if (mode == MODE_POWER) return;
        const size_t ms = tc ? 4 : vt;
        if (!dense && pkind == VNE_RADEMACHER)
            *bits = b.take<uint64_t>((size_t)n * ((s + 63) / 64));
        else
            *G = b.take<char>((size_t)n * s * ms);
        *Yb0 = b.take<char>((size_t)n * S * ms);
        *Yb1 = b.take<char>((size_t)n * S * ms);
        *Yb2 = b.take<char>((size_t)n * S * ms);
        if (dense && !tc) *Zpart = b.take<char>((size_t)splitk * S * n * vt);
        if (tc) *Sh = b.take<__nv_bfloat16>((size_t)2 * pieces * S_pad * ldk);
        *part = b.take<double>((size_t)ntiles0 * S + (size_t)T_steps * ntiles * S);
        *mom_c = b.take<double>((size_t)(m + 1) * s);
        *mom_t = b.take<double>((size_t)(m + 1) * s);
    };
    void *Rcopy, *Rop, *x0, *x1, *G, *Yb0, *Yb1, *Yb2, *Zpart, *symws;
    __nv_bfloat16 *Rpc[kMaxPieces], *Sh;
    double *sc, *ppart, *part, *mom_c, *mom_t;
    float* mws;
    unsigned int* counter;
    uint64_t* bits;
    {
        Bump b0(nullptr);
        plan(b0, &Rcopy, &Rop, Rpc, &sc, &ppart, &counter, &x0, &x1, &G, &bits, &Yb0, &Yb1,
             &Yb2, &Zpart, &Sh, &part, &mom_c, &mom_t, &mws, &symws);
        if (out.measure) {
            *out.measured = b0.off + 4096;
            return VNE_OK;
        }
        char* base = out.ws;
        if (!base) {
            vs = ensure_ws(h, b0.off + 4096);
            if (vs != VNE_OK) return vs;
            base = h->ws;
        }
        Bump b1(base);
        plan(b1, &Rcopy, &Rop, Rpc, &sc, &ppart, &counter, &x0, &x1, &G, &bits, &Yb0, &Yb1,
             &Yb2, &Zpart, &Sh, &part, &mom_c, &mom_t, &mws, &symws);
    }
    h->ev_used = 0;
    h->pending.clear();

    const bool pro = out.phase != 2;  // the prologue runs in phases 0 and 1
    if (pro) {
        c.chk(cudaMemsetAsync(sc, 0, SC_COUNT * sizeof(double), c.st));
        c.chk(cudaMemsetAsync(counter, 0, 64 * sizeof(unsigned int), c.st));
    }

    // ---- matrix to the device, trace check ----
    const void* Rdata = R.data;
    if (R.memory == VNE_MEM_HOST) {
        const size_t bytes = (size_t)(dense ? R.n : D) * R.ld * elt_size(R.dtype);
        // whole (an upper-layout matrix too: strided copies of its triangle
        // from host memory ran far below the link's rate)
        if (pro) c.chk(cudaMemcpyAsync(Rcopy, R.data, bytes, cudaMemcpyHostToDevice, c.st));
        Rdata = Rcopy;
    }
    if (upper) {  // in place on the host copy, else from the caller's matrix
        if (pro) c.launched(launch_dense_symmetrize(Rdata, R.ld, Rcopy, R.ld, R.n, R.dtype, c.st));
        Rdata = Rcopy;
    }
    if (pro && p->check_trace)
        c.launched(launch_trace(Rdata, dense ? VNE_DENSE : VNE_DIA, R.dtype, R.n, R.ld, ppart,
                                counter, sc, c.st));

    // ---- operands ----
    const void* Rk = Rdata;  // operand of the SIMT / DIA / power kernels
    int64_t ldr = R.ld;
    if (cplx) {
        const int edt = (f64 && !tc) ? VNE_F64 : VNE_F32;
        if (pro) c.launched(launch_hermitian_embed(Rdata, R.dtype, R.n, R.ld, Rop, edt, c.st));
        Rk = Rop;
        ldr = n;
        if (tc && pro)
            c.launched(launch_dense_convert_bf16(Rop, VNE_F32, n, n, Rpc, pieces, rows_pad, ldk, c.st));
    } else if (tc && (mode != MODE_POWER || pw_rdt == 2)) {
        if (pro)
            c.launched(launch_dense_convert_bf16(Rdata, R.dtype, n, R.ld, Rpc, pieces, rows_pad, ldk, c.st));
    } else if (Rop) {
        if (!pro) {
        } else if (dense) {
            if (f64) c.launched(launch_dense_convert_f64(Rdata, R.dtype, n, R.ld, (double*)Rop, c.st));
            else c.launched(launch_dense_convert_f32(Rdata, R.dtype, n, R.ld, (float*)Rop, c.st));
        } else {
            c.launched(launch_dia_convert(Rdata, R.dtype, n, R.ld, D, Rop, f64 ? VNE_F64 : VNE_F32, c.st));
        }
        Rk = Rop;
        ldr = n;
    }

    // ---- power method (Algorithm alg:power) or the given u ----
    if (pro && do_power) {
        if (pw_xdouble) c.launched(launch_power_init<double>((double*)x0, n, q, p->seed, sc, c.st));
        else c.launched(launch_power_init<float>((float*)x0, n, q, p->seed, sc, c.st));
        // a batch's persistent power launch takes the products from here
        const bool batch_pw = out.batch_power && out.phase == 1 && out.bmat && pw_rdt == 2 &&
                              !pw_xdouble && q == 1 && dense && !cplx && pieces == 1;
        if (batch_pw) {
            out.bmat->x[0] = (float*)x0;
            out.bmat->x[1] = (float*)x1;
            out.bmat->ppart = ppart;
        }
        void* xa = x0;
        void* xb = x1;
        const void* Rp = pw_rdt == 2 ? (const void*)Rpc[0] : Rk;
        const int64_t ldp = pw_rdt == 2 ? ldk : ldr;
        // the products are timed as one span: an event between two of them
        // would stop the next one from starting early (programmatic launch)
        c.prof_begin();
        if (use_sym && !batch_pw) {
            c.launched(launch_power_sym(Rpc, sym_pieces, n, rows_pad, ldk, (const float*)x0,
                                        p->power_iters, sc, symws, u_scale, sym_grid, sym_phased,
                                        c.st));
            if (sym_phased) h->launches += 2 * p->power_iters + 2;
        }
        for (int it = 0; it <= p->power_iters && c.ok() && !use_sym && !batch_pw; ++it) {
            const int fin = it == p->power_iters;
            if (dense)
                c.launched(launch_power_step_dense(Rp, pw_rdt, n, ldp, xa, xb, pw_xdouble, q, sc,
                                                   ppart, counter, fin, u_scale, power_blocks, c.st));
            else
                c.launched(launch_power_step_dia(Rk, f64 ? 0 : 1, n, ldr, D, xa, xb, q, sc, ppart,
                                                 counter, fin, u_scale, power_blocks, c.st));
            std::swap(xa, xb);
        }
        c.prof_end(3, p->power_iters + 1);
    } else if (pro) {
        c.launched(launch_set_u(sc, p->u_override > 0.0 ? p->u_override : 1.0, c.st));
    }

    // ---- probes, recurrence, combine ----
    if (mode != MODE_POWER && c.ok()) {
        Partials P{part, ntiles0, ntiles, S};
        // bf16 pieces of the probe blocks, double-buffered across steps: sh[b][k]
        __nv_bfloat16* sh[2][kMaxPieces] = {};
        if (tc) {
            if (pro)
                c.chk(cudaMemsetAsync(Sh, 0,
                                      (size_t)2 * pieces * S_pad * ldk * sizeof(__nv_bfloat16),
                                      c.st));
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < pieces; ++k)
                    sh[b][k] = Sh + (size_t)(b * pieces + k) * S_pad * ldk;
        }
        if (!pro) {
        } else if (dense) {
            if (f64)
                c.launched(launch_dense_init<double>((double*)G, (double*)Yb0, nullptr, 0, 0,
                                                     n, S, s, pkind, p->seed, P, 256, c.st,
                                                     R.n, p->probe_offset,
                                                     (const double*)out.probes));
            else
                c.launched(launch_dense_init<float>((float*)G, (float*)Yb0, sh[0], pieces, ldk, n, S, s,
                                                    pkind, p->seed, P, rows_per_tile0, c.st,
                                                    R.n, p->probe_offset,
                                                    (const float*)out.probes));
        } else {
            const int Wd = (s + 63) / 64;
            if (f64)
                c.launched(launch_dia_init<double>((double*)G, bits, Wd,
                                                   bits ? nullptr : (double*)Yb0, n, S, s,
                                                   pkind, p->seed, P, rows_per_tile0, c.st,
                                                   p->probe_offset, (const double*)out.probes));
            else
                c.launched(launch_dia_init<float>((float*)G, bits, Wd, bits ? nullptr : (float*)Yb0,
                                                  n, S, s, pkind, p->seed, P, rows_per_tile0,
                                                  c.st, p->probe_offset, (const float*)out.probes));
        }
        void* Yb[3] = {Yb0, Yb1, Yb2};
        if (out.phase == 1) {  // the batch's persistent kernel runs the steps
            if (out.bmat && tc && pieces == 1 && dense && !cplx) {
                TcBatchMat& b = *out.bmat;
                b.R = Rpc[0];
                b.sh[0] = sh[0][0];
                b.sh[1] = sh[1][0];
                b.G = (const float*)G;
                for (int k = 0; k < 3; ++k) b.Y[k] = (float*)Yb[k];
                b.sc = sc;
                b.flags = sc + SC_FLAGS;
                b.P = P;
                b.n = n;
                b.rows_pad = rows_pad;
                b.ldk = ldk;
                b.S = S;
                b.s = s;
                b.m = m;
                b.T = T_steps;
                b.tiles = (int)(rows_pad / tc_tile_m());
                b.has_cheb = has_cheb ? 1 : 0;
                b.has_tay = has_tay ? 1 : 0;
            }
            return c.ok() ? VNE_OK : map_err(h, c.err);
        }
        // tensor-core steps are timed as one span (consecutive launches overlap
        // their prologues with the previous step's tail; an event between them
        // would serialise them)
        if (tc && pro) c.prof_begin();
        for (int t = 1; t <= T_steps && c.ok() && pro; ++t) {
            StepCols cols{};
            const bool cheb_on = has_cheb && t <= m;
            cols.cheb_c0 = 0;
            cols.ncheb = cheb_on ? s : 0;
            cols.cheb_kind = cheb_on ? (t == 1 ? EPI_CHEB1 : EPI_CHEB) : EPI_NONE;
            cols.tay_c0 = has_cheb ? s : 0;
            cols.ntay = has_tay ? s : 0;
            const int col0 = cheb_on ? 0 : cols.tay_c0;
            const int ncols = cols.ncheb + cols.ntay;
            void* Yp = Yb[(t - 1) % 3];
            void* Yp2 = Yb[(t + 1) % 3];
            void* Yn = Yb[t % 3];
            if (!tc) c.prof_begin();
            if (tc) {
                TcStep a{};
                a.pieces = pieces;
                for (int k = 0; k < pieces; ++k) {
                    a.R[k] = Rpc[k];
                    a.Y[k] = sh[(t - 1) & 1][k];
                    a.Y_out[k] = sh[t & 1][k];
                }
                a.G = (const float*)G;
                a.Yprev = (const float*)Yp;
                a.Yprev2 = (const float*)Yp2;
                a.Ynew = (float*)Yn;
                a.n = n;
                a.rows_pad = rows_pad;
                a.ldk = ldk;
                a.S = S;
                a.s = s;
                a.split = 1;
                a.cols = cols;
                a.sc = sc;
                a.P = P;
                a.t = t;
                c.launched(launch_tc_step(a, h->sm_count, c.st));
            } else if (dense) {
                if (f64) {
                    c.launched(launch_dense_simt_step<double>((const double*)Rk, ldr, n,
                                                              (const double*)Yp, (double*)Zpart, S,
                                                              col0, ncols, splitk, c.st));
                    c.launched(launch_dense_simt_epilogue<double>(
                        (const double*)Zpart, splitk, (const double*)G, (const double*)Yp,
                        (const double*)Yp2, (double*)Yn, n, S, s, cols, sc, P, t, c.st));
                } else {
                    c.launched(launch_dense_simt_step<float>((const float*)Rk, ldr, n,
                                                             (const float*)Yp, (float*)Zpart, S,
                                                             col0, ncols, splitk, c.st));
                    c.launched(launch_dense_simt_epilogue<float>(
                        (const float*)Zpart, splitk, (const float*)G, (const float*)Yp,
                        (const float*)Yp2, (float*)Yn, n, S, s, cols, sc, P, t, c.st));
                }
                c.prof_end(1);
            } else {
                const int Wd = (s + 63) / 64;
                if (f64)
                    c.launched(launch_dia_step<double>((const double*)Rk, ldr, D, n,
                                                       (const double*)Yp, (const double*)Yp2,
                                                       (double*)Yn, (const double*)G, bits, Wd, S,
                                                       s, cols, sc, P, t, dia_grid, c.st,
                                                       dia_band_aligned));
                else
                    c.launched(launch_dia_step<float>((const float*)Rk, ldr, D, n,
                                                      (const float*)Yp, (const float*)Yp2,
                                                      (float*)Yn, (const float*)G, bits, Wd, S, s,
                                                      cols, sc, P, t, dia_grid, c.st,
                                                      dia_band_aligned));
                c.prof_end(2);
            }
        }
        if (tc && pro) c.prof_end(0, T_steps);
        if (c.ok())
            c.launched(launch_combine(P, s, m, has_cheb ? 0 : -1, has_tay ? (has_cheb ? s : 0) : -1,
                                      mom_c, mom_t, sc, c.st));
        if (c.ok() && out.mlp) {
            int cnt = 0;
            c.chk(launch_learned(mom_c, m, s, n, sc, out.mlp, mws, &cnt, c.st));
            h->launches += cnt;
        }
    }

    // ---- results ----
    double* host_slot = out.host_slot ? out.host_slot : h->host_sc;
    if (c.ok()) c.chk(cudaMemcpyAsync(host_slot, sc, SC_COUNT * sizeof(double),
                                      cudaMemcpyDeviceToHost, c.st));
    if (out.host_slot) {  // batched: the caller synchronises and reads the slot
        if (!c.ok()) return map_err(h, c.err);
        return VNE_OK;
    }
    if (c.ok() && out.mom_cheb && has_cheb)
        c.chk(cudaMemcpyAsync(out.mom_cheb, mom_c, (size_t)(m + 1) * s * sizeof(double),
                              cudaMemcpyDeviceToHost, c.st));
    if (c.ok() && out.mom_taylor && has_tay)
        c.chk(cudaMemcpyAsync(out.mom_taylor, mom_t, (size_t)(m + 1) * s * sizeof(double),
                              cudaMemcpyDeviceToHost, c.st));
    {
        cudaError_t e = cudaStreamSynchronize(c.st);
        c.chk(e);
    }
    if (!c.ok()) {
        cudaGetLastError();
        return map_err(h, c.err);
    }
    collect_profile(h);
    const double* hs = h->host_sc;
    vne_status fs = slot_status(hs, p->check_trace);
    if (fs != VNE_OK) return fs;
    if (out.H_cheb) *out.H_cheb = hs[SC_H_CHEB];
    if (out.H_taylor) *out.H_taylor = hs[SC_H_TAYLOR];
    if (out.u) *out.u = hs[SC_U];
    if (out.lam) *out.lam = hs[SC_LAM];
    if (out.H_learned) *out.H_learned = hs[SC_H_LEARNED];
    return VNE_OK;
}

// R X on the tensor cores for the projection paths (Algorithm alg:EN and the
// block-Krylov extension): X and the result FP32 [cols][n]; R and X are split
// into `pieces` bf16 pieces (2: bf16x3, 3: bf16x6) and the step kernel runs
// with the plain-product epilogue.
struct TcProduct {
    int pieces = 0;
    int64_t n = 0, rows_pad = 0, ldk = 0;
    int S_pad = 0;
    __nv_bfloat16* Rp[kMaxPieces] = {};
    __nv_bfloat16* Xp[kMaxPieces] = {};
    double* sc = nullptr;
    double* part = nullptr;
    void plan(Bump& b, int pieces_, int64_t n_, int cols) {
        pieces = pieces_;
        n = n_;
        if (!pieces) return;
        rows_pad = round_up(n, tc_tile_m());
        ldk = round_up(n, tc_tile_k());
        S_pad = (int)round_up(cols, 32);
        for (int k = 0; k < pieces; ++k) {
            Rp[k] = b.take<__nv_bfloat16>((size_t)rows_pad * ldk);
            Xp[k] = b.take<__nv_bfloat16>((size_t)S_pad * ldk);
        }
        sc = b.take<double>(SC_COUNT);
        part = b.take<double>((size_t)2 * (rows_pad / tc_tile_m()) * cols);
    }
    // once per call: R in pieces, u = 1 in the scalar block (read, unused)
    void prepare(Call& c, const void* Rdata, int dtype, int64_t ld) {
        c.chk(cudaMemsetAsync(sc, 0, SC_COUNT * sizeof(double), c.st));
        c.launched(launch_dense_convert_bf16(Rdata, dtype, n, ld, Rp, pieces, rows_pad, ldk, c.st));
        if (c.ok()) c.launched(launch_set_u(sc, 1.0, c.st));
    }
    void product(Call& c, const float* X, float* dst, int cols) {
        if (!c.ok()) return;
        c.launched(launch_convert_bf16_rect(X, VNE_F32, cols, n, n, Xp, pieces, S_pad, ldk, c.st));
        if (!c.ok()) return;
        TcStep a{};
        a.pieces = pieces;
        for (int k = 0; k < pieces; ++k) {
            a.R[k] = Rp[k];
            a.Y[k] = Xp[k];
            a.Y_out[k] = Xp[k];  // not written by the plain product
        }
        a.G = dst;
        a.Yprev = dst;
        a.Yprev2 = dst;
        a.Ynew = dst;
        a.n = n;
        a.rows_pad = rows_pad;
        a.ldk = ldk;
        a.S = cols;
        a.s = cols;
        a.split = 1;
        a.cols = StepCols{0, 0, 0, cols, EPI_PLAIN};
        a.sc = sc;
        const int nt = (int)(rows_pad / tc_tile_m());
        a.P = Partials{part, nt, nt, cols};
        a.t = 1;
        c.prof_begin();
        c.launched(launch_tc_step(a, c.h->sm_count, c.st));
        c.prof_end(0);
    }
};

// ---------------------------------------------------------------------------
// Random projection (Algorithm alg:EN): sketch -> R Pi -> Gram -> eigenvalues
// -> top-k singular values and H~.
// ---------------------------------------------------------------------------
template <typename T>
vne_status run_projection(vne_handle* h, const vne_matrix& R, int k, int s, int kind,
                          uint64_t seed, double* H_out, double* p_out, cudaStream_t st,
                          int pieces = 0) {
    Call c{h, st};
    TcProduct tcp;
    const int64_t n = R.n;
    const int want = sizeof(T) == 8 ? VNE_F64 : VNE_F32;
    const int splitk = dense_simt_splitk(n, s, h->sm_count, (int)sizeof(T));
    const int chunks = gram_chunks(n, s, h->sm_count);
    auto plan = [&](Bump& b, void** Rcopy, T** Rop, T** Pi, T** Zpart, T** Z, double** part,
                    double** C, double** W, double** de, double** ev, double** out) {
        *Rcopy = R.memory == VNE_MEM_HOST ? b.take<char>((size_t)n * R.ld * elt_size(R.dtype))
                                          : nullptr;
        *Rop = (R.dtype != want && !pieces) ? b.take<T>((size_t)n * n) : nullptr;
        *Pi = b.take<T>((size_t)n * s);
        *Zpart = b.take<T>((size_t)(pieces ? 1 : splitk) * s * n);
        *Z = (splitk > 1 && !pieces) ? b.take<T>((size_t)s * n) : *Zpart;
        tcp.plan(b, pieces, n, s);
        *part = b.take<double>((size_t)chunks * s * s);
        *C = b.take<double>((size_t)s * s);
        *W = b.take<double>((size_t)s * s);
        *de = b.take<double>((size_t)2 * s);
        *ev = b.take<double>((size_t)s);
        *out = b.take<double>((size_t)k + 1);
    };
    void* Rcopy;
    T *Rop, *Pi, *Zpart, *Z;
    double *part, *C, *W, *de, *ev, *out;
    {
        Bump b0(nullptr);
        plan(b0, &Rcopy, &Rop, &Pi, &Zpart, &Z, &part, &C, &W, &de, &ev, &out);
        vne_status vs = ensure_ws(h, b0.off + 4096);
        if (vs != VNE_OK) return vs;
        Bump b1(h->ws);
        plan(b1, &Rcopy, &Rop, &Pi, &Zpart, &Z, &part, &C, &W, &de, &ev, &out);
    }
    h->ev_used = 0;
    h->pending.clear();
    const void* Rdata = R.data;
    if (R.memory == VNE_MEM_HOST) {
        c.chk(cudaMemcpyAsync(Rcopy, R.data, (size_t)n * R.ld * elt_size(R.dtype),
                              cudaMemcpyHostToDevice, st));
        Rdata = Rcopy;
    }
    const T* Rk = (const T*)Rdata;
    int64_t ldr = R.ld;
    if (Rop) {
        if (sizeof(T) == 8)
            c.launched(launch_dense_convert_f64(Rdata, R.dtype, n, R.ld, (double*)Rop, st));
        else
            c.launched(launch_dense_convert_f32(Rdata, R.dtype, n, R.ld, (float*)Rop, st));
        Rk = Rop;
        ldr = n;
    }
    if (c.ok()) c.launched(launch_sketch<T>(Pi, n, s, kind, seed, h->sm_count, st));
    if (pieces) {
        if (c.ok()) tcp.prepare(c, Rdata, R.dtype, R.ld);
        tcp.product(c, (const float*)Pi, (float*)Z, s);
    } else {
        if (c.ok()) {
            c.prof_begin();
            c.launched(launch_dense_simt_step<T>(Rk, ldr, n, Pi, Zpart, s, 0, s, splitk, st));
            c.prof_end(1);
        }
        if (c.ok() && splitk > 1)
            c.launched(launch_split_sum<T>(Zpart, splitk, (int64_t)s * n, Z, h->sm_count, st));
    }
    if (c.ok()) c.launched(launch_gram<T>(Z, n, s, chunks, part, C, st));
    if (c.ok()) c.launched(launch_sym_eigvals(C, s, k, W, de, de + s, ev, st));
    if (c.ok()) c.launched(launch_proj_combine(ev, k, out, st));
    std::vector<double> host((size_t)k + 1);
    if (c.ok())
        c.chk(cudaMemcpyAsync(host.data(), out, (size_t)(k + 1) * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
    c.chk(cudaStreamSynchronize(st));
    if (!c.ok()) {
        cudaGetLastError();
        return map_err(h, c.err);
    }
    collect_profile(h);
    if (!std::isfinite(host[0])) return VNE_ERR_NONFINITE;
    *H_out = host[0];
    if (p_out) std::memcpy(p_out, host.data() + 1, (size_t)k * sizeof(double));
    return VNE_OK;
}

// ---------------------------------------------------------------------------
// Block Krylov extension of the projection path (not in the paper).
// ---------------------------------------------------------------------------
template <typename T>
vne_status run_krylov(vne_handle* h, const vne_matrix& R, int k, int b, int q, int kind,
                      uint64_t seed, double* H_out, double* p_out, cudaStream_t st,
                      int pieces = 0) {
    Call c{h, st};
    TcProduct tcp;
    const int64_t n = R.n;
    const int want = sizeof(T) == 8 ? VNE_F64 : VNE_F32;
    const int N = q * b;
    const int splitk = dense_simt_splitk(n, b, h->sm_count, (int)sizeof(T));
    const int chunks = gram_chunks(n, std::max(N, b), h->sm_count);
    const double drop = sizeof(T) == 8 ? 1e-12 : 1e-6;
    auto plan = [&](Bump& bp, void** Rcopy, T** Rop, T** Pi, T** V, T** Zpart, T** K, T** W,
                    double** part, double** C, double** G, double** lam, double** U, double** M,
                    double** Tm, double** Wg, double** de, double** ev, double** out,
                    double** lref) {
        *Rcopy = R.memory == VNE_MEM_HOST ? bp.take<char>((size_t)n * R.ld * elt_size(R.dtype))
                                          : nullptr;
        *Rop = (R.dtype != want && !pieces) ? bp.take<T>((size_t)n * n) : nullptr;
        *Pi = bp.take<T>((size_t)n * b);
        *V = bp.take<T>((size_t)n * b);
        *Zpart = bp.take<T>((size_t)(pieces ? 1 : splitk) * b * n);
        tcp.plan(bp, pieces, n, b);
        *K = bp.take<T>((size_t)N * n);
        *W = bp.take<T>((size_t)N * n);
        *part = bp.take<double>((size_t)chunks * N * N);
        *C = bp.take<double>((size_t)N * b);
        *G = bp.take<double>((size_t)b * b);
        *lam = bp.take<double>((size_t)b);
        *U = bp.take<double>((size_t)b * b);
        *M = bp.take<double>((size_t)b * b);
        *Tm = bp.take<double>((size_t)N * N);
        *Wg = bp.take<double>((size_t)N * N);
        *de = bp.take<double>((size_t)2 * N);
        *ev = bp.take<double>((size_t)N);
        *out = bp.take<double>((size_t)k + 1);
        *lref = bp.take<double>(1);
    };
    void* Rcopy;
    T *Rop, *Pi, *V, *Zpart, *K, *W;
    double *part, *C, *G, *lam, *U, *M, *Tm, *Wg, *de, *ev, *out, *lref;
    {
        Bump b0(nullptr);
        plan(b0, &Rcopy, &Rop, &Pi, &V, &Zpart, &K, &W, &part, &C, &G, &lam, &U, &M, &Tm, &Wg,
             &de, &ev, &out, &lref);
        vne_status vs = ensure_ws(h, b0.off + 4096);
        if (vs != VNE_OK) return vs;
        Bump b1(h->ws);
        plan(b1, &Rcopy, &Rop, &Pi, &V, &Zpart, &K, &W, &part, &C, &G, &lam, &U, &M, &Tm, &Wg,
             &de, &ev, &out, &lref);
    }
    h->ev_used = 0;
    h->pending.clear();
    const void* Rdata = R.data;
    if (R.memory == VNE_MEM_HOST) {
        c.chk(cudaMemcpyAsync(Rcopy, R.data, (size_t)n * R.ld * elt_size(R.dtype),
                              cudaMemcpyHostToDevice, st));
        Rdata = Rcopy;
    }
    const T* Rk = (const T*)Rdata;
    int64_t ldr = R.ld;
    if (Rop) {
        if (sizeof(T) == 8)
            c.launched(launch_dense_convert_f64(Rdata, R.dtype, n, R.ld, (double*)Rop, st));
        else
            c.launched(launch_dense_convert_f32(Rdata, R.dtype, n, R.ld, (float*)Rop, st));
        Rk = Rop;
        ldr = n;
    }
    if (pieces && c.ok()) tcp.prepare(c, Rdata, R.dtype, R.ld);
    // dst = R X (X stored [b][n])
    auto product = [&](const T* X, T* dst) {
        if (!c.ok()) return;
        if (pieces) {
            tcp.product(c, (const float*)X, (float*)dst, b);
            return;
        }
        c.prof_begin();
        c.launched(launch_dense_simt_step<T>(Rk, ldr, n, X, Zpart, b, 0, b, splitk, st));
        c.prof_end(1);
        if (c.ok()) c.launched(launch_split_sum<T>(Zpart, splitk, (int64_t)b * n, dst, h->sm_count, st));
    };
    if (c.ok()) c.launched(launch_sketch<T>(Pi, n, b, kind, seed, h->sm_count, st));
    product(Pi, V);
    for (int j = 0; j < q && c.ok(); ++j) {
        T* Kj = K + (size_t)j * b * n;
        if (j > 0) {
            c.chk(cudaMemcpyAsync(V, W + (size_t)(j - 1) * b * n, (size_t)b * n * sizeof(T),
                                  cudaMemcpyDeviceToDevice, st));
            for (int pass = 0; pass < 2 && c.ok(); ++pass) {
                c.launched(launch_xgram<T>(K, j * b, V, b, n, chunks, part, C, st));
                if (c.ok()) c.launched(launch_ts_mm<T>(K, j * b, C, b, -1.0, V, V, n, st));
            }
        }
        if (c.ok()) c.launched(launch_gram<T>(V, n, b, chunks, part, G, st));
        if (c.ok()) c.launched(launch_jacobi<T>(G, b, lam, U, st));
        if (c.ok()) c.launched(launch_basis_coeffs(lam, U, b, lref, j == 0, drop, M, st));
        if (c.ok()) c.launched(launch_ts_mm<T>(V, b, M, b, 1.0, nullptr, Kj, n, st));
        product(Kj, W + (size_t)j * b * n);
    }
    if (c.ok()) c.launched(launch_xgram<T>(K, N, W, N, n, chunks, part, Tm, st));
    if (c.ok()) c.launched(launch_symmetrize(Tm, N, st));
    if (c.ok()) c.launched(launch_sym_eigvals(Tm, N, k, Wg, de, de + N, ev, st));
    if (c.ok()) c.launched(launch_krylov_combine(ev, k, n, out, st));
    std::vector<double> host((size_t)k + 1);
    if (c.ok())
        c.chk(cudaMemcpyAsync(host.data(), out, (size_t)(k + 1) * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
    c.chk(cudaStreamSynchronize(st));
    if (!c.ok()) {
        cudaGetLastError();
        return map_err(h, c.err);
    }
    collect_profile(h);
    if (!std::isfinite(host[0])) return VNE_ERR_NONFINITE;
    *H_out = host[0];
    if (p_out) std::memcpy(p_out, host.data() + 1, (size_t)k * sizeof(double));
    return VNE_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

vne_status vne_create(vne_handle** out, int device) {
    if (!out) return VNE_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return VNE_ERR_INVALID_ARG;
    }
    vne_handle* h = new (std::nothrow) vne_handle();
    if (!h) return VNE_ERR_OOM;
    h->device = device;
    DeviceGuard guard(device);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return VNE_ERR_CUDA;
    }
    if (cudaMallocHost((void**)&h->host_sc, SC_COUNT * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return VNE_ERR_OOM;
    }
    *out = h;
    return VNE_OK;
}

void vne_destroy(vne_handle* h) {
    if (!h) return;
    DeviceGuard guard(h->device);
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    if (h->host_sc) cudaFreeHost(h->host_sc);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (cudaStream_t st : h->bstreams) cudaStreamDestroy(st);
    for (cudaEvent_t e : h->bevents) cudaEventDestroy(e);
    if (h->bws) cudaFree(h->bws);
    if (h->bhost) cudaFreeHost(h->bhost);
    if (h->btab_dev) cudaFree(h->btab_dev);
    if (h->btab_host) cudaFreeHost(h->btab_host);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (h->stage[k]) cudaFree(h->stage[k]);
        if (h->cev[k]) cudaEventDestroy(h->cev[k]);
    }
    if (h->cstream) cudaStreamDestroy(h->cstream);
    delete h;
}

vne_status vne_entropy_chebyshev(vne_handle* h, const vne_matrix* R, const vne_params* p,
                                 double* H_out, double* moments_out, double* u_out, void* stream) {
    if (!H_out) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_cheb = H_out;
    o.mom_cheb = moments_out;
    o.u = u_out;
    return run(h, R, p, MODE_CHEB, o, stream);
}

vne_status vne_entropy_taylor(vne_handle* h, const vne_matrix* R, const vne_params* p,
                              double* H_out, double* moments_out, double* u_out, void* stream) {
    if (!H_out) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_taylor = H_out;
    o.mom_taylor = moments_out;
    o.u = u_out;
    return run(h, R, p, MODE_TAYLOR, o, stream);
}

vne_status vne_entropy_both(vne_handle* h, const vne_matrix* R, const vne_params* p,
                            double* H_cheb, double* H_taylor, double* moments_cheb,
                            double* moments_taylor, double* u_out, void* stream) {
    if (!H_cheb || !H_taylor) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_cheb = H_cheb;
    o.H_taylor = H_taylor;
    o.mom_cheb = moments_cheb;
    o.mom_taylor = moments_taylor;
    o.u = u_out;
    return run(h, R, p, MODE_BOTH, o, stream);
}

int64_t vne_batch_queue(const int64_t* n, int32_t count, int32_t m, int32_t s, int32_t method,
                        double l2_mb, int32_t min_tiles, int32_t* items_out) {
    if (!n || count < 1 || m < 1 || s < 1 || !(l2_mb > 0.0) || min_tiles < 0) return -1;
    if (method != VNE_METHOD_TAYLOR && method != VNE_METHOD_CHEBYSHEV && method != VNE_METHOD_BOTH)
        return -1;
    const bool cheb = method != VNE_METHOD_TAYLOR, tay = method != VNE_METHOD_CHEBYSHEV;
    std::vector<TcBatchMat> bm((size_t)count, TcBatchMat{});
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1) return -1;
        TcBatchMat& b = bm[i];
        b.n = n[i];
        b.rows_pad = round_up(b.n, tc_tile_m());
        b.ldk = round_up(b.n, tc_tile_k());
        b.tiles = (int)(b.rows_pad / tc_tile_m());
        b.s = s;
        b.S = (cheb && tay) ? 2 * s : s;
        b.m = m;
        b.has_cheb = cheb ? 1 : 0;
        b.has_tay = tay ? 1 : 0;
        b.T = tay ? m + 1 : m;
    }
    return tc_batch_schedule(bm.data(), count, l2_mb * 1048576.0, min_tiles, items_out);
}

vne_status vne_entropy_chebyshev_probes(vne_handle* h, const vne_matrix* R, const void* G,
                                        const vne_params* p, double* H_out, double* moments_out,
                                        double* u_out, void* stream) {
    if (!H_out || !G) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_cheb = H_out;
    o.mom_cheb = moments_out;
    o.u = u_out;
    o.probes = G;
    return run(h, R, p, MODE_CHEB, o, stream);
}

vne_status vne_entropy_taylor_probes(vne_handle* h, const vne_matrix* R, const void* G,
                                     const vne_params* p, double* H_out, double* moments_out,
                                     double* u_out, void* stream) {
    if (!H_out || !G) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_taylor = H_out;
    o.mom_taylor = moments_out;
    o.u = u_out;
    o.probes = G;
    return run(h, R, p, MODE_TAYLOR, o, stream);
}

namespace {
uint64_t mix(uint64_t hsh, uint64_t v) { return splitmix_out(hsh ^ v, 0x51ull); }

// Streams of a batched call: VNE_BATCH_STREAMS (1..64), default 32 (measured on
// the 256-matrix batch: 6.40k entropies/s with 8 streams, 7.01k with 16, 7.34k with 32).
int batch_streams() {
    static int k = 0;
    if (!k) {
        k = 32;
        if (const char* e = getenv("VNE_BATCH_STREAMS")) {
            const int v = atoi(e);
            if (v >= 1 && v <= 64) k = v;
        }
    }
    return k;
}

// Batches run their recurrence in one persistent launch (BF16, dense real
// matrices, at most 64 step columns) unless VNE_BATCH_PERSISTENT=0 (read at
// each call).  VNE_BATCH_L2_MB (bf16 R of the matrices active at a time;
// default: no limit, every matrix in every round) and VNE_BATCH_MIN_TILES
// (default 2 per SM) shape its queue.  Measured on 256 matrices of n in
// [256, 4096]: 23.5 ms per batch with every matrix active, 28.1 ms with a
// 16-128 MiB active set (fewer independent items per round).
bool batch_persistent_enabled() {
    const char* e = getenv("VNE_BATCH_PERSISTENT");
    return !(e && e[0] == '0');
}
double batch_l2_budget() {
    const char* e = getenv("VNE_BATCH_L2_MB");
    const double v = e ? atof(e) : 0.0;
    return (v > 0.0 ? v * 1048576.0 : 1e300);
}
// Test hook of the persistent launches' bounded waits: VNE_BATCH_TEST_STALL=1
// (recurrence) or 2 (power method) makes every dependency wait for one tile
// more than the matrix has, so the waits expire and the call returns
// VNE_ERR_TIMEOUT; the GPU is not faulted and the next call runs normally.
int batch_test_stall() {
    const char* e = getenv("VNE_BATCH_TEST_STALL");
    return e ? atoi(e) : 0;
}

// The power launch's queue: VNE_BATCH_POWER_L2_MB (default: no limit) and
// VNE_BATCH_POWER_MIN_TILES (default 4 per SM).
double batch_power_l2_budget() {
    const char* e = getenv("VNE_BATCH_POWER_L2_MB");
    const double v = e ? atof(e) : 0.0;
    return (v > 0.0 ? v * 1048576.0 : 1e300);
}
int batch_power_min_tiles(int sm_count) {
    const char* e = getenv("VNE_BATCH_POWER_MIN_TILES");
    const int v = e ? atoi(e) : 4 * sm_count;
    return v >= 0 ? v : 4 * sm_count;
}
int batch_min_tiles(int sm_count) {
    const char* e = getenv("VNE_BATCH_MIN_TILES");
    const int v = e ? atoi(e) : 2 * sm_count;
    return v >= 0 ? v : 2 * sm_count;
}

// The pinned and device tables of the persistent launch (grown as needed; a
// captured graph that holds the old ones is dropped first).
vne_status batch_table(vne_handle* h, size_t bytes) {
    if (bytes <= h->btab_bytes) return VNE_OK;
    cudaDeviceSynchronize();
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (h->btab_dev) cudaFree(h->btab_dev);
    if (h->btab_host) cudaFreeHost(h->btab_host);
    h->btab_dev = h->btab_host = nullptr;
    h->btab_bytes = 0;
    if (cudaMalloc((void**)&h->btab_dev, bytes) != cudaSuccess ||
        cudaMallocHost((void**)&h->btab_host, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (h->btab_dev) cudaFree(h->btab_dev);
        h->btab_dev = nullptr;
        h->btab_host = nullptr;
        return VNE_ERR_OOM;
    }
    h->btab_bytes = bytes;
    return VNE_OK;
}

// The identity of a captured batch graph: the matrices' sizes, addresses and
// layouts, the parameters, the method, the handle's batch buffers and the
// queue settings; a call with the same key replays the graph.
uint64_t batch_key(const vne_handle* h, const vne_matrix* Rs, int count, const vne_params* p,
                   int method, bool pers, double l2_budget, int min_tiles, double pw_budget,
                   int pw_min_tiles, int stall) {
    uint64_t key = mix(0x9E3779B97F4A7C15ull, (uint64_t)count);
    for (int i = 0; i < count; ++i) {
        key = mix(key, (uint64_t)Rs[i].n);
        key = mix(key, (uint64_t)(uintptr_t)Rs[i].data);
        key = mix(key, (uint64_t)Rs[i].ld);
        key = mix(key, ((uint64_t)Rs[i].layout << 32) ^ ((uint64_t)Rs[i].dtype << 16) ^
                           (uint64_t)Rs[i].n_diags);
    }
    const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
    for (size_t b = 0; b < sizeof(vne_params); ++b) key = mix(key, pb[b] + (b << 8));
    key = mix(key, (uint64_t)method);
    key = mix(key, (uint64_t)(uintptr_t)h->bws);
    key = mix(key, (uint64_t)(uintptr_t)h->bhost);
    key = mix(key, pers ? (uint64_t)(uintptr_t)h->btab_dev ^ 0x70657273ull : 0ull);
    key = mix(key, (uint64_t)std::min(l2_budget / 1024.0, 1e18) ^ ((uint64_t)min_tiles << 40));
    key = mix(key, (uint64_t)std::min(pw_budget / 1024.0, 1e18) ^ ((uint64_t)pw_min_tiles << 40));
    key = mix(key, (uint64_t)stall);
    return key;
}

vne_status batch_resources(vne_handle* h, size_t ws_bytes, size_t count) {
    const int K = batch_streams();
    while ((int)h->bstreams.size() < K) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return VNE_ERR_CUDA;
        }
        h->bstreams.push_back(st);
    }
    while ((int)h->bevents.size() < K + 2) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return VNE_ERR_CUDA;
        }
        h->bevents.push_back(e);
    }
    if (ws_bytes > h->bws_bytes || count > h->bhost_count) {
        cudaDeviceSynchronize();
        if (h->graph) {  // the graph holds the old addresses
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
    }
    if (ws_bytes > h->bws_bytes) {
        if (h->bws) cudaFree(h->bws);
        h->bws = nullptr;
        h->bws_bytes = 0;
        if (cudaMalloc((void**)&h->bws, ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            h->bws = nullptr;
            return VNE_ERR_OOM;
        }
        h->bws_bytes = ws_bytes;
    }
    if (count > h->bhost_count) {
        if (h->bhost) cudaFreeHost(h->bhost);
        h->bhost = nullptr;
        h->bhost_count = 0;
        if (cudaMallocHost((void**)&h->bhost, count * SC_COUNT * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            h->bhost = nullptr;
            return VNE_ERR_OOM;
        }
        h->bhost_count = count;
    }
    return VNE_OK;
}

// The copy stream, its two events and `slots` device slots of `bytes` each
// for a sequence call (grown as needed; freed with the handle).
vne_status stage_resources(vne_handle* h, size_t bytes, int slots) {
    cudaError_t e = cudaSuccess;
    if (!h->cstream) e = cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!h->cev[k]) e = cudaEventCreateWithFlags(&h->cev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return map_err(h, e);
    }
    if (bytes > h->stage_bytes) {
        cudaDeviceSynchronize();
        for (int k = 0; k < 2; ++k) {
            if (h->stage[k]) cudaFree(h->stage[k]);
            h->stage[k] = nullptr;
        }
        h->stage_bytes = 0;
    }
    for (int k = 0; k < slots; ++k) {
        if (h->stage[k]) continue;
        const size_t want = bytes > h->stage_bytes ? bytes : h->stage_bytes;
        if (cudaMalloc((void**)&h->stage[k], want) != cudaSuccess) {
            cudaGetLastError();
            h->stage[k] = nullptr;
            return VNE_ERR_OOM;
        }
    }
    if (bytes > h->stage_bytes) h->stage_bytes = bytes;
    return VNE_OK;
}

}  // namespace

vne_status vne_entropy_batched(vne_handle* h, const vne_matrix* Rs, int32_t count,
                               const vne_params* p, int32_t method, int32_t use_graph,
                               double* H_cheb, double* H_taylor, double* u_out, void* stream) {
    if (!h || !Rs || !p || count < 1) return VNE_ERR_INVALID_ARG;
    if (method != VNE_METHOD_TAYLOR && method != VNE_METHOD_CHEBYSHEV && method != VNE_METHOD_BOTH)
        return VNE_ERR_INVALID_ARG;
    const int mode = method == VNE_METHOD_TAYLOR ? MODE_TAYLOR
                     : method == VNE_METHOD_CHEBYSHEV ? MODE_CHEB : MODE_BOTH;
    if ((mode & MODE_CHEB) && !H_cheb) return VNE_ERR_INVALID_ARG;
    if ((mode & MODE_TAYLOR) && !H_taylor) return VNE_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (Rs[i].memory != VNE_MEM_DEVICE) return VNE_ERR_UNSUPPORTED;
    DeviceGuard guard(h->device);
    // the recurrence (and power method) of the whole batch in persistent launches
    const int S_all = mode == MODE_BOTH ? 2 * p->s : p->s;
    bool pers = batch_persistent_enabled() && p->precision == VNE_PREC_BF16 && S_all <= 64;
    for (int i = 0; i < count && pers; ++i)
        if (Rs[i].layout != VNE_DENSE || is_complex(Rs[i].dtype)) pers = false;
    const double l2_budget = batch_l2_budget();
    const int min_tiles = batch_min_tiles(h->sm_count);
    const double pw_budget = batch_power_l2_budget();
    const int pw_min_tiles = batch_power_min_tiles(h->sm_count);
    const int stall = batch_test_stall();
    // results of the batch from the pinned host slots
    auto collect = [&]() -> vne_status {
        vne_status first = VNE_OK;
        for (int i = 0; i < count; ++i) {
            const double* hs = h->bhost + (size_t)i * SC_COUNT;
            vne_status fs = slot_status(hs, p->check_trace);
            if (fs != VNE_OK && first == VNE_OK) first = fs;
            const double nan = std::nan("");
            if (H_cheb && (mode & MODE_CHEB)) H_cheb[i] = fs == VNE_OK ? hs[SC_H_CHEB] : nan;
            if (H_taylor && (mode & MODE_TAYLOR)) H_taylor[i] = fs == VNE_OK ? hs[SC_H_TAYLOR] : nan;
            if (u_out) u_out[i] = hs[SC_U];
        }
        return first;
    };
    // replay: the same batch as the captured graph needs no planning at all
    if (use_graph && h->graph && !h->bstreams.empty() &&
        batch_key(h, Rs, count, p, method, pers, l2_budget, min_tiles, pw_budget, pw_min_tiles,
                  stall) == h->graph_key) {
        cudaStream_t user = (cudaStream_t)stream, origin = h->bstreams[0];
        cudaError_t e = cudaEventRecord(h->bevents[1], user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, h->bevents[1], 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(h->graph, origin);
        if (e == cudaSuccess) e = cudaEventRecord(h->bevents[1], origin);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->bevents[1], 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(user);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return map_err(h, e);
        }
        return collect();
    }
    // workspace of every matrix (the same plan as a single call)
    std::vector<size_t> off((size_t)count + 1, 0);
    for (int i = 0; i < count; ++i) {
        Outputs o;
        o.measure = 1;
        size_t bytes = 0;
        o.measured = &bytes;
        vne_status vs = run(h, &Rs[i], p, mode, o, nullptr);
        if (vs != VNE_OK) return vs;
        off[i + 1] = off[i] + round_up((int64_t)bytes, 256);
    }
    vne_status vs = batch_resources(h, off[count], (size_t)count);
    if (vs != VNE_OK) return vs;
    std::vector<TcBatchMat> bm;
    std::vector<int> items, pw_items;
    int64_t n_items = 0, pw_items_n = 0;
    bool pw_batch = false;
    size_t pw_tab = 0;  // bytes of the power launch's table, before the recurrence's
    if (pers) {
        bm.assign((size_t)count, TcBatchMat{});
        for (int i = 0; i < count; ++i) {
            TcBatchMat& b = bm[i];
            b.n = Rs[i].n;
            b.rows_pad = round_up(b.n, tc_tile_m());
            b.ldk = round_up(b.n, tc_tile_k());
            b.tiles = (int)(b.rows_pad / tc_tile_m());
            b.S = S_all;
            b.s = p->s;
            b.m = p->m;
            b.has_cheb = (mode & MODE_CHEB) ? 1 : 0;
            b.has_tay = (mode & MODE_TAYLOR) ? 1 : 0;
            b.T = b.has_tay ? p->m + 1 : p->m;
        }
        n_items = tc_batch_schedule(bm.data(), count, l2_budget, min_tiles, nullptr);
        items.assign((size_t)n_items * 4, 0);
        tc_batch_schedule(bm.data(), count, l2_budget, min_tiles, items.data());
        // the power method in a persistent launch too (one trial, no given u):
        // its own queue over t + 1 products
        pw_batch = !(p->u_override > 0.0) && p->power_trials <= 1;
        if (pw_batch) {
            std::vector<TcBatchMat> pm(bm);
            for (TcBatchMat& b : pm) b.T = p->power_iters + 1;
            pw_items_n = tc_batch_schedule(pm.data(), count, pw_budget, pw_min_tiles, nullptr);
            pw_items.assign((size_t)pw_items_n * 4, 0);
            tc_batch_schedule(pm.data(), count, pw_budget, pw_min_tiles, pw_items.data());
            pw_tab = (tc_batch_table_bytes(pm.data(), count, pw_items_n) + 255) & ~(size_t)255;
        }
        vs = batch_table(h, pw_tab + tc_batch_table_bytes(bm.data(), count, n_items));
        if (vs != VNE_OK) return vs;
    }
    const int K = batch_streams();
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t origin = h->bstreams[0];
    const int saved_prof = h->prof_on;
    h->prof_on = 0;
    // every matrix on one of the K streams, forked from and joined into origin
    auto enqueue = [&]() -> vne_status {
        cudaError_t e = cudaEventRecord(h->bevents[0], origin);
        for (int k = 1; k < K && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(h->bstreams[k], h->bevents[0], 0);
        if (e != cudaSuccess) return map_err(h, e);
        for (int i = 0; i < count; ++i) {
            Outputs o;
            o.ws = h->bws + off[i];
            o.host_slot = h->bhost + (size_t)i * SC_COUNT;
            if (pers) {
                o.phase = 1;
                o.bmat = &bm[i];
                o.batch_power = pw_batch ? 1 : 0;
            }
            vne_status r = run(h, &Rs[i], p, mode, o, h->bstreams[i % K]);
            if (r != VNE_OK) return r;
        }
        if (pers) {
            // join, one launch for every step of every matrix, fork again
            for (int k = 1; k < K && e == cudaSuccess; ++k) {
                e = cudaEventRecord(h->bevents[2 + k], h->bstreams[k]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, h->bevents[2 + k], 0);
            }
            if (e == cudaSuccess && pw_batch) {
                std::vector<TcBatchMat> pm(bm);
                for (TcBatchMat& b : pm) b.T = p->power_iters + 1;
                const double u_scale = p->u_scale > 0.0 ? p->u_scale : 1.0;
                e = launch_power_batch(pm.data(), count, pw_items.data(), pw_items_n,
                                       p->power_iters, u_scale, h->btab_host, h->btab_dev,
                                       h->sm_count, origin, stall == 2 ? 1 : 0);
                if (e == cudaSuccess) ++h->launches;
            }
            if (e == cudaSuccess)
                e = launch_tc_batch(bm.data(), count, items.data(), n_items,
                                    h->btab_host + pw_tab, h->btab_dev + pw_tab, h->sm_count,
                                    origin, stall == 1 ? 1 : 0);
            if (e == cudaSuccess) ++h->launches;
            if (e == cudaSuccess) e = cudaEventRecord(h->bevents[0], origin);
            for (int k = 1; k < K && e == cudaSuccess; ++k)
                e = cudaStreamWaitEvent(h->bstreams[k], h->bevents[0], 0);
            if (e != cudaSuccess) return map_err(h, e);
            for (int i = 0; i < count; ++i) {
                Outputs o;
                o.ws = h->bws + off[i];
                o.host_slot = h->bhost + (size_t)i * SC_COUNT;
                o.phase = 2;
                vne_status r = run(h, &Rs[i], p, mode, o, h->bstreams[i % K]);
                if (r != VNE_OK) return r;
            }
        }
        for (int k = 1; k < K && e == cudaSuccess; ++k) {
            e = cudaEventRecord(h->bevents[2 + k], h->bstreams[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, h->bevents[2 + k], 0);
        }
        return map_err(h, e);
    };
    cudaError_t e = cudaEventRecord(h->bevents[1], user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, h->bevents[1], 0);
    if (e != cudaSuccess) {
        h->prof_on = saved_prof;
        return map_err(h, e);
    }
    if (use_graph) {
        const uint64_t key = batch_key(h, Rs, count, p, method, pers, l2_budget, min_tiles,
                                       pw_budget, pw_min_tiles, stall);
        if (!h->graph || key != h->graph_key) {
            if (h->graph) {
                cudaGraphExecDestroy(h->graph);
                h->graph = nullptr;
            }
            e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                h->prof_on = saved_prof;
                return map_err(h, e);
            }
            vne_status r = enqueue();
            cudaGraph_t g = nullptr;
            cudaError_t ee = cudaStreamEndCapture(origin, &g);
            if (r != VNE_OK || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                h->prof_on = saved_prof;
                return r != VNE_OK ? r : map_err(h, ee);
            }
            ee = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            if (ee != cudaSuccess) {
                h->graph = nullptr;
                h->prof_on = saved_prof;
                return map_err(h, ee);
            }
            h->graph_key = key;
        }
        e = cudaGraphLaunch(h->graph, origin);
        if (e != cudaSuccess) {
            h->prof_on = saved_prof;
            return map_err(h, e);
        }
    } else {
        vne_status r = enqueue();
        if (r != VNE_OK) {
            h->prof_on = saved_prof;
            cudaStreamSynchronize(origin);
            return r;
        }
    }
    h->prof_on = saved_prof;
    e = cudaEventRecord(h->bevents[1], origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->bevents[1], 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(user);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return map_err(h, e);
    }
    return collect();
}

vne_status vne_entropy_sequence(vne_handle* h, const vne_matrix* Rs, int32_t count,
                                const vne_params* p, int32_t method, double* H_cheb,
                                double* H_taylor, double* u_out, void* stream) {
    if (!h || !Rs || !p || count < 1) return VNE_ERR_INVALID_ARG;
    if (method != VNE_METHOD_TAYLOR && method != VNE_METHOD_CHEBYSHEV && method != VNE_METHOD_BOTH)
        return VNE_ERR_INVALID_ARG;
    const int mode = method == VNE_METHOD_TAYLOR ? MODE_TAYLOR
                     : method == VNE_METHOD_CHEBYSHEV ? MODE_CHEB : MODE_BOTH;
    if ((mode & MODE_CHEB) && !H_cheb) return VNE_ERR_INVALID_ARG;
    if ((mode & MODE_TAYLOR) && !H_taylor) return VNE_ERR_INVALID_ARG;
    // every matrix is checked before any transfer starts
    size_t stage = 0;
    int nhost = 0;
    for (int i = 0; i < count; ++i) {
        vne_status vs = validate(&Rs[i], p, mode);
        if (vs != VNE_OK) return vs;
        if (Rs[i].memory == VNE_MEM_HOST) {
            const size_t b = (size_t)(Rs[i].layout != VNE_DIA ? Rs[i].n : Rs[i].n_diags) *
                             (size_t)Rs[i].ld * elt_size(Rs[i].dtype);
            if (b > stage) stage = b;
            ++nhost;
        }
    }
    const double nan = std::nan("");
    for (int i = 0; i < count; ++i) {
        if (H_cheb && (mode & MODE_CHEB)) H_cheb[i] = nan;
        if (H_taylor && (mode & MODE_TAYLOR)) H_taylor[i] = nan;
        if (u_out) u_out[i] = nan;
    }
    DeviceGuard guard(h->device);
    if (nhost > 0) {
        vne_status vs = stage_resources(h, stage, nhost < 2 ? 1 : 2);
        if (vs != VNE_OK) return vs;
    }
    cudaStream_t user = (cudaStream_t)stream;
    std::vector<int> host_idx;
    for (int i = 0; i < count; ++i)
        if (Rs[i].memory == VNE_MEM_HOST) host_idx.push_back(i);
    // host matrix number j goes to slot j & 1; it is requested once matrix
    // j - 1 has been estimated (the single call returns synchronised), so the
    // slot's previous matrix, j - 2, is no longer read
    int issued = 0, ord = 0;
    auto request = [&](int j) -> cudaError_t {
        const vne_matrix& R = Rs[host_idx[j]];
        const size_t b = (size_t)(R.layout != VNE_DIA ? R.n : R.n_diags) * (size_t)R.ld *
                         elt_size(R.dtype);
        cudaError_t e = cudaMemcpyAsync(h->stage[j & 1], R.data, b, cudaMemcpyHostToDevice,
                                        h->cstream);
        if (e == cudaSuccess) e = cudaEventRecord(h->cev[j & 1], h->cstream);
        return e;
    };
    vne_status first = VNE_OK;
    for (int i = 0; i < count; ++i) {
        vne_matrix M = Rs[i];
        if (M.memory == VNE_MEM_HOST) {
            cudaError_t e = cudaSuccess;
            while (e == cudaSuccess && issued < nhost && issued <= ord + 1) e = request(issued++);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->cev[ord & 1], 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                first = map_err(h, e);
                break;
            }
            M.data = h->stage[ord & 1];
            M.memory = VNE_MEM_DEVICE;
            if (M.layout == VNE_DENSE_UPPER) {  // the slot is the handle's: mirror in place
                e = launch_dense_symmetrize(M.data, M.ld, h->stage[ord & 1], M.ld, M.n, M.dtype,
                                            user);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    first = map_err(h, e);
                    break;
                }
                ++h->launches;
                M.layout = VNE_DENSE;
            }
            ++ord;
        }
        Outputs o;
        if (mode & MODE_CHEB) o.H_cheb = &H_cheb[i];
        if (mode & MODE_TAYLOR) o.H_taylor = &H_taylor[i];
        o.u = u_out ? &u_out[i] : nullptr;
        vne_status r = run(h, &M, p, mode, o, stream);
        if (r != VNE_OK) {
            first = r;
            break;
        }
    }
    // no copy from the caller's memory is in flight once this returns
    if (h->cstream) {
        cudaError_t e = cudaStreamSynchronize(h->cstream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (first == VNE_OK) first = map_err(h, e);
        }
    }
    return first;
}

vne_status vne_tc_shape(int64_t n, int32_t ncols, int32_t sm_count, int32_t* shape_out) {
    if (!shape_out) return VNE_ERR_INVALID_ARG;
    int sh[4];
    if (tc_plan(n, ncols, sm_count, sh) != 0) return VNE_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) shape_out[k] = sh[k];
    return VNE_OK;
}

vne_status vne_tc_autotune(vne_handle* h, const vne_matrix* R, const vne_params* p,
                           int32_t method, int32_t* shape_out, double* us_out, void* stream) {
    if (!h || !R || !p) return VNE_ERR_INVALID_ARG;
    if (R->layout != VNE_DENSE || p->precision < VNE_PREC_BF16) return VNE_ERR_UNSUPPORTED;
    if (method != VNE_METHOD_TAYLOR && method != VNE_METHOD_CHEBYSHEV && method != VNE_METHOD_BOTH)
        return VNE_ERR_INVALID_ARG;
    const int mode = method == VNE_METHOD_TAYLOR ? MODE_TAYLOR
                     : method == VNE_METHOD_CHEBYSHEV ? MODE_CHEB : MODE_BOTH;
    const int S = mode == MODE_BOTH ? 2 * p->s : p->s;
    int cand[16][4];
    const int cnt = tc_candidates(R->n, S, cand, 16);
    if (cnt < 1) return VNE_ERR_UNSUPPORTED;
    const int saved_prof = h->prof_on;
    h->prof_on = 1;
    int best = -1;
    double best_us = 0.0;
    vne_status st = VNE_OK;
    for (int i = 0; i < cnt && st == VNE_OK; ++i) {
        tc_set_tuned(R->n, S, cand[i][0], cand[i][1], cand[i][2], cand[i][3]);
        Outputs o;
        double H = 0.0, H2 = 0.0;
        o.H_cheb = &H;
        o.H_taylor = &H2;
        st = run(h, R, p, mode, o, stream);  // warm-up (tensor maps, caches)
        if (st != VNE_OK) break;
        h->prof_ms[0] = 0.0;
        h->prof_n[0] = 0;
        st = run(h, R, p, mode, o, stream);
        if (st != VNE_OK) break;
        const double us = h->prof_n[0] > 0 ? h->prof_ms[0] * 1e3 / (double)h->prof_n[0] : 1e30;
        if (best < 0 || us < best_us) {
            best = i;
            best_us = us;
        }
    }
    h->prof_on = saved_prof;
    for (int k = 0; k < 4; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    if (st != VNE_OK || best < 0) {
        tc_set_tuned(R->n, S, 0, 0, 0, 0);
        return st != VNE_OK ? st : VNE_ERR_UNSUPPORTED;
    }
    tc_set_tuned(R->n, S, cand[best][0], cand[best][1], cand[best][2], cand[best][3]);
    if (shape_out)
        for (int k = 0; k < 4; ++k) shape_out[k] = cand[best][k];
    if (us_out) *us_out = best_us;
    return VNE_OK;
}

vne_status vne_selftest_timeout(vne_handle* h, void* stream) {
    if (!h) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    vne_status vs = ensure_ws(h, SC_COUNT * sizeof(double) + 4096);
    if (vs != VNE_OK) return vs;
    double* sc = reinterpret_cast<double*>(h->ws);
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(sc, 0, SC_COUNT * sizeof(double), st);
    if (e == cudaSuccess) e = launch_wait_never(sc, st);
    h->launches++;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->host_sc, sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return map_err(h, e);
    return slot_status(h->host_sc, 0);
}

vne_status vne_lambda_max(vne_handle* h, const vne_matrix* R, const vne_params* p,
                          double* lam_out, void* stream) {
    if (!lam_out) return VNE_ERR_INVALID_ARG;
    if (p && p->u_override > 0.0) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.lam = lam_out;
    return run(h, R, p, MODE_POWER, o, stream);
}

vne_status vne_combine_moments(vne_handle* h, int32_t m, int32_t s, double u,
                               const double* moments_cheb, const double* moments_taylor,
                               double* H_cheb, double* H_taylor, void* stream) {
    if (!h || m < 1 || s < 1 || m > 100000) return VNE_ERR_INVALID_ARG;
    if (!moments_cheb && !moments_taylor) return VNE_ERR_INVALID_ARG;
    if ((moments_cheb && !H_cheb) || (moments_taylor && !H_taylor)) return VNE_ERR_INVALID_ARG;
    if ((int64_t)(m + 1) * s > ((int64_t)1 << 31)) return VNE_ERR_INVALID_ARG;
    if (!(u > 0.0) || !(u <= 1.0)) return VNE_ERR_BAD_INTERVAL;
    DeviceGuard guard(h->device);
    const size_t per = (size_t)(m + 1) * s;
    Bump b0(nullptr);
    b0.take<double>(SC_COUNT);
    b0.take<double>(per);
    b0.take<double>(per);
    vne_status vs = ensure_ws(h, b0.off + 4096);
    if (vs != VNE_OK) return vs;
    Bump b1(h->ws);
    double* sc = b1.take<double>(SC_COUNT);
    double* mc = b1.take<double>(per);
    double* mt = b1.take<double>(per);
    Call c{h, (cudaStream_t)stream};
    c.chk(cudaMemsetAsync(sc, 0, SC_COUNT * sizeof(double), c.st));
    if (moments_cheb)
        c.chk(cudaMemcpyAsync(mc, moments_cheb, per * sizeof(double), cudaMemcpyHostToDevice, c.st));
    if (moments_taylor)
        c.chk(cudaMemcpyAsync(mt, moments_taylor, per * sizeof(double), cudaMemcpyHostToDevice,
                              c.st));
    if (c.ok()) c.launched(launch_set_u(sc, u, c.st));
    if (c.ok())
        c.launched(launch_combine_final(s, m, moments_cheb ? mc : nullptr,
                                        moments_taylor ? mt : nullptr, sc, c.st));
    if (c.ok())
        c.chk(cudaMemcpyAsync(h->host_sc, sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                              c.st));
    c.chk(cudaStreamSynchronize(c.st));
    if (!c.ok()) {
        cudaGetLastError();
        return map_err(h, c.err);
    }
    const vne_status fs = slot_status(h->host_sc, 0);
    if (fs != VNE_OK) return fs;
    if (moments_cheb) *H_cheb = h->host_sc[SC_H_CHEB];
    if (moments_taylor) *H_taylor = h->host_sc[SC_H_TAYLOR];
    return VNE_OK;
}

vne_status vne_entropy_projection(vne_handle* h, const vne_matrix* R, int32_t k, int32_t s,
                                  int32_t sketch, int32_t krylov_iters, int32_t precision,
                                  uint64_t seed, double* H_out, double* p_out, void* stream) {
    if (!h || !R || !H_out || !R->data) return VNE_ERR_INVALID_ARG;
    if (R->n < 1 || R->ld < R->n) return VNE_ERR_INVALID_ARG;
    if (R->dtype != VNE_F64 && R->dtype != VNE_F32) return VNE_ERR_INVALID_ARG;
    if (R->memory != VNE_MEM_DEVICE && R->memory != VNE_MEM_HOST) return VNE_ERR_INVALID_ARG;
    if (R->layout != VNE_DENSE && R->layout != VNE_DIA) return VNE_ERR_INVALID_ARG;
    if (s < 1 || k < 1 || (krylov_iters <= 0 && k > s)) return VNE_ERR_INVALID_ARG;
    if (sketch < VNE_SKETCH_GAUSSIAN || sketch > VNE_SKETCH_COUNT) return VNE_ERR_INVALID_ARG;
    if (precision < VNE_PREC_F64 || precision > VNE_PREC_BF16X6 || krylov_iters < 0)
        return VNE_ERR_INVALID_ARG;
    if (R->layout != VNE_DENSE || s > 512 || precision == VNE_PREC_BF16 || is_complex(R->dtype))
        return VNE_ERR_UNSUPPORTED;
    // the split modes run R Pi (and R Q_j) on the tensor cores, FP32 results
    const int pieces = precision == VNE_PREC_BF16X3 ? 2 : precision == VNE_PREC_BF16X6 ? 3 : 0;
    if ((int64_t)s * R->n > ((int64_t)1 << 40)) return VNE_ERR_UNSUPPORTED;
    if (krylov_iters > 0) {
        if (s > 64 || (int64_t)krylov_iters * s > 512) return VNE_ERR_UNSUPPORTED;
        if (k > krylov_iters * s) return VNE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(h->device);
    if (krylov_iters > 0) {
        if (precision == VNE_PREC_F64)
            return run_krylov<double>(h, *R, k, s, krylov_iters, sketch, seed, H_out, p_out,
                                      (cudaStream_t)stream);
        return run_krylov<float>(h, *R, k, s, krylov_iters, sketch, seed, H_out, p_out,
                                 (cudaStream_t)stream, pieces);
    }
    if (precision == VNE_PREC_F64)
        return run_projection<double>(h, *R, k, s, sketch, seed, H_out, p_out, (cudaStream_t)stream);
    return run_projection<float>(h, *R, k, s, sketch, seed, H_out, p_out, (cudaStream_t)stream,
                                 pieces);
}

vne_status vne_entropy_chebyshev_learned(vne_handle* h, const vne_matrix* R, const vne_params* p,
                                         const float* params, double* H_out,
                                         double* H_plain_out, double* u_out, void* stream) {
    if (!H_out || !params || !p) return VNE_ERR_INVALID_ARG;
    if (p->m < VNE_MLP_N_MOMENTS - 1 || p->probe != VNE_GAUSSIAN) return VNE_ERR_INVALID_ARG;
    Outputs o;
    o.H_cheb = H_plain_out;
    o.u = u_out;
    o.mlp = params;
    o.H_learned = H_out;
    return run(h, R, p, MODE_CHEB, o, stream);
}

vne_status vne_spectral_samples(vne_handle* h, int32_t count, const int32_t* kind,
                                const int32_t* n, const float* a, const int32_t* ktop,
                                const float* floor, const float* c, const uint64_t* seeds,
                                int32_t m, int32_t s, float* features, float* target,
                                double* H_exact, double* H_low, double* totals, void* stream) {
    if (!h || count < 1 || s < 1 || !kind || !n || !a || !ktop || !floor || !c || !seeds ||
        !features || !target || !H_exact || !H_low)
        return VNE_ERR_INVALID_ARG;
    if (m < VNE_MLP_N_MOMENTS - 1 || m > 64) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    cudaError_t e = launch_spectral_sample(count, kind, n, a, ktop, floor, c, seeds, m, s, features,
                                           target, H_exact, H_low, totals, (cudaStream_t)stream);
    h->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return map_err(h, e);
}

namespace {
// workspace of the network calls: activations, row indices, gradient, loss
struct MlpWs {
    float* act;
    int* idx;
    float* grad;
    double* loss;
};
vne_status mlp_ws(vne_handle* h, int B, MlpWs* w) {
    auto plan = [&](Bump& b) {
        w->act = b.take<float>(mlp_workspace_floats(B));
        w->idx = b.take<int>((size_t)B);
        w->grad = b.take<float>(VNE_MLP_N_PARAMS);
        w->loss = b.take<double>(1);
    };
    Bump b0(nullptr);
    plan(b0);
    vne_status vs = ensure_ws(h, b0.off + 4096);
    if (vs != VNE_OK) return vs;
    Bump b1(h->ws);
    plan(b1);
    return VNE_OK;
}
}  // namespace

vne_status vne_mlp_forward(vne_handle* h, const float* params, const float* X, int32_t batch,
                           float* y, void* stream) {
    if (!h || !params || !X || !y || batch < 1) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    MlpWs w;
    vne_status vs = mlp_ws(h, batch, &w);
    if (vs != VNE_OK) return vs;
    int cnt = 0;
    cudaError_t e = mlp_forward(params, X, batch, y, w.act, &cnt, (cudaStream_t)stream);
    h->launches += cnt;
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return map_err(h, e);
}

vne_status vne_mlp_gradient(vne_handle* h, const float* params, const float* X,
                            const float* target, int32_t batch, float* grad, double* loss_out,
                            void* stream) {
    if (!h || !params || !X || !target || !grad || batch < 1) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    MlpWs w;
    vne_status vs = mlp_ws(h, batch, &w);
    if (vs != VNE_OK) return vs;
    int cnt = 0;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp_loss_grad(params, X, target, nullptr, batch, grad, w.loss, w.act, &cnt, st);
    h->launches += cnt;
    double loss = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && loss_out) *loss_out = loss;
    return map_err(h, e);
}

vne_status vne_mlp_train_step(vne_handle* h, float* params, float* adam_m, float* adam_v,
                              int32_t step, float lr, const float* X, const float* target,
                              int64_t rows, int32_t batch, int64_t first, uint64_t perm_seed,
                              double* loss_out, void* stream) {
    if (!h || !params || !adam_m || !adam_v || !X || !target || step < 1 || rows < 1 ||
        batch < 1 || first < 0 || !(lr > 0.f))
        return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    MlpWs w;
    vne_status vs = mlp_ws(h, batch, &w);
    if (vs != VNE_OK) return vs;
    int cnt = 0;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp_train_step(params, adam_m, adam_v, step, lr, X, target, rows, batch, first,
                                   perm_seed, w.idx, w.grad, w.loss, w.act, &cnt, st);
    h->launches += cnt;
    if (e == cudaSuccess && loss_out) {
        double loss = 0.0;
        e = cudaMemcpyAsync(&loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) *loss_out = loss;
    }
    return map_err(h, e);
}

vne_status vne_sketch_block(vne_handle* h, int64_t n, int32_t s, int32_t sketch, uint64_t seed,
                            double* out, void* stream) {
    if (!h || !out || n < 1 || s < 1) return VNE_ERR_INVALID_ARG;
    if (sketch < VNE_SKETCH_GAUSSIAN || sketch > VNE_SKETCH_COUNT) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    cudaError_t e = launch_sketch<double>(out, n, s, sketch, seed, h->sm_count, (cudaStream_t)stream);
    h->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return map_err(h, e);
}

vne_status vne_probe_block(vne_handle* h, int64_t n, int32_t s, int32_t probe, uint64_t seed,
                           double* out, void* stream) {
    if (!h || !out || n < 1 || s < 1) return VNE_ERR_INVALID_ARG;
    if (probe != VNE_RADEMACHER && probe != VNE_GAUSSIAN) return VNE_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    cudaError_t e = launch_probe_block_f64(out, n, s, probe, seed, (cudaStream_t)stream);
    h->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return map_err(h, e);
}

vne_status vne_profile_enable(vne_handle* h, int32_t on) {
    if (!h) return VNE_ERR_INVALID_ARG;
    h->prof_on = on ? 1 : 0;
    return VNE_OK;
}

vne_status vne_profile_read(vne_handle* h, int32_t kind, double* total_ms, int64_t* launches) {
    if (!h || kind < 0 || kind > 3) return VNE_ERR_INVALID_ARG;
    if (total_ms) *total_ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_n[kind];
    return VNE_OK;
}

vne_status vne_profile_reset(vne_handle* h) {
    if (!h) return VNE_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    return VNE_OK;
}

int64_t vne_launch_count(const vne_handle* h) { return h ? h->launches : -1; }

const char* vne_status_string(vne_status s) {
    switch (s) {
        case VNE_OK: return "VNE_OK";
        case VNE_ERR_INVALID_ARG: return "VNE_ERR_INVALID_ARG";
        case VNE_ERR_NOT_UNIT_TRACE: return "VNE_ERR_NOT_UNIT_TRACE";
        case VNE_ERR_BAD_INTERVAL: return "VNE_ERR_BAD_INTERVAL";
        case VNE_ERR_OOM: return "VNE_ERR_OOM";
        case VNE_ERR_CUDA: return "VNE_ERR_CUDA";
        case VNE_ERR_TIMEOUT: return "VNE_ERR_TIMEOUT";
        case VNE_ERR_NONFINITE: return "VNE_ERR_NONFINITE";
        case VNE_ERR_UNSUPPORTED: return "VNE_ERR_UNSUPPORTED";
    }
    return "VNE_ERR_UNKNOWN";
}

int32_t vne_last_cuda_error(const vne_handle* h) { return h ? h->last_err : 0; }

int32_t vne_suggest_m(int32_t method, double u, double ell, double eps) {
    if (!(u > 0.0 && u <= 1.0) || !(ell > 0.0 && ell <= u) || !(eps > 0.0 && eps < 1.0)) return -1;
    double m;
    if (method == VNE_METHOD_TAYLOR) m = std::ceil((u / ell) * std::log(1.0 / eps));
    else if (method == VNE_METHOD_CHEBYSHEV)
        m = std::ceil(std::sqrt(u / (2.0 * eps * ell * std::log(1.0 / (1.0 - ell)))));
    else return -1;
    if (!(m < 2.0e9)) return -1;
    return (int32_t)m;
}

}  // extern "C"
