// Check of the bounded-wait path: every mbarrier wait of the library gives up
// after a deadline, sets FLAG_TIMEOUT and lets its kernel return, so that a
// lost arrival becomes VNE_ERR_TIMEOUT and the context stays usable.  This
// kernel waits on a barrier that nothing arrives on.
#include "vne_common.cuh"
#include "vne_internal.h"
#include "vne_ptx.cuh"

namespace vne {

__global__ void k_wait_never(double* sc) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool got = mbar_wait(&bar, 0u, &abort_flag);  // no arrival ever comes
        if (!got) {
            unsigned long long* f = reinterpret_cast<unsigned long long*>(sc + SC_FLAGS);
            *f |= FLAG_TIMEOUT;
        }
    }
}

cudaError_t launch_wait_never(double* sc, cudaStream_t st) {
    k_wait_never<<<1, 32, 0, st>>>(sc);
    return cudaGetLastError();
}

}  // namespace vne
