// fa_selftest_wait_timeout: runs the bounded mbarrier wait of the staged tile
// loads against a barrier phase that can never complete, so that the timed-out
// path (flag in the status block, kernel returns, context stays usable) can be
// exercised on purpose without faulting or hanging the GPU.
#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

// One thread initialises an mbarrier that expects two arrivals, arrives once
// and waits for the phase with the same helper (and limit handling) as the
// tile solve's staged loads.  No copy is issued, so nothing is in flight when
// the wait gives up.
__global__ void k_wait_selftest(StatusBlock *st, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        st->flags = 0;
        st->count = 0;
        st->first = NO_INDEX;
        mbar_init(&bar, 2);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive(&bar);
        if (!mbar_wait(&bar, 0, limit_ns)) status_report(st, FA_FLAG_TIMEOUT, 1, NO_INDEX);
    }
}

}  // namespace fa

extern "C" fa_status fa_selftest_wait_timeout(int64_t limit_ns, int32_t *d_status, void *stream) {
    if (!d_status || ((uintptr_t)d_status & 7) || limit_ns < 0 || limit_ns > 10000000000ll)
        return FA_ERR_INVALID_ARG;
    fa::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<fa::StatusBlock *>(d_status), (uint64_t)limit_ns);
    return cudaGetLastError() == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
