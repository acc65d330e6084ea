// Diagnostic for the device-side failure path: the bounded mbarrier wait that every
// warp-specialised kernel uses (tc_ptx.cuh), run against a barrier that nothing arrives at,
// with a short limit.  The wait gives up, raises the CTA's abort flag, and the kernel writes
// FM_ERR_TIMEOUT to the status word it was given and returns, so the context stays usable.
#include "fm_internal.cuh"
#include "tc_ptx.cuh"

namespace fm {
namespace {

using namespace tc;

__global__ void k_diag_bounded_wait(long long limit_cycles, int *status)
{
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    const uint32_t b = su32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);                     // one arrival expected; none is ever made
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_ab<32>(b, 0u, &abort_flag, limit_cycles);
        *status = ok ? (int)FM_OK : (abort_flag ? (int)FM_ERR_TIMEOUT : (int)FM_ERR_CUDA);
    }
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" fm_status fm_diag_bounded_wait(int64_t limit_cycles, int *dev_status_out, fm_stream stream)
{
    if (!dev_status_out) {
        set_error("invalid argument: dev_status_out is NULL");
        return FM_ERR_INVALID_ARG;
    }
    if (limit_cycles < 1 || limit_cycles > WAIT_CYCLES) {
        set_error("invalid argument: limit_cycles must be in [1, %lld]", (long long)WAIT_CYCLES);
        return FM_ERR_INVALID_ARG;
    }
    k_diag_bounded_wait<<<1, 32, 0, stream>>>((long long)limit_cycles, dev_status_out);
    FM_CK_LAUNCH();
    return FM_OK;
}
