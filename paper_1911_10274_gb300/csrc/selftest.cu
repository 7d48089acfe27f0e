// selftest.cu -- proves the failure path of the bounded device waits without
// faulting the GPU.
//
// Every mbarrier wait in the library's kernels (TMA staging of the step
// kernels, the batch engine, the tensor-core GEMM) polls at most spin_limit
// times, then records the failure in a device flag that the host turns into
// TITAN_E_TIMEOUT.  Nothing in a healthy run makes one of those waits expire,
// so this entry point launches a one-CTA kernel whose thread waits on an
// mbarrier that nothing ever arrives on.  The wait must give up after its
// limit, the flag must reach the host, and the CUDA context must stay usable.
// No copy is ever in flight, so giving up leaves nothing behind.
#include <string>

#include "ptx.cuh"
#include "titan.h"

namespace titan {
void set_thread_error(const std::string &msg);   // defined in runtime.cu
}

namespace {

__global__ void k_wait_unarrived(uint32_t spin_limit, int *__restrict__ flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        titan::ptx::mbar_init(&bar, 1);      // one arrival expected; none comes
        titan::ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) *flag = titan::ptx::mbar_wait_bounded(&bar, 0, spin_limit) ? 2 : 1;
}

titan_status fail(titan_status st, const std::string &msg) {
    titan::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" titan_status titan_selftest_wait_timeout(int32_t device, uint32_t spin_limit) {
    if (spin_limit == 0 || spin_limit > (1u << 20))
        return fail(TITAN_E_INVALID, "titan_selftest_wait_timeout: spin_limit must be in [1, 2^20]");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(TITAN_E_CUDA, std::string("titan_selftest_wait_timeout: ") + cudaGetErrorString(e));
    int *flag = nullptr;
    int host = 0;
    titan_status st = TITAN_OK;
    std::string msg;
    if ((e = cudaMalloc(&flag, sizeof(int))) == cudaSuccess && (e = cudaMemset(flag, 0, sizeof(int))) == cudaSuccess) {
        k_wait_unarrived<<<1, 32>>>(spin_limit, flag);
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaDeviceSynchronize()) == cudaSuccess)
            e = cudaMemcpy(&host, flag, sizeof(int), cudaMemcpyDeviceToHost);
    }
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) {
        st = TITAN_E_CUDA;
        msg = std::string("titan_selftest_wait_timeout: ") + cudaGetErrorString(e);
    } else if (host == 1) {
        st = TITAN_E_TIMEOUT;
        msg = "titan_selftest_wait_timeout: the bounded wait expired (expected)";
    } else {
        st = TITAN_E_CUDA;
        msg = "titan_selftest_wait_timeout: the wait on an unarrived mbarrier did not expire";
    }
    cudaSetDevice(prev);
    return fail(st, msg);
}
