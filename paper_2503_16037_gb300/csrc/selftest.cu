// Self-test of the bounded device wait that the pipelined passes use: one
// thread waits, with the passes' own helper (a bounded number of polls of an
// mbarrier phase, then STATUS_TIMEOUT in the status word), on a barrier that
// receives its single expected arrival (arrive = 1) or none (arrive = 0).
// Nothing else runs in the kernel, so a wait that runs out leaves no copy in
// flight and the context stays usable.
#include <cuda_runtime.h>

#include <chrono>

#include "kern.h"
#include "stage.cuh"
#include "tursca.h"

namespace tk {

__global__ void k_wait_probe(int arrive, int *status) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(smem_addr(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) mbar_arrive(smem_addr(&bar));
    pipe_wait(smem_addr(&bar), 0u, &abort_flag, status, false);
}

}  // namespace tk

extern "C" tursca_status tursca_selftest_wait(void *cuda_stream, int arrive, double *seconds) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *d = nullptr, h = 0;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return TURSCA_E_NOMEM;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
    const auto t0 = std::chrono::steady_clock::now();
    if (e == cudaSuccess) {
        tk::k_wait_probe<<<1, 32, 0, st>>>(arrive ? 1 : 0, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const auto t1 = std::chrono::steady_clock::now();
    cudaFree(d);
    if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
    if (e != cudaSuccess) return TURSCA_E_CUDA;
    return (h & tk::STATUS_TIMEOUT) ? TURSCA_E_TIMEOUT : TURSCA_OK;
}
