// selftest.cu -- failure detection without a GPU fault: a kernel whose wait can never complete
// (an mbarrier expecting two arrivals that never come) must give up after the clock budget that
// bounds every pipeline wait of this library, record its error bit in the device error word and
// return, leaving the context usable for the next launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/corr.h"
#include "common.cuh"
#include "handle.cuh"

namespace gbx {
namespace {

constexpr unsigned kCompleted = 0x80000000u;   // the wait returned true: it should not have

__global__ void wait_selftest_kernel(unsigned* err, long long* cycles) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        const bool ok = mbar_wait(&bar, 0, err, ERR_WAIT_STAGE);   // phase 0 needs two arrivals: none come
        *cycles = clock64() - t0;
        if (ok) atomicOr(err, kCompleted);
    }
}

}  // namespace
}  // namespace gbx

using namespace gbx;

extern "C" int corr_wait_selftest(long long* cycles_out) {
    unsigned* d_err = nullptr;
    long long* d_cyc = nullptr;
    if (cudaMalloc(&d_err, sizeof(unsigned)) != cudaSuccess) return fail_code(CORR_E_CUDA, "cudaMalloc");
    if (cudaMalloc(&d_cyc, sizeof(long long)) != cudaSuccess) {
        cudaFree(d_err);
        return fail_code(CORR_E_CUDA, "cudaMalloc");
    }
    unsigned err = 0;
    long long cyc = 0;
    cudaError_t e = cudaMemset(d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32>>>(d_err, d_cyc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&err, d_err, sizeof err, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&cyc, d_cyc, sizeof cyc, cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    cudaFree(d_cyc);
    if (e != cudaSuccess) return fail_code(CORR_E_CUDA, cudaGetErrorString(e));
    if (cycles_out) *cycles_out = cyc;
    if ((err & ERR_WAIT_STAGE) == 0 || (err & kCompleted)) return fail_code(CORR_E_STATE, "the wait did not give up");
    return CORR_OK;
}
