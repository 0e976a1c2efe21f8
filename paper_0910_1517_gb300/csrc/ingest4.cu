// ingest4.cu -- ADC-format ingest of the paper's 33 MHz, 4-bit mode (Sec. 2.3.1, 2.3.2): each
// ADC card interleaves 4 inputs sample by sample, 4 bits each; the stream is demultiplexed into
// the 4 inputs' int8 rows, every 4-bit sample sign-extended.  Byte 2s of card c holds inputs 4c
// (bits 0-3) and 4c+1 (bits 4-7) of sample s, byte 2s+1 inputs 4c+2 and 4c+3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

__device__ __forceinline__ int8_t sext4(uint32_t nib) { return static_cast<int8_t>(static_cast<int>(nib << 28) >> 28); }

// grid-stride over (card, sample): one 2-byte load, four byte stores into consecutive samples of
// the four rows (coalesced across the warp)
__global__ void unpack4_kernel(const uint8_t* __restrict__ packed, int64_t ld, int n_cards, int64_t n,
                               int8_t* __restrict__ rows, int64_t ldr) {
    const int64_t total = static_cast<int64_t>(n_cards) * n;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(q / n);
        const int64_t s = q - static_cast<int64_t>(c) * n;
        const uint32_t w = *reinterpret_cast<const uint16_t*>(packed + c * ld + 2 * s);
        int8_t* r = rows + static_cast<int64_t>(4 * c) * ldr + s;
        r[0] = sext4(w & 0xFu);
        r[ldr] = sext4((w >> 4) & 0xFu);
        r[2 * ldr] = sext4((w >> 8) & 0xFu);
        r[3 * ldr] = sext4((w >> 12) & 0xFu);
    }
}

}  // namespace

cudaError_t launch_unpack4(const uint8_t* packed, int64_t ld, int n_cards, int64_t n, int8_t* rows, int64_t ldr,
                           int n_sm, cudaStream_t s) {
    if (n_cards < 1 || n < 0 || (ld & 1) || ld < 2 * n || ldr < n) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    const int64_t total = static_cast<int64_t>(n_cards) * n;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(n_sm) * 16));
    unpack4_kernel<<<grid, 256, 0, s>>>(packed, ld, n_cards, n, rows, ldr);
    return cudaGetLastError();
}

}  // namespace gbx
