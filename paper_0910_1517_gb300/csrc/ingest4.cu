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

// four 4-bit values in the low nibbles of the bytes of x (high nibbles zero), each sign-extended
// to its byte: bit 3 set adds 0xF0 to that byte (0x08 * 0x1E = 0xF0, no carry between bytes)
__device__ __forceinline__ uint32_t sext4x4(uint32_t x) { return x | ((x & 0x08080808u) * 0x1Eu); }

// Card c = blockIdx.y.  The four output rows share their alignment (ldr % 16 == 0): samples
// [h, h + 16 nb) form 16-sample blocks whose output is one aligned 16-byte store per row and
// whose input is 32 bytes (two 16-byte loads when aligned, else 2-byte loads); the head
// [0, h) and the tail [h + 16 nb, n) (under 32 samples) go one sample per thread.
__global__ void unpack4_kernel(const uint8_t* __restrict__ packed, int64_t ld, int64_t n,
                               int8_t* __restrict__ rows, int64_t ldr) {
    const int c = blockIdx.y;
    const uint8_t* in = packed + c * ld;
    int8_t* out = rows + static_cast<int64_t>(4 * c) * ldr;
    const int64_t h0 = (16 - static_cast<int64_t>(reinterpret_cast<uintptr_t>(out) & 15)) & 15;
    const int64_t h = n < h0 ? n : h0;
    const int64_t nb = (n - h) >> 4;
    const int64_t t0 = h + 16 * nb;
    const int64_t items = nb + h + (n - t0);
    const bool aligned = (reinterpret_cast<uintptr_t>(in + 2 * h) & 15) == 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < items; q += stride) {
        if (q < nb) {
            const int64_t s = h + 16 * q;
            uint32_t u[8];
            if (aligned) {
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(in + 2 * s));
                const uint4 b = __ldg(reinterpret_cast<const uint4*>(in + 2 * s + 16));
                u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
                u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
            } else {
                const uint16_t* w = reinterpret_cast<const uint16_t*>(in + 2 * s);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    u[j] = static_cast<uint32_t>(__ldg(w + 2 * j)) | (static_cast<uint32_t>(__ldg(w + 2 * j + 1)) << 16);
            }
            uint32_t r[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // e: the even bytes of samples s+4j .. s+4j+3 (inputs 4c, 4c+1), o: the odd bytes (4c+2, 4c+3)
                const uint32_t e = __byte_perm(u[2 * j], u[2 * j + 1], 0x6420);
                const uint32_t o = __byte_perm(u[2 * j], u[2 * j + 1], 0x7531);
                r[0][j] = sext4x4(e & 0x0F0F0F0Fu);
                r[1][j] = sext4x4((e >> 4) & 0x0F0F0F0Fu);
                r[2][j] = sext4x4(o & 0x0F0F0F0Fu);
                r[3][j] = sext4x4((o >> 4) & 0x0F0F0F0Fu);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<uint4*>(out + i * ldr + s) = make_uint4(r[i][0], r[i][1], r[i][2], r[i][3]);
        } else {
            const int64_t k = q - nb;
            const int64_t s = k < h ? k : t0 + (k - h);
            const uint32_t w = *reinterpret_cast<const uint16_t*>(in + 2 * s);
            out[s] = sext4(w & 0xFu);
            out[ldr + s] = sext4((w >> 4) & 0xFu);
            out[2 * ldr + s] = sext4((w >> 8) & 0xFu);
            out[3 * ldr + s] = sext4((w >> 12) & 0xFu);
        }
    }
}

}  // namespace

cudaError_t launch_unpack4(const uint8_t* packed, int64_t ld, int n_cards, int64_t n, int8_t* rows, int64_t ldr,
                           int n_sm, cudaStream_t s) {
    if (n_cards < 1 || n_cards > 65535 || n < 0 || (ld & 1) || ld < 2 * n || ldr < n || (ldr & 15) ||
        (reinterpret_cast<uintptr_t>(packed) & 1))
        return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    const int64_t per_card = n / 16 + 32;
    const int64_t cap = std::max<int64_t>(1, static_cast<int64_t>(n_sm) * 8 / n_cards);
    const dim3 grid(static_cast<unsigned>(std::min<int64_t>((per_card + 255) / 256, cap)), n_cards);
    unpack4_kernel<<<grid, 256, 0, s>>>(packed, ld, n, rows, ldr);
    return cudaGetLastError();
}

}  // namespace gbx
