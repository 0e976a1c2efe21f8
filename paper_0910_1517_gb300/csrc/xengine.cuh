// xengine.cuh -- launch interface of the X-engines (MAC over all N(N+1)/2
// baselines x n_pol^2 products, Sec. 2.1).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace gbx {

struct XParams {
    const void* spec;      // K-block layout spectra (fp32 for the CUDA-core engine, fp16 for tcgen05)
    int n_ant, n_pol, n_in, n_chan, n_int;
    const float* scale;    // [n_in][n_chan] requantisation scales (tensor-core engine) or nullptr
    float2* vis;           // [n_chan][n_bl][n_pol^2]
    int2* vis_int;         // [n_chan][n_bl][n_pol^2] exact integer sums (I8) or nullptr
    unsigned* err;
    int exact;             // tensor-core engine: 1 = int8-valued operands, integer flush
};

// Plain FP32 X-engine on CUDA cores: register-tiled upper-triangular complex MAC.
cudaError_t launch_xengine_fp32(const XParams& p, int n_sm, cudaStream_t s);

// tcgen05 X-engine: G = A A^T per channel on the tensor cores, TMEM accumulators.
// Supports 2*n_in <= 128.
cudaError_t launch_xengine_tc(const XParams& p, int n_sm, cudaStream_t s);
bool xengine_tc_supported(int n_in);

}  // namespace gbx
