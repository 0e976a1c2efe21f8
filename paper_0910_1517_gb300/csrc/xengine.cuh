// xengine.cuh -- launch interface of the X-engines (MAC over all N(N+1)/2
// baselines x n_pol^2 products, Sec. 2.1).
#pragma once
#include <cuda.h>
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
    float2* vis_part;      // CUDA-core engine: room for max_split partial visibility sets, or nullptr
    int max_split;
    int self;              // 1: self-polar (total-intensity) mode, only products pp, vis [n_chan][n_bl][n_pol]
};

// Index of product (p, q) within a baseline's products: full-polar p n_pol + q (RR*, RL*, LR*, LL*),
// self-polar p (RR*, LL*; only p = q exists)
__host__ __device__ constexpr int vis_prod(int self, int n_pol, int p, int q) { return self ? p : p * n_pol + q; }

// Plain FP32 X-engine on CUDA cores: register-tiled upper-triangular complex MAC.
cudaError_t launch_xengine_fp32(const XParams& p, int n_sm, cudaStream_t s);

// tcgen05 X-engine: G = A A^T per channel on the tensor cores, TMEM accumulators, over a
// table of sub-arrays and a list of (sub-array, channel, row block) items that the persistent
// CTAs stride (every wide item before the narrow ones, so that both kinds reach every CTA).
constexpr int kMaxSubX = 8;
constexpr int kStageMaxBytes = 32768;        // bytes of one operand stage (ks/8 K-blocks x 2 n_in rows x 16 B)
constexpr int kStage2Bytes = 32768;          // FP32 form: bytes of one FP32 stage (ks x rows_fp32(n_in) x 4 B)
struct alignas(128) XtSub {   // (the tensor map's own alignment)
    // FP32 form with quad = 1: the spectra are in the channel-quad layout (f32q_piece) and each
    // stage is one TMA copy through this 5-D tensor map over (16 floats, channel in quad, input,
    // K-block, quad), box (16, 1, n_in, ks / 8, 1); it lands [kb][2 n_in rows][8 frames]
    CUtensorMap tmap;
    int quad;
    const __half* spec;    // [k][kb][2 n_in][8] fp16 K-block layout
    // in8 = 1: spec holds the same layout in int8 bytes (rows of 8 bytes, the F-engine's OUT_I8B);
    // each stage lands in an input slot and converter warps widen it to the fp16 operand tile
    int in8;
    int n_ant, n_pol, n_in, n_chan, n_int;
    const float* scale;    // [n_in][n_chan]
    float2* vis;           // [n_chan][n_bl][n_pol^2]
    int2* vis_int;         // exact integer sums (int8-valued operands) or nullptr
    int exact;
    int ks;                // frames per operand stage: power of two, 16..512, ks/8 * 2 n_in * 16 <= kStageMaxBytes
                           // (FP32 form: ks * rows_fp32(n_in) * 4 <= kStage2Bytes)
    // FP32 form on the tensor cores: spec32 holds the FP32 spectra (the CUDA-core engine's
    // layout); each stage is split on chip into fp16 hi + lo planes of v = Y * split_scale, and
    // G = H H^T + H L^T + L H^T is multiplied by descale instead of divided by scale products.
    // nullptr: spec holds one fp16 plane.
    const float* spec32;
    float split_scale, descale;
    int chunk;             // frames per TMEM accumulation chunk: power of two, multiple of ks
    int self;              // self-polar mode: only products pp are written, vis [n_chan][n_bl][n_pol]
};
struct XtBatch {          // (the converted forms, spec32 or in8 set, run alone: launch with their form)
    int n_sub;
    XtSub sub[kMaxSubX];
    int n_items;
    const int4* items;     // (sub, channel, row block, 0)
    unsigned* err;
};
// Encode the tensor map of sub-array x's quad-layout FP32 spectra (x.spec32, x.n_in, x.n_chan,
// x.n_int, x.ks); false if the driver refuses it
bool xengine_tc_encode_quad(XtSub& x);
bool xengine_tc_supported(int n_in);                 // 2 n_in <= 256
int xengine_tc_max_ks(int n_in);                      // largest fp16 stage for the row count
int xengine_tc_ks_fp32(int n_in);                     // largest FP32-form stage (FP32 slot <= kStage2Bytes)
size_t xengine_tc_smem();
// form of every sub-array of the table: one fp16 plane (XT_FORM_F16), FP32 split on chip (spec32,
// XT_FORM_F32) or int8 bytes widened on chip (in8, XT_FORM_I8)
enum XtForm : int { XT_FORM_F16 = 0, XT_FORM_F32 = 1, XT_FORM_I8 = 2 };
cudaError_t launch_xengine_tc_table(const XtBatch* dtab, int n_items, int n_sm, cudaStream_t s, int form = XT_FORM_F16);

}  // namespace gbx
