// xengine_tc.cu -- X-engine on the tcgen05 tensor cores (sm_103a).
//
// Per channel k the visibilities are one dense contraction.  With the 2 n_in
// real rows A[r][t], r = 2i + c (c = 0 real, 1 imaginary part of Y_i[t]),
// the real Gram G = A A^T (K = n_int frames) holds every product:
//   Re V_ij = G[2i][2j] + G[2i+1][2j+1],  Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// A is the F-engine's K-block layout, which already is the no-swizzle K-major
// canonical operand layout (core matrices of 8 rows x 16 bytes), so one
// TMA-engine bulk copy per stage lands a ready operand tile and the same shared
// memory tile serves as both A and B.
//
// Work items are (sub-array, channel, row block): 128 Gram rows a0..a0+127 against
// columns b0..b0+N-1.  Up to 128 rows need one item (N <= 128, the rest of the 128
// rows is ignored); 256 rows need two (rows 0-127 x columns 0-255, rows 128-255 x
// columns 128-255).  A persistent CTA walks a cost-ordered item list; several
// sub-arrays of different sizes share one launch.
//
// Roles: warp 0 streams stages in (and owns the TMEM allocation), warp 1 issues
// tcgen05.mma from one thread.  One-plane forms (10 warps): warps 2-9 drain the
// accumulators (warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. Gram rows, and
// the column half (w - 2) / 4 of them; 168 registers a thread hold the running
// sums).  Converted forms (FP32 split, int8 bytes; 16 warps, 128 registers): warps 2-5 drain
// (all columns of their lanes, running sums in TMEM), warps 6-15 convert the input stages.
// Accumulation is chunked: every `chunk` frames the FP32 accumulator is drained
// and added into a running sum.  Items with N <= 128 rotate over four 128-column
// accumulators (the MMAs run up to three chunks ahead of the drain) and keep the
// running sums in the draining threads' registers (one Gram row per thread);
// wider items use one accumulator of N columns and a running sum in TMEM
// (columns 256-511).  For int8-valued operands (chunk 1024) every product is an
// integer of magnitude at most 127^2 = 16129 and a chunk sum at most 1024 * 16129 =
// 16,516,096 < 2^24, so the FP32 accumulator is exact and the running sum is kept
// as int32: the result equals the integer MAC.
//
// int8 form with byte operands (in8): the F-engine wrote the int8 values as bytes, so each stage
// lands in an input slot at half the fp16 size and the converter warps of the FP32 form widen it
// to the fp16 operand tile (exact: the fp16 bits 0x6400 | (b ^ 0x80) hold 1152 + b, one packed
// subtraction leaves b); one MMA per 16-frame step, chunks of 1024 frames over three rotating
// accumulators, int32 running sums in TMEM.
//
// FP32 form: the stages hold FP32 spectra in the CUDA-core engine's layout; ten
// converter warps split each FP32 value v (scaled by a power of two) into fp16
// hi (v rounded to 11 significant bits) and lo = v - hi rounded to fp16, so
// |v - hi - lo| <= 2^-22 |v|, and write both planes as canonical operand tiles;
// each 16-frame step then issues three MMAs, H H^T + H L^T + L H^T (the dropped
// L L^T is below 2^-22 of the product).  The F-engine thus writes FP32 once and
// the X-engine reads it once.  fp16 x fp16 products are exact in FP32, but the
// tensor core's FP32 accumulation drops low bits of every partial sum, a
// loss that grows with the accumulator's size and the number of steps.  So the
// dominant H H^T term is accumulated in 128-frame chunks that the CUDA cores add
// in FP32.  Items of 128 rows (64 inputs, the usual shape) are "paired": the
// converters lay each K-block out as its 128 hi rows followed by its 128 lo rows, so
// that one N = 256 MMA forms [H H^T | H L^T] = H [H; L]^T and a second, N = 128, adds
// L H^T onto the right half -- two MMAs per step instead of three (the tensor core's
// cost here is per instruction, nearly independent of N); two 256-column chunk
// accumulators fill TMEM, and the CUDA cores add both halves of every chunk into FP32
// running sums in shared memory.  Other narrow items keep three MMAs: the cross terms,
// 2^-11 of H H^T, go to a separate accumulator over the whole integration (columns
// 256-383), two chunk accumulators alternate in columns 0-255 and the running sums sit
// in columns 384-511.
#include <cudaTypedefs.h>

#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
namespace {

constexpr int kWarps1 = 10;                   // one-plane forms
constexpr int kWarps2 = 16;                   // FP32 form
constexpr int kEpiThreads1 = 8 * 32;          // drain threads, one-plane forms
constexpr int kEpiThreads2 = 4 * 32;          // drain threads, FP32 form
constexpr int kConvWarp0 = 6;                 // FP32 form: first converter warp
constexpr int kConvWarps = kWarps2 - kConvWarp0;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kStages = 5;                    // fp16 operand slots (one-plane forms)
constexpr int kSlot = kStageMaxBytes + 2048;  // rows past R stay in bounds
constexpr int kTailSlack = 32768;
// FP32 form: stages of kStage2Bytes of FP32 each, five in flight.  An operand slot takes ks * 2 n_in * 4 bytes plus the rows the
// 128-row MMA reads past R; ks * rows_fp32(n_in) * 4 <= kStage2Bytes bounds that by
// kStage2Bytes + (128 - 64) * 16 (R < 64 leaves more room).
constexpr int kOpStages2 = 2;                 // operand slots ...
constexpr int kF32Stages = 3;                 // ... the FP32 slots after them ...
constexpr int kRunBytes = 128 * 128 * 4;      // ... and the paired items' FP32 running sums, [column][row]
// int8 form: four operand slots, then five input slots of kStage2Bytes / 2 (an int8 stage is half
// the size of its fp16 operand tile)
constexpr int kOpStagesI8 = 4;
constexpr int kRawI8 = 5;
constexpr int kRawPitch = kStage2Bytes / 2;
constexpr int kInSlots = kRawI8 > kF32Stages ? kRawI8 : kF32Stages;
constexpr int kSlot2 = kStage2Bytes + 1024;
constexpr int kRunOff = kOpStages2 * kSlot2 + kF32Stages * kStage2Bytes;
constexpr int kSmemBytes = kRunOff + kRunBytes;
static_assert(kOpStagesI8 <= kStages && kOpStagesI8 * kSlot2 + kRawI8 * kRawPitch <= kSmemBytes, "int8-form slots");
static_assert(kStages * kSlot + kTailSlack <= kSmemBytes && kSmemBytes <= 227 * 1024 - 1024, "shared memory");
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColRun = 256;             // running-sum columns of wide items
constexpr int kAccBufs = 4;                   // 128-column accumulators of narrow items
constexpr uint32_t kColX = 256;               // FP32-form narrow items: the cross-term accumulator
constexpr uint32_t kColRun2 = 384;            // FP32-form narrow items: the running sums
constexpr int kXBit = 4;                      // the cross-term accumulator's parity bit in the phase words

struct Shared {
    uint64_t full[kStages];       // operand slot ready (bulk copy landed, or converted)
    uint64_t empty[kStages];      // operand slot consumed by the MMAs
    uint64_t f32full[kInSlots];     // input slot (FP32 or int8) landed
    uint64_t f32empty[kInSlots];    // input slot converted
    uint64_t accf[kAccBufs];
    uint64_t acce[kAccBufs];
    uint64_t xf;                  // cross-term accumulator complete (MMA -> epilogue)
    uint64_t xe;                  // cross-term accumulator drained (epilogue -> MMA)
    uint32_t taddr;
    int abort_flag;
    int consumed;                 // stages whose bulk copies the consumer has seen land
};

struct ItemGeo {
    int sub, k, a0, b0, N, R, ntb, n_stage, n_chunk, nkb_stage;
    int Rp, tb32, ntb32;   // FP32 form: padded rows, frames per FP32 K-block, FP32 K-blocks per channel
    bool dbl;      // N <= 128: rotating 128-column accumulators
    bool sep;      // dbl and a converted form: rotating chunk accumulators, TMEM running sums
    bool pair;     // sep, FP32 form, 128 rows: hi and lo rows of a K-block side by side, one N = 256 MMA
                   // H [H; L]^T and one L H^T per step into a 256-column chunk accumulator
    bool cross;    // sep and FP32 form otherwise: the cross terms in their own accumulator
    int nbuf;      // accumulators the item rotates over
};

__device__ __forceinline__ ItemGeo item_geo(const XtBatch& t, int it) {
    ItemGeo g;
    const int4 e = t.items[it];
    g.sub = e.x;
    g.k = e.y;
    const XtSub& s = t.sub[g.sub];
    g.R = 2 * s.n_in;
    g.a0 = 128 * e.z;
    g.b0 = (g.R > 128) ? g.a0 : 0;
    g.N = ((g.R - g.b0 + 15) / 16) * 16;
    g.Rp = rows_fp32(s.n_in);
    g.tb32 = tb_fp32(s.n_chan);
    g.ntb32 = s.n_int / g.tb32;
    g.dbl = g.N <= 128;
    g.sep = g.dbl && (s.spec32 != nullptr || s.in8);
    g.pair = g.sep && s.spec32 != nullptr && g.R == 128;
    g.cross = g.sep && s.spec32 != nullptr && !g.pair;
    g.nbuf = !g.dbl ? 1 : (g.sep ? (s.spec32 != nullptr ? 2 : 3) : kAccBufs);
    g.ntb = s.n_int / kTbHalf;
    g.nkb_stage = s.ks / kTbHalf;
    g.n_stage = (s.n_int + s.ks - 1) / s.ks;
    g.n_chunk = (s.n_int + s.chunk - 1) / s.chunk;
    return g;
}

// running sum + chunk sum: int32 for int8-valued operands (the FP32 chunk sum is an exact
// integer), FP32 otherwise
__device__ __forceinline__ uint32_t chunk_add(int exact, bool have, uint32_t run, uint32_t v) {
    if (exact) {
        const int x = __float2int_rn(__uint_as_float(v));
        return have ? static_cast<uint32_t>(static_cast<int>(run) + x) : static_cast<uint32_t>(x);
    }
    const float x = __uint_as_float(v);
    return __float_as_uint(have ? __uint_as_float(run) + x : x);
}

// Final sums of Gram row `row`, columns b0 + j0 .. b0 + j0 + W - 1 (every lane of the warp calls
// it): rows 2i and 2i+1 sit in adjacent lanes.  The even lane writes input pairs (i, j) for the
// first W/4 column pairs of the piece and the odd lane for the last W/4; per column pair each lane
// sends its partner the two sums the partner lacks.
template <int W>
__device__ __forceinline__ void write_piece(const XtSub& s, const ItemGeo& ig, int row, int j0,
                                            const uint32_t (&run)[W]) {
    constexpr int H = W / 2;                       // columns of the odd lane's half
    const int n_bl = s.n_ant * (s.n_ant + 1) / 2, npp = s.self ? s.n_pol : s.n_pol * s.n_pol;
    const bool odd = row & 1;
    const int i = row >> 1;
    // requantisation scales through the read-only path: the loads of every column pair can then
    // issue together instead of one L2 round trip per output behind the previous stores
    const float si = (!s.spec32 && i < s.n_in) ? __ldg(s.scale + static_cast<int64_t>(i) * s.n_chan + ig.k) : 1.0f;
#pragma unroll
    for (int jh = 0; jh < W / 4; ++jh) {
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, odd ? run[2 * jh] : run[2 * jh + H], 1);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, odd ? run[2 * jh + 1] : run[2 * jh + H + 1], 1);
        const int jp = jh + (odd ? W / 4 : 0);
        const int j = ((ig.b0 + j0) >> 1) + jp;
        // G[2i][2j], G[2i][2j+1], G[2i+1][2j], G[2i+1][2j+1]
        const uint32_t g_r0c0 = odd ? r0 : run[2 * jh];
        const uint32_t g_r0c1 = odd ? r1 : run[2 * jh + 1];
        const uint32_t g_r1c0 = odd ? run[2 * jh + H] : r0;
        const uint32_t g_r1c1 = odd ? run[2 * jh + H + 1] : r1;
        if (i >= s.n_in || j >= s.n_in) continue;
        const int a = i / s.n_pol, pp = i % s.n_pol, a2 = j / s.n_pol, qq = j % s.n_pol;
        if (a > a2 || (s.self && pp != qq)) continue;
        const int bl = a * s.n_ant - a * (a - 1) / 2 + (a2 - a);
        const int64_t o = (static_cast<int64_t>(ig.k) * n_bl + bl) * npp + vis_prod(s.self, s.n_pol, pp, qq);
        if (s.exact) {
            const float d = si * __ldg(s.scale + static_cast<int64_t>(j) * s.n_chan + ig.k);
            const int re = static_cast<int>(g_r0c0) + static_cast<int>(g_r1c1);
            const int im = static_cast<int>(g_r1c0) - static_cast<int>(g_r0c1);
            if (s.vis_int) s.vis_int[o] = make_int2(re, im);
            s.vis[o] = make_float2(static_cast<float>(re) / d, static_cast<float>(im) / d);
        } else {
            const float re = __uint_as_float(g_r0c0) + __uint_as_float(g_r1c1);
            const float im = __uint_as_float(g_r1c0) - __uint_as_float(g_r0c1);
            if (s.spec32) {
                s.vis[o] = make_float2(re * s.descale, im * s.descale);
            } else {
                const float d = si * __ldg(s.scale + static_cast<int64_t>(j) * s.n_chan + ig.k);
                s.vis[o] = make_float2(re / d, im / d);
            }
        }
    }
}

// One chunk of a wide item (N > 128, one accumulator at column 0): add this thread's W-column
// pieces (j_first, j_first + j_step, ...) into the running sums at kColRun, or write the final
// sums after the last chunk.
template <int W>
__device__ __forceinline__ void drain_wide(const XtSub& s, const ItemGeo ig, uint32_t tm, int row, int j_first,
                                           int j_step, int chunk) {
    const bool last = chunk == ig.n_chunk - 1;
    for (int j0 = j_first; j0 < ig.N; j0 += j_step) {   // this warp's pieces
        uint32_t v[W], rs[W];
        if constexpr (W == 32) {
            tmem_ld32(tm + j0, v);
            if (chunk > 0) tmem_ld32(tm + kColRun + j0, rs);
        } else {
            tmem_ld16(tm + j0, v);
            if (chunk > 0) tmem_ld16(tm + kColRun + j0, rs);
        }
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < W; ++e) rs[e] = chunk_add(s.exact, chunk > 0, rs[e], v[e]);
        if (!last) {
            if constexpr (W == 32) tmem_st32(tm + kColRun + j0, rs);
            else tmem_st16(tm + kColRun + j0, rs);
        } else {
            write_piece<W>(s, ig, row, j0, rs);
        }
    }
    if (!last) tmem_wait_st();
}

// One chunk of a converted-form narrow item (chunk accumulator b, running sums at kColRun2; the
// FP32 form's cross terms at kColX): running sums += chunk, or after the last chunk (+ cross
// terms) -> written.  kExact (int8 form): exact int32 running sums.
template <int kExact>
__device__ __forceinline__ void drain_split(const XtSub& s, const ItemGeo ig, uint32_t tm, int row, int b, int chunk) {
    const bool last = chunk == ig.n_chunk - 1;
    for (int j0 = 0; j0 < ig.N; j0 += 16) {        // 16-column pieces: few registers beside the converters
        uint32_t v[16], rs[16];
        tmem_ld16(tm + b * 128 + j0, v);
        if (chunk > 0) tmem_ld16(tm + kColRun2 + j0, rs);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) rs[e] = chunk_add(kExact, chunk > 0, rs[e], v[e]);
        if (!last) {
            tmem_st16(tm + kColRun2 + j0, rs);
        } else {
            if (ig.cross) {
                tmem_ld16(tm + kColX + j0, v);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; ++e) rs[e] = chunk_add(0, true, rs[e], v[e]);
            }
            write_piece<16>(s, ig, row, j0, rs);
        }
    }
    if (!last) tmem_wait_st();
}

// One chunk of a paired FP32-form item (chunk accumulator b: columns 256 b .. + 127 hold H H^T,
// 256 b + 128 .. + 255 hold H L^T + L H^T): the FP32 running sums of row `row` (shared memory,
// [column][row], so that a warp's rows are consecutive words) += the two halves, or after the
// last chunk the sums are written.
__device__ __forceinline__ void drain_pair(const XtSub& s, const ItemGeo ig, uint32_t tm, int row, int b, int chunk,
                                           float* run) {
    const bool last = chunk == ig.n_chunk - 1;
    const int lr = row - ig.a0;
    for (int j0 = 0; j0 < 128; j0 += 16) {
        uint32_t h[16], x[16], rs[16];
        tmem_ld16(tm + b * 256 + j0, h);
        tmem_ld16(tm + b * 256 + 128 + j0, x);
        float p[16];                                // (all loads, then all stores: no dependent chains)
#pragma unroll
        for (int e = 0; e < 16; ++e) p[e] = chunk > 0 ? run[(j0 + e) * 128 + lr] : 0.0f;
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float v = p[e] + (__uint_as_float(h[e]) + __uint_as_float(x[e]));
            if (!last) run[(j0 + e) * 128 + lr] = v;
            rs[e] = __float_as_uint(v);
        }
        if (last) write_piece<16>(s, ig, row, j0, rs);
    }
}

// run[0..63] (+)= this thread's 64 columns of the accumulator at TMEM address `col`
__device__ __forceinline__ void drain64(uint32_t (&run)[64], uint32_t col, bool have, int exact) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {           // four 16-column loads
        uint32_t v[16];
        tmem_ld16(col + 16 * h, v);
        tmem_wait_ld();
        if (!have) {
#pragma unroll
            for (int e = 0; e < 16; ++e) run[16 * h + e] = chunk_add(exact, false, 0u, v[e]);
        } else if (exact) {
#pragma unroll
            for (int e = 0; e < 16; ++e) run[16 * h + e] = chunk_add(1, true, run[16 * h + e], v[e]);
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) run[16 * h + e] = chunk_add(0, true, run[16 * h + e], v[e]);
        }
    }
}

// All chunks of a one-plane narrow item (N <= 128): chunk c (global chunk count cc + c) sits in
// accumulator (cc + c) % nbuf; the running sums of this thread's row and 64-column half stay in
// registers and are written after the last chunk.  `par`
// holds the accumulators' phase bits; the updated bits are returned.
__device__ __forceinline__ uint32_t drain_narrow(Shared& sh, const XtSub& s, const ItemGeo ig, uint32_t tm, int row,
                                              int half, int cc, uint32_t par, unsigned* err) {
    const int c0 = 64 * half;
    uint32_t run[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) run[e] = 0u;
    for (int chunk = 0; chunk < ig.n_chunk; ++chunk) {
        const int b = (cc + chunk) % ig.nbuf;
        if (!mbar_wait(&sh.accf[b], (par >> b) & 1, err, ERR_WAIT_MMA)) {
            sh.abort_flag = 1;
            return par;
        }
        par ^= 1u << b;
        tc_fence_after();
        if (c0 < ig.N) drain64(run, tm + b * 128 + c0, chunk > 0, s.exact);
        tc_fence_before();
        mbar_arrive(&sh.acce[b]);             // the accumulator goes back to the MMA issuer
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (c0 + 32 * j < ig.N) {
            uint32_t piece[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) piece[e] = run[32 * j + e];
            write_piece<32>(s, ig, row, c0 + 32 * j, piece);
        }
    }
    return par;
}

// Veltkamp's split of the pair v (both lanes at once; each packed operation rounds as its scalar
// counterpart): hi = v rounded to 11 significant bits (2^13 + 1), lo = v - hi exactly; both as
// fp16 pairs
__device__ __forceinline__ void split_pair(float2 v, uint32_t& hw, uint32_t& lw) {
    const float2 tt = __fmul2_rn(v, make_float2(8193.0f, 8193.0f));
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 hv = __ffma2_rn(__ffma2_rn(v, m1, tt), m1, tt);   // tt - (tt - v)
    const float2 lv = __ffma2_rn(hv, m1, v);                        // v - hi
    const __half2 hh = __floats2half2_rn(hv.x, hv.y);
    const __half2 ll = __floats2half2_rn(lv.x, lv.y);
    hw = *reinterpret_cast<const uint32_t*>(&hh);
    lw = *reinterpret_cast<const uint32_t*>(&ll);
}

// FP32 form: stage g's FP32 slot g % kF32Stages (after the operand slots) becomes operand slot
// g % kOpStages2 --
// for each 8-frame K-block j and row r (unit j * R + r; the converter threads stride over the
// units), the row's frames 8j..8j+7 (two 16-byte granules of the FP32 layout) scaled by the power
// of two split_scale, rounded to fp16 hi and the remainder to fp16 lo, stored as row r of K-block
// j of the hi tile and of the lo tile (full-stage offset).
// Each converter warp works on its own units and signals on its own: lane 0 waits for the FP32
// slot and the operand slot (the decision is shared by a shuffle), the warp converts, fences its
// shared stores for the tensor core's (async) proxy, and lane 0 arrives on both slots' barriers,
// which complete after all kConvWarps warps.  No barrier spans warps.
template <bool kIn8>
__device__ __noinline__ void convert_stages(const XtBatch& t, Shared& sh, unsigned char* smem, int ct) {
    constexpr int nop = kIn8 ? kOpStagesI8 : kOpStages2;      // operand slots
    constexpr int nin = kIn8 ? kRawI8 : kF32Stages, pin = kIn8 ? kRawPitch : kStage2Bytes;   // input slots
    volatile int* abort_flag = &sh.abort_flag;
    const int lane = ct & 31;
    int g = 0;
    for (int it = blockIdx.x; it < t.n_items; it += gridDim.x) {
        const ItemGeo ig = item_geo(t, it);
        const XtSub& s = t.sub[ig.sub];
        const int R = ig.R, Rp = ig.Rp, tb = ig.tb32;
        const float sc = s.split_scale;
        const int lo_off = ig.nkb_stage * R * 16;
        for (int st = 0; st < ig.n_stage; ++st, ++g) {
            const int fs = g % nin, os = g % nop;
            int ok = 1;
            if (lane == 0) {
                ok = !*abort_flag && mbar_wait(&sh.f32full[fs], (g / nin) & 1, t.err, ERR_WAIT_STAGE) &&
                     mbar_wait(&sh.empty[os], ((g / nop) & 1) ^ 1, t.err, ERR_WAIT_MMA);
                if (!ok) *abort_flag = 1;
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;   // the same decision in the whole warp
            const int frames = min(s.ks, s.n_int - st * s.ks);
            const float* src = reinterpret_cast<const float*>(smem + nop * kSlot2 + fs * pin);
            unsigned char* dst = smem + os * kSlot2;
            if constexpr (kIn8) {
                // the stage is [kb][R rows][8 frames] of int8: unit u = j R + r (8 bytes) becomes the
                // 16-byte row r of K-block j of the fp16 operand tile.  Only rows b0 .. R - 1 are
                // converted: the second item of a 256-row Gram (rows and columns 128 .. R - 1)
                // reads no others.
                const unsigned char* src8 = reinterpret_cast<const unsigned char*>(src);
                const __half2 bias = __float2half2_rn(1152.0f);
                auto widen = [&](int u) {
                    const uint2 q = *reinterpret_cast<const uint2*>(src8 + 8 * u);
                    const uint32_t x[2] = {q.x ^ 0x80808080u, q.y ^ 0x80808080u};
                    uint32_t w[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {   // bytes 2m, 2m + 1 -> fp16 1152 + b -> b
                        const uint32_t hb = __byte_perm(x[m >> 1], 0x64646464u, (m & 1) ? 0x4342 : 0x4140);
                        const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&hb), bias);
                        w[m] = *reinterpret_cast<const uint32_t*>(&v);
                    }
                    *reinterpret_cast<uint4*>(dst + 16 * u) = make_uint4(w[0], w[1], w[2], w[3]);
                };
                if (ig.b0 == 0) {
                    const int units = (frames / 8) * R;
#pragma unroll 4
                    for (int u = ct; u < units; u += kConvThreads) widen(u);
                } else {
                    // rows b0 .. R - 1 of each K-block: index v = j (R - b0) + (r - b0), stepped incrementally
                    const int Rs = R - ig.b0, units = (frames / 8) * Rs;
                    int r = ct % Rs, j = ct / Rs;
                    const int dr = kConvThreads % Rs, dj = kConvThreads / Rs;
#pragma unroll 2
                    for (int v = ct; v < units; v += kConvThreads) {
                        widen(j * R + ig.b0 + r);
                        r += dr;
                        j += dj;
                        if (r >= Rs) {
                            r -= Rs;
                            ++j;
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (ct == 0) sh.consumed = g + 1;
                    mbar_arrive(&sh.f32empty[fs]);
                    mbar_arrive(&sh.full[os]);
                }
                continue;
            }
            if (s.quad) {
                // the stage is [kb][R rows][8 frames]: unit u = (j R + r) 2 + h takes frames 4h .. 4h + 3 of
                // row r in K-block j (one 16-byte load; consecutive units, consecutive bytes) and writes
                // their hi and lo halves (8 bytes each) into row r of K-block j of the two operand tiles
                const int units = (frames / 8) * R * 2;
#pragma unroll 4
                for (int u = ct; u < units; u += kConvThreads) {
                    const float4 q = *reinterpret_cast<const float4*>(src + 4 * u);
                    const float2 sc2 = make_float2(sc, sc);
                    uint32_t hw[2], lw[2];
                    split_pair(__fmul2_rn(make_float2(q.x, q.y), sc2), hw[0], lw[0]);
                    split_pair(__fmul2_rn(make_float2(q.z, q.w), sc2), hw[1], lw[1]);
                    // paired items (128 rows): K-block j holds 128 hi rows then 128 lo rows (4096 bytes)
                    unsigned char* d = dst + u * 8 + (ig.pair ? (u >> 8) * 2048 : 0);
                    *reinterpret_cast<uint2*>(d) = make_uint2(hw[0], hw[1]);
                    *reinterpret_cast<uint2*>(d + (ig.pair ? 2048 : lo_off)) = make_uint2(lw[0], lw[1]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (ct == 0) sh.consumed = g + 1;
                    mbar_arrive(&sh.f32empty[fs]);
                    mbar_arrive(&sh.full[os]);
                }
                continue;
            }
            const int units = (frames / 8) * R;
            // unit u = j * R + r: thread ct takes u = ct, ct + kConvThreads, ... (r, j stepped incrementally)
            int r = ct % R, j = ct / R;
            const int dr = kConvThreads % R, dj = kConvThreads / R;
#pragma unroll 2
            for (int u = ct; u < units; u += kConvThreads) {
                // frames 0-3 and 4-7 of row r in the 8-frame span j (one FP32 K-block, or two of 4 frames)
                // (TB 8: rows r and r + 4 of a row group read opposite halves first, so that the 8
                // rows of a quarter warp hit 8 distinct bank groups)
                const bool sw = tb == 8 && ((r >> 2) & 1);
                const int oa = fp32_off(r, sw ? 4 : 0, tb);
                const int ob = tb == 8 ? fp32_off(r, sw ? 0 : 4, 8) : Rp * 4 + oa;
                const float* p = src + j * 8 * Rp;
                unsigned char* d = dst + u * 16 + (ig.pair ? j * 2048 : 0);
                const float4 qa = *reinterpret_cast<const float4*>(p + oa);
                const float4 qb = *reinterpret_cast<const float4*>(p + ob);
                const float4 q0 = sw ? qb : qa, q1 = sw ? qa : qb;
                // hi: v rounded to 11 significant bits in FP32 (Veltkamp's split, 2^13 + 1), exact in fp16
                // above 2^-14 (below, fp16 rounds it once more: under 2^-25 absolute, against values of
                // order 2^6); lo = v - hi is exact.  Two packed conversions per pair of values.
                const float2 sc2 = make_float2(sc, sc);
                uint32_t hw[4], lw[4];
                split_pair(__fmul2_rn(make_float2(q0.x, q0.y), sc2), hw[0], lw[0]);
                split_pair(__fmul2_rn(make_float2(q0.z, q0.w), sc2), hw[1], lw[1]);
                split_pair(__fmul2_rn(make_float2(q1.x, q1.y), sc2), hw[2], lw[2]);
                split_pair(__fmul2_rn(make_float2(q1.z, q1.w), sc2), hw[3], lw[3]);
                *reinterpret_cast<uint4*>(d) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(d + (ig.pair ? 2048 : lo_off)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                r += dr;
                j += dj;
                if (r >= R) {
                    r -= R;
                    ++j;
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (ct == 0) sh.consumed = g + 1;  // this FP32 copy has landed
                mbar_arrive(&sh.f32empty[fs]);
                mbar_arrive(&sh.full[os]);
            }
        }
    }
}

// kForm: XT_FORM_F16 (one plane, copied straight into the operand slots), XT_FORM_F32 (FP32 split),
// XT_FORM_I8 (int8 bytes widened); one instantiation per form keeps every role's branches static
template <int kForm>
__global__ void __launch_bounds__((kForm != XT_FORM_F16 ? kWarps2 : kWarps1) * 32, 1)
    xengine_tc_kernel(const XtBatch* __restrict__ tab) {
    constexpr bool kF32 = kForm != XT_FORM_F16;   // a converted form
    constexpr bool kIn8 = kForm == XT_FORM_I8;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Shared sh;
    const XtBatch& t = *tab;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh.full[s], kF32 ? kConvWarps : 1);   // converted by every converter warp, or one copy
            mbar_init(&sh.empty[s], 1);
        }
        for (int s = 0; s < kInSlots; ++s) {
            mbar_init(&sh.f32full[s], 1);
            mbar_init(&sh.f32empty[s], kConvWarps);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&sh.accf[b], 1);
            mbar_init(&sh.acce[b], kF32 ? kEpiThreads2 : kEpiThreads1);
        }
        mbar_init(&sh.xf, 1);
        mbar_init(&sh.xe, kEpiThreads2);
        fence_mbar_init();
        sh.abort_flag = 0;
        sh.consumed = 0;
    }
    if (warp == 0) {
        tmem_alloc(&sh.taddr, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.taddr;
    volatile int* abort_flag = &sh.abort_flag;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            constexpr bool f32 = kF32;
            constexpr bool in8 = kIn8;
            const int nsl = f32 ? (in8 ? kRawI8 : kF32Stages) : kStages;
            uint64_t* fullb = f32 ? sh.f32full : sh.full;
            uint64_t* emptyb = f32 ? sh.f32empty : sh.empty;
            unsigned char* slots = f32 ? smem + (in8 ? kOpStagesI8 : kOpStages2) * kSlot2 : smem;
            const int pitch = f32 ? (in8 ? kRawPitch : kStage2Bytes) : kSlot;
            int g = 0;
            for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
                const ItemGeo ig = item_geo(t, it);
                const XtSub& s = t.sub[ig.sub];
                for (int st = 0; st < ig.n_stage; ++st, ++g) {
                    const int slot = g % nsl;
                    if (!mbar_wait(&emptyb[slot], ((g / nsl) & 1) ^ 1, t.err, ERR_WAIT_MMA)) {
                        *abort_flag = 1;
                        break;
                    }
                    unsigned char* dst = slots + slot * pitch;
                    if (f32 && s.quad) {
                        // channel-quad layout: one 5-D tensor copy gathers the stage's pieces of channel k
                        // (a last, shorter stage reads zeros past the end and counts the whole box)
                        if (st == 0) tmap_acquire(&s.tmap);
                        const int nkb = s.ks / kTbHalf;
                        mbar_arrive_expect_tx(&fullb[slot], static_cast<uint32_t>(nkb) * s.n_in * 64);
                        tma_load_5d(dst, &s.tmap, 0, ig.k & 3, 0, st * nkb, ig.k >> 2, &fullb[slot]);
                    } else if (f32 && in8) {
                        // channel-quad int8 bytes: one 5-D tensor copy gathers the stage's 16-byte pieces
                        // of channel k into [kb][2 n_in rows][8 bytes] (half the fp16 bytes)
                        if (st == 0) tmap_acquire(&s.tmap);
                        const int nkb = s.ks / kTbHalf;
                        mbar_arrive_expect_tx(&fullb[slot], static_cast<uint32_t>(nkb) * s.n_in * 16);
                        tma_load_5d(dst, &s.tmap, 0, ig.k & 3, 0, st * nkb, ig.k >> 2, &fullb[slot]);
                    } else if (f32) {
                        // the stage's FP32 K-blocks of channel k are contiguous
                        const int frames = min(s.ks, s.n_int - st * s.ks);
                        const uint32_t bytes = static_cast<uint32_t>(frames) * ig.Rp * 4;
                        const float* src = s.spec32 +
                            (static_cast<int64_t>(ig.k) * ig.ntb32 + st * (s.ks / ig.tb32)) * ig.Rp * ig.tb32;
                        mbar_arrive_expect_tx(&fullb[slot], bytes);
                        bulk_g2s(dst, src, bytes, &fullb[slot]);
                    } else {
                        const int kb0 = st * ig.nkb_stage;
                        const int nkb = min(ig.nkb_stage, ig.ntb - kb0);
                        const uint32_t bytes = static_cast<uint32_t>(nkb) * ig.R * 16;
                        const int64_t off = (static_cast<int64_t>(ig.k) * ig.ntb + kb0) * ig.R * kTbHalf;
                        mbar_arrive_expect_tx(&fullb[slot], bytes);
                        bulk_g2s(dst, s.spec + off, bytes, &fullb[slot]);
                    }
                }
            }
            // let every issued copy land before the CTA can exit
            for (int q = *(volatile int*)&sh.consumed; q < g; ++q)
                mbar_wait(&fullb[q % nsl], (q / nsl) & 1, nullptr, 0);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int g = 0, cc = 0;
            uint32_t par = 0;                     // bit b: parity of accumulator b's uses so far
            int prev_nbuf = -1;
            constexpr int nsl = kF32 ? (kIn8 ? kOpStagesI8 : kOpStages2) : kStages;
            for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
                const ItemGeo ig = item_geo(t, it);
                const XtSub& s = t.sub[ig.sub];
                const uint32_t idesc = idesc_f16_f32(128, ig.N);
                const uint32_t lbo = static_cast<uint32_t>(ig.R) * 16, sbo = 128;
                const int stages_per_chunk = s.chunk / s.ks;
                const bool two = s.spec32 != nullptr;
                const uint32_t lo_off = static_cast<uint32_t>(ig.nkb_stage) * ig.R * 16;
                bool xfirst = true;                   // next cross-term MMA starts the accumulator
                if (ig.cross) {                       // the previous item's cross terms are drained
                    if (!mbar_wait(&sh.xe, ((par >> kXBit) & 1) ^ 1, t.err, ERR_WAIT_EPI)) {
                        *abort_flag = 1;
                        break;
                    }
                    par ^= 1u << kXBit;
                }
                for (int chunk = 0; chunk < ig.n_chunk && !*abort_flag; ++chunk, ++cc) {
                    const int b = cc % ig.nbuf;
                    // a single-buffered item, or a change of buffering, needs every earlier drain done
                    bool ok = true;
                    if (!ig.dbl || prev_nbuf != ig.nbuf) {
                        for (int q = 0; q < kAccBufs && ok; ++q)
                            ok = mbar_wait(&sh.acce[q], ((par >> q) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                        // (columns 256-383 may have held cross terms; a sep item already waited)
                        if (ok && !ig.cross)
                            ok = mbar_wait(&sh.xe, ((par >> kXBit) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    } else {
                        ok = mbar_wait(&sh.acce[b], ((par >> b) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    }
                    prev_nbuf = ig.nbuf;
                    if (!ok) {
                        *abort_flag = 1;
                        break;
                    }
                    par ^= 1u << b;
                    tc_fence_after();
                    const uint32_t dcol = tmem + (ig.dbl ? b * (ig.pair ? 256 : 128) : 0);
                    const int st0 = chunk * stages_per_chunk;
                    const int st1 = min(ig.n_stage, st0 + stages_per_chunk);
                    bool first = true;
                    for (int st = st0; st < st1; ++st, ++g) {
                        const int slot = g % nsl;
                        if (!mbar_wait(&sh.full[slot], (g / nsl) & 1, t.err, ERR_WAIT_STAGE)) {
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const int nkb = min(ig.nkb_stage, ig.ntb - st * ig.nkb_stage);
                        const uint32_t base = smem_u32(smem + slot * (kF32 ? kSlot2 : kSlot));
                        if constexpr (kForm == XT_FORM_F32) {
                            if (ig.pair) {
                                // K-block: 128 hi rows then 128 lo rows (LBO 4096 bytes); per 16 frames
                                // [H H^T | H L^T] = H [H; L]^T (N = 256), then L H^T onto the right half
                                constexpr uint32_t lbo2 = 4096;
                                const uint32_t idesc2 = idesc_f16_f32(128, 256);
                                for (int kk = 0; kk < nkb / 2; ++kk) {
                                    const uint32_t kbase = base + kk * 2 * lbo2;
                                    const uint64_t dh = smem_desc_noswizzle(kbase, lbo2, sbo);
                                    const uint64_t dl = smem_desc_noswizzle(kbase + 2048, lbo2, sbo);
                                    umma_f16(dcol, dh, dh, idesc2, first ? 0u : 1u);
                                    umma_f16(dcol + 128, dl, dh, idesc, 1u);
                                    first = false;
                                }
                                umma_commit(&sh.empty[slot]);   // frees the stage once these MMAs finish
                                continue;
                            }
                        }
                        for (int kk = 0; kk < nkb / 2; ++kk) {
                            const uint32_t kbase = base + kk * 2 * lbo;
                            const uint64_t da = smem_desc_noswizzle(kbase + ig.a0 * 16, lbo, sbo);
                            const uint64_t db = smem_desc_noswizzle(kbase + ig.b0 * 16, lbo, sbo);
                            umma_f16(dcol, da, db, idesc, first ? 0u : 1u);
                            first = false;
                            if (two) {
                                const uint64_t la = smem_desc_noswizzle(kbase + lo_off + ig.a0 * 16, lbo, sbo);
                                const uint64_t lb = smem_desc_noswizzle(kbase + lo_off + ig.b0 * 16, lbo, sbo);
                                const uint32_t xcol = ig.sep ? tmem + kColX : dcol;
                                umma_f16(xcol, da, lb, idesc, (ig.sep && xfirst) ? 0u : 1u);   // H L^T
                                umma_f16(xcol, la, db, idesc, 1u);                              // L H^T
                                xfirst = false;
                            }
                        }
                        umma_commit(&sh.empty[slot]);   // frees the stage once these MMAs finish
                        if (!kF32) sh.consumed = g + 1;
                    }
                    if (*abort_flag) break;
                    umma_commit(&sh.accf[b]);           // chunk complete
                }
                if (*abort_flag) break;
                if (ig.cross) umma_commit(&sh.xf);      // cross terms complete
            }
        }
    } else if (kF32 && warp >= kConvWarp0) {
        // ------------------------------------------------------------ converters (FP32 form)
        convert_stages<kIn8>(t, sh, smem, threadIdx.x - kConvWarp0 * 32);
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9 or 2..5)
        const int q = warp & 3;                   // TMEM lane quarter this warp may access
        const int lrow = 32 * q + lane;           // row within the item's 128 rows = TMEM lane
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        // one-plane forms: column half of the 8 drain warps; FP32 form: every column
        const int half = kF32 ? 0 : (warp - 2) >> 2;
        int cc = 0;
        uint32_t par = 0;                         // bit b: parity of accumulator b's uses so far
        for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
            const ItemGeo ig = item_geo(t, it);
            const XtSub& s = t.sub[ig.sub];
            if (kF32 && ig.sep) {           // (converted forms: every narrow item)
                for (int chunk = 0; chunk < ig.n_chunk; ++chunk, ++cc) {
                    const int b = cc % ig.nbuf;
                    const bool last = chunk == ig.n_chunk - 1;
                    bool ok = mbar_wait(&sh.accf[b], (par >> b) & 1, t.err, ERR_WAIT_MMA);
                    if (ok && last && ig.cross) ok = mbar_wait(&sh.xf, (par >> kXBit) & 1, t.err, ERR_WAIT_MMA);
                    if (!ok) {
                        sh.abort_flag = 1;
                        break;
                    }
                    par ^= 1u << b;
                    if (last && ig.cross) par ^= 1u << kXBit;
                    tc_fence_after();
                    if constexpr (kForm == XT_FORM_F32) {
                        if (ig.pair)
                            drain_pair(s, ig, tmem + lane_off, ig.a0 + lrow, b, chunk, reinterpret_cast<float*>(smem + kRunOff));
                        else
                            drain_split<0>(s, ig, tmem + lane_off, ig.a0 + lrow, b, chunk);
                    } else {
                        drain_split<kIn8 ? 1 : 0>(s, ig, tmem + lane_off, ig.a0 + lrow, b, chunk);
                    }
                    tc_fence_before();
                    mbar_arrive(&sh.acce[b]);
                    if (last && ig.cross) mbar_arrive(&sh.xe);
                }
            } else if (!kF32 && ig.dbl) {
                par = drain_narrow(sh, s, ig, tmem + lane_off, ig.a0 + lrow, half, cc, par, t.err);
                cc += ig.n_chunk;
            } else {
                for (int chunk = 0; chunk < ig.n_chunk; ++chunk, ++cc) {
                    if (!mbar_wait(&sh.accf[0], par & 1, t.err, ERR_WAIT_MMA)) {
                        sh.abort_flag = 1;
                        break;
                    }
                    par ^= 1u;
                    tc_fence_after();
                    if constexpr (kF32) drain_wide<16>(s, ig, tmem + lane_off, ig.a0 + lrow, 0, 16, chunk);
                    else drain_wide<32>(s, ig, tmem + lane_off, ig.a0 + lrow, 32 * half, 64, chunk);
                    tc_fence_before();
                    mbar_arrive(&sh.acce[0]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

bool xengine_tc_encode_quad(XtSub& x) {
    const bool b8 = x.in8 != 0;                    // int8 bytes (16-byte pieces) or FP32 (64-byte pieces)
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q{};
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t ntb = static_cast<cuuint64_t>(x.n_int / kTbHalf);
    const cuuint64_t dim[5] = {16, 4, static_cast<cuuint64_t>(x.n_in), ntb, static_cast<cuuint64_t>(x.n_chan / 4)};
    const cuuint64_t piece = b8 ? 16 : 64;         // bytes of one (channel, K-block, input) piece
    const cuuint64_t stride[4] = {piece, 4 * piece, 4 * piece * x.n_in, 4 * piece * x.n_in * ntb};   // bytes, dims 1..4
    const cuuint32_t box[5] = {16, 1, static_cast<cuuint32_t>(x.n_in), static_cast<cuuint32_t>(x.ks / kTbHalf), 1};
    const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
    void* base = b8 ? static_cast<void*>(const_cast<__half*>(x.spec)) : static_cast<void*>(const_cast<float*>(x.spec32));
    return encode(&x.tmap, b8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dim, stride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool xengine_tc_supported(int n_in) { return n_in >= 1 && 2 * n_in <= 256; }

int xengine_tc_max_ks(int n_in) {
    int ks = 512;                                  // stages of at most 512 frames
    while (ks > 16 && (ks / kTbHalf) * 2 * n_in * 16 > kStageMaxBytes) ks /= 2;
    return ks;
}

int xengine_tc_ks_fp32(int n_in) {
    // the FP32 slot holds ks * rows_fp32(n_in) floats; the operand slot's two planes then take
    // ks * 2 n_in * 4 <= that many bytes
    int ks = 512;
    while (ks > 16 && ks * rows_fp32(n_in) * 4 > kStage2Bytes) ks /= 2;
    return ks;
}

size_t xengine_tc_smem() { return static_cast<size_t>(kSmemBytes); }

cudaError_t launch_xengine_tc_table(const XtBatch* dtab, int n_items, int n_sm, cudaStream_t s, int form) {
    const size_t smem = xengine_tc_smem();
    auto kern = form == XT_FORM_F32 ? xengine_tc_kernel<XT_FORM_F32>
              : form == XT_FORM_I8  ? xengine_tc_kernel<XT_FORM_I8>
                                    : xengine_tc_kernel<XT_FORM_F16>;
    const bool convert = form != XT_FORM_F16;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(n_items, n_sm));
    kern<<<grid, (convert ? kWarps2 : kWarps1) * 32, smem, s>>>(dtab);
    return cudaGetLastError();
}

}  // namespace gbx
