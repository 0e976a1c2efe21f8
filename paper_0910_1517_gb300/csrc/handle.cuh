// handle.cuh -- the correlator handle shared by the C ABI translation units (capi.cu, batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/corr.h"
#include "fengine.cuh"
#include "xengine.cuh"

struct corr {
    int n_ant = 0, n_pol = 0, n_in = 0, n_fft = 0, n_chan = 0, n_int = 0, n_bl = 0, npp = 0;
    int xmode = CORR_FP32, beam_avg = 1, max_delay = 2048;
    int polmode = CORR_POL_FULL;         // CORR_POL_SELF: only the n_pol products pp (npp = n_pol)
    bool last_quad = false;              // the last integration's FP32 spectra are in the channel-quad layout
    int dev = 0, n_sm = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_done = nullptr, ev_aux = nullptr;
    // host-side model
    std::vector<double> tau, phi0, rate;
    bool scales_set = false;
    // streaming ingest: two sample rings; integration j is filled into ring j % 2 on the copy
    // stream while integration j - 1 is correlated on `stream` (the rings hand over their last
    // max_delay samples).  ev_ready[r]: ring r's samples have landed; ev_free[r]: the last
    // integration that read ring r is done with it.
    int8_t* d_ring = nullptr;
    int8_t* d_ring2 = nullptr;
    int cur_ring = 0;
    int64_t ring_ld = 0, fill = 0, seq_next = -1, seq_origin = -1, g_next = 0;
    bool ring_started = false;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr}, ev_copied = nullptr;
    int64_t n_streamed = 0;              // integrations launched from the rings since the stream started
    // ring of host output slots: integration j's visibilities / beams land in slot j % n_slots
    float* out_vis = nullptr;
    float* out_beams = nullptr;
    int n_slots = 0;
    std::vector<cudaEvent_t> ev_out;     // per slot: its last copy has landed
    std::vector<int64_t> slot_of;        // per slot: the integration it holds (or is receiving)
    // while an output ring is set the outputs are double-buffered: streamed integration j writes
    // buffer j % 2 (d_vis, d_beams_raw, d_beams point at the current one), and the output stream
    // copies it to the host slot while integration j + 1 runs
    float2* vis_b[2] = {nullptr, nullptr};
    float* beams_raw_b[2] = {nullptr, nullptr};
    float* beams_b[2] = {nullptr, nullptr};
    gbx::XtBatch* xtab_b1 = nullptr;     // tensor-core table naming buffer 1
    int out_buf = 0;
    cudaStream_t ostream = nullptr;
    cudaEvent_t ev_int_done = nullptr, ev_buf_free[2] = {nullptr, nullptr};
    int batch_refs = 0;                  // batches (captured graphs) holding this handle's buffers
    // device tables and outputs
    double* d_model = nullptr;          // tau | phi0 | rate, 3 * n_ant
    double* h_model = nullptr;          // pinned staging of the same: 1 + kModelSlots copies (the first
                                        // for graph-captured batches, the rest a ring for queued integrations)
    static constexpr int kModelSlots = 4;
    cudaEvent_t ev_model[kModelSlots] = {};
    int model_slot = 0;
    float2* d_pf = nullptr;
    float2* d_ff = nullptr;
    int* d_D = nullptr;
    float2* d_wcoh = nullptr;
    float* d_ginc = nullptr;
    float* d_scale = nullptr;
    float2* d_tw = nullptr;
    void* d_spec = nullptr;
    float* d_beams_raw = nullptr;
    float* d_beams = nullptr;
    float2* d_vis = nullptr;
    float2* d_vis_part = nullptr;   // kVisSplit partial visibility sets of the CUDA-core X-engine
    static constexpr int kVisSplit = 4;
    int2* d_vis_int = nullptr;
    unsigned* d_err = nullptr;
    // bookkeeping
    int64_t launched = 0, completed = 0;
    int last_mode = -1;
    // tensor-core X-engine table (one sub-array: this handle) and its work items
    gbx::XtBatch* d_xtab = nullptr;
    int4* d_items = nullptr;
    int n_items = 0;
    int ks = 0;                          // frames per operand stage (0 = largest that fits)
    // auto-power dumps for the RFI stage (0 = off)
    int dump = 0;
    float* d_power = nullptr;
    // time-domain voltage blanker (Sec. 5, Eq. 3-4; blank_M = 0: off): blocks of 2^blank_log2 samples,
    // noise table [n_in][noise_L], per-block statistics [n_in][blank_nb][4] of the last integration
    // (blank_cap blocks per input allocated), covering blank_n samples of each row
    double blank_M = 0.0;
    int blank_log2 = 0;
    float* d_noise = nullptr;
    int noise_L = 0;
    // multiple phased beams (n_mb = 0: off): weights [n_chan][multibeam_wstride] float2, output
    // [n_mb][n_int / mb_avg][n_chan] float4 of the last integration
    int n_mb = 0, mb_products = 0, mb_avg = 1;
    float2* d_mbw = nullptr;
    float4* d_mb = nullptr;
    // 4-bit ADC-format ingest.  Pushes go through a ring of kStage4Slots packed staging slots
    // (n_cards rows of up to kStage4 samples, pitch kStage4Pitch): host-to-device copies into a
    // slot on cstream, the unpack into the sample ring on ustream, a high-priority stream so that
    // unpacks take the next free SM slots ahead of queued correlator CTAs.  ev_s4[k]: slot k's
    // copy has landed; ev_s4_free[k]: slot k has been unpacked.  Device integrations unpack into
    // d_unpack.
    static constexpr int64_t kStage4 = int64_t(1) << 21;
    static constexpr int kStage4Slots = 8;
    static constexpr int64_t kStage4Pitch = 2 * kStage4 + 16;
    uint8_t* d_stage4 = nullptr;
    cudaStream_t ustream = nullptr;
    cudaEvent_t ev_s4[kStage4Slots] = {}, ev_s4_free[kStage4Slots] = {};
    int s4_next = 0;
    // the stream of the last writes into the sample rings (cstream, or ustream for 4-bit pushes);
    // a push from the other kind first waits for it through ev_ws
    cudaStream_t wstream = nullptr;
    cudaEvent_t ev_ws = nullptr;
    int8_t* d_unpack = nullptr;
    int64_t unpack_ld = 0;
    int32_t* d_blank = nullptr;
    int8_t* d_blanked = nullptr;        // the blanked rows the F-engine reads, stride blanked_ld
    int64_t blanked_ld = 0;
    int64_t blank_cap = 0, blank_nb = 0, blank_n = 0;
    // per-stage timing: kTimedMax integrations x 5 events (before set-up and after each stage)
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    int t_count = 0;
};

namespace gbx {
// Fill a one-entry tensor-core table describing handle h (its spectra, scales and outputs).
XtSub xt_sub_of(const corr* h);
// F-engine output layout (OutMode) of handle h's precision mode.
int fe_out_mode(const corr* h);
// Queue the integration's kernels of handle h (used by the C ABI and the batch code).
int run_integration(corr* h, const int8_t* x, int64_t ld, int64_t n_avail, int64_t g0, cudaStream_t s);
void set_last_error(const char* msg);
int fail_code(int code, const char* msg);
}  // namespace gbx
