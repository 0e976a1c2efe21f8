// capi.cu -- the C ABI declared in include/corr.h: handle state, the streaming
// ring with its delay overlap (Sec. 2.3.2), sequencing of the per-integration
// kernels, and result read-back.  All compute happens in the kernels of
// fengine.cu, xengine_fp32.cu and xengine_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/corr.h"
#include "fengine.cuh"
#include "handle.cuh"
#include "xengine.cuh"

using namespace gbx;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(CORR_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                 \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

}  // namespace

namespace gbx {
// Message reported by corr_last_error() on this thread (used by entry points in other files).
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace gbx

#include "handle.cuh"

namespace {

constexpr int kTimedMax = 4096;
constexpr int kStages = 4;

int64_t ring_need(const corr* h) { return static_cast<int64_t>(h->n_int) * h->n_fft + h->max_delay; }

// record the boundary event `b` (0..kStages) of the current timed integration
int mark(corr* h, int b, cudaStream_t s) {
    if (!h->timing || h->t_count >= kTimedMax) return CORR_OK;
    CU(cudaEventRecord(h->tev[static_cast<size_t>(h->t_count) * (kStages + 1) + b], s));
    return CORR_OK;
}

int alloc_ring(corr* h) {
    if (h->d_ring) cudaFree(h->d_ring);
    if (h->d_ring2) cudaFree(h->d_ring2);
    h->d_ring = h->d_ring2 = nullptr;
    h->cur_ring = 0;
    h->ring_ld = ((ring_need(h) + 64 + 255) / 256) * 256;
    const size_t bytes = static_cast<size_t>(h->ring_ld) * h->n_in;
    CU(dalloc(&h->d_ring, bytes));
    CU(dalloc(&h->d_ring2, bytes));
    CU(cudaMemset(h->d_ring, 0, bytes));
    CU(cudaMemset(h->d_ring2, 0, bytes));
    return CORR_OK;
}

int upload_beam_weights(corr* h, const float* gain, const float* theta, const uint8_t* inc, const uint8_t* coh) {
    std::vector<float2> w(static_cast<size_t>(h->n_ant) * h->n_chan);
    std::vector<float> g2(h->n_ant);
    for (int a = 0; a < h->n_ant; ++a) {
        const double g = gain ? gain[a] : 1.0;
        const bool in_inc = inc ? inc[a] != 0 : true;
        const bool in_coh = coh ? coh[a] != 0 : true;
        g2[a] = in_inc ? static_cast<float>(g * g) : 0.0f;
        for (int k = 0; k < h->n_chan; ++k) {
            const double th = theta ? theta[static_cast<size_t>(a) * h->n_chan + k] : 0.0;
            w[static_cast<size_t>(a) * h->n_chan + k] =
                in_coh ? make_float2(static_cast<float>(g * std::cos(th)), static_cast<float>(g * std::sin(th)))
                       : make_float2(0.f, 0.f);
        }
    }
    CU(cudaMemcpy(h->d_wcoh, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d_ginc, g2.data(), g2.size() * sizeof(float), cudaMemcpyHostToDevice));
    return CORR_OK;
}

// CORR_FP32TC hands its FP32 spectra over in the channel-quad layout (f32q_piece) where the
// warp-FFT F-engine runs (n_chan <= 1024) and no phased-beam kernel reads them
bool spec_quad(const corr* h) { return h->xmode == CORR_FP32TC && h->n_chan <= 1024 && h->n_mb == 0; }

// F-engine output mode of a handle's X-engine precision mode
int fe_mode(const corr* h) {
    switch (h->xmode) {
        case CORR_I8: return OUT_I8B;                                  // int8 bytes, 1 B a sample
        case CORR_F16: return OUT_F16;
        default: return spec_quad(h) ? OUT_F32Q : OUT_FP32;
    }
}

// CORR_FP32TC: v = Y * 2^-e with e = log2(n_fft) - 8 keeps |v| <= 128 * 256 (1 + eps) < 65504
int split_exp(const corr* h) {
    int e = -8;
    for (int n = h->n_fft; n > 1; n >>= 1) ++e;
    return e;
}

// frames per TMEM accumulation chunk of CORR_FP32TC: 128, and 256 where the X-engine pairs the
// hi and lo rows (64 inputs), whose drain then adds two accumulator halves per chunk
constexpr int kSplitChunk = 128;
constexpr int kSplitChunkPaired = 512;

int max_int_delay(const corr* h) {
    int m = 0;
    for (double t : h->tau) m = std::max(m, static_cast<int>(std::floor(t + 0.5)));
    return m;
}

}  // namespace

// Queue one integration (phasors, F-engine, X-engine, beam averaging) on stream s.
int gbx::run_integration(corr* h, const int8_t* x, int64_t ld, int64_t n_avail, int64_t g0, cudaStream_t s) {
    if ((h->xmode == CORR_I8 || h->xmode == CORR_F16) && !h->scales_set)
        return fail(CORR_E_STATE, "CORR_I8 / CORR_F16 need requantisation scales (corr_set_scales)");
    if (h->dump > 0 && h->xmode != CORR_FP32 && h->xmode != CORR_FP32TC)
        return fail(CORR_E_STATE, "power dumps need the FP32 spectra (CORR_FP32 or CORR_FP32TC)");
    if (h->n_mb > 0 && h->xmode != CORR_FP32 && h->xmode != CORR_FP32TC)
        return fail(CORR_E_STATE, "multiple beams need the FP32 spectra (CORR_FP32 or CORR_FP32TC)");
    const int nd = h->n_ant;
    // stage the model in a pinned slot no queued copy still reads (integrations may be queued
    // back to back while earlier ones run)
    const int ms = h->model_slot;
    h->model_slot = (ms + 1) % corr::kModelSlots;
    double* hm = h->h_model + 3 * static_cast<size_t>(nd) * (1 + ms);
    CU(cudaEventSynchronize(h->ev_model[ms]));
    std::memcpy(hm, h->tau.data(), nd * sizeof(double));
    std::memcpy(hm + nd, h->phi0.data(), nd * sizeof(double));
    std::memcpy(hm + 2 * nd, h->rate.data(), nd * sizeof(double));
    CU(cudaMemcpyAsync(h->d_model, hm, 3 * nd * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaEventRecord(h->ev_model[ms], s));
    if (int rc = mark(h, 0, s)) return rc;
    CU(launch_phasor_setup(h->n_ant, h->n_chan, h->n_fft, h->n_int, g0, h->d_model, h->d_model + nd,
                           h->d_model + 2 * nd, h->d_pf, h->d_ff, h->d_D, s));
    FeParams fp{};
    fp.x = x;
    fp.ld = ld;
    fp.n_avail = n_avail;
    fp.n_ant = h->n_ant;
    fp.n_pol = h->n_pol;
    fp.n_in = h->n_in;
    fp.n_fft = h->n_fft;
    fp.n_chan = h->n_chan;
    fp.n_int = h->n_int;
    fp.D = h->d_D;
    fp.pf = h->d_pf;
    fp.ff = h->d_ff;
    fp.wcoh = h->d_wcoh;
    fp.ginc = h->d_ginc;
    fp.scale = h->d_scale;
    fp.spec = h->d_spec;
    fp.beams = h->d_beams_raw;
    fp.tw = h->d_tw;
    fp.err = h->d_err;
    const int fmode = fe_mode(h);
    if (fmode == OUT_FP32 && h->last_quad) {   // back from the channel-quad layout: padding rows read as zero
        CU(cudaMemsetAsync(h->d_spec, 0,
                           static_cast<size_t>(h->n_chan) * h->n_int * rows_fp32(h->n_in) * sizeof(float), s));
    }
    h->last_quad = fmode == OUT_F32Q;
    if (int rc = mark(h, 1, s)) return rc;
    if (h->blank_M > 0.0) {   // voltage blanker: per-block statistics of every sample the F-engine reads
        const int64_t need = static_cast<int64_t>(h->n_int) * h->n_fft + max_int_delay(h);
        const int64_t nb = (need + (int64_t(1) << h->blank_log2) - 1) >> h->blank_log2;
        if (nb > h->blank_cap) return fail(CORR_E_STATE, "max_delay grew after corr_set_blanker: set the blanker again");
        CU(launch_blank(x, ld, h->n_in, need, 1 << h->blank_log2, h->blank_M, h->d_noise, h->noise_L - 1,
                        h->d_blank, h->d_blanked, h->blanked_ld, s));
        fp.x = h->d_blanked;            // the F-engine reads the blanked rows
        fp.ld = h->blanked_ld;
        fp.n_avail = need;
        h->blank_nb = nb;
        h->blank_n = need;
    }
    CU(launch_fengine(fp, fmode, s));
    if (int rc = mark(h, 2, s)) return rc;
    XParams xp{};
    xp.spec = h->d_spec;
    xp.n_ant = h->n_ant;
    xp.n_pol = h->n_pol;
    xp.n_in = h->n_in;
    xp.n_chan = h->n_chan;
    xp.n_int = h->n_int;
    xp.scale = h->d_scale;
    xp.vis = h->d_vis;
    xp.vis_int = h->xmode == CORR_I8 ? h->d_vis_int : nullptr;
    xp.err = h->d_err;
    xp.exact = h->xmode == CORR_I8 ? 1 : 0;
    xp.vis_part = h->d_vis_part;
    xp.max_split = corr::kVisSplit;
    xp.self = h->polmode == CORR_POL_SELF ? 1 : 0;
    if (h->xmode == CORR_FP32)
        CU(launch_xengine_fp32(xp, h->n_sm, s));
    else
        CU(launch_xengine_tc_table(h->out_buf == 1 ? h->xtab_b1 : h->d_xtab, h->n_items, h->n_sm, s,
                                   h->xmode == CORR_FP32TC ? XT_FORM_F32 : fmode == OUT_I8B ? XT_FORM_I8 : XT_FORM_F16));
    if (h->dump > 0) {
        CU(launch_power_dumps(static_cast<const float*>(h->d_spec), h->n_in, h->n_chan, h->n_int, h->dump,
                              h->d_power, s, fmode == OUT_F32Q));
    }
    if (int rc = mark(h, 3, s)) return rc;
    if (h->beam_avg > 1) CU(launch_beam_average(h->d_beams_raw, h->d_beams, h->n_int, h->n_chan, h->beam_avg, s));
    if (h->n_mb > 0)
        CU(launch_multibeam(static_cast<const float*>(h->d_spec), h->n_ant, h->n_pol, h->n_chan, h->n_int, h->d_mbw,
                            h->n_mb, h->mb_products, h->mb_avg, h->d_mb, h->d_err, s));
    if (int rc = mark(h, 4, s)) return rc;
    if (h->timing && h->t_count < kTimedMax) h->t_count += 1;
    CU(cudaEventRecord(h->ev_done, s));
    h->launched += 1;
    h->last_mode = h->xmode;
    return CORR_OK;
}

int gbx::fe_out_mode(const corr* h) { return fe_mode(h); }

gbx::XtSub gbx::xt_sub_of(const corr* h) {
    XtSub x{};
    x.spec = static_cast<const __half*>(h->d_spec);
    x.n_ant = h->n_ant;
    x.n_pol = h->n_pol;
    x.n_in = h->n_in;
    x.n_chan = h->n_chan;
    x.n_int = h->n_int;
    x.scale = h->d_scale;
    x.vis = h->d_vis;
    x.vis_int = h->xmode == CORR_I8 ? h->d_vis_int : nullptr;
    x.exact = h->xmode == CORR_I8 ? 1 : 0;
    x.self = h->polmode == CORR_POL_SELF ? 1 : 0;
    if (h->xmode == CORR_FP32TC) {
        const int max_ks = std::min(xengine_tc_ks_fp32(h->n_in), kSplitChunk);
        x.ks = h->ks > 0 ? std::min(h->ks, max_ks) : max_ks;
        x.spec32 = static_cast<const float*>(h->d_spec);
        x.split_scale = std::ldexp(1.0f, -split_exp(h));
        x.descale = std::ldexp(1.0f, 2 * split_exp(h));
        x.chunk = 2 * h->n_in == 128 ? kSplitChunkPaired : kSplitChunk;
        x.quad = spec_quad(h) ? 1 : 0;
    } else {
        const int max_ks = xengine_tc_max_ks(h->n_in);
        x.ks = h->ks > 0 ? std::min(h->ks, max_ks) : max_ks;
        x.chunk = 1024;
        x.in8 = fe_mode(h) == OUT_I8B ? 1 : 0;
    }
    return x;
}

int gbx::fail_code(int code, const char* msg) { return fail(code, "%s", msg); }

namespace {

// Rewrite the handle's one-entry tensor-core table (after a mode or stage-size change).
int upload_xtab(corr* h) {
    if (!h->d_xtab) return CORR_OK;
    XtBatch t{};
    t.n_sub = 1;
    t.sub[0] = xt_sub_of(h);
    t.n_items = h->n_items;
    t.items = h->d_items;
    t.err = h->d_err;
    if ((t.sub[0].quad || t.sub[0].in8) && !xengine_tc_encode_quad(t.sub[0]))
        return fail(CORR_E_CUDA, "the driver refused the tensor map of the spectra");
    CU(cudaDeviceSynchronize());
    if (h->xtab_b1) {                    // double-buffered outputs: one table per buffer
        t.sub[0].vis = h->vis_b[0];
        CU(cudaMemcpy(h->d_xtab, &t, sizeof t, cudaMemcpyHostToDevice));
        t.sub[0].vis = h->vis_b[1];
        CU(cudaMemcpy(h->xtab_b1, &t, sizeof t, cudaMemcpyHostToDevice));
        return CORR_OK;
    }
    CU(cudaMemcpy(h->d_xtab, &t, sizeof t, cudaMemcpyHostToDevice));
    return CORR_OK;
}

// Point the handle's outputs at buffer b of the double-buffered pair.
void select_outputs(corr* h, int b) {
    h->out_buf = b;
    h->d_vis = h->vis_b[b];
    h->d_beams_raw = h->beams_raw_b[b];
    h->d_beams = h->beams_b[b];
}

// Wait for (or poll) the last launched integration; check the device error word.
int settle(corr* h, int blocking) {
    if (h->launched == 0) return fail(CORR_E_AGAIN, "no integration has been launched");
    if (h->completed < h->launched) {
        if (blocking) {
            CU(cudaEventSynchronize(h->ev_done));
        } else {
            cudaError_t q = cudaEventQuery(h->ev_done);
            if (q == cudaErrorNotReady) return fail(CORR_E_AGAIN, "integration still in flight");
            if (q != cudaSuccess) return fail(CORR_E_CUDA, "integration failed: %s", cudaGetErrorString(q));
        }
        h->completed = h->launched;
    }
    unsigned err = 0;
    CU(cudaMemcpy(&err, h->d_err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(CORR_E_TIMEOUT, "a kernel wait timed out (error bits 0x%x); results invalid", err);
    return CORR_OK;
}

int check_handle(corr* h) {
    if (!h) return fail(CORR_E_INVAL, "null handle");
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return fail(CORR_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return CORR_OK;
}

// Append n samples per input (host or device rows of pitch spitch) to the ring,
// launching integrations as it fills.  kind is the cudaMemcpyKind of the copy.
// Results of the integration just queued on h->stream (in output buffer h->out_buf) into the
// host output ring: copied on the output stream, which then frees the buffer.
int enqueue_output(corr* h, int64_t index) {
    if (!h->out_vis) return CORR_OK;
    const int slot = static_cast<int>(index % h->n_slots), b = h->out_buf;
    const size_t nv = static_cast<size_t>(h->n_chan) * h->n_bl * h->npp * 2;
    const size_t nb = 2 * static_cast<size_t>(h->n_int / h->beam_avg) * h->n_chan;
    h->slot_of[slot] = index;
    CU(cudaEventRecord(h->ev_int_done, h->stream));
    CU(cudaStreamWaitEvent(h->ostream, h->ev_int_done, 0));
    CU(cudaMemcpyAsync(h->out_vis + nv * slot, h->vis_b[b], nv * sizeof(float), cudaMemcpyDeviceToHost,
                       h->ostream));
    if (h->out_beams)
        CU(cudaMemcpyAsync(h->out_beams + nb * slot, h->beams_b[b], nb * sizeof(float), cudaMemcpyDeviceToHost,
                           h->ostream));
    CU(cudaEventRecord(h->ev_out[slot], h->ostream));
    CU(cudaEventRecord(h->ev_buf_free[b], h->ostream));
    return CORR_OK;
}

// Streaming ingest of n samples per input: put(dst, take, done) queues the writes of samples
// done .. done + take - 1 of every input into the ring rows at dst (stride ring_ld), the last of
// them on ws (host copies run on the copy stream h->cstream).  A full ring launches its
// integration on h->stream (after ws) and the next integration fills the other ring, once the
// integration before that is done with it.  Returns when the host source has been read (host
// sources; device sources stay stream-ordered).
template <typename Put>
int ingest(corr* h, Put&& put, int64_t n, int64_t seq, bool from_host, cudaStream_t ws) {
    int rc = CORR_OK;
    if (h->wstream && h->wstream != ws) {   // ring writes switch streams: keep them in order
        CU(cudaEventRecord(h->ev_ws, h->wstream));
        CU(cudaStreamWaitEvent(ws, h->ev_ws, 0));
    }
    h->wstream = ws;
    if (!h->ring_started) {
        h->ring_started = true;
        h->seq_origin = seq;
        h->seq_next = seq;
        h->g_next = 0;
        h->fill = 0;
    } else if (seq != h->seq_next) {
        // gap or overlap: drop the partial integration, restart the current ring at seq
        const int64_t gap = seq - h->seq_next;
        h->fill = 0;
        h->seq_next = seq;
        h->g_next = (seq - h->seq_origin) >= 0 ? (seq - h->seq_origin) / h->n_fft : 0;
        fail(CORR_E_DATALOSS, "sequence gap of %lld samples: partial integration dropped", (long long)gap);
        rc = CORR_E_DATALOSS;
    }
    const int64_t need = ring_need(h);
    const int64_t body = static_cast<int64_t>(h->n_int) * h->n_fft;
    int64_t done = 0;
    while (done < n) {
        int8_t* ring = h->cur_ring ? h->d_ring2 : h->d_ring;
        const int64_t take = std::min(n - done, need - h->fill);
        if (int e = put(ring + h->fill, take, done)) return e;
        h->fill += take;
        done += take;
        if (h->fill == need) {
            if (max_int_delay(h) > h->max_delay)
                return fail(CORR_E_RANGE, "a delay exceeds max_delay = %d", h->max_delay);
            const int r = h->cur_ring, nx = r ^ 1;
            CU(cudaEventRecord(h->ev_ready[r], ws));
            CU(cudaStreamWaitEvent(h->stream, h->ev_ready[r], 0));
            if (h->out_vis) {            // output buffer j % 2, once its copy to the host slot is done
                const int b = static_cast<int>(h->n_streamed & 1);
                CU(cudaStreamWaitEvent(h->stream, h->ev_buf_free[b], 0));
                select_outputs(h, b);
            }
            if (int e = run_integration(h, ring, h->ring_ld, need, h->g_next, h->stream)) return e;
            CU(cudaEventRecord(h->ev_free[r], h->stream));
            if (int e = enqueue_output(h, h->n_streamed)) return e;
            // the next integration fills the other ring, once the integration two back is done
            // with it, beginning with this one's last max_delay samples (overlap, Sec. 2.3.2)
            int8_t* next = nx ? h->d_ring2 : h->d_ring;
            CU(cudaStreamWaitEvent(ws, h->ev_free[nx], 0));
            if (h->max_delay > 0)
                CU(cudaMemcpy2DAsync(next, h->ring_ld, ring + body, h->ring_ld, h->max_delay, h->n_in,
                                     cudaMemcpyDeviceToDevice, ws));
            h->cur_ring = nx;
            h->fill = h->max_delay;
            h->g_next += h->n_int;
            h->n_streamed += 1;
        }
    }
    h->seq_next += n;
    if (from_host) {   // the caller may reuse its buffer
        CU(cudaEventRecord(h->ev_copied, h->cstream));
        CU(cudaEventSynchronize(h->ev_copied));
    }
    return rc;
}

}  // namespace

extern "C" {

const char* corr_last_error(void) { return g_err.c_str(); }

int corr_create(corr_t** out, int n_ant, int n_pol, int n_fft, int n_int) {
    g_err.clear();
    if (!out) return fail(CORR_E_INVAL, "out is null");
    *out = nullptr;
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_ant * n_pol > 128)
        return fail(CORR_E_INVAL, "need 1 <= n_ant * n_pol <= 128 and n_pol in {1, 2}");
    if (n_fft < 64 || n_fft > 4096 || (n_fft & (n_fft - 1)))
        return fail(CORR_E_INVAL, "n_fft must be a power of two in [64, 4096]");
    if (n_int < 16 || n_int % 16) return fail(CORR_E_INVAL, "n_int must be a positive multiple of 16");
    corr* h = new corr();
    h->n_ant = n_ant;
    h->n_pol = n_pol;
    h->n_in = n_ant * n_pol;
    h->n_fft = n_fft;
    h->n_chan = n_fft / 2;
    h->n_int = n_int;
    h->n_bl = n_ant * (n_ant + 1) / 2;
    h->npp = n_pol * n_pol;
    h->tau.assign(n_ant, 0.0);
    h->phi0.assign(n_ant, 0.0);
    h->rate.assign(n_ant, 0.0);
    auto bail = [&](int rc) {
        corr_destroy(h);
        return rc;
    };
#define CUB(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return bail(fail(CORR_E_NOMEM, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)
    CUB(cudaGetDevice(&h->dev));
    CUB(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev));
    CUB(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CUB(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    CUB(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
    CUB(cudaEventCreateWithFlags(&h->ev_aux, cudaEventDisableTiming));
    CUB(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
    CUB(cudaEventCreateWithFlags(&h->ev_ws, cudaEventDisableTiming));
    for (int r = 0; r < 2; ++r) {
        CUB(cudaEventCreateWithFlags(&h->ev_ready[r], cudaEventDisableTiming));
        CUB(cudaEventCreateWithFlags(&h->ev_free[r], cudaEventDisableTiming));
    }
    const size_t nch = h->n_chan, na = n_ant, ni = h->n_in;
    CUB(dalloc(&h->d_model, 3 * na));
    CUB(cudaMallocHost(reinterpret_cast<void**>(&h->h_model), (1 + corr::kModelSlots) * 3 * na * sizeof(double)));
    for (cudaEvent_t& e : h->ev_model) CUB(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CUB(dalloc(&h->d_pf, na * nch));
    CUB(dalloc(&h->d_ff, na * static_cast<size_t>(n_int)));
    CUB(dalloc(&h->d_D, na));
    CUB(dalloc(&h->d_wcoh, na * nch));
    CUB(dalloc(&h->d_ginc, na));
    CUB(dalloc(&h->d_scale, ni * nch));
    const size_t spec_bytes = nch * static_cast<size_t>(n_int) * rows_fp32(h->n_in) * sizeof(float);
    CUB(cudaMalloc(&h->d_spec, spec_bytes));
    CUB(cudaMemset(h->d_spec, 0, spec_bytes));   // padding rows of the FP32 layout stay zero
    CUB(dalloc(&h->d_beams_raw, 2 * static_cast<size_t>(n_int) * nch));
    h->d_beams = h->d_beams_raw;
    const size_t nvis = nch * h->n_bl * h->npp;
    CUB(dalloc(&h->d_vis, nvis));
    CUB(dalloc(&h->d_vis_part, corr::kVisSplit * nvis));
    CUB(dalloc(&h->d_vis_int, nvis));
    CUB(dalloc(&h->d_err, 1));
    CUB(cudaMemset(h->d_err, 0, sizeof(unsigned)));
    CUB(cudaMemset(h->d_vis, 0, nvis * sizeof(float2)));
    CUB(cudaMemset(h->d_vis_int, 0, nvis * sizeof(int2)));
    CUB(cudaMemset(h->d_scale, 0, ni * nch * sizeof(float)));
    CUB(dalloc(&h->d_tw, static_cast<size_t>(fengine_tw_count(n_fft))));
    CUB(launch_fengine_twiddles(n_fft, h->d_tw, h->stream));
    CUB(cudaStreamSynchronize(h->stream));
#undef CUB
    if (xengine_tc_supported(h->n_in)) {
        const int rb = 2 * h->n_in > 128 ? 2 : 1;
        // row block outermost: the CTAs stride the list by the SM count, so interleaving a 256-row
        // Gram's wide (rows 0-127 x 256 columns) and narrow items per channel would hand each CTA
        // items of one kind only; wide ones first spreads both kinds over every CTA
        std::vector<int4> items;
        for (int r = 0; r < rb; ++r)
            for (int k = 0; k < h->n_chan; ++k) items.push_back(make_int4(0, k, r, 0));
        h->n_items = static_cast<int>(items.size());
        if (cudaMalloc(&h->d_xtab, sizeof(XtBatch)) != cudaSuccess ||
            cudaMalloc(&h->d_items, sizeof(int4) * items.size()) != cudaSuccess ||
            cudaMemcpy(h->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(CORR_E_NOMEM, "tensor-core tables"));
    }
    int rc = upload_beam_weights(h, nullptr, nullptr, nullptr, nullptr);
    if (rc == CORR_OK) rc = upload_xtab(h);
    if (rc != CORR_OK) return bail(rc);
    *out = h;
    return CORR_OK;
}

int corr_destroy(corr_t* h) {
    if (!h) return CORR_OK;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->cstream) cudaStreamSynchronize(h->cstream);
    if (h->ustream) cudaStreamSynchronize(h->ustream);
    if (h->ostream) cudaStreamSynchronize(h->ostream);
    if (h->d_power) cudaFree(h->d_power);
    if (h->d_noise) cudaFree(h->d_noise);
    if (h->d_blank) cudaFree(h->d_blank);
    if (h->d_blanked) cudaFree(h->d_blanked);
    if (h->d_mbw) cudaFree(h->d_mbw);
    if (h->d_mb) cudaFree(h->d_mb);
    if (h->d_stage4) cudaFree(h->d_stage4);
    if (h->d_unpack) cudaFree(h->d_unpack);
    if (h->d_xtab) cudaFree(h->d_xtab);
    if (h->d_items) cudaFree(h->d_items);
    if (h->vis_b[1]) {                   // the second output buffers (the current may be either)
        select_outputs(h, 0);
        if (h->beams_b[1] != h->beams_raw_b[1]) cudaFree(h->beams_b[1]);
        cudaFree(h->beams_raw_b[1]);
        cudaFree(h->vis_b[1]);
    }
    if (h->xtab_b1) cudaFree(h->xtab_b1);
    void* bufs[] = {h->d_ring, h->d_ring2, h->d_model, h->d_pf, h->d_ff, h->d_D, h->d_wcoh, h->d_ginc, h->d_scale,
                    h->d_tw, h->d_spec, h->d_beams_raw, h->d_vis, h->d_vis_part, h->d_vis_int, h->d_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->d_beams && h->d_beams != h->d_beams_raw) cudaFree(h->d_beams);
    if (h->h_model) cudaFreeHost(h->h_model);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    if (h->ev_aux) cudaEventDestroy(h->ev_aux);
    if (h->ev_copied) cudaEventDestroy(h->ev_copied);
    if (h->ev_ws) cudaEventDestroy(h->ev_ws);
    for (int k = 0; k < corr::kStage4Slots; ++k) {
        if (h->ev_s4[k]) cudaEventDestroy(h->ev_s4[k]);
        if (h->ev_s4_free[k]) cudaEventDestroy(h->ev_s4_free[k]);
    }
    for (int r = 0; r < 2; ++r) {
        if (h->ev_ready[r]) cudaEventDestroy(h->ev_ready[r]);
        if (h->ev_free[r]) cudaEventDestroy(h->ev_free[r]);
    }
    for (cudaEvent_t e : h->ev_out) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_model)
        if (e) cudaEventDestroy(e);
    if (h->ev_int_done) cudaEventDestroy(h->ev_int_done);
    for (cudaEvent_t e : h->ev_buf_free)
        if (e) cudaEventDestroy(e);
    if (h->ostream) cudaStreamDestroy(h->ostream);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->ustream) cudaStreamDestroy(h->ustream);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return CORR_OK;
}

int corr_set_mode(corr_t* h, int xmode, int polmode, int beam_avg) {
    if (int rc = check_handle(h)) return rc;
    if (xmode != CORR_FP32 && xmode != CORR_I8 && xmode != CORR_F16 && xmode != CORR_FP32TC)
        return fail(CORR_E_INVAL, "unknown xmode");
    if (xmode == CORR_FP32TC && h->batch_refs > 0)
        return fail(CORR_E_STATE, "CORR_FP32TC is not available to batch members");
    if (polmode != CORR_POL_FULL && polmode != CORR_POL_SELF)
        return fail(CORR_E_INVAL, "polmode must be CORR_POL_FULL or CORR_POL_SELF");
    if (h->out_vis && polmode != h->polmode)
        return fail(CORR_E_STATE, "polmode sizes the output ring and its buffers: remove the ring first");
    if (beam_avg < 1 || h->n_int % beam_avg) return fail(CORR_E_INVAL, "beam_avg must divide n_int");
    if (h->out_vis && beam_avg != h->beam_avg)
        return fail(CORR_E_STATE, "beam_avg sizes the output ring and its buffers: remove the ring first");
    if (xmode != CORR_FP32 && !xengine_tc_supported(h->n_in))
        return fail(CORR_E_INVAL, "tensor-core modes need n_in <= 128");
    if (xmode == CORR_I8 && h->n_int > 66571) return fail(CORR_E_INVAL, "CORR_I8 needs n_int <= 66571");
    CU(cudaStreamSynchronize(h->cstream));
    if (h->ustream) CU(cudaStreamSynchronize(h->ustream));
    CU(cudaStreamSynchronize(h->stream));
    if (beam_avg != h->beam_avg) {
        if (h->d_beams != h->d_beams_raw) cudaFree(h->d_beams);
        h->d_beams = h->d_beams_raw;
        if (beam_avg > 1) CU(dalloc(&h->d_beams, 2 * static_cast<size_t>(h->n_int / beam_avg) * h->n_chan));
    }
    const bool changed = h->xmode != xmode || h->polmode != polmode;
    if (h->xmode != xmode && xmode == CORR_FP32) {   // the FP32 layout's padding rows must read as zero again
        const size_t spec_bytes = static_cast<size_t>(h->n_chan) * h->n_int * rows_fp32(h->n_in) * sizeof(float);
        CU(cudaMemset(h->d_spec, 0, spec_bytes));
    }
    h->xmode = xmode;
    h->beam_avg = beam_avg;
    h->polmode = polmode;
    h->npp = polmode == CORR_POL_SELF ? h->n_pol : h->n_pol * h->n_pol;
    return changed ? upload_xtab(h) : CORR_OK;
}

int corr_set_xengine_stage(corr_t* h, int ks) {
    if (int rc = check_handle(h)) return rc;
    if (ks != 0 && (ks < 16 || ks > 512 || (ks & (ks - 1)) || ks > xengine_tc_max_ks(h->n_in)))
        return fail(CORR_E_INVAL, "stage must be 0 or a power of two in [16, %d]", xengine_tc_max_ks(h->n_in));
    h->ks = ks;
    return upload_xtab(h);
}

int corr_set_max_delay(corr_t* h, int max_delay) {
    if (int rc = check_handle(h)) return rc;
    if (h->ring_started) return fail(CORR_E_STATE, "max_delay is fixed once samples have been pushed");
    if (max_delay < 0 || max_delay > (1 << 24)) return fail(CORR_E_INVAL, "max_delay out of range");
    h->max_delay = max_delay;
    if (h->d_ring) return alloc_ring(h);
    return CORR_OK;
}

int corr_set_delays(corr_t* h, const double* delay, const double* phi0, const double* rate) {
    if (int rc = check_handle(h)) return rc;
    for (int a = 0; a < h->n_ant; ++a) {
        const double t = delay ? delay[a] : 0.0;
        if (!std::isfinite(t) || t < 0.0 || std::floor(t + 0.5) > 2.0e9)
            return fail(CORR_E_RANGE, "delay[%d] = %g must be finite and >= 0", a, t);
        if ((phi0 && !std::isfinite(phi0[a])) || (rate && !std::isfinite(rate[a])))
            return fail(CORR_E_INVAL, "fringe model of antenna %d is not finite", a);
    }
    for (int a = 0; a < h->n_ant; ++a) {
        h->tau[a] = delay ? delay[a] : 0.0;
        h->phi0[a] = phi0 ? phi0[a] : 0.0;
        h->rate[a] = rate ? rate[a] : 0.0;
    }
    return CORR_OK;
}

int corr_set_beam_weights(corr_t* h, const float* gain, const float* theta, const uint8_t* inc_mask,
                          const uint8_t* coh_mask) {
    if (int rc = check_handle(h)) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return upload_beam_weights(h, gain, theta, inc_mask, coh_mask);
}

int corr_set_scales(corr_t* h, const float* scale) {
    if (int rc = check_handle(h)) return rc;
    const size_t n = static_cast<size_t>(h->n_in) * h->n_chan;
    std::vector<float> s(n);
    if (scale) {
        for (size_t q = 0; q < n; ++q) {
            if (!(scale[q] > 0.0f) || !std::isfinite(scale[q]))
                return fail(CORR_E_INVAL, "scale[%zu] must be finite and > 0", q);
            s[q] = scale[q];
        }
    } else {
        if (int rc = settle(h, 1)) return rc;
        std::vector<float2> v(static_cast<size_t>(h->n_chan) * h->n_bl * h->npp);
        CU(cudaMemcpy(v.data(), h->d_vis, v.size() * sizeof(float2), cudaMemcpyDeviceToHost));
        for (int i = 0; i < h->n_in; ++i) {
            const int a = i / h->n_pol, p = i % h->n_pol;
            const int bl = a * h->n_ant - a * (a - 1) / 2;
            for (int k = 0; k < h->n_chan; ++k) {
                const double auto_p =
                    v[(static_cast<size_t>(k) * h->n_bl + bl) * h->npp + vis_prod(h->polmode == CORR_POL_SELF, h->n_pol, p, p)].x;
                // sigma of one component: half the channel's power for the circular statistics of
                // k > 0; at DC the spectrum of a real stream is real before the Eq. 2 rotation, so a
                // frame's whole power can sit in one component -- take the full power there
                const double sigma = std::sqrt(std::max(auto_p, 0.0) / ((k == 0 ? 1.0 : 2.0) * h->n_int));
                s[static_cast<size_t>(i) * h->n_chan + k] = sigma > 0 ? static_cast<float>(127.0 / (4.0 * sigma)) : 1.0f;
            }
        }
    }
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemcpy(h->d_scale, s.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    h->scales_set = true;
    return CORR_OK;
}

int corr_push_samples(corr_t* h, const int8_t* x, int64_t n, int64_t seq) {
    if (int rc = check_handle(h)) return rc;
    if (!x || n < 0) return fail(CORR_E_INVAL, "bad sample buffer");
    if (n == 0) return CORR_OK;
    if (!h->d_ring)
        if (int rc = alloc_ring(h)) return rc;
    auto put = [&](int8_t* dst, int64_t take, int64_t done) -> int {
        CU(cudaMemcpy2DAsync(dst, h->ring_ld, x + done, n, take, h->n_in, cudaMemcpyHostToDevice, h->cstream));
        return CORR_OK;
    };
    return ingest(h, put, n, seq, true, h->cstream);
}

int corr_push_samples_4bit(corr_t* h, const uint8_t* packed, int64_t ld, int64_t n, int64_t seq) {
    if (int rc = check_handle(h)) return rc;
    if (h->n_in % 4) return fail(CORR_E_INVAL, "4-bit ADC ingest needs n_in a multiple of 4 (4 inputs per card)");
    if (!packed || n < 0 || (ld & 1) || ld < 2 * n) return fail(CORR_E_INVAL, "bad packed buffer (ld even, >= 2 n)");
    if (n == 0) return CORR_OK;
    if (!h->d_ring)
        if (int rc = alloc_ring(h)) return rc;
    const int n_cards = h->n_in / 4;
    constexpr int64_t kS = corr::kStage4, kP = corr::kStage4Pitch;
    if (!h->d_stage4) {
        int lo = 0, hi = 0;
        CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        if (!h->ustream) CU(cudaStreamCreateWithPriority(&h->ustream, cudaStreamNonBlocking, hi));
        for (int k = 0; k < corr::kStage4Slots; ++k) {
            if (!h->ev_s4[k]) CU(cudaEventCreateWithFlags(&h->ev_s4[k], cudaEventDisableTiming));
            if (!h->ev_s4_free[k]) CU(cudaEventCreateWithFlags(&h->ev_s4_free[k], cudaEventDisableTiming));
        }
        CU(cudaMalloc(&h->d_stage4, static_cast<size_t>(corr::kStage4Slots) * n_cards * kP));
    }
    auto put = [&](int8_t* dst, int64_t take, int64_t done) -> int {
        for (int64_t q = 0; q < take; q += kS) {   // packed pieces through the staging slots
            const int64_t len = std::min<int64_t>(kS, take - q);
            const int k = h->s4_next;
            h->s4_next = (k + 1) % corr::kStage4Slots;
            // the copy lands at the offset that puts the input of the first 16-byte aligned
            // output sample on a 16-byte boundary (the unpack's vector path)
            const int64_t off = (2 * static_cast<int64_t>(reinterpret_cast<uintptr_t>(dst + q) & 15)) & 15;
            uint8_t* slot = h->d_stage4 + static_cast<size_t>(k) * n_cards * kP + off;
            CU(cudaStreamWaitEvent(h->cstream, h->ev_s4_free[k], 0));
            CU(cudaMemcpy2DAsync(slot, kP, packed + 2 * (done + q), ld, 2 * len, n_cards, cudaMemcpyHostToDevice,
                                 h->cstream));
            CU(cudaEventRecord(h->ev_s4[k], h->cstream));
            CU(cudaStreamWaitEvent(h->ustream, h->ev_s4[k], 0));
            CU(launch_unpack4(slot, kP, n_cards, len, dst + q, h->ring_ld, h->n_sm, h->ustream));
            CU(cudaEventRecord(h->ev_s4_free[k], h->ustream));
        }
        return CORR_OK;
    };
    return ingest(h, put, n, seq, true, h->ustream);
}

int corr_set_output_ring(corr_t* h, float* vis, float* beams, int n_slots) {
    if (int rc = check_handle(h)) return rc;
    if (vis && (n_slots < 1 || n_slots > 4096)) return fail(CORR_E_INVAL, "n_slots must be in [1, 4096]");
    if (vis && h->batch_refs > 0) return fail(CORR_E_STATE, "the handle belongs to a batch (captured graph)");
    CU(cudaStreamSynchronize(h->cstream));
    if (h->ustream) CU(cudaStreamSynchronize(h->ustream));
    CU(cudaStreamSynchronize(h->stream));
    if (h->ostream) CU(cudaStreamSynchronize(h->ostream));
    for (cudaEvent_t e : h->ev_out) cudaEventDestroy(e);
    h->ev_out.clear();
    h->slot_of.clear();
    h->out_vis = h->out_beams = nullptr;
    h->n_slots = 0;
    const size_t nv = static_cast<size_t>(h->n_chan) * h->n_bl * h->npp;
    const size_t nraw = 2 * static_cast<size_t>(h->n_int) * h->n_chan;
    const size_t navg = 2 * static_cast<size_t>(h->n_int / h->beam_avg) * h->n_chan;
    if (h->vis_b[1]) {
        // back to single outputs: keep the last results readable in buffer 0
        if (h->out_buf == 1) {
            CU(cudaMemcpy(h->vis_b[0], h->vis_b[1], nv * sizeof(float2), cudaMemcpyDeviceToDevice));
            CU(cudaMemcpy(h->beams_raw_b[0], h->beams_raw_b[1], nraw * sizeof(float), cudaMemcpyDeviceToDevice));
            if (h->beams_b[1] != h->beams_raw_b[1])
                CU(cudaMemcpy(h->beams_b[0], h->beams_b[1], navg * sizeof(float), cudaMemcpyDeviceToDevice));
            select_outputs(h, 0);
        }
        if (h->beams_b[1] != h->beams_raw_b[1]) cudaFree(h->beams_b[1]);
        cudaFree(h->beams_raw_b[1]);
        cudaFree(h->vis_b[1]);
        if (h->xtab_b1) cudaFree(h->xtab_b1);
        h->vis_b[1] = nullptr;
        h->beams_raw_b[1] = h->beams_b[1] = nullptr;
        h->xtab_b1 = nullptr;
        if (int rc = upload_xtab(h)) return rc;
    }
    if (!vis) return CORR_OK;
    h->vis_b[0] = h->d_vis;
    h->beams_raw_b[0] = h->d_beams_raw;
    h->beams_b[0] = h->d_beams;
    h->out_buf = 0;
    CU(dalloc(&h->vis_b[1], nv));
    CU(dalloc(&h->beams_raw_b[1], nraw));
    h->beams_b[1] = h->beams_raw_b[1];
    if (h->beam_avg > 1) CU(dalloc(&h->beams_b[1], navg));
    if (h->d_xtab) CU(cudaMalloc(&h->xtab_b1, sizeof(XtBatch)));
    if (int rc = upload_xtab(h)) return rc;
    if (!h->ostream) {
        CU(cudaStreamCreateWithFlags(&h->ostream, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&h->ev_int_done, cudaEventDisableTiming));
        for (cudaEvent_t& e : h->ev_buf_free) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    h->ev_out.resize(n_slots, nullptr);
    for (cudaEvent_t& e : h->ev_out) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->slot_of.assign(n_slots, -1);
    h->out_vis = vis;
    h->out_beams = beams;
    h->n_slots = n_slots;
    return CORR_OK;
}

int corr_wait_output(corr_t* h, int64_t index, int* slot) {
    if (int rc = check_handle(h)) return rc;
    if (!h->out_vis) return fail(CORR_E_STATE, "no output ring (corr_set_output_ring)");
    if (index < 0) return fail(CORR_E_INVAL, "index must be >= 0");
    if (index >= h->n_streamed) return fail(CORR_E_AGAIN, "integration %lld not launched yet", (long long)index);
    const int s = static_cast<int>(index % h->n_slots);
    if (h->slot_of[s] != index) return fail(CORR_E_STATE, "slot %d has been reused since integration %lld", s,
                                            (long long)index);
    CU(cudaEventSynchronize(h->ev_out[s]));
    unsigned err = 0;
    CU(cudaMemcpy(&err, h->d_err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(CORR_E_TIMEOUT, "a kernel wait timed out (error bits 0x%x); results invalid", err);
    if (slot) *slot = s;
    return CORR_OK;
}

int corr_push_samples_device(corr_t* h, const int8_t* x, int64_t n, int64_t seq, void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!x || n < 0) return fail(CORR_E_INVAL, "bad sample buffer");
    if (n == 0) return CORR_OK;
    if (!h->d_ring)
        if (int rc = alloc_ring(h)) return rc;
    // order the copy after the caller's producer work
    CU(cudaEventRecord(h->ev_aux, static_cast<cudaStream_t>(stream)));
    CU(cudaStreamWaitEvent(h->cstream, h->ev_aux, 0));
    auto put = [&](int8_t* dst, int64_t take, int64_t done) -> int {
        CU(cudaMemcpy2DAsync(dst, h->ring_ld, x + done, n, take, h->n_in, cudaMemcpyDeviceToDevice, h->cstream));
        return CORR_OK;
    };
    return ingest(h, put, n, seq, false, h->cstream);
}

int corr_integrate_4bit_device(corr_t* h, const uint8_t* packed, int64_t ld, int64_t n_avail, int64_t g0,
                               void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (h->n_in % 4) return fail(CORR_E_INVAL, "4-bit ADC ingest needs n_in a multiple of 4 (4 inputs per card)");
    if (!packed || (ld & 1) || ld < 2 * n_avail || (reinterpret_cast<uintptr_t>(packed) & 1))
        return fail(CORR_E_INVAL, "packed must be 2-byte aligned with an even ld >= 2 n_avail");
    const int64_t need = static_cast<int64_t>(h->n_int) * h->n_fft + max_int_delay(h);
    if (n_avail < need)
        return fail(CORR_E_RANGE, "n_avail = %lld < n_int * n_fft + max delay = %lld", (long long)n_avail,
                    (long long)need);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    const int64_t ldu = ((n_avail + 15) / 16) * 16 + 16;
    if (ldu > h->unpack_ld) {   // grow the unpacked rows (the stream is drained first)
        CU(cudaStreamSynchronize(s));
        CU(cudaStreamSynchronize(h->stream));
        if (h->d_unpack) cudaFree(h->d_unpack);
        h->d_unpack = nullptr;
        h->unpack_ld = 0;
        CU(cudaMalloc(&h->d_unpack, static_cast<size_t>(h->n_in) * ldu));
        h->unpack_ld = ldu;
    }
    CU(launch_unpack4(packed, ld, h->n_in / 4, n_avail, h->d_unpack, h->unpack_ld, h->n_sm, s));
    return run_integration(h, h->d_unpack, h->unpack_ld, n_avail, g0, s);
}

int corr_integrate_device(corr_t* h, const int8_t* x, int64_t ld, int64_t n_avail, int64_t g0, void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!x || (reinterpret_cast<uintptr_t>(x) & 15) || (ld & 15) || ld < n_avail)
        return fail(CORR_E_INVAL, "x and ld must be 16-byte aligned and ld >= n_avail");
    const int64_t need = static_cast<int64_t>(h->n_int) * h->n_fft + max_int_delay(h);
    if (n_avail < need)
        return fail(CORR_E_RANGE, "n_avail = %lld < n_int * n_fft + max delay = %lld", (long long)n_avail,
                    (long long)need);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    return run_integration(h, x, ld, n_avail, g0, s);
}

int corr_read_visibilities(corr_t* h, float* out, int blocking) {
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(CORR_E_INVAL, "out is null");
    if (int rc = settle(h, blocking)) return rc;
    CU(cudaMemcpy(out, h->d_vis, static_cast<size_t>(h->n_chan) * h->n_bl * h->npp * sizeof(float2),
                  cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int corr_read_beams(corr_t* h, float* out, int blocking) {
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(CORR_E_INVAL, "out is null");
    if (int rc = settle(h, blocking)) return rc;
    CU(cudaMemcpy(out, h->d_beams, 2 * static_cast<size_t>(h->n_int / h->beam_avg) * h->n_chan * sizeof(float),
                  cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int corr_read_vis_int(corr_t* h, int32_t* out, int blocking) {
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(CORR_E_INVAL, "out is null");
    if (int rc = settle(h, blocking)) return rc;
    if (h->last_mode != CORR_I8) return fail(CORR_E_STATE, "last integration was not CORR_I8");
    CU(cudaMemcpy(out, h->d_vis_int, static_cast<size_t>(h->n_chan) * h->n_bl * h->npp * sizeof(int2),
                  cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int corr_read_requant(corr_t* h, int k0, int nk, int8_t* q, float* scale) {
    if (int rc = check_handle(h)) return rc;
    if (int rc = settle(h, 1)) return rc;
    if (h->last_mode != CORR_I8) return fail(CORR_E_STATE, "last integration was not CORR_I8");
    if (k0 < 0 || nk < 0 || k0 + nk > h->n_chan) return fail(CORR_E_INVAL, "channel range");
    if (scale)
        CU(cudaMemcpy(scale, h->d_scale, static_cast<size_t>(h->n_in) * h->n_chan * sizeof(float),
                      cudaMemcpyDeviceToHost));
    if (q && nk > 0) {
        // int8 bytes in the channel-quad layout (OUT_I8B: i8q_piece): the quads covering k0 .. k0 + nk - 1
        const int R = 2 * h->n_in, ntb = h->n_int / kTbHalf;
        const size_t per_ch = static_cast<size_t>(ntb) * R * kTbHalf;
        const int q0 = k0 / 4, q1 = (k0 + nk + 3) / 4;
        std::vector<int8_t> buf8(per_ch * 4 * (q1 - q0));
        CU(cudaMemcpy(buf8.data(), static_cast<const int8_t*>(h->d_spec) + per_ch * 4 * q0, buf8.size(),
                      cudaMemcpyDeviceToHost));
        for (int c = 0; c < nk; ++c)
            for (int kb = 0; kb < ntb; ++kb)
                for (int r = 0; r < R; ++r)
                    for (int e = 0; e < kTbHalf; ++e) {
                        const int i = r / 2, cc = r % 2, t = kb * kTbHalf + e;
                        q[((static_cast<size_t>(i) * h->n_int + t) * nk + c) * 2 + cc] =
                            buf8[i8q_piece(k0 + c - 4 * q0, kb, i, ntb, h->n_in) + cc * kTbHalf + e];
                    }
    }
    return CORR_OK;
}

int corr_read_spectra(corr_t* h, int k0, int nk, float* out) {
    if (int rc = check_handle(h)) return rc;
    if (int rc = settle(h, 1)) return rc;
    if (h->last_mode != CORR_FP32 && h->last_mode != CORR_FP32TC)
        return fail(CORR_E_STATE, "last integration was not CORR_FP32 or CORR_FP32TC");
    if (!out || k0 < 0 || nk < 0 || k0 + nk > h->n_chan) return fail(CORR_E_INVAL, "channel range");
    const int tb = tb_fp32(h->n_chan);
    const int R = 2 * h->n_in, Rp = rows_fp32(h->n_in), ntb = h->n_int / tb;
    if (h->last_quad) {   // channel-quad layout: the quads covering channels k0 .. k0 + nk - 1
        const int q0 = k0 / 4, q1 = (k0 + nk + 3) / 4;
        const size_t per_q = static_cast<size_t>(ntb) * h->n_in * 64;
        std::vector<float> buf(per_q * (q1 - q0));
        CU(cudaMemcpy(buf.data(), static_cast<const float*>(h->d_spec) + per_q * q0, buf.size() * sizeof(float),
                      cudaMemcpyDeviceToHost));
        for (int c = 0; c < nk; ++c)
            for (int kb = 0; kb < ntb; ++kb)
                for (int i = 0; i < h->n_in; ++i)
                    for (int cc = 0; cc < 2; ++cc)
                        for (int e = 0; e < tb; ++e) {
                            const int k = k0 + c, t = kb * tb + e;
                            out[((static_cast<size_t>(i) * h->n_int + t) * nk + c) * 2 + cc] =
                                buf[f32q_piece(k, kb, i, ntb, h->n_in) - static_cast<int64_t>(per_q) * q0 + cc * 8 + e];
                        }
        return CORR_OK;
    }
    const size_t per_ch = static_cast<size_t>(ntb) * Rp * tb;
    std::vector<float> buf(per_ch * nk);
    CU(cudaMemcpy(buf.data(), static_cast<const float*>(h->d_spec) + per_ch * k0, buf.size() * sizeof(float),
                  cudaMemcpyDeviceToHost));
    for (int c = 0; c < nk; ++c)
        for (int kb = 0; kb < ntb; ++kb)
            for (int r = 0; r < R; ++r)
                for (int e = 0; e < tb; ++e) {
                    const int i = r / 2, cc = r % 2, t = kb * tb + e;
                    out[((static_cast<size_t>(i) * h->n_int + t) * nk + c) * 2 + cc] =
                        buf[(static_cast<size_t>(c) * ntb + kb) * Rp * tb + fp32_off(r, e, tb)];
                }
    return CORR_OK;
}

int corr_device_outputs(corr_t* h, void** vis, void** beams, void** stream) {
    if (int rc = check_handle(h)) return rc;
    if (vis) *vis = h->d_vis;
    if (beams) *beams = h->d_beams;
    if (stream) *stream = h->stream;
    return CORR_OK;
}

int corr_set_power_dump(corr_t* h, int dump) {
    if (int rc = check_handle(h)) return rc;
    if (dump < 0 || (dump > 0 && (dump % tb_fp32(h->n_chan) || h->n_int % dump)))
        return fail(CORR_E_INVAL, "dump must be 0 or a multiple of %d dividing n_int", tb_fp32(h->n_chan));
    CU(cudaStreamSynchronize(h->stream));
    if (h->d_power) cudaFree(h->d_power);
    h->d_power = nullptr;
    h->dump = dump;
    if (dump > 0) {
        CU(dalloc(&h->d_power, static_cast<size_t>(h->n_in) * (h->n_int / dump) * h->n_chan));
        CU(cudaMemset(h->d_power, 0, sizeof(float) * h->n_in * (h->n_int / dump) * h->n_chan));
    }
    return CORR_OK;
}

int corr_set_blanker(corr_t* h, double M, int block, const float* noise, int L) {
    if (int rc = check_handle(h)) return rc;
    if (!(M >= 0.0) || !std::isfinite(M)) return fail(CORR_E_INVAL, "M must be finite and >= 0");
    if (h->batch_refs > 0) return fail(CORR_E_STATE, "the voltage blanker runs per handle, not in batches");
    CU(cudaStreamSynchronize(h->stream));
    if (h->d_noise) cudaFree(h->d_noise);
    if (h->d_blank) cudaFree(h->d_blank);
    if (h->d_blanked) cudaFree(h->d_blanked);
    h->d_noise = nullptr;
    h->d_blank = nullptr;
    h->d_blanked = nullptr;
    h->blank_M = 0.0;
    h->blank_cap = h->blank_nb = h->blank_n = 0;
    if (M == 0.0) return CORR_OK;
    int lg = 0;
    while ((1 << lg) < block && lg < 30) ++lg;
    if (block < 4096 || block > 32768 || (1 << lg) != block)
        return fail(CORR_E_INVAL, "block must be a power of two in [4096, 32768]");
    if (!noise || L < 1 || L > (1 << 24) || (L & (L - 1))) return fail(CORR_E_INVAL, "noise table: L a power of two in [1, 2^24]");
    const size_t nn = static_cast<size_t>(h->n_in) * L;
    CU(dalloc(&h->d_noise, nn));
    CU(cudaMemcpy(h->d_noise, noise, nn * sizeof(float), cudaMemcpyHostToDevice));
    h->blank_cap = (static_cast<int64_t>(h->n_int) * h->n_fft + h->max_delay + block - 1) / block;
    CU(cudaMalloc(&h->d_blank, sizeof(int32_t) * 4 * static_cast<size_t>(h->n_in) * h->blank_cap));
    h->blanked_ld = h->blank_cap * block;   // block: a power of two >= 4096, so a multiple of 16
    CU(cudaMalloc(&h->d_blanked, static_cast<size_t>(h->n_in) * h->blanked_ld));
    h->blank_M = M;
    h->blank_log2 = lg;
    h->noise_L = L;
    return CORR_OK;
}

int corr_set_multibeam(corr_t* h, int n_beams, const float* weights, int products, int avg) {
    if (int rc = check_handle(h)) return rc;
    if (n_beams < 0 || n_beams > multibeam_max_beams())
        return fail(CORR_E_INVAL, "n_beams must be in [0, %d]", multibeam_max_beams());
    if (n_beams > 0) {
        const int fcta = avg > 64 ? avg : 64;
        if (avg < 1 || (avg & (avg - 1)) || h->n_int % fcta)
            return fail(CORR_E_INVAL, "avg must be a power of two with max(64, avg) dividing n_int");
        if (products != CORR_BEAM_FULLPOL && products != CORR_BEAM_VOLTAGE) return fail(CORR_E_INVAL, "unknown products");
        if (products == CORR_BEAM_VOLTAGE && avg != 1) return fail(CORR_E_INVAL, "beam voltages need avg = 1");
        if (!weights) return fail(CORR_E_INVAL, "weights required");
    }
    CU(cudaStreamSynchronize(h->stream));
    if (h->d_mbw) cudaFree(h->d_mbw);
    if (h->d_mb) cudaFree(h->d_mb);
    h->d_mbw = nullptr;
    h->d_mb = nullptr;
    h->n_mb = 0;
    // the layout of the CORR_FP32TC hand-off depends on whether phased beams read it
    if (n_beams == 0) return upload_xtab(h);
    // weights [beam][antenna][channel] -> [channel][beam * n_ant + antenna] (padded to even)
    const int ws = multibeam_wstride(n_beams, h->n_ant);
    std::vector<float2> w(static_cast<size_t>(h->n_chan) * ws, make_float2(0.0f, 0.0f));
    for (int b = 0; b < n_beams; ++b)
        for (int a = 0; a < h->n_ant; ++a)
            for (int k = 0; k < h->n_chan; ++k) {
                const float* src = weights + 2 * ((static_cast<size_t>(b) * h->n_ant + a) * h->n_chan + k);
                w[static_cast<size_t>(k) * ws + b * h->n_ant + a] = make_float2(src[0], src[1]);
            }
    CU(dalloc(&h->d_mbw, w.size()));
    CU(cudaMemcpy(h->d_mbw, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice));
    const size_t n_out = static_cast<size_t>(n_beams) * (h->n_int / avg) * h->n_chan;
    CU(dalloc(&h->d_mb, n_out));
    CU(cudaMemset(h->d_mb, 0, n_out * sizeof(float4)));
    h->n_mb = n_beams;
    h->mb_products = products;
    h->mb_avg = avg;
    return upload_xtab(h);
}

int corr_read_multibeam(corr_t* h, float* out, int blocking) {
    if (int rc = check_handle(h)) return rc;
    if (h->n_mb == 0) return fail(CORR_E_STATE, "multiple beams are off (corr_set_multibeam)");
    if (!out) return fail(CORR_E_INVAL, "out required");
    if (int rc = settle(h, blocking)) return rc;
    CU(cudaMemcpy(out, h->d_mb, sizeof(float4) * static_cast<size_t>(h->n_mb) * (h->n_int / h->mb_avg) * h->n_chan,
                  cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int corr_read_blank_stats(corr_t* h, int32_t* out, int64_t* n_blocks, int64_t* n_samples) {
    if (int rc = check_handle(h)) return rc;
    if (h->blank_M == 0.0) return fail(CORR_E_STATE, "the voltage blanker is off (corr_set_blanker)");
    if (h->blank_nb == 0) return fail(CORR_E_STATE, "no integration with the blanker yet");
    if (int rc = settle(h, 1)) return rc;
    if (n_blocks) *n_blocks = h->blank_nb;
    if (n_samples) *n_samples = h->blank_n;
    if (out)
        CU(cudaMemcpy(out, h->d_blank, sizeof(int32_t) * 4 * static_cast<size_t>(h->n_in) * h->blank_nb,
                      cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int corr_read_power(corr_t* h, float* out, void** device_ptr) {
    if (int rc = check_handle(h)) return rc;
    if (h->dump == 0) return fail(CORR_E_STATE, "power dumps are off (corr_set_power_dump)");
    if (device_ptr) *device_ptr = h->d_power;
    if (out) {
        if (int rc = settle(h, 1)) return rc;
        CU(cudaMemcpy(out, h->d_power, sizeof(float) * h->n_in * (h->n_int / h->dump) * h->n_chan,
                      cudaMemcpyDeviceToHost));
    }
    return CORR_OK;
}

int corr_set_timing(corr_t* h, int enable) {
    if (int rc = check_handle(h)) return rc;
    if (enable && h->tev.empty()) {
        h->tev.resize(static_cast<size_t>(kTimedMax) * (kStages + 1), nullptr);
        for (auto& e : h->tev) CU(cudaEventCreate(&e));
    }
    h->timing = enable != 0;
    h->t_count = 0;
    return CORR_OK;
}

int corr_stage_times(corr_t* h, float* ms4, int* n) {
    if (int rc = check_handle(h)) return rc;
    if (!ms4 || !n) return fail(CORR_E_INVAL, "null output");
    for (int b = 0; b < kStages; ++b) ms4[b] = 0.0f;
    *n = h->t_count;
    for (int t = 0; t < h->t_count; ++t) {
        cudaEvent_t* e = &h->tev[static_cast<size_t>(t) * (kStages + 1)];
        CU(cudaEventSynchronize(e[kStages]));
        for (int b = 0; b < kStages; ++b) {
            float ms = 0.0f;
            CU(cudaEventElapsedTime(&ms, e[b], e[b + 1]));
            ms4[b] += ms;
        }
    }
    h->t_count = 0;
    return CORR_OK;
}

int corr_info(corr_t* h, int64_t* out6) {
    if (!h || !out6) return fail(CORR_E_INVAL, "null argument");
    out6[0] = h->n_in;
    out6[1] = h->n_bl;
    out6[2] = h->n_chan;
    out6[3] = h->npp;
    out6[4] = h->n_int / h->beam_avg;
    out6[5] = h->completed;
    return CORR_OK;
}

}  // extern "C"
