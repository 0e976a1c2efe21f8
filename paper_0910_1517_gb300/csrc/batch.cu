// batch.cu -- several sub-arrays of uneven sizes in one graph-captured launch, and
// the autotuner that picks the tensor-core X-engine's stage size per sub-array.
//
// The graph refreshes the batch's small tables (frame counters, X-engine tables) from pinned
// host copies, then forks one branch per sub-array: the upload of its delay model, its phasor
// set-up, its F-engine (the kernel a single handle of that FFT size and mode runs) and its
// X-engine (the persistent tensor-core kernel over that sub-array's (channel, row block) items,
// in the operand form its F-engine writes), then the optional dumps and beam averages; the
// branches join at the end.  Independent branches let the F-engine of one sub-array overlap
// the X-engine of another.  The graph is captured once and replayed for every integration;
// each replay first sets the F-engine nodes' parameters (new sample pointers) in the
// executable graph -- except where the F-engine runs in 2-CTA clusters, whose parameters are
// only ever those of a capture: new ones for such a node capture the graph again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/corr.h"
#include "fengine.cuh"
#include "handle.cuh"
#include "xengine.cuh"

using namespace gbx;

struct corr_batch {
    int n_sub = 0;
    corr* h[kMaxSub] = {};
    int fmode[kMaxSub] = {};       // F-engine output layout of each sub-array
    int xmode = 0, n_sm = 0, dev = 0;
    cudaStream_t cap = nullptr;
    cudaStream_t br[kMaxSub] = {};    // capture branches, one per sub-array
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxSub] = {};
    int64_t* h_g0 = nullptr;     // pinned: global frame index of each sub-array's first frame
    int64_t* d_g0 = nullptr;
    FeParams fe_p[kMaxSub] = {};              // F-engine parameters of the next replay
    FeParams cap_p[kMaxSub] = {};             // ... and those the graph was captured with
    cudaGraphNode_t fe_node[kMaxSub] = {};    // the F-engine kernel node of each branch
    cudaKernelNodeParams fe_kp[kMaxSub] = {};
    XtBatch* h_xt = nullptr;     // pinned, one one-entry table per sub-array
    XtBatch* d_xt = nullptr;
    int4* d_items[kMaxSub] = {};
    int n_items[kMaxSub] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;  // the last launch: guards the pinned tables
    bool pending = false;
};

namespace {

int bfail(int code, const char* msg) { return fail_code(code, msg); }

#define BCU(call)                                                   \
    do {                                                            \
        if ((call) != cudaSuccess) return bfail(CORR_E_CUDA, #call); \
    } while (0)

bool tc_mode(int xmode) { return xmode == CORR_I8 || xmode == CORR_F16; }

// (channel, row block) items of sub-array q, for its one-entry table (sub index 0): a 256-row
// Gram has two row blocks per channel; every channel's wide block first, as in the handle's own
// list, so that the CTAs striding the list get both kinds.
std::vector<int4> make_items(const corr_batch* b, int q) {
    std::vector<int4> items;
    const int R = 2 * b->h[q]->n_in, rbs = R > 128 ? 2 : 1;
    for (int r = 0; r < rbs; ++r)
        for (int k = 0; k < b->h[q]->n_chan; ++k) items.push_back(make_int4(0, k, r, 0));
    return items;
}

// sub-array q's one-entry X-engine table; false if the driver refuses its tensor map
bool fill_xt(const corr_batch* b, int q, XtBatch* t, const int4* items, int n_items) {
    std::memset(t, 0, sizeof *t);
    t->n_sub = 1;
    t->sub[0] = xt_sub_of(b->h[q]);   // in8 where the F-engine writes int8 bytes (OUT_I8B)
    t->n_items = n_items;
    t->items = items;
    t->err = b->h[q]->d_err;
    return !t->sub[0].in8 || xengine_tc_encode_quad(t->sub[0]);
}

int xt_form(const corr_batch* b, int q) { return b->fmode[q] == OUT_I8B ? XT_FORM_I8 : XT_FORM_F16; }

FeParams fe_params(corr* h, const int8_t* x, int64_t ld, int64_t n_avail) {
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
    return fp;
}

// Branch q of the graph: sub-array q's whole integration on stream s.
bool capture_branch(corr_batch* b, int q, cudaStream_t s) {
    corr* h = b->h[q];
    const int nd = h->n_ant;
    bool ok = cudaMemcpyAsync(h->d_model, h->h_model, 3 * nd * sizeof(double), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              launch_phasor_setup(h->n_ant, h->n_chan, h->n_fft, h->n_int, 0, h->d_model, h->d_model + nd,
                                  h->d_model + 2 * nd, h->d_pf, h->d_ff, h->d_D, s, b->d_g0 + q) == cudaSuccess;
    ok = ok && launch_fengine(b->fe_p[q], b->fmode[q], s) == cudaSuccess;
    if (ok) {   // the node just captured: its parameters are set again before every replay
        cudaStreamCaptureStatus st{};
        const cudaGraphNode_t* deps = nullptr;
        size_t n_deps = 0;
        ok = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &n_deps) == cudaSuccess &&
             st == cudaStreamCaptureStatusActive && n_deps == 1;
        if (ok) b->fe_node[q] = deps[0];
    }
    if (ok && tc_mode(b->xmode)) {
        ok = launch_xengine_tc_table(b->d_xt + q, b->n_items[q], b->n_sm, s, xt_form(b, q)) == cudaSuccess;
    } else if (ok) {
        XParams xp{};
        xp.spec = h->d_spec;
        xp.n_ant = h->n_ant;
        xp.n_pol = h->n_pol;
        xp.n_in = h->n_in;
        xp.n_chan = h->n_chan;
        xp.n_int = h->n_int;
        xp.scale = h->d_scale;
        xp.vis = h->d_vis;
        xp.err = h->d_err;
        xp.vis_part = h->d_vis_part;
        xp.max_split = corr::kVisSplit;
        xp.self = h->polmode == CORR_POL_SELF ? 1 : 0;
        ok = launch_xengine_fp32(xp, b->n_sm, s) == cudaSuccess;
    }
    if (ok && h->dump > 0 && b->xmode == CORR_FP32)
        ok = launch_power_dumps(static_cast<const float*>(h->d_spec), h->n_in, h->n_chan, h->n_int, h->dump,
                                h->d_power, s) == cudaSuccess;
    if (ok && h->beam_avg > 1)
        ok = launch_beam_average(h->d_beams_raw, h->d_beams, h->n_int, h->n_chan, h->beam_avg, s) == cudaSuccess;
    return ok;
}

// Capture the integration of every sub-array into one graph: the table refresh on the batch's
// stream, then one branch per sub-array, joined before the capture ends.
int capture(corr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t s = b->cap;
    BCU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    bool ok = cudaMemcpyAsync(b->d_g0, b->h_g0, b->n_sub * sizeof(int64_t), cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (ok && tc_mode(b->xmode))
        ok = cudaMemcpyAsync(b->d_xt, b->h_xt, b->n_sub * sizeof(XtBatch), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaEventRecord(b->fork, s) == cudaSuccess;
    for (int q = 0; ok && q < b->n_sub; ++q) {
        if (cudaStreamWaitEvent(b->br[q], b->fork, 0) != cudaSuccess) {
            ok = false;
            break;
        }
        ok = capture_branch(b, q, b->br[q]);
        // join even a failed branch, so that the capture ends cleanly
        const bool joined = cudaEventRecord(b->join[q], b->br[q]) == cudaSuccess &&
                            cudaStreamWaitEvent(s, b->join[q], 0) == cudaSuccess;
        ok = ok && joined;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (!ok || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(CORR_E_CUDA, "capturing the batch graph failed");
    }
    b->graph = g;
    BCU(cudaGraphInstantiate(&b->exec, g, 0));
    for (int q = 0; q < b->n_sub; ++q) b->cap_p[q] = b->fe_p[q];
    for (int q = 0; q < b->n_sub; ++q) BCU(cudaGraphKernelNodeGetParams(b->fe_node[q], &b->fe_kp[q]));
    return CORR_OK;
}

}  // namespace

extern "C" {

int corr_batch_create(corr_batch_t** out, int n_sub, corr_t* const* subs) {
    if (!out || !subs || n_sub < 1 || n_sub > kMaxSub) return bfail(CORR_E_INVAL, "need 1..8 sub-array handles");
    *out = nullptr;
    for (int s = 0; s < n_sub; ++s) {
        if (!subs[s]) return bfail(CORR_E_INVAL, "null sub-array handle");
        if (subs[s]->xmode != subs[0]->xmode) return bfail(CORR_E_INVAL, "sub-arrays must share one precision mode");
        if (subs[s]->xmode == CORR_FP32TC) return bfail(CORR_E_INVAL, "CORR_FP32TC runs per handle, not in batches");
        if (subs[s]->blank_M > 0.0) return bfail(CORR_E_INVAL, "the voltage blanker runs per handle, not in batches");
        if (subs[s]->out_vis) return bfail(CORR_E_STATE, "a sub-array handle has an output ring (double-buffered outputs)");
        for (int q = 0; q < s; ++q)
            if (subs[q] == subs[s]) return bfail(CORR_E_INVAL, "a handle appears twice");
    }
    corr_batch* b = new corr_batch();
    b->n_sub = n_sub;
    b->xmode = subs[0]->xmode;
    for (int s = 0; s < n_sub; ++s) {
        b->h[s] = subs[s];
        b->fmode[s] = fe_out_mode(subs[s]);
        subs[s]->batch_refs += 1;
    }
    auto bail = [&](const char* m) {
        corr_batch_destroy(b);
        return bfail(CORR_E_NOMEM, m);
    };
    if (cudaGetDevice(&b->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_g0), kMaxSub * sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_xt), n_sub * sizeof(XtBatch)) != cudaSuccess ||
        cudaMalloc(&b->d_g0, kMaxSub * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_xt, n_sub * sizeof(XtBatch)) != cudaSuccess)
        return bail("batch tables");
    for (int s = 0; s < n_sub; ++s)
        if (cudaStreamCreateWithFlags(&b->br[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming) != cudaSuccess)
            return bail("batch streams");
    std::memset(b->h_g0, 0, kMaxSub * sizeof(int64_t));
    if (tc_mode(b->xmode)) {
        for (int s = 0; s < n_sub; ++s) {
            const std::vector<int4> items = make_items(b, s);
            b->n_items[s] = static_cast<int>(items.size());
            if (cudaMalloc(&b->d_items[s], sizeof(int4) * items.size()) != cudaSuccess ||
                cudaMemcpy(b->d_items[s], items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess)
                return bail("batch items");
        }
    }
    *out = b;
    return CORR_OK;
}

int corr_batch_destroy(corr_batch_t* b) {
    if (!b) return CORR_OK;
    if (b->cap) cudaStreamSynchronize(b->cap);
    if (b->done) cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_g0) cudaFree(b->d_g0);
    if (b->d_xt) cudaFree(b->d_xt);
    for (int q = 0; q < kMaxSub; ++q) {
        if (b->d_items[q]) cudaFree(b->d_items[q]);
        if (b->join[q]) cudaEventDestroy(b->join[q]);
        if (b->br[q]) cudaStreamDestroy(b->br[q]);
    }
    if (b->h_g0) cudaFreeHost(b->h_g0);
    if (b->h_xt) cudaFreeHost(b->h_xt);
    if (b->done) cudaEventDestroy(b->done);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int q = 0; q < b->n_sub; ++q)   // the handles outlive their batches
        if (b->h[q]) b->h[q]->batch_refs -= 1;
    delete b;
    return CORR_OK;
}

int corr_batch_integrate_device(corr_batch_t* b, const int8_t* const* x, const int64_t* ld, const int64_t* n_avail,
                                const int64_t* g0, void* stream) {
    if (!b || !x || !ld || !n_avail) return bfail(CORR_E_INVAL, "null argument");
    BCU(cudaSetDevice(b->dev));
    for (int s = 0; s < b->n_sub; ++s) {
        corr* h = b->h[s];
        if (h->xmode != b->xmode) return bfail(CORR_E_STATE, "a sub-array's mode changed after corr_batch_create");
        if (tc_mode(h->xmode) && !h->scales_set) return bfail(CORR_E_STATE, "a sub-array has no requantisation scales");
        if (!x[s] || (reinterpret_cast<uintptr_t>(x[s]) & 15) || (ld[s] & 15) || ld[s] < n_avail[s])
            return bfail(CORR_E_INVAL, "sample rows must be 16-byte aligned with ld >= n_avail");
        int dmax = 0;
        for (double t : h->tau) dmax = std::max(dmax, static_cast<int>(std::floor(t + 0.5)));
        if (n_avail[s] < static_cast<int64_t>(h->n_int) * h->n_fft + dmax)
            return bfail(CORR_E_RANGE, "a sub-array's n_avail is shorter than n_int * n_fft + its largest delay");
    }
    // the previous launch must have read the pinned tables before they are rewritten
    if (b->pending) BCU(cudaEventSynchronize(b->done));
    for (int s = 0; s < b->n_sub; ++s) {
        corr* h = b->h[s];
        b->fe_p[s] = fe_params(h, x[s], ld[s], n_avail[s]);
        b->h_g0[s] = g0 ? g0[s] : 0;
        const int nd = h->n_ant;
        std::memcpy(h->h_model, h->tau.data(), nd * sizeof(double));
        std::memcpy(h->h_model + nd, h->phi0.data(), nd * sizeof(double));
        std::memcpy(h->h_model + 2 * nd, h->rate.data(), nd * sizeof(double));
        if (tc_mode(b->xmode) && !fill_xt(b, s, b->h_xt + s, b->d_items[s], b->n_items[s]))
            return bfail(CORR_E_CUDA, "the driver refused the tensor map of a sub-array's spectra");
    }
    bool recapture = !b->exec;
    for (int q = 0; q < b->n_sub; ++q)
        if (fengine_clustered(b->h[q]->n_chan, b->fmode[q]) && std::memcmp(&b->fe_p[q], &b->cap_p[q], sizeof(FeParams)))
            recapture = true;
    if (recapture)
        if (int rc = capture(b)) return rc;
    for (int q = 0; q < b->n_sub; ++q) {   // this integration's sample pointers into the F-engine nodes
        if (fengine_clustered(b->h[q]->n_chan, b->fmode[q])) continue;
        cudaKernelNodeParams kp = b->fe_kp[q];
        void* args[1] = {&b->fe_p[q]};
        kp.kernelParams = args;
        kp.extra = nullptr;
        BCU(cudaGraphExecKernelNodeSetParams(b->exec, b->fe_node[q], &kp));
    }
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->cap;
    for (int q = 0; q < b->n_sub; ++q) {   // back from the channel-quad layout: padding rows read as zero
        corr* h = b->h[q];
        if (b->fmode[q] == OUT_FP32 && h->last_quad)
            BCU(cudaMemsetAsync(h->d_spec, 0,
                                static_cast<size_t>(h->n_chan) * h->n_int * rows_fp32(h->n_in) * sizeof(float), s));
    }
    BCU(cudaGraphLaunch(b->exec, s));
    BCU(cudaEventRecord(b->done, s));
    b->pending = true;
    for (int q = 0; q < b->n_sub; ++q) {
        corr* h = b->h[q];
        BCU(cudaEventRecord(h->ev_done, s));
        h->launched += 1;
        h->last_mode = h->xmode;
        h->last_quad = false;
    }
    return CORR_OK;
}

int corr_batch_tune(corr_batch_t* b, int* ks_out, float* ms_out) {
    if (!b) return bfail(CORR_E_INVAL, "null batch");
    if (!tc_mode(b->xmode)) return bfail(CORR_E_STATE, "the stage size applies to the tensor-core modes");
    if (!b->pending) return bfail(CORR_E_STATE, "run one batch integration first: tuning times its spectra");
    BCU(cudaSetDevice(b->dev));
    BCU(cudaEventSynchronize(b->done));
    XtBatch* d_tmp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CORR_OK;
    if (cudaMalloc(&d_tmp, sizeof(XtBatch)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = bfail(CORR_E_NOMEM, "tuning buffers");
    for (int s = 0; rc == CORR_OK && s < b->n_sub; ++s) {
        corr* h = b->h[s];
        int best = 0;
        float best_ms = 0.0f;
        for (int ks = 32; rc == CORR_OK && ks <= xengine_tc_max_ks(h->n_in); ks *= 2) {
            XtBatch t;
            if (!fill_xt(b, s, &t, b->d_items[s], b->n_items[s])) {
                rc = bfail(CORR_E_CUDA, "the driver refused the tensor map of a sub-array's spectra");
                break;
            }
            t.sub[0].ks = ks;
            if (t.sub[0].in8 && !xengine_tc_encode_quad(t.sub[0])) {   // the map's box follows ks
                rc = bfail(CORR_E_CUDA, "the driver refused the tensor map of a sub-array's spectra");
                break;
            }
            float ms = 0.0f;
            bool ok = cudaMemcpy(d_tmp, &t, sizeof t, cudaMemcpyHostToDevice) == cudaSuccess &&
                      launch_xengine_tc_table(d_tmp, t.n_items, b->n_sm, b->cap, xt_form(b, s)) == cudaSuccess &&
                      cudaEventRecord(e0, b->cap) == cudaSuccess;
            for (int r = 0; ok && r < 3; ++r)
                ok = launch_xengine_tc_table(d_tmp, t.n_items, b->n_sm, b->cap, xt_form(b, s)) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, b->cap) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (!ok) {
                rc = bfail(CORR_E_CUDA, "tuning launch failed");
                break;
            }
            ms /= 3.0f;
            if (best == 0 || ms < best_ms) {
                best = ks;
                best_ms = ms;
            }
        }
        if (rc == CORR_OK) {
            rc = corr_set_xengine_stage(h, best);
            if (ks_out) ks_out[s] = best;
            if (ms_out) ms_out[s] = best_ms;
        }
    }
    if (d_tmp) cudaFree(d_tmp);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
