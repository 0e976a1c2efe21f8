// batch.cu -- several sub-arrays of uneven sizes in one graph-captured launch, and
// the autotuner that picks the tensor-core X-engine's stage size per sub-array.
//
// The graph holds, per sub-array, the upload of its delay model and its phasor
// set-up, then ONE F-engine launch whose CTAs cover the frame blocks of every
// sub-array (each CTA dispatches on its sub-array's FFT size) and ONE persistent
// tensor-core X-engine launch whose CTAs walk a cost-ordered list of (sub-array,
// channel, row block) items of all of them.  The per-launch parameters live in
// device tables that memcpy nodes of the same graph refresh from pinned host
// copies, so the graph is captured once and replayed for every integration.
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
    int xmode = 0, n_sm = 0, dev = 0;
    cudaStream_t cap = nullptr;
    FeBatch* h_fe = nullptr;     // pinned
    FeBatch* d_fe = nullptr;
    XtBatch* h_xt = nullptr;     // pinned
    XtBatch* d_xt = nullptr;
    int4* d_items = nullptr;
    int n_items = 0;
    int fe_blocks = 0;
    size_t fe_smem = 0;
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

// (sub, channel, row block) items ordered by decreasing cost: wide sub-arrays first.
std::vector<int4> make_items(const corr_batch* b, int only_sub) {
    std::vector<int4> items;
    for (int s = 0; s < b->n_sub; ++s) {
        if (only_sub >= 0 && s != only_sub) continue;
        const int R = 2 * b->h[s]->n_in, rbs = R > 128 ? 2 : 1;
        for (int k = 0; k < b->h[s]->n_chan; ++k)
            for (int r = 0; r < rbs; ++r) items.push_back(make_int4(s, k, r, 0));
    }
    auto cost = [&](const int4& e) {
        const corr* h = b->h[e.x];
        return static_cast<double>(h->n_int) * std::min(2 * h->n_in, 256);
    };
    std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& c) { return cost(a) > cost(c); });
    return items;
}

void fill_xt(corr_batch* b, XtBatch* t, const int4* items, int n_items) {
    std::memset(t, 0, sizeof *t);
    t->n_sub = b->n_sub;
    for (int s = 0; s < b->n_sub; ++s) {
        t->sub[s] = xt_sub_of(b->h[s]);
        t->sub[s].in8 = 0;   // the batched F-engine writes int8 values in the fp16 layout
    }
    t->n_items = n_items;
    t->items = items;
    t->err = b->h[0]->d_err;
}

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

// Capture the integration of every sub-array into one graph on the batch's stream.
int capture(corr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t s = b->cap;
    BCU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    bool ok = cudaMemcpyAsync(b->d_fe, b->h_fe, sizeof(FeBatch), cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (ok && tc_mode(b->xmode))
        ok = cudaMemcpyAsync(b->d_xt, b->h_xt, sizeof(XtBatch), cudaMemcpyHostToDevice, s) == cudaSuccess;
    for (int q = 0; ok && q < b->n_sub; ++q) {
        corr* h = b->h[q];
        const int nd = h->n_ant;
        ok = cudaMemcpyAsync(h->d_model, h->h_model, 3 * nd * sizeof(double), cudaMemcpyHostToDevice, s) ==
                 cudaSuccess &&
             launch_phasor_setup(h->n_ant, h->n_chan, h->n_fft, h->n_int, 0, h->d_model, h->d_model + nd,
                                 h->d_model + 2 * nd, h->d_pf, h->d_ff, h->d_D, s, &b->d_fe->g0[q]) == cudaSuccess;
    }
    const int fmode = b->xmode == CORR_FP32 ? OUT_FP32 : (b->xmode == CORR_I8 ? OUT_I8 : OUT_F16);
    if (ok) ok = launch_fengine_batched(b->d_fe, b->fe_blocks, b->fe_smem, fmode, s) == cudaSuccess;
    if (ok && tc_mode(b->xmode)) {
        ok = launch_xengine_tc_table(b->d_xt, b->n_items, b->n_sm, s) == cudaSuccess;
    } else {
        for (int q = 0; ok && q < b->n_sub; ++q) {
            corr* h = b->h[q];
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
    }
    for (int q = 0; ok && q < b->n_sub; ++q) {
        corr* h = b->h[q];
        if (h->dump > 0 && b->xmode == CORR_FP32)
            ok = launch_power_dumps(static_cast<const float*>(h->d_spec), h->n_in, h->n_chan, h->n_int, h->dump,
                                    h->d_power, s) == cudaSuccess;
        if (ok && h->beam_avg > 1)
            ok = launch_beam_average(h->d_beams_raw, h->d_beams, h->n_int, h->n_chan, h->beam_avg, s) == cudaSuccess;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (!ok || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(CORR_E_CUDA, "capturing the batch graph failed");
    }
    b->graph = g;
    BCU(cudaGraphInstantiate(&b->exec, g, 0));
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
        cudaMallocHost(reinterpret_cast<void**>(&b->h_fe), sizeof(FeBatch)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_xt), sizeof(XtBatch)) != cudaSuccess ||
        cudaMalloc(&b->d_fe, sizeof(FeBatch)) != cudaSuccess || cudaMalloc(&b->d_xt, sizeof(XtBatch)) != cudaSuccess)
        return bail("batch tables");
    std::memset(b->h_fe, 0, sizeof(FeBatch));
    b->fe_blocks = 0;
    for (int s = 0; s < n_sub; ++s) {
        b->h_fe->first[s] = b->fe_blocks;
        b->fe_blocks += (fengine_blocks(subs[s]->n_fft, subs[s]->n_int) + 1) & ~1;   // even: cluster pairs
        b->fe_smem = std::max(b->fe_smem, fengine_smem_bytes(subs[s]->n_fft));
    }
    b->h_fe->first[n_sub] = b->fe_blocks;
    b->h_fe->n_sub = n_sub;
    if (tc_mode(b->xmode)) {
        const std::vector<int4> items = make_items(b, -1);
        b->n_items = static_cast<int>(items.size());
        if (cudaMalloc(&b->d_items, sizeof(int4) * items.size()) != cudaSuccess ||
            cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail("batch items");
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
    if (b->d_fe) cudaFree(b->d_fe);
    if (b->d_xt) cudaFree(b->d_xt);
    if (b->d_items) cudaFree(b->d_items);
    if (b->h_fe) cudaFreeHost(b->h_fe);
    if (b->h_xt) cudaFreeHost(b->h_xt);
    if (b->done) cudaEventDestroy(b->done);
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
        b->h_fe->p[s] = fe_params(h, x[s], ld[s], n_avail[s]);
        b->h_fe->g0[s] = g0 ? g0[s] : 0;
        const int nd = h->n_ant;
        std::memcpy(h->h_model, h->tau.data(), nd * sizeof(double));
        std::memcpy(h->h_model + nd, h->phi0.data(), nd * sizeof(double));
        std::memcpy(h->h_model + 2 * nd, h->rate.data(), nd * sizeof(double));
    }
    if (tc_mode(b->xmode)) fill_xt(b, b->h_xt, b->d_items, b->n_items);
    if (!b->exec)
        if (int rc = capture(b)) return rc;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->cap;
    BCU(cudaGraphLaunch(b->exec, s));
    BCU(cudaEventRecord(b->done, s));
    b->pending = true;
    for (int q = 0; q < b->n_sub; ++q) {
        corr* h = b->h[q];
        BCU(cudaEventRecord(h->ev_done, s));
        h->launched += 1;
        h->last_mode = h->xmode;
        h->last_quad = false;   // the batched F-engine writes the plain K-block layouts
        h->last_i8b = false;
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
    int4* d_it = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CORR_OK;
    if (cudaMalloc(&d_tmp, sizeof(XtBatch)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = bfail(CORR_E_NOMEM, "tuning buffers");
    for (int s = 0; rc == CORR_OK && s < b->n_sub; ++s) {
        corr* h = b->h[s];
        const std::vector<int4> items = make_items(b, s);
        if (d_it) cudaFree(d_it);
        d_it = nullptr;
        if (cudaMalloc(&d_it, sizeof(int4) * items.size()) != cudaSuccess ||
            cudaMemcpy(d_it, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = bfail(CORR_E_NOMEM, "tuning items");
            break;
        }
        int best = 0;
        float best_ms = 0.0f;
        for (int ks = 32; rc == CORR_OK && ks <= xengine_tc_max_ks(h->n_in); ks *= 2) {
            XtBatch t;
            fill_xt(b, &t, d_it, static_cast<int>(items.size()));
            t.sub[s].ks = ks;
            float ms = 0.0f;
            bool ok = cudaMemcpy(d_tmp, &t, sizeof t, cudaMemcpyHostToDevice) == cudaSuccess &&
                      launch_xengine_tc_table(d_tmp, t.n_items, b->n_sm, b->cap) == cudaSuccess &&
                      cudaEventRecord(e0, b->cap) == cudaSuccess;
            for (int r = 0; ok && r < 3; ++r) ok = launch_xengine_tc_table(d_tmp, t.n_items, b->n_sm, b->cap) == cudaSuccess;
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
    if (d_it) cudaFree(d_it);
    if (d_tmp) cudaFree(d_tmp);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
