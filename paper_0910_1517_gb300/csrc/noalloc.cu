// noalloc.cu -- corr_integrate_static: one FP32 integration with no allocation.
//
// Some callers cannot allocate device memory while they run: a real-time
// acquisition thread with a hard per-block deadline cannot afford cudaMalloc,
// which can synchronise the device and take driver locks for an unbounded
// time, and a process embedded in a larger pipeline often finds the whole
// device memory budget already reserved by its host framework.  For them this
// entry point runs the same F-engine and FP32 X-engine kernels as
// corr_integrate_device, but every intermediate buffer (integer delays,
// phasor and twiddle tables, beam weights, the F-to-X spectra hand-off and
// the error word) lives in one file-scope static device array of fixed size.
// The caller passes the samples and the output buffers; the delay model is
// passed by value in the kernel parameters, so no host-to-device copy and no
// host allocation is needed either.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/corr.h"
#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
void set_last_error(const char* msg);   // capi.cu: the message corr_last_error() returns
}

namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kStaticMaxAnt = 64;

// The scratch array.  In host code `g_scratch` names only a host-side stand-in;
// its device address comes from cudaGetSymbolAddress (once per device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

struct Model {
    double tau[kStaticMaxAnt];
    double phi0[kStaticMaxAnt];
    double rate[kStaticMaxAnt];
};

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

struct Layout {
    size_t err, D, ginc, pf, wcoh, ff, tw, spec, total;
};

Layout layout(int n_ant, int n_pol, int n_fft, int n_int) {
    const size_t nch = n_fft / 2;
    Layout L{};
    size_t o = 0;
    L.err = o;
    o = align256(o + sizeof(unsigned));
    L.D = o;
    o = align256(o + sizeof(int) * n_ant);
    L.ginc = o;
    o = align256(o + sizeof(float) * n_ant);
    L.pf = o;
    o = align256(o + sizeof(float2) * n_ant * nch);
    L.wcoh = o;
    o = align256(o + sizeof(float2) * n_ant * nch);
    L.ff = o;
    o = align256(o + sizeof(float2) * n_ant * static_cast<size_t>(n_int));
    L.tw = o;
    o = align256(o + sizeof(float2) * gbx::fengine_tw_count(n_fft));
    L.spec = o;
    o = align256(o + sizeof(float) * nch * static_cast<size_t>(n_int) * gbx::rows_fp32(n_ant * n_pol));
    L.total = o;
    return L;
}

// Fill the per-integration tables of the F-engine: integer delays, FSTC and fringe phasors
// (the delay-model helpers of fengine.cuh, as in the handle path) and unit beam weights over
// all antennas.  The twiddles come from launch_fengine_twiddles, as in the handle path.
__global__ void static_tables_kernel(Model m, int n_ant, int n_fft, int n_int, int64_t g0, unsigned char* base,
                                     Layout L) {
    const int M = n_fft / 2;
    int* D = reinterpret_cast<int*>(base + L.D);
    float* ginc = reinterpret_cast<float*>(base + L.ginc);
    float2* pf = reinterpret_cast<float2*>(base + L.pf);
    float2* wcoh = reinterpret_cast<float2*>(base + L.wcoh);
    float2* ff = reinterpret_cast<float2*>(base + L.ff);
    const int64_t n_pf = static_cast<int64_t>(n_ant) * M, n_ff = static_cast<int64_t>(n_ant) * n_int;
    const int64_t total = n_pf + n_ff + n_ant;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (q < n_pf) {
            const int a = static_cast<int>(q / M), k = static_cast<int>(q % M);
            pf[q] = gbx::model_fstc_phasor(m.tau[a], k, n_fft);
            wcoh[q] = make_float2(1.0f, 0.0f);
        } else if (q < n_pf + n_ff) {
            const int64_t r = q - n_pf;
            const int a = static_cast<int>(r / n_int), t = static_cast<int>(r % n_int);
            ff[r] = gbx::model_fringe_phasor(m.phi0[a], m.rate[a], g0 + t);
        } else {
            const int a = static_cast<int>(q - n_pf - n_ff);
            D[a] = gbx::model_int_delay(m.tau[a]);
            ginc[a] = 1.0f;
        }
    }
}

int fail(int code, const char* msg) {
    gbx::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int corr_integrate_static(int n_ant, int n_pol, int n_fft, int n_int, const int8_t* x, int64_t ld,
                                     int64_t n_avail, int64_t g0, const double* delay, const double* phi0,
                                     const double* rate, float* vis, float* beams, void* stream, int blocking) {
    if (n_ant < 1 || n_ant > kStaticMaxAnt || (n_pol != 1 && n_pol != 2))
        return fail(CORR_E_INVAL, "corr_integrate_static: need 1 <= n_ant <= 64 and n_pol in {1, 2}");
    if (n_fft < 64 || n_fft > 4096 || (n_fft & (n_fft - 1)) || n_int < 16 || n_int % 16)
        return fail(CORR_E_INVAL, "corr_integrate_static: n_fft a power of two in [64, 4096], n_int a multiple of 16");
    if (!x || !vis || !beams || !delay || (reinterpret_cast<uintptr_t>(x) & 15) || (ld & 15) || ld < n_avail)
        return fail(CORR_E_INVAL, "corr_integrate_static: null buffer, or x / ld not 16-byte aligned");
    const Layout L = layout(n_ant, n_pol, n_fft, n_int);
    if (L.total > kScratchBytes)
        return fail(CORR_E_RANGE, "corr_integrate_static: problem needs more than the 32 MiB static scratch");
    // the same delay-model checks as corr_set_delays, before any CUDA call: an integer delay
    // D = floor(tau + 1/2) must be a non-negative int no larger than 2e9 (the F-engine offsets
    // its sample reads by D), and the fringe model finite
    Model m{};
    int64_t dmax = 0;
    for (int a = 0; a < n_ant; ++a) {
        const double t = delay[a];
        if (!std::isfinite(t) || t < 0.0 || std::floor(t + 0.5) > 2.0e9)
            return fail(CORR_E_RANGE, "corr_integrate_static: delays must be finite, >= 0 and round to <= 2e9 samples");
        if ((phi0 && !std::isfinite(phi0[a])) || (rate && !std::isfinite(rate[a])))
            return fail(CORR_E_INVAL, "corr_integrate_static: fringe model is not finite");
        m.tau[a] = t;
        m.phi0[a] = phi0 ? phi0[a] : 0.0;
        m.rate[a] = rate ? rate[a] : 0.0;
        dmax = std::max(dmax, static_cast<int64_t>(std::floor(t + 0.5)));
    }
    if (n_avail < static_cast<int64_t>(n_int) * n_fft + dmax)
        return fail(CORR_E_RANGE, "corr_integrate_static: n_avail < n_int * n_fft + max delay");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(CORR_E_CUDA, "corr_integrate_static: no current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_dev[dev]) {   // once per device, with that device current
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr)
                return fail(CORR_E_CUDA, "corr_integrate_static: cudaGetSymbolAddress failed");
            g_scratch_dev[dev] = ptr;
        }
        scratch = g_scratch_dev[dev];
    }
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(CORR_E_CUDA, "corr_integrate_static: device query failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    const int64_t work = static_cast<int64_t>(n_ant) * (n_fft / 2 + n_int) + n_ant;
    static_tables_kernel<<<static_cast<int>(std::min<int64_t>((work + 255) / 256, 4096)), 256, 0, s>>>(
        m, n_ant, n_fft, n_int, g0, base, L);
    if (cudaGetLastError() != cudaSuccess ||
        gbx::launch_fengine_twiddles(n_fft, reinterpret_cast<float2*>(base + L.tw), s) != cudaSuccess)
        return fail(CORR_E_CUDA, "corr_integrate_static: table kernel");

    gbx::FeParams fp{};
    fp.x = x;
    fp.ld = ld;
    fp.n_avail = n_avail;
    fp.n_ant = n_ant;
    fp.n_pol = n_pol;
    fp.n_in = n_ant * n_pol;
    fp.n_fft = n_fft;
    fp.n_chan = n_fft / 2;
    fp.n_int = n_int;
    fp.D = reinterpret_cast<const int*>(base + L.D);
    fp.pf = reinterpret_cast<const float2*>(base + L.pf);
    fp.ff = reinterpret_cast<const float2*>(base + L.ff);
    fp.wcoh = reinterpret_cast<const float2*>(base + L.wcoh);
    fp.ginc = reinterpret_cast<const float*>(base + L.ginc);
    fp.scale = nullptr;
    fp.spec = base + L.spec;
    fp.beams = beams;
    fp.tw = reinterpret_cast<const float2*>(base + L.tw);
    fp.err = reinterpret_cast<unsigned*>(base + L.err);
    if (gbx::launch_fengine(fp, gbx::OUT_FP32, s) != cudaSuccess)
        return fail(CORR_E_CUDA, "corr_integrate_static: F-engine launch");
    gbx::XParams xp{};
    xp.spec = base + L.spec;
    xp.n_ant = n_ant;
    xp.n_pol = n_pol;
    xp.n_in = n_ant * n_pol;
    xp.n_chan = n_fft / 2;
    xp.n_int = n_int;
    xp.vis = reinterpret_cast<float2*>(vis);
    xp.err = fp.err;
    if (gbx::launch_xengine_fp32(xp, n_sm, s) != cudaSuccess)
        return fail(CORR_E_CUDA, "corr_integrate_static: X-engine launch");
    if (blocking) {
        // the error word is sticky: it collects the wait timeouts of this call and of every
        // non-blocking call since the last blocking one; read it, then clear it
        unsigned err = 0;
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(&err, base + L.err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemset(base + L.err, 0, sizeof err) != cudaSuccess)
            return fail(CORR_E_CUDA, "corr_integrate_static: synchronisation failed");
        if (err) return fail(CORR_E_TIMEOUT, "corr_integrate_static: a kernel wait timed out (this call or an earlier non-blocking one)");
    }
    return CORR_OK;
}
