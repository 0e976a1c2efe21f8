// fengine_blank.cu -- the F-engine with the time-domain voltage blanker (Sec. 5, Eq. 3-4)
// compiled in: a translation unit of its own, so that the plain kernels keep their register
// allocation and both halves build in parallel.
#include "fengine_impl.cuh"

namespace gbx {

cudaError_t launch_fengine_blank(const FeParams& p, int mode, cudaStream_t s) {
    if (p.n_chan * 2 != p.n_fft || !p.blank || (1 << p.blank_log2) < p.n_fft) return cudaErrorInvalidValue;
    switch (mode) {
        case OUT_FP32: return launch_mode<OUT_FP32, true>(p, s);
        case OUT_I8: return launch_mode<OUT_I8, true>(p, s);
        case OUT_F16: return launch_mode<OUT_F16, true>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbx
