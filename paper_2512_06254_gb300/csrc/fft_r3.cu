// S4-S5 transform lengths G = 3 2^a (image sizes 96 ... 6144): the kernels of
// fft_kernels.cuh with a final radix-3 Stockham pass.
#include "fft_kernels.cuh"

namespace toi {

cudaError_t fft_configure_r3(int G) {
  switch (G) {
    case 192: return configure_g<192>();
    case 384: return configure_g<384>();
    case 768: return configure_g<768>();
    case 1536: return configure_g<1536>();
    case 3072: return configure_g<3072>();
    case 6144: return configure_g<6144>();
    case 12288: return configure_g<12288>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fft_run_r3(toi_plan_s* p, FftOp op, Slot* s, float* out) {
  switch (p->G) {
    case 192: return run_g<192>(p, op, s, out);
    case 384: return run_g<384>(p, op, s, out);
    case 768: return run_g<768>(p, op, s, out);
    case 1536: return run_g<1536>(p, op, s, out);
    case 3072: return run_g<3072>(p, op, s, out);
    case 6144: return run_g<6144>(p, op, s, out);
    case 12288: return run_g<12288>(p, op, s, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace toi
