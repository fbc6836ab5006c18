// S4-S5 transform lengths G = 5 2^a (image sizes 160 ... 10240): the kernels
// of fft_kernels.cuh with a final radix-5 Stockham pass.
#include "fft_kernels.cuh"

namespace toi {

cudaError_t fft_configure_r5(int G) {
  switch (G) {
    case 320: return configure_g<320>();
    case 640: return configure_g<640>();
    case 1280: return configure_g<1280>();
    case 2560: return configure_g<2560>();
    case 5120: return configure_g<5120>();
    case 10240: return configure_g<10240>();
    case 20480: return configure_g<20480>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fft_run_r5(toi_plan_s* p, FftOp op, Slot* s, float* out) {
  switch (p->G) {
    case 320: return run_g<320>(p, op, s, out);
    case 640: return run_g<640>(p, op, s, out);
    case 1280: return run_g<1280>(p, op, s, out);
    case 2560: return run_g<2560>(p, op, s, out);
    case 5120: return run_g<5120>(p, op, s, out);
    case 10240: return run_g<10240>(p, op, s, out);
    case 20480: return run_g<20480>(p, op, s, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace toi
