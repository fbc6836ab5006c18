// S4-S5 transform lengths G = 2^a (image sizes 64 ... 8192) and the
// plan-facing FFT entry points, which dispatch on G to the translation unit
// of its length family (2^a here, 3 2^a in fft_r3.cu, 5 2^a in fft_r5.cu).
// The kernels themselves are in fft_kernels.cuh.
#include "fft_kernels.cuh"

namespace toi {

cudaError_t fft_configure_pow2(int G) {
  switch (G) {
    case 128: return configure_g<128>();
    case 256: return configure_g<256>();
    case 512: return configure_g<512>();
    case 1024: return configure_g<1024>();
    case 2048: return configure_g<2048>();
    case 4096: return configure_g<4096>();
    case 8192: return configure_g<8192>();
    case 16384: return configure_g<16384>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fft_run_pow2(toi_plan_s* p, FftOp op, Slot* s, float* out) {
  switch (p->G) {
    case 128: return run_g<128>(p, op, s, out);
    case 256: return run_g<256>(p, op, s, out);
    case 512: return run_g<512>(p, op, s, out);
    case 1024: return run_g<1024>(p, op, s, out);
    case 2048: return run_g<2048>(p, op, s, out);
    case 4096: return run_g<4096>(p, op, s, out);
    case 8192: return run_g<8192>(p, op, s, out);
    case 16384: return run_g<16384>(p, op, s, out);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

bool is_pow2_len(int G) { return G > 0 && (G & (G - 1)) == 0; }

cudaError_t run(toi_plan_s* p, FftOp op, Slot* s, float* out) {
  if (is_pow2_len(p->G)) return fft_run_pow2(p, op, s, out);
  if (p->G % 3 == 0) return fft_run_r3(p, op, s, out);
  return fft_run_r5(p, op, s, out);
}

}  // namespace

bool fft_length_supported(int G) {
  if (G < 128 || G % 8 != 0) return false;
  int m = G;
  while (m % 2 == 0) m /= 2;
  if (m == 1) return G <= 16384;
  if (m == 3) return G >= 192 && G <= 12288;
  if (m == 5) return G >= 320 && G <= 20480;
  return false;
}

cudaError_t fft_configure(int G) {
  if (is_pow2_len(G)) return fft_configure_pow2(G);
  if (G % 3 == 0) return fft_configure_r3(G);
  return fft_configure_r5(G);
}

cudaError_t launch_fft_to(toi_plan_s* p, Slot& s, float* out) { return run(p, FFT_FORWARD, &s, out); }

cudaError_t launch_fft(toi_plan_s* p, Slot& s) { return launch_fft_to(p, s, p->tilted); }

cudaError_t launch_fft_batch(toi_plan_s* p) { return run(p, FFT_BATCH, nullptr, nullptr); }

cudaError_t launch_fft_adjoint(toi_plan_s* p, Slot& s) { return run(p, FFT_ADJOINT, &s, nullptr); }

}  // namespace toi
