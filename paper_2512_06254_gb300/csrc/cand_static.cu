// tlisi_candidates_noalloc: the candidate search of tlisi_candidates with its
// scratch in a fixed device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory when they run the candidate
// search: a real-time pipeline that must never stall (cudaMalloc may
// synchronise the whole device), an application whose device memory is
// entirely owned by its own allocator, or code that runs where allocation is
// not allowed.  This entry point needs no allocation at all: it works in a
// file-scope __device__ array of kStaticScratchBytes that every GPU loading
// this library holds until the process exits.
//
// Host code cannot hand the array's name to a kernel (on the host it names a
// stand-in object, not device memory), so every call looks the device address
// up with cudaGetSymbolAddress for the calling thread's current device.  The
// lookup is cheap, and it is never stale: a cached address would outlive a
// cudaDeviceReset or a primary-context teardown, after which the module (and
// the array) is loaded again at a new address.
#include <string>

#include "toi_internal.cuh"

namespace toi {
size_t candidates_scratch_bytes(int S, int nt);
cudaError_t candidates_run(const float* cube, int S, int nty, int ntx, int T, int mode,
                           cudaStream_t st, void* scratch, double* scores_out, int max_boxes,
                           int* boxes_dev, double** thr_dev, int** nbox_dev, double* xbuf);
void set_planless_error(const std::string& msg);
}  // namespace toi

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB

__device__ __align__(256) unsigned char g_cand_scratch[kStaticScratchBytes];

toi_status nofail(toi_status s, const std::string& msg) {
  toi::set_planless_error(msg);
  return s;
}

}  // namespace

extern "C" toi_status tlisi_candidates_noalloc(const float* cube, int32_t S, int32_t nty,
                                               int32_t ntx, int32_t tile, int32_t mode,
                                               void* stream, double* threshold, int32_t* boxes,
                                               int32_t* nboxes, int32_t max_boxes,
                                               double* scores) {
  if (!cube || !threshold || !nboxes)
    return nofail(TOI_ERR_ARG, "cube, threshold and nboxes must be non-NULL");
  if (S < 1 || nty < 1 || ntx < 1 || tile < 1)
    return nofail(TOI_ERR_ARG, "S, nty, ntx, tile must be >= 1");
  if ((long long)nty * ntx > toi::kMaxCandTiles)
    return nofail(TOI_ERR_ARG, "more than 131072 tiles (the labelling runs in one block)");
  if (mode != TOI_CAND_PERIODIC && mode != TOI_CAND_NONPERIODIC)
    return nofail(TOI_ERR_ARG, "unknown mode");
  if (max_boxes < 0 || (max_boxes > 0 && !boxes))
    return nofail(TOI_ERR_ARG, "boxes must hold max_boxes entries");
  const int nt = nty * ntx;
  const size_t work = toi::candidates_scratch_bytes(S, nt);
  const size_t need = work + sizeof(int) * 4 * ((size_t)max_boxes + 1);
  if (need > kStaticScratchBytes)
    return nofail(TOI_ERR_ARG, "tlisi_candidates_noalloc: this cube needs " + std::to_string(need) +
                                   " bytes of scratch, more than its fixed " +
                                   std::to_string(kStaticScratchBytes) +
                                   " bytes; use tlisi_candidates for larger cubes");
  // the array's address on the current device (see the file comment)
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_cand_scratch);
  if (e != cudaSuccess || !base)
    return nofail(TOI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // Every kernel of the search writes each scratch word before reading it,
  // so the array's previous contents (it keeps those of the last call) need
  // no clearing.
  cudaStream_t st = (cudaStream_t)stream;
  int* boxes_dev = reinterpret_cast<int*>(reinterpret_cast<char*>(base) + work);
  double* thr_dev = nullptr;
  int* nbox_dev = nullptr;
  // no room for a folded copy of the series here: the search centres and
  // folds it per frequency instead (the same bits)
  e = toi::candidates_run(cube, S, nty, ntx, tile, mode, st, base, scores, max_boxes, boxes_dev,
                          &thr_dev, &nbox_dev, nullptr);
  int nb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(threshold, thr_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, nbox_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && max_boxes > 0 && nb > 0) {
    const int ncopy = nb < max_boxes ? nb : max_boxes;
    e = cudaMemcpyAsync(boxes, boxes_dev, sizeof(int) * 4 * (size_t)ncopy, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess)
    return nofail(TOI_ERR_CUDA, std::string("tlisi_candidates_noalloc: ") + cudaGetErrorString(e));
  *nboxes = nb;
  return TOI_OK;
}
