// status.cu -- the per-stream device status word.
//
// Kernels with bounded waits (the persistent CGLS launch) record why they
// stopped in a status word of their own workspace.  A call that returns
// without synchronising folds that word into one word per (device, stream)
// kept here; tomo_stream_status synchronises the stream, reads the word and
// resets it.  The first non-OK status wins (compare-and-swap from 0).
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace tomo {

namespace {

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, int *> g_words;

__global__ void k_fold_status(const int *src, int *dst) {
  const int s = *src;
  if (s != 0) atomicCAS(dst, 0, s);
}

}  // namespace

// The word of (current device, st), allocated and zeroed (in stream order) on
// first use; nullptr when the allocation fails.
int *stream_status_word(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, st);
  auto it = g_words.find(key);
  if (it != g_words.end()) return it->second;
  int *w = nullptr;
  if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) {
    cudaFree(w);
    return nullptr;
  }
  g_words[key] = w;
  return w;
}

tomo_status fold_status(const int *src, cudaStream_t st) {
  int *w = stream_status_word(st);
  if (!w) return fail(TOMO_ERR_OOM, "allocation of the stream status word failed");
  k_fold_status<<<1, 1, 0, st>>>(src, w);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status read_stream_status(cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return fail(TOMO_ERR_CUDA, std::string("stream synchronisation failed: ") + cudaGetErrorString(e));
  }
  int *w = nullptr;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(TOMO_ERR_CUDA, "no current device");
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_words.find(std::make_pair(dev, st));
    if (it == g_words.end()) return TOMO_OK;  // nothing was ever recorded on this stream
    w = it->second;
  }
  int v = 0;
  TOMO_CUDA(cudaMemcpyAsync(&v, w, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaMemsetAsync(w, 0, sizeof(int), st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  if (v != 0)
    return fail((tomo_status)v, "a launch queued on this stream stopped early: a bounded wait ran past its time limit");
  return TOMO_OK;
}

}  // namespace tomo

extern "C" tomo_status tomo_stream_status(void *stream) { return tomo::read_stream_status((cudaStream_t)stream); }
