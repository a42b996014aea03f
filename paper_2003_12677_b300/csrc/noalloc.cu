// noalloc.cu -- SIRT for callers that must not allocate GPU memory.
//
// tomo_sirt needs scratch (the residual and, for batched widths, interleaved
// copies of the sinogram and tomogram) and either takes it from the caller or
// allocates it itself.  Some callers can do neither: a reconstruction loop
// embedded in a detector's acquisition software, for example, runs against a
// fixed memory budget and cannot afford cudaMalloc / cudaFree in its steady
// state, because those calls may synchronise the whole device (stalling the
// other streams that are moving frames) and may fail under memory pressure
// half-way through a scan.  tomo_sirt_noalloc serves them from one scratch
// array that is part of the library image itself: kScratchBytes of device
// memory, reserved on every GPU that loads the library and held until the
// process exits.
//
// Its address is looked up with cudaGetSymbolAddress on the calling device
// (host code cannot use the array's name as a device pointer) and passed to
// the existing SIRT kernels as their workspace.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sirt_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_sirt_scratch on the current device.  It is looked up
// again on every call made outside stream capture (a device reset or a new
// primary context may load the module at another address) and remembered for
// calls made while `stream` is being captured, which may not query it.
tomo_status scratch_address(cudaStream_t stream, void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tomo::fail(TOMO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return tomo::fail(TOMO_ERR_UNSUPPORTED, "device ordinal out of range");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess)
    return tomo::fail(TOMO_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sirt_scratch);
    if (e != cudaSuccess || !p)
      return tomo::fail(TOMO_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                           cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  } else if (!g_scratch_addr[dev]) {
    return tomo::fail(TOMO_ERR_UNSUPPORTED,
                      "the first tomo_sirt_noalloc call on a device must come before any stream capture");
  }
  *out = g_scratch_addr[dev];
  return TOMO_OK;
}

// Makes `dev` current for the duration of the call and restores the previous device.
struct CurrentDevice {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit CurrentDevice(int dev) {
    err = cudaGetDevice(&prev);
    if (err != cudaSuccess) {
      prev = -1;
    } else if (prev != dev) {
      err = cudaSetDevice(dev);
      if (err != cudaSuccess) prev = -1;
    } else {
      prev = -1;
    }
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" tomo_status tomo_sirt_noalloc(const tomo_matrix *A, const float *sino, float *x, int32_t n_z,
                                         int32_t iters, float lambda, void *stream) {
  using namespace tomo;
  if (!A || !sino || !x) return fail(TOMO_ERR_INVALID_ARG, "matrix, sino and x must be non-NULL");
  if (((uintptr_t)sino & 15u) || ((uintptr_t)x & 15u))
    return fail(TOMO_ERR_INVALID_ARG, "sino and x must be 16-byte aligned");
  if (n_z < 1 || iters < 0) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1 and iters >= 0");
  if (!std::isfinite(lambda))
    return fail(TOMO_ERR_INVALID_ARG, "lambda must be finite");
  if (!A->sA.ent) return fail(TOMO_ERR_UNSUPPORTED, "matrix was built without the FP32 SELL form");
  CurrentDevice cd(A->device);
  if (cd.err != cudaSuccess)
    return fail(TOMO_ERR_CUDA, std::string("selecting the matrix's device: ") + cudaGetErrorString(cd.err));
  // widest batch (at most 16, at most the slice count) whose scratch fits
  Exec ex;
  ex.graph = false;
  int b = 1;
  while (b < n_z && b < 16) b <<= 1;
  for (; b >= 1; b >>= 1) {
    ex.B = b;
    if (workspace_bytes(A, TOMO_OP_SIRT, n_z, ex) <= kScratchBytes) break;
  }
  if (b < 1) {
    ex.B = 1;
    return fail(TOMO_ERR_INVALID_ARG, "geometry needs " + std::to_string(workspace_bytes(A, TOMO_OP_SIRT, n_z, ex)) +
                                          " bytes of scratch; the static scratch of tomo_sirt_noalloc holds " +
                                          std::to_string(kScratchBytes) + " bytes");
  }
  void *scratch = nullptr;
  TOMO_TRY(scratch_address((cudaStream_t)stream, &scratch));
  // never NULL here: run_sirt would otherwise allocate a workspace itself
  if (!scratch) return fail(TOMO_ERR_CUDA, "static scratch has no device address");
  if (iters == 0) return TOMO_OK;
  // every scratch word SIRT reads (residual, interleaved copies with zero
  // padding) is written earlier in the same call, so stale contents left by
  // a previous call are never read
  return run_sirt(A, sino, x, n_z, iters, lambda, ex, scratch, (cudaStream_t)stream);
}
