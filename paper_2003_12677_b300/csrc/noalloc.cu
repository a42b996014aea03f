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
// Its address is looked up once per device with cudaGetSymbolAddress (host
// code cannot use the array's name as a device pointer) and passed to the
// existing SIRT kernels as their workspace.
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

// Device address of g_sirt_scratch on the current device (looked up once).
tomo_status scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tomo::fail(TOMO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return tomo::fail(TOMO_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sirt_scratch);
    if (e != cudaSuccess || !p)
      return tomo::fail(TOMO_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                           cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TOMO_OK;
}

struct CurrentDevice {
  int prev = -1;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
      cudaSetDevice(dev);
    else
      prev = -1;
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
  TOMO_TRY(scratch_address(&scratch));
  if (iters == 0) return TOMO_OK;
  // every scratch word SIRT reads (residual, interleaved copies with zero
  // padding) is written earlier in the same call, so stale contents left by
  // a previous call are never read
  return run_sirt(A, sino, x, n_z, iters, lambda, ex, scratch, (cudaStream_t)stream);
}
