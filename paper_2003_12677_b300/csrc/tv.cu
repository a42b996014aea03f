// tv.cu -- the TV prior of the model-based objective (Sec. 2.1): value and
// gradient in one pass.
//
//   TV_eps(x_s) = sum_{iy,ix} sqrt(Dx^2 + Dy^2 + eps^2),
//   Dx = x[iy][ix+1] - x[iy][ix] (0 on the last column),
//   Dy = x[iy+1][ix] - x[iy][ix] (0 on the last row),
//
// per slice s.  Pixel (iy, ix) enters its own term and those of its left and
// upper neighbours, so one thread forms its gradient from three terms, recomputing
// the neighbours' instead of storing them:
//   g = -(Dx + Dy)/t (own) + Dx(iy, ix-1)/t(iy, ix-1) + Dy(iy-1, ix)/t(iy-1, ix).
// The value is summed per block in FP64 over a fixed tiling and the tiles in a
// fixed order (deterministic).
#include "internal.cuh"

namespace tomo {
namespace {

constexpr int kTx = 32, kTy = 8;

struct TvTerm {
  float dx, dy, t;
};

// the term at (iy, ix), or a null term outside the image
__device__ __forceinline__ TvTerm tv_term(const float *u, int ny, int nx, int iy, int ix, float eps2) {
  TvTerm r{0.f, 0.f, 1.f};
  if (iy < 0 || ix < 0) return r;
  const int64_t j = (int64_t)iy * nx + ix;
  const float c = u[j];
  r.dx = ix + 1 < nx ? u[j + 1] - c : 0.f;
  r.dy = iy + 1 < ny ? u[j + nx] - c : 0.f;
  r.t = sqrtf(r.dx * r.dx + r.dy * r.dy + eps2);
  return r;
}

// grid (tiles_x, tiles_y, nz), block kTx x kTy
__global__ void __launch_bounds__(kTx *kTy) k_tv(const float *x, int ny, int nx, float eps2, float *g,
                                                 double *part) {
  const int ix = blockIdx.x * kTx + threadIdx.x, iy = blockIdx.y * kTy + threadIdx.y, s = blockIdx.z;
  const float *u = x + (int64_t)s * ny * nx;
  double val = 0.0;
  if (ix < nx && iy < ny) {
    const TvTerm o = tv_term(u, ny, nx, iy, ix, eps2);
    const TvTerm l = tv_term(u, ny, nx, iy, ix - 1, eps2);
    const TvTerm a = tv_term(u, ny, nx, iy - 1, ix, eps2);
    g[(int64_t)s * ny * nx + (int64_t)iy * nx + ix] = -(o.dx + o.dy) / o.t + l.dx / l.t + a.dy / a.t;
    val = o.t;
  }
  __shared__ double red[kTx * kTy];
  const int t = threadIdx.y * kTx + threadIdx.x;
  red[t] = val;
  __syncthreads();
  for (int o = kTx * kTy / 2; o; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) part[((int64_t)s * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

// loss[s] = the slice's tile sums in tile order; one warp per slice
__global__ void k_tv_sum(const double *part, int tiles, double *loss) {
  const int s = blockIdx.x, lane = threadIdx.x;
  double v = 0.0;
  for (int i = lane; i < tiles; i += 32) v += part[(int64_t)s * tiles + i];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) loss[s] = v;
}

}  // namespace

tomo_status tv_loss_grad(const float *x, int32_t nz, int32_t ny, int32_t nx, float eps, double *loss, float *grad,
                         cudaStream_t st) {
  const dim3 grid((nx + kTx - 1) / kTx, (ny + kTy - 1) / kTy, nz);
  const int tiles = (int)(grid.x * grid.y);
  double *part = nullptr;
  if (cudaMallocAsync((void **)&part, sizeof(double) * (size_t)tiles * nz, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(TOMO_ERR_OOM, "TV scratch allocation failed");
  }
  k_tv<<<grid, dim3(kTx, kTy), 0, st>>>(x, ny, nx, eps * eps, grad, part);
  k_tv_sum<<<nz, 32, 0, st>>>(part, tiles, loss);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) return fail(TOMO_ERR_CUDA, std::string("TV kernels: ") + cudaGetErrorString(e));
  return TOMO_OK;
}

}  // namespace tomo
