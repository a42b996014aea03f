// bbstep.cuh -- the Barzilai-Borwein step of the paper's SIRT (Sec. 3.1) as
// used on the Fubini-Radon operator (fubini.cu) and on its normal operator
// (normal.cu): per-slice sums over a fixed split, reduced in a fixed order
// (deterministic), the BB1 rule, the update.  Internal linkage: each
// translation unit that includes it gets its own kernels.
#pragma once

#include <cstdint>

namespace tomo {
namespace {

// compensated FP32 sum of a thread's own terms (Kahan): its error stays
// near one FP32 rounding of the sum of magnitudes whatever the term count;
// the threads' sums are then combined in FP64
struct KSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// BB1 step of one slice from its sums (P = <gp,gp>, Q = <gp, g - gp>) and the
// state (alpha, frozen, stepped): alpha = 1 on the first step, frozen slices 0
__device__ __forceinline__ double bb_rule(double P, double Q, const double *in, double *frozen, double *stepped) {
  const double ap = in[0];
  *frozen = in[1];
  *stepped = in[2];
  if (*frozen != 0.0) return 0.0;
  if (*stepped == 0.0) {
    *stepped = 1.0;
    return 1.0;
  }
  const double ss = ap * ap * P, sy = -ap * Q;
  if (ss > 0.0 && sy > 0.0) return ss / sy;
  *frozen = 1.0;
  return 0.0;
}

// one warp per slice: the NB partial sums in a fixed order, the BB step, the
// state and ||g|| recorded, alpha[s] for the next pass
__global__ void k_bb_alpha(const double3 *part, int NB, const double *sc_in, double *sc_out, double *hist, int k,
                            int nz, float *alpha) {
  const int s = blockIdx.x, lane = threadIdx.x;
  double gg = 0.0, P = 0.0, Q = 0.0;
  for (int i = lane; i < NB; i += 32) {
    const double3 v = part[(int64_t)s * NB + i];
    gg += v.x;
    P += v.y;
    Q += v.z;
  }
  for (int o = 16; o; o >>= 1) {
    gg += __shfl_xor_sync(0xffffffffu, gg, o);
    P += __shfl_xor_sync(0xffffffffu, P, o);
    Q += __shfl_xor_sync(0xffffffffu, Q, o);
  }
  if (lane == 0) {
    double frozen, stepped;
    const double a = bb_rule(P, Q, sc_in + s * 4, &frozen, &stepped);
    sc_out[s * 4 + 0] = a;
    sc_out[s * 4 + 1] = frozen;
    sc_out[s * 4 + 2] = stepped;
    if (hist) hist[(int64_t)k * nz + s] = sqrt(gg);
    alpha[s] = (float)a;
  }
}

// x += alpha[s] g; grid (blocks over a slice, nz)
__global__ void k_bb_axpy(float *x, const float *g, const float *alpha, int64_t cols) {
  const float a = alpha[blockIdx.y];
  const int64_t off = (int64_t)blockIdx.y * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cols; i += (int64_t)gridDim.x * blockDim.x)
    x[off + i] = fmaf(a, g[off + i], x[off + i]);
}

// part[s NB + b].x = sum of y^2 over block b's share of slice s after
// y = b - y (the residual r = b - R x and its squared norm); grid (NB, nz)
__global__ void k_bb_resid(const float *b, float *y, int64_t rows, int NB, double3 *part) {
  const int64_t per = (rows + NB - 1) / NB, lo = blockIdx.x * per, hi = lo + per < rows ? lo + per : rows;
  const int64_t off = (int64_t)blockIdx.y * rows;
  KSum sr;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float r = b[off + i] - y[off + i];
    y[off + i] = r;
    sr.add(r * r);
  }
  __shared__ double red[256];
  red[threadIdx.x] = sr.value();
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * NB + blockIdx.x].x = red[0];
}

// part[s NB + b].y, .z = <gp,gp>, <gp, g - gp> over block b's share of slice
// s (0 when gp is null: no previous gradient); grid (NB, nz), 256 threads
__global__ void k_bb_dots(const float *g, const float *gp, int64_t cols, int NB, double3 *part) {
  const int64_t per = (cols + NB - 1) / NB, lo = blockIdx.x * per, hi = lo + per < cols ? lo + per : cols;
  const int64_t off = (int64_t)blockIdx.y * cols;
  KSum sp, sq;
  if (gp) {
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const float a = gp[off + i];
      sp.add(a * a);
      sq.add(a * g[off + i]);
    }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sp.value();
  red[1][threadIdx.x] = sq.value();
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double3 &q = part[(int64_t)blockIdx.y * NB + blockIdx.x];
    q.y = red[0][0];
    q.z = red[1][0] - red[0][0];
  }
}

}  // namespace
}  // namespace tomo
