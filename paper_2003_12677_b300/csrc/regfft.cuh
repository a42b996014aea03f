// regfft.cuh -- complex FFTs of length L = R1 R2 (a power of two, up to 2048)
// on one group of R2 lanes of a warp, for the fused passes of the
// Fubini-Radon operator's normal operator (normal.cu) and adjoint (fubini.cu).
// The four-step decomposition: R1-point DFTs in registers over x[j1 R2 + j2],
// the twiddles W_L^{j2 k1}, a transpose through a shared tile, R2-point DFTs
// in registers; X[k1 + R1 k2] ends in lane k1 mod R2.  R1 = R2 or 2 R2.
// Internal linkage: each translation unit that includes it gets its own copy.
#pragma once

#include <cmath>
#include <cstdint>

namespace tomo {
namespace {

struct Tw64 {
  float2 w[64];  // e^{-2 pi i k / 64}
};

__host__ __device__ constexpr int rev8(int i) {
  return ((i & 1) << 7) | ((i & 2) << 5) | ((i & 4) << 3) | ((i & 8) << 1) | ((i & 16) >> 1) | ((i & 32) >> 3) |
         ((i & 64) >> 5) | ((i & 128) >> 7);
}

__host__ __device__ constexpr int ilog2(int R) { return R <= 1 ? 0 : 1 + ilog2(R / 2); }

// bit reversal of i < R (R a power of two <= 256), loop-free so that unrolled
// register indexing folds to constants
template <int R>
__host__ __device__ constexpr int bitrev(int i) {
  return rev8(i) >> (8 - ilog2(R));
}
static_assert(bitrev<32>(1) == 16 && bitrev<32>(6) == 12 && bitrev<8>(3) == 6, "bit reversal");

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// in-register DFT of R <= 64 points, natural order in and out: radix-2
// decimation in time on the bit-reversed sequence, one template level per
// stage so that every loop unrolls; kInv: conjugate twiddles
template <int R, int LEN, bool kInv>
__device__ __forceinline__ void dft_stage(float2 *a, const Tw64 &tw) {
#pragma unroll
  for (int i = 0; i < R; i += LEN) {
#pragma unroll
    for (int j = 0; j < LEN / 2; ++j) {
      const float2 u = a[i + j];
      float2 t = a[i + j + LEN / 2];
      // the twiddle e^{-+2 pi i idx / 64}: multiplications by -+i are swaps,
      // the two diagonal ones take two multiplies, the rest a full product
      const int idx = j * (64 / LEN);
      if (idx == 16) {
        t = kInv ? make_float2(-t.y, t.x) : make_float2(t.y, -t.x);
      } else if (idx == 8 || idx == 24) {
        const float h = tw.w[8].x;  // cos(pi/4), as the table holds it
        const float p = h * (t.x + t.y), m = h * (t.x - t.y);
        if (idx == 8)
          t = kInv ? make_float2(m, p) : make_float2(p, -m);
        else
          t = kInv ? make_float2(-p, m) : make_float2(-m, -p);
      } else if (idx != 0) {
        float2 w = tw.w[idx];
        if (kInv) w.y = -w.y;
        t = cmulf(w, t);
      }
      a[i + j] = make_float2(u.x + t.x, u.y + t.y);
      a[i + j + LEN / 2] = make_float2(u.x - t.x, u.y - t.y);
    }
  }
  if constexpr (LEN < R) dft_stage<R, 2 * LEN, kInv>(a, tw);
}

template <int R, bool kInv>
__device__ __forceinline__ void dft_reg(float2 *v, const Tw64 &tw) {
  float2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) a[bitrev<R>(i)] = v[i];
  dft_stage<R, 2, kInv>(a, tw);
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}

// forward (kInv: the unnormalised inverse DFT, conjugate twiddles): lane l
// holds v[j1] = x[j1 R2 + l]; on return w[t R2 + k2] = X[(l + G t) + R1 k2].
// S: the group's R1 x (R2 + 1) shared tile.  twL holds
// W_L^{j2 k1} twice: [k1][j2] (first L entries) and [j2][k1], so that the
// lanes of a group read consecutive entries in both directions.
template <int R1, int R2, bool kInv = false>
__device__ __forceinline__ void fft_fwd(float2 *v, float2 *w, float2 *S, int l, const float2 *twL, const Tw64 &tw) {
  constexpr int G = R2, T = R1 / G;
  dft_reg<R1, kInv>(v, tw);
#pragma unroll
  for (int k1 = 1; k1 < R1; ++k1) {
    float2 t1 = __ldg(twL + k1 * R2 + l);
    if (kInv) t1.y = -t1.y;
    v[k1] = cmulf(v[k1], t1);
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) S[k1 * (R2 + 1) + l] = v[k1];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int k1 = l + G * t;
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) w[t * R2 + j2] = S[k1 * (R2 + 1) + j2];
    dft_reg<R2, kInv>(w + t * R2, tw);
  }
  __syncwarp();
}

// inverse (unnormalised) of fft_fwd: from w back to v[j1] = x[j1 R2 + l]
template <int R1, int R2>
__device__ __forceinline__ void fft_inv(float2 *w, float2 *v, float2 *S, int l, const float2 *twL, const Tw64 &tw) {
  constexpr int G = R2, T = R1 / G;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int k1 = l + G * t;
    dft_reg<R2, true>(w + t * R2, tw);
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) {
      float2 tw1 = __ldg(twL + R1 * R2 + j2 * R1 + k1);
      tw1.y = -tw1.y;
      S[k1 * (R2 + 1) + j2] = cmulf(w[t * R2 + j2], tw1);
    }
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) v[k1] = S[k1 * (R2 + 1) + l];
  __syncwarp();
  dft_reg<R1, true>(v, tw);
}

// W_L^{j2 k1} = e^{-2 pi i (j2 k1 mod L) / L} for L = R1 R2, FP64 arguments
// rounded once: tw[k1 R2 + j2], then tw[L + j2 R1 + k1]
__global__ void k_fft_twiddles(int R1, int R2, float2 *tw) {
  const int L = R1 * R2;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * L) return;
  const int k1 = e < L ? e / R2 : (e - L) % R1, j2 = e < L ? e % R2 : (e - L) / R1;
  double s, c;
  sincospi(-2.0 * (double)(((int64_t)j2 * k1) % L) / (double)L, &s, &c);
  tw[e] = make_float2((float)c, (float)s);
}

inline Tw64 tw64() {
  Tw64 t;
  for (int k = 0; k < 64; ++k)
    t.w[k] = make_float2((float)std::cos(2.0 * M_PI * k / 64.0), (float)-std::sin(2.0 * M_PI * k / 64.0));
  return t;
}

// the split L = R1 R2 the passes use (R1 = R2 or 2 R2)
inline int fft_r2(int L) {
  int R2 = 1;
  while (R2 * R2 < L) R2 *= 2;
  if (R2 * R2 > L) R2 /= 2;
  return R2;
}

}  // namespace
}  // namespace tomo
