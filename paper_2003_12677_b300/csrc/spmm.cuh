// spmm.cuh -- device building blocks shared by the SpMM kernels (ops.cu) and
// the persistent batched solver (persistent.cu): vector helpers, solver
// epilogues, deterministic block reductions and the SELL-32 row-group loops.
// Internal to libtomo.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "internal.cuh"

namespace tomo {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
template <int V>
struct Vec {
  float v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldg_vec(const float *p) {
  Vec<V> r;
  if constexpr (V == 4) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (V == 2) {
    float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = __ldg(p);
  }
  return r;
}

template <int V>
__device__ __forceinline__ Vec<V> ld_vec(const float *p) {
  Vec<V> r;
  if constexpr (V == 4) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (V == 2) {
    float2 t = *reinterpret_cast<const float2 *>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = *p;
  }
  return r;
}

template <int V>
__device__ __forceinline__ void st_vec(float *p, const Vec<V> &a) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(a.v[0], a.v[1]);
  } else {
    *p = a.v[0];
  }
}

// ---------------------------------------------------------------------------
// Epilogues.  Called once per (row, lane) with the lane's V accumulated slices
// starting at slice s0; `ss` collects per-slice squared norms when kNorm.
// ---------------------------------------------------------------------------
struct EpiStore {  // Y = acc
  static constexpr bool kNorm = false;
  float *Y;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    st_vec<V>(Y + row * ld + s0, a);
  }
};

struct EpiSirtResidual {  // r = R o (b - acc)
  static constexpr bool kNorm = false;
  float *r;
  const float *b, *R;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    float w = __ldg(R + row);
    Vec<V> bv = ldg_vec<V>(b + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) a.v[t] = w * (bv.v[t] - a.v[t]);
    st_vec<V>(r + row * ld + s0, a);
  }
};

// the same, times 1/a(theta) of the row's angle: the operand the 16-bit A^T
// pass gathers without a per-entry scale (separate type, so the FP32 kernels
// keep their register budget)
struct EpiSirtResidualScaled {
  static constexpr bool kNorm = false;
  float *r;
  const float *b, *R;
  int ld;
  const float *scale;  // per angle
  int np;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    const float w = __ldg(R + row) * __ldg(scale + row / np);
    Vec<V> bv = ldg_vec<V>(b + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) a.v[t] = w * (bv.v[t] - a.v[t]);
    st_vec<V>(r + row * ld + s0, a);
  }
};

struct EpiSirtUpdate {  // x += lambda C o acc
  static constexpr bool kNorm = false;
  float *x;
  const float *C;
  float lam;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    float w = lam * __ldg(C + row);
    Vec<V> xv = ld_vec<V>(x + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) xv.v[t] = fmaf(w, a.v[t], xv.v[t]);
    st_vec<V>(x + row * ld + s0, xv);
  }
};

struct EpiStoreNorm {  // Y = acc, ss += acc^2
  static constexpr bool kNorm = true;
  float *Y;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *ss) const {
    st_vec<V>(Y + row * ld + s0, a);
#pragma unroll
    for (int t = 0; t < V; ++t) ss[t] += (double)a.v[t] * (double)a.v[t];
  }
};

struct EpiResidual {  // r = b - acc
  static constexpr bool kNorm = false;
  float *r;
  const float *b;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    Vec<V> bv = ldg_vec<V>(b + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) a.v[t] = bv.v[t] - a.v[t];
    st_vec<V>(r + row * ld + s0, a);
  }
};

struct EpiResidualNorm {  // r = b - acc, ss += r^2
  static constexpr bool kNorm = true;
  float *r;
  const float *b;
  int ld;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *ss) const {
    Vec<V> bv = ldg_vec<V>(b + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      a.v[t] = bv.v[t] - a.v[t];
      ss[t] += (double)a.v[t] * (double)a.v[t];
    }
    st_vec<V>(r + row * ld + s0, a);
  }
};

// the same, also writing rs = r times 1/a(theta) of the row's angle (the
// operand of the 16-bit A^T pass)
struct EpiResidualNormScaled {
  static constexpr bool kNorm = true;
  float *r;
  const float *b;
  int ld;
  float *rs;
  const float *scale;
  int np;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *ss) const {
    Vec<V> bv = ldg_vec<V>(b + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      a.v[t] = bv.v[t] - a.v[t];
      ss[t] += (double)a.v[t] * (double)a.v[t];
    }
    st_vec<V>(r + row * ld + s0, a);
    const float sc = __ldg(scale + row / np);
#pragma unroll
    for (int t = 0; t < V; ++t) a.v[t] *= sc;
    st_vec<V>(rs + row * ld + s0, a);
  }
};

// Column bands of A (the image cut into bands of rows, each band stored as a
// matrix of its own): the pass over band b < last adds its sums into P (band 0
// stores them); the last band's pass adds P and hands the total to the real
// epilogue, which alone reduces norms.
struct EpiBandPartial {
  static constexpr bool kNorm = false;
  float *P;
  int ld;
  bool first;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *) const {
    if (!first) {
      const Vec<V> p = ld_vec<V>(P + row * ld + s0);
#pragma unroll
      for (int t = 0; t < V; ++t) a.v[t] += p.v[t];
    }
    st_vec<V>(P + row * ld + s0, a);
  }
};

template <class Epi>
struct EpiBandLast {
  static constexpr bool kNorm = Epi::kNorm;
  const float *P;
  int ld;
  Epi epi;
  template <int V>
  __device__ void operator()(int64_t row, int s0, Vec<V> &a, double *ss) const {
    const Vec<V> p = ld_vec<V>(P + row * ld + s0);
#pragma unroll
    for (int t = 0; t < V; ++t) a.v[t] += p.v[t];
    epi.template operator()<V>(row, s0, a, ss);
  }
};

// Deterministic per-block reduction of ss[V] (slices s0..s0+V-1 of each thread)
// into out[s], s < B.
// The reduction array doubles as the per-thread accumulators of the norm
// epilogues (norm_slots below): one 8 KB array per block, not two.
__device__ __forceinline__ double (*norm_red())[4] {
  __shared__ double red[kThreads][4];
  return red;
}

template <int V>
__device__ void block_norms_to(const double *ss, int s0, int B, double *out) {
  double(*red)[4] = norm_red();
  __shared__ int red_s0[kThreads];
#pragma unroll
  for (int t = 0; t < V; ++t) red[threadIdx.x][t] = ss[t];  // a no-op when ss is this thread's slot row
  red_s0[threadIdx.x] = s0;
  __syncthreads();
  for (int s = threadIdx.x; s < B; s += blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < kThreads; ++t) {
      int d = s - red_s0[t];
      if (d >= 0 && d < V) acc += red[t][d];
    }
    out[s] = acc;
  }
  __syncthreads();  // red[] may be reused by the caller's next reduction
}

// Per-thread FP64 accumulators of the norm epilogues.  They live in shared
// memory (each thread its own row of the reduction array, updated once per
// output row), so the SpMM row loop does not carry 2 V extra registers: with
// them in registers the norm variants needed 48-58 registers and lost one or
// two resident blocks per SM.  Epilogues without a norm get nullptr and never
// touch it.
template <int V, class Epi>
__device__ __forceinline__ double *norm_slots() {
  static_assert(V <= 4, "four slots per thread");
  if constexpr (Epi::kNorm) {
    double *p = norm_red()[threadIdx.x];
#pragma unroll
    for (int t = 0; t < V; ++t) p[t] = 0.0;
    return p;
  } else {
    return nullptr;
  }
}

// ... into part[blockIdx.x * B + s]
template <int V>
__device__ void block_norms(const double *ss, int s0, int B, double *part) {
  block_norms_to<V>(ss, s0, B, part + (int64_t)blockIdx.x * B);
}

// Order in which a pass visits its row groups.  IdentityMap: row order.
// TileMap (A^T, whose rows are pixels): the grid-stride schedule t is mapped
// so that the 8 warps of a block take 8 image rows x G pixels (a compact cell:
// rays through it hit few distinct bins, so their gathered residual rows are
// shared in L1) and consecutive blocks walk the image in tiles of 16 x 16
// cells (128 image rows x 16 G pixels: the residual rows that a tile's rays
// touch stay in L2 while the tile is in flight, instead of every angle's whole
// detector).  A bijection of [0, n_y n_x / G) when n_x % G == 0 and
// n_y % 8 == 0; gx = 0 selects row order.
struct IdentityMap {
  __device__ __forceinline__ int64_t operator()(int64_t t) const { return t; }
};

struct TileMap {
  int64_t gx;  // row groups per image row (n_x / G), 0 = row order
  int64_t cy;  // cell rows (n_y / 8)
  __device__ __forceinline__ int64_t operator()(int64_t t) const {
    if (gx == 0) return t;
    constexpr int64_t kTy = 16, kTx = 16;  // tile of kTy x kTx cells
    const int64_t w = t & 7, T = t >> 3;   // image row within the cell; cell in tiled order
    const int64_t band_cells = kTy * gx;
    const int64_t band = T / band_cells, r = T - band * band_cells;
    const int64_t ty = min(kTy, cy - band * kTy);
    const int64_t full = gx / kTx, tile_cells = ty * kTx;
    const int64_t ct = r / tile_cells;
    int64_t cyi, cxi;
    if (ct < full) {
      const int64_t u = r - ct * tile_cells;
      cyi = u / kTx;
      cxi = ct * kTx + u % kTx;
    } else {  // the narrower last tile of the band
      const int64_t tw = gx - full * kTx, u = r - full * tile_cells;
      cyi = u / tw;
      cxi = full * kTx + u % tw;
    }
    return ((band * kTy + cyi) * 8 + w) * gx + cxi;
  }
};

// Every SELL entry word is loaded exactly once per pass (one 128-bit load per
// pair or quad), so those loads carry the streaming (evict-first) hint and
// leave L2 to the gathered operand vector, which the whole pass reuses.  (The
// CSR kernels read each sector of indices with several loads and keep the
// default policy.)
// ---------------------------------------------------------------------------
// SELL-32 row groups (FP32 values).  V = min(B, 4) slices per lane, L = B/V
// lanes per row, G = 32/L rows per warp; the G rows of a warp are adjacent
// rows of one 32-row chunk, so each step loads one contiguous run of entry
// pairs (128-bit per lane) for all of them.  The calling warp handles row
// groups rg_begin, rg_begin + rg_step, ... below rg_end.
// ---------------------------------------------------------------------------
template <int V, bool kNC>
__device__ __forceinline__ Vec<V> gather(const float *p) {
  if constexpr (kNC)
    return ldg_vec<V>(p);
  else
    return ld_vec<V>(p);
}

template <int B>
struct Lanes {
  static constexpr int V = B >= 4 ? 4 : B;
  static constexpr int L = B / V;
  static constexpr int G = 32 / L;
};

// kNC: gather X through the read-only path (X unchanged during the launch);
// false for the persistent kernel, whose vectors change between phases.
template <int B, class Epi, bool kNC = true, class Map = IdentityMap>
__device__ __forceinline__ void sell_rowgroups(const int64_t *__restrict__ cp, const int32_t *__restrict__ rl,
                                               const int2 *__restrict__ ent, int64_t rows,
                                               const float *__restrict__ X, const Epi &epi, int64_t rg_begin,
                                               int64_t rg_step, int64_t rg_end, double *ss, Map map = Map()) {
  constexpr int V = Lanes<B>::V, L = Lanes<B>::L, G = Lanes<B>::G;
  const int lane = threadIdx.x & 31, l = lane % L, g = lane / L;
  const float *Xl = X + l * V;
  for (int64_t t = rg_begin; t < rg_end; t += rg_step) {
    const int64_t row = map(t) * G + g;
    if (row >= rows) continue;
    Vec<V> acc;
#pragma unroll
    for (int t = 0; t < V; ++t) acc.v[t] = 0.f;
    const int len = __ldg(rl + row);
    // entry pair (e, e+1), e even, of this row sits at p[(e/2)*32]
    const int4 *p = reinterpret_cast<const int4 *>(ent) + (__ldg(cp + (row >> 5)) >> 1) + (row & 31);
    int e = 0;
    // two entry pairs (4 gathers) per step: at 6 blocks per SM (40 registers)
    // this beat four pairs, which needs more registers than 6 blocks allow
    for (; e + 4 <= len; e += 4) {
      int4 pr[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) pr[u] = __ldcs(p + (size_t)((e >> 1) + u) * 32);
      Vec<V> xv[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        xv[2 * u] = gather<V, kNC>(Xl + (size_t)pr[u].x * B);
        xv[2 * u + 1] = gather<V, kNC>(Xl + (size_t)pr[u].z * B);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float w0 = __int_as_float(pr[u].y), w1 = __int_as_float(pr[u].w);
#pragma unroll
        for (int t = 0; t < V; ++t) acc.v[t] = fmaf(w0, xv[2 * u].v[t], acc.v[t]);
#pragma unroll
        for (int t = 0; t < V; ++t) acc.v[t] = fmaf(w1, xv[2 * u + 1].v[t], acc.v[t]);
      }
    }
    for (; e < len; e += 2) {
      const int4 pr = __ldcs(p + (size_t)(e >> 1) * 32);
      Vec<V> x0 = gather<V, kNC>(Xl + (size_t)pr.x * B);
      const float w0 = __int_as_float(pr.y);
#pragma unroll
      for (int t = 0; t < V; ++t) acc.v[t] = fmaf(w0, x0.v[t], acc.v[t]);
      if (e + 1 < len) {
        Vec<V> x1 = gather<V, kNC>(Xl + (size_t)pr.z * B);
        const float w1 = __int_as_float(pr.w);
#pragma unroll
        for (int t = 0; t < V; ++t) acc.v[t] = fmaf(w1, x1.v[t], acc.v[t]);
      }
    }
    epi.template operator()<V>(row, l * V, acc, ss);
  }
}

// ---------------------------------------------------------------------------
// 16-bit SELL-32 row groups: bf16 / f16 weights times a per-angle FP32 scale,
// uint16 column offsets against a 32-bit base per 16-slot row segment; a lane
// loads four slots per 128-bit load.  kTrans selects A^T (scale of each
// gathered column's angle) versus A (scale of the output row's angle).
// ---------------------------------------------------------------------------
template <bool kBf16>
__device__ __forceinline__ float w16(uint32_t ow) {
  if constexpr (kBf16) {
    return __uint_as_float(ow & 0xffff0000u);
  } else {
    return __half2float(__ushort_as_half((unsigned short)(ow >> 16)));
  }
}

// a / d for 0 <= a < 2^31 and small d: float estimate, then one exact correction
__device__ __forceinline__ int div_exact(int a, int d, float inv_d) {
  int q = (int)((float)a * inv_d);
  if (q * d > a) --q;
  else if ((q + 1) * d <= a) ++q;
  return q;
}

struct Sell16View {
  const int64_t *cpw, *cpb;
  const int32_t *rl;
  const uint32_t *ow;
  const int32_t *base;
  const float *scale;
  int np;
  float inv_np;
  int nb4 = 0;  // A in pair order (SellLp::nb4)
};

// kPre (A^T only): the gathered operand already carries the per-angle factor
// 1/a(theta) of its rows (the solvers write it that way), so the entries need
// no per-entry scale lookup.
template <int B, bool kBf16, bool kTrans, class Epi, bool kNC = true, bool kPre = false, class Map = IdentityMap>
__device__ __forceinline__ void sell16_rowgroups(const Sell16View &M, int64_t rows, const float *__restrict__ X,
                                                 const Epi &epi, int64_t rg_begin, int64_t rg_step, int64_t rg_end,
                                                 double *ss, Map map = Map()) {
  constexpr int V = Lanes<B>::V, L = Lanes<B>::L, G = Lanes<B>::G;
  const int lane = threadIdx.x & 31, l = lane % L, g = lane / L;
  const float *Xl = X + l * V;
  for (int64_t t = rg_begin; t < rg_end; t += rg_step) {
    const int64_t row = map(t) * G + g;
    if (row >= rows) continue;
    Vec<V> acc;
#pragma unroll
    for (int t = 0; t < V; ++t) acc.v[t] = 0.f;
    const int len = __ldg(M.rl + row);
    const int64_t c = row >> 5;
    const int q = (int)(row & 31);
    const uint4 *pw = reinterpret_cast<const uint4 *>(M.ow + __ldg(M.cpw + c)) + q;  // quad e/4 at pw[(e/4)*32]
    const int32_t *pb = M.base + __ldg(M.cpb + c) + q;                               // segment s at pb[s*32]
    for (int s = 0; s * 16 < len; ++s) {
      const int cb = __ldcs(pb + (size_t)s * 32);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 a0 = __ldcs(pw + (size_t)(4 * s + 2 * h) * 32);
        const uint4 a1 = __ldcs(pw + (size_t)(4 * s + 2 * h + 1) * 32);
        const uint32_t pk[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        int cc[8];
        Vec<V> xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          cc[u] = cb + (int)(pk[u] & 0xffffu);
          xv[u] = gather<V, kNC>(Xl + (size_t)cc[u] * B);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float w = w16<kBf16>(pk[u]);
          if constexpr (kTrans && !kPre) w *= __ldg(M.scale + div_exact(cc[u], M.np, M.inv_np));
#pragma unroll
          for (int t = 0; t < V; ++t) acc.v[t] = fmaf(w, xv[u].v[t], acc.v[t]);
        }
      }
    }
    int64_t out = row;
    if constexpr (!kTrans) {
      out = ray_of(row, M.nb4, M.np);
      const float sc = __ldg(M.scale + div_exact((int)out, M.np, M.inv_np));
#pragma unroll
      for (int t = 0; t < V; ++t) acc.v[t] *= sc;
    }
    epi.template operator()<V>(out, l * V, acc, ss);
  }
}

}  // namespace
}  // namespace tomo
