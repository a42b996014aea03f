// ops.cu -- batched projector / backprojector SpMM and the SIRT / CGLS drivers.
//
// Slices are independent (Sec. 3.1: each tomogram and sinogram is processed on
// its own), so a batch of B slices is one SpMM with B right-hand sides (Sec. 3:
// SpMV for one sinogram, SpMM for a stack).  Vectors live on the device
// interleaved as (rows, B): the B values of one row are contiguous, so every
// matrix entry is read once per batch and its gathered operand row is one
// coalesced B*4-byte segment.  The transpose is a stored matrix of its own
// (Sec. 3.1), so both directions are row-parallel and need no atomics.
//
// SIRT and CGLS (Sec. 2.1) are fused into the SpMM epilogues (residual and
// update of SIRT, norms of CGLS) plus small elementwise and scalar kernels;
// one iteration is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "spmm.cuh"

namespace tomo {

namespace {

constexpr int kMinBlocks = 6;  // fallback resident blocks per SM when occupancy is unknown

// ---------------------------------------------------------------------------
// SELL-32 kernels: grid-stride over row groups (see spmm.cuh)
// ---------------------------------------------------------------------------
// Six blocks (48 warps) per SM: at the unbounded 46 registers (5 blocks) the
// B = 64 pass ran 37% slower (gathers in flight limit it, not bandwidth).
// kTile: visit the row groups in image tiles (map) rather than in row order;
// a separate instantiation, so that the row-order kernels carry no mapping
template <int B, class Epi, bool kTile = false>
__global__ void __launch_bounds__(kThreads, 6) k_spmm_sell(const int64_t *__restrict__ cp,
                                                        const int32_t *__restrict__ rl,
                                                        const int2 *__restrict__ ent, int64_t rows,
                                                        const float *__restrict__ X, Epi epi,
                                                        double *__restrict__ part, TileMap map) {
  constexpr int V = Lanes<B>::V, G = Lanes<B>::G, L = Lanes<B>::L;
  double *ss = norm_slots<V, Epi>();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if constexpr (kTile)
    sell_rowgroups<B>(cp, rl, ent, rows, X, epi, warp, nwarps, (rows + G - 1) / G, ss, map);
  else
    sell_rowgroups<B>(cp, rl, ent, rows, X, epi, warp, nwarps, (rows + G - 1) / G, ss);
  if constexpr (Epi::kNorm) block_norms<V>(ss, ((threadIdx.x & 31) % L) * V, B, part);
}

template <int B, bool kBf16, bool kTrans, class Epi, bool kPre = false, bool kTile = false>
__global__ void __launch_bounds__(kThreads) k_spmm_sell16(Sell16View M, int64_t rows, const float *__restrict__ X,
                                                          Epi epi, double *__restrict__ part, TileMap map) {
  constexpr int V = Lanes<B>::V, G = Lanes<B>::G, L = Lanes<B>::L;
  double *ss = norm_slots<V, Epi>();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if constexpr (kTile)
    sell16_rowgroups<B, kBf16, kTrans, Epi, true, kPre>(M, rows, X, epi, warp, nwarps, (rows + G - 1) / G, ss, map);
  else
    sell16_rowgroups<B, kBf16, kTrans, Epi, true, kPre>(M, rows, X, epi, warp, nwarps, (rows + G - 1) / G, ss);
  if constexpr (Epi::kNorm) block_norms<V>(ss, ((threadIdx.x & 31) % L) * V, B, part);
}

// ---------------------------------------------------------------------------
// 16-bit A^T in image tiles (TileLp), B = 16, pre-scaled operand.  A
// persistent block walks the (tile, angle chunk) stream of its tiles
// (t = blockIdx.x, + gridDim.x, ...).  For every chunk it copies into shared
// memory, with cp.async and one chunk ahead of the chunk it computes (two
// buffers): the tile's detector window at the chunk's 8 angles (rows of the
// gathered operand, 64 B each), the chunk's entry blocks and its 9 group
// offsets.  The gathers then read shared memory instead of L2: the window
// holds each operand row once per tile, where the SELL pass fetches it once
// per pixel that meets it.  The global reads a copy needs (window bases,
// entry span) are loaded one chunk earlier still, so no thread waits on them.
// Warp w accumulates group w (tile rows 2w, 2w + 1); lane 4 i + l holds slices
// 4 l .. 4 l + 3 of the four pixels of quad i.  A slot's row load serves all
// four: the pixels of a 2 x 2 quad meet overlapping bins, so a quad walks
// about 0.55 rows per entry where a pixel walks one.  A shared-memory phase of
// a 128-bit load serves quads 2p and 2p + 1; rows are staged with bits 0 and
// 1 of their index swapped, so that rows 2 apart (the usual step between
// neighbouring quads) fall in opposite bank halves, and a padding slot reads
// its partner's row (a broadcast).  Every pixel adds its entries in its CSR
// order, the order of the SELL passes, with 0 times a staged row between them
// where its quad walks a bin it does not meet, as a SELL padding slot adds 0
// times a real column: the output is the same bits.
// ---------------------------------------------------------------------------
struct Tile16View {
  const uint32_t *qoff;
  const int32_t *win;
  const uint32_t *ent;
  int64_t tiles;
  int tiles_x, nch, W, max_blocks, nx, ny, np, nt;
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

constexpr int kTileQo = 12;     // group offsets copied per chunk (9 used, 16-byte pieces)
constexpr int kTilePieces = 4;  // window pieces (16 B) per thread and chunk: C W 4 <= 4 * 256, W <= 32
constexpr int kTileBlockF4 = kTileBlockBytes / 16;

// shared bytes of one launch: two buffers of (window rows, entry blocks, offsets)
inline size_t tile16_buf_bytes(const TileLp &T) {
  return (size_t)kTileChunk * T.W * kTileRow + (size_t)T.max_blocks * kTileBlockBytes + kTileQo * 4;
}
// two buffers, then the warps' FP64 norm sums (8 warps x 16 slices)
inline size_t tile16_smem(const TileLp &T) { return 2 * tile16_buf_bytes(T) + 8 * 16 * sizeof(double); }

// the four pixels' weights of a slot (2 bytes each, pixel 0 lowest) as FP32
template <bool kBf16>
__device__ __forceinline__ float tile_w(uint32_t wd, int half) {
  if constexpr (kBf16)
    return __uint_as_float(half ? (wd & 0xffff0000u) : (wd << 16));
  else
    return __half2float(__ushort_as_half((unsigned short)(half ? (wd >> 16) : (wd & 0xffffu))));
}

// Two FP32 lanes per instruction (a 64-bit register pair): d = a b + d, each
// lane rounded as one fmaf, so the sums keep the bits of the scalar form.
__device__ __forceinline__ void fma_x2(unsigned long long &d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ unsigned long long pack_x2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

// one slot of a quad: acc[2 p] holds slices (0, 1) of pixel p, acc[2 p + 1] slices (2, 3)
template <bool kBf16>
__device__ __forceinline__ void quad_fma(unsigned long long (&acc)[8], uint32_t w01, uint32_t w23, const char *row) {
  const float4 x = *reinterpret_cast<const float4 *>(row);
  const unsigned long long xa = pack_x2(x.x, x.y), xb = pack_x2(x.z, x.w);
  const float w[4] = {tile_w<kBf16>(w01, 0), tile_w<kBf16>(w01, 1), tile_w<kBf16>(w23, 0), tile_w<kBf16>(w23, 1)};
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const unsigned long long ww = pack_x2(w[p], w[p]);
    fma_x2(acc[2 * p], ww, xa);
    fma_x2(acc[2 * p + 1], ww, xb);
  }
}

template <bool kBf16, class Epi>
__global__ void __launch_bounds__(kThreads, Epi::kNorm ? 3 : 4) k_spmm_tile16(Tile16View M, const float *__restrict__ X, Epi epi,
                                                             double *__restrict__ part) {
  constexpr int B = 16, V = 4, C = kTileChunk;
  extern __shared__ float4 tile_sm[];
  const int W = M.W, Weff = min(M.W, M.np), W4 = W * 4;
  constexpr int RF4 = kTileRow / 16;  // float4 per window row slot
  const int buf_f4 = C * W * RF4 + M.max_blocks * kTileBlockF4 + kTileQo / 4;  // float4 per buffer
  // norm epilogues: each warp's FP64 sums per slice, added tile by tile in a
  // fixed order (1 KB of shared memory instead of 9 KB of per-thread slots).
  // Blocks per SM: 4 at 64 registers; the norm variants measured 0.6% faster
  // at 3 blocks with 80 registers.
  double *wss = reinterpret_cast<double *>(tile_sm + 2 * buf_f4);
  if constexpr (Epi::kNorm)
    for (int j = threadIdx.x; j < 8 * B; j += kThreads) wss[j] = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, i = lane >> 2, l = lane & 3;
  const int64_t my_tiles = (int64_t)blockIdx.x < M.tiles ? (M.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * M.nch;
  // buffer b: window rows at f4 [0, C W 4), entry blocks next, then the offsets
  auto win_of = [&](int b) { return tile_sm + b * buf_f4; };
  auto ent_of = [&](int b) { return tile_sm + b * buf_f4 + C * W * RF4; };
  auto qo_of = [&](int b) {
    return reinterpret_cast<uint32_t *>(tile_sm + b * buf_f4 + C * W * RF4 + M.max_blocks * kTileBlockF4);
  };
  // this thread's window pieces (16 B each): (angle in chunk << 16) | float offset
  // of the piece in its operand row run, -1 if none; and its staged position
  int pk[kTilePieces], pd[kTilePieces];
#pragma unroll
  for (int j = 0; j < kTilePieces; ++j) {
    const int p = threadIdx.x + j * kThreads, a = p / W4, rem = p % W4, w = rem >> 2;
    const bool on = p < C * W4 && w < Weff;
    pk[j] = on ? (a << 16) | (w * B + (rem & 3) * 4) : -1;
    pd[j] = on ? tile_swz(a * W + w) * RF4 + (rem & 3) : 0;
  }
  // (tile, chunk) of a step, advanced one step at a time
  struct Cursor {
    int64_t t;
    int k;
  };
  auto advance = [&](Cursor &c) {
    if (++c.k == M.nch) {
      c.k = 0;
      c.t += gridDim.x;
    }
  };
  // global reads of the next copy, loaded one chunk ahead
  int wnext[kTilePieces];
  uint32_t p0n = 0, p1n = 0;
  auto load_next = [&](const Cursor &c) {  // the reads of chunk c's copy
#pragma unroll
    for (int j = 0; j < kTilePieces; ++j) {
      const int m = c.k * C + (pk[j] >> 16);
      wnext[j] = (pk[j] >= 0 && m < M.nt) ? __ldg(M.win + c.t * M.nt + m) : 0;
    }
    const int64_t g0 = (c.t * M.nch + c.k) * 8;
    p0n = __ldg(M.qoff + g0);
    p1n = __ldg(M.qoff + g0 + 8);
  };
  auto stage = [&](const Cursor &c, int b) {  // copies of chunk c into buffer b (its reads are loaded)
    float4 *wb = win_of(b);
#pragma unroll
    for (int j = 0; j < kTilePieces; ++j) {
      const int m = c.k * C + (pk[j] >> 16);
      if (pk[j] >= 0 && m < M.nt)
        cp_async16(wb + pd[j], X + ((int64_t)m * M.np + wnext[j]) * B + (pk[j] & 0xffff));
    }
    const int n16 = (int)(p1n - p0n) * kTileBlockF4;
    const float4 *esrc = reinterpret_cast<const float4 *>(M.ent) + (size_t)p0n * kTileBlockF4;
    float4 *edst = ent_of(b);
    for (int p = threadIdx.x; p < n16; p += kThreads) cp_async16(edst + p, esrc + p);
    if (threadIdx.x < kTileQo / 4)
      cp_async16(qo_of(b) + 4 * threadIdx.x, M.qoff + (c.t * M.nch + c.k) * 8 + 4 * threadIdx.x);
  };

  unsigned long long acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0ull;  // +0.0f in both lanes
  Cursor cc{(int64_t)blockIdx.x, 0}, cn = cc;  // the chunk computed; the next chunk to copy
  if (total > 0) {
    load_next(cn);
    stage(cn, 0);
  }
  cp_async_commit();
  advance(cn);
  if (total > 1) load_next(cn);
  for (int64_t s = 0; s < total; ++s) {
    if (s + 1 < total) stage(cn, (int)((s + 1) & 1));
    cp_async_commit();
    advance(cn);
    if (s + 2 < total) load_next(cn);  // in flight while chunk s is computed
    cp_async_wait1();                  // this thread's copies of chunk s have landed
    __syncthreads();                   // ... and every thread's
    const int b = (int)(s & 1);
    const uint32_t *qo = qo_of(b);
    const char *wrow = reinterpret_cast<const char *>(win_of(b)) + l * 16;
    const char *eb = reinterpret_cast<const char *>(ent_of(b));
    const uint32_t q0 = qo[0];
    const int ba = (int)(qo[warp] - q0), bb = (int)(qo[warp + 1] - q0);
    for (int j = ba; j < bb; ++j) {
      const char *blk = eb + j * kTileBlockBytes;
      const uint4 w01 = *reinterpret_cast<const uint4 *>(blk + i * 16);
      const uint4 w23 = *reinterpret_cast<const uint4 *>(blk + 128 + i * 16);
      const uint32_t r = *reinterpret_cast<const uint32_t *>(blk + 256 + i * 4);
      quad_fma<kBf16>(acc, w01.x, w01.y, wrow + (r & 0xffu) * kTileRow);
      quad_fma<kBf16>(acc, w01.z, w01.w, wrow + ((r >> 8) & 0xffu) * kTileRow);
      quad_fma<kBf16>(acc, w23.x, w23.y, wrow + ((r >> 16) & 0xffu) * kTileRow);
      quad_fma<kBf16>(acc, w23.z, w23.w, wrow + (r >> 24) * kTileRow);
    }
    if (cc.k == M.nch - 1) {  // the tile is complete
      const int ty = (int)(cc.t / M.tiles_x), tx = (int)(cc.t - (int64_t)ty * M.tiles_x);
      double ss[V] = {};
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int iy = ty * kTileSide + 2 * warp + (p >> 1), ix = tx * kTileSide + 2 * i + (p & 1);
        Vec<V> v;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v.v[0]), "=f"(v.v[1]) : "l"(acc[2 * p]));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v.v[2]), "=f"(v.v[3]) : "l"(acc[2 * p + 1]));
        if (ix < M.nx && iy < M.ny) epi.template operator()<V>((int64_t)iy * M.nx + ix, l * V, v, ss);
        acc[2 * p] = acc[2 * p + 1] = 0ull;
      }
      if constexpr (Epi::kNorm) {  // over the warp's 8 quads (lanes 4 i + l), then into its sums
#pragma unroll
        for (int u = 0; u < V; ++u) {
          ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], 4);
          ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], 8);
          ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], 16);
        }
        if (i == 0)
#pragma unroll
          for (int u = 0; u < V; ++u) wss[warp * B + l * V + u] += ss[u];
      }
    }
    advance(cc);
    __syncthreads();  // buffer b is refilled by the next iteration's copies
  }
  if constexpr (Epi::kNorm) {  // the block's sums, warps in order, into part[blockIdx.x * B + s]
    __syncthreads();
    for (int s = threadIdx.x; s < B; s += kThreads) {
      double a = 0.0;
      for (int w = 0; w < 8; ++w) a += wss[w * B + s];
      part[(int64_t)blockIdx.x * B + s] = a;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 CSR SpMM, B >= 4: L = B/4 lanes per row own 4 slices each (float4),
// G = 32/L rows per warp.  Grid-stride over row groups.
// ---------------------------------------------------------------------------
template <int B, class Epi>
__device__ __forceinline__ void csr_spmm(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                         const float *__restrict__ val, int64_t rows, const float *__restrict__ X,
                                         Epi epi, double *__restrict__ part) {
  constexpr int L = B / 4, G = 32 / L;
  const int lane = threadIdx.x & 31, l = lane % L, g = lane / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float *Xl = X + l * 4;
  double ss[4] = {0, 0, 0, 0};
  for (int64_t rg = warp; rg * G < rows; rg += nwarps) {
    const int64_t row = rg * G + g;
    if (row >= rows) continue;
    Vec<4> acc = {{0.f, 0.f, 0.f, 0.f}};
    int64_t e = __ldg(rp + row);
    const int64_t end = __ldg(rp + row + 1);
    for (; e + 8 <= end; e += 8) {
      int c[8];
      float w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[u] = __ldg(ci + e + u);
        w[u] = __ldg(val + e + u);
      }
      Vec<4> xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = ldg_vec<4>(Xl + (size_t)c[u] * B);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc.v[t] = fmaf(w[u], xv[u].v[t], acc.v[t]);
    }
    for (; e < end; ++e) {
      int c = __ldg(ci + e);
      float w = __ldg(val + e);
      Vec<4> xv = ldg_vec<4>(Xl + (size_t)c * B);
#pragma unroll
      for (int t = 0; t < 4; ++t) acc.v[t] = fmaf(w, xv.v[t], acc.v[t]);
    }
    epi.template operator()<4>(row, l * 4, acc, ss);
  }
  if constexpr (Epi::kNorm) block_norms<4>(ss, l * 4, B, part);
}

template <int B, class Epi>
__global__ void __launch_bounds__(kThreads) k_spmm_f32(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                       const float *__restrict__ val, int64_t rows,
                                                       const float *__restrict__ X, Epi epi,
                                                       double *__restrict__ part) {
  csr_spmm<B>(rp, ci, val, rows, X, epi, part);
}

// The norm epilogues carry 2 x 4 FP64 accumulators through the row loop;
// unbounded they take 48 registers (5 blocks per SM).  Held at 6 blocks per
// SM they fit 40 registers unspilled.  Measured at 512x512x360 (CGLS passes):
// B = 64, 6 blocks 1.94 ms vs 5 blocks 2.63 ms; B = 16, 6 blocks 0.99 ms vs
// 5 blocks 0.90 ms.  So the bounded form serves B >= 32 only.
template <int B, class Epi>
__global__ void __launch_bounds__(kThreads, 6) k_spmm_f32_norm(const int64_t *__restrict__ rp,
                                                               const int32_t *__restrict__ ci,
                                                               const float *__restrict__ val, int64_t rows,
                                                               const float *__restrict__ X, Epi epi,
                                                               double *__restrict__ part) {
  csr_spmm<B>(rp, ci, val, rows, X, epi, part);
}

template <int B, class Epi>
constexpr auto csr_kernel() {
  if constexpr (Epi::kNorm && B >= 32)
    return k_spmm_f32_norm<B, Epi>;
  else
    return k_spmm_f32<B, Epi>;
}

// ---------------------------------------------------------------------------
// FP32 CSR SpMM for B in {1, 2}: P lanes split the entries of one row (CSR
// vector form), each lane holds all B slices, shuffle reduction at the end.
// ---------------------------------------------------------------------------
template <int B, int P, class Epi>
__global__ void __launch_bounds__(kThreads) k_spmv_f32(const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci,
                                                       const float *__restrict__ val, int64_t rows,
                                                       const float *__restrict__ X, Epi epi,
                                                       double *__restrict__ part) {
  constexpr int G = 32 / P;
  const int lane = threadIdx.x & 31, p = lane % P, g = lane / P;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double ss[B];
#pragma unroll
  for (int t = 0; t < B; ++t) ss[t] = 0.0;
  for (int64_t rg = warp; rg * G < rows; rg += nwarps) {
    const int64_t row = rg * G + g;
    const bool ok = row < rows;
    Vec<B> acc;
#pragma unroll
    for (int t = 0; t < B; ++t) acc.v[t] = 0.f;
    if (ok) {
      int64_t e = __ldg(rp + row) + p;
      const int64_t end = __ldg(rp + row + 1);
      for (; e + 3 * P < end; e += 4 * P) {
        int c[4];
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = __ldg(ci + e + u * P);
          w[u] = __ldg(val + e + u * P);
        }
        Vec<B> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ldg_vec<B>(X + (size_t)c[u] * B);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int t = 0; t < B; ++t) acc.v[t] = fmaf(w[u], xv[u].v[t], acc.v[t]);
      }
      for (; e < end; e += P) {
        int c = __ldg(ci + e);
        float w = __ldg(val + e);
        Vec<B> xv = ldg_vec<B>(X + (size_t)c * B);
#pragma unroll
        for (int t = 0; t < B; ++t) acc.v[t] = fmaf(w, xv.v[t], acc.v[t]);
      }
    }
#pragma unroll
    for (int o = P / 2; o; o >>= 1)
#pragma unroll
      for (int t = 0; t < B; ++t) acc.v[t] += __shfl_xor_sync(0xffffffffu, acc.v[t], o);
    if (ok && p == 0) epi.template operator()<B>(row, 0, acc, ss);
  }
  if constexpr (Epi::kNorm) block_norms<B>(ss, 0, B, part);
}

// ---------------------------------------------------------------------------
// Data fit ||b - A x|| of one slice with FP64 accumulation.  The product of an
// FP32 value and an FP32 operand is exact in FP64 (24 + 24 significand bits),
// so the only rounding left is the FP64 summation: the result is the data fit
// of the FP32-valued operator to about 1e-15 relative, whatever the row
// length.  A warp per row (lanes split its entries), slice-major vectors;
// per-block partials of r^2 in a fixed order, summed by k_sum_parts.
// ---------------------------------------------------------------------------
constexpr int kResidBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_resid_f64(const int64_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci,
                                                        const float *__restrict__ val, int64_t rows,
                                                        const float *__restrict__ x, const float *__restrict__ b,
                                                        double *__restrict__ part) {
  __shared__ double red[kWarps];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double ss = 0.0;
  for (int64_t row = warp; row < rows; row += nwarps) {
    double acc = 0.0;
    const int64_t end = __ldg(rp + row + 1);
    for (int64_t e = __ldg(rp + row) + lane; e < end; e += 32)
      acc = fma((double)__ldg(val + e), (double)__ldg(x + __ldg(ci + e)), acc);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double r = (double)__ldg(b + row) - acc;
    ss = fma(r, r, ss);
  }
  if (lane == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// out = sqrt(sum of part[0 .. n)), summed in index order by one thread
__global__ void k_sum_parts(const double *__restrict__ part, int n, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = sqrt(t);
  }
}

// ---------------------------------------------------------------------------
// Layout: slice-major (n_z, n) <-> interleaved (n, B), through shared memory.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(kThreads) k_interleave(const float *__restrict__ src, int64_t n, int cnt,
                                                         float *__restrict__ dst) {
  constexpr int TI = 32;
  __shared__ float tile[B][TI + 1];
  const int64_t i0 = (int64_t)blockIdx.x * TI;
  for (int t = threadIdx.x; t < B * TI; t += blockDim.x) {
    int s = t / TI, i = t % TI;
    float v = 0.f;
    if (s < cnt && i0 + i < n) v = src[(int64_t)s * n + i0 + i];
    tile[s][i] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * TI; t += blockDim.x) {
    int i = t / B, s = t % B;
    if (i0 + i < n) dst[(i0 + i) * B + s] = tile[s][i];
  }
}

template <int B>
__global__ void __launch_bounds__(kThreads) k_deinterleave(const float *__restrict__ src, int64_t n,
                                                           int cnt, float *__restrict__ dst) {
  constexpr int TI = 32;
  __shared__ float tile[B][TI + 1];
  const int64_t i0 = (int64_t)blockIdx.x * TI;
  for (int t = threadIdx.x; t < B * TI; t += blockDim.x) {
    int i = t / B, s = t % B;
    if (i0 + i < n) tile[s][i] = src[(i0 + i) * B + s];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * TI; t += blockDim.x) {
    int s = t / TI, i = t % TI;
    if (s < cnt && i0 + i < n) dst[(int64_t)s * n + i0 + i] = tile[s][i];
  }
}

// ---------------------------------------------------------------------------
// CGLS scalar and vector kernels.  Per-slice scalars (FP64), 8 per slice:
//   [0] gamma = ||s||^2   [1] alpha   [2] beta   [3] frozen (0/1)
// ---------------------------------------------------------------------------
__device__ double block_sum_slice(const double *part, int nblk, int B, int s) {
  __shared__ double red[kThreads];
  double a = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += part[(int64_t)b * B + s];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = kThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// one block per slice
__global__ void __launch_bounds__(kThreads) k_cgls_init(const double *part, int nblk, int B, double *scal,
                                                        int *it) {
  int s = blockIdx.x;
  double g = block_sum_slice(part, nblk, B, s);
  if (threadIdx.x == 0) {
    scal[s * 8 + 0] = g;
    scal[s * 8 + 1] = 0.0;
    scal[s * 8 + 2] = 0.0;
    scal[s * 8 + 3] = 0.0;
    if (s == 0) *it = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_cgls_alpha(const double *part, int nblk, int B, double *scal) {
  int s = blockIdx.x;
  double qq = block_sum_slice(part, nblk, B, s);
  if (threadIdx.x == 0) {
    double gam = scal[s * 8 + 0];
    bool frozen = scal[s * 8 + 3] != 0.0 || gam == 0.0 || qq == 0.0;
    scal[s * 8 + 3] = frozen ? 1.0 : 0.0;
    scal[s * 8 + 1] = frozen ? 0.0 : gam / qq;
  }
}

// gamma' = ||s||^2, beta = gamma'/gamma, history of ||r|| (rr partials optional)
__global__ void __launch_bounds__(kThreads) k_cgls_beta(const double *part_s, int nblk, const double *part_r,
                                                        int nblk_r, int B, double *scal, double *hist,
                                                        const int *it, int s0, int cnt, int nz) {
  int s = blockIdx.x;
  double gs = block_sum_slice(part_s, nblk, B, s);
  double rr = part_r ? block_sum_slice(part_r, nblk_r, B, s) : 0.0;
  if (threadIdx.x == 0) {
    bool frozen = scal[s * 8 + 3] != 0.0;
    if (frozen) {
      scal[s * 8 + 2] = 0.0;
    } else {
      scal[s * 8 + 2] = gs / scal[s * 8 + 0];
      scal[s * 8 + 0] = gs;
    }
    if (hist && s < cnt) hist[(int64_t)(*it) * nz + s0 + s] = sqrt(rr);
  }
}

// state in / out: per-slice gamma and frozen flag (padding slices frozen)
__global__ void k_cgls_load(double *scal, const double *gamma, const int32_t *frozen, int cnt, int B, int *it) {
  for (int s = threadIdx.x; s < B; s += blockDim.x) {
    const bool real = s < cnt;
    scal[s * 8 + 0] = real ? gamma[s] : 0.0;
    scal[s * 8 + 1] = 0.0;
    scal[s * 8 + 2] = 0.0;
    scal[s * 8 + 3] = (!real || frozen[s] != 0) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) *it = 0;
}

__global__ void k_cgls_save(const double *scal, double *gamma, int32_t *frozen, int cnt) {
  for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
    gamma[s] = scal[s * 8 + 0];
    frozen[s] = scal[s * 8 + 3] != 0.0 ? 1 : 0;
  }
}

// x += alpha p (cols); r -= alpha q (rows), optional ||r||^2 partials
// rs (nullable): also write r times 1/a(theta) of each row's angle (scale, per
// angle; np bins per angle), the operand of the 16-bit A^T pass
template <int B>
__global__ void __launch_bounds__(kThreads) k_cgls_step(float *__restrict__ x, const float *__restrict__ p,
                                                        int64_t ncols, float *__restrict__ r,
                                                        const float *__restrict__ q, int64_t nrows,
                                                        const double *__restrict__ scal,
                                                        double *__restrict__ part_r, float *__restrict__ rs,
                                                        const float *__restrict__ scale, int np) {
  constexpr int V = B >= 4 ? 4 : B;
  constexpr int PER = B / V;  // vectors per row
  const int64_t nvx = ncols * PER, nvr = nrows * PER;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  // every thread keeps one fixed slice offset (nth is a multiple of PER)
  const int s0 = (int)(tid % PER) * V;
  float al[V];
#pragma unroll
  for (int t = 0; t < V; ++t) al[t] = (float)scal[(s0 + t) * 8 + 1];
  for (int64_t i = tid; i < nvx; i += nth) {
    Vec<V> xv = ld_vec<V>(x + i * V), pv = ld_vec<V>(p + i * V);
#pragma unroll
    for (int t = 0; t < V; ++t) xv.v[t] = fmaf(al[t], pv.v[t], xv.v[t]);
    st_vec<V>(x + i * V, xv);
  }
  double ss[V];
#pragma unroll
  for (int t = 0; t < V; ++t) ss[t] = 0.0;
  for (int64_t i = tid; i < nvr; i += nth) {
    Vec<V> rv = ld_vec<V>(r + i * V), qv = ld_vec<V>(q + i * V);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      rv.v[t] = fmaf(-al[t], qv.v[t], rv.v[t]);
      ss[t] += (double)rv.v[t] * (double)rv.v[t];
    }
    st_vec<V>(r + i * V, rv);
    if (rs) {
      const float sc = __ldg(scale + (i / PER) / np);
#pragma unroll
      for (int t = 0; t < V; ++t) rv.v[t] *= sc;
      st_vec<V>(rs + i * V, rv);
    }
  }
  if (part_r) block_norms<V>(ss, s0, B, part_r);
}

// dst = src times 1/a(theta) of each row's angle, (rows, B) interleaved (dst may be src)
template <int B>
__global__ void __launch_bounds__(kThreads) k_scale_rows(const float *src, float *dst, int64_t nrows,
                                                         const float *__restrict__ scale, int np) {
  const int64_t n = nrows * B;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] * __ldg(scale + (i / B) / np);
}

// p = s + beta p (cols); advances the iteration counter
template <int B>
__global__ void __launch_bounds__(kThreads) k_cgls_dir(float *__restrict__ p, const float *__restrict__ s,
                                                       int64_t ncols, const double *__restrict__ scal,
                                                       int *it) {
  constexpr int V = B >= 4 ? 4 : B;
  constexpr int PER = B / V;
  const int64_t nv = ncols * PER;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int s0 = (int)(tid % PER) * V;
  float be[V];
#pragma unroll
  for (int t = 0; t < V; ++t) be[t] = (float)scal[(s0 + t) * 8 + 2];
  for (int64_t i = tid; i < nv; i += nth) {
    Vec<V> pv = ld_vec<V>(p + i * V), sv = ld_vec<V>(s + i * V);
#pragma unroll
    for (int t = 0; t < V; ++t) pv.v[t] = fmaf(be[t], pv.v[t], sv.v[t]);
    st_vec<V>(p + i * V, pv);
  }
  if (tid == 0 && it) ++*it;
}

// ---------------------------------------------------------------------------
// Preconditioned SIRT with the Barzilai-Borwein step (Sec. 3.1; the
// preconditioner P = F^dagger D^(1/2) F of Sec. 2.1).  Per-slice scalars
// (FP64), 4 per slice: [0] alpha of the last step  [1] frozen (0/1)
// [2] a previous step exists (0/1).
// ---------------------------------------------------------------------------

// rf = P^T P r on every projection row: rf[m, k, :] = sum_j tap[|k - j|] r[m, j, :]
// over the n_p bins of row m, j ascending (interleaved (rows, B) vectors).
// Block (256 threads) = 256/Q bin groups x Q slice groups of V slices; a
// thread owns KB adjacent output bins and keeps the KB taps it needs in
// registers, shifting them by one bin per step of j (the unrolled shift costs
// no moves).  Grid: (ceil(n_p / TK), n_theta).
constexpr int kRampKB = 8;  // output bins per thread

// output bins one block of k_ramp_filter<B> covers
template <int B>
constexpr int ramp_tile_bins() {
  return kRampKB * kThreads / (B >= 4 ? B / 4 : 1);
}

// scale (nullable): multiply projection row m's output by scale[m] (1/a(theta_m),
// for the 16-bit A^T pass that follows)
template <int B>
__global__ void __launch_bounds__(kThreads) k_ramp_filter(const float *__restrict__ r, float *__restrict__ rf,
                                                          const float *__restrict__ tap, int np,
                                                          const float *__restrict__ scale) {
  constexpr int V = B >= 4 ? 4 : B, Q = B / V, KB = kRampKB, TK = ramp_tile_bins<B>(), TJ = 32;
  __shared__ __align__(16) float rs[TJ * B];
  const int q = threadIdx.x % Q, kg = threadIdx.x / Q;
  const int64_t m = blockIdx.y;
  const int k0 = blockIdx.x * TK + kg * KB;
  const float *rm = r + m * np * B;
  auto tapv = [&](int d) { d = d < 0 ? -d : d; return d < np ? __ldg(tap + d) : 0.f; };
  float acc[KB][V];
#pragma unroll
  for (int i = 0; i < KB; ++i)
#pragma unroll
    for (int t = 0; t < V; ++t) acc[i][t] = 0.f;
  for (int j0 = 0; j0 < np; j0 += TJ) {
    __syncthreads();
    for (int t = threadIdx.x; t < TJ * B; t += kThreads) {
      const int jj = t / B;
      rs[t] = j0 + jj < np ? rm[(int64_t)(j0 + jj) * B + (t % B)] : 0.f;
    }
    __syncthreads();
    float w[KB];  // w[i] = tap at offset k0 + i - j
#pragma unroll
    for (int i = 0; i < KB; ++i) w[i] = tapv(k0 + i - j0);
#pragma unroll 8
    for (int jj = 0; jj < TJ; ++jj) {
      const Vec<V> xv = ld_vec<V>(rs + jj * B + q * V);
#pragma unroll
      for (int i = 0; i < KB; ++i)
#pragma unroll
        for (int t = 0; t < V; ++t) acc[i][t] = fmaf(w[i], xv.v[t], acc[i][t]);
#pragma unroll
      for (int i = KB - 1; i > 0; --i) w[i] = w[i - 1];
      w[0] = tapv(k0 - (j0 + jj) - 1);
    }
  }
  const float sc = scale ? __ldg(scale + m) : 1.0f;
#pragma unroll
  for (int i = 0; i < KB; ++i) {
    if (k0 + i >= np) break;
    Vec<V> o;
#pragma unroll
    for (int t = 0; t < V; ++t) o.v[t] = acc[i][t] * sc;
    st_vec<V>(rf + (m * np + k0 + i) * B + q * V, o);
  }
}

// per-slice partials of <g_prev, g_prev> and <g_prev, g - g_prev> (FP64)
template <int B>
__global__ void __launch_bounds__(kThreads) k_bb_dots(const float *__restrict__ gp, const float *__restrict__ gn,
                                                      int64_t ncols, double *__restrict__ part_p,
                                                      double *__restrict__ part_q) {
  constexpr int V = B >= 4 ? 4 : B;
  constexpr int PER = B / V;
  const int64_t nv = ncols * PER;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int s0 = (int)(tid % PER) * V;
  double pp[V], pq[V];
#pragma unroll
  for (int t = 0; t < V; ++t) pp[t] = pq[t] = 0.0;
  for (int64_t i = tid; i < nv; i += nth) {
    const Vec<V> a = ld_vec<V>(gp + i * V), b = ld_vec<V>(gn + i * V);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const double ga = a.v[t];
      pp[t] += ga * ga;
      pq[t] += ga * ((double)b.v[t] - ga);
    }
  }
  block_norms<V>(pp, s0, B, part_p);
  block_norms<V>(pq, s0, B, part_q);
}

// one block per slice: the step alpha (first step, BB1 or frozen) and ||r||
__global__ void __launch_bounds__(kThreads) k_bb_alpha(const double *part_p, const double *part_q, int nblk,
                                                       const double *part_r, int nblk_r, int B, double *scal,
                                                       double first_step, double *hist, const int *it, int s0,
                                                       int cnt, int nz) {
  const int s = blockIdx.x;
  const double P = block_sum_slice(part_p, nblk, B, s);
  const double Qd = block_sum_slice(part_q, nblk, B, s);
  const double rr = part_r ? block_sum_slice(part_r, nblk_r, B, s) : 0.0;
  if (threadIdx.x == 0) {
    const double a_prev = scal[s * 4 + 0];
    double a = 0.0;
    if (scal[s * 4 + 1] != 0.0) {
      a = 0.0;
    } else if (scal[s * 4 + 2] == 0.0) {
      a = first_step;
      scal[s * 4 + 2] = 1.0;
    } else {
      // s = a_prev g_prev, y = -(g - g_prev): <s,s> = a_prev^2 P, <s,y> = -a_prev Q
      const double ss = a_prev * a_prev * P, sy = -a_prev * Qd;
      if (ss > 0.0 && sy > 0.0) {
        a = ss / sy;
      } else {
        scal[s * 4 + 1] = 1.0;
      }
    }
    scal[s * 4 + 0] = a;
    if (hist && s < cnt) hist[(int64_t)(*it) * nz + s0 + s] = sqrt(rr);
  }
}

// x += alpha g; advances the iteration counter
template <int B>
__global__ void __launch_bounds__(kThreads) k_bb_update(float *__restrict__ x, const float *__restrict__ g,
                                                        int64_t ncols, const double *__restrict__ scal, int *it) {
  constexpr int V = B >= 4 ? 4 : B;
  constexpr int PER = B / V;
  const int64_t nv = ncols * PER;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int s0 = (int)(tid % PER) * V;
  float al[V];
#pragma unroll
  for (int t = 0; t < V; ++t) al[t] = (float)scal[(s0 + t) * 4 + 0];
  for (int64_t i = tid; i < nv; i += nth) {
    Vec<V> xv = ld_vec<V>(x + i * V);
    const Vec<V> gv = ld_vec<V>(g + i * V);
#pragma unroll
    for (int t = 0; t < V; ++t) xv.v[t] = fmaf(al[t], gv.v[t], xv.v[t]);
    st_vec<V>(x + i * V, xv);
  }
  if (tid == 0) ++*it;
}

// state in / out: alpha, frozen; padding slices (s >= cnt) frozen
__global__ void k_bb_load(double *scal, const double *alpha, const int32_t *frozen, int cnt, int B, int *it) {
  for (int s = threadIdx.x; s < B; s += blockDim.x) {
    const bool real = s < cnt;
    scal[s * 4 + 0] = (alpha && real) ? alpha[s] : 0.0;
    scal[s * 4 + 1] = (!real || (frozen && frozen[s] != 0)) ? 1.0 : 0.0;
    scal[s * 4 + 2] = (alpha && real && alpha[s] > 0.0) ? 1.0 : 0.0;  // alpha 0: no previous step
    scal[s * 4 + 3] = 0.0;
  }
  if (threadIdx.x == 0) *it = 0;
}

__global__ void k_bb_save(const double *scal, double *alpha, int32_t *frozen, int cnt) {
  for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
    alpha[s] = scal[s * 4 + 0];
    frozen[s] = scal[s * 4 + 1] != 0.0 ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------
struct Op {  // one SpMM operand (A or A^T) in the selected storage
  const Csr *m;
  const Sell *sell;
  const SellLp *lp;
  int format;
  bool trans;
  bool bf16;
  const float *scale;
  int np;
  bool pre = false;  // 16-bit A^T: the operand already carries 1/a(theta) per row
  int nx = 0, ny = 0;  // image shape (A^T rows are its pixels)
  const std::vector<SellLp> *bands = nullptr;  // 16-bit A stored as column bands
  float *partial = nullptr;                     // (rows, B) sums of the bands before the last
  int order = 0;                                // A^T row-group order (Exec::order)
  int blocks = 0;                               // resident blocks per SM to launch (0: all that fit)
  const TileLp *tl = nullptr;                   // 16-bit A^T in tiles, when the order allows it
  int nt = 0;
};

// blocks per SM a launch of the op uses: all that fit, or fewer when asked
inline int op_res(const Op &op, int res) { return op.blocks > 0 ? std::min(res, op.blocks) : res; }

// Row-group order of a SELL pass: row order for A; for A^T image tiles (see
// TileMap) when asked, or by default when the gathered batch of sinograms
// (rows of A times B floats) exceeds half of the L2.
inline TileMap tile_map(const Op &op, int G, int B) {
  if (!op.trans || op.order == 1 || op.nx % G != 0 || op.ny % 8 != 0) return TileMap{0, 0};
  if (op.order == 0 && op.m->cols * (int64_t)B * 4 <= (int64_t)(64 << 20)) return TileMap{0, 0};
  return TileMap{op.nx / G, op.ny / 8};
}

// rows one warp handles in the SpMM kernels of a format / width
inline int rows_per_warp(int format, int B) {
  if (format == TOMO_FMT_CSR && B < 4) return 1;  // CSR-vector: a warp per row
  const int V = B >= 4 ? 4 : B;
  return 32 / (B / V);
}

// Grid of a grid-stride SpMM launch: never more blocks than can be resident
// at once (a second partial wave would idle most SMs), never more than the
// row groups need.  `resident` is blocks per SM from the occupancy API.
inline int spmm_grid(int64_t rows, int G, int resident = kMinBlocks) {
  int64_t groups = (rows + G - 1) / G;
  int64_t blocks = (groups + kWarps - 1) / kWarps;
  int64_t cap = (int64_t)num_sms() * std::max(1, std::min(resident, 8));
  return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

template <typename K>
int resident_blocks(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, 0) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

inline int max_spmm_grid() { return num_sms() * 8; }

// The tiled 16-bit A^T pass serves the pre-scaled passes at B = 16 (op.tl is
// set only when the order allows it).
// (epilogues of the A^T passes: backprojection, SIRT update, CGLS s = A^T r)
template <class Epi>
constexpr bool kTile16Epi =
    std::is_same<Epi, EpiStore>::value || std::is_same<Epi, EpiStoreNorm>::value || std::is_same<Epi, EpiSirtUpdate>::value;
template <class Epi>
inline bool use_tile16(const Op &op, int B) {
  return kTile16Epi<Epi> && B == 16 && op.trans && op.pre && op.tl != nullptr && op.tl->W <= 32;
}

// Its kernels take more than the default 48 KB of dynamic shared memory: raise
// each instantiation's limit once, before any launch or occupancy query (the
// operators call this when they set op.tl, ahead of any graph capture).
template <class K>
void allow_tile16_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  cudaGetLastError();
}

void prepare_tile16() {
  static const bool done = [] {
    allow_tile16_smem(k_spmm_tile16<true, EpiStore>);
    allow_tile16_smem(k_spmm_tile16<false, EpiStore>);
    allow_tile16_smem(k_spmm_tile16<true, EpiStoreNorm>);
    allow_tile16_smem(k_spmm_tile16<false, EpiStoreNorm>);
    allow_tile16_smem(k_spmm_tile16<true, EpiSirtUpdate>);
    allow_tile16_smem(k_spmm_tile16<false, EpiSirtUpdate>);
    return true;
  }();
  (void)done;
}

// persistent grid of the tiled pass: the blocks that fit at once, at most one per tile
template <bool kBf16, class Epi>
int tile16_grid(const Op &op) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spmm_tile16<kBf16, Epi>, kThreads,
                                                    tile16_smem(*op.tl)) != cudaSuccess ||
      n <= 0) {
    cudaGetLastError();
    n = 1;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(op.tl->tiles, (int64_t)num_sms() * op_res(op, n)));
}

template <class Epi>
void launch_tile16(const Op &op, const float *X, Epi epi, double *part, cudaStream_t st) {
  const TileLp &T = *op.tl;
  const Tile16View v{T.qoff, T.win, T.ent, T.tiles, T.tiles_x, T.nch, T.W, T.max_blocks, op.nx, op.ny, op.np, op.nt};
  const size_t smem = tile16_smem(T);
  if (op.bf16)
    k_spmm_tile16<true, Epi><<<tile16_grid<true, Epi>(op), kThreads, smem, st>>>(v, X, epi, part);
  else
    k_spmm_tile16<false, Epi><<<tile16_grid<false, Epi>(op), kThreads, smem, st>>>(v, X, epi, part);
}

// The CSR gather kernels keep at most 6 blocks (48 warps) per SM: the
// 32-register norm variants would fit 8, and measured 20-30% slower there
// (more rows in flight share the same L1 for their gathered operand rows).
constexpr int kCsrMaxBlocks = 6;

template <int B, class Epi>
void launch_spmm(const Op &op, const float *X, Epi epi, double *part, cudaStream_t st) {
  const int G = rows_per_warp(op.format, B);
  const int64_t rows = op.m->rows;
  if (op.format == TOMO_FMT_SELL) {
    const Sell &S = *op.sell;
    const TileMap map = tile_map(op, G, B);
    if (map.gx) {
      static const int res = resident_blocks(k_spmm_sell<B, Epi, true>);
      k_spmm_sell<B, Epi, true><<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(S.cp, S.rl, S.ent, rows, X,
                                                                                           epi, part, map);
    } else {
      static const int res = resident_blocks(k_spmm_sell<B, Epi>);
      k_spmm_sell<B, Epi><<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(S.cp, S.rl, S.ent, rows, X, epi,
                                                                                    part, map);
    }
  } else if (op.format == TOMO_FMT_SELL16 && op.bands) {
    // one pass per column band; the bands' partial sums meet in op.partial
    const float inv_np = 1.0f / (float)op.np;
    const int K = (int)op.bands->size();
    for (int b = 0; b < K; ++b) {
      const SellLp &L = (*op.bands)[b];
      const Sell16View view{L.cpw, L.cpb, L.rl, L.ow, L.base, op.scale, op.np, inv_np, L.nb4};
      if (b < K - 1) {
        const EpiBandPartial ep{op.partial, B, b == 0};
        if (op.bf16) {
          static const int res = resident_blocks(k_spmm_sell16<B, true, false, EpiBandPartial>);
          k_spmm_sell16<B, true, false, EpiBandPartial>
              <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, ep, nullptr, TileMap{0, 0});
        } else {
          static const int res = resident_blocks(k_spmm_sell16<B, false, false, EpiBandPartial>);
          k_spmm_sell16<B, false, false, EpiBandPartial>
              <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, ep, nullptr, TileMap{0, 0});
        }
      } else {
        const EpiBandLast<Epi> el{op.partial, B, epi};
        if (op.bf16) {
          static const int res = resident_blocks(k_spmm_sell16<B, true, false, EpiBandLast<Epi>>);
          k_spmm_sell16<B, true, false, EpiBandLast<Epi>>
              <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, el, part, TileMap{0, 0});
        } else {
          static const int res = resident_blocks(k_spmm_sell16<B, false, false, EpiBandLast<Epi>>);
          k_spmm_sell16<B, false, false, EpiBandLast<Epi>>
              <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, el, part, TileMap{0, 0});
        }
      }
    }
  } else if (op.format == TOMO_FMT_SELL16 && use_tile16<Epi>(op, B)) {
    if constexpr (kTile16Epi<Epi>) launch_tile16(op, X, epi, part, st);
  } else if (op.format == TOMO_FMT_SELL16) {
    const SellLp &L = *op.lp;
    const float inv_np = 1.0f / (float)op.np;
    const Sell16View view{L.cpw, L.cpb, L.rl, L.ow, L.base, op.scale, op.np, inv_np, L.nb4};
    const TileMap map = tile_map(op, G, B);
#define TOMO_SELL16(BF, TR, PRE)                                                                               \
  do {                                                                                                         \
    if (TR && map.gx) {                                                                                        \
      static const int res = resident_blocks(k_spmm_sell16<B, BF, TR, Epi, PRE, true>);                        \
      k_spmm_sell16<B, BF, TR, Epi, PRE, true>                                                                 \
          <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, epi, part, map);          \
    } else {                                                                                                   \
      static const int res = resident_blocks(k_spmm_sell16<B, BF, TR, Epi, PRE>);                              \
      k_spmm_sell16<B, BF, TR, Epi, PRE>                                                                       \
          <<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(view, rows, X, epi, part, map);          \
    }                                                                                                          \
  } while (0)
    if (op.bf16) {
      if (op.trans && op.pre) TOMO_SELL16(true, true, true);
      else if (op.trans) TOMO_SELL16(true, true, false);
      else TOMO_SELL16(true, false, false);
    } else {
      if (op.trans && op.pre) TOMO_SELL16(false, true, true);
      else if (op.trans) TOMO_SELL16(false, true, false);
      else TOMO_SELL16(false, false, false);
    }
#undef TOMO_SELL16
  } else {
    if constexpr (B >= 4) {
      static const int res = std::min(resident_blocks(csr_kernel<B, Epi>()), kCsrMaxBlocks);
      csr_kernel<B, Epi>()<<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(op.m->rp, op.m->ci, op.m->v, rows, X, epi,
                                                                        part);
    } else {
      static const int res = resident_blocks(k_spmv_f32<B, 32, Epi>);
      k_spmv_f32<B, 32, Epi><<<spmm_grid(rows, G, op_res(op, res)), kThreads, 0, st>>>(op.m->rp, op.m->ci, op.m->v, rows, X,
                                                                            epi, part);
    }
  }
}

// grid the SpMM of (op, B, Epi) will use (the same instantiation launch_spmm
// picks); CGLS sizes its norm reductions with it
template <int B, class Epi>
int spmm_grid_of(const Op &op) {
  const int G = rows_per_warp(op.format, B);
  const bool tile = tile_map(op, G, B).gx != 0;
  int res = kMinBlocks;
  if constexpr (kTile16Epi<Epi>)
    if (op.format == TOMO_FMT_SELL16 && use_tile16<Epi>(op, B))
      return op.bf16 ? tile16_grid<true, Epi>(op) : tile16_grid<false, Epi>(op);
  if (op.format == TOMO_FMT_SELL) {
    res = tile ? resident_blocks(k_spmm_sell<B, Epi, true>) : resident_blocks(k_spmm_sell<B, Epi>);
  } else if (op.format == TOMO_FMT_SELL16 && op.bands) {  // the last band's pass reduces the norms
    res = op.bf16 ? resident_blocks(k_spmm_sell16<B, true, false, EpiBandLast<Epi>>)
                  : resident_blocks(k_spmm_sell16<B, false, false, EpiBandLast<Epi>>);
  } else if (op.format == TOMO_FMT_SELL16 && op.trans) {
    if (op.bf16)
      res = op.pre ? (tile ? resident_blocks(k_spmm_sell16<B, true, true, Epi, true, true>)
                           : resident_blocks(k_spmm_sell16<B, true, true, Epi, true>))
                   : (tile ? resident_blocks(k_spmm_sell16<B, true, true, Epi, false, true>)
                           : resident_blocks(k_spmm_sell16<B, true, true, Epi>));
    else
      res = op.pre ? (tile ? resident_blocks(k_spmm_sell16<B, false, true, Epi, true, true>)
                           : resident_blocks(k_spmm_sell16<B, false, true, Epi, true>))
                   : (tile ? resident_blocks(k_spmm_sell16<B, false, true, Epi, false, true>)
                           : resident_blocks(k_spmm_sell16<B, false, true, Epi>));
  } else if (op.format == TOMO_FMT_SELL16) {
    res = op.bf16 ? resident_blocks(k_spmm_sell16<B, true, false, Epi>)
                  : resident_blocks(k_spmm_sell16<B, false, false, Epi>);
  } else if constexpr (B >= 4) {
    res = std::min(resident_blocks(csr_kernel<B, Epi>()), kCsrMaxBlocks);
  } else {
    res = resident_blocks(k_spmv_f32<B, 32, Epi>);
  }
  return spmm_grid(op.m->rows, G, op_res(op, res));
}

inline int elem_grid(int64_t n_vec) {
  int64_t blocks = (n_vec + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)num_sms() * 8;
  return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

template <int B>
void interleave(const float *src, int64_t n, int cnt, float *dst, cudaStream_t st) {
  k_interleave<B><<<(unsigned)((n + 31) / 32), kThreads, 0, st>>>(src, n, cnt, dst);
}
template <int B>
void deinterleave(const float *src, int64_t n, int cnt, float *dst, cudaStream_t st) {
  k_deinterleave<B><<<(unsigned)((n + 31) / 32), kThreads, 0, st>>>(src, n, cnt, dst);
}

// carve a workspace into 256-byte aligned pieces (p == nullptr: size only)
struct Carver {
  char *p;
  size_t used = 0;
  template <typename T>
  T *take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T *r = p ? reinterpret_cast<T *>(p + used) : nullptr;
    used += bytes;
    return r;
  }
};

// Private stream used only to record graphs (capture executes nothing); the
// recorded graph is then launched on the caller's stream.  One per host thread.
tomo_status capture_stream(cudaStream_t *out) {
  thread_local cudaStream_t s = nullptr;
  thread_local int dev = -1;
  int cur = 0;
  TOMO_CUDA(cudaGetDevice(&cur));
  if (!s || dev != cur) {
    TOMO_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    dev = cur;
  }
  *out = s;
  return TOMO_OK;
}

// RAII for library-allocated workspaces (stream-ordered)
struct WsHolder {
  void *p = nullptr;
  cudaStream_t st = nullptr;
  ~WsHolder() {
    if (p) cudaFreeAsync(p, st);
  }
};

// Optional per-launch timing: an event pair around every kernel, summed per
// kind into the caller's tomo_timing when the call finishes.
enum Kind { kA = 0, kAT = 1, kOther = 2 };
struct Timer {
  tomo_timing *t = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kinds;
  void begin(cudaStream_t s) {
    if (!t) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.push_back(e);
  }
  void end(cudaStream_t s, int kind) {
    if (!t) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.push_back(e);
    kinds.push_back(kind);
  }
  tomo_status finish(cudaStream_t s) {
    if (!t) return TOMO_OK;
    TOMO_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < kinds.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      t->ms[kinds[i]] += ms;
      t->launches[kinds[i]] += 1;
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    kinds.clear();
    return TOMO_OK;
  }
};

#define TIMED(tm, st, kind, ...) \
  do {                           \
    (tm).begin(st);              \
    __VA_ARGS__;                 \
    (tm).end(st, kind);          \
  } while (0)

Op make_op(const tomo_matrix *h, bool trans, const Exec &ex) {
  Op op;
  op.m = trans ? &h->AT : &h->A;
  op.sell = trans ? &h->sAT : &h->sA;
  op.lp = trans ? &h->lpAT : &h->lpA;
  op.format = ex.format;
  op.trans = trans;
  op.bf16 = h->lp_dtype == TOMO_BF16;
  op.scale = h->ang_scale;
  op.np = h->np;
  op.nx = h->nx;
  op.ny = h->ny;
  op.order = ex.order;
  op.blocks = ex.blocks;
  op.nt = h->nt;
  if (!trans && ex.format == TOMO_FMT_SELL16 && !h->lpAb.empty()) op.bands = &h->lpAb;
  if (trans && ex.format == TOMO_FMT_SELL16 && h->lpATt.ent && (ex.order == 0 || ex.order == 3)) {
    op.tl = &h->lpATt;
    prepare_tile16();
  }
  return op;
}

// ---------------------------------------------------------------------------
// project / backproject
// ---------------------------------------------------------------------------
template <int B>
tomo_status project_t(const tomo_matrix *h, bool trans, const float *in, float *out, int32_t nz, int layout,
                      const Exec &ex, void *ws, cudaStream_t st) {
  Op op = make_op(h, trans, ex);
  Timer tm{ex.timing};
  const int kind = trans ? kAT : kA;
  const int64_t nin = op.m->cols, nout = op.m->rows;
  Carver cv{(char *)ws};
  float *xi = B > 1 ? cv.take<float>(nin * B) : nullptr;
  float *yi = B > 1 ? cv.take<float>(nout * B) : nullptr;
  if (op.bands) op.partial = cv.take<float>(nout * B);  // sums of the column bands
  if (layout == TOMO_INTERLEAVED || B == 1) {
    // interleaved with n_z == B (or a single slice per pass): operate in place
    for (int32_t s0 = 0; s0 < nz; s0 += B)
      TIMED(tm, st, kind,
            launch_spmm<B>(op, in + (int64_t)s0 * nin, EpiStore{out + (int64_t)s0 * nout, B}, nullptr, st));
    TOMO_CUDA(cudaGetLastError());
    return tm.finish(st);
  }
  // the 16-bit A^T pass gathers an operand scaled by 1/a(theta) per row (its own copy here)
  op.pre = trans && op.format == TOMO_FMT_SELL16;
  for (int32_t s0 = 0; s0 < nz; s0 += B) {
    int cnt = std::min<int32_t>(B, nz - s0);
    TIMED(tm, st, kOther, interleave<B>(in + (int64_t)s0 * nin, nin, cnt, xi, st));
    if (op.pre)
      TIMED(tm, st, kOther,
            (k_scale_rows<B><<<elem_grid(nin * B), kThreads, 0, st>>>(xi, xi, nin, h->ang_scale, h->np)));
    TIMED(tm, st, kind, launch_spmm<B>(op, xi, EpiStore{yi, B}, nullptr, st));
    TIMED(tm, st, kOther, deinterleave<B>(yi, nout, cnt, out + (int64_t)s0 * nout, st));
  }
  TOMO_CUDA(cudaGetLastError());
  return tm.finish(st);
}

// ---------------------------------------------------------------------------
// SIRT
// ---------------------------------------------------------------------------
template <int B>
tomo_status sirt_t(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters, float lam,
                   const Exec &ex, void *ws, cudaStream_t st) {
  Op A = make_op(h, false, ex), AT = make_op(h, true, ex);
  // 16-bit values: the residual is written times 1/a(theta), so A^T needs no per-entry scale
  AT.pre = ex.format == TOMO_FMT_SELL16;
  const float *rscale = AT.pre ? h->ang_scale : nullptr;
  const int64_t rows = h->A.rows, cols = h->A.cols;
  Carver cv{(char *)ws};
  float *r = cv.take<float>(rows * B);
  float *bi = B > 1 ? cv.take<float>(rows * B) : nullptr;
  float *xi = B > 1 ? cv.take<float>(cols * B) : nullptr;
  if (A.bands) A.partial = cv.take<float>(rows * B);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TOMO_CUDA(cudaStreamIsCapturing(st, &cs));
  Timer tm{ex.timing};
  const bool use_graph = ex.graph && !ex.timing && cs == cudaStreamCaptureStatusNone && iters > 1;
  cudaStream_t cap = nullptr;
  for (int32_t s0 = 0; s0 < nz; s0 += B) {
    int cnt = std::min<int32_t>(B, nz - s0);
    const float *bb = sino + (int64_t)s0 * rows;
    float *xx = x + (int64_t)s0 * cols;
    if (B > 1) {
      TIMED(tm, st, kOther, interleave<B>(bb, rows, cnt, bi, st));
      TIMED(tm, st, kOther, interleave<B>(xx, cols, cnt, xi, st));
      bb = bi;
      xx = xi;
    }
    auto one_iter = [&](cudaStream_t s) {
      if (rscale)
        TIMED(tm, s, kA, launch_spmm<B>(A, xx, EpiSirtResidualScaled{r, bb, h->R, B, rscale, h->np}, nullptr, s));
      else
        TIMED(tm, s, kA, launch_spmm<B>(A, xx, EpiSirtResidual{r, bb, h->R, B}, nullptr, s));
      TIMED(tm, s, kAT, launch_spmm<B>(AT, r, EpiSirtUpdate{xx, h->C, lam, B}, nullptr, s));
    };
    if (use_graph) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      TOMO_TRY(capture_stream(&cap));
      TOMO_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      one_iter(cap);
      TOMO_CUDA(cudaStreamEndCapture(cap, &graph));
      TOMO_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      for (int32_t it = 0; it < iters; ++it) TOMO_CUDA(cudaGraphLaunch(exec, st));
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
    } else {
      for (int32_t it = 0; it < iters; ++it) one_iter(st);
    }
    if (B > 1) TIMED(tm, st, kOther, deinterleave<B>(xi, cols, cnt, x + (int64_t)s0 * cols, st));
  }
  TOMO_CUDA(cudaGetLastError());
  return tm.finish(st);
}

// ---------------------------------------------------------------------------
// CGLS
// ---------------------------------------------------------------------------
template <int B>
tomo_status cgls_t(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                   int32_t recompute, double *hist, const tomo_cgls_state *sin, tomo_cgls_state *sout,
                   const Exec &ex, void *ws, cudaStream_t st) {
  Op A = make_op(h, false, ex), AT = make_op(h, true, ex);
  const int64_t rows = h->A.rows, cols = h->A.cols;
  const int pg = max_spmm_grid();
  Carver cv{(char *)ws};
  float *r = cv.take<float>(rows * B);
  float *q = cv.take<float>(rows * B);
  float *p = cv.take<float>(cols * B);
  float *s = cv.take<float>(cols * B);
  double *part_a = cv.take<double>((size_t)pg * B);
  double *part_b = cv.take<double>((size_t)pg * B);
  double *part_r = cv.take<double>((size_t)pg * B);
  double *scal = cv.take<double>(B * 8);
  int *itc = cv.take<int>(4);
  float *bi = B > 1 ? cv.take<float>(rows * B) : nullptr;
  float *xi = B > 1 ? cv.take<float>(cols * B) : nullptr;
  // 16-bit values: A^T gathers rs = r times 1/a(theta) (written beside r), not r
  AT.pre = ex.format == TOMO_FMT_SELL16;
  float *rs = AT.pre ? cv.take<float>(rows * B) : r;
  const float *rsc = AT.pre ? h->ang_scale : nullptr;
  if (A.bands) A.partial = cv.take<float>(rows * B);

  // the periodic residual r = b - A x: the solve's own values, or the FP32 ones
  Op Arec = A;
  if (ex.recompute_fp32 && ex.format == TOMO_FMT_SELL16) {
    Exec e32 = ex;
    e32.format = h->sA.ent ? TOMO_FMT_SELL : TOMO_FMT_CSR;
    Arec = make_op(h, false, e32);
  } else {
    Arec.partial = A.partial;
  }
  const int gA = spmm_grid_of<B, EpiStoreNorm>(A);        // q = A p
  const int gR = AT.pre ? spmm_grid_of<B, EpiResidualNormScaled>(Arec)   // r = b - A x
                        : spmm_grid_of<B, EpiResidualNorm>(Arec);
  const int gT = spmm_grid_of<B, EpiStoreNorm>(AT);    // s = A^T r
  constexpr int PER = B >= 4 ? B / 4 : 1;
  const int ge = elem_grid((rows > cols ? rows : cols) * PER);

  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TOMO_CUDA(cudaStreamIsCapturing(st, &cs));
  Timer tm{ex.timing};
  const bool use_graph = ex.graph && !ex.timing && cs == cudaStreamCaptureStatusNone && iters > 1;
  cudaStream_t cap = nullptr;

  for (int32_t s0 = 0; s0 < nz; s0 += B) {
    int cnt = std::min<int32_t>(B, nz - s0);
    const float *bb = sino + (int64_t)s0 * rows;
    float *xx = x + (int64_t)s0 * cols;
    if (B > 1) {
      TIMED(tm, st, kOther, interleave<B>(bb, rows, cnt, bi, st));
      bb = bi;
      xx = xi;
    }
    if (sin) {
      // resume: x, r, p, gamma and the frozen flags from the caller's state
      if (B > 1) {
        TIMED(tm, st, kOther, interleave<B>(x + (int64_t)s0 * cols, cols, cnt, xi, st));
        TIMED(tm, st, kOther, interleave<B>(sin->r + (int64_t)s0 * rows, rows, cnt, r, st));
        TIMED(tm, st, kOther, interleave<B>(sin->p + (int64_t)s0 * cols, cols, cnt, p, st));
      } else {
        TOMO_CUDA(cudaMemcpyAsync(r, sin->r + (int64_t)s0 * rows, sizeof(float) * rows, cudaMemcpyDeviceToDevice, st));
        TOMO_CUDA(cudaMemcpyAsync(p, sin->p + (int64_t)s0 * cols, sizeof(float) * cols, cudaMemcpyDeviceToDevice, st));
      }
      TIMED(tm, st, kOther, (k_cgls_load<<<1, 64, 0, st>>>(scal, sin->gamma + s0, sin->frozen + s0, cnt, B, itc)));
    } else {
      // x = 0, r = b, s = A^T r, p = s, gamma = ||s||^2
      TOMO_CUDA(cudaMemsetAsync(xx, 0, sizeof(float) * cols * B, st));
      TOMO_CUDA(cudaMemcpyAsync(r, bb, sizeof(float) * rows * B, cudaMemcpyDeviceToDevice, st));
      if (AT.pre)
        TIMED(tm, st, kOther, (k_scale_rows<B><<<elem_grid(rows * B), kThreads, 0, st>>>(r, rs, rows, rsc, h->np)));
      TIMED(tm, st, kAT, launch_spmm<B>(AT, rs, EpiStoreNorm{s, B}, part_b, st));
      TOMO_CUDA(cudaMemcpyAsync(p, s, sizeof(float) * cols * B, cudaMemcpyDeviceToDevice, st));
      TIMED(tm, st, kOther, (k_cgls_init<<<B, kThreads, 0, st>>>(part_b, gT, B, scal, itc)));
    }
    TOMO_CUDA(cudaGetLastError());

    // the residual-norm partials come from the residual SpMM grid (gR blocks)
    // on a recompute iteration and from the elementwise grid (ge blocks) otherwise
    auto one_iter = [&](cudaStream_t sm, bool recomp) {
      // q = A p, ||q||^2
      TIMED(tm, sm, kA, launch_spmm<B>(A, p, EpiStoreNorm{q, B}, part_a, sm));
      // alpha = gamma / ||q||^2
      TIMED(tm, sm, kOther, (k_cgls_alpha<<<B, kThreads, 0, sm>>>(part_a, gA, B, scal)));
      // x += alpha p, r -= alpha q
      TIMED(tm, sm, kOther,
            (k_cgls_step<B><<<ge, kThreads, 0, sm>>>(xx, p, cols, r, q, rows, scal, hist ? part_r : nullptr,
                                                     AT.pre && !recomp ? rs : nullptr, rsc, h->np)));
      // every `recompute` iterations: r = b - A x
      if (recomp && AT.pre)
        TIMED(tm, sm, kA, launch_spmm<B>(Arec, xx, EpiResidualNormScaled{r, bb, B, rs, rsc, h->np}, part_r, sm));
      else if (recomp)
        TIMED(tm, sm, kA, launch_spmm<B>(Arec, xx, EpiResidualNorm{r, bb, B}, part_r, sm));
      // s = A^T r, ||s||^2
      TIMED(tm, sm, kAT, launch_spmm<B>(AT, rs, EpiStoreNorm{s, B}, part_b, sm));
      // beta = ||s||^2 / gamma, residual history
      TIMED(tm, sm, kOther,
            (k_cgls_beta<<<B, kThreads, 0, sm>>>(part_b, gT, hist ? part_r : nullptr, recomp ? gR : ge, B, scal,
                                                 hist, itc, s0, cnt, nz)));
      // p = s + beta p
      TIMED(tm, sm, kOther, (k_cgls_dir<B><<<ge, kThreads, 0, sm>>>(p, s, cols, scal, itc)));
    };
    if (use_graph) {
      TOMO_TRY(capture_stream(&cap));
      cudaGraph_t g0 = nullptr, g1 = nullptr;
      cudaGraphExec_t e0 = nullptr, e1 = nullptr;
      TOMO_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      one_iter(cap, false);
      TOMO_CUDA(cudaStreamEndCapture(cap, &g0));
      TOMO_CUDA(cudaGraphInstantiate(&e0, g0, 0));
      if (recompute > 0) {
        TOMO_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        one_iter(cap, true);
        TOMO_CUDA(cudaStreamEndCapture(cap, &g1));
        TOMO_CUDA(cudaGraphInstantiate(&e1, g1, 0));
      }
      for (int32_t it = 0; it < iters; ++it) {
        bool rc = recompute > 0 && (it + 1) % recompute == 0;
        TOMO_CUDA(cudaGraphLaunch(rc ? e1 : e0, st));
      }
      cudaGraphExecDestroy(e0);
      cudaGraphDestroy(g0);
      if (e1) cudaGraphExecDestroy(e1);
      if (g1) cudaGraphDestroy(g1);
    } else {
      for (int32_t it = 0; it < iters; ++it) one_iter(st, recompute > 0 && (it + 1) % recompute == 0);
    }
    if (sout) {
      if (B > 1) {
        TIMED(tm, st, kOther, deinterleave<B>(r, rows, cnt, sout->r + (int64_t)s0 * rows, st));
        TIMED(tm, st, kOther, deinterleave<B>(p, cols, cnt, sout->p + (int64_t)s0 * cols, st));
      } else {
        TOMO_CUDA(cudaMemcpyAsync(sout->r + (int64_t)s0 * rows, r, sizeof(float) * rows, cudaMemcpyDeviceToDevice, st));
        TOMO_CUDA(cudaMemcpyAsync(sout->p + (int64_t)s0 * cols, p, sizeof(float) * cols, cudaMemcpyDeviceToDevice, st));
      }
      TIMED(tm, st, kOther, (k_cgls_save<<<1, 64, 0, st>>>(scal, sout->gamma + s0, sout->frozen + s0, cnt)));
    }
    if (B > 1) TIMED(tm, st, kOther, deinterleave<B>(xi, cols, cnt, x + (int64_t)s0 * cols, st));
  }
  TOMO_CUDA(cudaGetLastError());
  return tm.finish(st);
}

// ---------------------------------------------------------------------------
// BB-step SIRT driver.  One iteration: r = b - A x (+||r||^2), rf = P^T P r,
// g = A^T rf, the two dots, alpha, x += alpha g.  g and g_prev alternate
// between two buffers, so the iteration is captured as two graphs (even and
// odd) and replayed alternately.
// ---------------------------------------------------------------------------
template <int B>
tomo_status bb_t(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters, double first_step,
                 double *hist, const tomo_bb_state *sin, tomo_bb_state *sout, const Exec &ex, void *ws,
                 cudaStream_t st) {
  Op A = make_op(h, false, ex), AT = make_op(h, true, ex);
  AT.pre = ex.format == TOMO_FMT_SELL16;  // the filter writes P^T P r times 1/a(theta)
  const int64_t rows = h->A.rows, cols = h->A.cols;
  const int pg = max_spmm_grid();
  Carver cv{(char *)ws};
  float *r = cv.take<float>(rows * B);
  float *rf = cv.take<float>(rows * B);
  float *gb[2] = {cv.take<float>(cols * B), cv.take<float>(cols * B)};
  double *part_r = cv.take<double>((size_t)pg * B);
  double *part_p = cv.take<double>((size_t)pg * B);
  double *part_q = cv.take<double>((size_t)pg * B);
  double *scal = cv.take<double>(B * 4);
  int *itc = cv.take<int>(4);
  float *bi = B > 1 ? cv.take<float>(rows * B) : nullptr;
  float *xi = B > 1 ? cv.take<float>(cols * B) : nullptr;
  if (A.bands) A.partial = cv.take<float>(rows * B);

  const int gR = spmm_grid_of<B, EpiResidualNorm>(A);
  constexpr int PER = B >= 4 ? B / 4 : 1;
  constexpr int TK = ramp_tile_bins<B>();
  const int ge = elem_grid(cols * PER);
  const dim3 gf((unsigned)((h->np + TK - 1) / TK), (unsigned)h->nt);
  const double a0 = first_step > 0.0 ? first_step : 3.141592653589793 / (double)h->nt;

  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TOMO_CUDA(cudaStreamIsCapturing(st, &cs));
  Timer tm{ex.timing};
  const bool use_graph = ex.graph && !ex.timing && cs == cudaStreamCaptureStatusNone && iters > 2;
  cudaStream_t cap = nullptr;

  for (int32_t s0 = 0; s0 < nz; s0 += B) {
    const int cnt = std::min<int32_t>(B, nz - s0);
    const float *bb = sino + (int64_t)s0 * rows;
    float *xx = x + (int64_t)s0 * cols;
    if (B > 1) {
      TIMED(tm, st, kOther, interleave<B>(bb, rows, cnt, bi, st));
      TIMED(tm, st, kOther, interleave<B>(xx, cols, cnt, xi, st));
      bb = bi;
      xx = xi;
    }
    // the previous step's g (resume) sits in gb[1], the buffer iteration 0 reads
    if (sin) {
      if (B > 1) {
        TIMED(tm, st, kOther, interleave<B>(sin->g + (int64_t)s0 * cols, cols, cnt, gb[1], st));
      } else {
        TOMO_CUDA(cudaMemcpyAsync(gb[1], sin->g + (int64_t)s0 * cols, sizeof(float) * cols,
                                  cudaMemcpyDeviceToDevice, st));
      }
    } else {
      TOMO_CUDA(cudaMemsetAsync(gb[1], 0, sizeof(float) * cols * B, st));
    }
    TIMED(tm, st, kOther,
          (k_bb_load<<<1, 64, 0, st>>>(scal, sin ? sin->alpha + s0 : nullptr, sin ? sin->frozen + s0 : nullptr,
                                       cnt, B, itc)));
    TOMO_CUDA(cudaGetLastError());

    auto one_iter = [&](cudaStream_t sm, float *g, float *gp) {
      // the residual norm is only reduced when its history is asked for
      if (hist)
        TIMED(tm, sm, kA, launch_spmm<B>(A, xx, EpiResidualNorm{r, bb, B}, part_r, sm));
      else
        TIMED(tm, sm, kA, launch_spmm<B>(A, xx, EpiResidual{r, bb, B}, nullptr, sm));
      TIMED(tm, sm, kOther,
            (k_ramp_filter<B><<<gf, kThreads, 0, sm>>>(r, rf, h->ramp, h->np, AT.pre ? h->ang_scale : nullptr)));
      TIMED(tm, sm, kAT, launch_spmm<B>(AT, rf, EpiStore{g, B}, nullptr, sm));
      TIMED(tm, sm, kOther, (k_bb_dots<B><<<ge, kThreads, 0, sm>>>(gp, g, cols, part_p, part_q)));
      TIMED(tm, sm, kOther,
            (k_bb_alpha<<<B, kThreads, 0, sm>>>(part_p, part_q, ge, hist ? part_r : nullptr, gR, B, scal, a0, hist,
                                                itc, s0, cnt, nz)));
      TIMED(tm, sm, kOther, (k_bb_update<B><<<ge, kThreads, 0, sm>>>(xx, g, cols, scal, itc)));
    };
    if (use_graph) {
      TOMO_TRY(capture_stream(&cap));
      cudaGraph_t gr[2] = {nullptr, nullptr};
      cudaGraphExec_t ge2[2] = {nullptr, nullptr};
      for (int k = 0; k < 2; ++k) {
        TOMO_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        one_iter(cap, gb[k], gb[1 - k]);
        TOMO_CUDA(cudaStreamEndCapture(cap, &gr[k]));
        TOMO_CUDA(cudaGraphInstantiate(&ge2[k], gr[k], 0));
      }
      for (int32_t it = 0; it < iters; ++it) TOMO_CUDA(cudaGraphLaunch(ge2[it & 1], st));
      for (int k = 0; k < 2; ++k) {
        cudaGraphExecDestroy(ge2[k]);
        cudaGraphDestroy(gr[k]);
      }
    } else {
      for (int32_t it = 0; it < iters; ++it) one_iter(st, gb[it & 1], gb[1 - (it & 1)]);
    }
    if (sout) {
      const float *last = gb[iters > 0 ? (iters - 1) & 1 : 1];
      if (B > 1) {
        TIMED(tm, st, kOther, deinterleave<B>(last, cols, cnt, sout->g + (int64_t)s0 * cols, st));
      } else {
        TOMO_CUDA(cudaMemcpyAsync(sout->g + (int64_t)s0 * cols, last, sizeof(float) * cols,
                                  cudaMemcpyDeviceToDevice, st));
      }
      TIMED(tm, st, kOther, (k_bb_save<<<1, 64, 0, st>>>(scal, sout->alpha + s0, sout->frozen + s0, cnt)));
    }
    if (B > 1) TIMED(tm, st, kOther, deinterleave<B>(xi, cols, cnt, x + (int64_t)s0 * cols, st));
  }
  TOMO_CUDA(cudaGetLastError());
  return tm.finish(st);
}

template <template <int> class F, typename... Args>
tomo_status dispatch(int B, Args &&...args) {
  switch (B) {
    case 1: return F<1>::run(args...);
    case 2: return F<2>::run(args...);
    case 4: return F<4>::run(args...);
    case 8: return F<8>::run(args...);
    case 16: return F<16>::run(args...);
    case 32: return F<32>::run(args...);
    case 64: return F<64>::run(args...);
    default: return fail(TOMO_ERR_UNSUPPORTED, "batch width must be 1, 2, 4, 8, 16, 32 or 64");
  }
}

template <int B>
struct ProjectF {
  template <typename... A>
  static tomo_status run(A &&...a) { return project_t<B>(a...); }
};
template <int B>
struct SirtF {
  template <typename... A>
  static tomo_status run(A &&...a) { return sirt_t<B>(a...); }
};
template <int B>
struct CglsF {
  template <typename... A>
  static tomo_status run(A &&...a) { return cgls_t<B>(a...); }
};
template <int B>
struct BbF {
  template <typename... A>
  static tomo_status run(A &&...a) { return bb_t<B>(a...); }
};

bool valid_width(int b) { return b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32 || b == 64; }

tomo_status with_ws(const tomo_matrix *h, int op, int32_t nz, const Exec &ex, void *&ws, WsHolder &hold,
                    cudaStream_t st) {
  size_t need = workspace_bytes(h, op, nz, ex);
  if (ws || need == 0) return TOMO_OK;
  cudaError_t e = cudaMallocAsync(&hold.p, need, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TOMO_ERR_OOM, "workspace allocation of " + std::to_string(need) + " bytes failed");
  }
  hold.st = st;
  ws = hold.p;
  return TOMO_OK;
}

}  // namespace

tomo_status resolve_exec(const tomo_matrix *h, const tomo_exec_opts *o, int32_t nz, Exec *ex) {
  Exec e;
  const tomo_matrix::Tuned *tc = nullptr;  // tomo_autotune's choice for this slice count
  for (const auto &t : h->tuned)
    if (t.nz == nz) {
      tc = &t;
      break;
    }
  const bool tuned = tc != nullptr;
  int req = o ? o->batch_width : 0;
  if (req != 0 && !valid_width(req))
    return fail(TOMO_ERR_UNSUPPORTED, "batch_width must be 0, 1, 2, 4, 8, 16, 32 or 64");
  if (req == 0) {
    if (tuned) {
      req = tc->B;
    } else {
      int b = 1;
      while (b < nz && b < 16) b <<= 1;
      req = b;
    }
  }
  e.B = req;
  e.graph = o ? o->use_graph != 0 : true;
  e.timing = o ? o->timing : nullptr;
  e.format = o ? o->format : TOMO_FMT_SELL;
  if (e.format == TOMO_FMT_AUTO) e.format = tuned ? tc->fmt : TOMO_FMT_SELL;
  if (e.format != TOMO_FMT_SELL && e.format != TOMO_FMT_SELL16 && e.format != TOMO_FMT_CSR)
    return fail(TOMO_ERR_INVALID_ARG, "format must be a tomo_format value");
  if (e.format == TOMO_FMT_SELL16 && h->lp_dtype == TOMO_F32)
    return fail(TOMO_ERR_UNSUPPORTED, "matrix was built without 16-bit values");
  if (e.format == TOMO_FMT_SELL && !h->sA.ent)
    return fail(TOMO_ERR_UNSUPPORTED, "matrix was built without the FP32 SELL form (no_fp32_sell)");
  if (e.format == TOMO_FMT_CSR && !h->A.ci)
    return fail(TOMO_ERR_UNSUPPORTED, "matrix was built with drop_csr");
  e.recompute_fp32 = o ? o->recompute_fp32 != 0 : false;
  e.order = o ? o->order : 0;
  if (e.order < 0 || e.order > 3) return fail(TOMO_ERR_INVALID_ARG, "order must be 0, 1, 2 or 3");
  if (e.order == 0 && tuned) e.order = tc->order;
  e.blocks = o ? o->blocks_per_sm : 0;
  if (e.blocks < 0) return fail(TOMO_ERR_INVALID_ARG, "blocks_per_sm must be >= 0");
  if (e.blocks == 0 && tuned) e.blocks = tc->blocks;
  if (e.recompute_fp32 && !h->sA.ent && !h->A.ci)
    return fail(TOMO_ERR_UNSUPPORTED, "recompute_fp32 needs an FP32 form of A (FP32 SELL or CSR)");
  *ex = e;
  return TOMO_OK;
}

size_t workspace_bytes(const tomo_matrix *h, int op, int32_t nz, const Exec &ex) {
  (void)nz;
  const int64_t rows = h->A.rows, cols = h->A.cols;
  const int B = ex.B;
  // the 16-bit A stored as column bands sums its bands in a (rows, B) buffer
  const bool banded = ex.format == TOMO_FMT_SELL16 && !h->lpAb.empty();
  Carver cv{nullptr};
  switch (op) {
    case TOMO_OP_PROJECT:
    case TOMO_OP_BACKPROJECT:
      if (B > 1) {
        cv.take<float>(cols * B);
        cv.take<float>(rows * B);
      }
      if (banded && op == TOMO_OP_PROJECT) cv.take<float>(rows * B);
      break;
    case TOMO_OP_SIRT:
      cv.take<float>(rows * B);
      if (B > 1) {
        cv.take<float>(rows * B);
        cv.take<float>(cols * B);
      }
      if (banded) cv.take<float>(rows * B);
      break;
    case TOMO_OP_CGLS: {
      const int pg = max_spmm_grid();
      cv.take<float>(rows * B);
      cv.take<float>(rows * B);
      cv.take<float>(cols * B);
      cv.take<float>(cols * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>(B * 8);
      cv.take<int>(4);
      if (B > 1) {
        cv.take<float>(rows * B);
        cv.take<float>(cols * B);
      }
      if (ex.format == TOMO_FMT_SELL16) cv.take<float>(rows * B);  // r times 1/a(theta)
      if (banded) cv.take<float>(rows * B);
      break;
    }
    case TOMO_OP_SIRT_BB: {
      const int pg = max_spmm_grid();
      cv.take<float>(rows * B);
      cv.take<float>(rows * B);
      cv.take<float>(cols * B);
      cv.take<float>(cols * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>((size_t)pg * B);
      cv.take<double>(B * 4);
      cv.take<int>(4);
      if (B > 1) {
        cv.take<float>(rows * B);
        cv.take<float>(cols * B);
      }
      if (banded) cv.take<float>(rows * B);
      break;
    }
    default:
      return 0;
  }
  return cv.used;
}

tomo_status run_project(const tomo_matrix *h, bool transpose, const float *in, float *out, int32_t nz,
                        int layout, const Exec &ex, void *ws, cudaStream_t st) {
  WsHolder hold;
  TOMO_TRY(with_ws(h, transpose ? TOMO_OP_BACKPROJECT : TOMO_OP_PROJECT, nz, ex, ws, hold, st));
  return dispatch<ProjectF>(ex.B, h, transpose, in, out, nz, layout, ex, ws, st);
}

tomo_status run_sirt(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     float lambda, const Exec &ex, void *ws, cudaStream_t st) {
  WsHolder hold;
  TOMO_TRY(with_ws(h, TOMO_OP_SIRT, nz, ex, ws, hold, st));
  return dispatch<SirtF>(ex.B, h, sino, x, nz, iters, lambda, ex, ws, st);
}

tomo_status run_cgls(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     int32_t recompute, double *hist, const tomo_cgls_state *in, tomo_cgls_state *out,
                     const Exec &ex, void *ws, cudaStream_t st) {
  WsHolder hold;
  TOMO_TRY(with_ws(h, TOMO_OP_CGLS, nz, ex, ws, hold, st));
  return dispatch<CglsF>(ex.B, h, sino, x, nz, iters, recompute, hist, in, out, ex, ws, st);
}

int residual_parts() { return num_sms() * kResidBlocksPerSm; }

tomo_status run_residual_norm(const tomo_matrix *h, const float *sino, const float *x, int32_t nz, double *norms,
                              void *ws, cudaStream_t st) {
  const Csr &A = h->A;
  const int nb = residual_parts();
  double *part = static_cast<double *>(ws);
  WsHolder hold;
  if (!part) {
    if (cudaMallocAsync(&hold.p, sizeof(double) * nb, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(TOMO_ERR_OOM, "workspace allocation failed");
    }
    hold.st = st;
    part = static_cast<double *>(hold.p);
  }
  for (int32_t s = 0; s < nz; ++s) {
    k_resid_f64<<<nb, kThreads, 0, st>>>(A.rp, A.ci, A.v, A.rows, x + (int64_t)s * A.cols,
                                         sino + (int64_t)s * A.rows, part);
    k_sum_parts<<<1, 32, 0, st>>>(part, nb, norms + s);
  }
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

// Y = M X for an interleaved (rows, B) operand with the FP32 CSR kernels (the
// Fubini-Radon gridding matrices use it).
tomo_status spmm_csr_store(const Csr &M, int B, const float *X, float *Y, cudaStream_t st) {
  Op op{};
  op.m = &M;
  op.format = TOMO_FMT_CSR;
  switch (B) {
    case 1: launch_spmm<1>(op, X, EpiStore{Y, 1}, nullptr, st); break;
    case 2: launch_spmm<2>(op, X, EpiStore{Y, 2}, nullptr, st); break;
    case 4: launch_spmm<4>(op, X, EpiStore{Y, 4}, nullptr, st); break;
    case 8: launch_spmm<8>(op, X, EpiStore{Y, 8}, nullptr, st); break;
    case 16: launch_spmm<16>(op, X, EpiStore{Y, 16}, nullptr, st); break;
    case 32: launch_spmm<32>(op, X, EpiStore{Y, 32}, nullptr, st); break;
    case 64: launch_spmm<64>(op, X, EpiStore{Y, 64}, nullptr, st); break;
    default: return fail(TOMO_ERR_UNSUPPORTED, "SpMM width must be a power of two up to 64");
  }
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status run_sirt_bb(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                        double first_step, double *hist, const tomo_bb_state *in, tomo_bb_state *out,
                        const Exec &ex, void *ws, cudaStream_t st) {
  WsHolder hold;
  TOMO_TRY(with_ws(h, TOMO_OP_SIRT_BB, nz, ex, ws, hold, st));
  return dispatch<BbF>(ex.B, h, sino, x, nz, iters, first_step, hist, in, out, ex, ws, st);
}

// ---------------------------------------------------------------------------
// autotuner: time one SIRT iteration pair per (format, width) candidate
// ---------------------------------------------------------------------------
namespace {

template <int B>
tomo_status time_sirt_pair(const tomo_matrix *h, int format, int order, int blocks, float *x, float *r, float *b,
                           float *partial, cudaStream_t st, double *ms_out) {
  Exec ex;
  ex.B = B;
  ex.format = format;
  ex.order = order;
  ex.blocks = blocks;
  Op A = make_op(h, false, ex), AT = make_op(h, true, ex);
  A.partial = partial;
  AT.pre = format == TOMO_FMT_SELL16;
  const float *rscale = AT.pre ? h->ang_scale : nullptr;
  auto pair = [&]() {
    if (rscale)
      launch_spmm<B>(A, x, EpiSirtResidualScaled{r, b, h->R, B, rscale, h->np}, nullptr, st);
    else
      launch_spmm<B>(A, x, EpiSirtResidual{r, b, h->R, B}, nullptr, st);
    launch_spmm<B>(AT, r, EpiSirtUpdate{x, h->C, 0.0f, B}, nullptr, st);
  };
  for (int i = 0; i < 2; ++i) pair();
  cudaEvent_t e0, e1;
  TOMO_CUDA(cudaEventCreate(&e0));
  TOMO_CUDA(cudaEventCreate(&e1));
  const int reps = 5;
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps; ++i) pair();
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TOMO_CUDA(err);
  TOMO_CUDA(cudaGetLastError());
  *ms_out = ms / reps;
  return TOMO_OK;
}

// blocks per SM that the SIRT A pass of (B, format) fits (the autotuner's stage 2 starts below it)
template <int B>
int resident_of(const tomo_matrix *h, const Exec &ex) {
  const Op A = make_op(h, false, ex);
  const int G = rows_per_warp(ex.format, B);
  const int grid = spmm_grid_of<B, EpiSirtResidual>(A);
  const int64_t groups = (A.m->rows + G - 1) / G;
  const int64_t full = (groups + kWarps - 1) / kWarps;
  if (grid < full) return std::max(1, grid / num_sms());
  return std::max(1, (int)((full + num_sms() - 1) / num_sms()));
}

template <int B>
struct TimeF {
  template <typename... A>
  static tomo_status run(A &&...a) { return time_sirt_pair<B>(a...); }
};

}  // namespace

tomo_status run_autotune(tomo_matrix *h, int32_t nz, int allow16, tomo_exec_opts *best, double *rate,
                         tomo_tune_entry *table, int32_t cap, int32_t *n_table, cudaStream_t st) {
  int bmax = 1;
  while (bmax < nz && bmax < 64) bmax <<= 1;
  const bool lp16 = allow16 != 0 && h->lp_dtype != TOMO_F32;
  std::vector<int> fmts;
  if (allow16 != 2) {
    if (h->sA.ent) fmts.push_back(TOMO_FMT_SELL);
    if (h->A.ci) fmts.push_back(TOMO_FMT_CSR);
  }
  if (lp16) fmts.push_back(TOMO_FMT_SELL16);
  if (fmts.empty())
    return fail(TOMO_ERR_UNSUPPORTED, allow16 == 2 ? "matrix was built without 16-bit values"
                                                   : "no FP32 form to tune (built with no_fp32_sell and drop_csr)");
  const int64_t rows = h->A.rows, cols = h->A.cols;
  float *x = nullptr, *r = nullptr, *b = nullptr, *partial = nullptr;
  struct Free {
    float **p[4];
    ~Free() {
      for (auto q : p)
        if (*q) cudaFree(*q);
    }
  } guard{{&x, &r, &b, &partial}};
  TOMO_CUDA(cudaMalloc(&x, sizeof(float) * cols * bmax));
  TOMO_CUDA(cudaMalloc(&r, sizeof(float) * rows * bmax));
  TOMO_CUDA(cudaMalloc(&b, sizeof(float) * rows * bmax));
  if (!h->lpAb.empty()) TOMO_CUDA(cudaMalloc(&partial, sizeof(float) * rows * bmax));
  TOMO_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * cols * bmax, st));
  TOMO_CUDA(cudaMemsetAsync(b, 0, sizeof(float) * rows * bmax, st));
  int n = 0;
  double best_rate = -1.0;
  tomo_tune_entry bestc{};
  auto run = [&](int B, int f, int order, int blocks) -> tomo_status {
    double ms = 0.0;
    TOMO_TRY(dispatch<TimeF>(B, h, f, order, blocks, x, r, b, partial, st, &ms));
    const double chunks = (double)((nz + B - 1) / B);
    const double rt = ms > 0 ? nz / (chunks * ms) * 1000.0 : 0.0;
    const tomo_tune_entry ent{B, f, order, blocks, ms, rt};
    if (table && n < cap) table[n] = ent;
    ++n;
    if (rt > best_rate) {
      best_rate = rt;
      bestc = ent;
    }
    return TOMO_OK;
  };
  // stage 1: width x format x A^T order
  for (int f : fmts) {
    for (int B = 1; B <= bmax; B <<= 1) {
      const int G = rows_per_warp(f, B);
      const bool tileable = f != TOMO_FMT_CSR && h->nx % G == 0 && h->ny % 8 == 0;
      TOMO_TRY(run(B, f, 1, 0));
      if (tileable) TOMO_TRY(run(B, f, 2, 0));
      if (f == TOMO_FMT_SELL16 && B == 16 && h->lpATt.ent) TOMO_TRY(run(B, f, 3, 0));
    }
  }
  // stage 2: the best shape with fewer resident blocks per SM
  {
    Exec ex;
    ex.B = bestc.batch_width;
    ex.format = bestc.format;
    int res = 0;
    switch (ex.B) {  // blocks per SM the SIRT A pass of that shape fits
      case 1: res = resident_of<1>(h, ex); break;
      case 2: res = resident_of<2>(h, ex); break;
      case 4: res = resident_of<4>(h, ex); break;
      case 8: res = resident_of<8>(h, ex); break;
      case 16: res = resident_of<16>(h, ex); break;
      case 32: res = resident_of<32>(h, ex); break;
      default: res = resident_of<64>(h, ex); break;
    }
    const tomo_tune_entry s1 = bestc;
    for (int k = 1; k <= 2; ++k)
      if (res - k >= 1) TOMO_TRY(run(s1.batch_width, s1.format, s1.order, res - k));
  }
  if (n_table) *n_table = n;
  if (rate) *rate = best_rate;
  std::memset(best, 0, sizeof(*best));
  best->batch_width = bestc.batch_width;
  best->format = bestc.format;
  best->order = bestc.order;
  best->blocks_per_sm = bestc.blocks_per_sm;
  best->use_graph = 1;
  auto &tl = h->tuned;
  for (size_t k = 0; k < tl.size(); ++k)
    if (tl[k].nz == nz) {
      tl.erase(tl.begin() + k);
      break;
    }
  tl.insert(tl.begin(), tomo_matrix::Tuned{nz, bestc.batch_width, bestc.format, bestc.order, bestc.blocks_per_sm});
  if (tl.size() > 8) tl.pop_back();
  return TOMO_OK;
}

}  // namespace tomo
