// build.cu -- construction of the projector A, its explicit transpose A^T, the
// SIRT normalisers and the 16-bit encoding, all on the device.
//
// Sec. 2 defines the projection as the line integral of u along
// x cos(theta) + y sin(theta) = p; for a piecewise-constant pixel image that
// integral is sum_j u_j * chord(ray, pixel j), which is what A stores.  Sec. 3.1
// builds the entries, drops zero / out-of-range ones and keeps CSR sorted by
// row and column, with the transpose stored separately.  Here both A and A^T
// are generated directly from the geometry by the same FP64 predicate, so A^T
// is the exact transpose of A bit for bit and no sort is needed:
//   * A, row-driven: for ray (m,k) and pixel row iy the hit pixels form one
//     run of consecutive ix (the rounded predicate is monotone in x), so a warp
//     per ray finds each run's ends and writes the columns in ascending order;
//   * A^T, pixel-driven: for pixel (ix,iy) and angle m at most two bins k are
//     hit (three in the strip model), so a warp per pixel tests the candidates
//     of 32 angles at a time and compacts the hits in (m, k) order.
// Two discretisations share the enumeration: the line model (chord lengths)
// and the strip model (the area of the pixel inside the unit-width strip of
// bin k), which differ only in the support half width hs and the weight.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// The weight rules in IEEE FP64 without contraction:
//   t = fl(fl(x cs) + fl(y sn)), delta = |fl(p - t)|, hit iff delta < hs;
//   line:  length = 1/a if delta <= hm else fl(fl(h - delta) / (a e)), hs = h;
//   strip: F(delta + 1/2) - F(delta - 1/2), F odd, F(s) = s (1/a) for s <= hm,
//          hm (1/a) + (s - hm)(h - (s + hm)/2) / (a e) for hm < s < h,
//          1/2 for s >= h (F integrates the chord length), hs = h + 1/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double coord(int i, int n) {
  return __dsub_rn(__dadd_rn((double)i, 0.5), 0.5 * (double)n);  // exact
}

__device__ __forceinline__ double chord_delta(const AngleC &A, double pk, double x, double y) {
  double t = __dadd_rn(__dmul_rn(x, A.cs), __dmul_rn(y, A.sn));
  return fabs(__dsub_rn(pk, t));
}

__device__ __forceinline__ bool chord_hit(const AngleC &A, double pk, double x, double y) {
  return chord_delta(A, pk, x, y) < A.hs;
}

__device__ __forceinline__ double strip_F(const AngleC &A, double s) {
  if (s <= A.hm) return __dmul_rn(s, A.inv_a);
  if (s >= A.h) return 0.5;
  const double ramp = __dmul_rn(__dsub_rn(s, A.hm), __dsub_rn(A.h, __dmul_rn(0.5, __dadd_rn(s, A.hm))));
  return __dadd_rn(__dmul_rn(A.hm, A.inv_a), __ddiv_rn(ramp, A.ae));
}

__device__ __forceinline__ double chord_len(const AngleC &A, int model, double pk, double x, double y) {
  double del = chord_delta(A, pk, x, y);
  if (model == TOMO_MODEL_STRIP) {
    const double dp = __dadd_rn(del, 0.5), dm = __dsub_rn(del, 0.5);
    const double Fp = strip_F(A, dp);
    const double Fm = dm >= 0.0 ? strip_F(A, dm) : -strip_F(A, -dm);
    return __dsub_rn(Fp, Fm);
  }
  return del <= A.hm ? A.inv_a : __ddiv_rn(__dsub_rn(A.h, del), A.ae);
}

// Run [lo, hi] of hit pixels of ray (A, pk) in pixel row y (hi < lo: none).
// A cheap estimate of the run's ends seeds the search; the exact predicate then
// walks to the true ends, so the estimate only has to land near the run.
__device__ void row_run(const AngleC &A, double pk, int nx, double y, int &lo, int &hi) {
  lo = 0;
  hi = -1;
  auto pred = [&](int ix) { return chord_hit(A, pk, coord(ix, nx), y); };
  if (A.cs == 0.0) {
    // x drops out of the predicate: the whole row or nothing
    if (pred(0)) {
      lo = 0;
      hi = nx - 1;
    }
    return;
  }
  double r = pk - y * A.sn;
  double xa = (r - A.hs) * A.inv_cs, xb = (r + A.hs) * A.inv_cs;
  double off = 0.5 * nx - 0.5;
  double xl = fmin(xa, xb) + off, xh = fmax(xa, xb) + off;
  xl = fmin(fmax(xl, -16.0), nx + 16.0);
  xh = fmin(fmax(xh, -16.0), nx + 16.0);
  int s0 = max(0, (int)floor(xl) - 4);
  int s1 = min(nx - 1, (int)ceil(xh) + 4);
  if (s0 > s1) return;
  int a = s0;
  while (a <= s1 && !pred(a)) ++a;
  if (a > s1) return;
  int b = s1;
  while (b > a && !pred(b)) --b;
  while (a > 0 && pred(a - 1)) --a;
  while (b < nx - 1 && pred(b + 1)) ++b;
  lo = a;
  hi = b;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ---------------------------------------------------------------------------
// A: count and fill, one warp per ray
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_count_rays(const AngleC *__restrict__ ang, int nx, int ny,
                                                         int np, int nt, double c,
                                                         int32_t *__restrict__ cnt) {
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= (int64_t)nt * np) return;
  int m = (int)(w / np), k = (int)(w % np);
  AngleC A = ang[m];
  double pk = __dsub_rn(__dadd_rn((double)k, 0.5), c);
  int total = 0;
  for (int iy = lane; iy < ny; iy += 32) {
    int lo, hi;
    row_run(A, pk, nx, coord(iy, ny), lo, hi);
    total += max(0, hi - lo + 1);
  }
  total = warp_sum_i(total);
  if (lane == 0) cnt[w] = total;
}

__global__ void __launch_bounds__(kThreads) k_fill_rays(const AngleC *__restrict__ ang, int model, int nx,
                                                        int ny, int np, int nt, double c,
                                                        const int64_t *__restrict__ rp,
                                                        int32_t *__restrict__ ci, float *__restrict__ v,
                                                        float *__restrict__ R) {
  __shared__ int s_off[kThreads / 32][33];
  __shared__ int s_lo[kThreads / 32][32];
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  if (w >= (int64_t)nt * np) return;
  int m = (int)(w / np), k = (int)(w % np);
  AngleC A = ang[m];
  double pk = __dsub_rn(__dadd_rn((double)k, 0.5), c);
  int64_t pos = rp[w];
  double sum = 0.0;
  for (int iy0 = 0; iy0 < ny; iy0 += 32) {
    int iy = iy0 + lane;
    int lo = 0, hi = -1;
    if (iy < ny) row_run(A, pk, nx, coord(iy, ny), lo, hi);
    int len = max(0, hi - lo + 1);
    int incl = warp_incl_scan(len, lane);
    s_off[wl][lane + 1] = incl;
    if (lane == 0) s_off[wl][0] = 0;
    s_lo[wl][lane] = lo;
    __syncwarp();
    int T = __shfl_sync(0xffffffffu, incl, 31);
    for (int e = lane; e < T; e += 32) {
      int q = 0;  // largest q with s_off[q] <= e
#pragma unroll
      for (int step = 16; step; step >>= 1)
        if (q + step < 32 && s_off[wl][q + step] <= e) q += step;
      int ix = s_lo[wl][q] + (e - s_off[wl][q]);
      int yy = iy0 + q;
      double L = chord_len(A, model, pk, coord(ix, nx), coord(yy, ny));
      sum += L;
      ci[pos + e] = yy * nx + ix;
      v[pos + e] = __double2float_rn(L);
    }
    pos += T;
    __syncwarp();
  }
  sum = warp_sum_d(sum);
  if (lane == 0) R[w] = sum != 0.0 ? __double2float_rn(1.0 / sum) : 0.0f;
}

// ---------------------------------------------------------------------------
// A^T: count and fill, one warp per pixel, lanes over angles
// ---------------------------------------------------------------------------
template <bool kFill>
__global__ void __launch_bounds__(kThreads) k_pixels(const AngleC *__restrict__ ang, int model, int nx, int ny,
                                                     int np, int nt, double c,
                                                     int32_t *__restrict__ cnt,
                                                     const int64_t *__restrict__ rp,
                                                     int32_t *__restrict__ ci, float *__restrict__ v,
                                                     float *__restrict__ C, int *__restrict__ err) {
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= (int64_t)nx * ny) return;
  int ix = (int)(w % nx), iy = (int)(w / nx);
  double x = coord(ix, nx), y = coord(iy, ny);
  int total = 0;
  int64_t pos = kFill ? rp[w] : 0;
  double sum = 0.0;
  for (int m0 = 0; m0 < nt; m0 += 32) {
    int m = m0 + lane;
    constexpr int kMaxBins = 3;  // hits per angle: 2 (line), 3 (strip)
    int nh = 0;
    int kh[kMaxBins] = {0, 0, 0};
    double Lh[kMaxBins] = {0.0, 0.0, 0.0};
    if (m < nt) {
      AngleC A = ang[m];
      // |p_k - t| < hs <= 1.2072 puts k within 1.21 of u = t + c - 1/2
      double u = x * A.cs + y * A.sn + (c - 0.5);
      long long kf = (long long)floor(u);
      for (long long k = kf - 2; k <= kf + 2; ++k) {
        if (k < 0 || k >= np) continue;
        double pk = __dsub_rn(__dadd_rn((double)k, 0.5), c);
        if (chord_hit(A, pk, x, y)) {
          if (nh < kMaxBins) {
            kh[nh] = (int)k;
            if (kFill) Lh[nh] = chord_len(A, model, pk, x, y);
          } else if (err) {
            atomicExch(err, 1);  // impossible by the bound above; reported, never written
          }
          ++nh;
        }
      }
      nh = min(nh, kMaxBins);
    }
    if (!kFill) {
      total += nh;
    } else {
      int incl = warp_incl_scan(nh, lane);
      int base = incl - nh;
      for (int q = 0; q < nh; ++q) {
        ci[pos + base + q] = m * np + kh[q];
        v[pos + base + q] = __double2float_rn(Lh[q]);
        sum += Lh[q];
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (!kFill) {
    total = warp_sum_i(total);
    if (lane == 0) cnt[w] = total;
  } else {
    sum = warp_sum_d(sum);
    if (lane == 0) C[w] = sum != 0.0 ? __double2float_rn(1.0 / sum) : 0.0f;
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 counts into int64 offsets (three passes) + max.
// ---------------------------------------------------------------------------
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ int64_t block_excl_scan(int64_t v, int64_t *total) {
  __shared__ int64_t s_w[kThreads / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  int64_t woff = 0, tot = 0;
  for (int i = 0; i < kThreads / 32; ++i) {
    if (i < wid) woff += s_w[i];
    tot += s_w[i];
  }
  __syncthreads();
  *total = tot;
  return woff + incl - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t *__restrict__ in, int64_t n,
                                                          int64_t *__restrict__ part,
                                                          int *__restrict__ maxv) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  int mx = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) {
      s += in[base + i];
      mx = max(mx, in[base + i]);
    }
  int64_t tot;
  block_excl_scan(s, &tot);
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxv, mx);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_scan_parts(int64_t *part, int64_t nparts) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nparts; b0 += kThreads) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < nparts ? part[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan(v, &tot);
    if (i < nparts) part[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const int32_t *__restrict__ in, int64_t n,
                                                         const int64_t *__restrict__ part,
                                                         int64_t *__restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int64_t tot;
  int64_t ex = block_excl_scan(s, &tot) + part[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) {
      out[base + i] = ex;
      ex += in[base + i];
    }
  if (base + kScanItems >= n && base < n) out[n] = ex;  // thread owning the last item
}

// ---------------------------------------------------------------------------
// SELL-32 forms (see internal.cuh for the slot maps)
// ---------------------------------------------------------------------------
// per chunk of 32 rows: slots = W*32 with W the longest row rounded up to
// `align`, and (optionally) bases = (W/16)*32
__global__ void k_chunk_sizes(const int64_t *__restrict__ rp, int64_t rows, int align,
                              int32_t *__restrict__ slots, int32_t *__restrict__ bases) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t chunks = (rows + 31) / 32;
  if (c >= chunks) return;
  int64_t w = 0;
  for (int q = 0; q < 32; ++q) {
    int64_t r = c * 32 + q;
    if (r < rows) w = max(w, rp[r + 1] - rp[r]);
  }
  w = (w + align - 1) / align * align;
  slots[c] = (int32_t)(w * 32);
  if (bases) bases[c] = (int32_t)(w / 16 * 32);
}

__global__ void k_row_len(const int64_t *__restrict__ rp, int64_t rows, int32_t *__restrict__ rl) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) rl[r] = (int32_t)(rp[r + 1] - rp[r]);
}

// one warp per row; entries (column, value bits) in pairs
__global__ void __launch_bounds__(kThreads) k_sell_fill(const int64_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci,
                                                        const float *__restrict__ v, int64_t rows,
                                                        const int64_t *__restrict__ cp, int2 *__restrict__ ent) {
  int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= rows) return;
  int64_t b = rp[r], len = rp[r + 1] - b;
  int64_t base = cp[r >> 5];
  int q = (int)(r & 31);
  for (int64_t e = lane; e < len; e += 32)
    ent[base + (e >> 1) * 64 + 2 * q + (e & 1)] = make_int2(ci[b + e], __float_as_int(v[b + e]));
}

// 16-bit form, pass 1 (one thread per row): the row's padded length.  Entries
// are cut into segments of 16 with one 32-bit base each; a segment is closed
// early (padded with zero-weight entries) when the next column lies more than
// 65535 past its base, which happens where a pixel is seen by two separate
// ranges of angles (image corners).
// Only the entries with column in [c0, c1) are taken (one band of a banded A).
__global__ void k_sell16_len(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t rows,
                             int32_t *__restrict__ rl16, int32_t c0, int32_t c1, int nb4, int np) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t src = ray_of(r, nb4, np);  // the CSR row that row r holds
  int64_t b = rp[src], len = rp[src + 1] - b;
  int64_t slot = 0;
  int32_t cb = 0;
  for (int64_t e = 0; e < len; ++e) {
    int32_t col = ci[b + e];
    if (col < c0 || col >= c1) continue;
    if ((slot & 15) != 0 && (int64_t)col - cb > 65535) slot = (slot + 15) / 16 * 16;
    if ((slot & 15) == 0) cb = col;
    ++slot;
  }
  rl16[r] = (int32_t)((slot + 15) / 16 * 16);
}

// 16-bit form, pass 2 (one thread per row): same walk, writing the packed
// (offset | weight << 16) words and the segment bases; weights A_ij * a(theta)
// recomputed in FP64 from the geometry.  Padding slots stay zero.
template <bool kTranspose, typename W>
__global__ void k_sell16_fill(const AngleC *__restrict__ ang, int model, int nx, int ny, int np, double c,
                              const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t rows,
                              const int64_t *__restrict__ cpw, const int64_t *__restrict__ cpb,
                              uint32_t *__restrict__ ow, int32_t *__restrict__ base, int *__restrict__ err,
                              int32_t c0, int32_t c1, int nb4) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t src = ray_of(r, nb4, np);  // the CSR row that row r holds
  int64_t b = rp[src], len = rp[src + 1] - b;
  int64_t w0 = cpw[r >> 5], b0 = cpb[r >> 5];
  int q = (int)(r & 31);
  int64_t slot = 0;
  int32_t cb = 0;
  for (int64_t e = 0; e < len; ++e) {
    int32_t col = ci[b + e];
    if (col < c0 || col >= c1) continue;
    if ((slot & 15) != 0 && (int64_t)col - cb > 65535) slot = (slot + 15) / 16 * 16;
    if ((slot & 15) == 0) {
      cb = col;
      base[b0 + (slot >> 4) * 32 + q] = cb;
    }
    int64_t d = (int64_t)col - cb;
    if (d < 0 || d > 65535) atomicExch(err, 2);  // impossible after the early cut; reported
    int ray = kTranspose ? col : (int)src;
    int pix = kTranspose ? (int)src : col;
    int m = ray / np, k = ray % np;
    int ix = pix % nx, iy = pix / nx;
    AngleC A = ang[m];
    double pk = __dsub_rn(__dadd_rn((double)k, 0.5), c);
    double w = __dmul_rn(chord_len(A, model, pk, coord(ix, nx), coord(iy, ny)), A.a);
    uint16_t wbits;
    if constexpr (std::is_same<W, __nv_bfloat16>::value)
      wbits = __bfloat16_as_ushort(__double2bfloat16(w));
    else
      wbits = __half_as_ushort(__double2half(w));
    ow[w0 + (slot >> 2) * 128 + 4 * q + (slot & 3)] = (uint32_t)(uint16_t)d | ((uint32_t)wbits << 16);
    ++slot;
  }
}

// per chunk of 32 rows with explicit (already 16-aligned) row lengths
__global__ void k_chunk_sizes_rl(const int32_t *__restrict__ rl, int64_t rows, int32_t *__restrict__ slots,
                                 int32_t *__restrict__ bases) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t chunks = (rows + 31) / 32;
  if (c >= chunks) return;
  int32_t w = 0;
  for (int q = 0; q < 32; ++q) {
    int64_t r = c * 32 + q;
    if (r < rows) w = max(w, rl[r]);
  }
  slots[c] = w * 32;
  bases[c] = w / 16 * 32;
}

int grid_for_warps(int64_t warps) { return (int)((warps * 32 + kThreads - 1) / kThreads); }

tomo_status scan_counts(const int32_t *cnt, int64_t n, int64_t *out, int64_t *part, int *maxv,
                        cudaStream_t st) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)tiles, kThreads, 0, st>>>(cnt, n, part, maxv);
  k_scan_parts<<<1, kThreads, 0, st>>>(part, tiles);
  k_scan_apply<<<(unsigned)tiles, kThreads, 0, st>>>(cnt, n, part, out);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

template <typename T>
tomo_status dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TOMO_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  return TOMO_OK;
}

tomo_status build_sell(tomo_matrix *h, bool transpose, cudaStream_t st, int32_t *cnt, int64_t *part,
                       int *scratch) {
  const Csr &M = transpose ? h->AT : h->A;
  Sell &S = transpose ? h->sAT : h->sA;
  S.rows = M.rows;
  S.chunks = (M.rows + 31) / 32;
  TOMO_TRY(dmalloc(&S.cp, S.chunks + 1));
  TOMO_TRY(dmalloc(&S.rl, M.rows));
  k_row_len<<<(unsigned)((M.rows + 255) / 256), 256, 0, st>>>(M.rp, M.rows, S.rl);
  k_chunk_sizes<<<(unsigned)((S.chunks + 255) / 256), 256, 0, st>>>(M.rp, M.rows, 2, cnt, nullptr);
  TOMO_TRY(scan_counts(cnt, S.chunks, S.cp, part, scratch + 3, st));
  TOMO_CUDA(cudaMemcpyAsync(&S.slots, S.cp + S.chunks, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  TOMO_TRY(dmalloc(&S.ent, S.slots));
  TOMO_CUDA(cudaMemsetAsync(S.ent, 0, sizeof(int2) * S.slots, st));
  k_sell_fill<<<grid_for_warps(M.rows), kThreads, 0, st>>>(M.rp, M.ci, M.v, M.rows, S.cp, S.ent);
  TOMO_CUDA(cudaGetLastError());
  h->bytes_f32 += (S.chunks + 1) * 8 + M.rows * 4 + S.slots * 8;
  return TOMO_OK;
}

// The 16-bit SELL-32 form of A (or A^T) restricted to columns [c0, c1), into L.
tomo_status build_sell16(tomo_matrix *h, bool transpose, cudaStream_t st, int32_t *cnt, int64_t *part,
                         int *scratch, SellLp &L, int32_t c0, int32_t c1, bool pair_order = false) {
  const Csr &M = transpose ? h->AT : h->A;
  L.rows = M.rows;
  L.nb4 = (!transpose && pair_order && h->nt % 2 == 0 && h->np % 4 == 0) ? h->np / 4 : 0;
  L.chunks = (M.rows + 31) / 32;
  TOMO_TRY(dmalloc(&L.rl, M.rows));
  TOMO_TRY(dmalloc(&L.cpw, L.chunks + 1));
  TOMO_TRY(dmalloc(&L.cpb, L.chunks + 1));
  const unsigned gr = (unsigned)((M.rows + 255) / 256), gc = (unsigned)((L.chunks + 255) / 256);
  k_sell16_len<<<gr, 256, 0, st>>>(M.rp, M.ci, M.rows, L.rl, c0, c1, L.nb4, h->np);
  int32_t *cntb = cnt + L.chunks;  // cnt holds enough entries for two per-chunk arrays
  k_chunk_sizes_rl<<<gc, 256, 0, st>>>(L.rl, M.rows, cnt, cntb);
  TOMO_TRY(scan_counts(cnt, L.chunks, L.cpw, part, scratch + 3, st));
  TOMO_TRY(scan_counts(cntb, L.chunks, L.cpb, part, scratch + 3, st));
  TOMO_CUDA(cudaMemcpyAsync(&L.slots, L.cpw + L.chunks, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaMemcpyAsync(&L.bases, L.cpb + L.chunks, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  TOMO_TRY(dmalloc(&L.ow, L.slots));
  TOMO_TRY(dmalloc(&L.base, L.bases));
  TOMO_CUDA(cudaMemsetAsync(L.ow, 0, sizeof(uint32_t) * L.slots, st));
  TOMO_CUDA(cudaMemsetAsync(L.base, 0, sizeof(int32_t) * L.bases, st));
  const double c = h->center;
#define TOMO_FILL16(TR, W)                                                                                      \
  k_sell16_fill<TR, W><<<gr, 256, 0, st>>>(h->ang, h->model, h->nx, h->ny, h->np, c, M.rp, M.ci, M.rows, L.cpw,  \
                                           L.cpb, L.ow, L.base, scratch, c0, c1, L.nb4)
  if (h->lp_dtype == TOMO_BF16) {
    if (transpose) TOMO_FILL16(true, __nv_bfloat16);
    else TOMO_FILL16(false, __nv_bfloat16);
  } else {
    if (transpose) TOMO_FILL16(true, __half);
    else TOMO_FILL16(false, __half);
  }
#undef TOMO_FILL16
  TOMO_CUDA(cudaGetLastError());
  h->bytes_lp += (L.chunks + 1) * 16 + M.rows * 4 + L.slots * 4 + L.bases * 4;
  return TOMO_OK;
}

// ---------------------------------------------------------------------------
// 16-bit A^T in image tiles (TileLp): one block of 256 threads per tile, one
// thread per pixel (thread j: tile row j / 16, column j % 16), each walking its
// pixel's row of the A^T CSR (columns ascending: angle-major, bins ascending).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tile_pixel(int64_t t, int tiles_x, int nx, int ny, int &ix, int &iy) {
  const int ty = (int)(t / tiles_x), tx = (int)(t - (int64_t)ty * tiles_x);
  iy = ty * kTileSide + (int)(threadIdx.x >> 4);
  ix = tx * kTileSide + (int)(threadIdx.x & 15);
  return ix < nx && iy < ny;
}

// pass 1: per (tile, angle) the lowest bin any pixel meets (INT32_MAX if
// none) into win, and the widest span of bins over all (tile, angle) into *wmax
__global__ void __launch_bounds__(256) k_tile_window(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                     int nx, int ny, int np, int nt, int tiles_x,
                                                     int32_t *__restrict__ win, int *__restrict__ wmax) {
  extern __shared__ int tw_sm[];
  int *lo = tw_sm, *hi = tw_sm + nt;
  const int64_t t = blockIdx.x;
  for (int m = threadIdx.x; m < nt; m += blockDim.x) {
    lo[m] = INT32_MAX;
    hi[m] = -1;
  }
  __syncthreads();
  int ix, iy;
  if (tile_pixel(t, tiles_x, nx, ny, ix, iy)) {
    const int64_t row = (int64_t)iy * nx + ix;
    for (int64_t e = rp[row], end = rp[row + 1]; e < end; ++e) {
      const int col = ci[e], m = col / np, k = col - m * np;
      atomicMin(lo + m, k);
      atomicMax(hi + m, k);
    }
  }
  __syncthreads();
  int w = 0;
  for (int m = threadIdx.x; m < nt; m += blockDim.x) {
    win[t * nt + m] = lo[m];
    if (hi[m] >= 0) w = max(w, hi[m] - lo[m] + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
  if ((threadIdx.x & 31) == 0 && w > 0) atomicMax(wmax, w);
}

__global__ void k_tile_clamp(int32_t *__restrict__ win, int64_t n, int32_t hi) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    win[j] = min(win[j], hi);
}

// The quad of thread j's pixel (q = 8 g + i) and its place a = 2 dy + dx in it
__device__ __forceinline__ int tile_quad(int j) { return (j >> 5) * 8 + ((j & 15) >> 1); }
__device__ __forceinline__ int tile_quad_pixel(int j) { return ((j >> 4) & 1) * 2 + (j & 1); }

// Per (quad, angle of chunk k) the lowest and highest bin its pixels meet
// (INT32_MAX / -1 where none), from this thread's CSR cursor e, which it
// advances past the chunk.  Every thread of the block calls it.
__device__ __forceinline__ void quad_runs(const int32_t *__restrict__ ci, int64_t &e, int64_t end, int np, int nt,
                                          int k, int *lo, int *hi) {
  for (int j = threadIdx.x; j < 64 * kTileChunk; j += blockDim.x) {
    lo[j] = INT32_MAX;
    hi[j] = -1;
  }
  __syncthreads();
  const int q = tile_quad(threadIdx.x);
  const int64_t lim = (int64_t)min((k + 1) * kTileChunk, nt) * np;
  for (; e < end && ci[e] < lim; ++e) {
    const int col = ci[e], m = col / np, b = col - m * np, s = q * kTileChunk + m - k * kTileChunk;
    atomicMin(lo + s, b);
    atomicMax(hi + s, b);
  }
  __syncthreads();
}

// slots of quad q in the chunk: its angles' runs
__device__ __forceinline__ int quad_slots(const int *lo, const int *hi, int q) {
  int n = 0;
#pragma unroll
  for (int a = 0; a < kTileChunk; ++a) {
    const int j = q * kTileChunk + a;
    if (hi[j] >= 0) n += hi[j] - lo[j] + 1;
  }
  return n;
}

// pass 2: blocks of each (tile, chunk, group): the group's longest quad
__global__ void __launch_bounds__(256) k_tile_count(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                    int nx, int ny, int np, int nt, int tiles_x, int nch,
                                                    int32_t *__restrict__ cnt) {
  __shared__ int lo[64 * kTileChunk], hi[64 * kTileChunk];
  const int64_t t = blockIdx.x;
  int ix, iy;
  int64_t e = 0, end = 0;
  if (tile_pixel(t, tiles_x, nx, ny, ix, iy)) {
    const int64_t row = (int64_t)iy * nx + ix;
    e = rp[row];
    end = rp[row + 1];
  }
  for (int k = 0; k < nch; ++k) {
    quad_runs(ci, e, end, np, nt, k, lo, hi);
    if (threadIdx.x < 64) {  // thread q: quad q; a group's 8 quads are 8 consecutive threads
      int n = quad_slots(lo, hi, (int)threadIdx.x);
      n = max(n, __shfl_xor_sync(0xffffffffu, n, 1));
      n = max(n, __shfl_xor_sync(0xffffffffu, n, 2));
      n = max(n, __shfl_xor_sync(0xffffffffu, n, 4));
      if ((threadIdx.x & 7) == 0)
        cnt[(t * nch + k) * 8 + (threadIdx.x >> 3)] = (n + kTileBlockSlots - 1) / kTileBlockSlots;
    }
    __syncthreads();  // lo / hi are reset for the next chunk
  }
}

__global__ void k_tile_offsets(const int64_t *__restrict__ off, int64_t n, uint32_t *__restrict__ qoff) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += (int64_t)gridDim.x * blockDim.x)
    qoff[j] = (uint32_t)off[j];
}

// most blocks of one (tile, chunk): the size of the pass's staged entry buffer
__global__ void k_tile_max_blocks(const int64_t *__restrict__ off, int64_t chunks, int *__restrict__ mx) {
  int m = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < chunks; j += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(off[(j + 1) * 8] - off[j * 8]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// pass 3: weights (the FP64 rule and rounding of k_sell16_fill) and staged row
// positions of every slot
template <typename W>
__global__ void __launch_bounds__(256) k_tile_fill(const AngleC *__restrict__ ang, int model, double c,
                                                   const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                   int nx, int ny, int np, int nt, int tiles_x, int nch, int wlen,
                                                   const uint32_t *__restrict__ qoff, const int32_t *__restrict__ win,
                                                   uint32_t *__restrict__ ent) {
  constexpr int C = kTileChunk;
  __shared__ int lo[64 * C], hi[64 * C], st[64 * (C + 1)];
  const int64_t t = blockIdx.x;
  int ix, iy;
  int64_t e = 0, end = 0;
  const bool mine = tile_pixel(t, tiles_x, nx, ny, ix, iy);
  if (mine) {
    const int64_t row = (int64_t)iy * nx + ix;
    e = rp[row];
    end = rp[row + 1];
  }
  const double x = coord(ix, nx), y = coord(iy, ny);
  const int q = tile_quad(threadIdx.x), pa = tile_quad_pixel(threadIdx.x), i = q & 7;
  unsigned char *ent8 = reinterpret_cast<unsigned char *>(ent);
  for (int k = 0; k < nch; ++k) {
    const int64_t e0 = e;
    quad_runs(ci, e, end, np, nt, k, lo, hi);
    if (threadIdx.x < 64) {  // each quad's first slot per angle
      int n = 0;
      for (int a = 0; a < C; ++a) {
        const int j = threadIdx.x * C + a;
        st[threadIdx.x * (C + 1) + a] = n;
        if (hi[j] >= 0) n += hi[j] - lo[j] + 1;
      }
      st[threadIdx.x * (C + 1) + C] = n;
    }
    __syncthreads();
    const uint32_t *qg = qoff + (t * nch + k) * 8;
    for (int64_t f = e0; f < e; ++f) {  // this pixel's weights
      const int col = ci[f], m = col / np, b = col - m * np, a = m - k * C;
      const int s = st[q * (C + 1) + a] + (b - lo[q * C + a]);
      const AngleC A = ang[m];
      const double pk = __dsub_rn(__dadd_rn((double)b, 0.5), c);
      const double w = __dmul_rn(chord_len(A, model, pk, x, y), A.a);
      uint16_t wbits;
      if constexpr (std::is_same<W, __nv_bfloat16>::value)
        wbits = __bfloat16_as_ushort(__double2bfloat16(w));
      else
        wbits = __half_as_ushort(__double2half(w));
      const size_t blk = (size_t)qg[q >> 3] + (size_t)(s >> 2);
      reinterpret_cast<uint16_t *>(ent8 + blk * kTileBlockBytes)[((s & 3) >> 1) * 64 + i * 8 + (s & 1) * 4 + pa] =
          wbits;
    }
    if (threadIdx.x < 64) {  // the row positions of the quad's slots, padding included
      const int qq = (int)threadIdx.x, g = qq >> 3, qi = qq & 7, partner = qq ^ 1;
      const int S = (int)(qg[g + 1] - qg[g]) * kTileBlockSlots;
      // staged row of quad Q's slot s (s below its slot count)
      auto row_of = [&](int Q, int s) {
        int a = 0;
        while (s >= st[Q * (C + 1) + a + 1]) ++a;
        const int b = lo[Q * C + a] + (s - st[Q * (C + 1) + a]);
        return a * wlen + b - win[t * nt + k * C + a];
      };
      const int nq = st[qq * (C + 1) + C], npart = st[partner * (C + 1) + C];
      for (int s = 0; s < S; ++s) {
        const int r = s < nq ? row_of(qq, s) : (s < npart ? row_of(partner, s) : 0);
        const size_t blk = (size_t)qg[g] + (size_t)(s >> 2);
        ent8[blk * kTileBlockBytes + 256 + qi * 4 + (s & 3)] = (unsigned char)tile_swz(r);
      }
    }
    __syncthreads();  // lo / hi / st are reset for the next chunk
  }
}

// The tiled form of the 16-bit A^T (TileLp) from the A^T CSR.  Leaves it
// unbuilt (ent == nullptr) where the geometry does not suit it: more angles
// than the window pass's shared arrays hold, windows wider than 32 bins (a
// staged row position is one byte), or chunks whose staged entries would not
// leave room for two blocks of the pass per SM.
tomo_status build_tile16(tomo_matrix *h, cudaStream_t st) {
  TileLp &T = h->lpATt;
  const int nt = h->nt, np = h->np;
  const size_t win_smem = (size_t)2 * nt * sizeof(int);
  if (win_smem > (size_t)(160 << 10)) return TOMO_OK;
  T.tiles_x = (h->nx + kTileSide - 1) / kTileSide;
  T.tiles_y = (h->ny + kTileSide - 1) / kTileSide;
  T.tiles = (int64_t)T.tiles_x * T.tiles_y;
  T.nch = (nt + kTileChunk - 1) / kTileChunk;
  int *small = nullptr;  // [0] widest window, [1] most blocks of a chunk
  TOMO_TRY(dmalloc(&small, 2));
  DevBuf small_guard{small};
  TOMO_CUDA(cudaMemsetAsync(small, 0, 2 * sizeof(int), st));
  TOMO_TRY(dmalloc(&T.win, (size_t)T.tiles * nt));
  if (win_smem > (size_t)(48 << 10))
    TOMO_CUDA(cudaFuncSetAttribute(k_tile_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem));
  k_tile_window<<<(unsigned)T.tiles, 256, win_smem, st>>>(h->AT.rp, h->AT.ci, h->nx, h->ny, np, nt, T.tiles_x,
                                                          T.win, small);
  TOMO_CUDA(cudaGetLastError());
  int wmax = 0;
  TOMO_CUDA(cudaMemcpyAsync(&wmax, small, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  T.W = std::max(wmax, 1);
  if (T.W > 32) {  // wider than the pass stages (a unit-spaced detector needs at most 26): leave it unbuilt
    cudaFree(T.win);
    T = TileLp{};
    return TOMO_OK;
  }
  const int64_t nwin = T.tiles * nt;
  k_tile_clamp<<<(unsigned)std::min<int64_t>((nwin + 255) / 256, 4096), 256, 0, st>>>(T.win, nwin,
                                                                                      std::max(np - T.W, 0));
  const int64_t n = T.tiles * T.nch * 8;
  int32_t *cnt = nullptr;
  int64_t *off = nullptr, *part = nullptr;
  int *maxv = nullptr;
  TOMO_TRY(dmalloc(&cnt, n));
  DevBuf cnt_guard{cnt};
  TOMO_TRY(dmalloc(&off, n + 1));
  DevBuf off_guard{off};
  TOMO_TRY(dmalloc(&part, n / kScanTile + 2));
  DevBuf part_guard{part};
  TOMO_TRY(dmalloc(&maxv, 1));
  DevBuf maxv_guard{maxv};
  k_tile_count<<<(unsigned)T.tiles, 256, 0, st>>>(h->AT.rp, h->AT.ci, h->nx, h->ny, np, nt, T.tiles_x, T.nch, cnt);
  TOMO_CUDA(cudaGetLastError());
  TOMO_TRY(scan_counts(cnt, n, off, part, maxv, st));
  k_tile_max_blocks<<<(unsigned)std::min<int64_t>((T.tiles * T.nch + 255) / 256, 4096), 256, 0, st>>>(
      off, T.tiles * T.nch, small + 1);
  TOMO_CUDA(cudaGetLastError());
  int mb = 0;
  TOMO_CUDA(cudaMemcpyAsync(&T.blocks, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaMemcpyAsync(&mb, small + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  T.max_blocks = std::max(mb, 1);
  // block offsets are 32-bit; the pass's two staging buffers must leave room for 2 blocks per SM
  const int64_t buf = (int64_t)kTileChunk * T.W * kTileRow + (int64_t)T.max_blocks * kTileBlockBytes + 48;
  if (T.blocks >= ((int64_t)1 << 32) || 2 * buf > (100 << 10)) {
    cudaFree(T.win);
    T = TileLp{};
    return TOMO_OK;
  }
  TOMO_TRY(dmalloc(&T.qoff, n + 4));  // the pass copies 12 offsets per chunk (16-byte pieces)
  TOMO_CUDA(cudaMemsetAsync(T.qoff, 0, sizeof(uint32_t) * (n + 4), st));
  k_tile_offsets<<<(unsigned)std::min<int64_t>((n + 256) / 256, 4096), 256, 0, st>>>(off, n, T.qoff);
  const size_t ent_bytes = (size_t)std::max<int64_t>(T.blocks, 1) * kTileBlockBytes;
  TOMO_TRY(dmalloc(&T.ent, ent_bytes / 4));
  TOMO_CUDA(cudaMemsetAsync(T.ent, 0, ent_bytes, st));
#define TOMO_TFILL(WT)                                                                                        \
  k_tile_fill<WT><<<(unsigned)T.tiles, 256, 0, st>>>(h->ang, h->model, h->center, h->AT.rp, h->AT.ci, h->nx, h->ny, \
                                                    np, nt, T.tiles_x, T.nch, T.W, T.qoff, T.win, T.ent)
  if (h->lp_dtype == TOMO_BF16) TOMO_TFILL(__nv_bfloat16);
  else TOMO_TFILL(__half);
#undef TOMO_TFILL
  TOMO_CUDA(cudaGetLastError());
  TOMO_CUDA(cudaStreamSynchronize(st));  // the temporaries are freed on return
  h->bytes_lp += (n + 4) * 4 + nwin * 4 + T.blocks * kTileBlockBytes;
  return TOMO_OK;
}

}  // namespace

// Exclusive scan of n int32 counts into n+1 int64 offsets (other translation
// units use it for their transposes).
tomo_status exclusive_scan_i32(const int32_t *cnt, int64_t n, int64_t *out, cudaStream_t st) {
  int64_t *part = nullptr;
  int *maxv = nullptr;
  TOMO_TRY(dmalloc(&part, n / kScanTile + 2));
  DevBuf part_guard{part};
  TOMO_TRY(dmalloc(&maxv, 1));
  DevBuf max_guard{maxv};
  TOMO_CUDA(cudaMemsetAsync(maxv, 0, sizeof(int), st));
  TOMO_TRY(scan_counts(cnt, n, out, part, maxv, st));
  TOMO_CUDA(cudaStreamSynchronize(st));  // the scratch is freed on return
  return TOMO_OK;
}

// ---------------------------------------------------------------------------
// Taps of the preconditioning filter P^T P = F^dagger D F along the detector
// (Sec. 2.1), used by the BB-step SIRT of Sec. 3.1.  On the N-point DFT grid
// (N = the smallest power of two >= 2 n_p, so a projection row zero-padded to
// N never wraps), D_k = R_k w_k: R is the DFT of the sampled band-limited ramp
// (1/4 at n = 0, -1/(pi n)^2 at odd n, 0 at even n, |n| <= N/2) and w the
// Hamming window 0.54 + 0.46 cos(2 pi k / N).  The filter is then the
// symmetric Toeplitz operator tap[|k - j|] on the n_p bins of a row, with
// tap[d] = (1/N) sum_k D_k cos(2 pi k d / N).  FP64 sums, angles reduced
// exactly as (k d mod N) / N before the cosine; the taps are rounded to FP32.
// ---------------------------------------------------------------------------
__global__ void k_ramp_response(int N, double *D) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N / 2) return;
  const double pi = 3.141592653589793;
  double R = 0.25;
  for (int n = 1; n < N / 2; n += 2) {
    const int64_t kn = ((int64_t)k * n) % N;
    R -= 2.0 / (pi * pi * (double)n * (double)n) * cos(2.0 * pi * (double)kn / (double)N);
  }
  if ((N / 2) & 1) {  // n = -N/2 is odd only for N = 2
    const double hN = -1.0 / (pi * pi * (double)(N / 2) * (double)(N / 2));
    R += (k & 1) ? -hN : hN;
  }
  D[k] = R * (0.54 + 0.46 * cos(2.0 * pi * (double)k / (double)N));
}

__global__ void k_ramp_taps(int N, const double *D, int np, float *tap) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= np) return;
  const double pi = 3.141592653589793;
  double h = D[0] + ((d & 1) ? -D[N / 2] : D[N / 2]);
  for (int k = 1; k < N / 2; ++k) {
    const int64_t kd = ((int64_t)k * d) % N;
    h += 2.0 * D[k] * cos(2.0 * pi * (double)kd / (double)N);
  }
  tap[d] = (float)(h / (double)N);
}

tomo_status build_ramp(tomo_matrix *h, cudaStream_t st) {
  int N = 2;
  while (N < 2 * h->np) N *= 2;
  double *D = nullptr;
  TOMO_TRY(dmalloc(&D, N / 2 + 1));
  DevBuf D_guard{D};
  TOMO_TRY(dmalloc(&h->ramp, h->np));
  k_ramp_response<<<(N / 2 + 1 + 127) / 128, 128, 0, st>>>(N, D);
  TOMO_CUDA(cudaGetLastError());
  k_ramp_taps<<<(h->np + 127) / 128, 128, 0, st>>>(N, D, h->np, h->ramp);
  TOMO_CUDA(cudaGetLastError());
  TOMO_CUDA(cudaStreamSynchronize(st));  // D is freed on return
  return TOMO_OK;
}

void free_matrix(tomo_matrix *h) {
  if (!h) return;
  for (SellLp &L : h->lpAb)
    for (void *p : {(void *)L.cpw, (void *)L.cpb, (void *)L.rl, (void *)L.ow, (void *)L.base})
      if (p) cudaFree(p);
  void *ptrs[] = {h->ang,      h->ang_scale, h->A.rp,     h->A.ci,     h->A.v,       h->AT.rp,
                  h->AT.ci,    h->AT.v,      h->R,        h->C,        h->sA.cp,     h->sA.rl,
                  h->sA.ent,   h->sAT.cp,    h->sAT.rl,   h->sAT.ent,  h->lpA.cpw,   h->lpA.cpb,
                  h->lpA.ow,   h->lpA.base,  h->lpAT.cpw, h->lpAT.cpb, h->lpAT.ow,   h->lpAT.base,
                  h->lpA.rl,   h->lpAT.rl,   h->ramp,     h->lpATt.qoff, h->lpATt.win, h->lpATt.ent};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

tomo_status build_matrix(const tomo_geometry *g, const tomo_matrix_opts *o, cudaStream_t st,
                         tomo_matrix **out) {
  if (!g || !out) return fail(TOMO_ERR_INVALID_ARG, "geometry and out must be non-NULL");
  *out = nullptr;
  if (g->n_x <= 0 || g->n_y <= 0 || g->n_p <= 0 || g->n_theta <= 0)
    return fail(TOMO_ERR_INVALID_ARG, "n_x, n_y, n_p and n_theta must be positive");
  if ((int64_t)g->n_x * g->n_y >= (int64_t)INT32_MAX || (int64_t)g->n_p * g->n_theta >= (int64_t)INT32_MAX)
    return fail(TOMO_ERR_INVALID_ARG, "n_x*n_y and n_theta*n_p must fit in int32 column indices");
  int32_t lp = o ? o->values : TOMO_F32;
  if (lp != TOMO_F32 && lp != TOMO_BF16 && lp != TOMO_F16)
    return fail(TOMO_ERR_INVALID_ARG, "opts.values must be TOMO_F32, TOMO_BF16 or TOMO_F16");
  if (o && o->drop_csr && o->no_fp32_sell && lp == TOMO_F32)
    return fail(TOMO_ERR_INVALID_ARG, "drop_csr needs a SELL form (FP32 SELL or 16-bit values)");
  double c = std::isnan(g->center) ? 0.5 * (double)g->n_p : g->center;
  if (!std::isfinite(c)) return fail(TOMO_ERR_INVALID_ARG, "center must be finite or NaN");
  const int32_t model = o ? o->model : TOMO_MODEL_LINE;
  if (model != TOMO_MODEL_LINE && model != TOMO_MODEL_STRIP)
    return fail(TOMO_ERR_INVALID_ARG, "opts.model must be TOMO_MODEL_LINE or TOMO_MODEL_STRIP");
  int32_t bands = o ? o->col_blocks : 0;
  if (bands < 0 || bands > 64 || bands > g->n_y)
    return fail(TOMO_ERR_INVALID_ARG, "opts.col_blocks must be in [0, min(64, n_y)]");
  if (bands > 1 && lp == TOMO_F32)
    return fail(TOMO_ERR_INVALID_ARG, "opts.col_blocks > 1 needs 16-bit values (TOMO_BF16 or TOMO_F16)");
  if (bands == 0 && lp != TOMO_F32) {
    // auto: enough bands that one band of a 16-slice FP32 image batch fits in 48 MB of L2
    const int64_t batch_bytes = (int64_t)g->n_x * g->n_y * 16 * 4;
    bands = (int32_t)std::min<int64_t>({(batch_bytes + (48 << 20) - 1) / (48 << 20), 64, (int64_t)g->n_y});
  }
  const int nt = g->n_theta;
  std::vector<AngleC> ang(nt);
  std::vector<float> scale(nt);
  for (int m = 0; m < nt; ++m) {
    double th = g->angles ? g->angles[m] : (double)m * M_PI / (double)nt;
    if (!std::isfinite(th)) return fail(TOMO_ERR_INVALID_ARG, "angles must be finite");
    AngleC &A = ang[m];
    A.cs = std::cos(th);
    A.sn = std::sin(th);
    double acs = std::fabs(A.cs), asn = std::fabs(A.sn);
    A.a = acs > asn ? acs : asn;
    A.e = acs > asn ? asn : acs;
    A.h = 0.5 * (A.a + A.e);
    A.hm = 0.5 * (A.a - A.e);
    A.inv_a = 1.0 / A.a;
    A.ae = A.a * A.e;
    A.inv_cs = A.cs != 0.0 ? 1.0 / A.cs : 0.0;
    A.inv_sn = A.sn != 0.0 ? 1.0 / A.sn : 0.0;
    A.hs = model == TOMO_MODEL_STRIP ? A.h + 0.5 : A.h;
    scale[m] = (float)(1.0 / A.a);
  }

  tomo_matrix *h = new tomo_matrix();
  struct Guard {
    tomo_matrix *h;
    bool keep = false;
    ~Guard() {
      if (!keep) free_matrix(h);
    }
  } guard{h};
  cudaGetDevice(&h->device);
  h->nx = g->n_x;
  h->ny = g->n_y;
  h->np = g->n_p;
  h->nt = nt;
  h->model = model;
  h->center = c;
  h->lp_dtype = lp;
  const int64_t rows = (int64_t)nt * g->n_p, cols = (int64_t)g->n_x * g->n_y;
  h->A.rows = rows;
  h->A.cols = cols;
  h->AT.rows = cols;
  h->AT.cols = rows;

  TOMO_TRY(dmalloc(&h->ang, nt));
  TOMO_TRY(dmalloc(&h->ang_scale, nt));
  TOMO_CUDA(cudaMemcpyAsync(h->ang, ang.data(), sizeof(AngleC) * nt, cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemcpyAsync(h->ang_scale, scale.data(), sizeof(float) * nt, cudaMemcpyHostToDevice, st));

  int64_t nmax = rows > cols ? rows : cols;
  int32_t *cnt = nullptr;
  int64_t *part = nullptr;
  int *scratch = nullptr;  // [0] error flag, [1] max row length, [2] max column length, [3] unused max
  TOMO_TRY(dmalloc(&cnt, nmax + nmax / 16 + 64));  // also holds two per-chunk arrays
  DevBuf cnt_guard{cnt};
  TOMO_TRY(dmalloc(&part, nmax / kScanTile + 2));
  DevBuf part_guard{part};
  TOMO_TRY(dmalloc(&scratch, 4));
  DevBuf scratch_guard{scratch};
  TOMO_CUDA(cudaMemsetAsync(scratch, 0, 4 * sizeof(int), st));

  TOMO_TRY(dmalloc(&h->A.rp, rows + 1));
  TOMO_TRY(dmalloc(&h->AT.rp, cols + 1));
  TOMO_TRY(dmalloc(&h->R, rows));
  TOMO_TRY(dmalloc(&h->C, cols));

  k_count_rays<<<grid_for_warps(rows), kThreads, 0, st>>>(h->ang, h->nx, h->ny, h->np, nt, c, cnt);
  TOMO_CUDA(cudaGetLastError());
  TOMO_TRY(scan_counts(cnt, rows, h->A.rp, part, scratch + 1, st));
  k_pixels<false><<<grid_for_warps(cols), kThreads, 0, st>>>(h->ang, model, h->nx, h->ny, h->np, nt, c, cnt,
                                                               nullptr, nullptr, nullptr, nullptr, scratch);
  TOMO_CUDA(cudaGetLastError());
  TOMO_TRY(scan_counts(cnt, cols, h->AT.rp, part, scratch + 2, st));

  int64_t nnz_a = 0, nnz_t = 0;
  int hs[4] = {0, 0, 0, 0};
  TOMO_CUDA(cudaMemcpyAsync(&nnz_a, h->A.rp + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaMemcpyAsync(&nnz_t, h->AT.rp + cols, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaMemcpyAsync(hs, scratch, sizeof(hs), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  if (hs[0] != 0) return fail(TOMO_ERR_NUMERIC, "pixel enumeration found more bins per angle than the model allows");
  if (nnz_a != nnz_t)
    return fail(TOMO_ERR_NUMERIC, "ray-driven and pixel-driven entry counts differ: " + std::to_string(nnz_a) +
                                      " vs " + std::to_string(nnz_t));
  h->A.nnz = h->AT.nnz = nnz_a;
  h->A.max_len = hs[1];
  h->AT.max_len = hs[2];

  size_t freeb = 0, totalb = 0;
  TOMO_CUDA(cudaMemGetInfo(&freeb, &totalb));
  // CSR pair (16 B/nnz) [+ SELL pair (~17 B/nnz)] [+ 16-bit pair (~9.5 B/nnz)] [+ tiled 16-bit A^T (~5 B/nnz)]
  const bool sell32 = !(o && o->no_fp32_sell);
  const bool at_tiles = lp != TOMO_F32 && !(o && o->no_at_tiles);
  const bool pair_order = !(o && o->a_ray_order);
  size_t need = (size_t)nnz_a * (16 + (sell32 ? 18 : 0)) +
                (size_t)(lp != TOMO_F32 ? nnz_a * 10 + (rows + cols) * 64 : 0) +
                (size_t)(at_tiles ? nnz_a * 5 + (int64_t)nt * cols / 3 : 0);
  if (need + (size_t)(1ull << 30) > freeb)
    return fail(TOMO_ERR_OOM, "matrix needs " + std::to_string(need) + " bytes, device has " +
                                  std::to_string(freeb) + " free");
  TOMO_TRY(dmalloc(&h->A.ci, nnz_a));
  TOMO_TRY(dmalloc(&h->A.v, nnz_a));
  TOMO_TRY(dmalloc(&h->AT.ci, nnz_a));
  TOMO_TRY(dmalloc(&h->AT.v, nnz_a));
  k_fill_rays<<<grid_for_warps(rows), kThreads, 0, st>>>(h->ang, model, h->nx, h->ny, h->np, nt, c, h->A.rp,
                                                          h->A.ci, h->A.v, h->R);
  TOMO_CUDA(cudaGetLastError());
  k_pixels<true><<<grid_for_warps(cols), kThreads, 0, st>>>(h->ang, model, h->nx, h->ny, h->np, nt, c, nullptr,
                                                             h->AT.rp, h->AT.ci, h->AT.v, h->C, scratch);
  TOMO_CUDA(cudaGetLastError());
  h->bytes_f32 = (rows + 1 + cols + 1) * 8 + nnz_a * 16;

  if (!(o && o->no_fp32_sell)) {
    TOMO_TRY(build_sell(h, false, st, cnt, part, scratch));
    TOMO_TRY(build_sell(h, true, st, cnt, part, scratch));
  }
  if (lp != TOMO_F32) {
    if (bands > 1) {
      // band b holds the image rows [b n_y / bands, (b + 1) n_y / bands)
      h->lpAb.resize(bands);
      for (int b = 0; b < bands; ++b) {
        const int32_t y0 = (int32_t)((int64_t)g->n_y * b / bands), y1 = (int32_t)((int64_t)g->n_y * (b + 1) / bands);
        TOMO_TRY(build_sell16(h, false, st, cnt, part, scratch, h->lpAb[b], y0 * g->n_x, y1 * g->n_x, pair_order));
      }
    } else {
      TOMO_TRY(build_sell16(h, false, st, cnt, part, scratch, h->lpA, 0, INT32_MAX, pair_order));
    }
    TOMO_TRY(build_sell16(h, true, st, cnt, part, scratch, h->lpAT, 0, INT32_MAX));
    if (!(o && o->no_at_tiles)) TOMO_TRY(build_tile16(h, st));
  }
  TOMO_CUDA(cudaMemcpyAsync(hs, scratch, sizeof(hs), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  if (o && o->drop_csr) {
    for (void **p : {(void **)&h->A.ci, (void **)&h->A.v, (void **)&h->AT.ci, (void **)&h->AT.v}) {
      cudaFree(*p);
      *p = nullptr;
    }
    h->bytes_f32 -= nnz_a * 16;
  }
  if (hs[0] == 2)
    return fail(TOMO_ERR_UNSUPPORTED, "a 16-entry chunk spans more than 65535 columns (geometry too large "
                                      "for 16-bit offsets)");
  if (hs[0] != 0) return fail(TOMO_ERR_NUMERIC, "pixel enumeration found more bins per angle than the model allows");
  TOMO_TRY(build_ramp(h, st));
  guard.keep = true;
  *out = h;
  return TOMO_OK;
}

}  // namespace tomo
