// fubini.cu -- the Fubini-Radon transform (Sec. 3, Eq. 2) on the device.
//
// Radon(u) = F1^-1 S^H F2 (k* o u): deapodize the image, zero-pad it to a
// G x G grid (G = 2n), 2D FFT, grid phase, interpolate the spectrum onto the
// polar samples (angle m, radial frequency w_q = (q - floor(n_p/2)) / n_p)
// with the sparse gridding matrix S (Kaiser-Bessel window of kw x kw grid
// points), then a 1D inverse FFT along every radial line and the real part.
// The adjoint runs the transposed steps with the stored transpose S^T; with
// the ramp density on the polar samples and the weight pi/n_theta it is the
// filtered backprojection (iRadon of Sec. 3).
//
// S is real here: the paper folds FFT shifts and the axis phase ramp into
// complex entries of S; this build applies them as diagonal phase factors
// next to the FFTs instead, so one real SpMM kernel serves complex data
// stored as (re, im) column pairs.  On power-of-two grids (32..2048) the 2D
// transforms are register-FFT passes (regfft.cuh) fused with the padding,
// cropping, phases and layout changes around them; the 1D radial transforms
// and other grid sizes use cuFFT.
#include <cmath>
#include <cstring>
#include <vector>

#include "bbstep.cuh"
#include "regfft.cuh"
#include "fubini.cuh"


namespace tomo {

tomo_status spmm_csr_store(const Csr &M, int B, const float *X, float *Y, cudaStream_t st);
tomo_status exclusive_scan_i32(const int32_t *cnt, int64_t n, int64_t *out, cudaStream_t st);

namespace {

constexpr int kT = 256;

// phi(t) = I0(beta sqrt(1 - (2t/kw)^2)) on |t| <= kw/2 (t in grid units)
__device__ __forceinline__ double kb(double t, int kw, double beta) {
  const double a = 1.0 - (2.0 * t / kw) * (2.0 * t / kw);
  return a >= 0.0 ? cyl_bessel_i0(beta * sqrt(a)) : 0.0;
}

// One thread per polar sample r = m * np + q: its kw x kw window, in window
// order (ky, then kx), columns wrapped modulo G with a factor -1 per wrap.
__global__ void k_fub_fill_S(const double *cs, const double *sn, int nt, int np, int G, int kw, double beta,
                             int64_t *rp, int32_t *ci, float *v) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)nt * np) return;
  const int m = (int)(r / np), q = (int)(r % np);
  const double w = (double)(q - np / 2) / (double)np;
  const double tx = (double)G * (w * cs[m]), ty = (double)G * (w * sn[m]);
  const int64_t kx0 = (int64_t)floor(tx - 0.5 * kw) + 1, ky0 = (int64_t)floor(ty - 0.5 * kw) + 1;
  const int64_t base = r * kw * kw;
  if (r == 0) rp[0] = 0;
  rp[r + 1] = base + (int64_t)kw * kw;
  for (int a = 0; a < kw; ++a) {
    const int64_t ky = ky0 + a;
    const int64_t my = ((ky % G) + G) % G;
    const double wy = kb(ty - (double)ky, kw, beta) * ((((ky - my) / G) & 1) ? -1.0 : 1.0);
    for (int b = 0; b < kw; ++b) {
      const int64_t kx = kx0 + b;
      const int64_t mx = ((kx % G) + G) % G;
      const double wx = kb(tx - (double)kx, kw, beta) * ((((kx - mx) / G) & 1) ? -1.0 : 1.0);
      ci[base + a * kw + b] = (int32_t)(my * G + mx);
      v[base + a * kw + b] = (float)(wy * wx);
    }
  }
}

// transpose: counts, scatter, then each row sorted by the polar sample index
__global__ void k_fub_count(const int32_t *ci, int64_t nnz, int32_t *cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + ci[e], 1);
}

__global__ void k_fub_scatter(const int32_t *ci, const float *v, int64_t rows, int per_row, const int64_t *rpT,
                              int32_t *fill, int32_t *ciT, float *vT) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * per_row;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = ci[e];
    const int64_t pos = rpT[c] + atomicAdd(fill + c, 1);
    ciT[pos] = (int32_t)(e / per_row);
    vT[pos] = v[e];
  }
}

// S^T is kept as two parts: rows of at most kLongRow entries (the short
// part, long rows left empty) and the long rows (near the spectrum's centre,
// where the samples of every angle meet) in a compact list.  Both sorted by
// polar index within a row.
constexpr int kLongRow = 64;

__global__ void k_fub_split_count(const int64_t *rp, int64_t rows, int32_t *cnt_short, int32_t *is_long) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t len = rp[r + 1] - rp[r];
  cnt_short[r] = len <= kLongRow ? (int32_t)len : 0;
  is_long[r] = len > kLongRow;
}

__global__ void k_fub_long_list(const int64_t *rp, const int64_t *lpos, int64_t rows, int32_t *rows_l,
                                int32_t *cnt_l) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows || lpos[r + 1] == lpos[r]) return;
  rows_l[lpos[r]] = (int32_t)r;
  cnt_l[lpos[r]] = (int32_t)(rp[r + 1] - rp[r]);
}

// short rows: copy, then a stable insertion sort by polar index
__global__ void k_fub_copy_short(const int64_t *rp, const int32_t *ci, const float *v, int64_t rows,
                                 const int64_t *rps, int32_t *cis, float *vs) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t b = rps[r], len = rps[r + 1] - b, src = rp[r];
  for (int64_t i = 0; i < len; ++i) {
    const int32_t key = ci[src + i];
    const float val = v[src + i];
    int64_t j = b + i - 1;
    while (j >= b && cis[j] > key) {
      cis[j + 1] = cis[j];
      vs[j + 1] = vs[j];
      --j;
    }
    cis[j + 1] = key;
    vs[j + 1] = val;
  }
}

// long rows, one block each: every entry goes to its stable rank among the
// row's keys (a key repeats when the window is wider than the grid and wraps
// onto the same point more than once)
__global__ void k_fub_copy_long(const int64_t *rp, const int32_t *ci, const float *v, const int32_t *rows_l,
                                const int64_t *rpl, int32_t *cil, float *vl) {
  const int64_t src = rp[rows_l[blockIdx.x]], dst = rpl[blockIdx.x];
  const int len = (int)(rpl[blockIdx.x + 1] - dst);
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const int32_t key = ci[src + i];
    int rank = 0;
    for (int j = 0; j < len; ++j) {
      const int32_t kj = ci[src + j];
      rank += kj < key || (kj == key && j < i);
    }
    cil[dst + rank] = key;
    vl[dst + rank] = v[src + i];
  }
}

// Y[rows_l[b]] = (long row b of S^T) X for B interleaved columns: B/2 threads
// per entry (two columns each), 512/B entries at a time, partial sums
// combined in a fixed order (deterministic)
template <int B>
__global__ void __launch_bounds__(256) k_fub_long_spmm(const int64_t *rpl, const int32_t *cil, const float *vl,
                                                       const int32_t *rows_l, const float *X, float *Y) {
  constexpr int TPE = B / 2, SL = 256 / TPE;
  const int t = threadIdx.x % TPE, slot = threadIdx.x / TPE;
  float2 acc = make_float2(0.f, 0.f);
  for (int64_t e = rpl[blockIdx.x] + slot; e < rpl[blockIdx.x + 1]; e += SL) {
    const float w = vl[e];
    const float2 x = *reinterpret_cast<const float2 *>(X + (int64_t)cil[e] * B + 2 * t);
    acc.x = fmaf(w, x.x, acc.x);
    acc.y = fmaf(w, x.y, acc.y);
  }
  __shared__ float2 red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < TPE) {
    float2 sum = make_float2(0.f, 0.f);
    for (int k = 0; k < SL; ++k) {
      sum.x += red[k * TPE + threadIdx.x].x;
      sum.y += red[k * TPE + threadIdx.x].y;
    }
    *reinterpret_cast<float2 *>(Y + (int64_t)rows_l[blockIdx.x] * B + 2 * threadIdx.x) = sum;
  }
}

// 1 / phi_hat(x_i / G), phi_hat(s) = kw sinh(z)/z, z = sqrt(beta^2 - (pi kw s)^2)
__global__ void k_fub_deapod(int n, int G, int kw, double beta, float *d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = ((double)i + 0.5 - 0.5 * n) / (double)G;
  const double pk = 3.141592653589793 * kw * s;
  const double z = sqrt(beta * beta - pk * pk);
  d[i] = (float)(z / (kw * sinh(z)));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Phase tables, FP64 arguments reduced exactly, rounded to FP32 once:
//   grid  e^{i pi r / G},  r = (k (G - 1)) mod 2G  (= e^{2 pi i k (G/2 - 1/2)/G})
//   rad   e^{2 pi i (q - q0)(1/2 - c)/np}
//   bin   e^{2 pi i r / np}, r = (q0 k) mod np
__global__ void k_fub_tables(int G, int np, double c, float2 *ph_grid, float2 *ph_rad, float2 *ph_bin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s, co;
  if (i < G) {
    sincospi((double)(((int64_t)i * (G - 1)) % (2 * (int64_t)G)) / (double)G, &s, &co);
    ph_grid[i] = make_float2((float)co, (float)s);
  }
  if (i < np) {
    sincospi(2.0 * (double)(i - np / 2) * (0.5 - c) / (double)np, &s, &co);
    ph_rad[i] = make_float2((float)co, (float)s);
    sincospi(2.0 * (double)(((int64_t)(np / 2) * i) % np) / (double)np, &s, &co);
    ph_bin[i] = make_float2((float)co, (float)s);
  }
}

// forward 1: grid[s][gy][gx] = x[s][iy][ix] d[iy] d[ix] in the centre, 0 elsewhere
__global__ void k_fub_pad(const float *x, int cnt, int n, int G, const float *d, cufftComplex *grid, int Bf) {
  const int64_t total = (int64_t)Bf * G * G;
  const int o = (G - n) / 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((int64_t)G * G));
    const int gy = (int)((e / G) % G), gx = (int)(e % G);
    const int iy = gy - o, ix = gx - o;
    float val = 0.f;
    if (s < cnt && iy >= 0 && iy < n && ix >= 0 && ix < n) val = x[((int64_t)s * n + iy) * n + ix] * d[iy] * d[ix];
    grid[e] = make_float2(val, 0.f);
  }
}

// Slice-major complex data sm[s][i] (Bf x N) <-> interleaved (re, im) pairs
// il[i][s], times a per-point factor: a tiled transpose through shared memory
// so both sides are read and written coalesced.  kGrid: the factor is the grid
// phase ph[i / G] ph[i % G]; else the radial phase ph[i % np] times
// (w ? w[i % np] : 1) * scale.  kConj conjugates the phase (adjoint steps).
constexpr int kTile = 32;

template <bool kToIl, bool kGrid, bool kConj>
__global__ void __launch_bounds__(256) k_fub_transpose(cufftComplex *sm, float2 *il, int64_t N, int Bf,
                                                       const float2 *ph, int G, int np, const float *w, float scale) {
  __shared__ float2 tile[16][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;  // 32 x 8
  for (int64_t i0 = (int64_t)blockIdx.x * kTile; i0 < N; i0 += (int64_t)gridDim.x * kTile) {
    const int64_t i = i0 + tx;
    float2 f = make_float2(1.f, 0.f);
    if (i < N) {
      if (kGrid) {
        f = cmul(ph[i / G], ph[i % G]);
      } else {
        f = ph[i % np];
        const float sc = w ? w[i % np] * scale : scale;
        f = make_float2(f.x * sc, f.y * sc);
      }
      if (kConj) f = conjf2(f);
    }
    if (kToIl) {
      for (int s = ty; s < Bf; s += 8)
        if (i < N) tile[s][tx] = cmul(sm[(int64_t)s * N + i], f);
      __syncthreads();
      for (int l = threadIdx.x; l < kTile * Bf; l += 256) {
        const int ii = l / Bf, s = l % Bf;
        if (i0 + ii < N) il[(i0 + ii) * Bf + s] = tile[s][ii];
      }
    } else {
      for (int l = threadIdx.x; l < kTile * Bf; l += 256) {
        const int ii = l / Bf, s = l % Bf;
        if (i0 + ii < N) tile[s][ii] = il[(i0 + ii) * Bf + s];
      }
      __syncthreads();
      for (int s = ty; s < Bf; s += 8)
        if (i < N) sm[(int64_t)s * N + i] = cmul(tile[s][tx], f);
    }
    __syncthreads();
  }
}

// forward 7: y[s][m][k] = Re(pol[s][m][k] conj(ph_bin[k])) / np
__global__ void k_fub_out(const cufftComplex *pol, float *y, int cnt, int nt, int np, const float2 *ph_bin) {
  const int64_t total = (int64_t)cnt * nt * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % np);
    y[e] = cmul(pol[e], conjf2(ph_bin[k])).x / (float)np;
  }
}

// adjoint 1: pol[s][m][k] = y[s][m][k] ph_bin[k]
__global__ void k_fub_adj_in(const float *y, cufftComplex *pol, int cnt, int Bf, int nt, int np,
                             const float2 *ph_bin) {
  const int64_t total = (int64_t)Bf * nt * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((int64_t)nt * np));
    const int k = (int)(e % np);
    const float val = s < cnt ? y[e] : 0.f;
    const float2 ph = ph_bin[k];
    pol[e] = make_float2(val * ph.x, val * ph.y);
  }
}

// adjoint 7: x[s][iy][ix] = Re(grid[s][iy + o][ix + o]) d[iy] d[ix]
__global__ void k_fub_crop(const cufftComplex *grid, float *x, int cnt, int n, int G, const float *d) {
  const int64_t total = (int64_t)cnt * n * n;
  const int o = (G - n) / 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((int64_t)n * n));
    const int iy = (int)((e / n) % n), ix = (int)(e % n);
    x[e] = grid[((int64_t)s * G + iy + o) * G + ix + o].x * d[iy] * d[ix];
  }
}

// |w_q| with the DC sample weighted 1/(4 np) (the mean of |w| over its cell),
// and the same times the Hamming window 0.54 + 0.46 cos(2 pi w_q)
__global__ void k_fub_dens(int np, float *dens, float *dens_h) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int d = q - np / 2;
  const double r = d == 0 ? 1.0 / (4.0 * np) : fabs((double)d) / (double)np;
  dens[q] = (float)r;
  dens_h[q] = (float)(r * (0.54 + 0.46 * cospi(2.0 * (double)d / (double)np)));
}

// ---- the adjoint's last steps on power-of-two grids: the inverse 2D transform
// of the gridded spectrum, cropped to the image, in two register-FFT passes
// (regfft.cuh) that read and write only what the crop keeps:
//   columns  per (kx, 8 slices): c[ky] = gridI[ky G + kx][s] conj(ph[ky] ph[kx]),
//            inverse FFT over ky, rows gy in [o, o + n) -> T[s][kx][gy - o]
//   rows     per (slice, 8 image rows r): T[s][kx][r] over kx, inverse FFT,
//            columns gx in [o, o + n): x[s][r][gx - o] = Re(.) d[r] d[gx - o]
// Inputs are staged through shared memory so that global reads are whole rows.
constexpr int kFaSlices = 8;

template <int R1, int R2>
constexpr int fa_smem() {
  constexpr int stage = R1 * R2 * (kFaSlices + 1);
  constexpr int tiles = kFaSlices * (R1 * (R2 + 1) + 1);
  return (stage > tiles ? stage : tiles) * (int)sizeof(float2);
}

template <int R1, int R2>
__global__ void __launch_bounds__(kFaSlices *R2, (R1 <= 32 ? 3 : 1)) k_fa_cols(const float2 *gridI, int Bf, int cnt, int n,
                                                           const float2 *ph, float2 *T, const float2 *twL,
                                                           const __grid_constant__ Tw64 tw) {
  constexpr int G = R1 * R2;
  extern __shared__ float2 fa_sm[];
  // grid (slice groups, G): the groups of one column run next to each other,
  // so the second reads the other half of each 128-byte row from L2
  const int kx = blockIdx.y, q = threadIdx.x / R2, l = threadIdx.x % R2;
  const int s0 = blockIdx.x * kFaSlices, o = (G - n) / 2;
  for (int e = threadIdx.x; e < G * kFaSlices; e += blockDim.x) {
    const int ky = e / kFaSlices, qq = e % kFaSlices;
    fa_sm[ky * (kFaSlices + 1) + qq] =
        s0 + qq < cnt ? gridI[((int64_t)ky * G + kx) * Bf + s0 + qq] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2 pkx = conjf2(ph[kx]);
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) {
    const int ky = j1 * R2 + l;
    v[j1] = cmul(fa_sm[ky * (kFaSlices + 1) + q], cmul(conjf2(ph[ky]), pkx));
  }
  __syncthreads();
  fft_fwd<R1, R2, true>(v, w, fa_sm + q * (R1 * (R2 + 1) + 1), l, twL, tw);
  const int s = s0 + q;
  if (s >= cnt) return;
#pragma unroll
  for (int t = 0; t < R1 / R2; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int gy = (l + R2 * t) + R1 * k2;
      if (gy >= o && gy < o + n) T[((int64_t)s * G + kx) * n + gy - o] = w[t * R2 + k2];
    }
}

template <int R1, int R2>
__global__ void __launch_bounds__(kFaSlices *R2, (R1 <= 32 ? 3 : 1)) k_fa_rows(const float2 *T, int n, const float *d, float *x,
                                                           const float2 *twL, const __grid_constant__ Tw64 tw) {
  constexpr int G = R1 * R2;
  extern __shared__ float2 fa_sm[];
  const int s = blockIdx.y, r0 = blockIdx.x * kFaSlices, q = threadIdx.x / R2, l = threadIdx.x % R2;
  const int o = (G - n) / 2;
  for (int e = threadIdx.x; e < G * kFaSlices; e += blockDim.x) {
    const int kx = e / kFaSlices, qq = e % kFaSlices;
    fa_sm[kx * (kFaSlices + 1) + qq] =
        r0 + qq < n ? T[((int64_t)s * G + kx) * n + r0 + qq] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) v[j1] = fa_sm[(j1 * R2 + l) * (kFaSlices + 1) + q];
  __syncthreads();
  fft_fwd<R1, R2, true>(v, w, fa_sm + q * (R1 * (R2 + 1) + 1), l, twL, tw);
  const int r = r0 + q;
  if (r >= n) return;
  const float dr = d[r];
  float *xr = x + ((int64_t)s * n + r) * n;
#pragma unroll
  for (int t = 0; t < R1 / R2; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int gx = (l + R2 * t) + R1 * k2;
      if (gx >= o && gx < o + n) xr[gx - o] = w[t * R2 + k2].x * dr * d[gx - o];
    }
}

// ---- the forward transform's first steps on power-of-two grids: deapodize,
// zero-pad and transform the image in two register-FFT passes that touch only
// the image's rows and write the grid straight into the SpMM layout:
//   rows     per (slice, 8 image rows iy): u[iy][gx - o] d[iy] d[gx - o] over the
//            padded row, FFT -> T[s][kx][iy]
//   columns  per (kx, 8 slices): T[s][kx][gy - o] over the padded column, FFT,
//            the grid phase ph[ky] ph[kx] -> gridI[ky G + kx][s]
// Outputs are staged through shared memory so that global writes are whole rows.
template <int R1, int R2>
__global__ void __launch_bounds__(kFaSlices *R2, (R1 <= 32 ? 3 : 1)) k_ff_rows(const float *u, int n, const float *d, float2 *T,
                                                           const float2 *twL, const __grid_constant__ Tw64 tw) {
  constexpr int G = R1 * R2;
  extern __shared__ float2 fa_sm[];
  const int s = blockIdx.y, iy0 = blockIdx.x * kFaSlices, q = threadIdx.x / R2, l = threadIdx.x % R2;
  const int o = (G - n) / 2, iy = iy0 + q;
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) {
    const int gx = j1 * R2 + l;
    float val = 0.f;
    if (iy < n && gx >= o && gx < o + n) val = u[((int64_t)s * n + iy) * n + gx - o] * d[iy] * d[gx - o];
    v[j1] = make_float2(val, 0.f);
  }
  fft_fwd<R1, R2, false>(v, w, fa_sm + q * (R1 * (R2 + 1) + 1), l, twL, tw);
  __syncthreads();  // every group is done with its tile: the staging area overlaps them
#pragma unroll
  for (int t = 0; t < R1 / R2; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) fa_sm[((l + R2 * t) + R1 * k2) * (kFaSlices + 1) + q] = w[t * R2 + k2];
  __syncthreads();
  for (int e = threadIdx.x; e < G * kFaSlices; e += blockDim.x) {
    const int kx = e / kFaSlices, qq = e % kFaSlices;
    if (iy0 + qq < n) T[((int64_t)s * G + kx) * n + iy0 + qq] = fa_sm[kx * (kFaSlices + 1) + qq];
  }
}

// grid (ceil(Bf / 8), G): slices cnt .. Bf - 1 of the pass get zero columns
template <int R1, int R2>
__global__ void __launch_bounds__(kFaSlices *R2, (R1 <= 32 ? 3 : 1)) k_ff_cols(const float2 *T, int Bf, int cnt, int n,
                                                           const float2 *ph, float2 *gridI, const float2 *twL,
                                                           const __grid_constant__ Tw64 tw) {
  constexpr int G = R1 * R2;
  extern __shared__ float2 fa_sm[];
  const int kx = blockIdx.y, s0 = blockIdx.x * kFaSlices, q = threadIdx.x / R2, l = threadIdx.x % R2;
  const int o = (G - n) / 2, s = s0 + q;
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) {
    const int gy = j1 * R2 + l;
    v[j1] = (s < cnt && gy >= o && gy < o + n) ? T[((int64_t)s * G + kx) * n + gy - o] : make_float2(0.f, 0.f);
  }
  fft_fwd<R1, R2, false>(v, w, fa_sm + q * (R1 * (R2 + 1) + 1), l, twL, tw);
  const float2 pkx = ph[kx];
  __syncthreads();
#pragma unroll
  for (int t = 0; t < R1 / R2; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int ky = (l + R2 * t) + R1 * k2;
      fa_sm[ky * (kFaSlices + 1) + q] = cmul(w[t * R2 + k2], cmul(ph[ky], pkx));
    }
  __syncthreads();
  for (int e = threadIdx.x; e < G * kFaSlices; e += blockDim.x) {
    const int ky = e / kFaSlices, qq = e % kFaSlices;
    if (s0 + qq < Bf) gridI[((int64_t)ky * G + kx) * Bf + s0 + qq] = fa_sm[ky * (kFaSlices + 1) + qq];
  }
}

int tgrid(int64_t points) {
  const int64_t b = (points + kTile - 1) / kTile;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 16));
}

int egrid(int64_t n) {
  int64_t b = (n + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 16));
}

tomo_status cufft_check(cufftResult r, const char *what) {
  if (r != CUFFT_SUCCESS) return fail(TOMO_ERR_CUDA, std::string("cuFFT ") + what + " failed: " + std::to_string((int)r));
  return TOMO_OK;
}

template <class T>
tomo_status dalloc(T **p, size_t count) {
  if (cudaMalloc(p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TOMO_ERR_OOM, "device allocation of " + std::to_string(sizeof(T) * count) + " bytes failed");
  }
  return TOMO_OK;
}

void free_fubini(tomo_fubini *F) {
  if (!F) return;
  if (F->has_plan2) cufftDestroy(F->plan2);
  if (F->has_plan1) cufftDestroy(F->plan1);
  free_normal(F);
  void *ptrs[] = {F->S.rp, F->S.ci, F->S.v, F->STs.rp, F->STs.ci, F->STs.v, F->STl.rp, F->STl.ci, F->STl.v,
                  F->rows_l, F->faT, F->deapod, F->dens, F->dens_h, F->grid, F->gridI,
                  F->polI, F->pol, F->ph_grid, F->ph_rad, F->ph_bin, F->cs, F->sn, F->twP};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete F;
}

tomo_status long_rows(tomo_fubini *F, const float *X, float *Y, cudaStream_t st) {
  const unsigned nb = (unsigned)F->STl.rows;
  if (nb == 0) return TOMO_OK;
  const Csr &M = F->STl;
  switch (2 * F->Bf) {
    case 2: k_fub_long_spmm<2><<<nb, 256, 0, st>>>(M.rp, M.ci, M.v, F->rows_l, X, Y); break;
    case 4: k_fub_long_spmm<4><<<nb, 256, 0, st>>>(M.rp, M.ci, M.v, F->rows_l, X, Y); break;
    case 8: k_fub_long_spmm<8><<<nb, 256, 0, st>>>(M.rp, M.ci, M.v, F->rows_l, X, Y); break;
    case 16: k_fub_long_spmm<16><<<nb, 256, 0, st>>>(M.rp, M.ci, M.v, F->rows_l, X, Y); break;
    case 32: k_fub_long_spmm<32><<<nb, 256, 0, st>>>(M.rp, M.ci, M.v, F->rows_l, X, Y); break;
    default: return fail(TOMO_ERR_UNSUPPORTED, "Fubini batch width must be 1..16 slices");
  }
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

template <int R1, int R2>
tomo_status fa_run(tomo_fubini *F, int cnt, float *x, cudaStream_t st) {
  constexpr int G = R1 * R2, sm = fa_smem<R1, R2>();
  TOMO_CUDA(cudaFuncSetAttribute(k_fa_cols<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  TOMO_CUDA(cudaFuncSetAttribute(k_fa_rows<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  const Tw64 tw = tw64();
  k_fa_cols<R1, R2><<<dim3((cnt + kFaSlices - 1) / kFaSlices, G), kFaSlices * R2, sm, st>>>(
      (const float2 *)F->gridI, F->Bf, cnt, F->n, F->ph_grid, F->faT, F->twL, tw);
  k_fa_rows<R1, R2><<<dim3((F->n + kFaSlices - 1) / kFaSlices, cnt), kFaSlices * R2, sm, st>>>(
      F->faT, F->n, F->deapod, x, F->twL, tw);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

template <int R1, int R2>
tomo_status ff_run(tomo_fubini *F, int cnt, const float *u, cudaStream_t st) {
  constexpr int G = R1 * R2, sm = fa_smem<R1, R2>();
  TOMO_CUDA(cudaFuncSetAttribute(k_ff_rows<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  TOMO_CUDA(cudaFuncSetAttribute(k_ff_cols<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  const Tw64 tw = tw64();
  k_ff_rows<R1, R2><<<dim3((F->n + kFaSlices - 1) / kFaSlices, cnt), kFaSlices * R2, sm, st>>>(
      u, F->n, F->deapod, F->faT, F->twL, tw);
  k_ff_cols<R1, R2><<<dim3((F->Bf + kFaSlices - 1) / kFaSlices, G), kFaSlices * R2, sm, st>>>(
      F->faT, F->Bf, cnt, F->n, F->ph_grid, (float2 *)F->gridI, F->twL, tw);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

// the forward transform's deapodize, pad and 2D FFT by register FFTs (G a power of two, 32..2048)
tomo_status ff_dispatch(tomo_fubini *F, int cnt, const float *u, cudaStream_t st) {
  switch (F->G) {
    case 32: return ff_run<8, 4>(F, cnt, u, st);
    case 64: return ff_run<8, 8>(F, cnt, u, st);
    case 128: return ff_run<16, 8>(F, cnt, u, st);
    case 256: return ff_run<16, 16>(F, cnt, u, st);
    case 512: return ff_run<32, 16>(F, cnt, u, st);
    case 1024: return ff_run<32, 32>(F, cnt, u, st);
    case 2048: return ff_run<64, 32>(F, cnt, u, st);
  }
  return fail(TOMO_ERR_INVALID_ARG, "no register-FFT forward for this grid");
}

// the adjoint's inverse 2D transform and crop by register FFTs (G a power of two, 32..2048)
tomo_status fa_dispatch(tomo_fubini *F, int cnt, float *x, cudaStream_t st) {
  switch (F->G) {
    case 32: return fa_run<8, 4>(F, cnt, x, st);
    case 64: return fa_run<8, 8>(F, cnt, x, st);
    case 128: return fa_run<16, 8>(F, cnt, x, st);
    case 256: return fa_run<16, 16>(F, cnt, x, st);
    case 512: return fa_run<32, 16>(F, cnt, x, st);
    case 1024: return fa_run<32, 32>(F, cnt, x, st);
    case 2048: return fa_run<64, 32>(F, cnt, x, st);
  }
  return fail(TOMO_ERR_INVALID_ARG, "no register-FFT adjoint for this grid");
}

// ---- the radial 1D transforms by register FFTs (n_p a power of two, 32..1024) ----
// A block takes angle m and SB = 256 / R2 consecutive slices, one FFT of
// length L = n_p per group of R2 lanes.  The slice-interleaved rows of polI
// (SB slices of one row are 8 SB contiguous bytes) pass through a shared
// staging area of SB rows of L + 1 (the pad spreads a row's slices over the
// banks); the FFT tiles of regfft.cuh reuse the same memory afterwards.
inline bool radial_ok(int np) { return np >= 32 && np <= 1024 && (np & (np - 1)) == 0; }

template <int R1, int R2>
constexpr int rad_smem() {
  constexpr int L = R1 * R2, SB = 256 / R2;
  constexpr int stage = SB * (L + 1) * (int)sizeof(float2);
  constexpr int tiles = SB * (R1 * (R2 + 1) + 1) * (int)sizeof(float2);
  return stage > tiles ? stage : tiles;
}

// forward, after the gridding SpMM (steps 5-7): z[q] = polI[m np + q][s]
// ph_rad[q], Z = its unnormalised inverse DFT, y[s][m][k] = Re(Z[k]
// conj(ph_bin[k])) / np -- the transpose, the inverse 1D FFT and k_fub_out
template <int R1, int R2>
__global__ void __launch_bounds__(256) k_fub_rad_fwd(const float2 *__restrict__ polI, float *__restrict__ y, int cnt,
                                                     int Bf, int nt, const float2 *__restrict__ ph_rad,
                                                     const float2 *__restrict__ ph_bin, const float2 *twP,
                                                     const __grid_constant__ Tw64 tw) {
  constexpr int L = R1 * R2, G = R2, SB = 256 / G, T = R1 / G;
  extern __shared__ float2 rad_sm[];
  const int m = blockIdx.x, s0 = blockIdx.y * SB;
  if (s0 >= cnt) return;  // the whole block: no slice of it is written
  for (int e = threadIdx.x; e < L * SB; e += 256) {
    const int q = e / SB, sl = e % SB;
    const float2 z = s0 + sl < Bf ? polI[((int64_t)m * L + q) * Bf + s0 + sl] : make_float2(0.f, 0.f);
    rad_sm[sl * (L + 1) + q] = cmulf(z, __ldg(ph_rad + q));
  }
  __syncthreads();
  const int g = threadIdx.x / G, l = threadIdx.x % G;
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) v[j1] = rad_sm[g * (L + 1) + j1 * R2 + l];
  __syncthreads();  // the FFT tiles overwrite the staging area
  fft_fwd<R1, R2, true>(v, w, rad_sm + g * (R1 * (R2 + 1) + 1), l, twP, tw);
  const int s = s0 + g;
  if (s < cnt) {
    float *yr = y + ((int64_t)s * nt + m) * L;
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int k = (l + G * t) + R1 * k2;
        const float2 z = w[t * R2 + k2], pb = __ldg(ph_bin + k);
        yr[k] = (z.x * pb.x + z.y * pb.y) / (float)L;
      }
  }
}

// adjoint (steps 1-3): u[k] = y[s][m][k] ph_bin[k] (0 for slices >= cnt),
// P = its forward DFT, polI[m np + q][s] = P[q] conj(ph_rad[q] f[q]) with
// f = (w ? w[q] : 1) scale -- k_fub_adj_in, the forward 1D FFT and the
// transpose; every slice of the batch is written (zeros past cnt)
template <int R1, int R2>
__global__ void __launch_bounds__(256) k_fub_rad_adj(const float *__restrict__ y, float2 *__restrict__ polI, int cnt,
                                                     int Bf, int nt, const float2 *__restrict__ ph_rad,
                                                     const float2 *__restrict__ ph_bin, const float *__restrict__ wq,
                                                     float scale, const float2 *twP, const __grid_constant__ Tw64 tw) {
  constexpr int L = R1 * R2, G = R2, SB = 256 / G, T = R1 / G;
  extern __shared__ float2 rad_sm[];
  const int m = blockIdx.x, s0 = blockIdx.y * SB;
  const int g = threadIdx.x / G, l = threadIdx.x % G, s = s0 + g;
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) {
    const int k = j1 * R2 + l;
    const float val = s < cnt ? y[((int64_t)s * nt + m) * L + k] : 0.f;
    const float2 pb = __ldg(ph_bin + k);
    v[j1] = make_float2(val * pb.x, val * pb.y);
  }
  fft_fwd<R1, R2, false>(v, w, rad_sm + g * (R1 * (R2 + 1) + 1), l, twP, tw);
  __syncthreads();  // every group is done with its tile: the staging area takes the spectra
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int q = (l + G * t) + R1 * k2;
      float2 f = __ldg(ph_rad + q);
      const float sc = wq ? __ldg(wq + q) * scale : scale;
      f = make_float2(f.x * sc, -f.y * sc);
      rad_sm[g * (L + 1) + q] = cmulf(w[t * R2 + k2], f);
    }
  __syncthreads();
  for (int e = threadIdx.x; e < L * SB; e += 256) {
    const int q = e / SB, sl = e % SB;
    if (s0 + sl < Bf) polI[((int64_t)m * L + q) * Bf + s0 + sl] = rad_sm[sl * (L + 1) + q];
  }
}

template <int R1, int R2>
tomo_status rad_run(tomo_fubini *F, bool adj, int cnt, const float *y_in, float *y_out, const float *wq, float scale,
                    cudaStream_t st) {
  constexpr int sm = rad_smem<R1, R2>(), SB = 256 / R2;
  const Tw64 tw = tw64();
  const dim3 grid(F->nt, (F->Bf + SB - 1) / SB);
  if (adj) {
    TOMO_CUDA(cudaFuncSetAttribute(k_fub_rad_adj<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    k_fub_rad_adj<R1, R2><<<grid, 256, sm, st>>>(y_in, (float2 *)F->polI, cnt, F->Bf, F->nt, F->ph_rad, F->ph_bin,
                                                 wq, scale, F->twP, tw);
  } else {
    TOMO_CUDA(cudaFuncSetAttribute(k_fub_rad_fwd<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    k_fub_rad_fwd<R1, R2><<<grid, 256, sm, st>>>((const float2 *)F->polI, y_out, cnt, F->Bf, F->nt, F->ph_rad,
                                                 F->ph_bin, F->twP, tw);
  }
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status rad_dispatch(tomo_fubini *F, bool adj, int cnt, const float *y_in, float *y_out, const float *wq,
                         float scale, cudaStream_t st) {
  switch (F->np) {
    case 32: return rad_run<8, 4>(F, adj, cnt, y_in, y_out, wq, scale, st);
    case 64: return rad_run<8, 8>(F, adj, cnt, y_in, y_out, wq, scale, st);
    case 128: return rad_run<16, 8>(F, adj, cnt, y_in, y_out, wq, scale, st);
    case 256: return rad_run<16, 16>(F, adj, cnt, y_in, y_out, wq, scale, st);
    case 512: return rad_run<32, 16>(F, adj, cnt, y_in, y_out, wq, scale, st);
    case 1024: return rad_run<32, 32>(F, adj, cnt, y_in, y_out, wq, scale, st);
  }
  return fail(TOMO_ERR_INVALID_ARG, "no register-FFT radial transform for this n_p");
}

}  // namespace

tomo_status fubini_create(const tomo_geometry *g, int32_t kw, cudaStream_t st, tomo_fubini **out) {
  if (!g || !out) return fail(TOMO_ERR_INVALID_ARG, "geometry and out must be non-NULL");
  *out = nullptr;
  if (g->n_x <= 0 || g->n_x != g->n_y || g->n_p <= 0 || g->n_theta <= 0)
    return fail(TOMO_ERR_INVALID_ARG, "the Fubini-Radon transform needs a square image (n_x == n_y > 0), n_p, n_theta > 0");
  if (kw < 2 || kw > 16 || (kw & 1)) return fail(TOMO_ERR_INVALID_ARG, "kw must be even, 2..16");
  const int64_t G = 2 * (int64_t)g->n_x;
  if (G * G >= (int64_t)INT32_MAX || (int64_t)g->n_theta * g->n_p * kw * kw >= (int64_t)INT32_MAX * 4)
    return fail(TOMO_ERR_INVALID_ARG, "geometry too large for the Fubini-Radon transform");
  const double c = std::isnan(g->center) ? 0.5 * (double)g->n_p : g->center;
  if (!std::isfinite(c)) return fail(TOMO_ERR_INVALID_ARG, "center must be finite or NaN");
  std::vector<double> cs(g->n_theta), sn(g->n_theta);
  for (int m = 0; m < g->n_theta; ++m) {
    const double th = g->angles ? g->angles[m] : (double)m * M_PI / (double)g->n_theta;
    if (!std::isfinite(th)) return fail(TOMO_ERR_INVALID_ARG, "angles must be finite");
    cs[m] = std::cos(th);
    sn[m] = std::sin(th);
  }
  tomo_fubini *F = new tomo_fubini();
  struct Guard {
    tomo_fubini *F;
    bool keep = false;
    ~Guard() {
      if (!keep) free_fubini(F);
    }
  } guard{F};
  cudaGetDevice(&F->device);
  F->n = g->n_x;
  F->default_angles = g->angles == nullptr;
  F->np = g->n_p;
  F->nt = g->n_theta;
  F->kw = kw;
  F->G = (int32_t)G;
  F->center = c;
  const double sigma = 2.0;
  F->beta = M_PI * std::sqrt((kw / sigma) * (kw / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
  // batch of slices per pass: 16, fewer when the grid would pass 2 GiB
  F->Bf = 16;
  while (F->Bf > 1 && (int64_t)G * G * F->Bf * 16 > (int64_t)2 << 30) F->Bf /= 2;

  const int64_t rows = (int64_t)F->nt * F->np, cols = G * G, nnz = rows * kw * kw;
  TOMO_TRY(dalloc(&F->cs, F->nt));
  TOMO_TRY(dalloc(&F->sn, F->nt));
  double *dcs = F->cs, *dsn = F->sn;
  TOMO_CUDA(cudaMemcpyAsync(dcs, cs.data(), sizeof(double) * F->nt, cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemcpyAsync(dsn, sn.data(), sizeof(double) * F->nt, cudaMemcpyHostToDevice, st));
  F->S.rows = rows;
  F->S.cols = cols;
  F->S.nnz = nnz;
  F->S.max_len = (int64_t)kw * kw;
  TOMO_TRY(dalloc(&F->S.rp, rows + 1));
  TOMO_TRY(dalloc(&F->S.ci, nnz));
  TOMO_TRY(dalloc(&F->S.v, nnz));
  k_fub_fill_S<<<(unsigned)((rows + kT - 1) / kT), kT, 0, st>>>(dcs, dsn, F->nt, F->np, F->G, kw, F->beta, F->S.rp,
                                                                 F->S.ci, F->S.v);
  TOMO_CUDA(cudaGetLastError());
  // S^T: counting-sort transpose, then split into its short and long rows
  {
    Csr T;  // the whole transpose, unsorted rows; freed here
    int32_t *cnt = nullptr, *flag = nullptr, *cnt_l = nullptr;
    int64_t *lpos = nullptr;
    struct Tmp2 {
      Csr *T;
      int32_t **c, **f, **cl;
      int64_t **lp;
      ~Tmp2() {
        for (void *q : {(void *)T->rp, (void *)T->ci, (void *)T->v, (void *)*c, (void *)*f, (void *)*cl, (void *)*lp})
          if (q) cudaFree(q);
      }
    } tmp2{&T, &cnt, &flag, &cnt_l, &lpos};
    TOMO_TRY(dalloc(&T.rp, cols + 1));
    TOMO_TRY(dalloc(&T.ci, nnz));
    TOMO_TRY(dalloc(&T.v, nnz));
    TOMO_TRY(dalloc(&cnt, cols));
    TOMO_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * cols, st));
    k_fub_count<<<egrid(nnz), kT, 0, st>>>(F->S.ci, nnz, cnt);
    TOMO_CUDA(cudaGetLastError());
    TOMO_TRY(exclusive_scan_i32(cnt, cols, T.rp, st));
    TOMO_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * cols, st));
    k_fub_scatter<<<egrid(nnz), kT, 0, st>>>(F->S.ci, F->S.v, rows, kw * kw, T.rp, cnt, T.ci, T.v);
    TOMO_CUDA(cudaGetLastError());
    TOMO_TRY(dalloc(&flag, cols));
    TOMO_TRY(dalloc(&lpos, cols + 1));
    k_fub_split_count<<<(unsigned)((cols + kT - 1) / kT), kT, 0, st>>>(T.rp, cols, cnt, flag);
    TOMO_CUDA(cudaGetLastError());
    F->STs.rows = cols;
    F->STs.cols = rows;
    TOMO_TRY(dalloc(&F->STs.rp, cols + 1));
    TOMO_TRY(exclusive_scan_i32(cnt, cols, F->STs.rp, st));
    TOMO_TRY(exclusive_scan_i32(flag, cols, lpos, st));
    int64_t nl = 0;
    TOMO_CUDA(cudaMemcpyAsync(&F->STs.nnz, F->STs.rp + cols, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TOMO_CUDA(cudaMemcpyAsync(&nl, lpos + cols, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TOMO_CUDA(cudaStreamSynchronize(st));
    F->STs.max_len = kLongRow;
    TOMO_TRY(dalloc(&F->STs.ci, F->STs.nnz));
    TOMO_TRY(dalloc(&F->STs.v, F->STs.nnz));
    k_fub_copy_short<<<(unsigned)((cols + kT - 1) / kT), kT, 0, st>>>(T.rp, T.ci, T.v, cols, F->STs.rp, F->STs.ci,
                                                                       F->STs.v);
    TOMO_CUDA(cudaGetLastError());
    F->STl.rows = nl;
    F->STl.cols = rows;
    TOMO_TRY(dalloc(&F->STl.rp, nl + 1));
    TOMO_TRY(dalloc(&F->rows_l, nl));
    TOMO_TRY(dalloc(&cnt_l, nl));
    if (nl > 0) {
      k_fub_long_list<<<(unsigned)((cols + kT - 1) / kT), kT, 0, st>>>(T.rp, lpos, cols, F->rows_l, cnt_l);
      TOMO_CUDA(cudaGetLastError());
    }
    if (nl > 0) {
      TOMO_TRY(exclusive_scan_i32(cnt_l, nl, F->STl.rp, st));
      TOMO_CUDA(cudaMemcpyAsync(&F->STl.nnz, F->STl.rp + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      TOMO_CUDA(cudaStreamSynchronize(st));
    } else {
      TOMO_CUDA(cudaMemsetAsync(F->STl.rp, 0, sizeof(int64_t), st));
      F->STl.nnz = 0;
    }
    TOMO_TRY(dalloc(&F->STl.ci, F->STl.nnz));
    TOMO_TRY(dalloc(&F->STl.v, F->STl.nnz));
    if (nl > 0) {
      k_fub_copy_long<<<(unsigned)nl, kT, 0, st>>>(T.rp, T.ci, T.v, F->rows_l, F->STl.rp, F->STl.ci, F->STl.v);
      TOMO_CUDA(cudaGetLastError());
    }
    TOMO_CUDA(cudaStreamSynchronize(st));  // the temporaries are freed here
  }
  // factors and buffers
  TOMO_TRY(dalloc(&F->deapod, F->n));
  k_fub_deapod<<<(F->n + kT - 1) / kT, kT, 0, st>>>(F->n, F->G, kw, F->beta, F->deapod);
  TOMO_TRY(dalloc(&F->dens, F->np));
  TOMO_TRY(dalloc(&F->dens_h, F->np));
  k_fub_dens<<<(F->np + kT - 1) / kT, kT, 0, st>>>(F->np, F->dens, F->dens_h);
  TOMO_TRY(dalloc(&F->ph_grid, F->G));
  TOMO_TRY(dalloc(&F->ph_rad, F->np));
  TOMO_TRY(dalloc(&F->ph_bin, F->np));
  k_fub_tables<<<(std::max(F->G, F->np) + kT - 1) / kT, kT, 0, st>>>(F->G, F->np, c, F->ph_grid, F->ph_rad,
                                                                      F->ph_bin);
  TOMO_CUDA(cudaGetLastError());
  TOMO_TRY(dalloc(&F->gridI, (size_t)G * G * F->Bf * 2));
  TOMO_TRY(dalloc(&F->polI, (size_t)rows * F->Bf * 2));
  if (fused_ok(F->G)) {  // the adjoint's inverse 2D transform by register FFTs
    TOMO_TRY(ensure_twiddles(F, st));
    TOMO_TRY(dalloc(&F->faT, (size_t)F->Bf * F->G * F->n));
  }
  if (radial_ok(F->np)) {  // the radial 1D transforms by register FFTs
    const int R2 = fft_r2(F->np), R1 = F->np / R2;
    TOMO_TRY(dalloc(&F->twP, (size_t)2 * F->np));
    k_fft_twiddles<<<(2 * F->np + kT - 1) / kT, kT, 0, st>>>(R1, R2, F->twP);
    TOMO_CUDA(cudaGetLastError());
  }
  // cuFFT plans and their buffers, only for the sizes the register-FFT passes
  // do not take: G x G 2D transforms and length-np 1D transforms, contiguous batches
  if (!F->faT) {
    TOMO_TRY(dalloc(&F->grid, (size_t)G * G * F->Bf));
    int dims2[2] = {F->G, F->G};
    TOMO_TRY(cufft_check(cufftPlanMany(&F->plan2, 2, dims2, nullptr, 1, F->G * F->G, nullptr, 1, F->G * F->G,
                                       CUFFT_C2C, F->Bf), "plan 2D"));
    F->has_plan2 = true;
  }
  if (!F->twP) {
    TOMO_TRY(dalloc(&F->pol, (size_t)rows * F->Bf));
    int dims1[1] = {F->np};
    TOMO_TRY(cufft_check(cufftPlanMany(&F->plan1, 1, dims1, nullptr, 1, F->np, nullptr, 1, F->np, CUFFT_C2C,
                                       F->nt * F->Bf), "plan 1D"));
    F->has_plan1 = true;
  }
  TOMO_CUDA(cudaStreamSynchronize(st));
  guard.keep = true;
  *out = F;
  return TOMO_OK;
}

void fubini_destroy(tomo_fubini *F) { free_fubini(F); }

tomo_status fubini_project(tomo_fubini *F, const float *x, float *y, int32_t nz, cudaStream_t st) {
  const int G = F->G, n = F->n, nt = F->nt, np = F->np, Bf = F->Bf;
  const int64_t rows = (int64_t)nt * np;
  if (F->has_plan2) TOMO_TRY(cufft_check(cufftSetStream(F->plan2, st), "set stream"));
  if (F->has_plan1) TOMO_TRY(cufft_check(cufftSetStream(F->plan1, st), "set stream"));
  for (int32_t s0 = 0; s0 < nz; s0 += Bf) {
    const int cnt = std::min<int32_t>(Bf, nz - s0);
    if (F->faT) {
      TOMO_TRY(ff_dispatch(F, cnt, x + (int64_t)s0 * n * n, st));
    } else {
      k_fub_pad<<<egrid((int64_t)Bf * G * G), kT, 0, st>>>(x + (int64_t)s0 * n * n, cnt, n, G, F->deapod, F->grid,
                                                            Bf);
      TOMO_TRY(cufft_check(cufftExecC2C(F->plan2, F->grid, F->grid, CUFFT_FORWARD), "2D forward"));
      k_fub_transpose<true, true, false><<<tgrid((int64_t)G * G), 256, 0, st>>>(
          F->grid, (float2 *)F->gridI, (int64_t)G * G, Bf, F->ph_grid, G, np, nullptr, 1.f);
    }
    TOMO_TRY(spmm_csr_store(F->S, 2 * Bf, F->gridI, F->polI, st));
    if (F->twP) {  // steps 5-7 in one pass of register FFTs
      TOMO_TRY(rad_dispatch(F, false, cnt, nullptr, y + (int64_t)s0 * rows, nullptr, 1.f, st));
      continue;
    }
    k_fub_transpose<false, false, false><<<tgrid(rows), 256, 0, st>>>(F->pol, (float2 *)F->polI, rows, Bf, F->ph_rad,
                                                               G, np, nullptr, 1.f);
    TOMO_TRY(cufft_check(cufftExecC2C(F->plan1, F->pol, F->pol, CUFFT_INVERSE), "1D inverse"));
    k_fub_out<<<egrid(rows * cnt), kT, 0, st>>>(F->pol, y + (int64_t)s0 * rows, cnt, nt, np, F->ph_bin);
    TOMO_CUDA(cudaGetLastError());
  }
  return TOMO_OK;
}

tomo_status fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t nz, int filter, cudaStream_t st) {
  const int G = F->G, n = F->n, nt = F->nt, np = F->np, Bf = F->Bf;
  const int64_t rows = (int64_t)nt * np;
  if (F->has_plan2) TOMO_TRY(cufft_check(cufftSetStream(F->plan2, st), "set stream"));
  if (F->has_plan1) TOMO_TRY(cufft_check(cufftSetStream(F->plan1, st), "set stream"));
  const float scale = filter ? (float)(M_PI / ((double)np * nt)) : (float)(1.0 / np);
  const float *dens = filter == 1 ? F->dens : (filter == 2 ? F->dens_h : nullptr);
  for (int32_t s0 = 0; s0 < nz; s0 += Bf) {
    const int cnt = std::min<int32_t>(Bf, nz - s0);
    if (F->twP) {  // steps 1-3 in one pass of register FFTs
      TOMO_TRY(rad_dispatch(F, true, cnt, y + (int64_t)s0 * rows, nullptr, dens, scale, st));
    } else {
      k_fub_adj_in<<<egrid(rows * Bf), kT, 0, st>>>(y + (int64_t)s0 * rows, F->pol, cnt, Bf, nt, np, F->ph_bin);
      TOMO_TRY(cufft_check(cufftExecC2C(F->plan1, F->pol, F->pol, CUFFT_FORWARD), "1D forward"));
      k_fub_transpose<true, false, true><<<tgrid(rows), 256, 0, st>>>(F->pol, (float2 *)F->polI, rows, Bf, F->ph_rad,
                                                                G, np, dens, scale);
    }
    TOMO_TRY(spmm_csr_store(F->STs, 2 * Bf, F->polI, F->gridI, st));  // long rows come out 0 ...
    TOMO_TRY(long_rows(F, F->polI, F->gridI, st));                    // ... and are written here
    if (F->faT) {
      TOMO_TRY(fa_dispatch(F, cnt, x + (int64_t)s0 * n * n, st));
      continue;
    }
    k_fub_transpose<false, true, true><<<tgrid((int64_t)G * G), 256, 0, st>>>(F->grid, (float2 *)F->gridI, (int64_t)G * G,
                                                                          Bf, F->ph_grid, G, np, nullptr, 1.f);
    TOMO_TRY(cufft_check(cufftExecC2C(F->plan2, F->grid, F->grid, CUFFT_INVERSE), "2D inverse"));
    k_fub_crop<<<egrid((int64_t)cnt * n * n), kT, 0, st>>>(F->grid, x + (int64_t)s0 * n * n, cnt, n, G, F->deapod);
    TOMO_CUDA(cudaGetLastError());
  }
  return TOMO_OK;
}

tomo_status fubini_sirt_bb(tomo_fubini *F, const float *sino, float *x, int32_t nz, int32_t iters, double *hist,
                           cudaStream_t st) {
  // The paper's SIRT on this operator, per slice: r = b - R x (||r|| ->
  // hist[k]), g = iRadon_Hamming(r), the BB step from <gp,gp> and
  // <gp, g - gp> (alpha = 1 first), x += alpha g.  Sums over a fixed split of
  // each slice into NB blocks (bbstep.cuh).
  const int64_t rows = (int64_t)F->nt * F->np, cols = (int64_t)F->n * F->n;
  constexpr int NB = 32;
  if (nz > 65535) return fail(TOMO_ERR_INVALID_ARG, "n_z must be <= 65535");
  float *y = nullptr, *g0 = nullptr, *g1 = nullptr, *alpha = nullptr;
  double *scal = nullptr;
  double3 *part = nullptr;
  auto alloc = [&](void **p, size_t b) -> tomo_status {
    if (cudaMallocAsync(p, b, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(TOMO_ERR_OOM, "workspace allocation of " + std::to_string(b) + " bytes failed");
    }
    return TOMO_OK;
  };
  struct Free {
    void **p[6];
    cudaStream_t st;
    ~Free() {
      for (void **q : p)
        if (*q) cudaFreeAsync(*q, st);
    }
  } fr{{(void **)&y, (void **)&g0, (void **)&g1, (void **)&scal, (void **)&part, (void **)&alpha}, st};
  TOMO_TRY(alloc((void **)&y, sizeof(float) * rows * nz));
  TOMO_TRY(alloc((void **)&g0, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&g1, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&scal, sizeof(double) * 8 * nz));
  TOMO_TRY(alloc((void **)&part, sizeof(double3) * NB * nz));
  TOMO_TRY(alloc((void **)&alpha, sizeof(float) * nz));
  TOMO_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * cols * nz, st));
  TOMO_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 8 * nz, st));
  float *g = g0, *gp = nullptr;
  const int per = (int)std::min<int64_t>(64, (cols + kT - 1) / kT);
  for (int32_t k = 0; k < iters; ++k) {
    TOMO_TRY(fubini_project(F, x, y, nz, st));
    k_bb_resid<<<dim3(NB, nz), kT, 0, st>>>(sino, y, rows, NB, part);
    TOMO_TRY(fubini_backproject(F, y, g, nz, 2, st));
    k_bb_dots<<<dim3(NB, nz), kT, 0, st>>>(g, gp, cols, NB, part);
    k_bb_alpha<<<nz, 32, 0, st>>>(part, NB, scal + (k & 1) * 4 * nz, scal + ((k + 1) & 1) * 4 * nz, hist, k, nz,
                                  alpha);
    k_bb_axpy<<<dim3(per, nz), kT, 0, st>>>(x, g, alpha, cols);
    TOMO_CUDA(cudaGetLastError());
    gp = g;
    g = g == g0 ? g1 : g0;
  }
  return TOMO_OK;
}

}  // namespace tomo
