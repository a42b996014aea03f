// normal.cu -- the normal operator of the Fubini-Radon transform in one step
// (the Toeplitz route of the outlook in Sec. 5, which joins the transform and
// its adjoint and drops the 1D transforms).
//
// N = R^T W R for the exact transform R of real n x n images, with W the
// sinogram weight of the plain adjoint (filter 0), of the ramp (1) or of the
// Hamming-windowed ramp (2) filtered backprojection.  Its entries are
//   N[j, l] = t(x_j - x_l) + h(x_j + x_l)
//   t(d) = kappa sum_m f(d . theta_m),   f(s) = sum_q nu_q cos(2 pi w_q s)
//   h(s) = kappa (D_q0 / 2) sum_m cos(phi - pi s . theta_m),   phi = 2 pi (1/2 - c)
// with x the pixel centres (differences and sums are integer vectors).  The
// transform's real part pairs every radial sample w with -w; for even n_p the
// sample w = -1/2 has no partner, so it enters t with half its weight
// (nu_q0 = D_q0 / 2) and adds the Hankel part h.  Both parts are convolutions
// (h of the mirrored image), so on the L x L grid (L = 2n, no wrap-around)
//   N u = crop( IFFT2( Kt . U + Kh . conj(U) ) ),   U = FFT2(u zero-padded),
// the mirror folded into Kh as the phase e^{-2 pi i (kx + ky)(n - 1) / L}
// (for real u the mirrored image's spectrum is that phase times conj(U)).
// The taps are summed on the device in FP64 (Clenshaw's recurrence for the
// cosine series f), transformed once by a double-precision FFT and kept as
// FP32 spectra.  Each application is then a forward FFT of the padded image,
// one pointwise product and the inverse FFT: three fused register-FFT passes
// (regfft.cuh) when L is a power of two up to 2048, else cuFFT R2C / C2R with
// pad, product and crop kernels around them.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bbstep.cuh"
#include "regfft.cuh"
#include "fubini.cuh"

namespace tomo {

tomo_status fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t nz, int filter, cudaStream_t st);

namespace {

constexpr int kT = 256;


tomo_status cufft_ok(cufftResult r, const char *what) {
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

// signed offset of circular index i on an axis of length L = 2n; the unused
// index n maps to "no tap"
__device__ __forceinline__ bool tap_offset(int i, int n, int L, int *d) {
  if (i == n) return false;
  *d = i < n ? i : i - L;
  return true;
}

// Taps on the circular L x L grid.  One thread per position of the half plane
// (dy > 0, or dy == 0 and dx >= 0) computes t there and writes it at the
// position and its mirror (t is even), and h at both (h is not).
//   a[0..J]: cosine-series coefficients of f (nu_q paired with its mirror
//   folded: a_0 = D_0, a_j = 2 D_j, and for even n_p a_{n_p/2} = D_q0 / 2);
//   hc = kappa D_q0 / 2 (0: no Hankel part); cphi, sphi = cos, sin phi.
// with_t = false: h only (t from k_nrm_taps8, ct cleared beforehand).
__global__ void k_nrm_taps(int n, int L, int np, int nt, const double *cs, const double *sn, const double *a, int J,
                           double kappa, double hc, double cphi, double sphi, double *ct, double *ch, bool with_t) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * L) return;
  const int iy = (int)(e / L), ix = (int)(e % L);
  int dy, dx;
  if (!tap_offset(iy, n, L, &dy) || !tap_offset(ix, n, L, &dx)) {
    if (with_t) ct[e] = 0.0;
    if (ch) ch[e] = 0.0;
    return;
  }
  if (!with_t && !ch) return;
  if (dy < 0 || (dy == 0 && dx < 0)) return;  // written by the mirror thread
  const int64_t em = (int64_t)((L - iy) % L) * L + (L - ix) % L;
  double t = 0.0, hp = 0.0, hm = 0.0;
  const double inv = 2.0 / (double)np;
  for (int m = 0; m < nt; ++m) {
    const double c = cs[m], s = sn[m];
    const double p = (double)dx * c + (double)dy * s;
    if (with_t) {
      // f(p) = sum_j a_j cos(j th), th = 2 pi p / np: Clenshaw, b_k = a_k + 2 cos(th) b_{k+1} - b_{k+2}
      const double c1 = cospi(p * inv);
      const double c2 = 2.0 * c1;
      double b1 = 0.0, b2 = 0.0;
      for (int j = J; j >= 1; --j) {
        const double b0 = fma(c2, b1, __ldg(a + j) - b2);
        b2 = b1;
        b1 = b0;
      }
      t += fma(-c1, b1, __ldg(a) + c2 * b1 - b2);  // b_0 - cos(th) b_1
    }
    if (ch) {
      // s = x_j + x_l for the pair at offset (dx, dy) from the mirrored image: h(d) and h(-d)
      double sp, cp;
      sincospi(p, &sp, &cp);
      hp += fma(cphi, cp, sphi * sp);   // cos(phi - pi p)
      hm += fma(cphi, cp, -sphi * sp);  // cos(phi + pi p)
    }
  }
  if (with_t) {
    t *= kappa;
    ct[e] = t;
    ct[em] = t;
  }
  if (ch) {
    ch[e] = hc * hp;
    ch[em] = hc * hm;
  }
}

// t for the default angles m pi / n_theta with n_theta even: t is then
// invariant under the eight symmetries of the square (reflection: m ->
// n_theta - m; quarter turn: m -> m + n_theta / 2, f being even), so one thread
// per offset 0 <= ay <= ax < n sums it and writes all eight images.  Grid
// (ceil(n / 64), n) of 64 threads: one thread per (ax, ay).
__global__ void k_nrm_taps8(int n, int L, int np, int nt, const double *cs, const double *sn, const double *a, int J,
                            double kappa, double *ct) {
  const int ax = blockIdx.x * blockDim.x + threadIdx.x, ay = blockIdx.y;
  if (ax >= n || ay > ax) return;
  double t = 0.0;
  const double inv = 2.0 / (double)np;
  for (int m = 0; m < nt; ++m) {
    const double p = (double)ax * cs[m] + (double)ay * sn[m];
    const double c1 = cospi(p * inv);
    const double c2 = 2.0 * c1;
    double b1 = 0.0, b2 = 0.0;
    for (int j = J; j >= 1; --j) {
      const double b0 = fma(c2, b1, __ldg(a + j) - b2);
      b2 = b1;
      b1 = b0;
    }
    t += fma(-c1, b1, __ldg(a) + c2 * b1 - b2);
  }
  t *= kappa;
  const int u[2] = {ax, ay};
  for (int sw = 0; sw < 2; ++sw)
    for (int sx = -1; sx <= 1; sx += 2)
      for (int sy = -1; sy <= 1; sy += 2) {
        const int dx = sx * u[sw], dy = sy * u[1 - sw];
        const int ix = dx >= 0 ? dx : dx + L, iy = dy >= 0 ? dy : dy + L;
        ct[(int64_t)iy * L + ix] = t;
      }
}

// Kt = C_t / L^2; Kh = C_h e^{-2 pi i ((kx + ky)(n - 1) mod L) / L} / L^2
__global__ void k_nrm_spec(const double2 *Ct, const double2 *Ch, int n, int L, float2 *Kt, float2 *Kh) {
  const int W = L / 2 + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * W) return;
  const int ky = (int)(e / W), kx = (int)(e % W);
  const double sc = 1.0 / ((double)L * (double)L);
  Kt[e] = make_float2((float)(Ct[e].x * sc), (float)(Ct[e].y * sc));
  if (Kh) {
    const int64_t r = ((int64_t)(kx + ky) * (n - 1)) % L;
    double s, c;
    sincospi(-2.0 * (double)r / (double)L, &s, &c);
    const double2 v = Ch[e];
    Kh[e] = make_float2((float)((v.x * c - v.y * s) * sc), (float)((v.x * s + v.y * c) * sc));
  }
}

// P[s][gy][gx] = u[s][gy][gx] on the n x n corner, 0 elsewhere; grid (L rows,
// cnt slices; the pass's other slices are transformed too but never read)
__global__ void k_nrm_pad(const float *u, int n, int L, float *P) {
  const int gy = blockIdx.x, s = blockIdx.y;
  float *row = P + ((int64_t)s * L + gy) * L;
  const float *src = u + ((int64_t)s * n + gy) * n;
  for (int gx = threadIdx.x; gx < L; gx += blockDim.x) row[gx] = (gy < n && gx < n) ? src[gx] : 0.f;
}

// X = Kt X + Kh conj(X) on the half spectra; grid (ceil(per / kT), cnt slices)
__global__ void k_nrm_mul(float2 *X, int per, const float2 *Kt, const float2 *Kh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < per) {
    const int64_t e = (int64_t)blockIdx.y * per + k;
    const float2 x = X[e], kt = Kt[k];
    float re = kt.x * x.x - kt.y * x.y, im = kt.x * x.y + kt.y * x.x;
    if (Kh) {
      const float2 kh = Kh[k];  // times conj(x)
      re += kh.x * x.x + kh.y * x.y;
      im += kh.y * x.x - kh.x * x.y;
    }
    X[e] = make_float2(re, im);
  }
}

// y[s][iy][ix] = P[s][iy][ix] on the n x n corner; grid (n rows, cnt slices)
__global__ void k_nrm_crop(const float *P, int n, int L, float *y) {
  const int iy = blockIdx.x, s = blockIdx.y;
  const float *row = P + ((int64_t)s * L + iy) * L;
  float *dst = y + ((int64_t)s * n + iy) * n;
  for (int ix = threadIdx.x; ix < n; ix += blockDim.x) dst[ix] = row[ix];
}

// ---- the SIRT with N in one step --------------------------------------------
// per iteration: g = c - N x (g = c at x = 0), then x += alpha g with the BB1
// step of the gridded SIRT; per-slice sums in FP64 over a fixed split of each
// slice into NB blocks, reduced in a fixed order (deterministic).

__device__ double nrm_block_sum(double v) {
  __shared__ double red[kT];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kT / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// grid (NB, cnt): g = c - (P ? crop(P) : 0) for slices s0 .. s0 + cnt - 1;
// block b takes image rows [b rpb, (b + 1) rpb), rpb = ceil(n / NB), NB <= n;
// part[(s0 + s) NB + b] = (<g,g>, <gp,gp>, <gp, g - gp>) over those rows
__global__ void __launch_bounds__(kT) k_nrm_grad(const float *P, const float *c, const float *gp, float *g, int s0,
                                                 int n, int L, int NB, double3 *part) {
  const int b = blockIdx.x, s = blockIdx.y;
  const int rpb = (n + NB - 1) / NB;
  const int r0 = b * rpb, r1 = r0 + rpb < n ? r0 + rpb : n;
  const int64_t off = (int64_t)(s0 + s) * n * n;
  KSum sg, sp, sq;
  for (int r = r0; r < r1; ++r) {
    const float *prow = P ? P + ((int64_t)s * L + r) * L : nullptr;
    const int64_t ro = off + (int64_t)r * n;
    for (int col = threadIdx.x; col < n; col += kT) {
      const float gv = c[ro + col] - (prow ? prow[col] : 0.f);
      g[ro + col] = gv;
      const float a = gp[ro + col];
      sg.add(gv * gv);
      sp.add(a * a);
      sq.add(a * gv);  // <gp, g - gp> = <gp, g> - <gp, gp>, formed in FP64 below
    }
  }
  const double gg = nrm_block_sum(sg.value()), pp = nrm_block_sum(sp.value());
  const double pq = nrm_block_sum(sq.value()) - pp;
  if (threadIdx.x == 0) part[(int64_t)(s0 + s) * NB + b] = make_double3(gg, pp, pq);
}

// grid (NB, nz): alpha per slice from the partial sums (every block computes
// the same value in the same order; block 0 records it), then x += alpha g on
// the block's range.  sc_in / sc_out[s]: (alpha, frozen, stepped), double-buffered.
__global__ void __launch_bounds__(kT) k_nrm_step(float *x, const float *g, int64_t cols, int NB, const double3 *part,
                                                 const double *sc_in, double *sc_out, double *hist, int k, int nz) {
  const int b = blockIdx.x, s = blockIdx.y;
  __shared__ float alpha_s;
  if (threadIdx.x == 0) {
    double gg = 0.0, P = 0.0, Q = 0.0;
    for (int i = 0; i < NB; ++i) {
      const double3 v = part[(int64_t)s * NB + i];
      gg += v.x;
      P += v.y;
      Q += v.z;
    }
    double frozen, stepped;
    const double a = bb_rule(P, Q, sc_in + s * 4, &frozen, &stepped);
    if (b == 0) {
      sc_out[s * 4 + 0] = a;
      sc_out[s * 4 + 1] = frozen;
      sc_out[s * 4 + 2] = stepped;
      if (hist) hist[(int64_t)k * nz + s] = sqrt(gg);
    }
    alpha_s = (float)a;
  }
  __syncthreads();
  const float a = alpha_s;
  const int64_t per = (cols + NB - 1) / NB;
  const int64_t lo = b * per, hi = lo + per < cols ? lo + per : cols;
  const int64_t off = (int64_t)s * cols;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kT) x[off + i] = fmaf(a, g[off + i], x[off + i]);
}

// ---- fused convolution for L = 2n a power of two, 32 <= L <= 2048 ----------
// Three passes over the half spectrum H[s][kx][j] (kx = 0..n, image row j < n;
// column-major, so that the column pass reads each column contiguously):
//   rows     image rows a = 2p and b = 2p + 1 as one complex FFT of length L
//            (z = u_a + i u_b, zero-padded), split into the two half spectra;
//   columns  per column kx: the FFT over its n rows (zero-padded to L),
//            Kt V + Kh conj(V), the inverse FFT, rows < n kept;
//   rows^-1  the half spectra of rows a, b joined as Y_a + i Y_b (Hermitian
//            extension) and one inverse complex FFT: its real and imaginary
//            parts are rows a and b of N u.
// An FFT of length L = R1 R2 (R1 = R2 or 2 R2) runs on G = R2 lanes of one warp
// by the four-step decomposition: R1-point DFTs in registers over
// x[j1 R2 + j2], the twiddles W_L^{j2 k1}, a transpose through shared memory,
// R2-point DFTs in registers; X[k1 + R1 k2] ends in lane k1 mod G.  The
// inverse runs the same steps backwards with conjugate twiddles.

constexpr int kCvThreads = 256;

// a group's shared tile: R1 x (R2 + 1) plus one entry, so that the tiles of
// consecutive groups start in different banks
template <int R1, int R2>
constexpr int cv_tile() {
  return R1 * (R2 + 1) + 1;
}

template <int R1, int R2>
constexpr int cv_smem() {
  return (kCvThreads / R2) * cv_tile<R1, R2>() * (int)sizeof(float2);
}

// the rows passes move H through the tiles when a block's groups are
// consecutive row pairs of one slice (n/2 a multiple of the groups per block)
template <int R1, int R2>
constexpr bool cv_stage() {
  return (R1 * R2 / 4) % (kCvThreads / R2) == 0;
}

// rows: FFT id f = s (n/2) + p over rows 2p, 2p + 1 of slice s; kStep: the
// rows are x + alpha[s] g, written back to x first (the previous BB step)
template <int R1, int R2, bool kStep>
__global__ void __launch_bounds__(kCvThreads, (R1 <= 32 ? 3 : 1)) k_cv_rows(const float *u, float *x, const float *g,
                                                         const float *alpha, float2 *H, int nz, const float2 *twL,
                                                         const __grid_constant__ Tw64 tw) {
  constexpr int L = R1 * R2, n = L / 2, G = R2, W = n + 1;
  extern __shared__ float2 cv_sm[];
  const int l = threadIdx.x % G;
  float2 *S = cv_sm + (threadIdx.x / G) * cv_tile<R1, R2>();
  const int64_t f = ((int64_t)blockIdx.x * kCvThreads + threadIdx.x) / G;
  const bool act = f < (int64_t)nz * (n / 2);
  const int s = act ? (int)(f / (n / 2)) : 0, p = act ? (int)(f % (n / 2)) : 0;
  const int64_t ra = ((int64_t)s * n + 2 * p) * n, rb = ra + n;
  float2 v[R1], w[R1];
  const float al = (kStep && act) ? alpha[s] : 0.f;
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) {
    float a = 0.f, b = 0.f;
    if (j1 < R1 / 2 && act) {
      const int j = j1 * R2 + l;
      if (kStep) {
        a = fmaf(al, g[ra + j], x[ra + j]);
        b = fmaf(al, g[rb + j], x[rb + j]);
        x[ra + j] = a;
        x[rb + j] = b;
      } else {
        a = u[ra + j];
        b = u[rb + j];
      }
    }
    v[j1] = make_float2(a, b);
  }
  fft_fwd<R1, R2>(v, w, S, l, twL, tw);
  // Z in natural order through the tile, then A_k = (Z_k + conj Z_{L-k}) / 2,
  // B_k = (Z_k - conj Z_{L-k}) / 2i for k = 0..n
#pragma unroll
  for (int t = 0; t < R1 / G; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) S[(l + G * t) + R1 * k2] = w[t * R2 + k2];
  if constexpr (cv_stage<R1, R2>()) {
    // the block's NG row pairs together: row k of H gets NG consecutive pairs
    constexpr int NG = kCvThreads / G;
    __syncthreads();
    const int64_t f0 = (int64_t)blockIdx.x * NG;
    if (f0 < (int64_t)nz * (n / 2)) {
      const int s0 = (int)(f0 / (n / 2)), p0 = (int)(f0 % (n / 2));
      for (int e = threadIdx.x; e < W * NG; e += kCvThreads) {
        const int k = e / NG, q = e % NG;
        const float2 *Sq = cv_sm + q * cv_tile<R1, R2>();
        const float2 zk = Sq[k], zm = Sq[(L - k) & (L - 1)];
        *reinterpret_cast<float4 *>(H + ((int64_t)s0 * W + k) * n + 2 * (p0 + q)) =
            make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      }
    }
    return;
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < R1 / G; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = (l + G * t) + R1 * k2;
      if (k <= n && act) {
        const float2 zk = w[t * R2 + k2], zm = S[(L - k) & (L - 1)];
        const float4 o = make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y),
                                     -0.5f * (zk.x - zm.x));
        *reinterpret_cast<float4 *>(H + ((int64_t)s * W + k) * n + 2 * p) = o;
      }
    }
}

// columns: FFT id f = s W + kx; Kt2 / Kh2 in [kx][ky] order
template <int R1, int R2>
__global__ void __launch_bounds__(kCvThreads) k_cv_cols(float2 *H, int nz, const float2 *Kt2, const float2 *Kh2,
                                                         const float2 *twL, const __grid_constant__ Tw64 tw) {
  constexpr int L = R1 * R2, n = L / 2, G = R2, W = n + 1;
  extern __shared__ float2 cv_sm[];
  const int l = threadIdx.x % G;
  float2 *S = cv_sm + (threadIdx.x / G) * cv_tile<R1, R2>();
  const int64_t f = ((int64_t)blockIdx.x * kCvThreads + threadIdx.x) / G;
  const bool act = f < (int64_t)nz * W;
  const int kx = act ? (int)(f % W) : 0;
  float2 *col = H + (act ? f : 0) * n;
  float2 v[R1], w[R1];
#pragma unroll
  for (int j1 = 0; j1 < R1; ++j1) v[j1] = (j1 < R1 / 2 && act) ? col[j1 * R2 + l] : make_float2(0.f, 0.f);
  fft_fwd<R1, R2>(v, w, S, l, twL, tw);
  const float2 *kt = Kt2 + (int64_t)kx * L, *kh = Kh2 ? Kh2 + (int64_t)kx * L : nullptr;
#pragma unroll
  for (int t = 0; t < R1 / G; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int ky = (l + G * t) + R1 * k2;
      const float2 x = w[t * R2 + k2], a = __ldg(kt + ky);
      float re = a.x * x.x - a.y * x.y, im = a.x * x.y + a.y * x.x;
      if (kh) {
        const float2 b = __ldg(kh + ky);  // times conj(x)
        re += b.x * x.x + b.y * x.y;
        im += b.y * x.x - b.x * x.y;
      }
      w[t * R2 + k2] = make_float2(re, im);
    }
  fft_inv<R1, R2>(w, v, S, l, twL, tw);
  if (act) {
#pragma unroll
    for (int j1 = 0; j1 < R1 / 2; ++j1) col[j1 * R2 + l] = v[j1];
  }
}

// rows^-1: FFT id f = s (n/2) + p.  kGrad: g = c - N u on rows 2p, 2p + 1 and
// part[f] = (<g,g>, <gp,gp>, <gp, g - gp>) over them (the row-pair split of
// k_nrm_grad with NB = n/2); else y = N u
template <int R1, int R2, bool kGrad>
__global__ void __launch_bounds__(kCvThreads, (R1 <= 32 ? 3 : 1)) k_cv_rows_inv(const float2 *H, float *y, const float *c, const float *gp,
                                                             double3 *part, int nz, const float2 *twL,
                                                             const __grid_constant__ Tw64 tw) {
  constexpr int L = R1 * R2, n = L / 2, G = R2, W = n + 1;
  extern __shared__ float2 cv_sm[];
  const int l = threadIdx.x % G;
  float2 *S = cv_sm + (threadIdx.x / G) * cv_tile<R1, R2>();
  const int64_t f = ((int64_t)blockIdx.x * kCvThreads + threadIdx.x) / G;
  const bool act = f < (int64_t)nz * (n / 2);
  const int s = act ? (int)(f / (n / 2)) : 0, p = act ? (int)(f % (n / 2)) : 0;
  float2 v[R1], w[R1];
  if constexpr (cv_stage<R1, R2>()) {
    // the block's NG row pairs together: Z_q[k] = Y_a + i Y_b and its
    // Hermitian partner at L - k, written into the tiles in natural order
    constexpr int NG = kCvThreads / G;
    const int64_t f0 = (int64_t)blockIdx.x * NG;
    if (f0 < (int64_t)nz * (n / 2)) {
      const int s0 = (int)(f0 / (n / 2)), p0 = (int)(f0 % (n / 2));
      for (int e = threadIdx.x; e < W * NG; e += kCvThreads) {
        const int k = e / NG, q = e % NG;
        float4 y4 = *reinterpret_cast<const float4 *>(H + ((int64_t)s0 * W + k) * n + 2 * (p0 + q));
        if (k == 0 || k == n) y4.y = y4.w = 0.f;  // real for real rows
        float2 *Sq = cv_sm + q * cv_tile<R1, R2>();
        Sq[k] = make_float2(y4.x - y4.w, y4.y + y4.z);
        if (k > 0 && k < n) Sq[L - k] = make_float2(y4.x + y4.w, y4.z - y4.y);
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < R1 / G; ++t)
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) w[t * R2 + k2] = S[(l + G * t) + R1 * k2];
    __syncwarp();
  } else {
#pragma unroll
  for (int t = 0; t < R1 / G; ++t)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = (l + G * t) + R1 * k2;
      const bool cj = k > n;
      const int kk = cj ? L - k : k;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act) q = *reinterpret_cast<const float4 *>(H + ((int64_t)s * W + kk) * n + 2 * p);
      if (kk == 0 || kk == n) q.y = q.w = 0.f;  // real for real rows
      if (cj) q.y = -q.y, q.w = -q.w;
      w[t * R2 + k2] = make_float2(q.x - q.w, q.y + q.z);  // Y_a + i Y_b
    }
  }
  const int64_t ra = ((int64_t)s * n + 2 * p) * n, rb = ra + n;
  if (kGrad && act) {
    // the epilogue's c and gp rows (2 x n floats each) towards L2 while the FFT runs
    for (int j = 32 * l; j < 2 * n; j += 32 * R2) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(c + ra + j));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(gp + ra + j));
    }
  }
  fft_inv<R1, R2>(w, v, S, l, twL, tw);
  KSum sg, sp, sq;
  if (act) {
#pragma unroll
    for (int j1 = 0; j1 < R1 / 2; ++j1) {
      const int j = j1 * R2 + l;
      if (kGrad) {
        const float ga = c[ra + j] - v[j1].x, gb = c[rb + j] - v[j1].y;
        y[ra + j] = ga;
        y[rb + j] = gb;
        const float pa = gp[ra + j], pb = gp[rb + j];
        sg.add(ga * ga);
        sg.add(gb * gb);
        sp.add(pa * pa);
        sp.add(pb * pb);
        sq.add(pa * ga);
        sq.add(pb * gb);
      } else {
        y[ra + j] = v[j1].x;
        y[rb + j] = v[j1].y;
      }
    }
  }
  if (kGrad) {
    double gg = sg.value(), pp = sp.value(), pq = sq.value();
#pragma unroll
    for (int o = G / 2; o; o >>= 1) {
      gg += __shfl_xor_sync(0xffffffffu, gg, o);
      pp += __shfl_xor_sync(0xffffffffu, pp, o);
      pq += __shfl_xor_sync(0xffffffffu, pq, o);
    }
    if (act && l == 0) part[f] = make_double3(gg, pp, pq - pp);
  }
}

// part[s (n/2) + p] = (<c,c>, 0, 0) over rows 2p, 2p + 1: the sums of the
// first gradient g_0 = c (no previous one); one warp per row pair, grid
// (ceil(n / 16), nz)
__global__ void k_nrm_sumsq(const float *c, int n, double3 *part) {
  const int p = blockIdx.x * (kT / 32) + threadIdx.x / 32, s = blockIdx.y, lane = threadIdx.x & 31;
  if (p >= n / 2) return;  // whole warps
  const float *r = c + ((int64_t)s * n + 2 * p) * n;
  KSum sg;
  for (int j = lane; j < 2 * n; j += 32) sg.add(r[j] * r[j]);
  double gg = sg.value();
  for (int o = 16; o; o >>= 1) gg += __shfl_xor_sync(0xffffffffu, gg, o);
  if (lane == 0) part[(int64_t)s * (n / 2) + p] = make_double3(gg, 0.0, 0.0);
}

// [L][W] -> [W][L] for the column pass
__global__ void k_nrm_kT(const float2 *K, int L, float2 *KT) {
  const int W = L / 2 + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * W) return;
  const int ky = (int)(e / W), kx = (int)(e % W);
  KT[(int64_t)kx * L + ky] = K[e];
}

// FP64 weights of the backprojection: kappa and the density at |w| = j / np
double dens_at(int filter, int j, int np) {
  if (filter == 0) return 1.0;
  const double r = j == 0 ? 1.0 / (4.0 * np) : (double)j / (double)np;
  if (filter == 1) return r;
  return r * (0.54 + 0.46 * std::cos(2.0 * M_PI * (double)j / (double)np));
}

tomo_status build_kernel(tomo_fubini *F, int filter, cudaStream_t st) {
  NormalKernel &K = F->nk[filter];
  if (K.Kt) return TOMO_OK;
  const int n = F->n, L = F->G, np = F->np, nt = F->nt;
  const bool even = (np % 2) == 0;
  const double kappa = filter == 0 ? 1.0 / np : M_PI / ((double)nt * np);
  // cosine series of f: a_0 = D_0, a_j = 2 D_j for the paired samples, a_{np/2} = D_q0 / 2 (even np)
  const int J = np / 2;  // even: the unpaired sample at j = np/2; odd: the last pair
  std::vector<double> a(J + 1);
  a[0] = dens_at(filter, 0, np);
  for (int j = 1; j <= J; ++j) a[j] = (even && j == J) ? 0.5 * dens_at(filter, j, np) : 2.0 * dens_at(filter, j, np);
  const double hc = even ? kappa * 0.5 * dens_at(filter, J, np) : 0.0;
  const double phi = 2.0 * M_PI * (0.5 - F->center);
  const int W = L / 2 + 1;
  const int64_t LL = (int64_t)L * L, LW = (int64_t)L * W;

  double *da = nullptr, *ct = nullptr;
  double2 *C = nullptr;
  cufftHandle pd = 0;
  bool have_pd = false;
  struct Tmp {
    double **a, **ct;
    double2 **C;
    cufftHandle *pd;
    bool *have;
    ~Tmp() {
      if (*a) cudaFree(*a);
      if (*ct) cudaFree(*ct);
      if (*C) cudaFree(*C);
      if (*have) cufftDestroy(*pd);
    }
  } tmp{&da, &ct, &C, &pd, &have_pd};
  TOMO_TRY(dalloc(&da, J + 1));
  TOMO_TRY(dalloc(&ct, 2 * LL));  // ct then ch
  TOMO_TRY(dalloc(&C, 2 * LW));
  TOMO_CUDA(cudaMemcpyAsync(da, a.data(), sizeof(double) * (J + 1), cudaMemcpyHostToDevice, st));
  double *ch = even ? ct + LL : nullptr;
  if (!even) TOMO_CUDA(cudaMemsetAsync(ct + LL, 0, sizeof(double) * LL, st));
  // default angles, n_theta even: t from one octant of offsets (k_nrm_taps8)
  const bool sym8 = F->default_angles && (nt % 2) == 0;
  if (sym8) {
    TOMO_CUDA(cudaMemsetAsync(ct, 0, sizeof(double) * LL, st));
    k_nrm_taps8<<<dim3((n + 63) / 64, n), 64, 0, st>>>(n, L, np, nt, F->cs, F->sn, da, J, kappa, ct);
  }
  k_nrm_taps<<<(unsigned)((LL + kT - 1) / kT), kT, 0, st>>>(n, L, np, nt, F->cs, F->sn, da, J, kappa, hc,
                                                             std::cos(phi), std::sin(phi), ct, ch, !sym8);
  TOMO_CUDA(cudaGetLastError());
  int dims[2] = {L, L};
  TOMO_TRY(cufft_ok(cufftPlanMany(&pd, 2, dims, nullptr, 1, (int)LL, nullptr, 1, (int)LW, CUFFT_D2Z, 2), "plan D2Z"));
  have_pd = true;
  TOMO_TRY(cufft_ok(cufftSetStream(pd, st), "set stream"));
  TOMO_TRY(cufft_ok(cufftExecD2Z(pd, ct, (cufftDoubleComplex *)C), "taps D2Z"));
  TOMO_TRY(dalloc(&K.Kt, LW));
  if (even) {
    tomo_status s = dalloc(&K.Kh, LW);
    if (s != TOMO_OK) {
      cudaFree(K.Kt);
      K.Kt = nullptr;
      return s;
    }
  }
  k_nrm_spec<<<(unsigned)((LW + kT - 1) / kT), kT, 0, st>>>(C, C + LW, n, L, K.Kt, K.Kh);
  TOMO_CUDA(cudaGetLastError());
  if (fused_ok(L)) {  // the column pass reads the spectra column by column
    TOMO_TRY(dalloc(&K.Kt2, LW));
    k_nrm_kT<<<(unsigned)((LW + kT - 1) / kT), kT, 0, st>>>(K.Kt, L, K.Kt2);
    if (even) {
      TOMO_TRY(dalloc(&K.Kh2, LW));
      k_nrm_kT<<<(unsigned)((LW + kT - 1) / kT), kT, 0, st>>>(K.Kh, L, K.Kh2);
    }
    TOMO_CUDA(cudaGetLastError());
  }
  TOMO_CUDA(cudaStreamSynchronize(st));  // the temporaries are freed on return
  return TOMO_OK;
}

tomo_status ensure_plans(tomo_fubini *F) {
  if (F->nplans) return TOMO_OK;
  const int L = F->G, W = L / 2 + 1;
  const int64_t LL = (int64_t)L * L, LW = (int64_t)L * W;
  // slices per pass: 32, fewer while the two buffers would pass 1 GiB
  int Bn = 32;
  while (Bn > 1 && (LL * 4 + LW * 8) * Bn > ((int64_t)1 << 30)) Bn /= 2;
  TOMO_TRY(dalloc(&F->nP, (size_t)LL * Bn));
  TOMO_TRY(dalloc(&F->nX, (size_t)LW * Bn));
  int dims[2] = {L, L};
  TOMO_TRY(cufft_ok(cufftPlanMany(&F->planR, 2, dims, nullptr, 1, (int)LL, nullptr, 1, (int)LW, CUFFT_R2C, Bn),
                    "plan R2C"));
  cufftResult r = cufftPlanMany(&F->planC, 2, dims, nullptr, 1, (int)LW, nullptr, 1, (int)LL, CUFFT_C2R, Bn);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(F->planR);
    return cufft_ok(r, "plan C2R");
  }
  F->Bn = Bn;
  F->nplans = true;
  return TOMO_OK;
}

// P (first cnt slices of the pass) = N u for slices u[0 .. cnt)
tomo_status apply_pass(tomo_fubini *F, const NormalKernel &K, const float *u, int cnt, cudaStream_t st) {
  const int n = F->n, L = F->G, W = L / 2 + 1;
  k_nrm_pad<<<dim3(L, cnt), kT, 0, st>>>(u, n, L, F->nP);
  TOMO_TRY(cufft_ok(cufftExecR2C(F->planR, F->nP, (cufftComplex *)F->nX), "R2C"));
  k_nrm_mul<<<dim3((L * W + kT - 1) / kT, cnt), kT, 0, st>>>(F->nX, L * W, K.Kt, K.Kh);
  TOMO_TRY(cufft_ok(cufftExecC2R(F->planC, (cufftComplex *)F->nX, F->nP), "C2R"));
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status ensure_fused(tomo_fubini *F, cudaStream_t st) {
  if (F->H) return TOMO_OK;
  const int n = F->n, W = n + 1;
  // slices per fused pass: 64, fewer while the half spectrum would pass 1 GiB
  int Hc = 64;
  while (Hc > 1 && (int64_t)W * n * 8 * Hc > ((int64_t)1 << 30)) Hc /= 2;
  TOMO_TRY(ensure_twiddles(F, st));
  TOMO_TRY(dalloc(&F->H, (size_t)W * n * Hc));
  F->Hc = Hc;
  return TOMO_OK;
}

// the pointers of one fused pass set over cnt slices
struct CvArgs {
  const float *u = nullptr;      // rows: input image (plain) ...
  float *x = nullptr;            // ... or x += alpha g first (step)
  const float *g = nullptr;
  const float *alpha = nullptr;
  float *y = nullptr;            // rows^-1: N u (plain) or the new gradient c - N u (grad)
  const float *c = nullptr;
  const float *gp = nullptr;
  double3 *part = nullptr;
  bool step = false, grad = false;
};

template <class Kern>
tomo_status smem_attr(Kern k, int bytes) {
  TOMO_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return TOMO_OK;
}

template <int R1, int R2>
tomo_status cv_run(tomo_fubini *F, const NormalKernel &K, const CvArgs &a, int cnt, cudaStream_t st) {
  constexpr int L = R1 * R2, n = L / 2, W = n + 1, per = kCvThreads / R2, sm = cv_smem<R1, R2>();
  TOMO_TRY(smem_attr(k_cv_rows<R1, R2, true>, sm));
  TOMO_TRY(smem_attr(k_cv_rows<R1, R2, false>, sm));
  TOMO_TRY(smem_attr(k_cv_cols<R1, R2>, sm));
  TOMO_TRY(smem_attr(k_cv_rows_inv<R1, R2, true>, sm));
  TOMO_TRY(smem_attr(k_cv_rows_inv<R1, R2, false>, sm));
  const Tw64 tw = tw64();
  const unsigned gr = (unsigned)(((int64_t)cnt * (n / 2) + per - 1) / per);
  const unsigned gc = (unsigned)(((int64_t)cnt * W + per - 1) / per);
  if (a.step)
    k_cv_rows<R1, R2, true><<<gr, kCvThreads, sm, st>>>(nullptr, a.x, a.g, a.alpha, F->H, cnt, F->twL, tw);
  else
    k_cv_rows<R1, R2, false><<<gr, kCvThreads, sm, st>>>(a.u, nullptr, nullptr, nullptr, F->H, cnt, F->twL, tw);
  k_cv_cols<R1, R2><<<gc, kCvThreads, sm, st>>>(F->H, cnt, K.Kt2, K.Kh2, F->twL, tw);
  if (a.grad)
    k_cv_rows_inv<R1, R2, true><<<gr, kCvThreads, sm, st>>>(F->H, a.y, a.c, a.gp, a.part, cnt, F->twL, tw);
  else
    k_cv_rows_inv<R1, R2, false><<<gr, kCvThreads, sm, st>>>(F->H, a.y, nullptr, nullptr, nullptr, cnt, F->twL, tw);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status cv_dispatch(tomo_fubini *F, const NormalKernel &K, const CvArgs &a, int cnt, cudaStream_t st) {
  switch (F->G) {
    case 32: return cv_run<8, 4>(F, K, a, cnt, st);
    case 64: return cv_run<8, 8>(F, K, a, cnt, st);
    case 128: return cv_run<16, 8>(F, K, a, cnt, st);
    case 256: return cv_run<16, 16>(F, K, a, cnt, st);
    case 512: return cv_run<32, 16>(F, K, a, cnt, st);
    case 1024: return cv_run<32, 32>(F, K, a, cnt, st);
    case 2048: return cv_run<64, 32>(F, K, a, cnt, st);
  }
  return fail(TOMO_ERR_INVALID_ARG, "no fused convolution for this size");
}

tomo_status prepare(tomo_fubini *F, int filter, cudaStream_t st) {
  TOMO_TRY(build_kernel(F, filter, st));
  if (fused_ok(F->G)) return ensure_fused(F, st);
  TOMO_TRY(ensure_plans(F));
  TOMO_TRY(cufft_ok(cufftSetStream(F->planR, st), "set stream"));
  TOMO_TRY(cufft_ok(cufftSetStream(F->planC, st), "set stream"));
  return TOMO_OK;
}

}  // namespace

tomo_status ensure_twiddles(tomo_fubini *F, cudaStream_t st) {
  if (F->twL) return TOMO_OK;
  const int L = F->G, R2 = fft_r2(L);
  if (cudaMalloc(&F->twL, sizeof(float2) * 2 * L) != cudaSuccess) {
    cudaGetLastError();
    F->twL = nullptr;
    return fail(TOMO_ERR_OOM, "twiddle table allocation failed");
  }
  k_fft_twiddles<<<(2 * L + kT - 1) / kT, kT, 0, st>>>(L / R2, R2, F->twL);
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

void free_normal(tomo_fubini *F) {
  for (NormalKernel &K : F->nk) {
    for (float2 *q : {K.Kt, K.Kh, K.Kt2, K.Kh2})
      if (q) cudaFree(q);
    K = NormalKernel{};
  }
  if (F->twL) cudaFree(F->twL);
  if (F->H) cudaFree(F->H);
  F->twL = nullptr;
  F->H = nullptr;
  if (F->nplans) {
    cufftDestroy(F->planR);
    cufftDestroy(F->planC);
    F->nplans = false;
  }
  if (F->nP) cudaFree(F->nP);
  if (F->nX) cudaFree(F->nX);
  F->nP = nullptr;
  F->nX = nullptr;
}

tomo_status fubini_normal(tomo_fubini *F, const float *x, float *y, int32_t nz, int filter, cudaStream_t st) {
  TOMO_TRY(prepare(F, filter, st));
  const NormalKernel &K = F->nk[filter];
  const int n = F->n, L = F->G;
  if (fused_ok(L)) {
    for (int32_t s0 = 0; s0 < nz; s0 += F->Hc) {
      CvArgs a;
      a.u = x + (int64_t)s0 * n * n;
      a.y = y + (int64_t)s0 * n * n;
      TOMO_TRY(cv_dispatch(F, K, a, std::min<int32_t>(F->Hc, nz - s0), st));
    }
    return TOMO_OK;
  }
  for (int32_t s0 = 0; s0 < nz; s0 += F->Bn) {
    const int cnt = std::min<int32_t>(F->Bn, nz - s0);
    TOMO_TRY(apply_pass(F, K, x + (int64_t)s0 * n * n, cnt, st));
    k_nrm_crop<<<dim3(n, cnt), kT, 0, st>>>(F->nP, n, L, y + (int64_t)s0 * n * n);
    TOMO_CUDA(cudaGetLastError());
  }
  return TOMO_OK;
}

tomo_status fubini_sirt_bb_normal(tomo_fubini *F, const float *sino, float *x, int32_t nz, int32_t iters,
                                  double *hist, cudaStream_t st) {
  TOMO_TRY(prepare(F, 2, st));
  const NormalKernel &K = F->nk[2];
  const int n = F->n, L = F->G;
  const int64_t cols = (int64_t)n * n;
  const bool fused = fused_ok(L);
  // partial sums per slice: the fused path sums row pairs (n/2 per slice)
  const int NB = fused ? n / 2 : (int)std::max<int64_t>(1, std::min<int64_t>({32, (cols + 4095) / 4096, (int64_t)n}));
  float *c = nullptr, *g0 = nullptr, *g1 = nullptr, *alpha = nullptr;
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
  } fr{{(void **)&c, (void **)&g0, (void **)&g1, (void **)&scal, (void **)&part, (void **)&alpha}, st};
  TOMO_TRY(alloc((void **)&c, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&g0, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&g1, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&scal, sizeof(double) * 8 * nz));
  TOMO_TRY(alloc((void **)&part, sizeof(double3) * NB * nz));
  // c = the Hamming-filtered backprojection of b (gridded), once
  TOMO_TRY(fubini_backproject(F, sino, c, nz, 2, st));
  TOMO_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * cols * nz, st));
  if (!fused) TOMO_CUDA(cudaMemsetAsync(g1, 0, sizeof(float) * cols * nz, st));  // gp at k = 0
  TOMO_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 8 * nz, st));
  float *g = g0, *gp = g1;
  if (fused && iters > 0) {
    // per iteration k >= 1: alpha_{k-1} from the sums of g_{k-1}; then one fused
    // set of passes takes x_k = x_{k-1} + alpha g_{k-1} into the rows pass and
    // leaves g_k = c - N x_k and its sums after the inverse rows pass
    // g_0 = c itself; later gradients alternate between g0 and g1
    TOMO_TRY(alloc((void **)&alpha, sizeof(float) * nz));
    k_nrm_sumsq<<<dim3((n + 15) / 16, nz), kT, 0, st>>>(c, n, part);
    g = c;
    float *next = g0;
    for (int32_t k = 1; k <= iters; ++k) {
      const int m = k - 1;  // the step taken now: from g_{k-1}
      k_bb_alpha<<<nz, 32, 0, st>>>(part, NB, scal + (m & 1) * 4 * nz, scal + ((m + 1) & 1) * 4 * nz, hist, m, nz,
                                     alpha);
      TOMO_CUDA(cudaGetLastError());
      if (k == iters) {
        const int per = (int)std::min<int64_t>(64, (cols + kT - 1) / kT);
        k_bb_axpy<<<dim3(per, nz), kT, 0, st>>>(x, g, alpha, cols);
        TOMO_CUDA(cudaGetLastError());
        break;
      }
      for (int32_t s0 = 0; s0 < nz; s0 += F->Hc) {
        CvArgs a;
        a.step = a.grad = true;
        a.x = x + s0 * cols;
        a.g = g + s0 * cols;
        a.alpha = alpha + s0;
        a.y = next + s0 * cols;  // g_k
        a.c = c + s0 * cols;
        a.gp = g + s0 * cols;
        a.part = part + (int64_t)s0 * NB;
        TOMO_TRY(cv_dispatch(F, K, a, std::min<int32_t>(F->Hc, nz - s0), st));
      }
      float *prev = g;
      g = next;
      next = prev == c ? g1 : prev;
    }
    return TOMO_OK;
  }
  for (int32_t k = 0; k < iters; ++k) {
    if (k == 0) {
      k_nrm_grad<<<dim3(NB, nz), kT, 0, st>>>(nullptr, c, gp, g, 0, n, L, NB, part);
    } else {
      for (int32_t s0 = 0; s0 < nz; s0 += F->Bn) {
        const int cnt = std::min<int32_t>(F->Bn, nz - s0);
        TOMO_TRY(apply_pass(F, K, x + (int64_t)s0 * cols, cnt, st));
        k_nrm_grad<<<dim3(NB, cnt), kT, 0, st>>>(F->nP, c, gp, g, s0, n, L, NB, part);
      }
    }
    const double *sc_in = scal + (k & 1) * 4 * nz;
    double *sc_out = scal + ((k + 1) & 1) * 4 * nz;
    k_nrm_step<<<dim3(NB, nz), kT, 0, st>>>(x, g, cols, NB, part, sc_in, sc_out, hist, k, nz);
    TOMO_CUDA(cudaGetLastError());
    std::swap(g, gp);
  }
  return TOMO_OK;
}

}  // namespace tomo
