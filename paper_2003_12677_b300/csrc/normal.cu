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
// FP32 spectra; each application is an FP32 real-to-complex FFT, one
// pointwise product and the inverse FFT.
#include <cmath>
#include <vector>

#include "fubini.cuh"

namespace tomo {

tomo_status fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t nz, int filter, cudaStream_t st);

namespace {

constexpr int kT = 256;

int egrid(int64_t n) {
  int64_t b = (n + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 16));
}

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
__global__ void k_nrm_taps(int n, int L, int np, int nt, const double *cs, const double *sn, const double *a, int J,
                           double kappa, double hc, double cphi, double sphi, double *ct, double *ch) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * L) return;
  const int iy = (int)(e / L), ix = (int)(e % L);
  int dy, dx;
  if (!tap_offset(iy, n, L, &dy) || !tap_offset(ix, n, L, &dx)) {
    ct[e] = 0.0;
    if (ch) ch[e] = 0.0;
    return;
  }
  if (dy < 0 || (dy == 0 && dx < 0)) return;  // written by the mirror thread
  const int64_t em = (int64_t)((L - iy) % L) * L + (L - ix) % L;
  double t = 0.0, hp = 0.0, hm = 0.0;
  const double inv = 2.0 / (double)np;
  for (int m = 0; m < nt; ++m) {
    const double c = cs[m], s = sn[m];
    const double p = (double)dx * c + (double)dy * s;
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
    if (ch) {
      // s = x_j + x_l for the pair at offset (dx, dy) from the mirrored image: h(d) and h(-d)
      double sp, cp;
      sincospi(p, &sp, &cp);
      hp += fma(cphi, cp, sphi * sp);   // cos(phi - pi p)
      hm += fma(cphi, cp, -sphi * sp);  // cos(phi + pi p)
    }
  }
  t *= kappa;
  ct[e] = t;
  ct[em] = t;
  if (ch) {
    ch[e] = hc * hp;
    ch[em] = hc * hm;
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

// P[s][gy][gx] = u[s][gy][gx] on the n x n corner, 0 elsewhere (s < cnt; the
// pass's other slices are transformed too but never read)
__global__ void k_nrm_pad(const float *u, int cnt, int n, int L, float *P) {
  const int64_t total = (int64_t)cnt * L * L;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((int64_t)L * L));
    const int gy = (int)((e / L) % L), gx = (int)(e % L);
    P[e] = (gy < n && gx < n) ? u[((int64_t)s * n + gy) * n + gx] : 0.f;
  }
}

// X = Kt X + Kh conj(X) on the half spectra of cnt slices
__global__ void k_nrm_mul(float2 *X, int cnt, int64_t per, const float2 *Kt, const float2 *Kh) {
  const int64_t total = (int64_t)cnt * per;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % per;
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

// y[s][iy][ix] = P[s][iy][ix] on the n x n corner
__global__ void k_nrm_crop(const float *P, int cnt, int n, int L, float *y) {
  const int64_t total = (int64_t)cnt * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((int64_t)n * n));
    const int iy = (int)((e / n) % n), ix = (int)(e % n);
    y[e] = P[((int64_t)s * L + iy) * L + ix];
  }
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
// part[(s0 + s) NB + b] = (<g,g>, <gp,gp>, <gp, g - gp>) of block b's range
__global__ void __launch_bounds__(kT) k_nrm_grad(const float *P, const float *c, const float *gp, float *g, int s0,
                                                 int n, int L, int NB, double3 *part) {
  const int b = blockIdx.x, s = blockIdx.y;
  const int64_t cols = (int64_t)n * n;
  const int64_t per = (cols + NB - 1) / NB;
  const int64_t lo = b * per, hi = lo + per < cols ? lo + per : cols;
  const int64_t off = (int64_t)(s0 + s) * cols;
  double gg = 0.0, pp = 0.0, pq = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kT) {
    float nx = 0.f;
    if (P) nx = P[((int64_t)s * L + i / n) * L + i % n];
    const float gv = c[off + i] - nx;
    g[off + i] = gv;
    const double a = gp[off + i];
    gg += (double)gv * (double)gv;
    pp += a * a;
    pq += a * ((double)gv - a);
  }
  gg = nrm_block_sum(gg);
  pp = nrm_block_sum(pp);
  pq = nrm_block_sum(pq);
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
    const double ap = sc_in[s * 4 + 0];
    double frozen = sc_in[s * 4 + 1], stepped = sc_in[s * 4 + 2];
    double a = 0.0;
    if (frozen != 0.0) {
      a = 0.0;
    } else if (stepped == 0.0) {
      a = 1.0;
      stepped = 1.0;
    } else {
      const double ss = ap * ap * P, sy = -ap * Q;
      if (ss > 0.0 && sy > 0.0)
        a = ss / sy;
      else
        frozen = 1.0;
    }
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
  k_nrm_taps<<<(unsigned)((LL + kT - 1) / kT), kT, 0, st>>>(n, L, np, nt, F->cs, F->sn, da, J, kappa, hc,
                                                             std::cos(phi), std::sin(phi), ct, ch);
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
  k_nrm_pad<<<egrid((int64_t)cnt * L * L), kT, 0, st>>>(u, cnt, n, L, F->nP);
  TOMO_TRY(cufft_ok(cufftExecR2C(F->planR, F->nP, (cufftComplex *)F->nX), "R2C"));
  k_nrm_mul<<<egrid((int64_t)cnt * L * W), kT, 0, st>>>(F->nX, cnt, (int64_t)L * W, K.Kt, K.Kh);
  TOMO_TRY(cufft_ok(cufftExecC2R(F->planC, (cufftComplex *)F->nX, F->nP), "C2R"));
  TOMO_CUDA(cudaGetLastError());
  return TOMO_OK;
}

tomo_status prepare(tomo_fubini *F, int filter, cudaStream_t st) {
  TOMO_TRY(build_kernel(F, filter, st));
  TOMO_TRY(ensure_plans(F));
  TOMO_TRY(cufft_ok(cufftSetStream(F->planR, st), "set stream"));
  TOMO_TRY(cufft_ok(cufftSetStream(F->planC, st), "set stream"));
  return TOMO_OK;
}

}  // namespace

void free_normal(tomo_fubini *F) {
  for (NormalKernel &K : F->nk) {
    if (K.Kt) cudaFree(K.Kt);
    if (K.Kh) cudaFree(K.Kh);
    K = NormalKernel{};
  }
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
  for (int32_t s0 = 0; s0 < nz; s0 += F->Bn) {
    const int cnt = std::min<int32_t>(F->Bn, nz - s0);
    TOMO_TRY(apply_pass(F, K, x + (int64_t)s0 * n * n, cnt, st));
    k_nrm_crop<<<egrid((int64_t)cnt * n * n), kT, 0, st>>>(F->nP, cnt, n, L, y + (int64_t)s0 * n * n);
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
  const int NB = (int)std::max<int64_t>(1, std::min<int64_t>(32, (cols + 4095) / 4096));
  float *c = nullptr, *g0 = nullptr, *g1 = nullptr;
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
    void **p[5];
    cudaStream_t st;
    ~Free() {
      for (void **q : p)
        if (*q) cudaFreeAsync(*q, st);
    }
  } fr{{(void **)&c, (void **)&g0, (void **)&g1, (void **)&scal, (void **)&part}, st};
  TOMO_TRY(alloc((void **)&c, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&g0, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&g1, sizeof(float) * cols * nz));
  TOMO_TRY(alloc((void **)&scal, sizeof(double) * 8 * nz));
  TOMO_TRY(alloc((void **)&part, sizeof(double3) * NB * nz));
  // c = the Hamming-filtered backprojection of b (gridded), once
  TOMO_TRY(fubini_backproject(F, sino, c, nz, 2, st));
  TOMO_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * cols * nz, st));
  TOMO_CUDA(cudaMemsetAsync(g1, 0, sizeof(float) * cols * nz, st));
  TOMO_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 8 * nz, st));
  float *g = g0, *gp = g1;
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
