// fubini.cuh -- the handle of the Fubini-Radon transform (Sec. 3, Eq. 2),
// shared by the transform (fubini.cu) and its normal operator (normal.cu).
#pragma once

#include <cufft.h>

#include "internal.cuh"

namespace tomo {

// The normal operator N = R^T W R of one filter, applied as a 2n x 2n
// circular convolution: spectra of its Toeplitz taps (over pixel differences)
// and of its Hankel taps (over pixel sums, times the phase that turns the
// mirrored image's spectrum into the conjugate of the image's), each scaled
// by 1 / L^2 for the unnormalised inverse transform.
struct NormalKernel {
  float2 *Kt = nullptr;   // [L][L/2+1]
  float2 *Kh = nullptr;   // [L][L/2+1]; null when n_p is odd (no Hankel part)
  float2 *Kt2 = nullptr;  // [L/2+1][L]: the same, column-major (fused convolution)
  float2 *Kh2 = nullptr;
};

}  // namespace tomo

struct tomo_fubini {
  int32_t n = 0, np = 0, nt = 0, kw = 0, G = 0, Bf = 0;
  double center = 0, beta = 0;
  int device = 0;
  tomo::Csr S;                    // (nt*np) x (G*G)
  tomo::Csr STs;                  // S^T with its long rows emptied (rows of <= 64 entries)
  tomo::Csr STl;                  // the long rows of S^T, compact; rows_l[i] is row i's index
  int32_t *rows_l = nullptr;
  bool default_angles = false;    // theta_m = m pi / nt (no user angles)
  double *cs = nullptr;           // [nt] cos theta_m
  double *sn = nullptr;           // [nt] sin theta_m
  float *deapod = nullptr;        // [n] 1 / phi_hat(x / G)
  float *dens = nullptr;          // [np] ramp density of the filtered backprojection
  float *dens_h = nullptr;        // [np] the same times the Hamming window
  float2 *ph_grid = nullptr;      // [G]  e^{2 pi i k (G/2 - 1/2)/G}
  float2 *ph_rad = nullptr;       // [np] e^{2 pi i (q - q0)(1/2 - c)/np}
  float2 *ph_bin = nullptr;       // [np] e^{2 pi i q0 k / np}
  cufftComplex *grid = nullptr;   // [Bf][G][G]
  float *gridI = nullptr;         // [G*G][2 Bf] interleaved (re, im)
  float *polI = nullptr;          // [nt*np][2 Bf]
  cufftComplex *pol = nullptr;    // [Bf][nt][np]
  float2 *faT = nullptr;          // [Bf][G][n] the adjoint's column-transformed grid (register-FFT path)
  float2 *twP = nullptr;          // [2 np] W_np^{j2 k1} in both orders (register-FFT radial transforms)
  cufftHandle plan2 = 0, plan1 = 0;  // only for sizes the register-FFT passes do not take
  bool has_plan2 = false, has_plan1 = false;
  // normal operator (normal.cu), built on first use per filter
  tomo::NormalKernel nk[3];
  int32_t Bn = 0;                 // slices per convolution pass
  float *nP = nullptr;            // [Bn][G][G] real padded image / result
  float2 *nX = nullptr;           // [Bn][G][G/2+1] its half spectrum
  cufftHandle planR = 0, planC = 0;
  bool nplans = false;
  float2 *twL = nullptr;          // [2 G] W_G^{j2 k1} in both orders (fused convolution)
  float2 *H = nullptr;            // [Hc][n + 1][n] half spectra, column-major
  int32_t Hc = 0;                 // slices per fused pass
};

namespace tomo {
void free_normal(tomo_fubini *F);
// the W_L^{j2 k1} tables of regfft.cuh for L = G (built once per handle)
tomo_status ensure_twiddles(tomo_fubini *F, cudaStream_t st);
// grids with the register-FFT passes (G a power of two, 32..2048)
inline bool fused_ok(int L) { return L >= 32 && L <= 2048 && (L & (L - 1)) == 0; }
}
