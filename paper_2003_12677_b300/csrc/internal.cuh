// internal.cuh -- shared definitions of libtomo (handle layout, error plumbing,
// per-angle constants).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "tomo.h"

namespace tomo {

// Per-angle constants of the chord-length rule (Sec. 2 projection integral),
// computed once on the host in IEEE FP64:
//   a = max(|cos|,|sin|), e = min(|cos|,|sin|), h = (a+e)/2, hm = (a-e)/2,
//   inv_a = 1/a, ae = a*e.  inv_cs / inv_sn only seed candidate searches.
struct AngleC {
  double cs, sn, a, e, h, hm, inv_a, ae, inv_cs, inv_sn;
};

struct Csr {
  int64_t rows = 0, cols = 0, nnz = 0, max_len = 0;
  int64_t *rp = nullptr;  // [rows+1]
  int32_t *ci = nullptr;  // [nnz]
  float *v = nullptr;     // [nnz]
};

// 16-bit encoding of one CSR operand.  Each row is cut into chunks of 16
// entries (the last one padded with zero weights); chunk c holds a 32-bit
// column base (the first column of the chunk) and, per entry, one uint32 that
// packs the uint16 column offset against that base (low half) with the 16-bit
// float weight (high half).  Weights are A_ij * a(theta) so that a full chord
// is exactly 1.0; the FP32 factor 1/a(theta) of the angle is applied by the
// kernels (per output row for A, per gathered input for A^T).
struct Lp {
  int64_t rows = 0, chunks = 0;
  int64_t *cp = nullptr;       // [rows+1] chunk pointers
  int32_t *base = nullptr;     // [chunks]
  uint32_t *ow = nullptr;      // [chunks*16] offset | weight << 16
};

}  // namespace tomo

struct tomo_matrix {
  int32_t nx = 0, ny = 0, np = 0, nt = 0;
  double center = 0;
  int device = 0;
  tomo::AngleC *ang = nullptr;   // device [nt]
  float *ang_scale = nullptr;    // device [nt]: 1/a(theta_m) in FP32
  tomo::Csr A, AT;
  float *R = nullptr, *C = nullptr;
  int32_t lp_dtype = TOMO_F32;
  tomo::Lp lpA, lpAT;
  int64_t bytes_f32 = 0, bytes_lp = 0;
};

namespace tomo {

void set_error(const std::string &msg);
tomo_status fail(tomo_status s, const std::string &msg);

#define TOMO_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess)                                                              \
      return ::tomo::fail(_e == cudaErrorMemoryAllocation ? TOMO_ERR_OOM : TOMO_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(_e));          \
  } while (0)

#define TOMO_TRY(expr)                   \
  do {                                   \
    tomo_status _s = (expr);             \
    if (_s != TOMO_OK) return _s;        \
  } while (0)

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// ---- matrix build (build.cu) ----
tomo_status build_matrix(const tomo_geometry *g, const tomo_matrix_opts *o, cudaStream_t st,
                         tomo_matrix **out);
void free_matrix(tomo_matrix *h);

// ---- operators (ops.cu) ----
struct Exec {
  int B = 0;          // slices per SpMM pass
  bool graph = true;
  bool lp = false;
  tomo_timing *timing = nullptr;
};
tomo_status resolve_exec(const tomo_matrix *h, const tomo_exec_opts *o, int32_t nz, Exec *ex);
size_t workspace_bytes(const tomo_matrix *h, int op, int32_t nz, const Exec &ex);
tomo_status run_project(const tomo_matrix *h, bool transpose, const float *in, float *out,
                        int32_t nz, int layout, const Exec &ex, void *ws, cudaStream_t st);
tomo_status run_sirt(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     float lambda, const Exec &ex, void *ws, cudaStream_t st);
tomo_status run_cgls(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     int32_t recompute, double *hist, const Exec &ex, void *ws, cudaStream_t st);

}  // namespace tomo
