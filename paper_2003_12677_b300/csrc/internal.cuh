// internal.cuh -- shared definitions of libtomo (handle layout, error plumbing,
// per-angle constants).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tomo.h"

namespace tomo {

// Per-angle constants of the chord-length rule (Sec. 2 projection integral),
// computed once on the host in IEEE FP64:
//   a = max(|cos|,|sin|), e = min(|cos|,|sin|), h = (a+e)/2, hm = (a-e)/2,
//   inv_a = 1/a, ae = a*e.  inv_cs / inv_sn only seed candidate searches.
struct AngleC {
  double cs, sn, a, e, h, hm, inv_a, ae, inv_cs, inv_sn;
  double hs;  // support half width: h (line model) or h + 1/2 (strip model)
};

struct Csr {
  int64_t rows = 0, cols = 0, nnz = 0, max_len = 0;
  int64_t *rp = nullptr;  // [rows+1]
  int32_t *ci = nullptr;  // [nnz]
  float *v = nullptr;     // [nnz]
};

// SELL-32 form of one operand (FP32).  Rows are grouped in chunks of 32
// consecutive rows; chunk c is stored column-major with width W_c (the
// longest row of the chunk, rounded up to even), entries packed as int2
// (column, value bits) and kept in pairs so that one 128-bit load brings two
// consecutive entries of one row:
//   slot(c, q, e) = cp[c] + (e/2)*64 + 2*q + (e%2),   q = row % 32.
// The G rows a warp handles are adjacent in every column, so their entry
// loads are contiguous.  rl holds each row's true length; the kernels never
// read past it.
struct Sell {
  int64_t rows = 0, chunks = 0, slots = 0;
  int64_t *cp = nullptr;   // [chunks+1] slot offset of each chunk
  int32_t *rl = nullptr;   // [rows]
  int2 *ent = nullptr;     // [slots]
};

// 16-bit SELL-32 form.  Per entry one uint32 packs the uint16 column offset
// (low half) with the 16-bit float weight (high half); the offset is taken
// against a 32-bit base per row segment of 16 slots (the segment's first
// column).  A segment is closed early, padded with zero-weight slots, when the
// next column lies more than 65535 past its base; rl holds each row's padded
// slot count (a multiple of 16).  Quads of consecutive slots of a row are
// adjacent:
//   slot(c, q, e) = cpw[c] + (e/4)*128 + 4*q + (e%4),   width W_c % 16 == 0
//   base(c, q, s) = cpb[c] + s*32 + q,                    s = e/16.
// Weights are A_ij * a(theta) so that a full chord is exactly 1.0; the FP32
// factor 1/a(theta) of the angle is applied by the kernels (per output row
// for A, per gathered entry for A^T).  Padding slots carry weight 0 and
// offset 0 (column = the segment base).
// The 16-bit A may store its rows in pair order (nb4 > 0, n_theta even and n_p
// a multiple of 4): row rho holds ray ray_of(rho), so that each group of 8
// consecutive rows (the rows one warp takes at batch width 16) is 2 adjacent
// angles x 4 adjacent bins, whose gathers meet the same image rows more often
// than 8 bins of one angle do.
struct SellLp {
  int64_t rows = 0, chunks = 0, slots = 0, bases = 0;
  int32_t nb4 = 0;          // n_p / 4 when the rows are in pair order, else 0
  int64_t *cpw = nullptr;   // [chunks+1]
  int64_t *cpb = nullptr;   // [chunks+1]
  int32_t *rl = nullptr;    // [rows] padded slot count per row
  uint32_t *ow = nullptr;   // [slots]
  int32_t *base = nullptr;  // [bases]
};

// the ray (row of A) that row rho of a 16-bit A in pair order holds
__host__ __device__ __forceinline__ int64_t ray_of(int64_t rho, int nb4, int np) {
  if (nb4 == 0) return rho;
  const int64_t grp = rho >> 3, m2 = grp / nb4;
  const int j = (int)(rho & 7), b4 = (int)(grp - m2 * nb4);
  return (2 * m2 + (j >> 2)) * np + 4 * b4 + (j & 3);
}

// 16-bit A^T in image tiles, for a pass that stages each tile's detector
// window in shared memory (k_spmm_tile16).  The image is cut into tiles of
// kTileSide x kTileSide pixels (t = ty * tiles_x + tx; the last column and row
// of tiles may be ragged) and the angles into chunks of kTileChunk.  For tile t
// and angle m, win[t * n_theta + m] is the first bin of a window of W bins that
// holds every bin the tile's pixels meet at m (clamped into [0, n_p - W] when
// n_p >= W); window row r = (m - k kTileChunk) W + bin - win of chunk k is
// staged at position swz(r) (bits 0 and 1 of r swapped).  W <= 32.
//
// The pixels form 2 x 2 quads: group g (0..7) is the tile's pixel rows 2g and
// 2g + 1, quad i (0..7) of a group its pixel columns 2i and 2i + 1, pixel
// a = 2 dy + dx of a quad.  At angle m a quad walks the bins from the lowest
// to the highest that any of its pixels meets, in that order, one slot per
// bin: a slot carries the staged row of its bin and the 16-bit weights of the
// four pixels there (0 where a pixel has no entry).  A quad's slots for chunk
// k are its angles' runs in angle order; each pixel meets its entries in its
// CSR order.  The group's quads are padded with weight-0 slots to its longest
// quad, rounded up to blocks of kTileBlockSlots slots.  Block j of group g of
// (t, k) is ent + 72 (qoff[(t * nch + k) * 8 + g] + j) words:
//   bytes   0..127  slots 0, 1: quad i at 16 i (slot 0: 8 bytes, then slot 1)
//   bytes 128..255  slots 2, 3: the same
//   bytes 256..287  staged row positions: quad i at 4 i, slot s in byte s
// where a slot's 8 bytes hold the weights of pixels 0..3 (2 bytes each, in
// order).  A padding slot reads the row of the other quad of its
// shared-memory phase (quad i ^ 1) at that slot, or row 0.  The offsets run
// over (t, k, g) in that order; qoff[.. + 1] - qoff[..] is the group's block
// count.
constexpr int kTileSide = 16;
constexpr int kTileChunk = 8;
constexpr int kTileRow = 64;          // bytes of a staged window row (16 slices)
constexpr int kTileBlockSlots = 4;    // slots of one entry block
constexpr int kTileBlockBytes = 288;  // bytes of one entry block
__host__ __device__ constexpr int tile_swz(int r) { return (r & ~3) | ((r & 1) << 1) | ((r >> 1) & 1); }
struct TileLp {
  int64_t tiles = 0, blocks = 0;
  int32_t tiles_x = 0, tiles_y = 0, nch = 0, W = 0;
  int32_t max_blocks = 0;     // most blocks of one (tile, chunk)
  uint32_t *qoff = nullptr;   // [tiles * nch * 8 + 4] (3 zero words of padding)
  int32_t *win = nullptr;     // [tiles * n_theta]
  uint32_t *ent = nullptr;    // [blocks * 72]
};

}  // namespace tomo

struct tomo_matrix {
  int32_t nx = 0, ny = 0, np = 0, nt = 0;
  int32_t model = TOMO_MODEL_LINE;
  double center = 0;
  int device = 0;
  tomo::AngleC *ang = nullptr;   // device [nt]
  float *ang_scale = nullptr;    // device [nt]: 1/a(theta_m) in FP32
  tomo::Csr A, AT;
  float *R = nullptr, *C = nullptr;
  float *ramp = nullptr;         // device [np]: taps |d| = 0..np-1 of the preconditioning filter
  int32_t lp_dtype = TOMO_F32;
  tomo::Sell sA, sAT;
  tomo::SellLp lpA, lpAT;
  // 16-bit A stored as column bands (bands of image rows, each its own 16-bit
  // SELL-32 matrix over all rows of A) when built with col_blocks > 1; lpA is
  // then empty
  std::vector<tomo::SellLp> lpAb;
  // the 16-bit A^T also in image tiles (ent == nullptr when not built)
  tomo::TileLp lpATt;
  int64_t bytes_f32 = 0, bytes_lp = 0;
  // tomo_autotune's choice per slice count (most recent first)
  struct Tuned {
    int32_t nz, B, fmt, order, blocks;
  };
  std::vector<Tuned> tuned;
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
  int B = 0;            // slices per SpMM pass
  bool graph = true;
  int format = TOMO_FMT_SELL;
  tomo_timing *timing = nullptr;
  bool recompute_fp32 = false;  // CGLS on 16-bit values: residual recompute with the FP32 values
  int order = 0;                // A^T row-group order: 0 auto, 1 rows, 2 image tiles, 3 staged tiles
  int blocks = 0;               // SpMM blocks per SM (0: all that fit)
};
tomo_status resolve_exec(const tomo_matrix *h, const tomo_exec_opts *o, int32_t nz, Exec *ex);
size_t workspace_bytes(const tomo_matrix *h, int op, int32_t nz, const Exec &ex);
tomo_status run_project(const tomo_matrix *h, bool transpose, const float *in, float *out,
                        int32_t nz, int layout, const Exec &ex, void *ws, cudaStream_t st);
tomo_status run_sirt(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     float lambda, const Exec &ex, void *ws, cudaStream_t st);
tomo_status run_cgls(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                     int32_t recompute, double *hist, const tomo_cgls_state *in, tomo_cgls_state *out,
                     const Exec &ex, void *ws, cudaStream_t st);
// ||b - A x|| per slice with FP64 accumulation (ops.cu); ws: residual_parts() doubles
int residual_parts();
tomo_status run_residual_norm(const tomo_matrix *h, const float *sino, const float *x, int32_t nz, double *norms,
                              void *ws, cudaStream_t st);
tomo_status run_sirt_bb(const tomo_matrix *h, const float *sino, float *x, int32_t nz, int32_t iters,
                        double first_step, double *hist, const tomo_bb_state *in, tomo_bb_state *out,
                        const Exec &ex, void *ws, cudaStream_t st);
tomo_status batched_workspace(const tomo_request *reqs, int32_t n, const tomo_exec_opts *o, size_t *bytes);
// Fubini-Radon transform (fubini.cu)
tomo_status fubini_create(const tomo_geometry *g, int32_t kw, cudaStream_t st, tomo_fubini **out);
void fubini_destroy(tomo_fubini *F);
tomo_status fubini_project(tomo_fubini *F, const float *x, float *y, int32_t nz, cudaStream_t st);
tomo_status fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t nz, int filter, cudaStream_t st);
tomo_status fubini_sirt_bb(tomo_fubini *F, const float *sino, float *x, int32_t nz, int32_t iters, double *hist,
                           cudaStream_t st);
// TV prior value and gradient (tv.cu)
tomo_status tv_loss_grad(const float *x, int32_t nz, int32_t ny, int32_t nx, float eps, double *loss, float *grad,
                         cudaStream_t st);
// its normal operator in one step (normal.cu)
tomo_status fubini_normal(tomo_fubini *F, const float *x, float *y, int32_t nz, int filter, cudaStream_t st);
tomo_status fubini_sirt_bb_normal(tomo_fubini *F, const float *sino, float *x, int32_t nz, int32_t iters,
                                  double *hist, cudaStream_t st);
// per-stream status word (status.cu)
int *stream_status_word(cudaStream_t st);
tomo_status fold_status(const int *src, cudaStream_t st);
tomo_status read_stream_status(cudaStream_t st);
tomo_status run_cgls_batched(const tomo_request *reqs, int32_t n, int32_t iters, const tomo_exec_opts *o,
                             void *ws, size_t ws_bytes, cudaStream_t st);
tomo_status run_autotune(tomo_matrix *h, int32_t nz, int allow16, tomo_exec_opts *best, double *rate,
                         tomo_tune_entry *table, int32_t cap, int32_t *n_table, cudaStream_t st);

}  // namespace tomo
