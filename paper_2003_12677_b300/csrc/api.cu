// api.cu -- the extern "C" boundary of libtomo (declared in include/tomo.h).
// Argument checking, device selection and error strings live here; every
// computation is queued by build.cu / ops.cu.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace tomo {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

tomo_status fail(tomo_status s, const std::string &msg) {
  set_error(msg);
  return s;
}

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
      cudaSetDevice(dev);
    else
      prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static tomo_status check_vec(const void *p, const char *name) {
  if (!p) return fail(TOMO_ERR_INVALID_ARG, std::string(name) + " must be non-NULL");
  if (!aligned16(p)) return fail(TOMO_ERR_INVALID_ARG, std::string(name) + " must be 16-byte aligned");
  return TOMO_OK;
}

static bool pow2_width(int b) { return b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32 || b == 64; }

static tomo_status check_ws(const tomo_matrix *A, int op, int32_t n_z, const Exec &ex, void *ws, size_t bytes) {
  size_t need = workspace_bytes(A, op, n_z, ex);
  if (ws && bytes < need) return fail(TOMO_ERR_INVALID_ARG, "workspace too small: need " + std::to_string(need));
  if (ws && !aligned16(ws)) return fail(TOMO_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  return TOMO_OK;
}

}  // namespace tomo

using namespace tomo;

extern "C" {

tomo_status tomo_build_matrix(const tomo_geometry *geom, const tomo_matrix_opts *opts, void *stream,
                              tomo_matrix **out) {
  return build_matrix(geom, opts, (cudaStream_t)stream, out);
}

tomo_status tomo_matrix_destroy(tomo_matrix *A) {
  if (!A) return TOMO_OK;
  DeviceGuard dg(A->device);
  free_matrix(A);
  return TOMO_OK;
}

tomo_status tomo_matrix_info(const tomo_matrix *A, tomo_matrix_info_t *info) {
  if (!A || !info) return fail(TOMO_ERR_INVALID_ARG, "matrix and info must be non-NULL");
  std::memset(info, 0, sizeof(*info));
  info->rows = A->A.rows;
  info->cols = A->A.cols;
  info->nnz = A->A.nnz;
  info->bytes_f32 = A->bytes_f32;
  info->bytes_lp = A->bytes_lp;
  info->max_row_len = A->A.max_len;
  info->max_col_len = A->AT.max_len;
  info->lp_dtype = A->lp_dtype;
  info->at_tiles = A->lpATt.ent != nullptr ? 1 : 0;
  return TOMO_OK;
}

tomo_status tomo_matrix_export_rows(const tomo_matrix *A, int32_t transpose, int64_t row_begin, int64_t row_end,
                                    int64_t *row_ptr, int32_t *col, float *val, int64_t cap) {
  if (!A || !row_ptr) return fail(TOMO_ERR_INVALID_ARG, "matrix and row_ptr must be non-NULL");
  const Csr &M = transpose ? A->AT : A->A;
  if (row_begin < 0 || row_end < row_begin || row_end > M.rows)
    return fail(TOMO_ERR_INVALID_ARG, "row range out of bounds");
  if (!M.ci) return fail(TOMO_ERR_UNSUPPORTED, "matrix was built with drop_csr: nothing to export");
  DeviceGuard dg(A->device);
  const int64_t n = row_end - row_begin;
  if (cudaMemcpy(row_ptr, M.rp + row_begin, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(TOMO_ERR_CUDA, "copy of row pointers failed");
  const int64_t first = row_ptr[0], cnt = row_ptr[n] - first;
  for (int64_t i = 0; i <= n; ++i) row_ptr[i] -= first;
  if (cnt > cap) return fail(TOMO_ERR_INVALID_ARG, "export capacity too small: need " + std::to_string(cnt));
  if (cnt > 0) {
    if (!col || !val) return fail(TOMO_ERR_INVALID_ARG, "col and val must be non-NULL");
    if (cudaMemcpy(col, M.ci + first, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(val, M.v + first, sizeof(float) * cnt, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(TOMO_ERR_CUDA, "copy of entries failed");
  }
  return TOMO_OK;
}

tomo_status tomo_matrix_export_csr(const tomo_matrix *A, int32_t transpose, int64_t *row_ptr, int32_t *col, float *val,
                                   void *stream) {
  if (!A || !row_ptr || !col || !val) return fail(TOMO_ERR_INVALID_ARG, "matrix, row_ptr, col and val must be non-NULL");
  const Csr &M = transpose ? A->AT : A->A;
  if (!M.ci) return fail(TOMO_ERR_UNSUPPORTED, "matrix was built with drop_csr: nothing to export");
  DeviceGuard dg(A->device);
  const cudaStream_t st = (cudaStream_t)stream;
  TOMO_CUDA(cudaMemcpyAsync(row_ptr, M.rp, sizeof(int64_t) * (M.rows + 1), cudaMemcpyDeviceToHost, st));
  if (M.nnz > 0) {
    TOMO_CUDA(cudaMemcpyAsync(col, M.ci, sizeof(int32_t) * M.nnz, cudaMemcpyDeviceToHost, st));
    TOMO_CUDA(cudaMemcpyAsync(val, M.v, sizeof(float) * M.nnz, cudaMemcpyDeviceToHost, st));
  }
  TOMO_CUDA(cudaStreamSynchronize(st));
  return TOMO_OK;
}

tomo_status tomo_matrix_export_norms(const tomo_matrix *A, float *R, float *C) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  DeviceGuard dg(A->device);
  if (R && cudaMemcpy(R, A->R, sizeof(float) * A->A.rows, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(TOMO_ERR_CUDA, "copy of R failed");
  if (C && cudaMemcpy(C, A->C, sizeof(float) * A->A.cols, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(TOMO_ERR_CUDA, "copy of C failed");
  return TOMO_OK;
}

tomo_status tomo_workspace_size(const tomo_matrix *A, int32_t op, int32_t n_z, const tomo_exec_opts *opts,
                                size_t *bytes) {
  if (!A || !bytes) return fail(TOMO_ERR_INVALID_ARG, "matrix and bytes must be non-NULL");
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (op < TOMO_OP_PROJECT || op > TOMO_OP_RESIDUAL) return fail(TOMO_ERR_INVALID_ARG, "unknown op");
  if (op == TOMO_OP_RESIDUAL) {
    *bytes = sizeof(double) * (size_t)residual_parts();
    return TOMO_OK;
  }
  Exec ex;
  TOMO_TRY(resolve_exec(A, opts, n_z, &ex));
  *bytes = workspace_bytes(A, op, n_z, ex);
  return TOMO_OK;
}

static tomo_status project_common(const tomo_matrix *A, bool trans, const float *in, float *out, int32_t n_z,
                                  int32_t layout, const tomo_exec_opts *opts, void *ws, size_t ws_bytes,
                                  void *stream) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  TOMO_TRY(check_vec(in, trans ? "y" : "x"));
  TOMO_TRY(check_vec(out, trans ? "x" : "y"));
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (layout != TOMO_SLICE_MAJOR && layout != TOMO_INTERLEAVED)
    return fail(TOMO_ERR_INVALID_ARG, "layout must be TOMO_SLICE_MAJOR or TOMO_INTERLEAVED");
  DeviceGuard dg(A->device);
  Exec ex;
  tomo_exec_opts o = opts ? *opts : tomo_exec_opts{};
  if (!opts) o.use_graph = 1;
  if (layout == TOMO_INTERLEAVED) {
    if (!pow2_width(n_z)) return fail(TOMO_ERR_UNSUPPORTED, "interleaved layout needs n_z in {1,2,4,8,16,32,64}");
    o.batch_width = n_z;
  }
  TOMO_TRY(resolve_exec(A, &o, n_z, &ex));
  TOMO_TRY(check_ws(A, trans ? TOMO_OP_BACKPROJECT : TOMO_OP_PROJECT, n_z, ex, ws, ws_bytes));
  return run_project(A, trans, in, out, n_z, layout, ex, ws, (cudaStream_t)stream);
}

tomo_status tomo_project(const tomo_matrix *A, const float *x, float *y, int32_t n_z, int32_t layout,
                         const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes, void *stream) {
  return project_common(A, false, x, y, n_z, layout, opts, workspace, workspace_bytes, stream);
}

tomo_status tomo_backproject(const tomo_matrix *A, const float *y, float *x, int32_t n_z, int32_t layout,
                             const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes, void *stream) {
  return project_common(A, true, y, x, n_z, layout, opts, workspace, workspace_bytes, stream);
}

tomo_status tomo_sirt(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters, float lambda,
                      const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes, void *stream) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  if (n_z < 1 || iters < 0) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1 and iters >= 0");
  if (!std::isfinite(lambda)) return fail(TOMO_ERR_INVALID_ARG, "lambda must be finite");
  DeviceGuard dg(A->device);
  Exec ex;
  TOMO_TRY(resolve_exec(A, opts, n_z, &ex));
  TOMO_TRY(check_ws(A, TOMO_OP_SIRT, n_z, ex, workspace, workspace_bytes));
  if (iters == 0) return TOMO_OK;
  return run_sirt(A, sino, x, n_z, iters, lambda, ex, workspace, (cudaStream_t)stream);
}

tomo_status tomo_residual_norm(const tomo_matrix *A, const float *sino, const float *x, int32_t n_z, double *norms,
                               void *workspace, size_t workspace_bytes, void *stream) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  if (!norms || ((uintptr_t)norms & 7u)) return fail(TOMO_ERR_INVALID_ARG, "norms must be non-NULL and 8-byte aligned");
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (!A->A.ci) return fail(TOMO_ERR_UNSUPPORTED, "matrix was built with drop_csr");
  DeviceGuard dg(A->device);
  if (workspace) {
    if (!aligned16(workspace)) return fail(TOMO_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    if (workspace_bytes < sizeof(double) * (size_t)residual_parts())
      return fail(TOMO_ERR_INVALID_ARG,
                  "workspace too small: need " + std::to_string(sizeof(double) * (size_t)residual_parts()));
  }
  return run_residual_norm(A, sino, x, n_z, norms, workspace, (cudaStream_t)stream);
}

static tomo_status check_state(const tomo_cgls_state *s, const char *name) {
  if (!s) return TOMO_OK;
  if (!s->gamma || !s->frozen) return fail(TOMO_ERR_INVALID_ARG, std::string(name) + ": gamma and frozen must be set");
  TOMO_TRY(check_vec(s->r, "state r"));
  TOMO_TRY(check_vec(s->p, "state p"));
  if (((uintptr_t)s->gamma & 7u) || ((uintptr_t)s->frozen & 3u))
    return fail(TOMO_ERR_INVALID_ARG, std::string(name) + ": gamma / frozen misaligned");
  return TOMO_OK;
}

tomo_status tomo_cgls_resume(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                             int32_t recompute_every, double *resnorm_hist, const tomo_cgls_state *in,
                             tomo_cgls_state *out, const tomo_exec_opts *opts, void *workspace,
                             size_t workspace_bytes, void *stream) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  TOMO_TRY(check_state(in, "in"));
  TOMO_TRY(check_state(out, "out"));
  if (n_z < 1 || iters < 0 || recompute_every < 0)
    return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1, iters >= 0 and recompute_every >= 0");
  DeviceGuard dg(A->device);
  Exec ex;
  TOMO_TRY(resolve_exec(A, opts, n_z, &ex));
  TOMO_TRY(check_ws(A, TOMO_OP_CGLS, n_z, ex, workspace, workspace_bytes));
  return run_cgls(A, sino, x, n_z, iters, recompute_every, resnorm_hist, in, out, ex, workspace,
                  (cudaStream_t)stream);
}

tomo_status tomo_cgls(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                      int32_t recompute_every, double *resnorm_hist, const tomo_exec_opts *opts, void *workspace,
                      size_t workspace_bytes, void *stream) {
  return tomo_cgls_resume(A, sino, x, n_z, iters, recompute_every, resnorm_hist, nullptr, nullptr, opts, workspace,
                          workspace_bytes, stream);
}

static tomo_status check_bb_state(const tomo_bb_state *s, const char *name) {
  if (!s) return TOMO_OK;
  if (!s->alpha || !s->frozen) return fail(TOMO_ERR_INVALID_ARG, std::string(name) + ": alpha and frozen must be set");
  TOMO_TRY(check_vec(s->g, "state g"));
  if (((uintptr_t)s->alpha & 7u) || ((uintptr_t)s->frozen & 3u))
    return fail(TOMO_ERR_INVALID_ARG, std::string(name) + ": alpha / frozen misaligned");
  return TOMO_OK;
}

tomo_status tomo_sirt_bb(const tomo_matrix *A, const float *sino, float *x, int32_t n_z, int32_t iters,
                         double first_step, double *resnorm_hist, const tomo_bb_state *in, tomo_bb_state *out,
                         const tomo_exec_opts *opts, void *workspace, size_t workspace_bytes, void *stream) {
  if (!A) return fail(TOMO_ERR_INVALID_ARG, "matrix must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  TOMO_TRY(check_bb_state(in, "in"));
  TOMO_TRY(check_bb_state(out, "out"));
  if (n_z < 1 || iters < 0) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1 and iters >= 0");
  if (!std::isfinite(first_step)) return fail(TOMO_ERR_INVALID_ARG, "first_step must be finite");
  if (resnorm_hist && ((uintptr_t)resnorm_hist & 7u)) return fail(TOMO_ERR_INVALID_ARG, "resnorm_hist misaligned");
  DeviceGuard dg(A->device);
  Exec ex;
  TOMO_TRY(resolve_exec(A, opts, n_z, &ex));
  TOMO_TRY(check_ws(A, TOMO_OP_SIRT_BB, n_z, ex, workspace, workspace_bytes));
  return run_sirt_bb(A, sino, x, n_z, iters, first_step, resnorm_hist, in, out, ex, workspace,
                     (cudaStream_t)stream);
}

tomo_status tomo_cgls_batched(const tomo_request *reqs, int32_t n_reqs, int32_t iters, const tomo_exec_opts *opts,
                              void *workspace, size_t workspace_bytes, void *stream) {
  if (!reqs || n_reqs < 1 || !reqs[0].A) return fail(TOMO_ERR_INVALID_ARG, "need at least one request");
  if (workspace && !aligned16(workspace)) return fail(TOMO_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  DeviceGuard dg(reqs[0].A->device);
  return run_cgls_batched(reqs, n_reqs, iters, opts, workspace, workspace_bytes, (cudaStream_t)stream);
}

tomo_status tomo_cgls_batched_workspace(const tomo_request *reqs, int32_t n_reqs, const tomo_exec_opts *opts,
                                        size_t *bytes) {
  if (!bytes) return fail(TOMO_ERR_INVALID_ARG, "bytes must be non-NULL");
  return batched_workspace(reqs, n_reqs, opts, bytes);
}

tomo_status tomo_autotune(tomo_matrix *A, int32_t n_z, int32_t allow_16bit, tomo_exec_opts *best, double *rate,
                          tomo_tune_entry *table, int32_t cap, int32_t *n_table, void *stream) {
  if (!A || !best) return fail(TOMO_ERR_INVALID_ARG, "matrix and best must be non-NULL");
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (cap < 0 || (cap > 0 && !table)) return fail(TOMO_ERR_INVALID_ARG, "table must hold cap entries");
  DeviceGuard dg(A->device);
  return run_autotune(A, n_z, allow_16bit, best, rate, table, cap, n_table, (cudaStream_t)stream);
}

tomo_status tomo_fubini_create(const tomo_geometry *geom, int32_t kw, void *stream, tomo_fubini **out) {
  return fubini_create(geom, kw, (cudaStream_t)stream, out);
}

tomo_status tomo_fubini_destroy(tomo_fubini *F) {
  fubini_destroy(F);
  return TOMO_OK;
}

tomo_status tomo_fubini_project(tomo_fubini *F, const float *x, float *y, int32_t n_z, void *stream) {
  if (!F) return fail(TOMO_ERR_INVALID_ARG, "handle must be non-NULL");
  TOMO_TRY(check_vec(x, "x"));
  TOMO_TRY(check_vec(y, "y"));
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  return fubini_project(F, x, y, n_z, (cudaStream_t)stream);
}

tomo_status tomo_fubini_backproject(tomo_fubini *F, const float *y, float *x, int32_t n_z, int32_t filter,
                                    void *stream) {
  if (!F) return fail(TOMO_ERR_INVALID_ARG, "handle must be non-NULL");
  TOMO_TRY(check_vec(y, "y"));
  TOMO_TRY(check_vec(x, "x"));
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (filter < 0 || filter > 2) return fail(TOMO_ERR_INVALID_ARG, "filter must be 0, 1 or 2");
  return fubini_backproject(F, y, x, n_z, filter, (cudaStream_t)stream);
}

tomo_status tomo_fubini_sirt_bb(tomo_fubini *F, const float *sino, float *x, int32_t n_z, int32_t iters,
                                double *resnorm_hist, void *stream) {
  if (!F) return fail(TOMO_ERR_INVALID_ARG, "handle must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  if (n_z < 1 || iters < 0) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1 and iters >= 0");
  if (resnorm_hist && ((uintptr_t)resnorm_hist & 7u)) return fail(TOMO_ERR_INVALID_ARG, "resnorm_hist misaligned");
  return fubini_sirt_bb(F, sino, x, n_z, iters, resnorm_hist, (cudaStream_t)stream);
}

tomo_status tomo_tv(const float *x, int32_t n_z, int32_t n_y, int32_t n_x, float eps, double *loss, float *grad,
                    void *stream) {
  TOMO_TRY(check_vec(x, "x"));
  TOMO_TRY(check_vec(grad, "grad"));
  if (!loss || ((uintptr_t)loss & 7u)) return fail(TOMO_ERR_INVALID_ARG, "loss must be non-NULL and 8-byte aligned");
  if (n_z < 1 || n_z > 65535 || n_y < 1 || n_x < 1)
    return fail(TOMO_ERR_INVALID_ARG, "need 1 <= n_z <= 65535, n_y >= 1, n_x >= 1");
  if (!(eps > 0.f) || !std::isfinite(eps)) return fail(TOMO_ERR_INVALID_ARG, "eps must be positive and finite");
  // the kernel works with eps^2 in FP32: below ~1.1e-19 it underflows, and flat regions would divide by 0
  if (eps * eps < FLT_MIN) return fail(TOMO_ERR_INVALID_ARG, "eps must be at least 1.1e-19 (eps^2 is a normal FP32)");
  return tv_loss_grad(x, n_z, n_y, n_x, eps, loss, grad, (cudaStream_t)stream);
}

tomo_status tomo_fubini_normal(tomo_fubini *F, const float *x, float *y, int32_t n_z, int32_t filter, void *stream) {
  if (!F) return fail(TOMO_ERR_INVALID_ARG, "handle must be non-NULL");
  TOMO_TRY(check_vec(x, "x"));
  TOMO_TRY(check_vec(y, "y"));
  if (n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1");
  if (filter < 0 || filter > 2) return fail(TOMO_ERR_INVALID_ARG, "filter must be 0, 1 or 2");
  return fubini_normal(F, x, y, n_z, filter, (cudaStream_t)stream);
}

tomo_status tomo_fubini_sirt_bb_normal(tomo_fubini *F, const float *sino, float *x, int32_t n_z, int32_t iters,
                                       double *gradnorm_hist, void *stream) {
  if (!F) return fail(TOMO_ERR_INVALID_ARG, "handle must be non-NULL");
  TOMO_TRY(check_vec(sino, "sino"));
  TOMO_TRY(check_vec(x, "x"));
  if (n_z < 1 || iters < 0) return fail(TOMO_ERR_INVALID_ARG, "n_z must be >= 1 and iters >= 0");
  if (n_z > 65535) return fail(TOMO_ERR_INVALID_ARG, "n_z must be <= 65535");
  if (gradnorm_hist && ((uintptr_t)gradnorm_hist & 7u)) return fail(TOMO_ERR_INVALID_ARG, "gradnorm_hist misaligned");
  return fubini_sirt_bb_normal(F, sino, x, n_z, iters, gradnorm_hist, (cudaStream_t)stream);
}

const char *tomo_status_string(tomo_status s) {
  switch (s) {
    case TOMO_OK: return "TOMO_OK";
    case TOMO_ERR_INVALID_ARG: return "TOMO_ERR_INVALID_ARG";
    case TOMO_ERR_OOM: return "TOMO_ERR_OOM";
    case TOMO_ERR_CUDA: return "TOMO_ERR_CUDA";
    case TOMO_ERR_TIMEOUT: return "TOMO_ERR_TIMEOUT";
    case TOMO_ERR_UNSUPPORTED: return "TOMO_ERR_UNSUPPORTED";
    case TOMO_ERR_NUMERIC: return "TOMO_ERR_NUMERIC";
    case TOMO_ERR_IO: return "TOMO_ERR_IO";
  }
  return "TOMO_ERR_UNKNOWN";
}

const char *tomo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
