/*
 * tomo_oracle.c -- FP64 CPU oracle for the parallel-beam line-model projector.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper: "Sparse Matrix-Based HPC Tomography"):
 *   - the projection integral of Sec. 2, P_theta(p) = integral of u along the
 *     line x cos(theta) + y sin(theta) = p, discretised for a piecewise-constant
 *     pixel image: A[(m,k),(ix,iy)] = length of the chord that the ray of angle
 *     theta_m through bin k cuts from pixel (ix,iy);
 *   - Sec. 3.1: entries are generated, zero / out-of-range ones dropped, and the
 *     result stored as CSR sorted by row and column; the transpose is stored
 *     separately (here: the plain counting-sort transpose of that CSR);
 *   - Sec. 2.1: SIRT and CGLS on the least-squares problem, and the gradient of
 *     the model-based objective ||A x - b||^2 + mu * TV(x).
 *
 * Geometry (the paper fixes the integral, not the grid; the readings are):
 *   pixel (ix,iy) is the unit square centred at x = ix+1/2-nx/2, y = iy+1/2-ny/2,
 *   column j = iy*nx + ix; row i = m*n_p + k; bin centre p_k = k + 1/2 - c,
 *   c = n_p/2 when the rotation axis is centred (Sec. 3).
 *
 * Chord length of the line {x cs + y sn = p} through the square centred at
 * (x, y): with a = max(|cs|,|sn|), e = min(|cs|,|sn|), h = (a+e)/2 and
 * delta = |p - (x cs + y sn)|, the chord is 1/a on the plateau delta <= (a-e)/2,
 * falls linearly to 0 at delta = h, and the pixel is hit iff delta < h.
 * Every quantity is evaluated in IEEE FP64, round-to-nearest, in the order
 * written, with no contraction (build with -ffp-contract=off).
 *
 * Parity status of each function is recorded beside it; all are pinned by the
 * CPU tests (special angles, brute-force clipping, closed-form projections,
 * mass conservation, adjointness, Krylov / least-squares minimisers, finite
 * differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Default angle set theta_m = m*pi/n_theta over [0, pi). */
void oracle_default_angles(int32_t nt, double *theta) {
  for (int32_t m = 0; m < nt; ++m) theta[m] = (double)m * M_PI / (double)nt;
}

/* cos / sin table of the angles (FP64, C library). */
void oracle_trig(int32_t nt, const double *theta, double *cs, double *sn) {
  for (int32_t m = 0; m < nt; ++m) {
    cs[m] = cos(theta[m]);
    sn[m] = sin(theta[m]);
  }
}

/* Strip model: F(s) = integral of the chord length over offsets [0, s], s >= 0.
 * The chord length at offset s from the pixel centre's projection is a
 * trapezoid: 1/a for |s| <= hm, (h - |s|)/(a e) for hm < |s| < h, 0 beyond;
 * F reaches 1/2 (half the pixel's area) at s = h.  Operation order fixed. */
static double strip_F(double s, double inv_a, double ae, double h, double hm) {
  if (s <= hm) return s * inv_a;
  if (s >= h) return 0.5;
  return hm * inv_a + (s - hm) * (h - 0.5 * (s + hm)) / ae;
}

/* Weight of ray (cs, sn, bin k) and pixel (ix, iy).  model 0 (line): the
 * chord length of the line x cos + y sin = p_k through the pixel square, hit
 * iff delta < h.  model 1 (strip): the area of the pixel square inside the
 * strip |x cos + y sin - p_k| < 1/2, i.e. the line integral of Sec. 2 averaged
 * over a detector bin of unit width: F(delta + 1/2) - F(delta - 1/2) with F
 * odd, hit iff delta < h + 1/2.  Returns 1 and stores the weight on a hit.
 * Pinned: Liang-Barsky clipping (line) and polygon clipping (strip) on 8x8
 * grids, theta = 0 and pi/2 special cases, exact mass of the strip model. */
int oracle_weight(int32_t nx, int32_t ny, double c, double cs, double sn,
                  int32_t k, int32_t ix, int32_t iy, double *len, int32_t model) {
  double acs = fabs(cs), asn = fabs(sn);
  double a = acs > asn ? acs : asn;
  double e = acs > asn ? asn : acs;
  double h = 0.5 * (a + e);
  double hm = 0.5 * (a - e);
  double x = ((double)ix + 0.5) - 0.5 * (double)nx;
  double y = ((double)iy + 0.5) - 0.5 * (double)ny;
  double pk = ((double)k + 0.5) - c;
  double t = x * cs + y * sn;
  double d = pk - t;
  double del = fabs(d);
  if (model == 1) {
    if (!(del < h + 0.5)) return 0;
    double inv_a = 1.0 / a, ae = a * e;
    double dp = del + 0.5, dm = del - 0.5;
    double Fp = strip_F(dp, inv_a, ae, h, hm);
    double Fm = dm >= 0.0 ? strip_F(dm, inv_a, ae, h, hm) : -strip_F(-dm, inv_a, ae, h, hm);
    *len = Fp - Fm;
    return 1;
  }
  if (!(del < h)) return 0;
  if (del <= hm)
    *len = 1.0 / a;
  else
    *len = (h - del) / (a * e);
  return 1;
}

/* Bins k whose ray can hit the pixel centred at t = x cs + y sn.
 * |p_k - t| < h <= 1/sqrt(2) (line) or < h + 1/2 <= 1.21 (strip) means k lies
 * within 1.21 of u = t + c - 1/2, so the five integers floor(u)-2 .. floor(u)+2
 * contain every hit; each candidate is then decided by oracle_weight itself. */
static void candidate_bins(double c, double cs, double sn, int32_t nx, int32_t ny,
                           int32_t ix, int32_t iy, int64_t *k0) {
  double x = ((double)ix + 0.5) - 0.5 * (double)nx;
  double y = ((double)iy + 0.5) - 0.5 * (double)ny;
  double u = x * cs + y * sn + c - 0.5;
  *k0 = (int64_t)floor(u) - 2;
}

/* Number of entries in each row of A (rows = n_theta * n_p).  Returns nnz. */
int64_t oracle_count(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c,
                     const double *cs, const double *sn, int64_t *row_count, int32_t model) {
  int64_t rows = (int64_t)nt * np_;
  memset(row_count, 0, sizeof(int64_t) * rows);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t m = 0; m < nt; ++m) {
    for (int32_t iy = 0; iy < ny; ++iy)
      for (int32_t ix = 0; ix < nx; ++ix) {
        int64_t k0;
        candidate_bins(c, cs[m], sn[m], nx, ny, ix, iy, &k0);
        for (int64_t k = k0; k < k0 + 5; ++k) {
          double L;
          if (k < 0 || k >= np_) continue;
          if (oracle_weight(nx, ny, c, cs[m], sn[m], (int32_t)k, ix, iy, &L, model))
            row_count[(int64_t)m * np_ + k]++;
        }
      }
  }
  int64_t nnz = 0;
  for (int64_t i = 0; i < rows; ++i) nnz += row_count[i];
  return nnz;
}

/* Fill CSR of A given row_ptr (exclusive prefix sum of the counts).
 * Within a row, columns come out ascending because pixels are visited in
 * increasing j = iy*nx + ix. */
void oracle_fill(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c,
                 const double *cs, const double *sn, const int64_t *row_ptr,
                 int32_t *col, double *val, int32_t model) {
#pragma omp parallel
  {
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)np_);
#pragma omp for schedule(dynamic, 1)
    for (int32_t m = 0; m < nt; ++m) {
      for (int32_t k = 0; k < np_; ++k) cursor[k] = row_ptr[(int64_t)m * np_ + k];
      for (int32_t iy = 0; iy < ny; ++iy)
        for (int32_t ix = 0; ix < nx; ++ix) {
          int64_t k0;
          candidate_bins(c, cs[m], sn[m], nx, ny, ix, iy, &k0);
          for (int64_t k = k0; k < k0 + 5; ++k) {
            double L;
            if (k < 0 || k >= np_) continue;
            if (oracle_weight(nx, ny, c, cs[m], sn[m], (int32_t)k, ix, iy, &L, model)) {
              int64_t e = cursor[k]++;
              col[e] = iy * nx + ix;
              val[e] = L;
            }
          }
        }
    }
    free(cursor);
  }
}

/* One row of A by brute force over every pixel (for sampling huge matrices).
 * Returns the entry count; writes at most cap entries. */
int64_t oracle_row(int32_t nx, int32_t ny, int32_t np_, double c, double cs, double sn,
                   int32_t k, int32_t *col, double *val, int64_t cap, int32_t model) {
  int64_t n = 0;
  for (int32_t iy = 0; iy < ny; ++iy)
    for (int32_t ix = 0; ix < nx; ++ix) {
      double L;
      if (oracle_weight(nx, ny, c, cs, sn, k, ix, iy, &L, model)) {
        if (n < cap) {
          col[n] = iy * nx + ix;
          val[n] = L;
        }
        ++n;
      }
    }
  (void)np_;
  return n;
}

/* One row of A^T (pixel j = iy*nx + ix): its rays (m, k) in increasing
 * m*n_p + k with their chord lengths, from the same candidate bins as
 * oracle_count.  Returns the entry count; writes at most cap entries. */
int64_t oracle_pixel_row(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c, const double *cs,
                         const double *sn, int64_t j, int32_t *col, double *val, int64_t cap, int32_t model) {
  int32_t ix = (int32_t)(j % nx), iy = (int32_t)(j / nx);
  int64_t n = 0;
  for (int32_t m = 0; m < nt; ++m) {
    int64_t k0;
    candidate_bins(c, cs[m], sn[m], nx, ny, ix, iy, &k0);
    for (int64_t k = k0; k < k0 + 5; ++k) {
      double L;
      if (k < 0 || k >= np_) continue;
      if (oracle_weight(nx, ny, c, cs[m], sn[m], (int32_t)k, ix, iy, &L, model)) {
        if (n < cap) {
          col[n] = (int32_t)((int64_t)m * np_ + k);
          val[n] = L;
        }
        ++n;
      }
    }
  }
  return n;
}

/* Plain CSR transpose (counting sort by column; rows of the result come out
 * with ascending column indices because source rows are scanned in order). */
void oracle_transpose(int64_t rows, int64_t cols, const int64_t *rp, const int32_t *ci,
                      const double *v, int64_t *trp, int32_t *tci, double *tv) {
  memset(trp, 0, sizeof(int64_t) * (cols + 1));
  int64_t nnz = rp[rows];
  for (int64_t e = 0; e < nnz; ++e) trp[ci[e] + 1]++;
  for (int64_t j = 0; j < cols; ++j) trp[j + 1] += trp[j];
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)cols);
  memcpy(cur, trp, sizeof(int64_t) * cols);
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t d = cur[ci[e]]++;
      tci[d] = (int32_t)i;
      tv[d] = v[e];
    }
  free(cur);
}

/* y_s = M x_s for every slice s; x is (nz, cols), y is (nz, rows), slice-major. */
void oracle_spmv(int64_t rows, int64_t cols, const int64_t *rp, const int32_t *ci,
                 const double *v, int32_t nz, const double *x, double *y) {
  for (int32_t s = 0; s < nz; ++s) {
    const double *xs = x + (int64_t)s * cols;
    double *ys = y + (int64_t)s * rows;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i) {
      double acc = 0.0;
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) acc += v[e] * xs[ci[e]];
      ys[i] = acc;
    }
  }
}

/* Matrix-free y = A x: same weights, generated on the fly (no storage).
 * Each row's terms are summed in increasing pixel order, as in the CSR form. */
void oracle_project_mf(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c,
                       const double *cs, const double *sn, int32_t nz,
                       const double *x, double *y, int32_t model) {
  int64_t cols = (int64_t)nx * ny, rows = (int64_t)nt * np_;
  memset(y, 0, sizeof(double) * rows * nz);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t m = 0; m < nt; ++m)
    for (int32_t iy = 0; iy < ny; ++iy)
      for (int32_t ix = 0; ix < nx; ++ix) {
        int64_t k0;
        candidate_bins(c, cs[m], sn[m], nx, ny, ix, iy, &k0);
        for (int64_t k = k0; k < k0 + 5; ++k) {
          double L;
          if (k < 0 || k >= np_) continue;
          if (oracle_weight(nx, ny, c, cs[m], sn[m], (int32_t)k, ix, iy, &L, model)) {
            int64_t j = (int64_t)iy * nx + ix, i = (int64_t)m * np_ + k;
            for (int32_t s = 0; s < nz; ++s) y[s * rows + i] += L * x[s * cols + j];
          }
        }
      }
}

/* Matrix-free x' = A^T y; each pixel sums its terms in increasing row order. */
void oracle_backproject_mf(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c,
                           const double *cs, const double *sn, int32_t nz,
                           const double *y, double *x, int32_t model) {
  int64_t cols = (int64_t)nx * ny, rows = (int64_t)nt * np_;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < cols; ++j) {
    int32_t ix = (int32_t)(j % nx), iy = (int32_t)(j / nx);
    for (int32_t s = 0; s < nz; ++s) x[s * cols + j] = 0.0;
    for (int32_t m = 0; m < nt; ++m) {
      int64_t k0;
      candidate_bins(c, cs[m], sn[m], nx, ny, ix, iy, &k0);
      for (int64_t k = k0; k < k0 + 5; ++k) {
        double L;
        if (k < 0 || k >= np_) continue;
        if (oracle_weight(nx, ny, c, cs[m], sn[m], (int32_t)k, ix, iy, &L, model)) {
          int64_t i = (int64_t)m * np_ + k;
          for (int32_t s = 0; s < nz; ++s) x[s * cols + j] += L * y[s * rows + i];
        }
      }
    }
  }
}

/* Reciprocal sums used by SIRT: out[i] = 1 / sum_e v[e] over row i (0 if the
 * sum is 0).  Applied to A gives R (rows), applied to A^T gives C (columns). */
void oracle_inv_row_sums(int64_t rows, const int64_t *rp, const double *v, double *out) {
  for (int64_t i = 0; i < rows; ++i) {
    double s = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e];
    out[i] = s != 0.0 ? 1.0 / s : 0.0;
  }
}

/* SIRT (Sec. 2.1): x <- x + lambda * C o A^T (R o (b - A x)), per slice, from
 * the given x (in: start, out: result).  Pinned: fixed point equals the
 * R-weighted least-squares solution; exact recovery on consistent data. */
void oracle_sirt(int64_t rows, int64_t cols,
                 const int64_t *arp, const int32_t *aci, const double *av,
                 const int64_t *trp, const int32_t *tci, const double *tv,
                 int32_t nz, const double *b, double *x, int32_t iters, double lambda) {
  double *R = (double *)malloc(sizeof(double) * rows);
  double *C = (double *)malloc(sizeof(double) * cols);
  double *r = (double *)malloc(sizeof(double) * rows * nz);
  double *g = (double *)malloc(sizeof(double) * cols * nz);
  oracle_inv_row_sums(rows, arp, av, R);
  oracle_inv_row_sums(cols, trp, tv, C);
  for (int32_t it = 0; it < iters; ++it) {
    oracle_spmv(rows, cols, arp, aci, av, nz, x, r);
    for (int32_t s = 0; s < nz; ++s)
      for (int64_t i = 0; i < rows; ++i) r[s * rows + i] = R[i] * (b[s * rows + i] - r[s * rows + i]);
    oracle_spmv(cols, rows, trp, tci, tv, nz, r, g);
    for (int32_t s = 0; s < nz; ++s)
      for (int64_t j = 0; j < cols; ++j) x[s * cols + j] += lambda * C[j] * g[s * cols + j];
  }
  free(R);
  free(C);
  free(r);
  free(g);
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* The two products CGLS takes, q = A p and s = A^T r, for one slice: from the
 * stored CSR pair, or generated on the fly (matrix-free, for geometries whose
 * matrix does not fit in host memory).  Both forms sum every row's terms in
 * the same order, so they give the same bits. */
typedef struct {
  const int64_t *arp, *trp;
  const int32_t *aci, *tci;
  const double *av, *tv;
  int32_t mf, nx, ny, np_, nt, model;
  double c;
  const double *cs, *sn;
} cgls_ops;

static void cgls_A(const cgls_ops *o, int64_t rows, int64_t cols, const double *p, double *q) {
  if (o->mf)
    oracle_project_mf(o->nx, o->ny, o->np_, o->nt, o->c, o->cs, o->sn, 1, p, q, o->model);
  else
    oracle_spmv(rows, cols, o->arp, o->aci, o->av, 1, p, q);
}

static void cgls_AT(const cgls_ops *o, int64_t rows, int64_t cols, const double *r, double *s) {
  if (o->mf)
    oracle_backproject_mf(o->nx, o->ny, o->np_, o->nt, o->c, o->cs, o->sn, 1, r, s, o->model);
  else
    oracle_spmv(cols, rows, o->trp, o->tci, o->tv, 1, r, s);
}

/* CGLS (Sec. 2.1; Hestenes-Stiefel form for min ||A x - b||), independently per
 * slice.  One iteration from the state (x, r = b - A x, p, gamma = ||A^T r||^2):
 *   q = A p, alpha = gamma/||q||^2, x += alpha p, r -= alpha q,
 *   s = A^T r, gamma' = ||s||^2, beta = gamma'/gamma, p = s + beta p.
 * A slice whose gamma or ||q||^2 is 0 is converged and stops changing (frozen).
 * hist (nullable, iters x nz) receives ||r|| after each iteration.
 * Pinned: iterate k equals the minimiser of ||A x - b|| over the Krylov space
 * K_k(A^T A, A^T b); after rank-many steps it equals the lstsq solution. */
static void cgls_iterate(const cgls_ops *o, int64_t rows, int64_t cols, double *xz, double *r,
                         double *p, double *gamma, int32_t *frozen, int32_t iters, double *hist, int32_t nz,
                         int32_t z, double *q, double *s) {
  for (int32_t it = 0; it < iters; ++it) {
    if (!*frozen) {
      cgls_A(o, rows, cols, p, q);
      double qq = dot(rows, q, q);
      if (*gamma == 0.0 || qq == 0.0) {
        *frozen = 1;
      } else {
        double alpha = *gamma / qq;
        for (int64_t j = 0; j < cols; ++j) xz[j] += alpha * p[j];
        for (int64_t i = 0; i < rows; ++i) r[i] -= alpha * q[i];
        cgls_AT(o, rows, cols, r, s);
        double gnew = dot(cols, s, s);
        double beta = gnew / *gamma;
        for (int64_t j = 0; j < cols; ++j) p[j] = s[j] + beta * p[j];
        *gamma = gnew;
      }
    }
    if (hist) hist[(int64_t)it * nz + z] = sqrt(dot(rows, r, r));
  }
}

/* CGLS from x0 = 0 for every slice: r = b, s = A^T r, p = s, gamma = ||s||^2,
 * then `iters` iterations (see cgls_iterate). */
static void cgls_run(const cgls_ops *o, int64_t rows, int64_t cols, int32_t nz, const double *b, double *x,
                     int32_t iters, double *hist) {
  double *r = (double *)malloc(sizeof(double) * rows);
  double *q = (double *)malloc(sizeof(double) * rows);
  double *s = (double *)malloc(sizeof(double) * cols);
  double *p = (double *)malloc(sizeof(double) * cols);
  for (int32_t z = 0; z < nz; ++z) {
    double *xz = x + (int64_t)z * cols;
    memset(xz, 0, sizeof(double) * cols);
    memcpy(r, b + (int64_t)z * rows, sizeof(double) * rows);
    cgls_AT(o, rows, cols, r, s);
    memcpy(p, s, sizeof(double) * cols);
    double gamma = dot(cols, s, s);
    int32_t frozen = 0;
    cgls_iterate(o, rows, cols, xz, r, p, &gamma, &frozen, iters, hist, nz, z, q, s);
  }
  free(r);
  free(q);
  free(s);
  free(p);
}

/* CGLS continued from a given state: x (nz, cols), r (nz, rows), p (nz, cols),
 * gamma (nz), frozen (nz), all updated in place by `iters` iterations. */
static void cgls_resume_run(const cgls_ops *o, int64_t rows, int64_t cols, int32_t nz, double *x, double *r,
                            double *p, double *gamma, int32_t *frozen, int32_t iters, double *hist) {
  double *q = (double *)malloc(sizeof(double) * rows);
  double *s = (double *)malloc(sizeof(double) * cols);
  for (int32_t z = 0; z < nz; ++z)
    cgls_iterate(o, rows, cols, x + (int64_t)z * cols, r + (int64_t)z * rows, p + (int64_t)z * cols, gamma + z,
                 frozen + z, iters, hist, nz, z, q, s);
  free(q);
  free(s);
}

static cgls_ops stored_ops(const int64_t *arp, const int32_t *aci, const double *av, const int64_t *trp,
                           const int32_t *tci, const double *tv) {
  cgls_ops o;
  memset(&o, 0, sizeof(o));
  o.arp = arp; o.aci = aci; o.av = av;
  o.trp = trp; o.tci = tci; o.tv = tv;
  return o;
}

static cgls_ops mf_ops(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c, const double *cs,
                       const double *sn, int32_t model) {
  cgls_ops o;
  memset(&o, 0, sizeof(o));
  o.mf = 1;
  o.nx = nx; o.ny = ny; o.np_ = np_; o.nt = nt; o.c = c; o.cs = cs; o.sn = sn; o.model = model;
  return o;
}

void oracle_cgls(int64_t rows, int64_t cols,
                 const int64_t *arp, const int32_t *aci, const double *av,
                 const int64_t *trp, const int32_t *tci, const double *tv,
                 int32_t nz, const double *b, double *x, int32_t iters, double *hist) {
  cgls_ops o = stored_ops(arp, aci, av, trp, tci, tv);
  cgls_run(&o, rows, cols, nz, b, x, iters, hist);
}

void oracle_cgls_resume(int64_t rows, int64_t cols,
                        const int64_t *arp, const int32_t *aci, const double *av,
                        const int64_t *trp, const int32_t *tci, const double *tv,
                        int32_t nz, double *x, double *r, double *p, double *gamma, int32_t *frozen,
                        int32_t iters, double *hist) {
  cgls_ops o = stored_ops(arp, aci, av, trp, tci, tv);
  cgls_resume_run(&o, rows, cols, nz, x, r, p, gamma, frozen, iters, hist);
}

/* The same two CGLS calls with the matrix-free projector pair: the iterates
 * equal those of the stored form bit for bit. */
void oracle_cgls_mf(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c, const double *cs,
                    const double *sn, int32_t model, int32_t nz, const double *b, double *x, int32_t iters,
                    double *hist) {
  cgls_ops o = mf_ops(nx, ny, np_, nt, c, cs, sn, model);
  cgls_run(&o, (int64_t)nt * np_, (int64_t)nx * ny, nz, b, x, iters, hist);
}

void oracle_cgls_resume_mf(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c, const double *cs,
                           const double *sn, int32_t model, int32_t nz, double *x, double *r, double *p,
                           double *gamma, int32_t *frozen, int32_t iters, double *hist) {
  cgls_ops o = mf_ops(nx, ny, np_, nt, c, cs, sn, model);
  cgls_resume_run(&o, (int64_t)nt * np_, (int64_t)nx * ny, nz, x, r, p, gamma, frozen, iters, hist);
}

/* TV term of the model-based objective: adds mu * sum sqrt(Dx^2 + Dy^2 + eps^2)
 * over every slice to the returned value and its gradient to grad. */
static double tv_add(int32_t nx, int32_t ny, int32_t nz, const double *x, double mu, double eps, double *grad) {
  int64_t cols = (int64_t)nx * ny;
  double f = 0.0;
  for (int32_t s = 0; s < nz; ++s) {
    const double *u = x + (int64_t)s * cols;
    double *g = grad + (int64_t)s * cols;
    for (int32_t iy = 0; iy < ny; ++iy)
      for (int32_t ix = 0; ix < nx; ++ix) {
        int64_t j = (int64_t)iy * nx + ix;
        double dx = ix + 1 < nx ? u[j + 1] - u[j] : 0.0;
        double dy = iy + 1 < ny ? u[j + nx] - u[j] : 0.0;
        double t = sqrt(dx * dx + dy * dy + eps * eps);
        f += mu * t;
        /* d t / d u[j] = -(dx + dy)/t (only the differences that exist) */
        if (ix + 1 < nx) {
          g[j] -= mu * dx / t;
          g[j + 1] += mu * dx / t;
        }
        if (iy + 1 < ny) {
          g[j] -= mu * dy / t;
          g[j + nx] += mu * dy / t;
        }
      }
  }
  return f;
}

/* Model-based objective of Sec. 2.1 with an unweighted norm and TV prior:
 *   f(x) = sum_s ||A x_s - b_s||^2 + mu * sum_s sum_pixels sqrt(Dx^2 + Dy^2 + eps^2),
 * Dx, Dy forward differences within the slice, 0 on the last column / row.
 * Returns f; grad (nz, cols) receives 2 A^T (A x - b) + mu * dTV/dx.
 * Pinned: central finite differences; TV value of hand-computed images. */
double oracle_loss_grad(int64_t rows, int64_t cols,
                        const int64_t *arp, const int32_t *aci, const double *av,
                        const int64_t *trp, const int32_t *tci, const double *tv,
                        int32_t nx, int32_t ny, int32_t nz, const double *x, const double *b,
                        double mu, double eps, double *grad) {
  double *r = (double *)malloc(sizeof(double) * rows * nz);
  oracle_spmv(rows, cols, arp, aci, av, nz, x, r);
  double f = 0.0;
  for (int64_t i = 0; i < rows * nz; ++i) {
    r[i] -= b[i];
    f += r[i] * r[i];
  }
  oracle_spmv(cols, rows, trp, tci, tv, nz, r, grad);
  for (int64_t j = 0; j < cols * nz; ++j) grad[j] *= 2.0;
  f += tv_add(nx, ny, nz, x, mu, eps, grad);
  free(r);
  return f;
}

/* The same objective and gradient with the matrix-free projector pair. */
double oracle_loss_grad_mf(int32_t nx, int32_t ny, int32_t np_, int32_t nt, double c, const double *cs,
                           const double *sn, int32_t nz, const double *x, const double *b, double mu, double eps,
                           double *grad, int32_t model) {
  int64_t rows = (int64_t)nt * np_, cols = (int64_t)nx * ny;
  double *r = (double *)malloc(sizeof(double) * rows * nz);
  oracle_project_mf(nx, ny, np_, nt, c, cs, sn, nz, x, r, model);
  double f = 0.0;
  for (int64_t i = 0; i < rows * nz; ++i) {
    r[i] -= b[i];
    f += r[i] * r[i];
  }
  oracle_backproject_mf(nx, ny, np_, nt, c, cs, sn, nz, r, grad, model);
  for (int64_t j = 0; j < cols * nz; ++j) grad[j] *= 2.0;
  f += tv_add(nx, ny, nz, x, mu, eps, grad);
  free(r);
  return f;
}
