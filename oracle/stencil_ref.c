/*
 * FP64 reference stencil (test infrastructure only).
 *
 * This file is the oracle: a plain, slow, obviously correct CPU restatement of the
 * iterated constant-coefficient stencil that SparStencil computes (Sec. 2.2, the
 * Box-2D9P pseudo-code fixes the orientation: out[i][j] = sum_ab c_ab * in[i+a][j+b],
 * i.e. a correlation with offset-indexed weights, no flip).  Only tests/, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * Conventions
 *   - grid: ndim in {1,2,3}; dims[0] is the slowest axis, dims[ndim-1] the fastest;
 *     row-major contiguous.
 *   - weights: dense cube of side 2r+1 in the same axis order, entry (o_0,..,o_{d-1})
 *     stored at index sum_i (o_i + r) * (2r+1)^(d-1-i).  Zero entries are not part of
 *     the stencil and are skipped.
 *   - bc = 0: Dirichlet zero (values outside the grid are 0 at every step).
 *     bc = 1: periodic (indices taken modulo the extent).
 *   - one step: u_{s+1}[x] = sum_o w[o] * u_s[x + o], accumulated in FP64 in
 *     lexicographic offset order; T steps, no intermediate rounding.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Largest weight cube (entries): 2D radius up to 31, 3D radius up to 7, 1D radius up to 2047. */
#define ORACLE_MAX_CUBE 4096

typedef struct {
  int npts;
  int off[ORACLE_MAX_CUBE][3]; /* offsets, padded to 3 axes (leading axes 0) */
  double w[ORACLE_MAX_CUBE];
} stencil_pts;

static int build_points(int ndim, int radius, const double* weights, stencil_pts* sp) {
  if (radius > 2047) return -1;
  int side = 2 * radius + 1;
  int64_t total = 1;
  for (int i = 0; i < ndim; i++) total *= side;
  if (total > ORACLE_MAX_CUBE) return -1;
  sp->npts = 0;
  for (int idx = 0; idx < (int)total; idx++) {
    if (weights[idx] == 0.0) continue;
    int rem = idx;
    int o[3] = {0, 0, 0};
    for (int a = ndim - 1; a >= 0; a--) {
      o[3 - ndim + a] = rem % side - radius;
      rem /= side;
    }
    sp->off[sp->npts][0] = o[0];
    sp->off[sp->npts][1] = o[1];
    sp->off[sp->npts][2] = o[2];
    sp->w[sp->npts] = weights[idx];
    sp->npts++;
  }
  return 0;
}

static int64_t wrap(int64_t i, int64_t n) {
  int64_t m = i % n;
  return m < 0 ? m + n : m;
}

/* one step on the whole grid; dims padded to 3 axes */
static void step(const int64_t d[3], const stencil_pts* sp, int bc, const double* in, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < d[0]; z++) {
    for (int64_t y = 0; y < d[1]; y++) {
      for (int64_t x = 0; x < d[2]; x++) {
        double acc = 0.0;
        for (int p = 0; p < sp->npts; p++) {
          int64_t zz = z + sp->off[p][0], yy = y + sp->off[p][1], xx = x + sp->off[p][2];
          double v;
          if (bc == 1) {
            v = in[(wrap(zz, d[0]) * d[1] + wrap(yy, d[1])) * d[2] + wrap(xx, d[2])];
          } else if (zz < 0 || zz >= d[0] || yy < 0 || yy >= d[1] || xx < 0 || xx >= d[2]) {
            v = 0.0;
          } else {
            v = in[(zz * d[1] + yy) * d[2] + xx];
          }
          acc += sp->w[p] * v;
        }
        out[(z * d[1] + y) * d[2] + x] = acc;
      }
    }
  }
}

/* Runs T steps.  in and out hold prod(dims) doubles and may alias; scratch holds
 * prod(dims) doubles.  Returns 0 on success, -1 on bad arguments. */
int oracle_stencil_run(int ndim, const int64_t* dims, int radius, const double* weights, int bc, int64_t T,
                       const double* in, double* out, double* scratch, int nthreads) {
  if (ndim < 1 || ndim > 3 || radius < 0 || T < 0 || (bc != 0 && bc != 1)) return -1;
  int64_t d[3] = {1, 1, 1};
  int64_t n = 1;
  for (int i = 0; i < ndim; i++) {
    if (dims[i] <= 0) return -1;
    d[3 - ndim + i] = dims[i];
    n *= dims[i];
  }
  stencil_pts* sp = (stencil_pts*)malloc(sizeof(stencil_pts));
  if (!sp) return -1;
  if (build_points(ndim, radius, weights, sp) != 0) {
    free(sp);
    return -1;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  if (out != in) memcpy(out, in, (size_t)n * sizeof(double));
  double* a = out;
  double* b = scratch;
  for (int64_t s = 0; s < T; s++) {
    step(d, sp, bc, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != out) memcpy(out, a, (size_t)n * sizeof(double));
  free(sp);
  return 0;
}

/* Value of one grid point after T steps, from the dependence cone only: a window of
 * half-width T*r around the point (periodic: wrapped coordinates; Dirichlet: points
 * outside the grid are held at zero).  Step s (s = 0 .. T-1) updates only the cells within
 * (T-1-s)*r of the point along every axis: those are the cells a later step reads, and each
 * reads neighbours within (T-s)*r, all updated by the step before (or initial values), so
 * every value computed is the full-grid value of that cell.  Returns 0 on success. */
int oracle_stencil_point(int ndim, const int64_t* dims, int radius, const double* weights, int bc, int64_t T,
                         const double* in, const int64_t* point, double* value) {
  if (ndim < 1 || ndim > 3 || radius < 0 || T < 0 || (bc != 0 && bc != 1)) return -1;
  stencil_pts* sp = (stencil_pts*)malloc(sizeof(stencil_pts));
  if (!sp) return -1;
  if (build_points(ndim, radius, weights, sp) != 0) {
    free(sp);
    return -1;
  }
  int64_t d[3] = {1, 1, 1}, p[3] = {0, 0, 0};
  for (int i = 0; i < ndim; i++) {
    d[3 - ndim + i] = dims[i];
    p[3 - ndim + i] = point[i];
  }
  int64_t h = T * radius;
  int64_t wd[3];
  for (int a = 0; a < 3; a++) wd[a] = (a < 3 - ndim) ? 1 : 2 * h + 1;
  int64_t wn = wd[0] * wd[1] * wd[2];
  double* cur = (double*)calloc((size_t)wn, sizeof(double));
  double* nxt = (double*)calloc((size_t)wn, sizeof(double));
  unsigned char* outside = (unsigned char*)calloc((size_t)wn, 1);
  if (!cur || !nxt || !outside) {
    free(cur);
    free(nxt);
    free(outside);
    free(sp);
    return -1;
  }
  int64_t hz = (3 - ndim > 0) ? 0 : h;
  int64_t hy = (3 - ndim > 1) ? 0 : h;
  for (int64_t z = 0; z < wd[0]; z++)
    for (int64_t y = 0; y < wd[1]; y++)
      for (int64_t x = 0; x < wd[2]; x++) {
        int64_t gz = p[0] + z - hz, gy = p[1] + y - hy, gx = p[2] + x - h;
        int64_t wi = (z * wd[1] + y) * wd[2] + x;
        if (bc == 1) {
          cur[wi] = in[(wrap(gz, d[0]) * d[1] + wrap(gy, d[1])) * d[2] + wrap(gx, d[2])];
        } else if (gz < 0 || gz >= d[0] || gy < 0 || gy >= d[1] || gx < 0 || gx >= d[2]) {
          outside[wi] = 1;
          cur[wi] = 0.0;
        } else {
          cur[wi] = in[(gz * d[1] + gy) * d[2] + gx];
        }
      }
  for (int64_t s = 0; s < T; s++) {
    const int64_t keep = (T - 1 - s) * radius; /* half-width of the cells still needed */
    const int64_t z0 = hz - (hz ? keep : 0), z1 = hz + (hz ? keep : 0);
    const int64_t y0 = hy - (hy ? keep : 0), y1 = hy + (hy ? keep : 0);
    for (int64_t z = z0; z <= z1; z++)
      for (int64_t y = y0; y <= y1; y++)
        for (int64_t x = h - keep; x <= h + keep; x++) {
          int64_t wi = (z * wd[1] + y) * wd[2] + x;
          if (outside[wi]) {
            nxt[wi] = 0.0;
            continue;
          }
          double acc = 0.0;
          for (int q = 0; q < sp->npts; q++) {
            int64_t zz = z + sp->off[q][0], yy = y + sp->off[q][1], xx = x + sp->off[q][2];
            if (zz < 0 || zz >= wd[0] || yy < 0 || yy >= wd[1] || xx < 0 || xx >= wd[2]) continue;
            acc += sp->w[q] * cur[(zz * wd[1] + yy) * wd[2] + xx];
          }
          nxt[wi] = acc;
        }
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  *value = cur[(hz * wd[1] + hy) * wd[2] + h];
  free(cur);
  free(nxt);
  free(outside);
  free(sp);
  return 0;
}
