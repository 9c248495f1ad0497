/*
 * Multi-core CPU baseline for tiled Hogbom CLEAN with feedback (arXiv
 * 2501.01461): the oracle's float32 algorithm with the tiles of a round run
 * by OpenMP threads, the CPU analogue of the paper's distribution of tiles
 * over workers (Section 4).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle beside it: the
 * CUDA library never links, loads or calls it.
 *
 * Arithmetic is the oracle's, operation for operation, so the outputs equal
 * oracle_clean_f32's bit for bit (tests check this): within a round every
 * tile changes only its own pixels, so tiles can run at once; each tile
 * writes its components to its own buffer and the round's list is then
 * concatenated in tile order; the feedback updates each tile's pixels with
 * the round's other-tile components in list order, one thread per tile.
 * Flux triggers and replay are not offered (the timed workload uses
 * neither).
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static float absf(float v) { return v < 0 ? -v : v; }

static void bounds(int32_t t, int32_t ny, int32_t nx, int32_t ty, int32_t tx, int32_t* y0,
                   int32_t* y1, int32_t* x0, int32_t* x1) {
  int32_t i = t / tx, j = t % tx;
  *y0 = (int32_t)(((int64_t)i * ny) / ty);
  *y1 = (int32_t)(((int64_t)(i + 1) * ny) / ty);
  *x0 = (int32_t)(((int64_t)j * nx) / tx);
  *x1 = (int32_t)(((int64_t)(j + 1) * nx) / tx);
}

/* largest |R| in the rectangle, lowest row-major index on ties */
static int64_t peak(const float* R, int32_t nx, int32_t y0, int32_t y1, int32_t x0, int32_t x1) {
  int64_t best = -1;
  float bv = 0;
  for (int32_t y = y0; y < y1; ++y)
    for (int32_t x = x0; x < x1; ++x) {
      float a = absf(R[(int64_t)y * nx + x]);
      if (best < 0 || a > bv) {
        bv = a;
        best = (int64_t)y * nx + x;
      }
    }
  return best;
}

/* R <- R - f * P shifted to (py, px), over the rectangle, PSF range only */
static void sub_psf(float* R, int32_t nx, const float* P, int32_t pny, int32_t pnx, int32_t py,
                    int32_t px, float f, int32_t y0, int32_t y1, int32_t x0, int32_t x1) {
  const int32_t cy = pny / 2, cx = pnx / 2;
  for (int32_t y = y0; y < y1; ++y) {
    const int32_t sy = y - py + cy;
    if (sy < 0 || sy >= pny) continue;
    for (int32_t x = x0; x < x1; ++x) {
      const int32_t sx = x - px + cx;
      if (sx < 0 || sx >= pnx) continue;
      const float t = f * P[(int64_t)sy * pnx + sx];
      float* r = &R[(int64_t)y * nx + x];
      *r = *r - t;
    }
  }
}

/*
 * Same arguments and results as oracle_clean_f32 without the trigger
 * (which must be 0); max_rounds limits the rounds (-1: to completion).
 * Returns the number of components, -1 bad arguments, -2 out of memory,
 * -3 component list capacity exceeded.
 */
int64_t parallel_clean_f32(const float* dirty, int32_t ny, int32_t nx, const float* psf,
                           int32_t pny, int32_t pnx, double gain, int64_t niter,
                           double threshold, int32_t ty, int32_t tx, int32_t K,
                           int32_t max_rounds, float* residual, float* model, int32_t* out_y,
                           int32_t* out_x, float* out_f, int32_t* out_tile, int32_t* out_round,
                           int64_t cap, int32_t* rounds_out) {
  if (ny < 1 || nx < 1 || pny < 1 || pnx < 1 || !(gain > 0.0) || !(gain <= 1.0) || niter < 0 ||
      !(threshold >= 0.0) || ty < 1 || tx < 1 || ty > ny || tx > nx || K < 0)
    return -1;
  const float g = (float)gain, thr = (float)threshold;
  const int32_t T = ty * tx;
  const int feedback = K > 0 && T > 1;
  const int64_t npix = (int64_t)ny * nx;
  int64_t* budget = malloc(sizeof(int64_t) * (size_t)T);
  int32_t* active = malloc(sizeof(int32_t) * (size_t)T);
  int64_t* count = malloc(sizeof(int64_t) * (size_t)T);
  int64_t per = niter / T + 1;
  if (K > 0 && K < per) per = K;
  int32_t* ty_ = malloc(sizeof(int32_t) * (size_t)T * (size_t)per);
  int32_t* tx_ = malloc(sizeof(int32_t) * (size_t)T * (size_t)per);
  float* tf = malloc(sizeof(float) * (size_t)T * (size_t)per);
  if (!budget || !active || !count || !ty_ || !tx_ || !tf) {
    free(budget); free(active); free(count); free(ty_); free(tx_); free(tf);
    return -2;
  }
  for (int64_t i = 0; i < npix; ++i) residual[i] = dirty[i];
  for (int32_t t = 0; t < T; ++t) budget[t] = niter / T + (t < niter % T ? 1 : 0);

  int64_t ncomp = 0;
  int32_t round = 0;
  int rc = 0;
  for (;;) {
    if (max_rounds >= 0 && round >= max_rounds) break;
    int any = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : any)
    for (int32_t t = 0; t < T; ++t) {
      int32_t y0, y1, x0, x1;
      bounds(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
      const int64_t p = peak(residual, nx, y0, y1, x0, x1);
      active[t] = budget[t] > 0 && absf(residual[p]) > thr;
      any |= active[t];
    }
    if (!any) break;
    const int64_t round_start = ncomp;
    /* minor loops: every tile on its own pixels, at once */
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t t = 0; t < T; ++t) {
      count[t] = 0;
      if (!active[t]) continue;
      int32_t y0, y1, x0, x1;
      bounds(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
      const int64_t kmax = (K > 0 && K < budget[t]) ? K : budget[t];
      for (int64_t k = 0; k < kmax; ++k) {
        const int64_t p = peak(residual, nx, y0, y1, x0, x1);
        const float v = residual[p];
        if (absf(v) <= thr) break;
        const float f = g * v;
        const int32_t py = (int32_t)(p / nx), px = (int32_t)(p % nx);
        const int64_t slot = (int64_t)t * per + count[t];
        ty_[slot] = py;
        tx_[slot] = px;
        tf[slot] = f;
        count[t] += 1;
        sub_psf(residual, nx, psf, pny, pnx, py, px, f, y0, y1, x0, x1);
      }
    }
    /* the round's list, in tile order */
    for (int32_t t = 0; t < T; ++t) {
      if (ncomp + count[t] > cap) {
        rc = -3;
        break;
      }
      for (int64_t k = 0; k < count[t]; ++k) {
        const int64_t slot = (int64_t)t * per + k;
        out_y[ncomp] = ty_[slot];
        out_x[ncomp] = tx_[slot];
        out_f[ncomp] = tf[slot];
        out_tile[ncomp] = t;
        out_round[ncomp] = round;
        ++ncomp;
      }
      budget[t] -= count[t];
    }
    if (rc) break;
    /* feedback: each tile takes the other tiles' new components in list order */
    if (feedback) {
#pragma omp parallel for schedule(dynamic, 1)
      for (int32_t t = 0; t < T; ++t) {
        int32_t y0, y1, x0, x1;
        bounds(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
        for (int64_t c = round_start; c < ncomp; ++c) {
          if (out_tile[c] == t) continue;
          sub_psf(residual, nx, psf, pny, pnx, out_y[c], out_x[c], out_f[c], y0, y1, x0, x1);
        }
      }
    }
    ++round;
  }
  if (!rc) {
    memset(model, 0, sizeof(float) * (size_t)npix);
    for (int64_t c = 0; c < ncomp; ++c) {
      float* m = &model[(int64_t)out_y[c] * nx + out_x[c]];
      *m = *m + out_f[c];
    }
    if (rounds_out) *rounds_out = round;
  }
  free(budget); free(active); free(count); free(ty_); free(tx_); free(tf);
  return rc ? rc : ncomp;
}

/* OpenMP threads for the calls that follow (n <= 0: leave as is); returns
 * the number the next parallel region will use. */
int parallel_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}
