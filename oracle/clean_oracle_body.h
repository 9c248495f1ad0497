/*
 * Body of the CPU oracle for tiled Hogbom CLEAN with feedback.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is included twice by
 * clean_oracle.c, once with REAL = float and once with REAL = double.  It is
 * plain single-threaded C, written step by step from the paper; it shares no
 * code with the CUDA library and must never be linked into it.
 *
 * Notation (paper, Section 3):
 *   R        residual image, starts as the dirty image
 *   P        point spread function, centre c = (pny / 2, pnx / 2)
 *   g        loop gain
 *   component (position p, flux f = g * R[p])            -- first equation
 *   R[q] <- R[q] - f * P[q - p + c]  for every q          -- second equation
 * A tile (Section 2, Fig. 1) is a rectangle of the image; tile (i, j) of a
 * Ty x Tx grid covers rows [floor(i ny / Ty), floor((i+1) ny / Ty)) and the
 * columns likewise.  Feedback (Section 3, Figs. 2-3): the components a tile
 * found since the last feedback, convolved with the full PSF, are subtracted
 * from every other tile.
 *
 * Every multiply and every subtract is rounded separately to REAL (the
 * library is built with -ffp-contract=off, so no fused multiply-add).
 */

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SFX)

static REAL FN(absr)(REAL v) { return v < 0 ? -v : v; }

/* Bounds of tile t (row-major tile index). */
static void FN(tile_bounds)(int32_t t, int32_t ny, int32_t nx, int32_t ty,
                            int32_t tx, int32_t* y0, int32_t* y1, int32_t* x0,
                            int32_t* x1) {
  int32_t i = t / tx, j = t % tx;
  *y0 = (int32_t)(((int64_t)i * ny) / ty);
  *y1 = (int32_t)(((int64_t)(i + 1) * ny) / ty);
  *x0 = (int32_t)(((int64_t)j * nx) / tx);
  *x1 = (int32_t)(((int64_t)(j + 1) * nx) / tx);
}

/* Peak search of the first equation over rows [y0,y1) x cols [x0,x1):
 * the pixel with the largest |R|; among equal |R| the lowest row-major
 * index wins (the scan is row-major and only a strictly larger value
 * replaces the current best). */
static int64_t FN(argmax_abs)(const REAL* R, int32_t nx, int32_t y0,
                              int32_t y1, int32_t x0, int32_t x1) {
  int64_t best = -1;
  REAL bv = 0;
  for (int32_t y = y0; y < y1; ++y)
    for (int32_t x = x0; x < x1; ++x) {
      REAL a = FN(absr)(R[(int64_t)y * nx + x]);
      if (best < 0 || a > bv) {
        bv = a;
        best = (int64_t)y * nx + x;
      }
    }
  return best;
}

/* Second equation restricted to the rectangle [y0,y1) x [x0,x1): subtract
 * f * P shifted so that its centre sits on (py, px).  Pixels whose PSF index
 * falls outside the PSF array are left unchanged. */
static void FN(subtract_psf)(REAL* R, int32_t nx, const REAL* P, int32_t pny,
                             int32_t pnx, int32_t py, int32_t px, REAL f,
                             int32_t y0, int32_t y1, int32_t x0, int32_t x1) {
  int32_t cy = pny / 2, cx = pnx / 2;
  for (int32_t y = y0; y < y1; ++y) {
    int32_t sy = y - py + cy;
    if (sy < 0 || sy >= pny) continue;
    for (int32_t x = x0; x < x1; ++x) {
      int32_t sx = x - px + cx;
      if (sx < 0 || sx >= pnx) continue;
      REAL t = f * P[(int64_t)sy * pnx + sx];
      REAL* r = &R[(int64_t)y * nx + x];
      *r = *r - t;
    }
  }
}

/*
 * Run CLEAN.  Returns the number of components written, or a negative
 * error code.  Arguments are described in clean_oracle.c.
 *
 * replay_n >= 0 selects replay mode: positions, tiles and rounds are taken
 * from (replay_y, replay_x, replay_tile, replay_round) in list order, and only
 * the fluxes and residuals are computed (in REAL).
 */
static int64_t FN(clean_run)(
    const float* dirty, int32_t ny, int32_t nx, const float* psf, int32_t pny,
    int32_t pnx, double gain_in, int64_t niter, double threshold_in,
    int32_t ty, int32_t tx, int32_t K, double trigger_in, int32_t max_rounds,
    const int32_t* replay_y, const int32_t* replay_x,
    const int32_t* replay_tile, const int32_t* replay_round, int64_t replay_n,
    REAL* residual, REAL* model, int32_t* out_y, int32_t* out_x, REAL* out_f,
    int32_t* out_tile, int32_t* out_round, int64_t cap, int32_t* rounds_out) {
  const REAL g = (REAL)gain_in;
  const REAL thr = (REAL)threshold_in;
  const REAL trig = (REAL)trigger_in;
  /* feedback happens after every round when an interval or a trigger is set */
  const int feedback = (K > 0 || trigger_in > 0) && ty * tx > 1;
  const int32_t T = ty * tx;
  const int64_t npix = (int64_t)ny * nx;
  const int replay = replay_n >= 0;
  int64_t ncomp = 0, rp = 0;
  int32_t round = 0;

  REAL* P = (REAL*)malloc(sizeof(REAL) * (size_t)pny * (size_t)pnx);
  int64_t* budget = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
  int32_t* active = (int32_t*)malloc(sizeof(int32_t) * (size_t)T);
  if (!P || !budget || !active) {
    free(P); free(budget); free(active);
    return -2;
  }
  for (int64_t i = 0; i < (int64_t)pny * pnx; ++i) P[i] = (REAL)psf[i];
  for (int64_t i = 0; i < npix; ++i) residual[i] = (REAL)dirty[i];

  /* Iteration budget: niter split over the tiles, the remainder going to
   * the lowest tile indices. */
  for (int32_t t = 0; t < T; ++t)
    budget[t] = niter / T + (t < niter % T ? 1 : 0);

  for (;;) {
    if (max_rounds >= 0 && round >= max_rounds) break;
    int64_t round_start = ncomp;

    if (replay) {
      if (rp >= replay_n) break;
      int32_t r = replay_round[rp];
      /* the components of round r, tile by tile in list order */
      for (int32_t t = 0; t < T; ++t) {
        int32_t y0, y1, x0, x1;
        FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
        for (int64_t k = rp; k < replay_n && replay_round[k] == r; ++k) {
          if (replay_tile[k] != t) continue;
          if (ncomp >= cap) goto overflow;
          int32_t py = replay_y[k], px = replay_x[k];
          REAL v = residual[(int64_t)py * nx + px];
          REAL f = g * v;
          out_y[ncomp] = py; out_x[ncomp] = px; out_f[ncomp] = f;
          out_tile[ncomp] = t; out_round[ncomp] = round;
          ++ncomp;
          FN(subtract_psf)(residual, nx, P, pny, pnx, py, px, f, y0, y1, x0, x1);
        }
      }
      while (rp < replay_n && replay_round[rp] == r) ++rp;
    } else {
      /* a tile takes part in this round while it has budget left and its
       * peak is above the threshold */
      int any = 0;
      for (int32_t t = 0; t < T; ++t) {
        int32_t y0, y1, x0, x1;
        FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
        int64_t p = FN(argmax_abs)(residual, nx, y0, y1, x0, x1);
        active[t] = budget[t] > 0 && FN(absr)(residual[p]) > thr;
        any |= active[t];
      }
      if (!any) break;

      /* flux trigger (Section 3): this round ends for a tile once its
       * |peak| is at most trigger x the largest |peak| among the tiles taking
       * part in the round (that tile always makes progress) */
      REAL level = 0;
      if (trig > 0) {
        REAL top = 0;
        for (int32_t t = 0; t < T; ++t) {
          if (!active[t]) continue;
          int32_t y0, y1, x0, x1;
          FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
          REAL a = FN(absr)(residual[FN(argmax_abs)(residual, nx, y0, y1, x0, x1)]);
          if (a > top) top = a;
        }
        level = trig * top;
      }
      /* minor loops: every tile on its own pixels, up to K iterations
       * (K = 0: no interval; without a trigger, no feedback and the whole
       * budget in one round) */
      for (int32_t t = 0; t < T; ++t) {
        if (!active[t]) continue;
        int32_t y0, y1, x0, x1;
        FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
        int64_t kmax = (K > 0 && K < budget[t]) ? K : budget[t];
        for (int64_t k = 0; k < kmax; ++k) {
          int64_t p = FN(argmax_abs)(residual, nx, y0, y1, x0, x1);
          REAL v = residual[p];
          if (FN(absr)(v) <= thr || FN(absr)(v) <= level) break;
          if (ncomp >= cap) goto overflow;
          REAL f = g * v;                            /* first equation */
          int32_t py = (int32_t)(p / nx), px = (int32_t)(p % nx);
          out_y[ncomp] = py; out_x[ncomp] = px; out_f[ncomp] = f;
          out_tile[ncomp] = t; out_round[ncomp] = round;
          ++ncomp;
          budget[t] -= 1;
          /* second equation, on this tile's pixels only */
          FN(subtract_psf)(residual, nx, P, pny, pnx, py, px, f, y0, y1, x0, x1);
        }
      }
    }

    /* Feedback: each new component, placed on the full image and convolved
     * with the full PSF, is subtracted from every tile except its own.  Per
     * pixel the components are taken in list order (tile, then iteration),
     * one rounded multiply and one rounded subtract each. */
    if (feedback) {
      for (int64_t c = round_start; c < ncomp; ++c) {
        for (int32_t t = 0; t < T; ++t) {
          if (t == out_tile[c]) continue;
          int32_t y0, y1, x0, x1;
          FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);
          FN(subtract_psf)(residual, nx, P, pny, pnx, out_y[c], out_x[c],
                           out_f[c], y0, y1, x0, x1);
        }
      }
    }
    ++round;
  }

  /* Model image: the component fluxes summed per pixel in list order. */
  for (int64_t i = 0; i < npix; ++i) model[i] = 0;
  for (int64_t c = 0; c < ncomp; ++c) {
    REAL* m = &model[(int64_t)out_y[c] * nx + out_x[c]];
    *m = *m + out_f[c];
  }
  if (rounds_out) *rounds_out = round;
  free(P); free(budget); free(active);
  return ncomp;

overflow:
  free(P); free(budget); free(active);
  return -3;
}

#undef FN
#undef CAT
#undef CAT_
