/*
 * Test driver for the CPU oracle under AddressSanitizer and
 * UndefinedBehaviorSanitizer: runs both precisions on random small images
 * over many tile grids, intervals, thresholds, flux triggers, clipped PSFs,
 * replay and a too-small component list, and checks the return codes.
 * Exit status 0 means every run completed with no sanitizer report.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int64_t oracle_clean_f32(const float*, int32_t, int32_t, const float*, int32_t, int32_t, double,
                         int64_t, double, int32_t, int32_t, int32_t, double, int32_t, float*,
                         float*, int32_t*, int32_t*, float*, int32_t*, int32_t*, int64_t,
                         int32_t*);
int64_t oracle_clean_f64(const float*, int32_t, int32_t, const float*, int32_t, int32_t, double,
                         int64_t, double, int32_t, int32_t, int32_t, double, int32_t,
                         const int32_t*, const int32_t*, const int32_t*, const int32_t*, int64_t,
                         double*, double*, int32_t*, int32_t*, double*, int32_t*, int32_t*,
                         int64_t, int32_t*);

static uint64_t rng = 88172645463325252ull;
static double uni(void) {  /* xorshift64 */
  rng ^= rng << 13;
  rng ^= rng >> 7;
  rng ^= rng << 17;
  return (double)(rng >> 11) / 9007199254740992.0;
}

int main(void) {
  int failures = 0;
  const int sizes[][4] = {{16, 16, 32, 32}, {13, 17, 26, 34}, {20, 9, 12, 7}, {7, 7, 15, 15}};
  const int grids[][2] = {{1, 1}, {2, 2}, {3, 2}, {4, 4}, {1, 3}};
  const int Ks[] = {0, 1, 3, 7};
  const double trig[] = {0.0, 0.5};
  for (int si = 0; si < 4; ++si) {
    const int ny = sizes[si][0], nx = sizes[si][1], pny = sizes[si][2], pnx = sizes[si][3];
    float* dirty = malloc(sizeof(float) * ny * nx);
    float* psf = malloc(sizeof(float) * pny * pnx);
    for (int i = 0; i < ny * nx; ++i) dirty[i] = (float)(2.0 * uni() - 1.0);
    for (int i = 0; i < pny * pnx; ++i) psf[i] = (float)(0.8 * uni() - 0.4);
    psf[(pny / 2) * pnx + pnx / 2] = 1.0f;
    const int64_t niter = 60, cap = 60;
    float *r32 = malloc(sizeof(float) * ny * nx), *m32 = malloc(sizeof(float) * ny * nx);
    double *r64 = malloc(sizeof(double) * ny * nx), *m64 = malloc(sizeof(double) * ny * nx);
    int32_t *y = malloc(4 * cap), *x = malloc(4 * cap), *t = malloc(4 * cap), *rd = malloc(4 * cap);
    float* f32 = malloc(4 * cap);
    double* f64 = malloc(8 * cap);
    for (int gi = 0; gi < 5; ++gi) {
      const int ty = grids[gi][0], tx = grids[gi][1];
      if (ty > ny || tx > nx) continue;
      for (int ki = 0; ki < 4; ++ki)
        for (int tr = 0; tr < 2; ++tr) {
          int32_t rounds = 0;
          const int64_t n = oracle_clean_f32(dirty, ny, nx, psf, pny, pnx, 0.3, niter, 0.05, ty,
                                             tx, Ks[ki], trig[tr], -1, r32, m32, y, x, f32, t,
                                             rd, cap, &rounds);
          if (n < 0 || n > niter) ++failures;
          /* float64 replay of the float32 list, then an independent run */
          const int64_t n2 = oracle_clean_f64(dirty, ny, nx, psf, pny, pnx, 0.3, niter, 0.05, ty,
                                              tx, Ks[ki], trig[tr], -1, y, x, t, rd, n, r64, m64,
                                              y, x, f64, t, rd, cap, &rounds);
          if (n2 != n) ++failures;
          const int64_t n3 = oracle_clean_f64(dirty, ny, nx, psf, pny, pnx, 0.3, niter, 0.05, ty,
                                              tx, Ks[ki], trig[tr], 3, 0, 0, 0, 0, -1, r64, m64,
                                              y, x, f64, t, rd, cap, &rounds);
          if (n3 < 0) ++failures;
        }
    }
    /* too small a component list, and bad arguments */
    int32_t rounds = 0;
    if (oracle_clean_f32(dirty, ny, nx, psf, pny, pnx, 0.3, niter, 0.0, 1, 1, 0, 0.0, -1, r32,
                         m32, y, x, f32, t, rd, 5, &rounds) != -3)
      ++failures;
    if (oracle_clean_f32(dirty, ny, nx, psf, pny, pnx, 1.5, niter, 0.0, 1, 1, 0, 0.0, -1, r32,
                         m32, y, x, f32, t, rd, cap, &rounds) != -1)
      ++failures;
    if (oracle_clean_f32(dirty, ny, nx, psf, pny, pnx, 0.3, niter, 0.0, ny + 1, 1, 0, 0.0, -1,
                         r32, m32, y, x, f32, t, rd, cap, &rounds) != -1)
      ++failures;
    free(dirty); free(psf); free(r32); free(m32); free(r64); free(m64);
    free(y); free(x); free(t); free(rd); free(f32); free(f64);
  }
  if (failures) fprintf(stderr, "%d unexpected return codes\n", failures);
  return failures ? 1 : 0;
}
