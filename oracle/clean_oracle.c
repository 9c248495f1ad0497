/*
 * CPU oracle for tiled Hogbom CLEAN with feedback (arXiv 2501.01461).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, by the package's smoke check
 * and by the benchmark's CPU-baseline leg.  The CUDA library never links,
 * loads or calls it, and the two share no code.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 *
 * oracle_clean_f32 computes in float with every multiply and subtract
 * rounded separately; oracle_clean_f64 is the same algorithm in double.
 *
 * Arguments (both variants):
 *   dirty[ny*nx], psf[pny*pnx]   row-major float32 inputs (read only)
 *   gain, niter, threshold        loop gain, total iteration budget over all
 *                                 tiles, stop a tile while |peak| <= threshold
 *   ty, tx                        tile grid (1 x 1 = untiled)
 *   K                             feedback interval in minor iterations per
 *                                 tile; 0 = no interval
 *   trigger                       0, or in (0, 1): a tile's round also ends
 *                                 once its |peak| <= trigger x the largest
 *                                 |peak| among the round's active tiles at
 *                                 the round's start;
 *                                 feedback follows every round when K > 0 or
 *                                 trigger > 0 (else independent tiles)
 *   max_rounds                    stop after this many rounds (-1 = run to
 *                                 completion); every round ends with feedback
 *   replay_*                      FP64 replay list (replay_n < 0: off)
 *   residual[ny*nx], model[ny*nx] outputs
 *   out_y/x/f/tile/round[cap]     component list in list order
 *   rounds_out                    rounds executed
 * Returns the number of components, -1 bad arguments, -2 out of memory,
 * -3 component list capacity exceeded.
 */
#include <stdint.h>
#include <stdlib.h>

#define REAL float
#define SFX _f32
#include "clean_oracle_body.h"
#undef REAL
#undef SFX

#define REAL double
#define SFX _f64
#include "clean_oracle_body.h"
#undef REAL
#undef SFX

static int bad_args(int32_t ny, int32_t nx, int32_t pny, int32_t pnx,
                    double gain, int64_t niter, double threshold, int32_t ty,
                    int32_t tx, int32_t K, double trigger) {
  return ny < 1 || nx < 1 || pny < 1 || pnx < 1 || !(gain > 0.0) ||
         !(gain <= 1.0) || niter < 0 || !(threshold >= 0.0) || ty < 1 ||
         tx < 1 || ty > ny || tx > nx || K < 0 || !(trigger >= 0.0) ||
         !(trigger < 1.0);
}

int64_t oracle_clean_f32(const float* dirty, int32_t ny, int32_t nx,
                         const float* psf, int32_t pny, int32_t pnx,
                         double gain, int64_t niter, double threshold,
                         int32_t ty, int32_t tx, int32_t K, double trigger,
                         int32_t max_rounds, float* residual, float* model,
                         int32_t* out_y,
                         int32_t* out_x, float* out_f, int32_t* out_tile,
                         int32_t* out_round, int64_t cap, int32_t* rounds_out) {
  if (bad_args(ny, nx, pny, pnx, gain, niter, threshold, ty, tx, K, trigger))
    return -1;
  return clean_run_f32(dirty, ny, nx, psf, pny, pnx, gain, niter, threshold,
                       ty, tx, K, trigger, max_rounds, 0, 0, 0, 0, -1, residual, model,
                       out_y, out_x, out_f, out_tile, out_round, cap,
                       rounds_out);
}

int64_t oracle_clean_f64(const float* dirty, int32_t ny, int32_t nx,
                         const float* psf, int32_t pny, int32_t pnx,
                         double gain, int64_t niter, double threshold,
                         int32_t ty, int32_t tx, int32_t K, double trigger,
                         int32_t max_rounds, const int32_t* replay_y,
                         const int32_t* replay_x,
                         const int32_t* replay_tile,
                         const int32_t* replay_round, int64_t replay_n,
                         double* residual, double* model, int32_t* out_y,
                         int32_t* out_x, double* out_f, int32_t* out_tile,
                         int32_t* out_round, int64_t cap,
                         int32_t* rounds_out) {
  if (bad_args(ny, nx, pny, pnx, gain, niter, threshold, ty, tx, K, trigger))
    return -1;
  return clean_run_f64(dirty, ny, nx, psf, pny, pnx, gain, niter, threshold,
                       ty, tx, K, trigger, max_rounds, replay_y, replay_x, replay_tile,
                       replay_round, replay_n, residual, model, out_y, out_x,
                       out_f, out_tile, out_round, cap, rounds_out);
}
