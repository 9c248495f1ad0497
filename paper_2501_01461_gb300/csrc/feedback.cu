// Feedback between tiles (Section 3, Figs. 2-3) by gather, and the close of
// a round.
//
// The cross-coupling image of tile s is its components placed on a full-size
// image and convolved with the full PSF; feedback subtracts it from every
// other tile.  Evaluated per pixel q of tile t: for every component
// (p, f) of the round that tile s != t found, in list order (tile index, then
// iteration), R[q] <- R[q] - f * PSF[q - p + c], one rounded multiply and
// one rounded subtract each.  This is the convolution written out term by
// term in a fixed order, so the result is bit-reproducible.
//
// Each CTA owns a kRows x kCols block of one tile; every thread keeps its
// kRowsPerWarp x kColsPerLane pixels in registers for the whole component
// list, so the residual is read and written once per round.  The CTA also
// reduces its pixels' peak key (largest |R|, lowest index) into the tile's
// next-round peak with a 64-bit atomic max.
//
// The last CTA to finish closes the round: it appends the round's
// components to the list (round-major, then tile, then iteration), records
// the round's list offset, and decides whether any tile can still run
// (budget left and |peak| > threshold).
#include <cudaTypedefs.h>

#include <mutex>

#include "cleangb_internal.cuh"
#include "ptx.cuh"
#include "round_close.cuh"

namespace cleangb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRowsPerWarp = 8;
constexpr int kColsPerLane = 2;
constexpr int kRows = kWarps * kRowsPerWarp;  // 64
constexpr int kCols = 32 * kColsPerLane;      // 64
constexpr int kChunk = 512;                   // components staged at once

struct __align__(16) Comp4 {
  int32_t y, x;
  float f;
  int32_t pad;
};

// Sum of the round's component counts over all tiles (0: the round changed
// nothing, so the image's residual and peaks need no new pass).
__device__ __forceinline__ int round_total(const PlanDev& d) {
  int n = 0;
  for (int s = 0; s < d.T; ++s) n += d.rcount[s];
  return n;
}

// Block (bxi, byi) of tile t; blocks_x * blocks_y blocks per tile.
__device__ __forceinline__ void feedback_body(const PlanDev& d, int parity, int apply, int t,
                                              int bxi, int byi, int blocks_x, int blocks_y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Comp4* s_comp = reinterpret_cast<Comp4*>(smem_raw);
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_comp + kChunk);
  int32_t* s_pre = s_cnt + d.T;  // [T + 1]
  __shared__ uint64_t s_warp[kWarps];

  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int by0 = rc.y0 + byi * kRows;
  const int bx0 = rc.x0 + bxi * kCols;
  const bool live = by0 < rc.y1 && bx0 < rc.x1 && *(volatile int32_t*)&d.st->status == 0 &&
                    round_total(d) > 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (live) {
    // the other tiles' components of this round, in list order
    const bool fb = apply && feedback_on(d);  // this image feeds back at all
    for (int s = threadIdx.x; s < d.T; s += kThreads) s_cnt[s] = (s == t || !fb) ? 0 : d.rcount[s];
    block_prefix(s_cnt, s_pre, d.T);
    const int n_other = s_pre[d.T];

    float r[kRowsPerWarp][kColsPerLane];
    bool in[kRowsPerWarp][kColsPerLane];
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
      for (int j = 0; j < kColsPerLane; ++j) {
        const int y = by0 + warp * kRowsPerWarp + i;
        const int x = bx0 + lane + 32 * j;
        in[i][j] = y < rc.y1 && x < rc.x1;
        r[i][j] = in[i][j] ? d.R[(int64_t)y * d.nx + x] : 0.f;
      }

    const int y_first = by0 + warp * kRowsPerWarp;
    const int x_first = bx0 + lane;
    for (int base = 0; base < n_other; base += kChunk) {
      const int n = min(kChunk, n_other - base);
      __syncthreads();
      for (int jj = threadIdx.x; jj < n; jj += kThreads) {
        const int g = base + jj;
        const int s = find_tile(s_pre, d.T, g);
        const clean_component cc = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
        Comp4 c4;
        c4.y = cc.y;
        c4.x = cc.x;
        c4.f = cc.flux;
        c4.pad = 0;
        s_comp[jj] = c4;
      }
      __syncthreads();
      for (int jj = 0; jj < n; ++jj) {
        const Comp4 c4 = s_comp[jj];
        const int sy0 = y_first - c4.y + d.cy;
        const int sx0 = x_first - c4.x + d.cx;
#pragma unroll
        for (int i = 0; i < kRowsPerWarp; ++i) {
          const int sy = sy0 + i;
          const bool yin = (unsigned)sy < (unsigned)d.pny;
#pragma unroll
          for (int j = 0; j < kColsPerLane; ++j) {
            const int sx = sx0 + 32 * j;
            if (in[i][j] && yin && (unsigned)sx < (unsigned)d.pnx) {
              const float p = __ldg(d.P + (int64_t)sy * d.pnx + sx);
              r[i][j] = __fsub_rn(r[i][j], __fmul_rn(c4.f, p));
            }
          }
        }
      }
    }

    // write back and reduce this block's peak key
    float best_a = -1.f, best_v = 0.f;
    int best_i = 0x7fffffff;
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
      for (int j = 0; j < kColsPerLane; ++j) {
        if (!in[i][j]) continue;
        const int y = by0 + warp * kRowsPerWarp + i;
        const int x = bx0 + lane + 32 * j;
        const int gi = y * d.nx + x;
        if (n_other > 0) d.R[(int64_t)gi] = r[i][j];
        const float a = fabsf(r[i][j]);
        if (a > best_a || (a == best_a && gi < best_i)) {
          best_a = a;
          best_i = gi;
          best_v = r[i][j];
        }
      }
    uint64_t k = best_a >= 0.f ? make_key(best_v, best_i) : 0ull;
    k = warp_max_key(k);
    if (lane == 0) s_warp[warp] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t m = 0;
      for (int w = 0; w < kWarps; ++w) m = umax64(m, s_warp[w]);
      if (m) atomicMax((unsigned long long*)&d.peak[(parity ^ 1) * d.T + t],
                       (unsigned long long)m);
    }
  }

  close_round_if_last(d, parity, blocks_x * blocks_y * d.T, s_cnt, s_pre);
}

__global__ void __launch_bounds__(kThreads)
    feedback_kernel(PlanDev d, int parity, int apply, int blocks_x, int blocks_y) {
  feedback_body(d, parity, apply, blockIdx.z, blockIdx.x, blockIdx.y, blocks_x, blocks_y);
}


// ---------------------------------------------------------------------------
// TMA variant.  The same arithmetic, with the PSF window of every component
// staged into shared memory by one 2-D TMA box load (kBoxW x kRows floats at
// an x rounded down to 4 floats) through a ring of kStages buffers.  A
// producer warp issues the loads; eight consumer warps apply the updates
// from shared memory and release each buffer through an mbarrier.  Every
// mbarrier wait is bounded (status bit ST_TIMEOUT on expiry).
// ---------------------------------------------------------------------------
namespace tma {

// A block is 32 rows x 128 columns: a 132-float window row wastes 4 of 132
// floats and 1 of 17 L2 sectors, against 4 of 68 and 1 of 9 for 64 columns
// (measured: 2.63 vs 3.00 ms per 4096^2 round).  A 256-column block would
// need a 260-float box, past the 256-element limit of a TMA box.
constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kRowsPerWarp = 4;
constexpr int kColsPerLane = 4;
constexpr int kRows = kConsumerWarps * kRowsPerWarp;  // 32
constexpr int kCols = 32 * kColsPerLane;              // 128
constexpr int kBoxW = kCols + 4;                      // 132: covers any 4-float misalignment
constexpr int kStages = 3;
constexpr int kStageFloats = kBoxW * kRows;
constexpr int kStageBytes = kStageFloats * 4;         // 16896 (multiple of 128)
// 4 CTAs per SM: at most 56 registers a thread (65536 / (4 x 288)) and
// 4 x 55 KB of shared memory; 3 CTAs of 4 stages were 8 % slower
constexpr int kMinBlocks = 4;
constexpr int kListCap = 256;                        // components staged per chunk
constexpr uint32_t kFull = 1u << 8;                   // window lies inside the PSF

struct __align__(16) Win {
  int32_t x;    // TMA x (PSF column of the window, rounded down to 4 floats)
  int32_t y;    // PSF row of the block's first row
  float f;      // component flux
  uint32_t off; // bits 0-1: column offset within the box; kFull flag
};

size_t smem_bytes(int T) {
  return 128 + (size_t)kStages * kStageBytes + (size_t)kListCap * sizeof(Win) +
         sizeof(int32_t) * (2 * (size_t)T + 1);
}

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t limit,
                                              volatile int* abort, int32_t* status) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer_ns();
  for (;;) {
    if (ptx::mbar_try_wait_hint(bar, parity, ptx::kWaitHintNs)) return true;
    if (*abort) return false;
    if (ptx::globaltimer_ns() - t0 > limit) {
      *abort = 1;
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void feedback_tma_body(const PlanDev& d, const CUtensorMap* psf_map,
                                                  int parity, int apply, int t, int bxi, int byi,
                                                  int blocks_x, int blocks_y, uint64_t limit_ns) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* s_win = reinterpret_cast<float*>(base);
  Win* s_list = reinterpret_cast<Win*>(base + (size_t)kStages * kStageBytes);
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_list + kListCap);
  int32_t* s_pre = s_cnt + d.T;
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ uint64_t s_warp[kConsumerWarps];
  __shared__ int s_abort;

  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int by0 = rc.y0 + byi * kRows;
  const int bx0 = rc.x0 + bxi * kCols;
  const bool live = by0 < rc.y1 && bx0 < rc.x1 && *(volatile int32_t*)&d.st->status == 0 &&
                    round_total(d) > 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = warp == kConsumerWarps;

  if (live) {
    if (threadIdx.x == 0) {
      s_abort = 0;
      for (int i = 0; i < kStages; ++i) {
        ptx::mbar_init(&full_bar[i], 1);
        ptx::mbar_init(&empty_bar[i], kConsumerWarps);
      }
      ptx::fence_barrier_init();
    }
    if (producer && lane == 0) ptx::prefetch_tensormap(psf_map);
    for (int s = threadIdx.x; s < d.T; s += kThreads)
      s_cnt[s] = (s == t || !(apply && feedback_on(d))) ? 0 : d.rcount[s];
    block_prefix(s_cnt, s_pre, d.T);  // also orders the barrier set-up
    const int n_other = s_pre[d.T];

    float r[kRowsPerWarp][kColsPerLane];
    const int y_first = by0 + warp * kRowsPerWarp;
    if (!producer) {
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
        for (int j = 0; j < kColsPerLane; ++j) {
          const int y = y_first + i, x = bx0 + lane + 32 * j;
          r[i][j] = (y < rc.y1 && x < rc.x1) ? d.R[(int64_t)y * d.nx + x] : 0.f;
        }
    }

    int issued = 0;  // producer: loads issued so far
    for (int cbase = 0; cbase < n_other; cbase += kListCap) {
      const int n = min(kListCap, n_other - cbase);
      __syncthreads();
      for (int jj = threadIdx.x; jj < n; jj += kThreads) {
        const int g = cbase + jj;
        const int s = find_tile(s_pre, d.T, g);
        const clean_component cc = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
        const int sy0 = by0 - cc.y + d.cy;
        const int sx0 = bx0 - cc.x + d.cx;
        Win w;
        w.x = sx0 & ~3;
        w.y = sy0;
        w.f = cc.flux;
        const bool inside = sy0 >= 0 && sy0 + kRows <= d.pny && sx0 >= 0 && sx0 + kCols <= d.pnx;
        w.off = (uint32_t)(sx0 - w.x) | (inside ? kFull : 0u);
        s_list[jj] = w;
      }
      __syncthreads();
      if (producer) {
        if (lane == 0) {
          for (int jj = 0; jj < n; ++jj) {
            const int j = cbase + jj;
            const int st = j % kStages;
            if (j >= kStages &&
                !wait_or_abort(&empty_bar[st], (uint32_t)((j / kStages) - 1) & 1u, limit_ns,
                               &s_abort, &d.st->status))
              break;
            ptx::mbar_arrive_expect_tx(&full_bar[st], kStageBytes);
            ptx::tma_load_2d(s_win + (size_t)st * kStageFloats, psf_map, s_list[jj].x,
                             s_list[jj].y, &full_bar[st]);
            ++issued;
          }
        }
      } else {
        for (int jj = 0; jj < n; ++jj) {
          const int j = cbase + jj;
          const int st = j % kStages;
          if (!wait_or_abort(&full_bar[st], (uint32_t)(j / kStages) & 1u, limit_ns, &s_abort,
                             &d.st->status))
            break;
          const Win w = s_list[jj];
          const float* win = s_win + (size_t)st * kStageFloats +
                             (warp * kRowsPerWarp) * kBoxW + (w.off & 3u) + lane;
          if (w.off & kFull) {
#pragma unroll
            for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
              for (int c = 0; c < kColsPerLane; ++c)
                r[i][c] = __fsub_rn(r[i][c], __fmul_rn(w.f, win[i * kBoxW + 32 * c]));
          } else {
            // window partly off the PSF array: those pixels stay unchanged
            const int sxl = w.x + (int)(w.off & 3u) + lane;
#pragma unroll
            for (int i = 0; i < kRowsPerWarp; ++i) {
              const bool yin = (unsigned)(w.y + warp * kRowsPerWarp + i) < (unsigned)d.pny;
#pragma unroll
              for (int c = 0; c < kColsPerLane; ++c)
                if (yin && (unsigned)(sxl + 32 * c) < (unsigned)d.pnx)
                  r[i][c] = __fsub_rn(r[i][c], __fmul_rn(w.f, win[i * kBoxW + 32 * c]));
            }
          }
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&empty_bar[st]);
        }
      }
    }
    __syncthreads();
    if (producer && lane == 0 && s_abort) {
      // after an expired wait: let this CTA's own loads in flight land
      for (int j = max(0, issued - kStages); j < issued; ++j) {
        const uint64_t t0 = ptx::globaltimer_ns();
        while (!ptx::mbar_try_wait(&full_bar[j % kStages], (uint32_t)(j / kStages) & 1u))
          if (ptx::globaltimer_ns() - t0 > limit_ns) break;
      }
    }

    // write back and reduce this block's peak key
    uint64_t k = 0ull;
    if (!producer) {
      float best_a = -1.f, best_v = 0.f;
      int best_i = 0x7fffffff;
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
        for (int c = 0; c < kColsPerLane; ++c) {
          const int y = y_first + i, x = bx0 + lane + 32 * c;
          if (y >= rc.y1 || x >= rc.x1) continue;
          const int gi = y * d.nx + x;
          if (n_other > 0) d.R[(int64_t)gi] = r[i][c];
          const float a = fabsf(r[i][c]);
          if (a > best_a || (a == best_a && gi < best_i)) {
            best_a = a;
            best_i = gi;
            best_v = r[i][c];
          }
        }
      k = best_a >= 0.f ? make_key(best_v, best_i) : 0ull;
      k = warp_max_key(k);
      if (lane == 0) s_warp[warp] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t m = 0;
      for (int w = 0; w < kConsumerWarps; ++w) m = umax64(m, s_warp[w]);
      if (m) atomicMax((unsigned long long*)&d.peak[(parity ^ 1) * d.T + t],
                       (unsigned long long)m);
    }
  }
  close_round_if_last(d, parity, blocks_x * blocks_y * d.T, s_cnt, s_pre);
}

__global__ void __launch_bounds__(kThreads, kMinBlocks)
    feedback_tma_kernel(PlanDev d, const __grid_constant__ CUtensorMap psf_map, int parity,
                        int apply, int blocks_x, int blocks_y, uint64_t limit_ns) {
  feedback_tma_body(d, &psf_map, parity, apply, blockIdx.z, blockIdx.x, blockIdx.y, blocks_x,
                    blocks_y, limit_ns);
}

}  // namespace tma

// ---------------------------------------------------------------------------
// Batched feedback: the blocks of many images in one flattened grid; block
// b belongs to the image whose [block0, block0 + nblocks) range holds it.
// Each image closes its own round (its own last block).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_image(const BatchImage* imgs, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (imgs[mid].block0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads)
    feedback_batch_kernel(const PlanDev* __restrict__ plans, const BatchImage* __restrict__ imgs,
                          int n_images, int round, int apply) {
  const int i = batch_image(imgs, n_images, blockIdx.x);
  const BatchImage im = imgs[i];
  const PlanDev d = plans[i];
  const int local = blockIdx.x - im.block0;
  const int per_tile = im.bx * im.by;
  const int t = local / per_tile, rem = local - t * per_tile;
  feedback_body(d, (round - d.round0) & 1, apply, t, rem % im.bx, rem / im.bx, im.bx, im.by);
}

__global__ void __launch_bounds__(tma::kThreads, tma::kMinBlocks)
    feedback_tma_batch_kernel(const PlanDev* __restrict__ plans,
                              const BatchImage* __restrict__ imgs, const CUtensorMap* maps,
                              int n_images, int round, int apply, uint64_t limit_ns) {
  const int i = batch_image(imgs, n_images, blockIdx.x);
  const BatchImage im = imgs[i];
  const PlanDev d = plans[i];
  const int local = blockIdx.x - im.block0;
  const int per_tile = im.bx * im.by;
  const int t = local / per_tile, rem = local - t * per_tile;
  tma::feedback_tma_body(d, maps + i, (round - d.round0) & 1, apply, t, rem % im.bx, rem / im.bx,
                         im.bx, im.by, limit_ns);
}


}  // namespace

cudaError_t launch_feedback(const PlanDev& d, const CUtensorMap* psf_map, int parity,
                            int apply, uint64_t limit_ns, cudaStream_t s) {
  // blocks sized for the largest tile; blocks past a smaller tile's edge
  // only take part in the round close
  int maxH = 0, maxW = 0;
  for (int i = 0; i < d.ty; ++i)
    maxH = max(maxH, (int)(((int64_t)(i + 1) * d.ny) / d.ty - ((int64_t)i * d.ny) / d.ty));
  for (int j = 0; j < d.tx; ++j)
    maxW = max(maxW, (int)(((int64_t)(j + 1) * d.nx) / d.tx - ((int64_t)j * d.nx) / d.tx));
  if (psf_map) {
    const int bx = (maxW + tma::kCols - 1) / tma::kCols, by = (maxH + tma::kRows - 1) / tma::kRows;
    const size_t smem = tma::smem_bytes(d.T);
    tma::feedback_tma_kernel<<<dim3(bx, by, d.T), tma::kThreads, smem, s>>>(
        d, *psf_map, parity, apply, bx, by, limit_ns);
    return cudaGetLastError();
  }
  const int bx = (maxW + kCols - 1) / kCols, by = (maxH + kRows - 1) / kRows;
  const size_t smem = sizeof(Comp4) * kChunk + sizeof(int32_t) * (2 * (size_t)d.T + 1);
  feedback_kernel<<<dim3(bx, by, d.T), kThreads, smem, s>>>(d, parity, apply, bx, by);
  return cudaGetLastError();
}


void feedback_blocks(const PlanDev& d, bool use_tma, int* bx, int* by) {
  int maxH = 0, maxW = 0;
  for (int i = 0; i < d.ty; ++i)
    maxH = max(maxH, (int)(((int64_t)(i + 1) * d.ny) / d.ty - ((int64_t)i * d.ny) / d.ty));
  for (int j = 0; j < d.tx; ++j)
    maxW = max(maxW, (int)(((int64_t)(j + 1) * d.nx) / d.tx - ((int64_t)j * d.nx) / d.tx));
  const int kc = use_tma ? tma::kCols : kCols, kr = use_tma ? tma::kRows : kRows;
  *bx = (maxW + kc - 1) / kc;
  *by = (maxH + kr - 1) / kr;
}

cudaError_t launch_feedback_batch(const PlanDev* plans, const BatchImage* imgs, int n_images,
                                  int total_blocks, int max_T, const CUtensorMap* maps,
                                  int round, int apply, uint64_t limit_ns, cudaStream_t s) {
  if (n_images <= 0 || total_blocks <= 0) return cudaSuccess;
  if (maps) {
    const size_t smem = tma::smem_bytes(max_T);
    cudaError_t e = allow_max_smem((const void*)feedback_tma_batch_kernel);
    if (e != cudaSuccess) return e;
    feedback_tma_batch_kernel<<<total_blocks, tma::kThreads, smem, s>>>(plans, imgs, maps,
                                                                         n_images, round, apply,
                                                                         limit_ns);
  } else {
    const size_t smem = sizeof(Comp4) * kChunk + sizeof(int32_t) * (2 * (size_t)max_T + 1);
    cudaError_t e = allow_max_smem((const void*)feedback_batch_kernel);
    if (e != cudaSuccess) return e;
    feedback_batch_kernel<<<total_blocks, kThreads, smem, s>>>(plans, imgs, n_images, round,
                                                               apply);
  }
  return cudaGetLastError();
}

cudaError_t feedback_prepare(int T) {
  (void)T;
  cudaError_t e = allow_max_smem((const void*)feedback_kernel);
  if (e != cudaSuccess) return e;
  e = allow_max_smem((const void*)tma::feedback_tma_kernel);
  if (e != cudaSuccess) return e;
  return fft_prepare();
}


// 2-D tiled tensor map of a row-major float array, box_w x box_h floats.
// L2 misses are promoted to 128-byte lines: with 256-byte promotion the
// feedback round took 2.606 ms, with 128 bytes or none 2.580 (4096^2).
bool encode_tensor_map_2d(CUtensorMap* map, const float* base, int rows, int cols, int box_w,
                          int box_h) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cudaGetLastError();
  });
  if (!encode) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base),
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_psf_tensor_map(CUtensorMap* map, const float* psf, int pny, int pnx) {
  if ((reinterpret_cast<uintptr_t>(psf) & 15u) != 0 || (pnx % 4) != 0) return false;
  if (pnx < tma::kBoxW || pny < tma::kRows) return false;
  return encode_tensor_map_2d(map, psf, pny, pnx, tma::kBoxW, tma::kRows);
}

}  // namespace cleangb
