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

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) {
  return a > b ? a : b;
}

__device__ __forceinline__ uint64_t warp_max_key(uint64_t k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = umax64(k, __shfl_xor_sync(0xffffffffu, k, o));
  return k;
}

// Exclusive prefix of cnt[0..T) into pre[0..T]; whole block participates.
__device__ void block_prefix(const int32_t* cnt, int32_t* pre, int T) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int carry = 0;
    for (int b = 0; b < T; b += 32) {
      int v = (b + lane < T) ? cnt[b + lane] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
      }
      if (b + lane < T) pre[b + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) pre[T] = carry;
  }
  __syncthreads();
}

// Largest s with pre[s] <= g (pre non-decreasing, pre[0] = 0 <= g < pre[T]).
__device__ __forceinline__ int find_tile(const int32_t* pre, int T, int g) {
  int lo = 0, hi = T - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}


// The last CTA of the feedback launch closes the round: appends the round's
// components to the list (tile order, then iteration), records the round's
// list offset, and decides whether any tile can run again.  Every thread of
// every CTA calls this once, after its pixels are final.
__device__ void close_round_if_last(const PlanDev& d, int parity, int total_blocks,
                                    int32_t* s_cnt, int32_t* s_pre, float* clear_grid = nullptr,
                                    int64_t clear_pitch = 0) {
  __shared__ int s_last;
  __shared__ int64_t s_mb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nthr = blockDim.x, nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&d.st->fb_done, 1u);
    s_last = (done == (unsigned)total_blocks - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  for (int s = threadIdx.x; s < d.T; s += nthr) s_cnt[s] = ((volatile int32_t*)d.rcount)[s];
  block_prefix(s_cnt, s_pre, d.T);
  const int n_all = s_pre[d.T];
  const int64_t total0 = d.st->total;
  for (int g = threadIdx.x; g < n_all; g += nthr) {
    const int s = find_tile(s_pre, d.T, g);
    const clean_component cc = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
    d.list[total0 + g] = cc;
    if (clear_grid) clear_grid[(int64_t)cc.y * clear_pitch + cc.x] = 0.f;
  }
  // any tile that can run next round; largest remaining budget; the largest
  // |peak| among those tiles (the flux trigger's reference)
  int act = 0;
  int64_t mb = 0;
  uint32_t top = 0u;  // |peak| bits: non-negative floats order like integers
  for (int s = threadIdx.x; s < d.T; s += nthr) {
    const int64_t b = ((volatile int64_t*)d.budget)[s];
    const uint64_t pk = ((volatile unsigned long long*)d.peak)[(parity ^ 1) * d.T + s];
    if (b > 0 && pk != 0ull && key_abs(pk) > d.thr) {
      act = 1;
      top = max(top, (uint32_t)(pk >> 32));
    }
    mb = b > mb ? b : mb;
  }
  act = __syncthreads_or(act);
  __shared__ uint32_t s_top;
  if (threadIdx.x == 0) s_top = 0u;
  __syncthreads();
  if (top) atomicMax(&s_top, top);
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t other = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = other > mb ? other : mb;
  }
  if (lane == 0) s_mb[warp] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t m = 0;
    for (int w = 0; w < nwarps; ++w) m = s_mb[w] > m ? s_mb[w] : m;
    if (n_all > 0) {
      d.round_off[d.st->n_rounds] = total0;
      d.st->n_rounds += 1;
    }
    d.st->total = total0 + n_all;
    d.st->round_comps = n_all;
    d.st->active = act;
    d.st->max_budget = m;
    d.st->level = d.trigger > 0.f ? __fmul_rn(d.trigger, __uint_as_float(s_top)) : 0.f;
    d.st->fb_done = 0u;
  }
}

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
// Pipelined-load variant.  The same arithmetic and block layout as
// feedback_kernel, with the PSF values of the next kDepth components already
// in flight (register buffers) while the current component is applied, so
// the read latency of L2 is hidden without staging windows in shared memory.
// The loads go through L1, where windows of nearby components overlap.
// Components whose window is clipped by the PSF array take a checked path.
// ---------------------------------------------------------------------------
namespace ldg {

constexpr int kDepth = 4;     // components whose PSF values are in flight
constexpr int kChunk = 1024;  // components staged in shared memory at once

struct __align__(16) Win {
  int32_t sy0, sx0;  // PSF row and column of the block's first pixel
  float f;           // component flux
  int32_t inside;    // the block's whole window lies inside the PSF array
};

size_t smem_bytes(int T) {
  return sizeof(Win) * kChunk + sizeof(int32_t) * (2 * (size_t)T + 1);
}

__device__ __forceinline__ void feedback_ldg_body(const PlanDev& d, int parity, int apply, int t,
                                                  int bxi, int byi, int blocks_x, int blocks_y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Win* s_win = reinterpret_cast<Win*>(smem_raw);
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_win + kChunk);
  int32_t* s_pre = s_cnt + d.T;  // [T + 1]
  __shared__ uint64_t s_warp[kWarps];

  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int by0 = rc.y0 + byi * kRows;
  const int bx0 = rc.x0 + bxi * kCols;
  const bool live = by0 < rc.y1 && bx0 < rc.x1 && *(volatile int32_t*)&d.st->status == 0 &&
                    round_total(d) > 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (live) {
    const bool fb = apply && feedback_on(d);
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

    const float* __restrict__ P = d.P;
    const int pnx = d.pnx;
    const int wrow = warp * kRowsPerWarp;
    float buf[kDepth][kRowsPerWarp][kColsPerLane];

    // PSF values of staged component jj for this thread (whole window inside)
    auto issue = [&](float(&b)[kRowsPerWarp][kColsPerLane], int jj, int n) {
      if (jj < n) {
        const Win w = s_win[jj];
        if (w.inside) {
          const float* q = P + ((int64_t)(w.sy0 + wrow) * pnx + w.sx0 + lane);
#pragma unroll
          for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
            for (int j = 0; j < kColsPerLane; ++j) b[i][j] = __ldg(q + (int64_t)i * pnx + 32 * j);
        }
      }
    };

    for (int base = 0; base < n_other; base += kChunk) {
      const int n = min(kChunk, n_other - base);
      __syncthreads();
      for (int jj = threadIdx.x; jj < n; jj += kThreads) {
        const int g = base + jj;
        const int s = find_tile(s_pre, d.T, g);
        const clean_component cc = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
        Win w;
        w.sy0 = by0 - cc.y + d.cy;
        w.sx0 = bx0 - cc.x + d.cx;
        w.f = cc.flux;
        w.inside = w.sy0 >= 0 && w.sy0 + kRows <= d.pny && w.sx0 >= 0 && w.sx0 + kCols <= d.pnx;
        s_win[jj] = w;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kDepth; ++u) issue(buf[u], u, n);
      for (int j0 = 0; j0 < n; j0 += kDepth) {
#pragma unroll
        for (int u = 0; u < kDepth; ++u) {
          const int jj = j0 + u;
          if (jj < n) {
            const Win w = s_win[jj];
            if (w.inside) {
#pragma unroll
              for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
                for (int j = 0; j < kColsPerLane; ++j)
                  r[i][j] = __fsub_rn(r[i][j], __fmul_rn(w.f, buf[u][i][j]));
            } else {
              // window partly off the PSF array: those pixels stay unchanged
#pragma unroll
              for (int i = 0; i < kRowsPerWarp; ++i) {
                const int sy = w.sy0 + wrow + i;
                const bool yin = (unsigned)sy < (unsigned)d.pny;
#pragma unroll
                for (int j = 0; j < kColsPerLane; ++j) {
                  const int sx = w.sx0 + lane + 32 * j;
                  if (in[i][j] && yin && (unsigned)sx < (unsigned)pnx)
                    r[i][j] = __fsub_rn(r[i][j], __fmul_rn(w.f, __ldg(P + (int64_t)sy * pnx + sx)));
                }
              }
            }
            issue(buf[u], jj + kDepth, n);
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
        const int y = by0 + wrow + i;
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

__global__ void __launch_bounds__(kThreads, 2)
    feedback_ldg_kernel(PlanDev d, int parity, int apply, int blocks_x, int blocks_y) {
  feedback_ldg_body(d, parity, apply, blockIdx.z, blockIdx.x, blockIdx.y, blocks_x, blocks_y);
}

}  // namespace ldg

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


// ---------------------------------------------------------------------------
// FFT feedback (tolerance-exact alternative to the gather).  The round's
// components, scattered onto an L x L grid (L >= 2N - 1 in each axis),
// convolved circularly with the PSF kernel K[d mod L] = P[d + c] give, at
// every image pixel q, S[q] = sum_c f_c P[q - p_c + c] with no wrap-around.
// The residual after the round is then the residual at the round's start
// minus S on every pixel of every tile (the minor loops' own-tile
// subtractions included), so no per-tile correction is needed.
// ---------------------------------------------------------------------------
constexpr int kFftThreads = 256;
constexpr int kFftRows = 16;

// K[(dy mod Ly), (dx mod Lx)] = P[dy + cy, dx + cx] for |dy| < ny, |dx| < nx
// inside the PSF; zero elsewhere.  One thread per grid element.
__global__ void fft_kernel_image(const float* __restrict__ P, int pny, int pnx, int cy, int cx,
                                 int ny, int nx, int Ly, int Lx, float* __restrict__ Kimg) {
  const int64_t n = (int64_t)Ly * Lx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int my = (int)(i / Lx), mx = (int)(i - (int64_t)my * Lx);
    const int dy = my < ny ? my : my - Ly;   // represent m as d in (-(L - ny), ny)
    const int dx = mx < nx ? mx : mx - Lx;
    float v = 0.f;
    if (dy > -ny && dx > -nx) {
      const int sy = dy + cy, sx = dx + cx;
      if ((unsigned)sy < (unsigned)pny && (unsigned)sx < (unsigned)pnx)
        v = P[(int64_t)sy * pnx + sx];
    }
    Kimg[i] = v;
  }
}

// The round's components onto the (zeroed) grid: one warp per tile (a
// tile's components lie inside it, so tiles never share a cell).  Lane l
// takes components l, l + 32, ...; the first component at a cell sums every
// component of the tile at that cell in iteration order and writes the cell
// once, so each cell gets ((0 + f1) + f2) + ... exactly as one thread adding
// them in order would.  Above kScatterQuadMax components the quadratic
// search gives way to one thread in order.
constexpr int kScatterQuadMax = 4096;
__global__ void fft_scatter(PlanDev d, float* __restrict__ A, int64_t pitch) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= d.T) return;
  const int n = d.rcount[t];
  const clean_component* c = d.rcomps + (int64_t)t * d.cap_round;
  if (n > kScatterQuadMax) {
    if (lane == 0)
      for (int k = 0; k < n; ++k) {
        float* a = &A[(int64_t)c[k].y * pitch + c[k].x];
        *a = *a + c[k].flux;
      }
    return;
  }
  for (int k = lane; k < n; k += 32) {
    const clean_component ck = c[k];
    bool first = true;
    for (int j = 0; j < k && first; ++j) first = !(c[j].y == ck.y && c[j].x == ck.x);
    if (!first) continue;
    float* a = &A[(int64_t)ck.y * pitch + ck.x];
    float acc = *a + ck.flux;
    for (int j = k + 1; j < n; ++j)
      if (c[j].y == ck.y && c[j].x == ck.x) acc = acc + c[j].flux;
    *a = acc;
  }
}

// X <- X * K / (Ly Lx), complex, element by element.
__global__ void fft_multiply(float2* __restrict__ X, const float2* __restrict__ Kh, int64_t n,
                             float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = X[i], b = Kh[i];
    X[i] = make_float2((a.x * b.x - a.y * b.y) * scale, (a.x * b.y + a.y * b.x) * scale);
  }
}

// R <- R0 - S on tile t's rows [ya, ya + kFftRows); R0 <- R; the block's
// peak into the tile's next-round key; the last block closes the round and
// clears the scattered grid cells.
__global__ void __launch_bounds__(kFftThreads)
    fft_subtract(PlanDev d, float* __restrict__ R0, const float* __restrict__ S, int64_t pitch,
                 float* __restrict__ A, int parity, int blocks_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t* s_cnt = reinterpret_cast<int32_t*>(smem_raw);
  int32_t* s_pre = s_cnt + d.T;
  __shared__ uint64_t s_warp[kFftThreads / 32];
  const int t = blockIdx.y;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int ya = rc.y0 + blockIdx.x * kFftRows, yb = min(rc.y1, ya + kFftRows);
  const bool live = *(volatile int32_t*)&d.st->status == 0;
  float best_a = -1.f, best_v = 0.f;
  int best_i = 0x7fffffff;
  if (live) {
    for (int y = ya; y < yb; ++y)
      for (int x = rc.x0 + threadIdx.x; x < rc.x1; x += kFftThreads) {
        const int64_t gi = (int64_t)y * d.nx + x;
        const float r = R0[gi] - S[(int64_t)y * pitch + x];
        d.R[gi] = r;
        R0[gi] = r;
        const float a = fabsf(r);
        if (a > best_a || (a == best_a && (int)gi < best_i)) {
          best_a = a;
          best_i = (int)gi;
          best_v = r;
        }
      }
  }
  uint64_t k = best_a >= 0.f ? make_key(best_v, best_i) : 0ull;
  k = warp_max_key(k);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t m = 0;
    for (int w = 0; w < kFftThreads / 32; ++w) m = umax64(m, s_warp[w]);
    if (m) atomicMax((unsigned long long*)&d.peak[(parity ^ 1) * d.T + t], (unsigned long long)m);
  }
  close_round_if_last(d, parity, blocks_x * d.T, s_cnt, s_pre, A, pitch);
}

}  // namespace

cudaError_t launch_feedback_ldg(const PlanDev& d, int parity, int apply, cudaStream_t s) {
  int bx, by;
  feedback_blocks(d, false, &bx, &by);
  ldg::feedback_ldg_kernel<<<dim3(bx, by, d.T), kThreads, ldg::smem_bytes(d.T), s>>>(
      d, parity, apply, bx, by);
  return cudaGetLastError();
}

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


cudaError_t fft_build_kernel_image(const PlanDev& d, int Ly, int Lx, float* Kimg,
                                   cudaStream_t s) {
  fft_kernel_image<<<4096, 256, 0, s>>>(d.P, d.pny, d.pnx, d.cy, d.cx, d.ny, d.nx, Ly, Lx, Kimg);
  return cudaGetLastError();
}

cudaError_t fft_launch_scatter(const PlanDev& d, float* A, int64_t pitch, cudaStream_t s) {
  fft_scatter<<<(d.T + 3) / 4, 128, 0, s>>>(d, A, pitch);  // a warp per tile
  return cudaGetLastError();
}

cudaError_t fft_launch_multiply(void* X, const void* Kh, int64_t n, float scale,
                                cudaStream_t s) {
  fft_multiply<<<4096, 256, 0, s>>>(reinterpret_cast<float2*>(X),
                                    reinterpret_cast<const float2*>(Kh), n, scale);
  return cudaGetLastError();
}

cudaError_t fft_launch_subtract(const PlanDev& d, float* R0, const float* S, int64_t pitch,
                                float* A, int parity, cudaStream_t s) {
  int maxH = 0;
  for (int i = 0; i < d.ty; ++i)
    maxH = max(maxH, (int)(((int64_t)(i + 1) * d.ny) / d.ty - ((int64_t)i * d.ny) / d.ty));
  const int bx = (maxH + kFftRows - 1) / kFftRows;
  const size_t smem = sizeof(int32_t) * (2 * (size_t)d.T + 1);
  fft_subtract<<<dim3(bx, d.T), kFftThreads, smem, s>>>(d, R0, S, pitch, A, parity, bx);
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
  e = allow_max_smem((const void*)ldg::feedback_ldg_kernel);
  if (e != cudaSuccess) return e;
  return allow_max_smem((const void*)fft_subtract);
}


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
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_psf_tensor_map(CUtensorMap* map, const float* psf, int pny, int pnx) {
  if ((reinterpret_cast<uintptr_t>(psf) & 15u) != 0 || (pnx % 4) != 0) return false;
  if (pnx < tma::kBoxW || pny < tma::kRows) return false;
  return encode_tensor_map_2d(map, psf, pny, pnx, tma::kBoxW, tma::kRows);
}

}  // namespace cleangb
