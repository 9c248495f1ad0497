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
#include "cleangb_internal.cuh"

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

__global__ void __launch_bounds__(kThreads)
    feedback_kernel(PlanDev d, int parity, int apply, int blocks_x, int blocks_y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Comp4* s_comp = reinterpret_cast<Comp4*>(smem_raw);
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_comp + kChunk);
  int32_t* s_pre = s_cnt + d.T;  // [T + 1]
  __shared__ uint64_t s_warp[kWarps];
  __shared__ int s_last;

  const int t = blockIdx.z;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int by0 = rc.y0 + blockIdx.y * kRows;
  const int bx0 = rc.x0 + blockIdx.x * kCols;
  const bool live = by0 < rc.y1 && bx0 < rc.x1 && *(volatile int32_t*)&d.st->status == 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (live) {
    // the other tiles' components of this round, in list order
    for (int s = threadIdx.x; s < d.T; s += kThreads) s_cnt[s] = (s == t || !apply) ? 0 : d.rcount[s];
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

  // ---- last CTA closes the round ----
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned total_blocks = (unsigned)(blocks_x * blocks_y * d.T);
    const unsigned done = atomicAdd(&d.st->fb_done, 1u);
    s_last = (done == total_blocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  for (int s = threadIdx.x; s < d.T; s += kThreads) s_cnt[s] = ((volatile int32_t*)d.rcount)[s];
  block_prefix(s_cnt, s_pre, d.T);
  const int n_all = s_pre[d.T];
  const int64_t total0 = d.st->total;
  for (int g = threadIdx.x; g < n_all; g += kThreads) {
    const int s = find_tile(s_pre, d.T, g);
    d.list[total0 + g] = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
  }
  // any tile that can run next round; largest remaining budget
  int act = 0;
  int64_t mb = 0;
  for (int s = threadIdx.x; s < d.T; s += kThreads) {
    const int64_t b = ((volatile int64_t*)d.budget)[s];
    const uint64_t pk = ((volatile unsigned long long*)d.peak)[(parity ^ 1) * d.T + s];
    if (b > 0 && pk != 0ull && key_abs(pk) > d.thr) act = 1;
    mb = b > mb ? b : mb;
    d.gbar[s] = 0u;
  }
  act = __syncthreads_or(act);
  // max of mb over the block
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t other = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = other > mb ? other : mb;
  }
  __shared__ int64_t s_mb[kWarps];
  if (lane == 0) s_mb[warp] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t m = 0;
    for (int w = 0; w < kWarps; ++w) m = s_mb[w] > m ? s_mb[w] : m;
    if (n_all > 0) {
      d.round_off[d.st->n_rounds] = total0;
      d.st->n_rounds += 1;
    }
    d.st->total = total0 + n_all;
    d.st->round_comps = n_all;
    d.st->active = act;
    d.st->max_budget = m;
    d.st->fb_done = 0u;
  }
}

}  // namespace

cudaError_t launch_feedback(const PlanDev& d, int parity, int apply, cudaStream_t s) {
  // blocks sized for the largest tile; blocks past a smaller tile's edge
  // only take part in the round close
  int maxH = 0, maxW = 0;
  for (int i = 0; i < d.ty; ++i)
    maxH = max(maxH, (int)(((int64_t)(i + 1) * d.ny) / d.ty - ((int64_t)i * d.ny) / d.ty));
  for (int j = 0; j < d.tx; ++j)
    maxW = max(maxW, (int)(((int64_t)(j + 1) * d.nx) / d.tx - ((int64_t)j * d.nx) / d.tx));
  const int bx = (maxW + kCols - 1) / kCols, by = (maxH + kRows - 1) / kRows;
  const size_t smem = sizeof(Comp4) * kChunk + sizeof(int32_t) * (2 * (size_t)d.T + 1);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(feedback_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sizeof(Comp4) * kChunk + sizeof(int32_t) * (2 * 4096 + 1));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  feedback_kernel<<<dim3(bx, by, d.T), kThreads, smem, s>>>(d, parity, apply, bx, by);
  return cudaGetLastError();
}

}  // namespace cleangb
