// Device helpers shared by the feedback kernels (gather and FFT): 64-bit
// key maxima, the block-wide prefix of the tiles' component counts, and the
// close of a round by the last CTA of a feedback launch.  Included by one
// translation unit each; everything here has internal linkage.
#pragma once

#include "cleangb_internal.cuh"

namespace cleangb {
namespace {

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

}  // namespace
}  // namespace cleangb
