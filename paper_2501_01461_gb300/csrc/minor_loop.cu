// Minor loop of tiled Hogbom CLEAN (Section 3, first and second equations;
// Section 2, Fig. 1): one round of up to K iterations in every tile at once.
//
// Each tile is served by a group of G CTAs; CTA `rank` owns the tile rows
// [y0 + floor(rank H / G), y0 + floor((rank + 1) H / G)).  Per iteration:
//   1. every CTA knows the tile's peak (index p, signed value v) from the
//      previous iteration's exchange (the first from the round's input key);
//   2. f = gain * v (rounded); rank 0 records the component and adds f to
//      the model pixel (the model is thus summed in list order);
//   3. each CTA subtracts f * PSF[q - p + c] from its rows (a rounded
//      multiply, then a rounded subtract) and, in the same pass, finds the
//      largest |R| of its rows (ties: lowest index);
//   4. the G partial keys are exchanged and reduced identically by every CTA:
//      through distributed shared memory after a hardware cluster barrier
//      (G CTAs form one thread-block cluster), or through global memory after
//      a bounded grid barrier (cooperative launch, all CTAs co-resident).
// The loop stops when the tile's budget or K is reached or |v| <= threshold.
// With `resident`, a CTA holds its rows in shared memory for the whole round
// and only the PSF window streams in per iteration.
//
// The kernels in this file, as the plan picks them:
//   minor_kernel         plain loads (resident slabs; the allocation-free
//                        whole-GPU entry point)
//   minor_pipe_kernel    a TMA producer warp streams each chunk's residual and
//                        PSF boxes through an mbarrier ring to 15 consumer
//                        warps; with TM, each CTA's first chunks keep their
//                        residual in tensor memory for the launch
//   minor_pair_kernel    the pipeline with groups of 2G CTAs serving two tiles
//                        alternately (grid groups, streamed rows, even T)
//   minor_batch_kernel,  the same bodies over the (image, tile) items of a
//   minor_pipe_batch_kernel  batch (one CTA or one cluster per item)
// Every variant gives the same bits.
#include <algorithm>

#include "cleangb_internal.cuh"
#include "ptx.cuh"

namespace cleangb {

namespace {

constexpr int kThreads = 1024;
constexpr int kUnroll = 8;
constexpr int kSyncNone = 3;  // one CTA per tile (batched launches)

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) {
  return a > b ? a : b;
}

__device__ __forceinline__ uint64_t warp_max_key(uint64_t k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = umax64(k, __shfl_xor_sync(0xffffffffu, k, o));
  return k;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t ld_cluster_u64(const uint64_t* local, uint32_t rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), ra;
  uint64_t v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One fused pass over rows [ya, yb) x cols [x0, x1): subtract f * PSF
// shifted to (py, px) and track the largest |R| (lowest index on ties).
// Rows are mapped to threads as (tid / tpr, tid % tpr), tpr = threads per
// row (a power of two); kUnroll rows are in flight per thread.
template <bool RES>
__device__ __forceinline__ void subtract_pass(const PlanDev& d, float* __restrict__ sR,
                                              int ya, int yb, int x0, int x1,
                                              float f, int py, int px, float& best_a,
                                              int& best_i, float& best_v) {
  const int W = x1 - x0;
  // threads per row: a power of two (so it divides the block) >= W, <= block
  int tpr = 32;
  while (tpr < W && tpr < kThreads) tpr <<= 1;
  const int rps = kThreads / tpr;  // rows per step
  const int col = threadIdx.x % tpr;
  const int row = threadIdx.x / tpr;
  const int dy = d.cy - py, dx = d.cx - px;  // PSF index = pixel + (dy, dx)
  float* __restrict__ R = d.R;
  const float* __restrict__ P = d.P;
  for (int yb0 = ya + row; yb0 < yb; yb0 += rps * kUnroll) {
    for (int c = col; c < W; c += tpr) {
      const int x = x0 + c;
      const int sx = x + dx;
      const bool xin = (unsigned)sx < (unsigned)d.pnx;
      float rv[kUnroll], pv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int y = yb0 + u * rps;
        const int sy = y + dy;
        const bool in = y < yb;
        const bool pin = in && xin && (unsigned)sy < (unsigned)d.pny;
        if (RES)
          rv[u] = in ? sR[(y - ya) * W + c] : 0.f;
        else
          rv[u] = in ? R[(int64_t)y * d.nx + x] : 0.f;
        pv[u] = pin ? __ldg(P + (int64_t)sy * d.pnx + sx) : 0.f;
        if (pin) rv[u] = __fsub_rn(rv[u], __fmul_rn(f, pv[u]));
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int y = yb0 + u * rps;
        if (y < yb) {
          if (RES)
            sR[(y - ya) * W + c] = rv[u];
          else
            R[(int64_t)y * d.nx + x] = rv[u];
          const float a = fabsf(rv[u]);
          const int gi = y * d.nx + x;
          if (a > best_a || (a == best_a && gi < best_i)) {
            best_a = a;
            best_i = gi;
            best_v = rv[u];
          }
        }
      }
    }
  }
}

// Block-wide max of keys; the result is valid in warp 0.
__device__ __forceinline__ uint64_t block_max_key(uint64_t k, uint64_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  k = warp_max_key(k);
  if (lane == 0) s_warp[warp] = k;
  __syncthreads();
  if (warp == 0) {
    k = lane < nwarps ? s_warp[lane] : 0ull;
    k = warp_max_key(k);
  }
  return k;
}

// Step 4: every CTA of the tile group publishes its partial key `mine`
// (valid in thread 0) and gets the group maximum back, identical in every
// CTA.  Called by all threads; ends with a CTA barrier.
//
// Cluster groups read the partial keys through distributed shared memory
// after a cluster barrier.  Grid groups exchange through global memory with
// no counter and no fence: exchange g (g = seq0 + k counts the tile's
// exchanges since the run started) writes slot set g & 1 and marks each key
// with bit 63 = (g >> 1) & 1, a bit no key uses (|R| is non-negative).  The
// previous write to a slot (exchange g - 2) carries the other mark, so a
// reader polls the G slots until all carry the current mark.  A writer can
// reach exchange g + 2 only after every CTA published exchange g + 1, which
// each does after reading exchange g, so no slot is overwritten early.
// Slots start with mark 1 (the run's first two exchanges expect 0).  An
// expired wait sets ST_TIMEOUT and *s_abort.
template <int SYNC>
__device__ __forceinline__ uint64_t exchange_keys(const PlanDev& d, const MinorCfg& c, int t,
                                                  int rank, int64_t k, uint32_t seq0,
                                                  uint64_t mine, uint64_t* s_part,
                                                  uint64_t* s_best, int* s_abort) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = c.G;
  if (SYNC == kSyncNone) {
    if (threadIdx.x == 0) *s_best = mine;  // one CTA per tile: nothing to exchange
  } else if (SYNC == CLEAN_SYNC_CLUSTER) {
    if (threadIdx.x == 0) s_part[k & 1] = mine;
    cluster_sync_all();
    if (warp == 0) {
      uint64_t kk = lane < G ? ld_cluster_u64(&s_part[k & 1], (uint32_t)lane) : 0ull;
      kk = warp_max_key(kk);
      if (lane == 0) *s_best = kk;
    }
  } else {
    if (warp == 0) {
      const uint32_t g = seq0 + (uint32_t)k;
      uint64_t* slot = d.gkeys + (int64_t)t * G + (int64_t)(g & 1u) * ((int64_t)d.T * G);
      const uint64_t mark = (uint64_t)((g >> 1) & 1u) << 63;
      // a forced timeout waits for a mark no CTA writes
      const uint64_t want = c.force_timeout ? (mark ^ (1ull << 63)) : mark;
      if (lane == 0) st_relaxed_u64(slot + rank, mine | mark);
      uint64_t kk = 0ull;
      int abort = 0;
      const uint64_t t0 = globaltimer_ns();
      constexpr int kPoll = 8;  // slots per lane polled with all loads in flight
      if (G <= 32 * kPoll) {
        unsigned pend = 0u;
#pragma unroll
        for (int i = 0; i < kPoll; ++i)
          if (lane + 32 * i < G) pend |= 1u << i;
        while (pend) {
          uint64_t v[kPoll];
#pragma unroll
          for (int i = 0; i < kPoll; ++i)
            v[i] = (pend >> i) & 1u ? ld_relaxed_u64(slot + lane + 32 * i) : 0ull;
#pragma unroll
          for (int i = 0; i < kPoll; ++i)
            if (((pend >> i) & 1u) && (v[i] & (1ull << 63)) == want) {
              kk = umax64(kk, v[i] & ~(1ull << 63));
              pend &= ~(1u << i);
            }
          if (pend && globaltimer_ns() - t0 > (uint64_t)c.spin_limit_ns) {
            abort = 1;
            break;
          }
        }
      } else {
        for (int j = lane; j < G && !abort; j += 32) {
          uint64_t v = ld_relaxed_u64(slot + j);
          while ((v & (1ull << 63)) != want) {
            if (globaltimer_ns() - t0 > (uint64_t)c.spin_limit_ns) {
              abort = 1;
              break;
            }
            v = ld_relaxed_u64(slot + j);
          }
          kk = umax64(kk, v & ~(1ull << 63));
        }
      }
      abort = __any_sync(0xffffffffu, abort);
      kk = warp_max_key(kk);
      if (lane == 0) {
        *s_best = abort ? 0ull : kk;
        if (abort) {
          atomicOr(&d.st->status, ST_TIMEOUT);
          d.st->timeout_where = ((int64_t)t << 32) | (int64_t)k;
          *s_abort = 1;
        }
      }
    }
  }
  __syncthreads();
  return *s_best;
}

// One tile group member: CTA `rank` of the G serving tile t.
template <int SYNC, bool RES>
__device__ __forceinline__ void minor_body(const PlanDev& d, const MinorCfg& c, int parity,
                                           int t, int rank) {
  extern __shared__ __align__(16) float sR[];
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_part[2];
  __shared__ uint64_t s_best;
  __shared__ int s_abort;

  const int G = c.G;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int H = rc.y1 - rc.y0;
  const int ya = rc.y0 + (int)(((int64_t)rank * H) / G);
  const int yb = rc.y0 + (int)(((int64_t)(rank + 1) * H) / G);
  const int W = rc.x1 - rc.x0;

  // Status bits only change inside grid-synchronised launches (timeouts), so
  // every CTA of a cluster reads the same value here.
  if (*(volatile int32_t*)&d.st->status != 0) return;

  uint64_t key = d.peak[parity * d.T + t];
  const int64_t budget = d.budget[t];
  const int64_t kmax = (d.K > 0 && (int64_t)d.K < budget) ? (int64_t)d.K : budget;
  const float level = d.trigger > 0.f ? *(volatile float*)&d.st->level : 0.f;
  const uint32_t seq0 = d.gbar[t];  // the tile's exchanges so far in this run
  if (threadIdx.x == 0) {
    s_abort = 0;
    // the feedback of this round accumulates the tile's next peak here
    if (rank == 0) d.peak[(parity ^ 1) * d.T + t] = 0ull;
  }

  if (RES) {
    const int n = (yb - ya) * W;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int r = i / W, cc = i - r * W;
      sR[i] = d.R[(int64_t)(ya + r) * d.nx + rc.x0 + cc];
    }
  }
  __syncthreads();

  int64_t k = 0;
  while (k < kmax && key != 0ull) {
    const float v = key_value(key);
    if (!(fabsf(v) > d.thr) || !(fabsf(v) > level)) break;  // threshold, flux trigger
    const int idx = key_index(key);
    const float f = __fmul_rn(d.gain, v);  // first equation
    const int py = idx / d.nx, px = idx - py * d.nx;
    if (rank == 0 && threadIdx.x == 0) {
      clean_component cc;
      cc.y = py;
      cc.x = px;
      cc.flux = f;
      cc.tile = t;
      d.rcomps[(int64_t)t * d.cap_round + k] = cc;
      d.model[idx] = __fadd_rn(d.model[idx], f);
    }

    float best_a = -1.f, best_v = 0.f;
    int best_i = 0x7fffffff;
    subtract_pass<RES>(d, sR, ya, yb, rc.x0, rc.x1, f, py, px, best_a, best_i, best_v);
    uint64_t mine = (best_a >= 0.f) ? make_key(best_v, best_i) : 0ull;
    mine = block_max_key(mine, s_warp);

    key = exchange_keys<SYNC>(d, c, t, rank, k, seq0, mine, s_part, &s_best, &s_abort);
    if (s_abort) break;
    ++k;
  }

  // No CTA may leave while a peer can still read its shared memory.
  if (SYNC == CLEAN_SYNC_CLUSTER) cluster_sync_all();

  if (RES) {
    __syncthreads();
    const int n = (yb - ya) * W;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int r = i / W, cc = i - r * W;
      d.R[(int64_t)(ya + r) * d.nx + rc.x0 + cc] = sR[i];
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    d.rcount[t] = (int32_t)k;
    d.budget[t] = budget - k;
    d.gbar[t] = seq0 + (uint32_t)k;
  }
}

template <int SYNC, bool RES>
__global__ void __launch_bounds__(kThreads, 1)
    minor_kernel(PlanDev d, MinorCfg c, int parity) {
  const int t = blockIdx.x / c.G;
  const int rank = (SYNC == CLEAN_SYNC_CLUSTER) ? (int)cluster_rank() : (int)(blockIdx.x % c.G);
  minor_body<SYNC, RES>(d, c, parity, t, rank);
}

// Batched launch: one CTA per (image, tile) item, each image's plan state in
// `plans`.  Tiles are independent within a round, so no CTA waits on another.
template <int SYNC, bool RES>
__global__ void __launch_bounds__(kThreads, 1)
    minor_batch_kernel(const PlanDev* __restrict__ plans, const BatchItem* __restrict__ items,
                       MinorCfg c, int round) {
  const BatchItem it = items[blockIdx.x / c.G];
  const PlanDev d = plans[it.image];
  const int rank = (SYNC == CLEAN_SYNC_CLUSTER) ? (int)cluster_rank() : 0;
  minor_body<SYNC, RES>(d, c, (round - d.round0) & 1, it.tile, rank);
}


// ---------------------------------------------------------------------------
// TMA pipeline variant (same arithmetic, same results).  The CTA's rows are
// cut into chunks of chunk_h rows x chunk_w columns.  A producer warp loads,
// per chunk, one 2-D TMA box of the residual (unless the rows are resident in
// shared memory) and one box of the PSF window, each box_w x chunk_h floats
// at an x rounded down to 4 floats, into a ring of mbarrier-guarded stages;
// 15 consumer warps apply the subtraction from shared memory, write the
// residual (to global memory with 16-byte stores, or to the resident slab)
// and track the peak.  Each mbarrier wait is bounded; a CTA whose wait
// expires stops working but keeps joining the group exchange, so every CTA
// of a cluster executes the same barriers.
// ---------------------------------------------------------------------------
// 15 consumer warps + the producer: 4 warps per scheduler, so up to 128
// registers a thread
constexpr int kPipeConsumers = 480;
constexpr int kPipeThreads = kPipeConsumers + 32;
constexpr int kPipeMaxStages = 8;

// (r0, r1) - f * (p0, p1), each lane a rounded multiply then a rounded
// subtract.  Scalar on purpose: ptxas contracts a packed mul.rn.f32x2
// followed by sub.rn.f32x2 into one fused multiply-add (a single rounding),
// even with explicit .rn and --fmad=false, which would change the results;
// the scalar __fmul_rn / __fsub_rn pair is never contracted.
__device__ __forceinline__ void fms2(float& r0, float& r1, float p0, float p1, float f) {
  r0 = __fsub_rn(r0, __fmul_rn(f, p0));
  r1 = __fsub_rn(r1, __fmul_rn(f, p1));
}

__device__ __forceinline__ bool pipe_wait(uint64_t* bar, uint32_t parity, uint64_t limit,
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

// Keeps the larger |r| (ties: the lower index).
__device__ __forceinline__ void take_peak(float r, int idx, float& best_a, int& best_i,
                                          float& best_v) {
  const float a = fabsf(r);
  if (a > best_a || (a == best_a && idx < best_i)) {
    best_a = a;
    best_i = idx;
    best_v = r;
  }
}

// Vector path over one chunk.  The chunk's rows form slabs of 32 / LPR rows
// (LPR = 1 << lpr_log2 lanes per row, 4 pixels per lane, so a slab row is
// CW = 4 LPR pixels wide); slab s goes to consumer warp (s + rot) mod 15,
// continuing the round-robin of the previous chunk so the warps stay
// balanced across a ragged last slab.  A warp step loads the residual and
// PSF vectors of four slabs (two or one for a chunk's tail) before any
// arithmetic, then subtracts and stores (global or the resident slab).  The
// step has no branches: rows past the chunk are read from a valid staged row
// and masked.  The peak is kept
// per 4-pixel group: the largest group maximum |R|, ties to the lower group
// base index.  Groups are aligned runs of 4 pixels of one row, so the lowest
// index holding the largest |R| lies in that group; resolve_group() finds it
// once per iteration.
constexpr int kSlabUnroll = 4;

// The running best 4-pixel group: a group replaces it only if its maximum
// |R| is larger, or equal with a lower base index.  Past the first few groups
// a new maximum is rare, so the common case is one comparison (m >= best_a)
// that skips the update.
__device__ __forceinline__ void keep_group(bool valid, float m, int base, const float4& r,
                                           float& best_a, int& best_base, float4& best_r) {
  if (valid && m >= best_a) {
    if (m > best_a || base < best_base) {
      best_a = m;
      best_base = base;
      best_r = r;
    }
  }
}

// One thread's four groups of a chunk (rows w, w + 15, w + 30, w + 45, so in
// increasing index order) into the running best: the chunk's best group is
// found as a two-level tournament in which a later group wins only with a
// strictly larger maximum (the lowest index among equal maxima), then merged
// once by keep_group.  Same choice as four keep_group calls, with a dependency
// chain of three steps instead of four.  m < 0 marks a group that takes no
// part.
__device__ __forceinline__ void keep_chunk4(const float (&m)[4], const float4 (&r)[4], int base0,
                                            int row_step, float& best_a, int& best_base,
                                            float4& best_r) {
  const bool s01 = m[1] > m[0], s23 = m[3] > m[2];
  const float m01 = s01 ? m[1] : m[0], m23 = s23 ? m[3] : m[2];
  const float4 r01 = s01 ? r[1] : r[0], r23 = s23 ? r[3] : r[2];
  const int u01 = s01 ? 1 : 0, u23 = s23 ? 3 : 2;
  const bool s = m23 > m01;
  const float mc = s ? m23 : m01;
  keep_group(mc >= 0.f, mc, base0 + (s ? u23 : u01) * row_step, s ? r23 : r01, best_a, best_base,
             best_r);
}

// U slabs s, s + 15, ... of one chunk for this lane (rows past r1 masked).
template <bool RES, int OFF, int U>
__device__ __forceinline__ void slab_step(const PlanDev& d, float* sRes, int WR, int ya,
                                          const float* stgR, const float* stgP, int BW, int r0,
                                          int r1, int x, int x0, int g, int rps, int sub, int s,
                                          float f, float& best_a, int& best_base,
                                          float4& best_r) {
  constexpr int kWarps = kPipeConsumers / 32;
  float4 rv[U], pa[U], pb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int y = r0 + (s + u * kWarps) * rps + sub;
    const int ly = y < r1 ? y - r0 : 0;  // masked rows read staged row 0
    const float4* rowP4 = reinterpret_cast<const float4*>(stgP + ly * BW);
    pa[u] = rowP4[g];
    if (OFF != 0) pb[u] = rowP4[g + 1];
    rv[u] = RES ? *reinterpret_cast<const float4*>(sRes + (r0 + ly - ya) * WR + (x - x0))
                : reinterpret_cast<const float4*>(stgR + ly * BW)[g];
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int y = r0 + (s + u * kWarps) * rps + sub;
    const bool valid = y < r1;
    const float4 a = pa[u];
    float4 p;
    if (OFF == 0) {
      p = a;
    } else {
      const float4 b = pb[u];
      p = OFF == 1 ? make_float4(a.y, a.z, a.w, b.x)
                   : OFF == 2 ? make_float4(a.z, a.w, b.x, b.y) : make_float4(a.w, b.x, b.y, b.z);
    }
    float4 r = rv[u];
    fms2(r.x, r.y, p.x, p.y, f);
    fms2(r.z, r.w, p.z, p.w, f);
    if (valid) {
      if (RES)
        *reinterpret_cast<float4*>(sRes + (y - ya) * WR + (x - x0)) = r;
      else
        *reinterpret_cast<float4*>(d.R + (int64_t)y * d.nx + x) = r;
    }
    const float m = fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w)));
    keep_group(valid, m, y * d.nx + x, r, best_a, best_base, best_r);
  }
}

template <bool RES, int OFF>
__device__ __forceinline__ void chunk_slabs(const PlanDev& d, float* sRes, int WR, int ya,
                                            const float* stgR, const float* stgP, int BW,
                                            int r0, int r1, int c0, int c1, int x0, float f,
                                            int lpr_log2, int s_first, float& best_a,
                                            int& best_base, float4& best_r) {
  constexpr int kWarps = kPipeConsumers / 32;
  const int lane = threadIdx.x & 31;
  const int g = lane & ((1 << lpr_log2) - 1);
  const int rps = 32 >> lpr_log2;  // rows per slab
  const int sub = lane >> lpr_log2;
  const int x = c0 + 4 * g;
  if (x >= c1) return;
  const int nslabs = (r1 - r0 + rps - 1) / rps;
  // warp-uniform step sizes: whole 4-slab steps, then at most one 2-slab and
  // one 1-slab step, so a chunk whose slab count is not a multiple of 60
  // wastes no work on absent slabs
  int s = s_first;
  for (; s + (kSlabUnroll - 1) * kWarps < nslabs; s += kSlabUnroll * kWarps)
    slab_step<RES, OFF, kSlabUnroll>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, x, x0, g, rps,
                                     sub, s, f, best_a, best_base, best_r);
  if (s + kWarps < nslabs) {
    slab_step<RES, OFF, 2>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, x, x0, g, rps, sub, s, f,
                           best_a, best_base, best_r);
    s += 2 * kWarps;
  }
  if (s < nslabs)
    slab_step<RES, OFF, 1>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, x, x0, g, rps, sub, s, f,
                           best_a, best_base, best_r);
}

// The pixel of the best 4-pixel group that holds |R| = best_a first (lowest
// index), and its signed value, from the group's values kept in registers.
__device__ __forceinline__ void resolve_group(float best_a, int base, const float4& r,
                                              int& best_i, float& best_v) {
  const int k4 = fabsf(r.x) == best_a ? 0 : fabsf(r.y) == best_a ? 1 : fabsf(r.z) == best_a ? 2 : 3;
  best_i = base + k4;
  best_v = k4 == 0 ? r.x : k4 == 1 ? r.y : k4 == 2 ? r.z : r.w;
}

// One chunk whose residual lives in tensor memory (a full CW = 128, 60-row
// chunk: warp w owns rows w, w + 15, w + 30, w + 45, lane l the pixels
// 4l..4l+3 of each, 16 TMEM columns from taddr).  On a launch's first
// iteration the residual comes from the staged box instead.  Same arithmetic
// and peak tracking as slab_step.
template <int OFF>
__device__ __forceinline__ void tmem_chunk(const PlanDev& d, uint32_t taddr, bool from_box,
                                           const float* stgR, const float* stgP, int BW,
                                           int r0, int c0, float f, float& best_a,
                                           int& best_base, float4& best_r) {
  constexpr int kWarps = kPipeConsumers / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 rv[kSlabUnroll], pa[kSlabUnroll], pb[kSlabUnroll];
  float m[kSlabUnroll];
#pragma unroll
  for (int u = 0; u < kSlabUnroll; ++u) {
    const float4* rowP4 = reinterpret_cast<const float4*>(stgP + (warp + u * kWarps) * BW);
    pa[u] = rowP4[lane];
    if (OFF != 0) pb[u] = rowP4[lane + 1];
  }
  if (from_box) {
#pragma unroll
    for (int u = 0; u < kSlabUnroll; ++u)
      rv[u] = reinterpret_cast<const float4*>(stgR + (warp + u * kWarps) * BW)[lane];
  } else {
    __syncwarp();
    ptx::tmem_ld16(taddr, rv);
  }
#pragma unroll
  for (int u = 0; u < kSlabUnroll; ++u) {
    const float4 a = pa[u];
    float4 p;
    if (OFF == 0) {
      p = a;
    } else {
      const float4 b = pb[u];
      p = OFF == 1 ? make_float4(a.y, a.z, a.w, b.x)
                   : OFF == 2 ? make_float4(a.z, a.w, b.x, b.y) : make_float4(a.w, b.x, b.y, b.z);
    }
    float4 r = rv[u];
    fms2(r.x, r.y, p.x, p.y, f);
    fms2(r.z, r.w, p.z, p.w, f);
    rv[u] = r;
    m[u] = fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w)));
  }
  keep_chunk4(m, rv, (r0 + warp) * d.nx + c0 + 4 * lane, kWarps * d.nx, best_a, best_base,
              best_r);
  __syncwarp();
  ptx::tmem_st16(taddr, rv);
}

template <int N>
struct IntTag {
  static constexpr int value = N;
};

// One streamed chunk of 4 lanes' pixels a row and at most 60 rows (CW = 128):
// warp w owns rows w, w + 15, w + 30, w + 45 as in tmem_chunk, reads the
// residual from the staged box and writes it back to global memory.  Rows
// past the chunk (nrows) and lanes past its right edge (c1) read a valid
// staged value and neither store nor take part in the peak.  Same
// arithmetic and peak tracking as slab_step, with the row addresses formed
// once a chunk.
template <int OFF>
__device__ __forceinline__ void stream_chunk(const PlanDev& d, const float* stgR,
                                             const float* stgP, int BW, int r0, int nrows,
                                             int c0, int c1, float f, float& best_a,
                                             int& best_base, float4& best_r) {
  constexpr int kWarps = kPipeConsumers / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool lane_in = c0 + 4 * lane < c1;
  float4 rv[kSlabUnroll], pa[kSlabUnroll], pb[kSlabUnroll];
  float m[kSlabUnroll];
#pragma unroll
  for (int u = 0; u < kSlabUnroll; ++u) {
    const int row = warp + u * kWarps;
    const int ly = row < nrows ? row : 0;
    const float4* rowP4 = reinterpret_cast<const float4*>(stgP + ly * BW);
    pa[u] = rowP4[lane];
    if (OFF != 0) pb[u] = rowP4[lane + 1];
    rv[u] = reinterpret_cast<const float4*>(stgR + ly * BW)[lane];
  }
  float* out = d.R + (int64_t)(r0 + warp) * d.nx + c0 + 4 * lane;
#pragma unroll
  for (int u = 0; u < kSlabUnroll; ++u) {
    const bool valid = lane_in && warp + u * kWarps < nrows;
    const float4 a = pa[u];
    float4 p;
    if (OFF == 0) {
      p = a;
    } else {
      const float4 b = pb[u];
      p = OFF == 1 ? make_float4(a.y, a.z, a.w, b.x)
                   : OFF == 2 ? make_float4(a.z, a.w, b.x, b.y) : make_float4(a.w, b.x, b.y, b.z);
    }
    float4 r = rv[u];
    fms2(r.x, r.y, p.x, p.y, f);
    fms2(r.z, r.w, p.z, p.w, f);
    if (valid) *reinterpret_cast<float4*>(out + (int64_t)u * kWarps * d.nx) = r;
    rv[u] = r;
    m[u] = valid ? fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w))) : -1.f;
  }
  keep_chunk4(m, rv, (r0 + warp) * d.nx + c0 + 4 * lane, kWarps * d.nx, best_a, best_base,
              best_r);
}

// CTA `rank` of the group serving tile t; r_map and p_map describe the
// residual and PSF boxes (r_map unused when the rows are resident).
//
// TM: the CTA's first (up to 8) full chunks keep their residual in tensor
// memory for the whole launch (16 columns per chunk and consumer warp; warps
// w, w + 4, w + 8, w + 12 share lane quarter w mod 4 and take columns
// 128 (w / 4) ..), so those chunks stream only their PSF box: a third fewer
// bytes per iteration at 4096^2.  Used when every window of the CTA's rows is
// inside the PSF array (the vector path applies to every iteration) and the
// CTA owns its SM (shared memory above half of it), so the 512-column
// allocation never waits.  The residual is read from the staged box in the
// launch's first iteration and written back to global memory at the end.
constexpr int kTmemCols = 512;
constexpr int kTmemChunks = 8;       // 4 warps per lane quarter x 8 chunks x 16 columns
constexpr int kTmemChunkRows = 60;   // 15 warps x 4 slabs of one row

// PERSIST: one unit of a persistent launch (the caller checks the plan's
// status uniformly before; at the end the barriers are invalidated so the
// next unit can initialise the same shared memory again).
template <int SYNC, bool RES, bool TM = false, bool PERSIST = false>
__device__ __forceinline__ void minor_pipe_body(const PlanDev& d, const MinorCfg& c, int parity,
                                                const CUtensorMap* r_map,
                                                const CUtensorMap* p_map, int t, int rank) {
  extern __shared__ __align__(128) float smem[];
  float* sRes = smem;                       // resident slab (RES), row stride WR
  float* sStage = smem + c.res_floats;      // ring of stages
  __shared__ __align__(8) uint64_t full_bar[kPipeMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kPipeMaxStages];
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_part[2];
  __shared__ uint64_t s_best;
  __shared__ int s_abort;    // grid-barrier timeout: leave the loop
  __shared__ int s_dead;     // mbarrier timeout: stop working, keep exchanging
  __shared__ uint32_t s_tmem;  // TMEM base address (TM)

  const int G = c.G;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int H = rc.y1 - rc.y0;
  const int ya = rc.y0 + (int)(((int64_t)rank * H) / G);
  const int yb = rc.y0 + (int)(((int64_t)(rank + 1) * H) / G);
  const int x0 = rc.x0, x1 = rc.x1, W = x1 - x0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = warp == kPipeConsumers / 32;
  const int S = c.stages, BH = c.chunk_h, CW = c.chunk_w, BW = c.box_w;
  const int box_floats = (BW * BH + 31) & ~31;  // each box starts 128-byte aligned
  const int stage_floats = (RES ? 1 : 2) * box_floats;
  const uint32_t stage_bytes = (uint32_t)((RES ? 1 : 2) * BW * BH) * 4u;  // bytes the boxes land
  const uint32_t p_box_bytes = (uint32_t)(BW * BH) * 4u;
  const int nrb = (yb - ya + BH - 1) / BH, ncb = (W + CW - 1) / CW;
  const int nch = nrb * ncb;                // chunks per iteration
  const uint64_t limit = (uint64_t)c.spin_limit_ns;
  const int WR = (W + 3) & ~3;              // resident slab row stride

  if (!PERSIST && *(volatile int32_t*)&d.st->status != 0) return;  // uniform, see minor_kernel

  // consumer geometry within a chunk: row slabs of 4-pixel groups (vector
  // path, CW = 32, 64 or 128) or single pixels, threads per row a power of two
  const bool vec_cols = (x0 % 4) == 0 && (W % 4) == 0 && (CW == 32 || CW == 64 || CW == 128);

  // tensor-memory chunks: the leading full chunks, when every peak of the
  // tile puts this CTA's whole window inside the PSF array
  int n_tm = 0;
  if (TM && c.tmem && vec_cols && CW == 128 && BH == kTmemChunkRows &&
      ya + d.cy - (rc.y1 - 1) >= 0 && yb - 1 + d.cy - rc.y0 < d.pny &&
      x0 + d.cx - (x1 - 1) >= 0 && x1 - 1 + d.cx - x0 < d.pnx) {
    while (n_tm < kTmemChunks && n_tm < nch) {
      const int rb = n_tm / ncb, cb = n_tm - rb * ncb;
      if (ya + (rb + 1) * BH > yb || x0 + (cb + 1) * CW > x1) break;
      ++n_tm;
    }
  }
  const bool tm_on = TM && n_tm > 0;
  if (tm_on && warp == 0) {
    ptx::tmem_alloc(&s_tmem, kTmemCols);
    // a persistent CTA allocates again for its next unit: it keeps the permit
    // (it owns its SM, so no other CTA waits for the columns)
    if (!PERSIST) ptx::tmem_relinquish();
    ptx::tmem_fence_before_sync();
  }

  uint64_t key = d.peak[parity * d.T + t];
  const int64_t budget = d.budget[t];
  const int64_t kmax = (d.K > 0 && (int64_t)d.K < budget) ? (int64_t)d.K : budget;
  const float level = d.trigger > 0.f ? *(volatile float*)&d.st->level : 0.f;
  const uint32_t seq0 = d.gbar[t];  // the tile's exchanges so far in this run
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_dead = 0;
    if (rank == 0) d.peak[(parity ^ 1) * d.T + t] = 0ull;
    for (int i = 0; i < S; ++i) {
      ptx::mbar_init(&full_bar[i], 1);
      ptx::mbar_init(&empty_bar[i], kPipeConsumers / 32);
    }
    ptx::fence_barrier_init();
  }
  if (producer && lane == 0) {
    if (!RES) ptx::prefetch_tensormap(r_map);
    ptx::prefetch_tensormap(p_map);
  }
  if (RES) {
    const int n = (yb - ya) * W;
    for (int i = threadIdx.x; i < n; i += kPipeThreads) {
      const int r = i / W, cc = i - r * W;
      sRes[r * WR + cc] = d.R[(int64_t)(ya + r) * d.nx + x0 + cc];
    }
  }
  __syncthreads();
  if (tm_on) ptx::tmem_fence_after_sync();
  // this warp's lane quarter and first column (the producer warp's is unused)
  const uint32_t tm_base =
      tm_on ? s_tmem + (((uint32_t)(warp & 3) * 32u) << 16) + (uint32_t)(warp >> 2) * 128u : 0u;
  bool tm_filled = false;  // tensor memory holds this launch's residual

  const int lpr_log2 = CW == 128 ? 5 : CW == 64 ? 4 : 3;
  const int slabs = (BH + (32 >> lpr_log2) - 1) / (32 >> lpr_log2);  // per full chunk
  int tpr = 1;
  while (tpr < CW && tpr < kPipeConsumers) tpr <<= 1;
  const int rpp = kPipeConsumers / tpr;
  const int crow = threadIdx.x / tpr, ccol = threadIdx.x % tpr;

  // ring state, advanced chunk by chunk (no division in the loop): the
  // producer's next stage and phase, the consumers' likewise, and the slab
  // rotation of the consumers
  constexpr int kW = kPipeConsumers / 32;
  const int rot_step = slabs % kW;
  int p_st = 0, c_st = 0, rot = 0;
  uint32_t p_ph = 0, c_ph = 0;
  int64_t jnext = 0;   // producer: chunks issued so far
  int64_t k = 0;
  while (k < kmax && key != 0ull) {
    const float v = key_value(key);
    if (!(fabsf(v) > d.thr) || !(fabsf(v) > level)) break;  // threshold, flux trigger
    const int idx = key_index(key);
    const float f = __fmul_rn(d.gain, v);  // first equation
    const int py = idx / d.nx, px = idx - py * d.nx;
    const int dy = d.cy - py, dx = d.cx - px;  // PSF index = pixel + (dy, dx)
    // whole window inside the PSF array and 16-byte-aligned columns: the
    // vector path with no per-pixel range checks
    const bool fast = vec_cols && ya + dy >= 0 && yb - 1 + dy < d.pny && x0 + dx >= 0 &&
                      x1 - 1 + dx < d.pnx;
    if (rank == 0 && threadIdx.x == 0) {
      clean_component cc;
      cc.y = py;
      cc.x = px;
      cc.flux = f;
      cc.tile = t;
      d.rcomps[(int64_t)t * d.cap_round + k] = cc;
      d.model[idx] = __fadd_rn(d.model[idx], f);
    }

    float best_a = -1.f, best_v = 0.f;
    int best_i = 0x7fffffff;
    if (producer) {
      if (lane == 0) {
        int rb = 0, cb = 0;
        for (int ch = 0; ch < nch && !*(volatile int*)&s_dead; ++ch) {
          if (jnext >= S && !pipe_wait(&empty_bar[p_st], p_ph ^ 1u, limit, &s_dead,
                                       &d.st->status))
            break;
          const int r0 = ya + rb * BH, c0 = x0 + cb * CW;
          float* stg = sStage + (size_t)p_st * stage_floats;
          // a tensor-memory chunk needs its residual box only in iteration 0
          const bool r_box = !RES && !(TM && ch < n_tm && k > 0);
          ptx::mbar_arrive_expect_tx(&full_bar[p_st], r_box ? stage_bytes : p_box_bytes);
          if (r_box) ptx::tma_load_2d(stg, r_map, c0 & ~3, r0, &full_bar[p_st]);
          ptx::tma_load_2d(stg + (RES ? 0 : box_floats), p_map, (c0 + dx) & ~3, r0 + dy,
                           &full_bar[p_st]);
          ++jnext;
          if (++p_st == S) {
            p_st = 0;
            p_ph ^= 1u;
          }
          if (++cb == ncb) {
            cb = 0;
            ++rb;
          }
        }
      }
    } else {
      int best_base = 0x7fffffff;
      float4 best_r = make_float4(0.f, 0.f, 0.f, 0.f);
      int rb = 0, cb = 0;
      // the previous iteration's tensor-memory stores land before this
      // iteration reads them back
      if (tm_on && k > 0) {
        __syncwarp();
        ptx::tmem_wait_st();
      }
      // streamed 128-wide chunks with the window inside the PSF: the pass is
      // specialised once on the PSF realignment, which every chunk shares (as
      // in the tile-pair body)
      auto fast_pass = [&](auto off) {
        constexpr int OFF = decltype(off)::value;
        int rb = 0, cb = 0;
        for (int ch = 0; ch < nch; ++ch) {
          const int st = c_st;
          bool ok = pipe_wait(&full_bar[st], c_ph, limit, &s_dead, &d.st->status);
          if (TM) ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          if (++c_st == S) {
            c_st = 0;
            c_ph ^= 1u;
          }
          const int r0 = ya + rb * BH, r1 = min(yb, r0 + BH);
          const int c0 = x0 + cb * CW, c1 = min(x1, c0 + CW);
          if (++cb == ncb) {
            cb = 0;
            ++rb;
          }
          const float* stgR = sStage + (size_t)st * stage_floats;
          const float* stgP = stgR + box_floats;
          if (TM && ch < n_tm)
            tmem_chunk<OFF>(d, tm_base + (uint32_t)ch * 16u, k == 0, stgR, stgP, BW, r0, c0, f,
                            best_a, best_base, best_r);
          else
            stream_chunk<OFF>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base,
                              best_r);
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&empty_bar[st]);
        }
      };
      const bool lean = !RES && fast && CW == 128 && BH <= kSlabUnroll * kW;
      if (lean) {
        switch ((x0 + dx) & 3) {
          case 0:
            fast_pass(IntTag<0>{});
            break;
          case 1:
            fast_pass(IntTag<1>{});
            break;
          case 2:
            fast_pass(IntTag<2>{});
            break;
          default:
            fast_pass(IntTag<3>{});
            break;
        }
      }
      for (int ch = 0; ch < nch && !lean; ++ch) {
        const int st = c_st;
        bool ok = !*(volatile int*)&s_dead &&
                  pipe_wait(&full_bar[st], c_ph, limit, &s_dead, &d.st->status);
        // tensor-memory accesses are warp-wide: the whole warp stops or none
        if (TM) ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        if (++c_st == S) {
          c_st = 0;
          c_ph ^= 1u;
        }
        const int r0 = ya + rb * BH, r1 = min(yb, r0 + BH);
        const int c0 = x0 + cb * CW, c1 = min(x1, c0 + CW);
        if (++cb == ncb) {
          cb = 0;
          ++rb;
        }
        const float* stg = sStage + (size_t)st * stage_floats;
        const float* stgR = stg;                            // streamed residual box
        const float* stgP = stg + (RES ? 0 : box_floats);   // PSF box
        const int offR = c0 - (c0 & ~3), offP = (c0 + dx) - ((c0 + dx) & ~3);
        if (TM && fast && ch < n_tm) {
          // full chunk, rot == 0 (60 slabs a chunk): warp w owns slabs w + 15u
          const uint32_t ta = tm_base + (uint32_t)ch * 16u;
          const bool from_box = k == 0;
          switch (offP) {
            case 0:
              tmem_chunk<0>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base,
                            best_r);
              break;
            case 1:
              tmem_chunk<1>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base,
                            best_r);
              break;
            case 2:
              tmem_chunk<2>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base,
                            best_r);
              break;
            default:
              tmem_chunk<3>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base,
                            best_r);
              break;
          }
        } else if (!RES && fast && CW == 128 && BH <= kSlabUnroll * kW) {
          switch (offP) {
            case 0:
              stream_chunk<0>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
              break;
            case 1:
              stream_chunk<1>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
              break;
            case 2:
              stream_chunk<2>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
              break;
            default:
              stream_chunk<3>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
              break;
          }
        } else if (fast) {
          // continue the slab round-robin where the previous chunk ended
          const int s_first = warp >= rot ? warp - rot : warp + kW - rot;
          switch (offP) {
            case 0:
              chunk_slabs<RES, 0>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, c0, c1, x0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
              break;
            case 1:
              chunk_slabs<RES, 1>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, c0, c1, x0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
              break;
            case 2:
              chunk_slabs<RES, 2>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, c0, c1, x0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
              break;
            default:
              chunk_slabs<RES, 3>(d, sRes, WR, ya, stgR, stgP, BW, r0, r1, c0, c1, x0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
              break;
          }
        } else {
          for (int y = r0 + crow; crow < rpp && y < r1; y += rpp) {
            const bool yin = (unsigned)(y + dy) < (unsigned)d.pny;
            const float* rowP = stgP + (y - r0) * BW + offP - c0;  // index by x
            const float* rowR = stgR + (y - r0) * BW + offR - c0;  // index by x (streamed)
            float* rowRes = sRes + (y - ya) * WR - x0;             // index by x (resident)
            for (int x = c0 + ccol; x < c1; x += tpr) {
              float r = RES ? rowRes[x] : rowR[x];
              if (yin && (unsigned)(x + dx) < (unsigned)d.pnx)
                r = __fsub_rn(r, __fmul_rn(f, rowP[x]));
              if (RES)
                rowRes[x] = r;
              else
                d.R[(int64_t)y * d.nx + x] = r;
              take_peak(r, y * d.nx + x, best_a, best_i, best_v);
            }
          }
        }
        rot += rot_step;
        if (rot >= kW) rot -= kW;
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&empty_bar[st]);
      }
      if (fast && best_a >= 0.f) resolve_group(best_a, best_base, best_r, best_i, best_v);
      tm_filled = tm_on && !*(volatile int*)&s_dead;
      // residual rows written through the generic proxy are read back by TMA
      // (async proxy) in the next iteration
      if (!RES) asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    uint64_t mine = (best_a >= 0.f) ? make_key(best_v, best_i) : 0ull;
    mine = block_max_key(mine, s_warp);
    key = exchange_keys<SYNC>(d, c, t, rank, k, seq0, mine, s_part, &s_best, &s_abort);
    if (s_abort) break;
    ++k;
  }

  if (tm_on) {
    // tensor-memory chunks back to global memory, then free the columns
    if (!producer) {
      __syncwarp();
      ptx::tmem_wait_st();
      const bool wb = __shfl_sync(0xffffffffu, (int)(tm_filled && !*(volatile int*)&s_dead), 0);
      if (wb) {
        for (int ch = 0; ch < n_tm; ++ch) {
          const int rb = ch / ncb, cb = ch - rb * ncb;
          const int r0 = ya + rb * BH, c0 = x0 + cb * CW;
          float4 v[kSlabUnroll];
          __syncwarp();
          ptx::tmem_ld16(tm_base + (uint32_t)ch * 16u, v);
#pragma unroll
          for (int u = 0; u < kSlabUnroll; ++u)
            *reinterpret_cast<float4*>(d.R + (int64_t)(r0 + warp + u * (kW)) * d.nx + c0 +
                                       4 * lane) = v[u];
        }
      }
    }
    ptx::tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      ptx::tmem_fence_after_sync();
      __syncwarp();
      ptx::tmem_dealloc(s_tmem, kTmemCols);
    }
  }
  if (SYNC == CLEAN_SYNC_CLUSTER) cluster_sync_all();
  if (producer && lane == 0 && s_dead) {
    // after an expired wait: let this CTA's own copies in flight land
    for (int64_t j = max((int64_t)0, jnext - S); j < jnext; ++j) {
      const uint64_t t0 = ptx::globaltimer_ns();
      while (!ptx::mbar_try_wait(&full_bar[j % S], (uint32_t)(j / S) & 1u))
        if (ptx::globaltimer_ns() - t0 > limit) break;
    }
  }
  if (RES) {
    __syncthreads();
    const int n = (yb - ya) * W;
    for (int i = threadIdx.x; i < n; i += kPipeThreads) {
      const int r = i / W, cc = i - r * W;
      d.R[(int64_t)(ya + r) * d.nx + x0 + cc] = sRes[r * WR + cc];
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    d.rcount[t] = (int32_t)k;
    d.budget[t] = budget - k;
    d.gbar[t] = seq0 + (uint32_t)k;
  }
  if (PERSIST) {
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < S; ++i) {
        ptx::mbar_inval(&full_bar[i]);
        ptx::mbar_inval(&empty_bar[i]);
      }
    __syncthreads();
  }
}

template <int SYNC, bool RES, bool TM>
__global__ void __launch_bounds__(kPipeThreads, 1)
    minor_pipe_kernel(PlanDev d, MinorCfg c, int parity,
                      const __grid_constant__ CUtensorMap r_map,
                      const __grid_constant__ CUtensorMap p_map) {
  const int t = blockIdx.x / c.G;
  const int rank = (SYNC == CLEAN_SYNC_CLUSTER) ? (int)cluster_rank() : (int)(blockIdx.x % c.G);
  minor_pipe_body<SYNC, RES, TM>(d, c, parity, &r_map, &p_map, t, rank);
}

// ---------------------------------------------------------------------------
// Tile pairs.  The exchange that ends a tile's iteration (every CTA of the
// group publishes its partial peak, then waits for all of them) and the
// latency of the next iteration's first window leave the SMs idle for a few
// microseconds per iteration.  Two tiles have no dependence on each other
// within a round, so a group of 2G CTAs serves a pair of tiles and
// alternates between them: while the consumer warps subtract the window of
// one tile, the producer warp waits for the other tile's exchange and starts
// loading its next windows.  CTA q of the pair's group owns row band q mod G
// of column half q / G of both tiles (halves split at a whole number of
// 128-pixel chunks), so its chunks keep their full 128 x 60 shape and up to
// 4 chunks of each tile live in tensor memory (columns 64 X + 16 ch of its
// warp's 128).
//
// Step s serves tile X = s mod 2 (steps of a finished tile are skipped on
// both sides alike).  The producer's lane 0 publishes the step's key in
// s_key[n mod 2] (key n; 0: the tile is finished) and arrives on
// key_bar[n mod 2]; the consumers wait there (phase n / 2), process the
// tile's chunks and leave their partial keys in shared memory; the last warp
// to finish posts the CTA's key to the tile's exchange slot with the usual
// phase mark.  The producer warp reads the exchange of the tile's previous
// iteration, which every CTA posted one step earlier, so the wait overlaps
// the other tile's pass.  Exchange g of
// tile t is posted after reading exchange g - 1, so the argument that keeps
// slots from being overwritten early is the single-tile one.  The last
// exchange of a launch is posted and never read; the next launch's count
// continues past it.
//
// Keys n and n + 1 can both be posted before the consumers wait for key n:
// the first key of each tile needs no exchange, and a finished tile's key is
// posted at once.  On one barrier that is two phases, and a parity wait for
// the older one would then test the newer, incomplete phase and never
// return.  Key n + 2 needs the exchange of key n's pass, so with one barrier
// per buffer no barrier runs more than one phase ahead of its waiters.
// ---------------------------------------------------------------------------
struct Piece {
  int t;                 // tile
  int ya, yb, x0, x1;    // this CTA's rows and columns of the tile
  int ncb, nch;          // chunks per row of chunks, chunks per pass
  int n_tm;              // leading full chunks kept in tensor memory (<= 4)
  bool vec;              // 16-byte-aligned columns: the vector path is possible
};

__device__ __forceinline__ Piece pair_piece(const PlanDev& d, int t, int band, int half, int G,
                                            int BH, int CW, bool tm_ok) {
  Piece p;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int H = rc.y1 - rc.y0, W = rc.x1 - rc.x0;
  p.t = t;
  p.ya = rc.y0 + (int)(((int64_t)band * H) / G);
  p.yb = rc.y0 + (int)(((int64_t)(band + 1) * H) / G);
  const int w0 = min(W, ((W / 2) + CW - 1) / CW * CW);
  p.x0 = half == 0 ? rc.x0 : rc.x0 + w0;
  p.x1 = half == 0 ? rc.x0 + w0 : rc.x1;
  const int Wp = p.x1 - p.x0;
  const int nrb = Wp > 0 ? (p.yb - p.ya + BH - 1) / BH : 0;
  p.ncb = (Wp + CW - 1) / CW;
  p.nch = nrb * p.ncb;
  p.vec = (p.x0 % 4) == 0 && (Wp % 4) == 0 && (CW == 32 || CW == 64 || CW == 128);
  p.n_tm = 0;
  if (tm_ok && p.vec && CW == 128 && BH == kTmemChunkRows && p.nch > 0 &&
      p.ya + d.cy - (rc.y1 - 1) >= 0 && p.yb - 1 + d.cy - rc.y0 < d.pny &&
      p.x0 + d.cx - (rc.x1 - 1) >= 0 && p.x1 - 1 + d.cx - rc.x0 < d.pnx) {
    while (p.n_tm < kTmemChunks / 2 && p.n_tm < p.nch) {
      const int rb = p.n_tm / p.ncb, cb = p.n_tm - rb * p.ncb;
      if (p.ya + (rb + 1) * BH > p.yb || p.x0 + (cb + 1) * CW > p.x1) break;
      ++p.n_tm;
    }
  }
  return p;
}

// Exchange g of tile t over the group's G2 slots, read by one whole warp:
// the maximum key once every slot carries exchange g's mark.  *timed_out on
// expiry (then the result is 0).
__device__ __forceinline__ uint64_t pair_poll(const PlanDev& d, const MinorCfg& c, int t, int G2,
                                              uint32_t g, bool* timed_out) {
  const int lane = threadIdx.x & 31;
  const uint64_t* slot = d.gkeys + (int64_t)t * G2 + (int64_t)(g & 1u) * ((int64_t)d.T * G2);
  const uint64_t mark = (uint64_t)((g >> 1) & 1u) << 63;
  const uint64_t want = c.force_timeout ? (mark ^ (1ull << 63)) : mark;
  constexpr int kPoll = 8;  // slots per lane, all loads in flight (G2 <= 256)
  unsigned pend = 0u;
#pragma unroll
  for (int i = 0; i < kPoll; ++i)
    if (lane + 32 * i < G2) pend |= 1u << i;
  uint64_t kk = 0ull;
  int abort = 0;
  const uint64_t t0 = globaltimer_ns();
  while (pend) {
    uint64_t v[kPoll];
#pragma unroll
    for (int i = 0; i < kPoll; ++i)
      v[i] = (pend >> i) & 1u ? ld_relaxed_u64(slot + lane + 32 * i) : 0ull;
#pragma unroll
    for (int i = 0; i < kPoll; ++i)
      if (((pend >> i) & 1u) && (v[i] & (1ull << 63)) == want) {
        kk = umax64(kk, v[i] & ~(1ull << 63));
        pend &= ~(1u << i);
      }
    if (pend && globaltimer_ns() - t0 > (uint64_t)c.spin_limit_ns) {
      abort = 1;
      break;
    }
  }
  abort = __any_sync(0xffffffffu, abort);
  kk = warp_max_key(kk);
  *timed_out = abort != 0;
  return abort ? 0ull : kk;
}

// PERSIST: one unit of the persistent batched launch (as in minor_pipe_body).
template <bool TM, bool PERSIST = false>
__device__ __forceinline__ void minor_pair_body(const PlanDev& d, const MinorCfg& c, int parity,
                                                const CUtensorMap* r_map,
                                                const CUtensorMap* p_map, int pair, int q) {
  extern __shared__ __align__(128) float smem[];
  float* sStage = smem;  // ring of stages (the residual is streamed)
  constexpr int kW = kPipeConsumers / 32;
  __shared__ __align__(8) uint64_t full_bar[kPipeMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kPipeMaxStages];
  __shared__ __align__(8) uint64_t key_bar[2];  // key n: barrier n mod 2, phase n / 2
  __shared__ int s_arrived[2];  // consumer warps done with the pass, per key buffer
  __shared__ uint64_t s_key[2];
  __shared__ uint64_t s_warp[2][kW];
  __shared__ int s_abort;    // an exchange or key wait expired: stop both tiles
  __shared__ int s_dead;     // an mbarrier wait expired: stop working, keep exchanging
  __shared__ uint32_t s_tmem;

  const int G = c.G, G2 = 2 * G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = warp == kW;
  const int S = c.stages, BH = c.chunk_h, CW = c.chunk_w, BW = c.box_w;
  const int box_floats = (BW * BH + 31) & ~31;
  const int stage_floats = 2 * box_floats;
  const uint32_t stage_bytes = (uint32_t)(2 * BW * BH) * 4u;
  const uint32_t p_box_bytes = (uint32_t)(BW * BH) * 4u;
  const uint64_t limit = (uint64_t)c.spin_limit_ns;

  if (!PERSIST && *(volatile int32_t*)&d.st->status != 0) return;  // uniform, see minor_kernel

  // per-tile state in named pairs (selected per step, no local arrays)
  const Piece pc0 = pair_piece(d, 2 * pair, q % G, q / G, G, BH, CW, TM && c.tmem);
  const Piece pc1 = pair_piece(d, 2 * pair + 1, q % G, q / G, G, BH, CW, TM && c.tmem);
  const bool tm_on = TM && (pc0.n_tm > 0 || pc1.n_tm > 0);
  if (tm_on && warp == 0) {
    ptx::tmem_alloc(&s_tmem, kTmemCols);
    if (!PERSIST) ptx::tmem_relinquish();  // a persistent CTA allocates again later
    ptx::tmem_fence_before_sync();
  }

  const uint64_t key00 = d.peak[parity * d.T + pc0.t], key01 = d.peak[parity * d.T + pc1.t];
  const int64_t budget0 = d.budget[pc0.t], budget1 = d.budget[pc1.t];
  const int64_t kmax0 = (d.K > 0 && (int64_t)d.K < budget0) ? (int64_t)d.K : budget0;
  const int64_t kmax1 = (d.K > 0 && (int64_t)d.K < budget1) ? (int64_t)d.K : budget1;
  const uint32_t seq00 = d.gbar[pc0.t], seq01 = d.gbar[pc1.t];
  const float level = d.trigger > 0.f ? *(volatile float*)&d.st->level : 0.f;
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_dead = 0;
    if (q == 0) {
      d.peak[(parity ^ 1) * d.T + pc0.t] = 0ull;
      d.peak[(parity ^ 1) * d.T + pc1.t] = 0ull;
    }
    for (int i = 0; i < S; ++i) {
      ptx::mbar_init(&full_bar[i], 1);
      ptx::mbar_init(&empty_bar[i], kW);
    }
    ptx::mbar_init(&key_bar[0], 1);
    ptx::mbar_init(&key_bar[1], 1);
    s_arrived[0] = 0;
    s_arrived[1] = 0;
    ptx::fence_barrier_init();
  }
  if (producer && lane == 0) {
    ptx::prefetch_tensormap(r_map);
    ptx::prefetch_tensormap(p_map);
  }
  __syncthreads();
  if (tm_on) ptx::tmem_fence_after_sync();
  const uint32_t tm_base =
      tm_on ? s_tmem + (((uint32_t)(warp & 3) * 32u) << 16) + (uint32_t)(warp >> 2) * 128u : 0u;
  bool filled0 = false, filled1 = false;

  const int lpr_log2 = CW == 128 ? 5 : CW == 64 ? 4 : 3;
  const int slabs = (BH + (32 >> lpr_log2) - 1) / (32 >> lpr_log2);
  int tpr = 1;
  while (tpr < CW && tpr < kPipeConsumers) tpr <<= 1;
  const int rpp = kPipeConsumers / tpr;
  const int crow = threadIdx.x / tpr, ccol = threadIdx.x % tpr;
  const int rot_step = slabs % kW;

  int p_st = 0, c_st = 0, rot = 0;
  uint32_t p_ph = 0, c_ph = 0;
  int64_t jnext = 0;
  int64_t kx0 = 0, kx1 = 0;
  bool done0 = false, done1 = false;
  uint32_t n_pub = 0;   // keys published (producer) / taken (consumers)
  uint32_t n_pass = 0;  // consumers: passes, for the partial-key buffer

  for (int s = 0; !(done0 && done1); ++s) {
    const int X = s & 1;
    if (X ? done1 : done0) continue;
    const Piece P = X ? pc1 : pc0;
    const int64_t kX = X ? kx1 : kx0;
    const uint32_t seqX = X ? seq01 : seq00;
    if (producer) {
      // the key of the tile's next iteration: the exchange of its previous
      // iteration, posted by every CTA one step earlier
      // one view of the abort flag for the whole warp (the poll is warp-wide)
      const int ab = __shfl_sync(0xffffffffu, *(volatile int*)&s_abort, 0);
      bool to = false;
      uint64_t key = X ? key01 : key00;
      if (kX > 0 && !ab) key = pair_poll(d, c, P.t, G2, seqX + (uint32_t)(kX - 1), &to);
      bool active = !to && !ab && kX < (X ? kmax1 : kmax0) && key != 0ull;
      if (active) {
        const float v = key_value(key);
        active = fabsf(v) > d.thr && fabsf(v) > level;  // threshold, flux trigger
      }
      if (lane == 0) {
        if (to) {
          atomicOr(&d.st->status, ST_TIMEOUT);
          d.st->timeout_where = ((int64_t)P.t << 32) | (int64_t)kX;
          s_abort = 1;
        }
        s_key[n_pub & 1u] = active ? key : 0ull;
        ptx::mbar_arrive(&key_bar[n_pub & 1u]);
      }
      ++n_pub;
      if (!active) {
        if (X) done1 = true; else done0 = true;
        continue;
      }
      const int idx = key_index(key);
      const float f = __fmul_rn(d.gain, key_value(key));  // first equation
      const int py = idx / d.nx, px = idx - py * d.nx;
      const int dy = d.cy - py, dx = d.cx - px;
      if (lane == 0) {
        if (q == 0) {
          clean_component cc;
          cc.y = py;
          cc.x = px;
          cc.flux = f;
          cc.tile = P.t;
          d.rcomps[(int64_t)P.t * d.cap_round + kX] = cc;
          d.model[idx] = __fadd_rn(d.model[idx], f);
        }
        int rb = 0, cb = 0;
        for (int ch = 0; ch < P.nch && !*(volatile int*)&s_dead; ++ch) {
          if (jnext >= S && !pipe_wait(&empty_bar[p_st], p_ph ^ 1u, limit, &s_dead,
                                       &d.st->status))
            break;
          const int r0 = P.ya + rb * BH, c0 = P.x0 + cb * CW;
          float* stg = sStage + (size_t)p_st * stage_floats;
          // a tensor-memory chunk needs its residual box only in iteration 0
          const bool r_box = !(TM && ch < P.n_tm && kX > 0);
          ptx::mbar_arrive_expect_tx(&full_bar[p_st], r_box ? stage_bytes : p_box_bytes);
          if (r_box) ptx::tma_load_2d(stg, r_map, c0 & ~3, r0, &full_bar[p_st]);
          ptx::tma_load_2d(stg + box_floats, p_map, (c0 + dx) & ~3, r0 + dy, &full_bar[p_st]);
          ++jnext;
          if (++p_st == S) {
            p_st = 0;
            p_ph ^= 1u;
          }
          if (++cb == P.ncb) {
            cb = 0;
            ++rb;
          }
        }
      }
      __syncwarp();
      if (X) ++kx1; else ++kx0;
      continue;
    }

    // ---- consumers ----
    // the producer publishes within its own bounded waits (at most two
    // limits), so this wait gets four
    bool got = pipe_wait(&key_bar[n_pub & 1u], (n_pub >> 1) & 1u, 4 * limit, &s_dead,
                         &d.st->status);
    got = __all_sync(0xffffffffu, got);
    const uint64_t key = got ? s_key[n_pub & 1u] : 0ull;
    ++n_pub;
    if (!got) s_abort = 1;
    if (key == 0ull) {
      if (X || !got) done1 = true;
      if (!X || !got) done0 = true;
      continue;
    }
    const int idx = key_index(key);
    const float f = __fmul_rn(d.gain, key_value(key));
    const int py = idx / d.nx, px = idx - py * d.nx;
    const int dy = d.cy - py, dx = d.cx - px;
    const bool fast = P.vec && P.ya + dy >= 0 && P.yb - 1 + dy < d.pny && P.x0 + dx >= 0 &&
                      P.x1 - 1 + dx < d.pnx;
    float best_a = -1.f, best_v = 0.f;
    int best_i = 0x7fffffff, best_base = 0x7fffffff;
    float4 best_r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tm_on && kX > 0) {
      __syncwarp();
      ptx::tmem_wait_st();
    }
    // 128-wide chunks with the window inside the PSF: every chunk is a
    // tensor-memory or a streamed one, and the PSF realignment (c0 + dx) mod 4
    // is the same for every chunk of the pass (chunk columns step by 128), so
    // the pass is specialised on it once instead of switching per chunk.  A
    // wait whose producer gave up returns false from its bounded slow path.
    auto fast_pass = [&](auto off) {
      constexpr int OFF = decltype(off)::value;
      int rb = 0, cb = 0;
      for (int ch = 0; ch < P.nch; ++ch) {
        const int st = c_st;
        bool ok = pipe_wait(&full_bar[st], c_ph, limit, &s_dead, &d.st->status);
        if (TM) ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        if (++c_st == S) {
          c_st = 0;
          c_ph ^= 1u;
        }
        const int r0 = P.ya + rb * BH, r1 = min(P.yb, r0 + BH);
        const int c0 = P.x0 + cb * CW, c1 = min(P.x1, c0 + CW);
        if (++cb == P.ncb) {
          cb = 0;
          ++rb;
        }
        const float* stgR = sStage + (size_t)st * stage_floats;
        const float* stgP = stgR + box_floats;
        if (TM && ch < P.n_tm)
          tmem_chunk<OFF>(d, tm_base + (uint32_t)(X * 64 + ch * 16), kX == 0, stgR, stgP, BW, r0,
                          c0, f, best_a, best_base, best_r);
        else
          stream_chunk<OFF>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&empty_bar[st]);
      }
    };
    const bool lean = fast && CW == 128 && BH <= kSlabUnroll * kW;
    if (lean) {
      switch ((P.x0 + dx) & 3) {
        case 0:
          fast_pass(IntTag<0>{});
          break;
        case 1:
          fast_pass(IntTag<1>{});
          break;
        case 2:
          fast_pass(IntTag<2>{});
          break;
        default:
          fast_pass(IntTag<3>{});
          break;
      }
    }
    int rb = 0, cb = 0;
    for (int ch = 0; ch < P.nch && !lean; ++ch) {
      const int st = c_st;
      bool ok = !*(volatile int*)&s_dead &&
                pipe_wait(&full_bar[st], c_ph, limit, &s_dead, &d.st->status);
      if (TM) ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      if (++c_st == S) {
        c_st = 0;
        c_ph ^= 1u;
      }
      const int r0 = P.ya + rb * BH, r1 = min(P.yb, r0 + BH);
      const int c0 = P.x0 + cb * CW, c1 = min(P.x1, c0 + CW);
      if (++cb == P.ncb) {
        cb = 0;
        ++rb;
      }
      const float* stgR = sStage + (size_t)st * stage_floats;
      const float* stgP = stgR + box_floats;
      const int offR = c0 - (c0 & ~3), offP = (c0 + dx) - ((c0 + dx) & ~3);
      if (TM && fast && ch < P.n_tm) {
        const uint32_t ta = tm_base + (uint32_t)(X * 64 + ch * 16);
        const bool from_box = kX == 0;
        switch (offP) {
          case 0:
            tmem_chunk<0>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base, best_r);
            break;
          case 1:
            tmem_chunk<1>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base, best_r);
            break;
          case 2:
            tmem_chunk<2>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base, best_r);
            break;
          default:
            tmem_chunk<3>(d, ta, from_box, stgR, stgP, BW, r0, c0, f, best_a, best_base, best_r);
            break;
        }
      } else if (fast && CW == 128 && BH <= kSlabUnroll * kW) {
        switch (offP) {
          case 0:
            stream_chunk<0>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
            break;
          case 1:
            stream_chunk<1>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
            break;
          case 2:
            stream_chunk<2>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
            break;
          default:
            stream_chunk<3>(d, stgR, stgP, BW, r0, r1 - r0, c0, c1, f, best_a, best_base, best_r);
            break;
        }
      } else if (fast) {
        const int s_first = warp >= rot ? warp - rot : warp + kW - rot;
        switch (offP) {
          case 0:
            chunk_slabs<false, 0>(d, nullptr, 0, 0, stgR, stgP, BW, r0, r1, c0, c1, 0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
            break;
          case 1:
            chunk_slabs<false, 1>(d, nullptr, 0, 0, stgR, stgP, BW, r0, r1, c0, c1, 0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
            break;
          case 2:
            chunk_slabs<false, 2>(d, nullptr, 0, 0, stgR, stgP, BW, r0, r1, c0, c1, 0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
            break;
          default:
            chunk_slabs<false, 3>(d, nullptr, 0, 0, stgR, stgP, BW, r0, r1, c0, c1, 0, f,
                                  lpr_log2, s_first, best_a, best_base, best_r);
            break;
        }
      } else {
        for (int y = r0 + crow; crow < rpp && y < r1; y += rpp) {
          const bool yin = (unsigned)(y + dy) < (unsigned)d.pny;
          const float* rowP = stgP + (y - r0) * BW + offP - c0;  // index by x
          const float* rowR = stgR + (y - r0) * BW + offR - c0;
          for (int x = c0 + ccol; x < c1; x += tpr) {
            float r = rowR[x];
            if (yin && (unsigned)(x + dx) < (unsigned)d.pnx) r = __fsub_rn(r, __fmul_rn(f, rowP[x]));
            d.R[(int64_t)y * d.nx + x] = r;
            take_peak(r, y * d.nx + x, best_a, best_i, best_v);
          }
        }
      }
      rot += rot_step;
      if (rot >= kW) rot -= kW;
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty_bar[st]);
    }
    if (fast && best_a >= 0.f) resolve_group(best_a, best_base, best_r, best_i, best_v);
    const bool fill = tm_on && !*(volatile int*)&s_dead;
    if (X) filled1 = fill; else filled0 = fill;
    // residual rows written through the generic proxy are read back by TMA
    asm volatile("fence.proxy.async.global;" ::: "memory");
    // the CTA's partial key: each consumer warp leaves its maximum and counts
    // itself in; the last warp to arrive reduces, posts and resets the count,
    // so no warp waits for another.  Buffers alternate: a warp refills this
    // one two passes later, after taking a key that needed this pass's post.
    uint64_t mine = (best_a >= 0.f) ? make_key(best_v, best_i) : 0ull;
    mine = warp_max_key(mine);
    const uint32_t buf = n_pass & 1u;
    if (lane == 0) {
      s_warp[buf][warp] = mine;
      __threadfence_block();
      if (atomicAdd(&s_arrived[buf], 1) == kW - 1) {
        __threadfence_block();
        uint64_t m = 0ull;
        for (int w = 0; w < kW; ++w) m = umax64(m, *(volatile uint64_t*)&s_warp[buf][w]);
        const uint32_t g = seqX + (uint32_t)kX;
        uint64_t* slot = d.gkeys + (int64_t)P.t * G2 + (int64_t)(g & 1u) * ((int64_t)d.T * G2);
        st_relaxed_u64(slot + q, m | ((uint64_t)((g >> 1) & 1u) << 63));
        s_arrived[buf] = 0;
      }
    }
    __syncwarp();
    ++n_pass;
    if (X) ++kx1; else ++kx0;
  }

  if (tm_on) {
    // tensor-memory chunks back to global memory, then free the columns
    if (!producer) {
      __syncwarp();
      ptx::tmem_wait_st();
#pragma unroll
      for (int X = 0; X < 2; ++X) {
        const Piece P = X ? pc1 : pc0;
        const bool wb = __shfl_sync(0xffffffffu,
                                    (int)((X ? filled1 : filled0) && !*(volatile int*)&s_dead),
                                    0) != 0;
        if (!wb) continue;
        for (int ch = 0; ch < P.n_tm; ++ch) {
          const int rb = ch / P.ncb, cb = ch - rb * P.ncb;
          const int r0 = P.ya + rb * BH, c0 = P.x0 + cb * CW;
          float4 v[kSlabUnroll];
          __syncwarp();
          ptx::tmem_ld16(tm_base + (uint32_t)(X * 64 + ch * 16), v);
#pragma unroll
          for (int u = 0; u < kSlabUnroll; ++u)
            *reinterpret_cast<float4*>(d.R + (int64_t)(r0 + warp + u * kW) * d.nx + c0 +
                                       4 * lane) = v[u];
        }
      }
    }
    ptx::tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      ptx::tmem_fence_after_sync();
      __syncwarp();
      ptx::tmem_dealloc(s_tmem, kTmemCols);
    }
  }
  if (producer && lane == 0 && s_dead) {
    // after an expired wait: let this CTA's own copies in flight land
    for (int64_t j = max((int64_t)0, jnext - S); j < jnext; ++j) {
      const uint64_t t0 = ptx::globaltimer_ns();
      while (!ptx::mbar_try_wait(&full_bar[j % S], (uint32_t)(j / S) & 1u))
        if (ptx::globaltimer_ns() - t0 > limit) break;
    }
  }
  if (q == 0 && threadIdx.x == 0) {
    d.rcount[pc0.t] = (int32_t)kx0;
    d.budget[pc0.t] = budget0 - kx0;
    d.gbar[pc0.t] = seq00 + (uint32_t)kx0;
    d.rcount[pc1.t] = (int32_t)kx1;
    d.budget[pc1.t] = budget1 - kx1;
    d.gbar[pc1.t] = seq01 + (uint32_t)kx1;
  }
  if (PERSIST) {
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < S; ++i) {
        ptx::mbar_inval(&full_bar[i]);
        ptx::mbar_inval(&empty_bar[i]);
      }
      ptx::mbar_inval(&key_bar[0]);
      ptx::mbar_inval(&key_bar[1]);
    }
    __syncthreads();
  }
}

template <bool TM>
__global__ void __launch_bounds__(kPipeThreads, 1)
    minor_pair_kernel(PlanDev d, MinorCfg c, int parity,
                      const __grid_constant__ CUtensorMap r_map,
                      const __grid_constant__ CUtensorMap p_map) {
  const int G2 = 2 * c.G;
  minor_pair_body<TM>(d, c, parity, &r_map, &p_map, (int)blockIdx.x / G2,
                      (int)blockIdx.x % G2);
}

// Batched pipeline launch: one CTA (kSyncNone) or one cluster of G CTAs per
// (image, tile) item, each image's plan state in `plans` and its residual and
// PSF box maps in rmaps / pmaps (global memory, indexed like `plans`).
template <int SYNC, bool RES, bool TM>
__global__ void __launch_bounds__(kPipeThreads, 1)
    minor_pipe_batch_kernel(const PlanDev* __restrict__ plans,
                            const BatchItem* __restrict__ items, const CUtensorMap* rmaps,
                            const CUtensorMap* pmaps, MinorCfg c, int round) {
  const BatchItem it = items[blockIdx.x / c.G];
  const PlanDev d = plans[it.image];
  const int rank = (SYNC == CLEAN_SYNC_CLUSTER) ? (int)cluster_rank() : 0;
  minor_pipe_body<SYNC, RES, TM>(d, c, (round - d.round0) & 1, rmaps + it.image,
                                 pmaps + it.image, it.tile, rank);
}

// Persistent batched minor loop: one CTA per SM, each working through its
// column of a host-built schedule of waves.  units[w * gridDim.x + b] is the
// (item, rank) that CTA b serves in wave w (item -1: idle).  An item is one
// tile of one image with its own launch configuration; its G ranks sit in
// one wave, so they run at the same time on distinct CTAs (the launch is
// cooperative: every CTA is resident) and exchange their peaks through the
// bounded grid exchange.  A CTA goes on to its next wave as soon as its unit
// ends.  A CTA can only wait for the ranks of its own unit, and the ranks of
// the earliest unfinished wave are all resident and at that unit, so the
// schedule always progresses.  Each unit runs the pipelined body of the
// single-plan and clustered kernels, so the results are bit for bit theirs.
__global__ void __launch_bounds__(kPipeThreads, 1)
    minor_batch_persistent_kernel(const PlanDev* __restrict__ plans,
                                  const BatchUnitItem* __restrict__ items,
                                  const int2* __restrict__ units, int n_waves,
                                  const CUtensorMap* rmaps, const CUtensorMap* pmaps, int round) {
  __shared__ int s_skip;
  for (int w = 0; w < n_waves; ++w) {
    const int2 u = units[(int64_t)w * gridDim.x + blockIdx.x];
    if (u.x < 0) continue;  // the same for the whole CTA
    const BatchUnitItem it = items[u.x];
    const PlanDev d = plans[it.image];
    if (threadIdx.x == 0) s_skip = *(volatile int32_t*)&d.st->status != 0;
    __syncthreads();
    const bool skip = s_skip != 0;
    __syncthreads();
    if (skip) continue;
    const int parity = (round - d.round0) & 1;
    const CUtensorMap* rm = rmaps + it.image;
    const CUtensorMap* pm = pmaps + it.image;
    switch (it.kind) {
      case kUnitResident:
        minor_pipe_body<CLEAN_SYNC_GRID, true, false, true>(d, it.cfg, parity, rm, pm, it.tile, u.y);
        break;
      case kUnitTmem:
        minor_pipe_body<CLEAN_SYNC_GRID, false, true, true>(d, it.cfg, parity, rm, pm, it.tile, u.y);
        break;
      case kUnitPair:  // it.tile: the pair, tiles 2 it.tile and 2 it.tile + 1
        minor_pair_body<true, true>(d, it.cfg, parity, rm, pm, it.tile, u.y);
        break;
      default:
        minor_pipe_body<CLEAN_SYNC_GRID, false, false, true>(d, it.cfg, parity, rm, pm, it.tile, u.y);
        break;
    }
  }
}

template <int SYNC, bool RES>
void* kernel_ptr(bool pipe, bool tmem) {
  if (!pipe) return (void*)minor_kernel<SYNC, RES>;
  if (!RES && tmem) return (void*)minor_pipe_kernel<SYNC, false, true>;
  return (void*)minor_pipe_kernel<SYNC, RES, false>;
}

void* pick(const MinorCfg& c) {
  const bool p = c.pipe != 0, tm = c.tmem != 0;
  if (p && c.pair && !c.resident && c.sync == CLEAN_SYNC_GRID)
    return tm ? (void*)minor_pair_kernel<true> : (void*)minor_pair_kernel<false>;
  if (c.sync == CLEAN_SYNC_CLUSTER)
    return c.resident ? kernel_ptr<CLEAN_SYNC_CLUSTER, true>(p, tm)
                      : kernel_ptr<CLEAN_SYNC_CLUSTER, false>(p, tm);
  return c.resident ? kernel_ptr<CLEAN_SYNC_GRID, true>(p, tm)
                    : kernel_ptr<CLEAN_SYNC_GRID, false>(p, tm);
}

}  // namespace

namespace {
const void* batch_fn(int G, int resident) {
  if (G > 1)
    return resident ? (const void*)minor_batch_kernel<CLEAN_SYNC_CLUSTER, true>
                    : (const void*)minor_batch_kernel<CLEAN_SYNC_CLUSTER, false>;
  return resident ? (const void*)minor_batch_kernel<kSyncNone, true>
                  : (const void*)minor_batch_kernel<kSyncNone, false>;
}
}  // namespace

int minor_batch_cluster(int want, int resident, int smem) {
  for (int G = std::min(16, std::max(1, want)); G > 1; G /= 2) {
    const void* fn = batch_fn(G, resident);
    if (allow_max_smem(fn) != cudaSuccess) break;
    if (G > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess)
      continue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = resident ? smem : 0;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) return G;
  }
  cudaGetLastError();
  return 1;
}

// ---- batched pipeline --------------------------------------------------------

// tmem: the streamed variant that keeps each CTA's leading chunks in tensor
// memory (every CTA owns its SM: the ring takes more than half of its
// shared memory, so a later CTA starts there only after this one freed its
// columns)
const void* pipe_batch_fn(int G, int resident, int tmem) {
  if (G > 1)
    return resident ? (const void*)minor_pipe_batch_kernel<CLEAN_SYNC_CLUSTER, true, false>
           : tmem   ? (const void*)minor_pipe_batch_kernel<CLEAN_SYNC_CLUSTER, false, true>
                    : (const void*)minor_pipe_batch_kernel<CLEAN_SYNC_CLUSTER, false, false>;
  return resident ? (const void*)minor_pipe_batch_kernel<kSyncNone, true, false>
         : tmem   ? (const void*)minor_pipe_batch_kernel<kSyncNone, false, true>
                  : (const void*)minor_pipe_batch_kernel<kSyncNone, false, false>;
}

bool minor_pipe_batch_geometry(MinorCfg& c, int G, int resident, int max_rows, int max_w) {
  c = MinorCfg{};
  c.G = G;
  c.sync = G > 1 ? CLEAN_SYNC_CLUSTER : kSyncNone;
  c.resident = resident;
  c.spin_limit_ns = 2000000000ll;
  c.chunk_w = 128;
  c.box_w = kBatchBoxW;
  c.chunk_h = kBatchBoxRows;
  const int64_t box = (int64_t)((c.box_w * c.chunk_h + 31) & ~31) * 4;
  const int64_t stage = (resident ? 1 : 2) * box;
  c.res_floats = resident ? ((max_rows * ((max_w + 3) & ~3) + 31) & ~31) : 0;
  const int64_t budget = 200 * 1024 - (int64_t)c.res_floats * 4;
  c.stages = (int)std::min<int64_t>(kPipeMaxStages, budget / stage);
  if (c.stages < 2) return false;
  c.smem = (int)((int64_t)c.res_floats * 4 + c.stages * stage);
  c.threads = kPipeThreads;
  c.pipe = 1;
  c.tmem = (!resident && c.smem > 114 * 1024) ? 1 : 0;
  return true;
}

int minor_pipe_batch_cluster(int want, int resident, int smem) {
  for (int G = std::min(16, std::max(1, want)); G > 1; G /= 2) {
    const void* fn = pipe_batch_fn(G, resident, 0);
    if (allow_max_smem(fn) != cudaSuccess) break;
    if (G > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess)
      continue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G, 1, 1);
    cfg.blockDim = dim3(kPipeThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) return G;
  }
  cudaGetLastError();
  return 1;
}

cudaError_t launch_minor_pipe_batch(const PlanDev* plans, const BatchItem* items, int n_items,
                                    const MinorCfg& c, const CUtensorMap* rmaps,
                                    const CUtensorMap* pmaps, int round, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const void* fn = pipe_batch_fn(c.G, c.resident, c.tmem);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  if (c.G > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(n_items * c.G), 1, 1);
  cfg.blockDim = dim3(kPipeThreads, 1, 1);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = c.G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = c.G > 1 ? 1 : 0;
  MinorCfg cc = c;
  void* args[] = {const_cast<PlanDev**>(&plans), const_cast<BatchItem**>(&items),
                  const_cast<CUtensorMap**>(&rmaps), const_cast<CUtensorMap**>(&pmaps), &cc,
                  &round};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

int minor_batch_persistent_grid(int smem) {
  const void* fn = (const void*)minor_batch_persistent_kernel;
  int dev = 0, sms = 0, per_sm = 0;
  if (allow_max_smem(fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPipeThreads, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm >= 1 ? sms : 0;  // one CTA per SM (the tensor-memory units own their SM)
}

cudaError_t launch_minor_batch_persistent(const PlanDev* plans, const BatchUnitItem* items,
                                          const int2* units, int n_waves, int grid, int smem,
                                          const CUtensorMap* rmaps, const CUtensorMap* pmaps,
                                          int round, cudaStream_t s) {
  if (n_waves <= 0 || grid <= 0) return cudaSuccess;
  const void* fn = (const void*)minor_batch_persistent_kernel;
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kPipeThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<PlanDev**>(&plans), const_cast<BatchUnitItem**>(&items),
                  const_cast<int2**>(&units), &n_waves, const_cast<CUtensorMap**>(&rmaps),
                  const_cast<CUtensorMap**>(&pmaps), &round};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_minor_batch(const PlanDev* plans, const BatchItem* items, int n_items, int G,
                               int resident, int smem, int round, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  MinorCfg c{};
  c.G = G;
  c.sync = G > 1 ? CLEAN_SYNC_CLUSTER : kSyncNone;
  c.resident = resident;
  c.smem = resident ? smem : 0;
  c.threads = kThreads;
  c.spin_limit_ns = 2000000000ll;
  const void* fn = batch_fn(G, resident);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  if (G > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(n_items * G), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = G > 1 ? 1 : 0;
  void* args[] = {const_cast<PlanDev**>(&plans), const_cast<BatchItem**>(&items), &c, &round};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t minor_prepare(const MinorCfg& c) {
  const void* fn = pick(c);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  if (c.sync == CLEAN_SYNC_CLUSTER && c.G > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int minor_threads() { return kThreads; }

bool make_box_tensor_map(CUtensorMap* map, const float* base, int rows, int cols, int box_w,
                         int box_h) {
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || (cols % 4) != 0) return false;
  if (box_w > 256 || box_h > 256 || box_w < 4 || (box_w % 4) != 0 || box_h < 1) return false;
  return encode_tensor_map_2d(map, base, rows, cols, box_w, box_h);
}

bool minor_pipe_geometry(MinorCfg& c, int max_rows, int max_w, int chunk_px, int max_stages) {
  // measured on GB300: few large TMA boxes per byte keep the copy engine
  // busy; streamed slabs take 8192-pixel chunks, resident ones 4096
  if (chunk_px <= 0) chunk_px = c.resident ? 4096 : 8192;
  if (max_stages <= 0 || max_stages > kPipeMaxStages) max_stages = kPipeMaxStages;
  // columns: 128 (one warp per row, 4 pixels per lane), or 64 / 32 for narrow
  // tiles; the box is 4 floats wider to cover any misalignment of the PSF
  // window; rows: up to the CTA's row count
  c.chunk_w = max_w > 64 ? 128 : max_w > 32 ? 64 : 32;
  c.box_w = c.chunk_w + 4;
  // rows: a whole number of warp steps (15 warps x kSlabUnroll slabs of
  // 128 / CW rows), so every consumer warp gets the same share of a chunk
  const int unit = (kPipeConsumers / 32) * kSlabUnroll * (128 / c.chunk_w);
  const int h = std::max(unit, (chunk_px / c.chunk_w) / unit * unit);
  c.chunk_h = std::max(1, std::min(std::min(256, max_rows), h));
  const int64_t stage = (int64_t)(c.resident ? 1 : 2) * ((c.box_w * c.chunk_h + 31) & ~31) * 4;
  c.res_floats = c.resident ? max_rows * ((max_w + 3) & ~3) : 0;
  c.res_floats = (c.res_floats + 31) & ~31;  // keep the stages 128-byte aligned
  const int64_t budget = 200 * 1024 - (int64_t)c.res_floats * 4;
  c.stages = (int)std::min<int64_t>(max_stages, budget / stage);
  if (c.stages < 2) return false;
  const int64_t total = (int64_t)c.res_floats * 4 + c.stages * stage;
  c.smem = (int)total;
  c.threads = kPipeThreads;
  c.pipe = 1;
  // tensor-memory chunks: streamed 128 x 60 chunks, and shared memory above
  // half of an SM's 228 KB so that no second CTA of this kernel shares the SM
  // (the 512-column allocation then never waits)
  c.tmem = (!c.resident && c.chunk_w == 128 && c.chunk_h == kTmemChunkRows &&
            c.smem > 114 * 1024) ? 1 : 0;
  return true;
}

// Number of G-CTA clusters that can be co-resident (0 if none).
int minor_max_cluster_ctas(int G, int resident, int smem, int threads) {
  MinorCfg c{};
  c.G = G;
  c.sync = CLEAN_SYNC_CLUSTER;
  c.resident = resident;
  c.smem = smem;
  c.pipe = threads == kPipeThreads ? 1 : 0;
  if (minor_prepare(c) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(G, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, pick(c), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_minor(const PlanDev& d, const MinorCfg& c, int parity,
                         const CUtensorMap* r_map, const CUtensorMap* p_map, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(d.T * c.G), 1, 1);
  cfg.blockDim = dim3(c.pipe ? kPipeThreads : kThreads, 1, 1);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (c.sync == CLEAN_SYNC_CLUSTER) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c.G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
  } else {
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
  }
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PlanDev dd = d;
  MinorCfg cc = c;
  if (c.pipe) {
    if (!p_map || (!c.resident && !r_map)) return cudaErrorInvalidValue;
    CUtensorMap rm = c.resident ? *p_map : *r_map, pm = *p_map;
    void* args[] = {&dd, &cc, &parity, &rm, &pm};
    return cudaLaunchKernelExC(&cfg, pick(c), args);
  }
  void* args[] = {&dd, &cc, &parity};
  return cudaLaunchKernelExC(&cfg, pick(c), args);
}

}  // namespace cleangb
