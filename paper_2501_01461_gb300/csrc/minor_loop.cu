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
#include "cleangb_internal.cuh"

namespace cleangb {

namespace {

constexpr int kThreads = 1024;
constexpr int kUnroll = 8;

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

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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
  k = warp_max_key(k);
  if (lane == 0) s_warp[warp] = k;
  __syncthreads();
  if (warp == 0) {
    k = lane < (kThreads / 32) ? s_warp[lane] : 0ull;
    k = warp_max_key(k);
  }
  return k;
}

template <int SYNC, bool RES>
__global__ void __launch_bounds__(kThreads, 1)
    minor_kernel(PlanDev d, MinorCfg c, int parity) {
  extern __shared__ __align__(16) float sR[];
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_part[2];
  __shared__ uint64_t s_best;
  __shared__ int s_abort;

  const int G = c.G;
  const int t = blockIdx.x / G;
  const int rank = (SYNC == CLEAN_SYNC_CLUSTER) ? (int)cluster_rank() : (int)(blockIdx.x % G);
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int H = rc.y1 - rc.y0;
  const int ya = rc.y0 + (int)(((int64_t)rank * H) / G);
  const int yb = rc.y0 + (int)(((int64_t)(rank + 1) * H) / G);
  const int W = rc.x1 - rc.x0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Status bits only change inside grid-synchronised launches (timeouts), so
  // every CTA of a cluster reads the same value here.
  if (*(volatile int32_t*)&d.st->status != 0) return;

  uint64_t key = d.peak[parity * d.T + t];
  const int64_t budget = d.budget[t];
  const int64_t kmax = (d.K > 0 && (int64_t)d.K < budget) ? (int64_t)d.K : budget;
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

  uint64_t* gslot0 = d.gkeys + (int64_t)t * G;
  const int64_t gstride = (int64_t)d.T * G;
  int64_t k = 0;
  while (k < kmax && key != 0ull) {
    const float v = key_value(key);
    if (!(fabsf(v) > d.thr)) break;
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

    if (SYNC == CLEAN_SYNC_CLUSTER) {
      if (threadIdx.x == 0) s_part[k & 1] = mine;
      cluster_sync_all();
      if (warp == 0) {
        uint64_t kk = lane < G ? ld_cluster_u64(&s_part[k & 1], (uint32_t)lane) : 0ull;
        kk = warp_max_key(kk);
        if (lane == 0) s_best = kk;
      }
    } else {
      if (warp == 0) {
        uint64_t* slot = gslot0 + (k & 1) * gstride;
        int abort = 0;
        if (lane == 0) {
          st_relaxed_u64(slot + rank, mine);
          red_release_add_u32(d.gbar + t, 1u);
          const uint32_t target = (uint32_t)((k + 1) * G) + (uint32_t)(c.force_timeout ? 1 : 0);
          const uint64_t t0 = globaltimer_ns();
          while (ld_acquire_u32(d.gbar + t) < target) {
            if (globaltimer_ns() - t0 > (uint64_t)c.spin_limit_ns) {
              atomicOr(&d.st->status, ST_TIMEOUT);
              d.st->timeout_where = ((int64_t)t << 32) | (int64_t)k;
              abort = 1;
              break;
            }
          }
        }
        abort = __shfl_sync(0xffffffffu, abort, 0);
        __syncwarp();
        uint64_t kk = 0ull;
        if (!abort)
          for (int j = lane; j < G; j += 32) kk = umax64(kk, ld_relaxed_u64(slot + j));
        kk = warp_max_key(kk);
        if (lane == 0) {
          s_best = kk;
          s_abort = abort;
        }
      }
    }
    __syncthreads();
    if (s_abort) break;
    key = s_best;
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
  }
}

template <int SYNC, bool RES>
void* kernel_ptr() {
  return (void*)minor_kernel<SYNC, RES>;
}

void* pick(const MinorCfg& c) {
  if (c.sync == CLEAN_SYNC_CLUSTER)
    return c.resident ? kernel_ptr<CLEAN_SYNC_CLUSTER, true>()
                      : kernel_ptr<CLEAN_SYNC_CLUSTER, false>();
  return c.resident ? kernel_ptr<CLEAN_SYNC_GRID, true>()
                    : kernel_ptr<CLEAN_SYNC_GRID, false>();
}

}  // namespace

cudaError_t minor_prepare(const MinorCfg& c) {
  const void* fn = pick(c);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       c.smem);
  if (e != cudaSuccess) return e;
  if (c.sync == CLEAN_SYNC_CLUSTER && c.G > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int minor_threads() { return kThreads; }

// Number of G-CTA clusters that can be co-resident (0 if none).
int minor_max_cluster_ctas(int G, int resident, int smem, int threads) {
  MinorCfg c{};
  c.G = G;
  c.sync = CLEAN_SYNC_CLUSTER;
  c.resident = resident;
  c.smem = smem;
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
                         cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(d.T * c.G), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
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
  void* args[] = {&dd, &cc, &parity};
  return cudaLaunchKernelExC(&cfg, pick(c), args);
}

}  // namespace cleangb
