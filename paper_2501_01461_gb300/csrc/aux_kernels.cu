// Set-up, input checks and restoration.
//
// init_kernel      R <- dirty, model <- 0, finiteness of the dirty image, the
//                  first peak key of every tile, and the per-tile budgets
//                  (niter split evenly, the remainder to the lowest tiles).
// validate_psf     finiteness of the PSF and |P| <= P[centre] everywhere.
// restore_kernel   model convolved with a Gaussian clean beam, plus residual.
#include <cmath>

#include "cleangb_internal.cuh"

namespace cleangb {

namespace {

constexpr int kInitThreads = 256;
constexpr int kInitRows = 16;  // tile rows per init block

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) {
  return a > b ? a : b;
}

__device__ __forceinline__ uint64_t warp_max_key(uint64_t k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = umax64(k, __shfl_xor_sync(0xffffffffu, k, o));
  return k;
}

__global__ void __launch_bounds__(kInitThreads)
    init_kernel(PlanDev d, const float* dirty, int64_t niter) {
  __shared__ uint64_t s_warp[kInitThreads / 32];
  const int t = blockIdx.y;
  const Rect rc = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
  const int W = rc.x1 - rc.x0;
  const int ya = rc.y0 + blockIdx.x * kInitRows;
  const int yb = min(rc.y1, ya + kInitRows);
  float best_a = -1.f, best_v = 0.f;
  int best_i = 0x7fffffff;
  int bad = 0;
  for (int y = ya; y < yb; ++y)
    for (int c = threadIdx.x; c < W; c += kInitThreads) {
      const int64_t gi = (int64_t)y * d.nx + rc.x0 + c;
      const float v = dirty[gi];
      d.R[gi] = v;
      d.model[gi] = 0.f;
      if (!isfinite(v)) bad = 1;
      const float a = fabsf(v);
      if (a > best_a || (a == best_a && (int)gi < best_i)) {
        best_a = a;
        best_i = (int)gi;
        best_v = v;
      }
    }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&d.st->status, ST_NONFINITE_DIRTY);
  uint64_t k = best_a >= 0.f ? make_key(best_v, best_i) : 0ull;
  k = warp_max_key(k);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t m = 0;
    for (int w = 0; w < kInitThreads / 32; ++w) m = umax64(m, s_warp[w]);
    if (m) atomicMax((unsigned long long*)&d.peak[t], (unsigned long long)m);
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    const int64_t T = d.T;
    for (int s = threadIdx.x; s < d.T; s += kInitThreads) {
      d.budget[s] = niter / T + ((int64_t)s < niter % T ? 1 : 0);
      d.rcount[s] = 0;
      d.gbar[s] = 0u;
    }
    if (threadIdx.x == 0) {
      d.st->active = 1;
      d.st->max_budget = niter / T + (niter % T ? 1 : 0);
    }
  }
}

__global__ void validate_psf_kernel(const float* __restrict__ P, int64_t n, int64_t centre,
                                    int32_t* status) {
  const float pc = P[centre];
  int bad = 0, off = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = P[i];
    if (!isfinite(v)) bad = 1;
    if (fabsf(v) > pc) off = 1;
  }
  if (!isfinite(pc)) bad = 1;
  bad = __syncthreads_or(bad);
  off = __syncthreads_or(off);
  if (threadIdx.x == 0) {
    if (bad) atomicOr(status, ST_NONFINITE_PSF);
    if (off) atomicOr(status, ST_PSF_OFFCENTRE);
  }
}

// Restore: out[q] = R[q] + sum over offsets o in the disc |o| <= r of
// model[q - o] * B(o), B the clean beam (symmetric, so B(o) = B(-o)).
constexpr int kRB = 32;  // output block side

__global__ void __launch_bounds__(kRB * 8)
    restore_kernel(PlanDev d, const float* __restrict__ beam, int r, float* __restrict__ out) {
  extern __shared__ __align__(16) float sm[];
  const int side = kRB + 2 * r;
  float* s_model = sm;                 // side x side
  float* s_beam = sm + side * side;    // (2r+1)^2
  const int y0 = blockIdx.y * kRB, x0 = blockIdx.x * kRB;
  const int nb = (2 * r + 1) * (2 * r + 1);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s_beam[i] = beam[i];
  for (int i = threadIdx.x; i < side * side; i += blockDim.x) {
    const int yy = y0 - r + i / side, xx = x0 - r + i % side;
    s_model[i] = (yy >= 0 && yy < d.ny && xx >= 0 && xx < d.nx)
                     ? d.model[(int64_t)yy * d.nx + xx] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x % kRB, ty0 = threadIdx.x / kRB;  // 8 rows of threads
  for (int ty = ty0; ty < kRB; ty += 8) {
    const int y = y0 + ty, x = x0 + tx;
    if (y >= d.ny || x >= d.nx) continue;
    float acc = 0.f;
    for (int oy = -r; oy <= r; ++oy)
      for (int ox = -r; ox <= r; ++ox) {
        const float b = s_beam[(oy + r) * (2 * r + 1) + (ox + r)];
        if (b == 0.f) continue;
        const float m = s_model[(ty - oy + r) * side + (tx - ox + r)];
        acc = fmaf(m, b, acc);
      }
    out[(int64_t)y * d.nx + x] = d.R[(int64_t)y * d.nx + x] + acc;
  }
}

__global__ void beam_table_kernel(float* beam, int r, float smaj, float smin, float pa) {
  const int n = 2 * r + 1;
  const float c = cosf(pa), s = sinf(pa);
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < n * n; i += blockDim.x * gridDim.x) {
    const int oy = i / n - r, ox = i % n - r;
    float v = 0.f;
    if (oy * oy + ox * ox <= r * r) {
      const float u = ox * c + oy * s, w = -ox * s + oy * c;
      v = expf(-0.5f * ((u / smaj) * (u / smaj) + (w / smin) * (w / smin)));
    }
    beam[i] = v;
  }
}

// The flux-trigger level of the first round: trigger x the largest |peak|
// among the tiles that can run (budget left, |peak| > threshold).
__global__ void first_level_kernel(PlanDev d) {
  __shared__ uint32_t s_top;
  if (threadIdx.x == 0) s_top = 0u;
  __syncthreads();
  uint32_t top = 0u;
  for (int s = threadIdx.x; s < d.T; s += blockDim.x) {
    const uint64_t pk = d.peak[s];
    if (d.budget[s] > 0 && pk != 0ull && key_abs(pk) > d.thr) top = max(top, (uint32_t)(pk >> 32));
  }
  if (top) atomicMax(&s_top, top);
  __syncthreads();
  if (threadIdx.x == 0) d.st->level = __fmul_rn(d.trigger, __uint_as_float(s_top));
}

}  // namespace

cudaError_t launch_first_level(const PlanDev& d, cudaStream_t s) {
  if (!(d.trigger > 0.f)) return cudaSuccess;
  first_level_kernel<<<1, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_init(const PlanDev& d, const float* dirty, int64_t niter, cudaStream_t s) {
  int maxH = 0;
  for (int i = 0; i < d.ty; ++i)
    maxH = max(maxH, (int)(((int64_t)(i + 1) * d.ny) / d.ty - ((int64_t)i * d.ny) / d.ty));
  dim3 grid((maxH + kInitRows - 1) / kInitRows, d.T, 1);
  init_kernel<<<grid, kInitThreads, 0, s>>>(d, dirty, niter);
  return cudaGetLastError();
}

cudaError_t launch_validate_psf(const PlanDev& d, cudaStream_t s) {
  const int64_t n = (int64_t)d.pny * d.pnx;
  const int64_t centre = (int64_t)d.cy * d.pnx + d.cx;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  validate_psf_kernel<<<blocks, 256, 0, s>>>(d.P, n, centre, &d.st->status);
  return cudaGetLastError();
}

// Beam table scratch: a plan-owned buffer of (2r+1)^2 floats is passed in.
cudaError_t launch_restore_with(const PlanDev& d, float bmaj, float bmin, float bpa,
                                float* beam_buf, int r, float* out, cudaStream_t s) {
  const float k = 1.0f / (2.0f * sqrtf(2.0f * logf(2.0f)));
  beam_table_kernel<<<8, 256, 0, s>>>(beam_buf, r, bmaj * k, bmin * k, bpa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int side = kRB + 2 * r;
  const size_t smem = sizeof(float) * ((size_t)side * side + (size_t)(2 * r + 1) * (2 * r + 1));
  e = allow_max_smem((const void*)restore_kernel);
  if (e != cudaSuccess) return e;
  dim3 grid((d.nx + kRB - 1) / kRB, (d.ny + kRB - 1) / kRB, 1);
  restore_kernel<<<grid, kRB * 8, smem, s>>>(d, beam_buf, r, out);
  return cudaGetLastError();
}

}  // namespace cleangb
