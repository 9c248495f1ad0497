// FFT feedback (Section 3): the round's components, every tile's, convolved
// with the full PSF through cuFFT transforms, with this library's scatter,
// spectrum multiply and subtract kernels around them.
// Within a tolerance of the exact gather, not bit-exact; the cuFFT plans live
// with the plan (capi.cu).
#include "cleangb_internal.cuh"
#include "round_close.cuh"

namespace cleangb {

namespace {

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
  // 16-byte rows (tile columns, image width and grid pitch multiples of 4):
  // four pixels a thread and step, the peak kept per 4-pixel group as in the
  // minor loop (largest |R|, lowest base index) and resolved once at the end
  const bool vec = ((rc.x0 | (rc.x1 - rc.x0) | d.nx | (int)pitch) & 3) == 0;
  if (live && vec) {
    int best_base = 0x7fffffff;
    float4 best_r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int y = ya; y < yb; ++y)
      for (int x = rc.x0 + 4 * threadIdx.x; x < rc.x1; x += 4 * kFftThreads) {
        const int64_t gi = (int64_t)y * d.nx + x;
        const float4 a = *reinterpret_cast<const float4*>(R0 + gi);
        const float4 b = *reinterpret_cast<const float4*>(S + (int64_t)y * pitch + x);
        const float4 r = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        *reinterpret_cast<float4*>(d.R + gi) = r;
        *reinterpret_cast<float4*>(R0 + gi) = r;
        const float m = fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w)));
        const bool better = m > best_a || (m == best_a && (int)gi < best_base);
        best_a = better ? m : best_a;
        best_base = better ? (int)gi : best_base;
        best_r = better ? r : best_r;
      }
    if (best_a >= 0.f) {
      const int k4 = fabsf(best_r.x) == best_a   ? 0
                     : fabsf(best_r.y) == best_a ? 1
                     : fabsf(best_r.z) == best_a ? 2
                                                 : 3;
      best_i = best_base + k4;
      best_v = k4 == 0 ? best_r.x : k4 == 1 ? best_r.y : k4 == 2 ? best_r.z : best_r.w;
    }
  } else if (live) {
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

cudaError_t fft_prepare() { return allow_max_smem((const void*)fft_subtract); }

}  // namespace cleangb
