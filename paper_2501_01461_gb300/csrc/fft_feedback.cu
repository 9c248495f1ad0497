// FFT feedback (Section 3, Figs. 2-3): the round's components, every tile's,
// convolved with the full PSF by this library's own transforms.  Within a
// tolerance of the exact gather, not bit-exact.
//
// The components, placed on an Ly x Lx grid (Ly >= 2 ny - 1, Lx >= 2 nx - 1),
// convolved circularly with the PSF kernel K[d mod L] = P[d + c], give at
// every image pixel q
//     S[q] = sum_c f_c P[q - p_c + c]
// with no wrap-around.  The residual after the round is the residual at the
// round's start minus S on every pixel of every tile (the minor loops'
// own-tile subtractions included), so no per-tile correction is needed.
//
// The 2-D transforms are split by axis and pruned to what the round needs:
//   columns (one CTA per frequency k of the x axis, k = 0 .. Lx/2):
//       the column's input is the x-axis DFT of the component grid at k,
//       sum over the components of a row of f e^{-2 pi i k x / Lx}, evaluated
//       directly (a round has few components: the grid is sparse); then a
//       forward FFT along y, the product with the cached kernel spectrum, an
//       inverse FFT along y, and only rows 0 .. ny - 1 are stored;
//   rows (one CTA per pair of image rows): the Hermitian half of each row's
//       x-axis spectrum is extended to the full length, two real rows ride in
//       one complex inverse FFT (one as the real, one as the imaginary part),
//       and only columns 0 .. nx - 1 are kept; the same CTA then sets
//       R <- R_round_start - S, reduces the next peaks and closes the round.
// The kernel spectrum is built the same way once per PSF (dense rows, two
// per complex FFT, then columns).
//
// Every 1-D transform is a mixed-radix (8, 4, 2, 3, 5, 7) Stockham FFT in
// shared memory: each stage reads a thread's butterfly inputs into
// registers, applies the stage twiddles, synchronises, and writes the small
// DFT's outputs back to the autosorted positions.  Twiddles come from a
// table exp(-2 pi i t / L) computed in double precision on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cleangb_internal.cuh"
#include "ptx.cuh"
#include "round_close.cuh"

namespace cleangb {

namespace {

__device__ __forceinline__ int fpad(int i) { return i + (i >> 5); }  // shared-memory padding

constexpr uint64_t kFftWaitNs = 2000000000ull;  // bound of every bulk-copy wait

// 1-D bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completion on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(ptx::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(ptx::smem_u32(bar))
      : "memory");
}

int fft_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return std::max(n, 1);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 rot(float2 a, bool inv) {
  return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs X[m] = sum_r v[r] w^(r m), w = e^(-2 pi i / R) (e^(+...) when inv).
template <int R>
struct Dft;

template <>
struct Dft<2> {
  __device__ __forceinline__ static void run(float2 (&v)[2], bool, const float2*, int) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <>
struct Dft<4> {
  __device__ __forceinline__ static void run(float2 (&v)[4], bool inv, const float2*, int) {
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = rot(csub(v[1], v[3]), inv);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <>
struct Dft<8> {
  // radix 2 over (r, r + 4), then two DFT-4s, the odd one after the
  // twiddles w8^r
  __device__ __forceinline__ static void run(float2 (&v)[8], bool inv, const float2*, int) {
    const float h = 0.70710678118654752f;  // sqrt(2) / 2
    float2 b[4], c[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      b[r] = cadd(v[r], v[r + 4]);
      c[r] = csub(v[r], v[r + 4]);
    }
    // c[r] *= w8^r, w8 = (1 - i) / sqrt(2) forward, (1 + i) / sqrt(2) inverse
    c[1] = inv ? make_float2((c[1].x - c[1].y) * h, (c[1].x + c[1].y) * h)
               : make_float2((c[1].x + c[1].y) * h, (c[1].y - c[1].x) * h);
    c[2] = rot(c[2], inv);
    c[3] = inv ? make_float2(-(c[3].x + c[3].y) * h, (c[3].x - c[3].y) * h)
               : make_float2((c[3].y - c[3].x) * h, -(c[3].x + c[3].y) * h);
    Dft<4>::run(b, inv, nullptr, 0);
    Dft<4>::run(c, inv, nullptr, 0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 * m] = b[m];
      v[2 * m + 1] = c[m];
    }
  }
};

// Odd radices: the roots of unity from the length-L table (R divides L).
template <int R>
struct Dft {
  __device__ __forceinline__ static void run(float2 (&v)[R], bool inv, const float2* tw, int L) {
    float2 w[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      w[m] = __ldg(&tw[m * (L / R)]);
      if (inv) w[m].y = -w[m].y;
    }
    float2 out[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      float2 acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], w[(r * m) % R]));
      out[m] = acc;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = out[m];
  }
};

// One Stockham stage of radix R over buf[0 .. L): sub-transforms of size Ns
// become sub-transforms of size Ns R.  tws: the stage's twiddles
// exp(-2 pi i r k / (Ns R)) at r Ns + k.  Every thread of the block calls it.
template <int R>
__device__ __forceinline__ void fft_stage(float2* buf, int L, int Ns, const float2* __restrict__ tw,
                                          const float2* __restrict__ tws, bool inv) {
  constexpr int kMaxB = (kFftValsPerThread + R - 1) / R;
  const int nb = L / R;
  const int nthr = blockDim.x;
  float2 v[kMaxB][R];
#pragma unroll
  for (int b = 0; b < kMaxB; ++b) {
    const int j = threadIdx.x + b * nthr;
    if (j < nb) {
      const int k = j % Ns;
      v[b][0] = buf[fpad(j)];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(&tws[r * Ns + k]);
        if (inv) w.y = -w.y;
        v[b][r] = cmul(buf[fpad(j + r * nb)], w);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < kMaxB; ++b) {
    const int j = threadIdx.x + b * nthr;
    if (j < nb) {
      Dft<R>::run(v[b], inv, tw, L);
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[fpad(base + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

// The same stage reading `in` and writing `out` (another buffer): each
// butterfly goes through registers alone (one at a time per thread), and the
// stage needs one barrier, after its stores.
template <int R>
__device__ __forceinline__ void fft_stage_pp(const float2* in, float2* out, int L, int Ns,
                                             const float2* __restrict__ tw,
                                             const float2* __restrict__ tws, bool inv) {
  const int nb = L / R;
#pragma unroll 1
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    float2 v[R];
    v[0] = in[fpad(j)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = __ldg(&tws[r * Ns + k]);
      if (inv) w.y = -w.y;
      v[r] = cmul(in[fpad(j + r * nb)], w);
    }
    Dft<R>::run(v, inv, tw, L);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[fpad(base + r * Ns)] = v[r];
  }
  __syncthreads();
}

// ---- power-of-two lengths 2048 .. 8192: radix-16 stages, L / 16 threads --------
// Each thread holds one 16-point butterfly per stage in registers; all index
// arithmetic is compile-time.  A stage's twiddles w^r (w = e^(-2 pi i k /
// (16 Ns))) are built from w, w^2, w^4, w^8 read from the table (at most three
// products deep).

// w16^p, p = 0 .. 15 (forward e^(-2 pi i p / 16))
__device__ __forceinline__ float2 w16(int p, bool inv) {
  const float C = 0.92387953251128674f, S = 0.38268343236508977f, H = 0.70710678118654752f;
  float2 w;
  switch (p & 15) {
    case 0: w = make_float2(1.f, 0.f); break;
    case 1: w = make_float2(C, -S); break;
    case 2: w = make_float2(H, -H); break;
    case 3: w = make_float2(S, -C); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 5: w = make_float2(-S, -C); break;
    case 6: w = make_float2(-H, -H); break;
    case 7: w = make_float2(-C, -S); break;
    case 8: w = make_float2(-1.f, 0.f); break;
    case 9: w = make_float2(-C, S); break;
    case 10: w = make_float2(-H, H); break;
    case 11: w = make_float2(-S, C); break;
    case 12: w = make_float2(0.f, 1.f); break;
    case 13: w = make_float2(S, C); break;
    case 14: w = make_float2(H, H); break;
    default: w = make_float2(C, S); break;
  }
  if (inv) w.y = -w.y;
  return w;
}

// X[m + 4q] = sum_t x[t] w16^(t (m + 4q)): DFT-4s over t = r + 4s for each r,
// twiddles w16^(r m), DFT-4s over r.
__device__ __forceinline__ void dft16(float2 (&x)[16], bool inv) {
  float2 b[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 t[4] = {x[r], x[r + 4], x[r + 8], x[r + 12]};
    Dft<4>::run(t, inv, nullptr, 0);
#pragma unroll
    for (int m = 0; m < 4; ++m) b[r][m] = (r == 0 || m == 0) ? t[m] : cmul(t[m], w16(r * m, inv));
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float2 t[4] = {b[0][m], b[1][m], b[2][m], b[3][m]};
    Dft<4>::run(t, inv, nullptr, 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[m + 4 * q] = t[q];
  }
}

// The default input of a transform's first stage and output of its last:
// the shared-memory buffer itself.  Kernels pass their own to fuse the pass
// before the transform into its first loads, or the pass after it into its
// last stores.
struct BufIO {
  float2* buf;
  __device__ __forceinline__ float2 load(int i) const { return buf[fpad(i)]; }
  __device__ __forceinline__ void store(int i, float2 v) const { buf[fpad(i)] = v; }
};

template <int L, int NS, bool FIRST, bool LAST, class Pro, class Epi>
__device__ __forceinline__ void p2_stage16(float2* buf, const float2* __restrict__ tws, bool inv,
                                           const Pro& pro, const Epi& epi) {
  constexpr int NB = L / 16;  // one butterfly a thread
  const int j = threadIdx.x;
  const int k = j & (NS - 1);
  float2 x[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) x[r] = FIRST ? pro.load(j + r * NB) : buf[fpad(j + r * NB)];
  if (NS > 1) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(tws) + 2 * k);
    const float4 c = __ldg(reinterpret_cast<const float4*>(tws) + 2 * k + 1);
    const float sg = inv ? -1.f : 1.f;
    float2 w[16];
    w[1] = make_float2(a.x, sg * a.y);
    w[2] = make_float2(a.z, sg * a.w);
    w[4] = make_float2(c.x, sg * c.y);
    w[8] = make_float2(c.z, sg * c.w);
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
#pragma unroll
    for (int r = 1; r < 16; ++r) x[r] = cmul(x[r], w[r]);
  }
  __syncthreads();
  dft16(x, inv);
  const int base = (j - k) * 16 + k;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if (LAST)
      epi.store(base + r * NS, x[r]);
    else
      buf[fpad(base + r * NS)] = x[r];
  }
  __syncthreads();
}

// Last stage of radix R = L / NS < 16: 16 / R butterflies a thread; twiddles
// exp(-2 pi i r k / L) at r NS + k.
template <int L, int NS, class Epi>
__device__ __forceinline__ void p2_tail(float2* buf, const float2* __restrict__ tws, bool inv,
                                        const Epi& epi) {
  constexpr int R = L / NS, NB = L / R, NT = L / 16, MB = 16 / R;
  float2 v[MB][R];
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int j = threadIdx.x + b * NT;
    const int k = j & (NS - 1);
    v[b][0] = buf[fpad(j)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = __ldg(&tws[r * NS + k]);
      if (inv) w.y = -w.y;
      v[b][r] = cmul(buf[fpad(j + r * NB)], w);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int j = threadIdx.x + b * NT;
    const int k = j & (NS - 1);
    Dft<R>::run(v[b], inv, nullptr, 0);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) epi.store(base + r * NS, v[b][r]);
  }
  __syncthreads();
}

// Radix-16 stages, then a smaller last one if L is not a power of 16 (the
// first stage is always radix 16: L >= 2048).  pro feeds the first stage,
// epi takes the last stage's outputs.
template <int L, int NS, int S, class Pro, class Epi>
__device__ __forceinline__ void p2_fft(float2* buf, const FftAxis& ax, const float2* __restrict__ tw,
                                       bool inv, const Pro& pro, const Epi& epi) {
  if constexpr (NS * 16 <= L) {
    constexpr bool last = NS * 16 == L;
    p2_stage16<L, NS, NS == 1, last>(buf, tw + ax.tw_off[S], inv, pro, epi);
    p2_fft<L, NS * 16, S + 1>(buf, ax, tw, inv, pro, epi);
  } else if constexpr (NS < L) {
    p2_tail<L, NS>(buf, tw + ax.tw_off[S], inv, epi);
  }
}

// The radix-16 transform of one length with fused first loads / last stores.
template <class Pro, class Epi>
__device__ __forceinline__ void fft_p2_io(float2* buf, const FftAxis& ax,
                                          const float2* __restrict__ tw, bool inv, const Pro& pro,
                                          const Epi& epi) {
  switch (ax.L) {
    case 8192: p2_fft<8192, 1, 0>(buf, ax, tw, inv, pro, epi); return;
    case 4096: p2_fft<4096, 1, 0>(buf, ax, tw, inv, pro, epi); return;
    default: p2_fft<2048, 1, 0>(buf, ax, tw, inv, pro, epi); return;
  }
}

// Whole 1-D transform of buf (length ax.L, natural order in and out,
// unnormalised).  The caller synchronises before (inputs written) and the
// last stage synchronises after.  P2: the radix-16 path (ax.p2 set); each
// kernel is compiled once per path, so neither path's registers burden the
// other.
template <bool P2>
__device__ __forceinline__ void fft_1d(float2* buf, const FftAxis& ax,
                                       const float2* __restrict__ tw, bool inv,
                                       float2* tmp = nullptr) {
  if constexpr (P2) {
    fft_p2_io(buf, ax, tw, inv, BufIO{buf}, BufIO{buf});
    return;
  }
  if (tmp) {
    // mixed radix with a scratch buffer: stages alternate between the two,
    // and the result comes back to buf if it ends in tmp
    float2* a = buf;
    float2* b = tmp;
    int Ns = 1;
    for (int s = 0; s < ax.nrad; ++s) {
      const int R = ax.rad[s];
      const float2* tws = tw + ax.tw_off[s];
      switch (R) {
        case 8: fft_stage_pp<8>(a, b, ax.L, Ns, tw, tws, inv); break;
        case 4: fft_stage_pp<4>(a, b, ax.L, Ns, tw, tws, inv); break;
        case 2: fft_stage_pp<2>(a, b, ax.L, Ns, tw, tws, inv); break;
        case 3: fft_stage_pp<3>(a, b, ax.L, Ns, tw, tws, inv); break;
        case 5: fft_stage_pp<5>(a, b, ax.L, Ns, tw, tws, inv); break;
        default: fft_stage_pp<7>(a, b, ax.L, Ns, tw, tws, inv); break;
      }
      float2* t = a;
      a = b;
      b = t;
      Ns *= R;
    }
    if (a != buf) {
      for (int i = threadIdx.x; i < ax.L; i += blockDim.x) buf[fpad(i)] = a[fpad(i)];
      __syncthreads();
    }
    return;
  }
  int Ns = 1;
  for (int s = 0; s < ax.nrad; ++s) {
    const int R = ax.rad[s];
    const float2* tws = tw + ax.tw_off[s];
    switch (R) {
      case 8: fft_stage<8>(buf, ax.L, Ns, tw, tws, inv); break;
      case 4: fft_stage<4>(buf, ax.L, Ns, tw, tws, inv); break;
      case 2: fft_stage<2>(buf, ax.L, Ns, tw, tws, inv); break;
      case 3: fft_stage<3>(buf, ax.L, Ns, tw, tws, inv); break;
      case 5: fft_stage<5>(buf, ax.L, Ns, tw, tws, inv); break;
      default: fft_stage<7>(buf, ax.L, Ns, tw, tws, inv); break;
    }
    Ns *= R;
  }
}

// ---- PSF kernel spectrum (once per PSF) -------------------------------------

// Kernel image value K(my, mx) = P[dy + cy, dx + cx] with d the signed
// representative of m (|dy| < ny, |dx| < nx), zero elsewhere.
__device__ __forceinline__ float kernel_image(const PlanDev& d, int Ly, int Lx, int my, int mx) {
  const int dy = my < d.ny ? my : my - Ly;
  const int dx = mx < d.nx ? mx : mx - Lx;
  if (dy <= -d.ny || dx <= -d.nx) return 0.f;
  const int sy = dy + d.cy, sx = dx + d.cx;
  if ((unsigned)sy >= (unsigned)d.pny || (unsigned)sx >= (unsigned)d.pnx) return 0.f;
  return d.P[(int64_t)sy * d.pnx + sx];
}

// Rows 2a and 2a + 1 of the kernel image through one complex FFT along x;
// their Hermitian halves go to Kspec[k][2a], Kspec[k][2a + 1] (k <= Lx/2).
template <bool P2>
__global__ void __launch_bounds__(kFftMaxThreads, 1) fft_psf_rows_kernel(PlanDev d, FftAxis ax, int Ly, const float2* __restrict__ twx,
                                    float2* __restrict__ Kspec) {
  extern __shared__ float2 fbuf[];
  const int Lx = ax.L, a = blockIdx.x;
  for (int mx = threadIdx.x; mx < Lx; mx += blockDim.x)
    fbuf[fpad(mx)] = make_float2(kernel_image(d, Ly, Lx, 2 * a, mx),
                                 kernel_image(d, Ly, Lx, 2 * a + 1, mx));
  __syncthreads();
  fft_1d<P2>(fbuf, ax, twx, false, P2 ? nullptr : fbuf + fpad(Lx) + 2);
  for (int k = threadIdx.x; k <= Lx / 2; k += blockDim.x) {
    const float2 z1 = fbuf[fpad(k)];
    const float2 z = fbuf[fpad(k == 0 ? 0 : Lx - k)];
    const float2 z2 = make_float2(z.x, -z.y);  // conj(Z[L - k])
    const float2 A = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y + z2.y));
    const float2 B = make_float2(0.5f * (z1.y - z2.y), -0.5f * (z1.x - z2.x));  // (z1 - z2) / 2i
    Kspec[(int64_t)k * Ly + 2 * a] = A;
    Kspec[(int64_t)k * Ly + 2 * a + 1] = B;
  }
}

// Column k of the row transforms through a forward FFT along y, scaled by
// 1 / (Ly Lx), in place.
template <bool P2>
__global__ void __launch_bounds__(kFftMaxThreads, 1) fft_psf_cols_kernel(FftAxis ay, const float2* __restrict__ twy,
                                    float2* __restrict__ Kspec, float scale) {
  extern __shared__ float2 fbuf[];
  const int Ly = ay.L;
  float2* col = Kspec + (int64_t)blockIdx.x * Ly;
  for (int i = threadIdx.x; i < Ly; i += blockDim.x) fbuf[fpad(i)] = col[i];
  __syncthreads();
  fft_1d<P2>(fbuf, ay, twy, false, P2 ? nullptr : fbuf + fpad(Ly) + 2);
  for (int i = threadIdx.x; i < Ly; i += blockDim.x) {
    const float2 v = fbuf[fpad(i)];
    col[i] = make_float2(v.x * scale, v.y * scale);
  }
}

// ---- one round ----------------------------------------------------------------

// The round's components of every tile in list order (tile, then iteration)
// as comps[1 + g] = (y, x, flux bits, next), where next is the list index of
// the next component on the same image row (-1: none); comps[0] = (n, number
// of rows with components); lead[0 .. rows) the first component of each such
// row (in no particular order).  One block: a histogram of the rows and its
// prefix give each row its range of `bucket`; one warp then places the
// components 32 at a time in list order (within a step, lanes of one row by
// lane), so every row's range holds its components in list order, and the
// chains follow the ranges.
constexpr int kCompThreads = 1024;
constexpr int kCompSmem = 8192;  // components whose rows are kept in shared memory
__global__ void __launch_bounds__(kCompThreads)
    fft_comp_list_kernel(PlanDev d, int4* __restrict__ comps, int* __restrict__ lead,
                         int* __restrict__ bucket) {
  extern __shared__ int32_t s_int[];
  int32_t* s_cnt = s_int;               // [T] then reused: [ny] row counts
  int32_t* s_pre = s_int + d.T;         // [T + 1]
  int32_t* s_rc = s_pre + d.T + 1;      // [ny] row counts, then running fill
  int32_t* s_ro = s_rc + d.ny;          // [ny + 1] row offsets
  int32_t* s_y = s_ro + d.ny + 1;       // the components' rows, when they fit
  __shared__ int s_rows;
  const bool live = *(volatile int32_t*)&d.st->status == 0;
  for (int s = threadIdx.x; s < d.T; s += blockDim.x) s_cnt[s] = live ? d.rcount[s] : 0;
  for (int y = threadIdx.x; y < d.ny; y += blockDim.x) s_rc[y] = 0;
  if (threadIdx.x == 0) s_rows = 0;
  block_prefix(s_cnt, s_pre, d.T);
  const int n = s_pre[d.T];
  const bool in_smem = n <= kCompSmem;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const int s = find_tile(s_pre, d.T, g);
    const clean_component cc = d.rcomps[(int64_t)s * d.cap_round + (g - s_pre[s])];
    comps[1 + g] = make_int4(cc.y, cc.x, __float_as_int(cc.flux), -1);
    if (in_smem) s_y[g] = cc.y;
    atomicAdd(&s_rc[cc.y], 1);
  }
  block_prefix(s_rc, s_ro, d.ny);  // synchronises before and after
  for (int y = threadIdx.x; y < d.ny; y += blockDim.x) s_rc[y] = 0;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int base = 0; base < n; base += 32) {
      const int g = base + lane;
      const bool valid = g < n;
      const int y = valid ? (in_smem ? s_y[g] : comps[1 + g].x) : -1 - lane;
      const unsigned grp = __match_any_sync(0xffffffffu, y);
      const int rank = __popc(grp & ((1u << lane) - 1u));
      const int filled = valid ? s_rc[y] : 0;
      __syncwarp();
      if (valid) {
        bucket[s_ro[y] + filled + rank] = g;
        if ((grp >> lane) == 1u) s_rc[y] = filled + rank + 1;  // the group's last lane
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int g = bucket[p];
    const int y = in_smem ? s_y[g] : comps[1 + g].x;
    comps[1 + g].w = p + 1 < s_ro[y + 1] ? bucket[p + 1] : -1;
    if (p == s_ro[y]) lead[atomicAdd(&s_rows, 1)] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) comps[0] = make_int4(n, s_rows, 0, 0);
}

// Columns k = blockIdx.x, blockIdx.x + gridDim.x, ... (one CTA per SM):
// the components' x-axis DFT at k placed on their rows, forward FFT along y,
// times the kernel spectrum, inverse FFT along y; rows 0 .. ny - 1 to Y
// (pair-major, below).  The components of one row are summed in list order (their
// chain), so the result is deterministic.  The kernel spectrum's column
// arrives by one bulk copy into shared memory, issued a column ahead, so
// its load overlaps the previous column's transforms.
// Fused first loads / last stores of the radix-16 path (see BufIO).
struct RowsIn {  // the column's input: component rows from rowv, zero elsewhere
  const float2* rowv;
  int ny;
  __device__ __forceinline__ float2 load(int i) const {
    return i < ny ? rowv[i] : make_float2(0.f, 0.f);
  }
};
struct TimesK {  // the forward transform's outputs times the spectrum column
  float2* buf;
  const float2* kst;
  __device__ __forceinline__ void store(int i, float2 v) const { buf[fpad(i)] = cmul(v, kst[i]); }
};
struct ToY {  // the inverse transform's image rows, pair-major into Y
  float2* Y;
  int ny, ncols, k;
  __device__ __forceinline__ void store(int q, float2 v) const {
    if (q < ny) Y[(((int64_t)(q >> 1) * ncols + k) << 1) + (q & 1)] = v;
  }
};

template <bool P2>
__global__ void __launch_bounds__(kFftMaxThreads, 1)
    fft_cols_kernel(PlanDev d, FftAxis ay, int Lx, const int4* __restrict__ comps,
                    const int* __restrict__ lead, const float2* __restrict__ twx,
                    const float2* __restrict__ twy, const float2* __restrict__ Kspec,
                    float2* __restrict__ Y, uint64_t limit_ns) {
  extern __shared__ __align__(128) unsigned char fsm[];
  const int Ly = ay.L, ny = d.ny, ncols = Lx / 2 + 1;
  float2* kst = reinterpret_cast<float2*>(fsm);  // the spectrum column, Ly
  float2* fbuf = kst + Ly;                        // the transform, padded
  float2* rowv = fbuf + fpad(Ly) + 2;             // radix-16 path: the component rows' inputs
  float2* scratch = rowv;                         // mixed radix: the transforms' second buffer
  __shared__ __align__(8) uint64_t kbar;
  __shared__ int s_abort;
  const uint32_t kbytes = (uint32_t)Ly * (uint32_t)sizeof(float2);
  const int rows = comps[0].y;
  if (threadIdx.x == 0) {
    s_abort = *(volatile int32_t*)&d.st->status != 0;
    ptx::mbar_init(&kbar, 1);
    ptx::fence_barrier_init();
    if (!s_abort && blockIdx.x < ncols) {
      ptx::mbar_arrive_expect_tx(&kbar, kbytes);
      bulk_load(kst, Kspec + (int64_t)blockIdx.x * Ly, kbytes, &kbar);
    }
  }
  if (P2)  // rows without components stay zero for every column
    for (int q = threadIdx.x; q < ny; q += blockDim.x) rowv[q] = make_float2(0.f, 0.f);
  __syncthreads();
  if (s_abort) return;  // uniform: written before the barrier
  uint32_t phase = 0;
  for (int k = blockIdx.x; k < ncols; k += gridDim.x) {
    if (!P2) {
#pragma unroll
      for (int u = 0; u < kFftValsPerThread; ++u) {
        const int i = threadIdx.x + u * blockDim.x;
        if (i < Ly) fbuf[fpad(i)] = make_float2(0.f, 0.f);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      int j = lead[i];
      const int y = comps[1 + j].x;
      float2 acc = make_float2(0.f, 0.f);
      while (j >= 0) {
        const int4 e = comps[1 + j];  // (y, x, flux bits, next)
        const float2 w = __ldg(&twx[(int)(((int64_t)k * e.y) % Lx)]);
        const float f = __int_as_float(e.z);
        acc = cadd(acc, make_float2(f * w.x, f * w.y));
        j = e.w;
      }
      if (P2)
        rowv[y] = acc;
      else
        fbuf[fpad(y)] = acc;
    }
    if (P2) {
      // the spectrum column (every thread waits, bounded), then the forward
      // transform from the rows, times the column in its last stage
      if (!ptx::mbar_wait_bounded(&kbar, phase, limit_ns)) {
        atomicOr(&d.st->status, ST_TIMEOUT);
        s_abort = 1;
      }
      phase ^= 1u;
      __syncthreads();
      if (s_abort) return;
      fft_p2_io(fbuf, ay, twy, false, RowsIn{rowv, ny}, TimesK{fbuf, kst});
      // the staging buffer is free: fetch the next column's spectrum
      if (threadIdx.x == 0 && k + (int)gridDim.x < ncols) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ptx::mbar_arrive_expect_tx(&kbar, kbytes);
        bulk_load(kst, Kspec + (int64_t)(k + gridDim.x) * Ly, kbytes, &kbar);
      }
      fft_p2_io(fbuf, ay, twy, true, BufIO{fbuf}, ToY{Y, ny, ncols, k});
      continue;
    }
    __syncthreads();
    fft_1d<P2>(fbuf, ay, twy, false, scratch);
    // the spectrum column: every thread waits (bounded) for the bulk copy
    if (!ptx::mbar_wait_bounded(&kbar, phase, limit_ns)) {
      atomicOr(&d.st->status, ST_TIMEOUT);
      s_abort = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (s_abort) return;
#pragma unroll
    for (int u = 0; u < kFftValsPerThread; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < Ly) fbuf[fpad(i)] = cmul(fbuf[fpad(i)], kst[i]);
    }
    __syncthreads();
    // the staging buffer is free: fetch the next column's spectrum
    if (threadIdx.x == 0 && k + (int)gridDim.x < ncols) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ptx::mbar_arrive_expect_tx(&kbar, kbytes);
      bulk_load(kst, Kspec + (int64_t)(k + gridDim.x) * Ly, kbytes, &kbar);
    }
    fft_1d<P2>(fbuf, ay, twy, true, scratch);
    // pair-major: row q's bin k at ((q / 2) ncols + k) 2 + q % 2, so a pair
    // of rows is one contiguous run for the row pass
#pragma unroll
    for (int u = 0; u < kFftValsPerThread; ++u) {
      const int q = threadIdx.x + u * blockDim.x;
      if (q < ny) Y[(((int64_t)(q >> 1) * ncols + k) << 1) + (q & 1)] = fbuf[fpad(q)];
    }
    __syncthreads();
  }
}

struct PairIn {  // Z = Y_q0 + i Y_q1 over the whole length, from the staged half spectra
  const float2* ystg;
  int L;
  bool has1;
  __device__ __forceinline__ float2 load(int i) const {
    const bool lo = 2 * i <= L;
    const int k = lo ? i : L - i;
    float2 a = ystg[2 * k], c = has1 ? ystg[2 * k + 1] : make_float2(0.f, 0.f);
    if (k == 0 || 2 * k == L) a.y = c.y = 0.f;  // real in exact arithmetic
    return lo ? make_float2(a.x - c.y, a.y + c.x) : make_float2(a.x + c.y, c.x - a.y);
  }
};
struct PairOut {  // R <- R0 - S for the pair's image columns; (R q0, R q1) back to buf
  float2* buf;
  float* R;
  float* R0;
  const float* rstg;
  int64_t g0;
  int nx;
  bool bulk, has1;
  __device__ __forceinline__ void store(int x, float2 v) const {
    if (x >= nx) return;
    const float r0 = bulk ? rstg[x] : R0[g0 + x];
    const float r1 = has1 ? (bulk ? rstg[nx + x] : R0[g0 + nx + x]) : 0.f;
    const float a = r0 - v.x, c = r1 - v.y;
    R[g0 + x] = a;
    R0[g0 + x] = a;
    if (has1) {
      R[g0 + nx + x] = c;
      R0[g0 + nx + x] = c;
    }
    buf[fpad(x)] = make_float2(a, c);
  }
};

// Pairs of rows b = blockIdx.x, blockIdx.x + gridDim.x, ... (one CTA per
// SM), rows q0 = 2b and q1 = 2b + 1: their x-axis spectra (one contiguous
// run of Y) extended to length Lx and combined as Z = Y_q0 + i Y_q1; the
// inverse FFT gives row q0 in the real and row q1 in the imaginary part.
// R <- R0 - S, R0 <- R on columns 0 .. nx - 1; each tile's peak of these
// rows into the next-round key; the last CTA closes the round.  The pair's
// spectra and its R0 rows (when nx is a multiple of 4) arrive by bulk
// copies into shared memory issued a pair ahead, overlapping the current
// pair's transform.
template <bool P2>
__global__ void __launch_bounds__(kFftMaxThreads, 1)
    fft_rows_kernel(PlanDev d, FftAxis ax, const float2* __restrict__ twx,
                    const float2* __restrict__ Y, float* __restrict__ R0, int parity,
                    uint64_t limit_ns, int scratch) {
  extern __shared__ __align__(128) unsigned char fsm[];
  const int Lx = ax.L, ncols = Lx / 2 + 1, nx = d.nx, ny = d.ny;
  const int npairs = (ny + 1) / 2;
  float2* ystg = reinterpret_cast<float2*>(fsm);                    // 2 ncols
  float* rstg = reinterpret_cast<float*>(ystg + 2 * ((ncols + 1) & ~1));  // 2 nx
  float2* fbuf = reinterpret_cast<float2*>(rstg + 2 * ((nx + 3) & ~3));
  int32_t* s_cnt = reinterpret_cast<int32_t*>(fbuf + fpad(Lx) + 1);
  int32_t* s_pre = s_cnt + d.T;
  // mixed radix, when the launch made room: the transform's second buffer
  float2* tmp = nullptr;
  if (!P2 && scratch)
    tmp = reinterpret_cast<float2*>(
        (reinterpret_cast<uintptr_t>(s_pre + d.T + 1) + 15) & ~static_cast<uintptr_t>(15));
  __shared__ uint64_t s_warp[2][32];
  __shared__ __align__(8) uint64_t ybar, rbar;
  __shared__ int s_abort;
  const bool bulk_r = (nx & 3) == 0;
  const uint32_t ybytes = (uint32_t)ncols * 16u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nthr = blockDim.x;
  auto issue = [&](int b) {  // thread 0: the pair's spectra and R0 rows
    const int rows = 2 * b + 1 < ny ? 2 : 1;
    ptx::mbar_arrive_expect_tx(&ybar, ybytes);
    bulk_load(ystg, Y + (int64_t)b * ncols * 2, ybytes, &ybar);
    if (bulk_r) {
      ptx::mbar_arrive_expect_tx(&rbar, (uint32_t)(rows * nx) * 4u);
      bulk_load(rstg, R0 + (int64_t)2 * b * nx, (uint32_t)(rows * nx) * 4u, &rbar);
    }
  };
  if (threadIdx.x == 0) {
    s_abort = *(volatile int32_t*)&d.st->status != 0;
    ptx::mbar_init(&ybar, 1);
    ptx::mbar_init(&rbar, 1);
    ptx::fence_barrier_init();
    if (!s_abort && (int)blockIdx.x < npairs) issue(blockIdx.x);
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int b = blockIdx.x; b < npairs && !s_abort; b += gridDim.x) {
    const int q0 = 2 * b, q1 = q0 + 1;
    const bool has1 = q1 < ny;
    if (!ptx::mbar_wait_bounded(&ybar, phase, limit_ns)) {
      atomicOr(&d.st->status, ST_TIMEOUT);
      s_abort = 1;
    }
    if (P2 && bulk_r && !ptx::mbar_wait_bounded(&rbar, phase, limit_ns)) {
      atomicOr(&d.st->status, ST_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();
    if (s_abort) break;
    const int64_t g0 = (int64_t)q0 * nx;
    if (P2) {
      // the pair's spectrum feeds the first stage, the subtraction takes the
      // last stage's outputs
      fft_p2_io(fbuf, ax, twx, true, PairIn{ystg, Lx, has1},
                PairOut{fbuf, d.R, R0, rstg, g0, nx, bulk_r, has1});
    }
    for (int k = threadIdx.x; k < ncols && !P2; k += nthr) {
      float2 a = ystg[2 * k], c = has1 ? ystg[2 * k + 1] : make_float2(0.f, 0.f);
      const bool edge = k == 0 || 2 * k == Lx;  // real in exact arithmetic
      if (edge) a.y = c.y = 0.f;
      fbuf[fpad(k)] = make_float2(a.x - c.y, a.y + c.x);
      if (!edge) fbuf[fpad(Lx - k)] = make_float2(a.x + c.y, c.x - a.y);
    }
    if (!P2) {
      __syncthreads();
      fft_1d<P2>(fbuf, ax, twx, true, tmp);
      // R <- R0 - S; the results back into fbuf as (row q0, row q1)
      if (bulk_r && !ptx::mbar_wait_bounded(&rbar, phase, limit_ns)) {
        atomicOr(&d.st->status, ST_TIMEOUT);
        s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
    }
    for (int x = threadIdx.x; x < nx && !P2; x += nthr) {
      const float r0 = bulk_r ? rstg[x] : R0[g0 + x];
      const float r1 = has1 ? (bulk_r ? rstg[nx + x] : R0[g0 + nx + x]) : 0.f;
      const float2 sv = fbuf[fpad(x)];
      const float a = r0 - sv.x, c = r1 - sv.y;
      d.R[g0 + x] = a;
      R0[g0 + x] = a;
      if (has1) {
        d.R[g0 + nx + x] = c;
        R0[g0 + nx + x] = c;
      }
      fbuf[fpad(x)] = make_float2(a, c);
    }
    __syncthreads();
    phase ^= 1u;
    // both staging buffers are free: the next pair's copies
    if (threadIdx.x == 0 && b + (int)gridDim.x < npairs) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(b + gridDim.x);
    }
    // tile rows of q0 and q1
    int t_row0 = 0, t_row1 = 0;
    for (int i = 0; i < d.ty; ++i) {
      const Rect r = tile_rect(i * d.tx, ny, nx, d.ty, d.tx);
      if (q0 >= r.y0 && q0 < r.y1) t_row0 = i;
      if (has1 && q1 >= r.y0 && q1 < r.y1) t_row1 = i;
    }
    for (int j = 0; j < d.tx; ++j) {
      const Rect rc = tile_rect(j, ny, nx, d.ty, d.tx);
      float b0a = -1.f, b0v = 0.f, b1a = -1.f, b1v = 0.f;
      int b0i = 0x7fffffff, b1i = 0x7fffffff;
      for (int x = rc.x0 + threadIdx.x; x < rc.x1; x += nthr) {
        const float2 v = fbuf[fpad(x)];
        const int i0 = (int)g0 + x;
        const float a0 = fabsf(v.x);
        if (a0 > b0a || (a0 == b0a && i0 < b0i)) {
          b0a = a0;
          b0i = i0;
          b0v = v.x;
        }
        if (has1) {
          const int i1 = i0 + nx;
          const float a1 = fabsf(v.y);
          if (a1 > b1a || (a1 == b1a && i1 < b1i)) {
            b1a = a1;
            b1i = i1;
            b1v = v.y;
          }
        }
      }
      uint64_t k0 = b0a >= 0.f ? make_key(b0v, b0i) : 0ull;
      uint64_t k1 = b1a >= 0.f ? make_key(b1v, b1i) : 0ull;
      k0 = warp_max_key(k0);
      k1 = warp_max_key(k1);
      if (lane == 0) {
        s_warp[0][warp] = k0;
        s_warp[1][warp] = k1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t m0 = 0, m1 = 0;
        for (int w = 0; w < nw; ++w) {
          m0 = umax64(m0, s_warp[0][w]);
          m1 = umax64(m1, s_warp[1][w]);
        }
        const int t0 = t_row0 * d.tx + j, t1 = t_row1 * d.tx + j;
        if (has1 && t1 == t0) m0 = umax64(m0, m1), m1 = 0;
        if (m0) atomicMax((unsigned long long*)&d.peak[(parity ^ 1) * d.T + t0], (unsigned long long)m0);
        if (m1) atomicMax((unsigned long long*)&d.peak[(parity ^ 1) * d.T + t1], (unsigned long long)m1);
      }
      __syncthreads();
    }
  }
  close_round_if_last(d, parity, gridDim.x, s_cnt, s_pre);
}

}  // namespace

// Smallest even n >= m whose only prime factors are 2, 3, 5 and 7.
int fft_grid_size(int m) {
  for (int n = std::max(m, 2);; ++n) {
    if (n & 1) continue;
    int r = n;
    for (int f : {2, 3, 5, 7})
      while (r % f == 0) r /= f;
    if (r == 1) return n;
  }
}

bool fft_axis_init(FftAxis* a, int L) {
  if (L < 2 || L > kFftMaxL || (L & 1)) return false;
  FftAxis x{};
  x.L = L;
  int r = L;
  for (int f : {8, 4, 2, 3, 5, 7})
    while (r % f == 0) {
      if (x.nrad == kFftMaxRadices) return false;
      x.rad[x.nrad++] = f;
      r /= f;
    }
  if (r != 1) return false;
  if (L == 2048 || L == 4096 || L == 8192) {  // radix-16 stages, then the rest
    x.p2 = 1;
    x.nrad = 0;
    for (int m = L; m > 1;) {
      const int f = m >= 16 ? 16 : m;
      x.rad[x.nrad++] = f;
      m /= f;
    }
  }
  int off = L, Ns = 1;
  for (int st = 0; st < x.nrad; ++st) {
    x.tw_off[st] = off;
    off += (x.rad[st] == 16 ? 4 : x.rad[st]) * Ns;  // radix 16: w, w^2, w^4, w^8 per k
    Ns *= x.rad[st];
  }
  x.tw_len = off;
  // at most kFftValsPerThread values a thread in every stage (the radix-16
  // path: exactly one butterfly of 16 a thread)
  const int need = (L + kFftValsPerThread - 1) / kFftValsPerThread;
  x.nthr = x.p2 ? L / 16 : std::min(kFftMaxThreads, std::max(128, (need + 31) / 32 * 32));
  *a = x;
  return true;
}

size_t fft_comps_bytes(int64_t n_max) {
  return sizeof(int4) * (size_t)(1 + n_max) + 2 * sizeof(int) * (size_t)n_max;
}

size_t fft_smem_bytes(int L) { return sizeof(float2) * ((size_t)L + (size_t)L / 32 + 2); }

cudaError_t fft_make_twiddles(float2* d_tw, const FftAxis& a, cudaStream_t s) {
  std::vector<float2> h((size_t)a.tw_len);
  const double two_pi = 6.283185307179586476925286766559;
  auto root = [&](int64_t t, int64_t n) {  // exp(-2 pi i t / n)
    const double ang = two_pi * (double)t / (double)n;
    return make_float2((float)std::cos(ang), (float)-std::sin(ang));
  };
  for (int t = 0; t < a.L; ++t) h[(size_t)t] = root(t, a.L);
  int Ns = 1;
  for (int st = 0; st < a.nrad; ++st) {
    const int R = a.rad[st];
    if (R == 16) {
      for (int k = 0; k < Ns; ++k)
        for (int e = 0; e < 4; ++e)
          h[(size_t)a.tw_off[st] + 4 * (size_t)k + e] = root((int64_t)k << e, (int64_t)Ns * R);
    } else {
      for (int r = 0; r < R; ++r)
        for (int k = 0; k < Ns; ++k)
          h[(size_t)a.tw_off[st] + (size_t)r * Ns + k] = root((int64_t)r * k, (int64_t)Ns * R);
    }
    Ns *= R;
  }
  cudaError_t e = cudaMemcpyAsync(d_tw, h.data(), sizeof(float2) * (size_t)a.tw_len,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // h goes out of scope
  return e;
}

cudaError_t fft_build_psf_spectrum(const PlanDev& d, const FftAxis& ay, const FftAxis& ax,
                                   const float2* twy, const float2* twx, float2* Kspec,
                                   cudaStream_t s) {
  if (ax.p2)
    fft_psf_rows_kernel<true><<<ay.L / 2, ax.nthr, fft_smem_bytes(ax.L), s>>>(d, ax, ay.L, twx, Kspec);
  else
    fft_psf_rows_kernel<false><<<ay.L / 2, ax.nthr, 2 * fft_smem_bytes(ax.L), s>>>(d, ax, ay.L, twx, Kspec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const float scale = (float)(1.0 / ((double)ay.L * (double)ax.L));
  if (ay.p2)
    fft_psf_cols_kernel<true><<<ax.L / 2 + 1, ay.nthr, fft_smem_bytes(ay.L), s>>>(ay, twy, Kspec, scale);
  else
    fft_psf_cols_kernel<false><<<ax.L / 2 + 1, ay.nthr, 2 * fft_smem_bytes(ay.L), s>>>(ay, twy, Kspec, scale);
  return cudaGetLastError();
}

cudaError_t fft_feedback_round(const PlanDev& d, const FftAxis& ay, const FftAxis& ax,
                               const float2* twy, const float2* twx, const float2* Kspec,
                               float2* Y, int4* comps, float* R0, int parity, cudaStream_t s) {
  const int64_t n_max = (int64_t)d.T * d.cap_round;
  int* lead = reinterpret_cast<int*>(comps + 1 + n_max);
  int* bucket = lead + n_max;
  const size_t csmem = sizeof(int32_t) * (2 * (size_t)d.T + 2 + 2 * (size_t)d.ny +
                                          (size_t)std::min<int64_t>(n_max, kCompSmem));
  fft_comp_list_kernel<<<1, kCompThreads, csmem, s>>>(d, comps, lead, bucket);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ncols = ax.L / 2 + 1;
  const int grid = std::min(ncols, fft_sm_count());
  // the spectrum column, the transform, then the radix-16 path's component
  // rows or the mixed-radix path's second buffer
  const size_t cs = sizeof(float2) * (size_t)ay.L + fft_smem_bytes(ay.L) +
                    (ay.p2 ? sizeof(float2) * (size_t)d.ny : fft_smem_bytes(ay.L));
  if (ay.p2)
    fft_cols_kernel<true><<<grid, ay.nthr, cs, s>>>(d, ay, ax.L, comps, lead, twx, twy, Kspec, Y,
                                                    kFftWaitNs);
  else
    fft_cols_kernel<false><<<grid, ay.nthr, cs, s>>>(d, ay, ax.L, comps, lead, twx, twy, Kspec, Y,
                                                     kFftWaitNs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int npairs = (d.ny + 1) / 2;
  const int rgrid = std::min(npairs, fft_sm_count());
  size_t smem = sizeof(float2) * 2 * (size_t)((ncols + 1) & ~1) +
                sizeof(float) * 2 * (size_t)((d.nx + 3) & ~3) + fft_smem_bytes(ax.L) +
                sizeof(int32_t) * (2 * (size_t)d.T + 1);
  if (ax.p2) {
    fft_rows_kernel<true><<<rgrid, ax.nthr, smem, s>>>(d, ax, twx, Y, R0, parity, kFftWaitNs, 0);
    return cudaGetLastError();
  }
  // mixed radix: a second transform buffer after the counters when it fits
  // under the device's per-block limit (all but the largest lengths)
  int scratch = 0;
  {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    const size_t need = ((smem + 15) & ~(size_t)15) + fft_smem_bytes(ax.L);
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ==
            cudaSuccess &&
        cudaFuncGetAttributes(&fa, (const void*)fft_rows_kernel<false>) == cudaSuccess &&
        need + fa.sharedSizeBytes <= (size_t)optin) {
      smem = need;
      scratch = 1;
    }
    cudaGetLastError();
  }
  fft_rows_kernel<false><<<rgrid, ax.nthr, smem, s>>>(d, ax, twx, Y, R0, parity, kFftWaitNs,
                                                      scratch);
  return cudaGetLastError();
}

cudaError_t fft_prepare() {
  const void* fns[] = {(const void*)fft_psf_rows_kernel<true>, (const void*)fft_psf_rows_kernel<false>,
                       (const void*)fft_psf_cols_kernel<true>, (const void*)fft_psf_cols_kernel<false>,
                       (const void*)fft_cols_kernel<true>,     (const void*)fft_cols_kernel<false>,
                       (const void*)fft_rows_kernel<true>,     (const void*)fft_rows_kernel<false>,
                       (const void*)fft_comp_list_kernel};
  cudaError_t e = cudaSuccess;
  for (const void* f : fns)
    if (e == cudaSuccess) e = allow_max_smem(f);
  return e;
}

}  // namespace cleangb
