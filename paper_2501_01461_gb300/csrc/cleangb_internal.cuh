// Internal declarations shared by the kernels and the C-ABI host code of
// libcleangb.so.  Nothing here is part of the public ABI (include/cleangb.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "cleangb.h"

namespace cleangb {

// ---------------------------------------------------------------------------
// Peak keys.  The peak search of Section 3 (first equation) picks the pixel
// of largest |R|, ties to the lowest row-major index.  A pixel is encoded as
// a 64-bit key whose unsigned order is exactly that order:
//   bits 63..32  bit pattern of |R| (monotone in |R| for non-negative floats)
//   bits 31..1   0x7fffffff - index (larger for lower indices)
//   bit  0       sign bit of R, so the signed value is recovered exactly
// Key 0 means "no pixel".  Requires index < 2^31 - 1.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t make_key(float v, int32_t idx) {
  uint32_t bits;
#ifdef __CUDA_ARCH__
  bits = __float_as_uint(v);
#else
  __builtin_memcpy(&bits, &v, 4);
#endif
  uint32_t hi = bits & 0x7fffffffu;
  uint32_t lo = ((0x7fffffffu - (uint32_t)idx) << 1) | (bits >> 31);
  return ((uint64_t)hi << 32) | lo;
}
__host__ __device__ __forceinline__ int32_t key_index(uint64_t k) {
  return (int32_t)(0x7fffffffu - ((uint32_t)k >> 1));
}
__device__ __forceinline__ float key_value(uint64_t k) {
  uint32_t hi = (uint32_t)(k >> 32);
  return __uint_as_float(hi | ((uint32_t)(k & 1u) << 31));
}
__device__ __forceinline__ float key_abs(uint64_t k) {
  return __uint_as_float((uint32_t)(k >> 32));
}

// Tile bounds: tile (i, j) covers rows [floor(i ny / Ty), floor((i+1) ny / Ty))
// and columns likewise (Section 2, Fig. 1; the split of a non-divisible size
// is this library's reading).
struct Rect {
  int32_t y0, y1, x0, x1;
};
__host__ __device__ __forceinline__ Rect tile_rect(int32_t t, int32_t ny,
                                                   int32_t nx, int32_t ty,
                                                   int32_t tx) {
  int32_t i = t / tx, j = t - (t / tx) * tx;
  Rect r;
  r.y0 = (int32_t)(((int64_t)i * ny) / ty);
  r.y1 = (int32_t)(((int64_t)(i + 1) * ny) / ty);
  r.x0 = (int32_t)(((int64_t)j * nx) / tx);
  r.x1 = (int32_t)(((int64_t)(j + 1) * nx) / tx);
  return r;
}

// Status bits (DevState::status).  Sticky for the run.
enum : int32_t {
  ST_NONFINITE_DIRTY = 1,
  ST_NONFINITE_PSF = 2,
  ST_PSF_OFFCENTRE = 4,
  ST_TIMEOUT = 8,
};

// Device-resident control block of a plan.
struct DevState {
  int32_t status;        // ST_* bits
  int32_t active;        // a tile can run in the next round
  uint32_t fb_done;      // feedback blocks finished (last-block pattern)
  int32_t pad0;
  int64_t total;         // components in the list
  int64_t n_rounds;      // rounds recorded (>= 1 component)
  int64_t round_comps;   // components of the last closed round
  int64_t max_budget;    // max over tiles of the remaining budget
  int64_t timeout_where; // diagnostic: tile * 2^32 + barrier index of a timeout
  float level;           // flux-trigger level of the next round (0: none)
  int32_t pad1;
};

// Pointers and sizes every kernel of a plan sees.
struct PlanDev {
  float* R;                 // residual, ny x nx
  float* model;             // model image, ny x nx
  const float* P;           // PSF, pny x pnx
  int32_t ny, nx, pny, pnx, cy, cx;
  int32_t ty, tx, T;        // tile grid and tile count
  float gain, thr;
  int32_t K;                // feedback interval (0 = none)
  float trigger;            // flux trigger (0 = none)
  int32_t cap_round;        // per-tile capacity of the round buffer
  int32_t round0;           // batched runs: the batch round at which this image started
  int64_t* budget;          // [T] remaining iterations per tile
  uint64_t* peak;           // [2][T] peak key per tile, indexed by round parity
  int32_t* rcount;          // [T] components of the current round per tile
  clean_component* rcomps;  // [T][cap_round] current round's components
  clean_component* list;    // [niter] all components, list order
  int64_t* round_off;       // [niter + 1] list offset of each recorded round
  uint64_t* gkeys;          // [2][T * G] per-CTA partial keys (grid sync)
  uint32_t* gbar;           // [T] grid-barrier exchanges done per tile in this run
  DevState* st;
};

// A batched work item: tile `tile` of image `image`.
struct BatchItem {
  int32_t image;
  int32_t tile;
};

// Per-image geometry of a batched feedback launch.
struct BatchImage {
  int32_t block0;    // first flattened block of this image
  int32_t bx, by;    // blocks per tile in x and y
  int32_t nblocks;   // bx * by * T
};

// Minor-loop launch configuration.
struct MinorCfg {
  int32_t G;          // CTAs per tile
  int32_t sync;       // CLEAN_SYNC_CLUSTER or CLEAN_SYNC_GRID
  int32_t resident;   // 1: residual rows live in shared memory for the round
  int32_t threads;    // threads per CTA
  int32_t smem;       // dynamic shared memory bytes
  int64_t spin_limit_ns;
  int32_t force_timeout;
  // bulk-copy pipeline (pipe = 1): rows stream through a ring of `stages`
  // shared-memory buffers, `chunk_rows` rows per buffer
  int32_t pipe;
  int32_t chunk_w;    // columns per chunk (multiple of 4, <= 128)
  int32_t chunk_h;    // rows per chunk
  int32_t box_w;      // TMA box width in floats (chunk_w + 4)
  int32_t stages;
  int32_t res_floats; // resident slab floats (0 when streamed)
  int32_t tmem;       // 1: each CTA's leading full chunks keep their residual
                      // in tensor memory for the launch (streamed pipeline)
  int32_t pair;       // 1: groups of 2G CTAs serve pairs of tiles, alternating
                      // between them (streamed pipeline, grid groups, T even)
};

// Pipeline geometry and shared-memory size for a minor-loop configuration
// (fills the pipe fields of c; returns false if it does not fit).
// chunk_px: target pixels per chunk (0: 4096); max_stages: ring depth cap
// (0: 8).
bool minor_pipe_geometry(MinorCfg& c, int max_rows, int max_w, int chunk_px = 0,
                         int max_stages = 0);

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum.
// The cap is process-wide state of the kernel, so every plan sets the same
// value (setting a plan's own size would break launches of plans that need
// more); each launch still requests only its own size.
inline cudaError_t allow_max_smem(const void* fn) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);  // static shared memory counts too
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  return e;
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_init(const PlanDev& d, const float* dirty, int64_t niter,
                        cudaStream_t s);
cudaError_t launch_validate_psf(const PlanDev& d, cudaStream_t s);
// Flux-trigger level of a run's first round (after launch_init); no-op
// without a trigger.
cudaError_t launch_first_level(const PlanDev& d, cudaStream_t s);
// Whether rounds of this plan end with a feedback.
__host__ __device__ __forceinline__ bool feedback_on(const PlanDev& d) {
  return (d.K > 0 || d.trigger > 0.f) && d.T > 1;
}
// r_map / p_map: 2-D tensor maps of the residual and the PSF with the box
// (c.box_w x c.chunk_h) of a pipelined configuration (ignored otherwise).
cudaError_t launch_minor(const PlanDev& d, const MinorCfg& c, int parity,
                         const CUtensorMap* r_map, const CUtensorMap* p_map, cudaStream_t s);
// Encodes a 2-D float32 tensor map (rows x cols, row pitch cols floats) with
// the given box; false if the base or pitch is not 16-byte aligned.
bool make_box_tensor_map(CUtensorMap* map, const float* base, int rows, int cols, int box_w,
                         int box_h);
bool encode_tensor_map_2d(CUtensorMap* map, const float* base, int rows, int cols, int box_w,
                          int box_h);
cudaError_t minor_prepare(const MinorCfg& c);  // sets function attributes
// G CTAs per item (G = 1: independent CTAs; G > 1: one thread-block cluster
// per item), each reading its image's plan state from `plans` (device
// arrays); resident: each CTA's rows fit `smem` bytes of shared memory.
// Image i runs its round (round - plans[i].round0).
cudaError_t launch_minor_batch(const PlanDev* plans, const BatchItem* items, int n_items,
                               int G, int resident, int smem, int round, cudaStream_t s);
// Largest cluster size <= want that can be scheduled for the batched kernel.
int minor_batch_cluster(int want, int resident, int smem);

// One tile of one image in the persistent batched minor loop: its launch
// configuration (G CTAs with the grid exchange) and the body it takes.
enum { kUnitResident = 0, kUnitTmem = 1, kUnitStreamed = 2, kUnitPair = 3 };
struct BatchUnitItem {
  MinorCfg cfg;
  int32_t image;
  int32_t tile;   // the tile, or for kUnitPair the pair (tiles 2 tile, 2 tile + 1)
  int32_t kind;
  int32_t ranks;  // CTAs of the unit: cfg.G, or 2 cfg.G for a pair
};
// CTAs of the persistent launch with `smem` bytes of dynamic shared memory
// (one per SM; 0 if it cannot be resident).
int minor_batch_persistent_grid(int smem);
// One round of every item: units[w * grid + b] = (item, rank) of CTA b in
// wave w, item -1 idle.  Cooperative launch.
cudaError_t launch_minor_batch_persistent(const PlanDev* plans, const BatchUnitItem* items,
                                          const int2* units, int n_waves, int grid, int smem,
                                          const CUtensorMap* rmaps, const CUtensorMap* pmaps,
                                          int round, cudaStream_t s);

// Batched TMA pipeline: every image's residual and PSF box maps have boxes of
// kBatchBoxW x kBatchBoxRows floats (chunks of 128 columns x 60 rows).
constexpr int kBatchBoxW = 132;
constexpr int kBatchBoxRows = 60;
// Pipeline geometry for a batch group of G CTAs per tile whose CTAs hold at
// most max_rows x max_w pixels (resident in shared memory or streamed);
// false if the ring does not fit.
bool minor_pipe_batch_geometry(MinorCfg& c, int G, int resident, int max_rows, int max_w);
// Largest cluster size <= want (a power of two) the device can schedule for
// the batched pipeline with `smem` bytes of dynamic shared memory (1 if none).
int minor_pipe_batch_cluster(int want, int resident, int smem);
cudaError_t launch_minor_pipe_batch(const PlanDev* plans, const BatchItem* items, int n_items,
                                    const MinorCfg& c, const CUtensorMap* rmaps,
                                    const CUtensorMap* pmaps, int round, cudaStream_t s);
// Feedback for many images in one launch (plain loads, or TMA when maps is
// non-NULL: one PSF tensor map per image in device memory, 64-byte aligned).
cudaError_t launch_feedback_batch(const PlanDev* plans, const BatchImage* imgs, int n_images,
                                  int total_blocks, int max_T, const CUtensorMap* maps,
                                  int round, int apply, uint64_t limit_ns, cudaStream_t s);
// Feedback block grid of one image (blocks per tile in x and y).
void feedback_blocks(const PlanDev& d, bool tma, int* bx, int* by);
int minor_max_cluster_ctas(int G, int resident, int smem, int threads);
// psf_map: a 2-D tensor map of the PSF (box 132 x 32 floats) selects the TMA
// kernel; NULL selects the plain-load kernel.
cudaError_t launch_feedback(const PlanDev& d, const CUtensorMap* psf_map, int parity,
                            int apply, uint64_t limit_ns, cudaStream_t s);
cudaError_t feedback_prepare(int T);
// ---- FFT feedback (fft_feedback.cu) -----------------------------------------
// One axis of the 2-D transforms: length L (even, 7-smooth, <= kFftMaxL),
// its radices in stage order and the threads of a block that transforms it
// (every thread holds at most kFftValsPerThread values in a stage).
constexpr int kFftMaxL = 8192;
constexpr int kFftMaxThreads = 512;
constexpr int kFftMaxRadices = 16;
constexpr int kFftValsPerThread = 16;
struct FftAxis {
  int32_t L, nthr, nrad;
  int32_t rad[kFftMaxRadices];
  // twiddle table: entries [0, L) hold exp(-2 pi i t / L); stage s (radix R,
  // Ns = product of the earlier radices) reads exp(-2 pi i r k / (Ns R)) at
  // tw_off[s] + r Ns + k, so neighbouring lanes read neighbouring entries
  int32_t tw_off[kFftMaxRadices];
  int32_t tw_len;
  int32_t p2;  // 1: L is 2048, 4096 or 8192 and takes the radix-16 path (L / 16 threads)
};
// Smallest even n >= m whose prime factors are 2, 3, 5 and 7.
int fft_grid_size(int m);
// Fills *a for length L; false if L is odd, above kFftMaxL or not 7-smooth.
bool fft_axis_init(FftAxis* a, int L);
// The twiddle table of an axis (a.tw_len float2, layout in FftAxis),
// computed in double precision on the host and copied to d_tw; synchronises s.
cudaError_t fft_make_twiddles(float2* d_tw, const FftAxis& a, cudaStream_t s);
// Bytes of the per-round component work area for up to n_max components.
size_t fft_comps_bytes(int64_t n_max);
// Kernel spectrum Kspec[k][m] (k <= Lx / 2, m < Ly) of the PSF kernel image
// K[d mod L] = P[d + c] (|d| < image size), scaled by 1 / (Ly Lx).
cudaError_t fft_build_psf_spectrum(const PlanDev& d, const FftAxis& ay, const FftAxis& ax,
                                   const float2* twy, const float2* twx, float2* Kspec,
                                   cudaStream_t s);
// One FFT feedback: R <- R0 - (round components (*) PSF) on every pixel,
// R0 <- R, next peaks, round close.  Y: (Lx/2 + 1) x (ny rounded up to
// even) float2 work area;
// comps: fft_comps_bytes(T cap_round) bytes of work area.
cudaError_t fft_feedback_round(const PlanDev& d, const FftAxis& ay, const FftAxis& ax,
                               const float2* twy, const float2* twx, const float2* Kspec,
                               float2* Y, int4* comps, float* R0, int parity, cudaStream_t s);
cudaError_t fft_prepare();  // kernel attributes of the FFT feedback
// Encodes the PSF tensor map for the TMA feedback kernel; false if the PSF's
// address or row pitch is not 16-byte aligned (or the driver lacks TMA).
bool make_psf_tensor_map(CUtensorMap* map, const float* psf, int pny, int pnx);
cudaError_t launch_restore_with(const PlanDev& d, float bmaj, float bmin, float bpa,
                                float* beam_buf, int r, float* out, cudaStream_t s);
int minor_threads();

// Accessors the batch code uses on single-image plans (defined with the C ABI).
PlanDev plan_device_state(const clean_plan_s* pl);
bool plan_psf_tensor_map(const clean_plan_s* pl, CUtensorMap* out);
int64_t plan_niter(const clean_plan_s* pl);
// FFT feedback of a plan on the state `d` (a batch job's copy of the plan's
// device state, with its own control block and round phase).
bool plan_uses_fft(const clean_plan_s* pl);
cudaError_t plan_fft_start(clean_plan_s* pl, const PlanDev& d, cudaStream_t s);
cudaError_t plan_fft_round(clean_plan_s* pl, const PlanDev& d, int parity, cudaStream_t s);

}  // namespace cleangb
