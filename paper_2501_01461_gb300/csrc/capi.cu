// C ABI of libcleangb.so (declared in include/cleangb.h): plan state,
// argument checks, the round loop and the status conventions.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cleangb_internal.cuh"

using namespace cleangb;

namespace {

std::atomic<int64_t> g_alloc_limit{-1};

constexpr int64_t kResidentMaxBytes = 200 * 1024;  // residual rows per CTA in smem
constexpr int kMaxBeamRadius = 64;
constexpr int64_t kDefaultSpinNs = 2000000000ll;
// FFT feedback cost model of AUTO: seconds per spectrum cell and per round's
// launches, fitted to GB300 rounds on 2048- and 8192-point grids (0.087 and
// 0.665 ms); grids off the radix-16 path take the mixed-radix kernels, about
// kFftMixedFactor times slower per cell
constexpr double kFftCellS = 18e-12;
constexpr double kFftLaunchS = 48e-6;
constexpr double kFftMixedFactor = 2.5;

}  // namespace

struct clean_plan_s {
  clean_params p{};
  int device = 0;
  int sm_count = 0;
  PlanDev d{};
  MinorCfg mc{};       // plain-load minor loop
  MinorCfg mc_pipe{};  // bulk-copy pipeline minor loop (valid when pipe_ok)
  bool pipe_ok = false;      // image rows 16-byte aligned and the pipeline fits
  bool psf_aligned = false;  // PSF base and row pitch 16-byte aligned
  int minor_path = 0;        // 0 auto, 1 plain loads, 2 pipeline
  int pipe_chunk_px = 0;     // pipeline tuning (0: defaults)
  int pipe_stages = 0;
  bool tmem_allowed = true;  // CLEAN_DEBUG_MINOR_TMEM
  bool pair_allowed = true;  // CLEAN_DEBUG_MINOR_PAIR
  int max_rows = 0, max_w = 0;  // largest CTA slab of the minor loop
  float* psf_own = nullptr;
  bool psf_set = false;
  int psf_status = CLEAN_OK;
  int poisoned = CLEAN_OK;
  bool started = false;
  bool pending = false;
  int parity = 0;
  int64_t rounds_launched = 0;
  DevState* h_st = nullptr;
  float* beam_buf = nullptr;
  std::vector<void*> allocs;
  // launch accounting and optional per-launch CUDA-event timing
  int64_t kernel_launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;  // pairs: [2i] start, [2i+1] stop
  std::vector<int> ev_kind;          // 0 minor, 1 feedback, per used pair
  int64_t minor_launches = 0, feedback_launches = 0;
  double minor_ms = 0.0, feedback_ms = 0.0;
  // PSF tensor map for the TMA feedback kernel (valid when psf_map_ok)
  CUtensorMap psf_map{};
  bool psf_map_ok = false;
  // residual and PSF tensor maps with the pipelined minor loop's box
  CUtensorMap r_map{}, p_map_minor{};
  bool pipe_maps_ok = false;
  // FFT feedback (feedback_mode FFT, or AUTO when it is estimated faster)
  bool fft = false;
  int Ly = 0, Lx = 0;
  FftAxis fft_ay{}, fft_ax{};
  float2* fft_twy = nullptr;  // twiddle tables exp(-2 pi i t / L) of both axes
  float2* fft_twx = nullptr;
  float2* fft_K = nullptr;    // PSF kernel spectrum, (Lx/2 + 1) x Ly
  float2* fft_Y = nullptr;    // round work area, (Lx/2 + 1) x ny rounded up to even
  int4* fft_comps = nullptr;  // round work area: the round's components
  float* R0 = nullptr;        // residual at the start of the current round
  int feedback_path = 0;  // 0 auto, 1 plain loads, 2 TMA
  // two rounds (minor + feedback, twice) captured as a CUDA graph, one per
  // starting parity, together with the launch configuration they captured
  struct GraphKey {
    PlanDev d;
    MinorCfg mc;
    CUtensorMap r_map, p_map, psf_map;
    int32_t pipe, fb_path, tma, apply;
  };
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pair[2] = {nullptr, nullptr};
  GraphKey pair_key[2];
  bool use_graphs = true;
  bool graphs_refused = false;
  int64_t graph_launches = 0;
  // phases of the last clean_deconvolve_host call: events before the input
  // copies, after them, after the run, after the output copies
  cudaEvent_t host_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double host_ms[3] = {0.0, 0.0, 0.0};  // inputs in, run, outputs out
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// CLEANGB_FORCE_FEEDBACK=gather|fft|auto overrides a plan's feedback_mode
// (for experiments without code changes); anything else leaves it alone.
int forced_feedback_mode(int mode) {
  const char* v = std::getenv("CLEANGB_FORCE_FEEDBACK");
  if (!v) return mode;
  if (std::strcmp(v, "gather") == 0) return CLEAN_FB_GATHER;
  if (std::strcmp(v, "fft") == 0) return CLEAN_FB_FFT;
  if (std::strcmp(v, "auto") == 0) return CLEAN_FB_AUTO;
  return mode;
}

int poison(clean_plan_s* pl, int code) {
  if (pl->poisoned == CLEAN_OK) pl->poisoned = code;
  return pl->poisoned;
}

int cuda_fail(clean_plan_s* pl, cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return poison(pl, CLEAN_ERR_CUDA);
}

bool finite_pos(float v) { return std::isfinite(v); }

int max_extent(int n, int parts) {
  int m = 0;
  for (int i = 0; i < parts; ++i)
    m = std::max(m, (int)(((int64_t)(i + 1) * n) / parts - ((int64_t)i * n) / parts));
  return m;
}

// Event pair for one timed launch (created on first use, reused after).
int timed_begin(clean_plan_s* pl, int kind, cudaStream_t s) {
  if (!pl->timing) return -1;
  const size_t i = pl->ev_kind.size();
  while (pl->ev_pool.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    pl->ev_pool.push_back(e);
  }
  pl->ev_kind.push_back(kind);
  cudaEventRecord(pl->ev_pool[2 * i], s);
  return (int)i;
}

void timed_end(clean_plan_s* pl, int i, cudaStream_t s) {
  if (i >= 0) cudaEventRecord(pl->ev_pool[2 * i + 1], s);
}

// Folds the durations of completed timed launches into the totals (called
// after a synchronisation).
void timed_collect(clean_plan_s* pl) {
  for (size_t i = 0; i < pl->ev_kind.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pl->ev_pool[2 * i], pl->ev_pool[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (pl->ev_kind[i] == 0) {
      pl->minor_ms += ms;
      ++pl->minor_launches;
    } else {
      pl->feedback_ms += ms;
      ++pl->feedback_launches;
    }
  }
  pl->ev_kind.clear();
}

// Reads the device control block into the pinned mirror (synchronises).
int read_state(clean_plan_s* pl, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(pl->h_st, pl->d.st, sizeof(DevState),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  timed_collect(pl);
  if (pl->h_st->status & ST_TIMEOUT) return poison(pl, CLEAN_ERR_TIMEOUT);
  return CLEAN_OK;
}

// PSF kernel spectrum for the FFT feedback (after every PSF change).
int fft_prepare_psf(clean_plan_s* pl, cudaStream_t s) {
  if (!pl->fft) return CLEAN_OK;
  cudaError_t e = fft_build_psf_spectrum(pl->d, pl->fft_ay, pl->fft_ax, pl->fft_twy, pl->fft_twx,
                                         pl->fft_K, s);
  pl->kernel_launches += 2;
  if (e != cudaSuccess) return cuda_fail(pl, e);
  return CLEAN_OK;
}

// Tensor maps for the pipelined minor loop (box = its chunk geometry).
void refresh_pipe_maps(clean_plan_s* pl) {
  const MinorCfg& q = pl->mc_pipe;
  pl->pipe_maps_ok =
      pl->pipe_ok && pl->d.R && pl->d.P &&
      make_box_tensor_map(&pl->p_map_minor, pl->d.P, pl->d.pny, pl->d.pnx, q.box_w, q.chunk_h) &&
      (q.resident || make_box_tensor_map(&pl->r_map, pl->d.R, pl->d.ny, pl->d.nx, q.box_w,
                                         q.chunk_h));
}

int check_psf(clean_plan_s* pl, cudaStream_t s) {
  pl->psf_map_ok = make_psf_tensor_map(&pl->psf_map, pl->d.P, pl->d.pny, pl->d.pnx);
  pl->psf_aligned = (reinterpret_cast<uintptr_t>(pl->d.P) & 15u) == 0 && (pl->d.pnx % 4) == 0;
  refresh_pipe_maps(pl);
  cudaError_t e = cudaMemsetAsync(pl->d.st, 0, sizeof(DevState), s);
  if (e == cudaSuccess) e = launch_validate_psf(pl->d, s);
  ++pl->kernel_launches;
  if (e != cudaSuccess) return cuda_fail(pl, e);
  int rc = read_state(pl, s);
  if (rc != CLEAN_OK) return rc;
  const int bits = pl->h_st->status;
  pl->psf_set = true;
  pl->psf_status = (bits & ST_NONFINITE_PSF)   ? CLEAN_ERR_NONFINITE
                   : (bits & ST_PSF_OFFCENTRE) ? CLEAN_ERR_INVALID_ARG
                                               : CLEAN_OK;
  pl->started = false;  // a run's state refers to the old PSF
  if (pl->psf_status == CLEAN_OK && (rc = fft_prepare_psf(pl, s)) != CLEAN_OK) return rc;
  return pl->psf_status;
}

// One FFT feedback: scatter the round's components, convolve with the PSF
// through the cached spectrum, R <- R0 - S everywhere, next peaks, close.
cudaError_t launch_fft_feedback(clean_plan_s* pl, cudaStream_t s) {
  pl->kernel_launches += 2;  // component list and columns (the caller counts the rows)
  return plan_fft_round(pl, pl->d, pl->parity, s);
}

int launch_round_feedback(clean_plan_s* pl, cudaStream_t s) {
  const int apply = feedback_on(pl->d) ? 1 : 0;
  if (apply && pl->fft) {
    const int ev = timed_begin(pl, 1, s);
    cudaError_t e = launch_fft_feedback(pl, s);
    timed_end(pl, ev, s);
    ++pl->kernel_launches;
    if (e != cudaSuccess) return cuda_fail(pl, e);
    pl->parity ^= 1;
    pl->pending = false;
    ++pl->rounds_launched;
    return CLEAN_OK;
  }
  const bool use_tma = pl->psf_map_ok && pl->feedback_path != 1;
  const int ev = timed_begin(pl, 1, s);
  cudaError_t e = launch_feedback(pl->d, use_tma ? &pl->psf_map : nullptr, pl->parity, apply,
                                  (uint64_t)pl->mc.spin_limit_ns, s);
  timed_end(pl, ev, s);
  ++pl->kernel_launches;
  if (e != cudaSuccess) return cuda_fail(pl, e);
  pl->parity ^= 1;
  pl->pending = false;
  ++pl->rounds_launched;
  return CLEAN_OK;
}

// Minor-loop variant for this plan.  Automatic choice, from GB300
// measurements: the TMA pipeline whenever the slab is streamed (it wins for
// every streamed tile shape measured), plain loads for resident slabs.
bool use_pipe(const clean_plan_s* pl) {
  if (!pl->pipe_ok || !pl->pipe_maps_ok || !pl->psf_aligned || pl->minor_path == 1) return false;
  if (pl->minor_path == 2) return true;
  return !pl->mc_pipe.resident;
}

int launch_round_minor(clean_plan_s* pl, cudaStream_t s) {
  const bool pipe = use_pipe(pl);
  const int ev = timed_begin(pl, 0, s);
  cudaError_t e = launch_minor(pl->d, pipe ? pl->mc_pipe : pl->mc, pl->parity, &pl->r_map,
                               &pl->p_map_minor, s);
  timed_end(pl, ev, s);
  ++pl->kernel_launches;
  if (e != cudaSuccess) return cuda_fail(pl, e);
  pl->pending = true;
  return CLEAN_OK;
}

// ---- CUDA-graph replay of two rounds --------------------------------------

void drop_graphs(clean_plan_s* pl) {
  for (cudaGraphExec_t& g : pl->pair)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

clean_plan_s::GraphKey graph_key(const clean_plan_s* pl) {
  clean_plan_s::GraphKey k;
  std::memset(&k, 0, sizeof(k));
  const bool pipe = use_pipe(pl);
  k.d = pl->d;
  k.mc = pipe ? pl->mc_pipe : pl->mc;
  k.r_map = pl->r_map;
  k.p_map = pl->p_map_minor;
  k.psf_map = pl->psf_map;
  k.pipe = pipe ? 1 : 0;
  k.fb_path = pl->feedback_path;
  k.tma = (pl->psf_map_ok && pl->feedback_path != 1) ? 1 : 0;
  k.apply = feedback_on(pl->d) ? 1 : 0;
  return k;
}

// One round (minor loop of parity q, then its feedback) on stream s.
cudaError_t launch_round_pair_part(const clean_plan_s* pl, const clean_plan_s::GraphKey& k,
                                   int q, cudaStream_t s) {
  cudaError_t e = launch_minor(k.d, k.mc, q, &k.r_map, &k.p_map, s);
  if (e != cudaSuccess) return e;
  return launch_feedback(k.d, k.tma ? &k.psf_map : nullptr, q, k.apply,
                         (uint64_t)pl->mc.spin_limit_ns, s);
}

bool capture_pair(clean_plan_s* pl, int par, const clean_plan_s::GraphKey& k) {
  if (!pl->cap_stream &&
      cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t l = launch_round_pair_part(pl, k, par, pl->cap_stream);
    if (l == cudaSuccess) l = launch_round_pair_part(pl, k, par ^ 1, pl->cap_stream);
    e = cudaStreamEndCapture(pl->cap_stream, &graph);
    if (l != cudaSuccess) e = l;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->pair[par], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    pl->pair[par] = nullptr;
    cudaGetLastError();
    return false;
  }
  pl->pair_key[par] = k;
  return true;
}

bool graphs_usable(const clean_plan_s* pl) {
  return pl->use_graphs && !pl->graphs_refused && !pl->timing && !pl->fft && !pl->pending;
}

// Two rounds from the graph of the current parity (captured, or recaptured
// when the launch configuration changed).  Returns CLEAN_OK, an error, or
// -1 when graphs are refused (the caller launches directly).
int launch_pair(clean_plan_s* pl, cudaStream_t s) {
  const clean_plan_s::GraphKey k = graph_key(pl);
  const int par = pl->parity;
  if (!pl->pair[par] || std::memcmp(&k, &pl->pair_key[par], sizeof(k)) != 0) {
    if (pl->pair[par]) {
      cudaGraphExecDestroy(pl->pair[par]);
      pl->pair[par] = nullptr;
    }
    if (!capture_pair(pl, par, k)) {
      pl->graphs_refused = true;
      return -1;
    }
  }
  const cudaError_t e = cudaGraphLaunch(pl->pair[par], s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  pl->kernel_launches += 4;
  pl->rounds_launched += 2;
  ++pl->graph_launches;
  return CLEAN_OK;
}

int start_run(clean_plan_s* pl, const float* d_dirty, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl->d.peak, 0, sizeof(uint64_t) * 2 * pl->d.T, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d.st, 0, sizeof(DevState), s);
  // grid-barrier key slots start with mark bit 63 set (see exchange_keys)
  if (e == cudaSuccess)
    e = cudaMemsetAsync(pl->d.gkeys, 0x80, sizeof(uint64_t) * 4 * (size_t)pl->d.T * pl->mc.G, s);
  if (e == cudaSuccess) e = launch_init(pl->d, d_dirty, pl->p.niter, s);
  ++pl->kernel_launches;
  if (e == cudaSuccess && pl->d.trigger > 0.f) {
    e = launch_first_level(pl->d, s);
    ++pl->kernel_launches;
  }
  if (e == cudaSuccess && pl->fft)
    e = cudaMemcpyAsync(pl->R0, pl->d.R, sizeof(float) * (size_t)pl->d.ny * pl->d.nx,
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  pl->started = true;
  pl->pending = false;
  pl->parity = 0;
  pl->rounds_launched = 0;
  return CLEAN_OK;
}

// Tile pairs (see minor_loop.cu): streamed rows in grid groups, an even
// number of tiles, each at least two chunks wide (both column halves hold a
// chunk), and at most 128 CTAs a tile (the pair's 2G exchange slots are
// polled by one warp).
bool pair_ok(const clean_plan_s* pl, const MinorCfg& q) {
  if (!pl->pair_allowed || q.resident || q.sync != CLEAN_SYNC_GRID || q.G > 128) return false;
  const int T = pl->p.tiles_y * pl->p.tiles_x;
  if (T < 2 || (T % 2) != 0) return false;
  for (int j = 0; j < pl->p.tiles_x; ++j) {
    const int w = (int)(((int64_t)(j + 1) * pl->p.nx) / pl->p.tiles_x -
                        ((int64_t)j * pl->p.nx) / pl->p.tiles_x);
    if (w < 2 * q.chunk_w) return false;
  }
  return true;
}

// Pipeline geometry for the plan's group: resident slab when it fits beside
// the ring, else streamed rows.
bool configure_pipe(clean_plan_s* pl) {
  MinorCfg q = pl->mc;
  q.resident = 1;
  bool ok = minor_pipe_geometry(q, pl->max_rows, pl->max_w, pl->pipe_chunk_px, pl->pipe_stages);
  if (!ok) {
    q = pl->mc;
    q.resident = 0;
    ok = minor_pipe_geometry(q, pl->max_rows, pl->max_w, pl->pipe_chunk_px, pl->pipe_stages);
  }
  if (ok) {
    if (!pl->tmem_allowed) q.tmem = 0;
    q.pair = pair_ok(pl, q) ? 1 : 0;
    pl->mc_pipe = q;
  }
  return ok;
}

// Whether every CTA of a tensor-memory configuration keeps its leading
// chunks in TMEM: the PSF array holds every window of every tile pixel.
bool tmem_in_use(const clean_plan_s* pl) {
  if (!pl->mc_pipe.tmem) return false;
  int maxH = 0, maxW = 0;
  for (int i = 0; i < pl->d.ty; ++i)
    maxH = std::max(maxH, (int)(((int64_t)(i + 1) * pl->d.ny) / pl->d.ty -
                                ((int64_t)i * pl->d.ny) / pl->d.ty));
  for (int j = 0; j < pl->d.tx; ++j)
    maxW = std::max(maxW, (int)(((int64_t)(j + 1) * pl->d.nx) / pl->d.tx -
                                ((int64_t)j * pl->d.nx) / pl->d.tx));
  return pl->d.cy >= maxH - 1 && pl->d.pny - pl->d.cy >= maxH && pl->d.cx >= maxW - 1 &&
         pl->d.pnx - pl->d.cx >= maxW;
}

int common_checks(clean_plan_s* pl) {
  if (!pl) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  if (!pl->psf_set) return CLEAN_ERR_INVALID_ARG;
  if (pl->psf_status != CLEAN_OK) return pl->psf_status;
  return CLEAN_OK;
}

int run_rounds(clean_plan_s* pl, int32_t max_rounds, cudaStream_t s) {
  int rc;
  if (pl->pending && (rc = launch_round_feedback(pl, s)) != CLEAN_OK) return rc;
  if ((rc = read_state(pl, s)) != CLEAN_OK) return rc;
  if (pl->h_st->status & ST_NONFINITE_DIRTY) {
    pl->started = false;
    return CLEAN_ERR_NONFINITE;
  }
  int64_t done = 0;
  while (max_rounds < 0 || done < max_rounds) {
    if (!pl->h_st->active) break;
    int64_t chunk = 1;
    if (pl->d.K > 0) chunk = (pl->h_st->max_budget + pl->d.K - 1) / pl->d.K;
    chunk = std::max<int64_t>(chunk, 1);
    if (max_rounds >= 0) chunk = std::min<int64_t>(chunk, max_rounds - done);
    NvtxRange range("clean_rounds");
    for (int64_t i = 0; i < chunk;) {
      if (chunk - i >= 2 && graphs_usable(pl)) {
        rc = launch_pair(pl, s);
        if (rc == CLEAN_OK) {
          i += 2;
          continue;
        }
        if (rc != -1) return rc;
      }
      if ((rc = launch_round_minor(pl, s)) != CLEAN_OK) return rc;
      if ((rc = launch_round_feedback(pl, s)) != CLEAN_OK) return rc;
      ++i;
    }
    done += chunk;
    if ((rc = read_state(pl, s)) != CLEAN_OK) return rc;
  }
  return CLEAN_OK;
}

}  // namespace

namespace cleangb {

PlanDev plan_device_state(const clean_plan_s* pl) { return pl->d; }

bool plan_psf_tensor_map(const clean_plan_s* pl, CUtensorMap* out) {
  if (!pl->psf_map_ok) return false;
  *out = pl->psf_map;
  return true;
}

int64_t plan_niter(const clean_plan_s* pl) { return pl->p.niter; }

bool plan_uses_fft(const clean_plan_s* pl) { return pl->fft; }

cudaError_t plan_fft_start(clean_plan_s* pl, const PlanDev& d, cudaStream_t s) {
  return cudaMemcpyAsync(pl->R0, d.R, sizeof(float) * (size_t)d.ny * d.nx,
                         cudaMemcpyDeviceToDevice, s);
}

cudaError_t plan_fft_round(clean_plan_s* pl, const PlanDev& d, int parity, cudaStream_t s) {
  return fft_feedback_round(d, pl->fft_ay, pl->fft_ax, pl->fft_twy, pl->fft_twx, pl->fft_K,
                            pl->fft_Y, pl->fft_comps, pl->R0, parity, s);
}

}  // namespace cleangb

extern "C" {

int clean_params_default(clean_params* p) {
  if (!p) return CLEAN_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->gain = 0.1f;
  p->threshold = 0.f;
  p->tiles_y = p->tiles_x = 1;
  p->feedback_interval = 0;
  p->feedback_mode = CLEAN_FB_GATHER;
  p->mode = CLEAN_TILED;
  p->group_ctas = 0;
  p->group_sync = CLEAN_SYNC_AUTO;
  return CLEAN_OK;
}

int clean_params_check(const clean_params* p) {
  if (!p) return CLEAN_ERR_INVALID_ARG;
  if (p->ny < 1 || p->nx < 1 || p->psf_ny < 1 || p->psf_nx < 1) return CLEAN_ERR_INVALID_ARG;
  if ((int64_t)p->ny * p->nx >= 0x7fffffffll) return CLEAN_ERR_INVALID_ARG;
  if ((int64_t)p->psf_ny * p->psf_nx >= 0x7fffffffll) return CLEAN_ERR_INVALID_ARG;
  if (!finite_pos(p->gain) || !(p->gain > 0.f) || !(p->gain <= 1.f)) return CLEAN_ERR_INVALID_ARG;
  if (!finite_pos(p->threshold) || !(p->threshold >= 0.f)) return CLEAN_ERR_INVALID_ARG;
  if (p->niter < 0 || p->niter > (int64_t)1 << 40) return CLEAN_ERR_INVALID_ARG;
  if (p->tiles_y < 1 || p->tiles_x < 1 || p->tiles_y > 64 || p->tiles_x > 64 ||
      p->tiles_y > p->ny || p->tiles_x > p->nx)
    return CLEAN_ERR_INVALID_ARG;
  if (p->feedback_interval < 0) return CLEAN_ERR_INVALID_ARG;
  if (p->feedback_mode != CLEAN_FB_GATHER && p->feedback_mode != CLEAN_FB_FFT &&
      p->feedback_mode != CLEAN_FB_AUTO)
    return CLEAN_ERR_INVALID_ARG;
  if (p->mode != CLEAN_TILED && p->mode != CLEAN_UNTILED_GRID) return CLEAN_ERR_INVALID_ARG;
  if (p->mode == CLEAN_UNTILED_GRID && (p->tiles_y != 1 || p->tiles_x != 1))
    return CLEAN_ERR_INVALID_ARG;
  if (p->group_ctas < 0 || p->group_ctas > 1024) return CLEAN_ERR_INVALID_ARG;
  if (p->group_sync != CLEAN_SYNC_AUTO && p->group_sync != CLEAN_SYNC_CLUSTER &&
      p->group_sync != CLEAN_SYNC_GRID)
    return CLEAN_ERR_INVALID_ARG;
  if (p->group_sync == CLEAN_SYNC_CLUSTER && p->group_ctas > 16) return CLEAN_ERR_INVALID_ARG;
  if (!std::isfinite(p->feedback_trigger) || !(p->feedback_trigger >= 0.f) ||
      !(p->feedback_trigger < 1.f))
    return CLEAN_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (p->reserved[i] != 0) return CLEAN_ERR_INVALID_ARG;
  return CLEAN_OK;
}

void clean_debug_alloc_limit(int64_t bytes) { g_alloc_limit.store(bytes); }

void clean_destroy(clean_plan_t pl) {
  if (!pl) return;
  {
    DeviceGuard g(pl->device);
    cudaDeviceSynchronize();
    drop_graphs(pl);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    for (void* a : pl->allocs) cudaFree(a);
    for (cudaEvent_t e : pl->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : pl->host_ev)
      if (e) cudaEventDestroy(e);
    if (pl->h_st) cudaFreeHost(pl->h_st);
    cudaGetLastError();
  }
  delete pl;
}

int clean_plan(clean_plan_t* out, const clean_params* p, const float* d_psf, void* stream) {
  if (!out) return CLEAN_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = clean_params_check(p);
  if (rc != CLEAN_OK) return rc;


  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  clean_plan_s* pl = new (std::nothrow) clean_plan_s();
  if (!pl) return CLEAN_ERR_OOM;
  pl->p = *p;
  pl->device = dev;
  pl->sm_count = sms;
  cudaStream_t s = as_stream(stream);

  const int T = p->tiles_y * p->tiles_x;
  const int maxH = max_extent(p->ny, p->tiles_y);
  const int maxW = max_extent(p->nx, p->tiles_x);
  const int threads = minor_threads();

  // ---- minor-loop group: G CTAs per tile, cluster or grid barrier ----
  MinorCfg& mc = pl->mc;
  mc.threads = threads;
  mc.spin_limit_ns = kDefaultSpinNs;
  mc.force_timeout = 0;
  int sync = p->group_sync;
  int G = p->group_ctas;
  if (p->mode == CLEAN_UNTILED_GRID) {
    sync = CLEAN_SYNC_GRID;
    if (G == 0) G = sms;
  } else {
    const int per = std::max(1, sms / T);
    const int64_t tile_px = (int64_t)maxH * maxW;
    // A grid-synchronised group needs all T * G CTAs resident (one per SM).
    // Measured on GB300 (plain Hogbom, 256^2 to 4096^2): tiles of up to 2^17
    // pixels run fastest as one 16-CTA cluster (256^2: 3.3 us per iteration
    // vs 5.8 with 152 grid CTAs, the exchange dominating); larger tiles on a
    // grid group of about one CTA per 8192 pixels, at most SMs / T (512^2:
    // 32 CTAs, 5.3 us; 1024^2 and up: all SMs).  Grids with more tiles than
    // SMs use clusters.
    if (sync == CLEAN_SYNC_AUTO) {
      if (T > sms)
        sync = CLEAN_SYNC_CLUSTER;
      else if (tile_px <= (int64_t)1 << 17 && 16 * T <= sms && G == 0)
        sync = CLEAN_SYNC_CLUSTER;
      else
        sync = CLEAN_SYNC_GRID;
    }
    if (G == 0) {
      if (sync == CLEAN_SYNC_GRID) {
        G = (int)std::min<int64_t>(per, std::max<int64_t>(1, (tile_px + 8191) / 8192));
      } else {
        G = 1;
        while (G * 2 <= std::min(per, 16)) G *= 2;
      }
    }
  }
  G = std::max(1, std::min(G, maxH));
  auto slab_bytes = [&](int g) { return (int64_t)((maxH + g - 1) / g) * maxW * 4; };
  // both minor-loop variants for group size g: plain loads, and the
  // bulk-copy pipeline (resident slab if it fits beside the ring)
  auto configure = [&](int g) {
    mc.sync = sync;
    mc.G = g;
    mc.pipe = 0;
    mc.resident = slab_bytes(g) <= kResidentMaxBytes ? 1 : 0;
    mc.smem = mc.resident ? (int)slab_bytes(g) : 0;
    pl->max_rows = (maxH + g - 1) / g;
    pl->max_w = maxW;
    pl->pipe_ok = configure_pipe(pl) && (p->nx % 4) == 0;
  };
  configure(G);
  if (sync == CLEAN_SYNC_CLUSTER) {
    for (;;) {
      bool fits = minor_max_cluster_ctas(mc.G, mc.resident, mc.smem, threads) >= 1;
      if (fits && pl->pipe_ok)
        fits = minor_max_cluster_ctas(mc.G, pl->mc_pipe.resident, pl->mc_pipe.smem,
                                      pl->mc_pipe.threads) >= 1;
      if (fits) break;
      if (p->group_ctas != 0 || mc.G == 1) {
        delete pl;
        return mc.G == 1 ? CLEAN_ERR_CUDA : CLEAN_ERR_INVALID_ARG;
      }
      configure(mc.G / 2);
    }
  }
  if (minor_prepare(mc) != cudaSuccess || (pl->pipe_ok && minor_prepare(pl->mc_pipe) != cudaSuccess) ||
      feedback_prepare(T) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return CLEAN_ERR_CUDA;
  }
  if (sync == CLEAN_SYNC_GRID && (int64_t)T * mc.G > sms) {
    // a grid-synchronised launch needs every CTA resident (one per SM)
    delete pl;
    return CLEAN_ERR_INVALID_ARG;
  }

  // ---- device state ----
  const int64_t npix = (int64_t)p->ny * p->nx;
  const int64_t per_tile_max = p->niter / T + (p->niter % T ? 1 : 0);
  int64_t cap_round = p->feedback_interval > 0
                          ? std::min<int64_t>(p->feedback_interval, per_tile_max)
                          : per_tile_max;
  cap_round = std::max<int64_t>(cap_round, 1);
  if (cap_round * T > 0x7fffffffll) {
    delete pl;
    return CLEAN_ERR_INVALID_ARG;
  }
  const int64_t list_cap = std::max<int64_t>(p->niter, 1);
  struct Req {
    void** dst;
    size_t bytes;
  };
  // FFT feedback: a grid of at least (2 ny - 1) x (2 nx - 1) so the circular
  // convolution never wraps onto an image pixel.  AUTO takes it when a round's
  // gather (about 0.21 ns per pixel-component update on GB300) would cost more
  // than the transforms (estimated per spectrum cell, plus the launches).
  // Grids longer than kFftMaxL per axis are not served.
  const bool fb_on = (p->feedback_interval > 0 || p->feedback_trigger > 0.f) && T > 1;
  const int fb_mode = forced_feedback_mode(p->feedback_mode);
  pl->Ly = fft_grid_size(2 * p->ny - 1);
  pl->Lx = fft_grid_size(2 * p->nx - 1);
  const bool fft_ok = fft_axis_init(&pl->fft_ay, pl->Ly) && fft_axis_init(&pl->fft_ax, pl->Lx);
  if (fb_on && fb_mode == CLEAN_FB_FFT) {
    if (!fft_ok) {
      delete pl;
      return CLEAN_ERR_UNSUPPORTED;
    }
    pl->fft = true;
  }
  if (fb_on && fb_mode == CLEAN_FB_AUTO && fft_ok) {
    const double comps =
        (double)(p->feedback_interval > 0 ? std::min<int64_t>(p->feedback_interval, per_tile_max)
                                          : per_tile_max) * T;
    const double gather_s = comps * ((double)npix - (double)npix / T) * 0.21e-9;
    const double per_cell = kFftCellS * (pl->fft_ay.p2 && pl->fft_ax.p2 ? 1.0 : kFftMixedFactor);
    const double fft_s = (double)pl->Ly * (pl->Lx / 2 + 1) * per_cell + kFftLaunchS;
    pl->fft = fft_s < gather_s;
  }
  const size_t spec_bytes = sizeof(float2) * (size_t)pl->Ly * (pl->Lx / 2 + 1);
  const int beam_n = (2 * kMaxBeamRadius + 1) * (2 * kMaxBeamRadius + 1);
  std::vector<Req> req = {
      {(void**)&pl->d.R, sizeof(float) * (size_t)npix},
      {(void**)&pl->d.model, sizeof(float) * (size_t)npix},
      {(void**)&pl->d.budget, sizeof(int64_t) * (size_t)T},
      {(void**)&pl->d.peak, sizeof(uint64_t) * 2 * (size_t)T},
      {(void**)&pl->d.rcount, sizeof(int32_t) * (size_t)T},
      {(void**)&pl->d.rcomps, sizeof(clean_component) * (size_t)(cap_round * T)},
      {(void**)&pl->d.list, sizeof(clean_component) * (size_t)list_cap},
      {(void**)&pl->d.round_off, sizeof(int64_t) * (size_t)(list_cap + 1)},
      // 2 slot sets x T tiles x 2G slots (tile pairs exchange over 2G CTAs)
      {(void**)&pl->d.gkeys, sizeof(uint64_t) * 4 * (size_t)T * (size_t)mc.G},
      {(void**)&pl->d.gbar, sizeof(uint32_t) * (size_t)T},
      {(void**)&pl->d.st, sizeof(DevState)},
      {(void**)&pl->beam_buf, sizeof(float) * (size_t)beam_n},
  };
  if (!d_psf) req.push_back({(void**)&pl->psf_own, sizeof(float) * (size_t)p->psf_ny * p->psf_nx});
  if (pl->fft) {
    req.push_back({(void**)&pl->fft_K, spec_bytes});
    // pair-major rows: room for a whole last pair when ny is odd
    req.push_back({(void**)&pl->fft_Y,
                   sizeof(float2) * (size_t)(pl->Lx / 2 + 1) * (size_t)(p->ny + (p->ny & 1))});
    req.push_back({(void**)&pl->fft_comps, fft_comps_bytes(cap_round * T)});
    req.push_back({(void**)&pl->fft_twy, sizeof(float2) * (size_t)pl->fft_ay.tw_len});
    req.push_back({(void**)&pl->fft_twx, sizeof(float2) * (size_t)pl->fft_ax.tw_len});
    req.push_back({(void**)&pl->R0, sizeof(float) * (size_t)npix});
  }
  size_t total = 0;
  for (auto& r : req) total += r.bytes;
  const int64_t lim = g_alloc_limit.load();
  if (lim >= 0 && (int64_t)total > lim) {
    delete pl;
    return CLEAN_ERR_OOM;
  }
  for (auto& r : req) {
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, r.bytes) != cudaSuccess) {
      cudaGetLastError();
      clean_destroy(pl);
      return CLEAN_ERR_OOM;
    }
    pl->allocs.push_back(ptr);
    *r.dst = ptr;
  }
  if (cudaMallocHost((void**)&pl->h_st, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    clean_destroy(pl);
    return CLEAN_ERR_OOM;
  }
  std::memset(pl->h_st, 0, sizeof(DevState));

  PlanDev& d = pl->d;
  d.P = d_psf ? d_psf : pl->psf_own;
  d.ny = p->ny;
  d.nx = p->nx;
  d.pny = p->psf_ny;
  d.pnx = p->psf_nx;
  d.cy = p->psf_ny / 2;
  d.cx = p->psf_nx / 2;
  d.ty = p->tiles_y;
  d.tx = p->tiles_x;
  d.T = T;
  d.gain = p->gain;
  d.thr = p->threshold;
  d.K = p->feedback_interval;
  d.trigger = p->feedback_trigger;
  d.cap_round = (int32_t)cap_round;

  if (pl->fft && (fft_make_twiddles(pl->fft_twy, pl->fft_ay, s) != cudaSuccess ||
                  fft_make_twiddles(pl->fft_twx, pl->fft_ax, s) != cudaSuccess)) {
    cudaGetLastError();
    clean_destroy(pl);
    return CLEAN_ERR_CUDA;
  }
  if (cudaMemsetAsync(d.gbar, 0, sizeof(uint32_t) * T, s) != cudaSuccess ||
      cudaMemsetAsync(d.st, 0, sizeof(DevState), s) != cudaSuccess) {
    cudaGetLastError();
    clean_destroy(pl);
    return CLEAN_ERR_CUDA;
  }
  refresh_pipe_maps(pl);
  if (d_psf) {
    rc = check_psf(pl, s);
    if (rc != CLEAN_OK) {
      clean_destroy(pl);
      return rc;
    }
  }
  *out = pl;
  return CLEAN_OK;
}

int clean_set_psf(clean_plan_t pl, const float* psf, int32_t on_host, void* stream) {
  if (!pl || !psf) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  if (on_host) {
    if (!pl->psf_own) return CLEAN_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(pl->psf_own, psf,
                                    sizeof(float) * (size_t)pl->d.pny * pl->d.pnx,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(pl, e);
  } else {
    if (pl->psf_own) return CLEAN_ERR_INVALID_ARG;
    pl->d.P = psf;
  }
  return check_psf(pl, s);
}

int clean_run(clean_plan_t pl, const float* d_dirty, int32_t max_rounds, void* stream) {
  int rc = common_checks(pl);
  if (rc != CLEAN_OK) return rc;
  if (max_rounds < -1) return CLEAN_ERR_INVALID_ARG;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  if (d_dirty) {
    if ((rc = start_run(pl, d_dirty, s)) != CLEAN_OK) return rc;
  } else if (!pl->started) {
    return CLEAN_ERR_INVALID_ARG;
  }
  return run_rounds(pl, max_rounds, s);
}

int clean_step(clean_plan_t pl, void* stream) {
  int rc = common_checks(pl);
  if (rc != CLEAN_OK) return rc;
  if (!pl->started) return CLEAN_ERR_INVALID_ARG;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  if (pl->pending && (rc = launch_round_feedback(pl, s)) != CLEAN_OK) return rc;
  return launch_round_minor(pl, s);
}

int clean_feedback(clean_plan_t pl, void* stream) {
  int rc = common_checks(pl);
  if (rc != CLEAN_OK) return rc;
  if (!pl->started) return CLEAN_ERR_INVALID_ARG;
  if (!pl->pending) return CLEAN_OK;
  DeviceGuard g(pl->device);
  return launch_round_feedback(pl, as_stream(stream));
}

int clean_restore(clean_plan_t pl, float bmaj, float bmin, float bpa, float* d_out,
                  void* stream) {
  int rc = common_checks(pl);
  if (rc != CLEAN_OK) return rc;
  if (!pl->started || !d_out) return CLEAN_ERR_INVALID_ARG;
  if (!std::isfinite(bmaj) || !std::isfinite(bmin) || !std::isfinite(bpa) || !(bmin > 0.f) ||
      !(bmaj >= bmin))
    return CLEAN_ERR_INVALID_ARG;
  const double smaj = (double)bmaj / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  const int r = (int)std::floor(5.0 * smaj);
  if (r > kMaxBeamRadius) return CLEAN_ERR_UNSUPPORTED;
  DeviceGuard g(pl->device);
  cudaError_t e = launch_restore_with(pl->d, bmaj, bmin, bpa, pl->beam_buf, r, d_out,
                                      as_stream(stream));
  pl->kernel_launches += 2;
  if (e != cudaSuccess) return cuda_fail(pl, e);
  return CLEAN_OK;
}

int clean_get(clean_plan_t pl, float* d_residual_out, float* d_model_out,
              clean_component* d_comps_out, int64_t comps_cap, int64_t* n_comps,
              void* stream) {
  if (!pl) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  if (!pl->started) return CLEAN_ERR_INVALID_ARG;
  if (d_comps_out && comps_cap < 0) return CLEAN_ERR_INVALID_ARG;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  const size_t img = sizeof(float) * (size_t)pl->d.ny * pl->d.nx;
  cudaError_t e = cudaSuccess;
  if (d_residual_out) e = cudaMemcpyAsync(d_residual_out, pl->d.R, img, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_model_out)
    e = cudaMemcpyAsync(d_model_out, pl->d.model, img, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  if (d_comps_out || n_comps) {
    int rc = read_state(pl, s);
    if (rc != CLEAN_OK) return rc;
    const int64_t n = pl->h_st->total;
    if (n_comps) *n_comps = n;
    if (d_comps_out) {
      const int64_t m = std::min(n, comps_cap);
      if (m > 0) {
        e = cudaMemcpyAsync(d_comps_out, pl->d.list, sizeof(clean_component) * (size_t)m,
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(pl, e);
      }
    }
  }
  return CLEAN_OK;
}

int clean_get_rounds(clean_plan_t pl, int64_t* h_offsets, int64_t cap, int64_t* n_rounds,
                     void* stream) {
  if (!pl) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  if (!pl->started || (h_offsets && cap < 0)) return CLEAN_ERR_INVALID_ARG;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  int rc = read_state(pl, s);
  if (rc != CLEAN_OK) return rc;
  const int64_t n = pl->h_st->n_rounds;
  if (n_rounds) *n_rounds = n;
  if (h_offsets && cap > 0 && n > 0) {
    const int64_t m = std::min(n, cap);
    cudaError_t e = cudaMemcpyAsync(h_offsets, pl->d.round_off, sizeof(int64_t) * (size_t)m,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(pl, e);
  }
  return CLEAN_OK;
}

// ---- checkpoint / resume ---------------------------------------------------

namespace {

constexpr uint64_t kCkptMagic = 0x31544b50424c4743ull;  // bytes "CGLBPKT1"
constexpr int32_t kCkptVersion = 1;

struct CkptHeader {
  uint64_t magic;
  int32_t version;
  int32_t parity;
  clean_params params;
  int64_t rounds_launched;
  int64_t total;     // components in the list
  int64_t n_rounds;  // recorded rounds (list offsets)
  int64_t npix;
  int64_t T;
  int64_t bytes;     // the whole checkpoint
};

int64_t ckpt_bytes(int64_t npix, int64_t T, int64_t total, int64_t n_rounds) {
  return (int64_t)sizeof(CkptHeader) + 2 * npix * (int64_t)sizeof(float) +
         total * (int64_t)sizeof(clean_component) + n_rounds * (int64_t)sizeof(int64_t) +
         T * (int64_t)(sizeof(int64_t) + 2 * sizeof(uint64_t) + sizeof(int32_t)) +
         (int64_t)sizeof(DevState);
}

// (device pointer, bytes) of each checkpoint section after the header, in order.
std::vector<std::pair<void*, size_t>> ckpt_sections(clean_plan_s* pl, int64_t total,
                                                    int64_t n_rounds) {
  const size_t npix = (size_t)pl->d.ny * pl->d.nx, T = (size_t)pl->d.T;
  return {{pl->d.R, sizeof(float) * npix},
          {pl->d.model, sizeof(float) * npix},
          {pl->d.list, sizeof(clean_component) * (size_t)total},
          {pl->d.round_off, sizeof(int64_t) * (size_t)n_rounds},
          {pl->d.budget, sizeof(int64_t) * T},
          {pl->d.peak, sizeof(uint64_t) * 2 * T},
          {pl->d.rcount, sizeof(int32_t) * T},
          {pl->d.st, sizeof(DevState)}};
}

}  // namespace

int clean_checkpoint(clean_plan_t pl, void* h_buf, int64_t capacity, int64_t* bytes,
                     void* stream) {
  if (!pl || !bytes || (h_buf && capacity < 0)) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  if (!pl->started || pl->pending) return CLEAN_ERR_INVALID_ARG;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  int rc = read_state(pl, s);
  if (rc != CLEAN_OK) return rc;
  const DevState st = *pl->h_st;
  const int64_t npix = (int64_t)pl->d.ny * pl->d.nx;
  const int64_t need = ckpt_bytes(npix, pl->d.T, st.total, st.n_rounds);
  *bytes = need;
  if (!h_buf) return CLEAN_OK;
  if (capacity < need) return CLEAN_ERR_INVALID_ARG;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kCkptMagic;
  h.version = kCkptVersion;
  h.parity = pl->parity;
  h.params = pl->p;
  h.rounds_launched = pl->rounds_launched;
  h.total = st.total;
  h.n_rounds = st.n_rounds;
  h.npix = npix;
  h.T = pl->d.T;
  h.bytes = need;
  std::memcpy(h_buf, &h, sizeof(h));
  unsigned char* out = static_cast<unsigned char*>(h_buf) + sizeof(h);
  cudaError_t e = cudaSuccess;
  for (const auto& sec : ckpt_sections(pl, st.total, st.n_rounds)) {
    if (sec.second && e == cudaSuccess)
      e = cudaMemcpyAsync(out, sec.first, sec.second, cudaMemcpyDeviceToHost, s);
    out += sec.second;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  return CLEAN_OK;
}

int clean_resume(clean_plan_t pl, const void* h_buf, int64_t bytes, void* stream) {
  if (!pl || !h_buf || bytes < (int64_t)sizeof(CkptHeader)) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  CkptHeader h;
  std::memcpy(&h, h_buf, sizeof(h));
  const int64_t npix = (int64_t)pl->d.ny * pl->d.nx;
  if (h.magic != kCkptMagic || h.version != kCkptVersion || h.npix != npix ||
      h.T != pl->d.T || std::memcmp(&h.params, &pl->p, sizeof(clean_params)) != 0 ||
      h.total < 0 || h.total > pl->p.niter || h.n_rounds < 0 || h.n_rounds > h.total ||
      (h.parity != 0 && h.parity != 1) || h.bytes != bytes ||
      ckpt_bytes(npix, h.T, h.total, h.n_rounds) != bytes)
    return CLEAN_ERR_INVALID_ARG;
  if (!pl->psf_set) return CLEAN_ERR_INVALID_ARG;
  if (pl->psf_status != CLEAN_OK) return pl->psf_status;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  const unsigned char* in = static_cast<const unsigned char*>(h_buf) + sizeof(h);
  cudaError_t e = cudaSuccess;
  for (const auto& sec : ckpt_sections(pl, h.total, h.n_rounds)) {
    if (sec.second && e == cudaSuccess)
      e = cudaMemcpyAsync(sec.first, in, sec.second, cudaMemcpyHostToDevice, s);
    in += sec.second;
  }
  // the grid exchange restarts its count; its key slots start marked
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d.gbar, 0, sizeof(uint32_t) * pl->d.T, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(pl->d.gkeys, 0x80, sizeof(uint64_t) * 4 * (size_t)pl->d.T * pl->mc.G, s);
  if (e == cudaSuccess && pl->fft)
    e = cudaMemcpyAsync(pl->R0, pl->d.R, sizeof(float) * (size_t)npix, cudaMemcpyDeviceToDevice,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host buffer may go now
  if (e != cudaSuccess) return cuda_fail(pl, e);
  pl->started = true;
  pl->pending = false;
  pl->parity = h.parity;
  pl->rounds_launched = h.rounds_launched;
  return read_state(pl, s);
}

int clean_deconvolve_host(clean_plan_t pl, const float* h_dirty, const float* h_psf,
                          float* h_residual, float* h_model, clean_component* h_comps,
                          int64_t comps_cap, int64_t* n_comps, void* stream) {
  if (!pl || !h_dirty) return CLEAN_ERR_INVALID_ARG;
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  DeviceGuard g(pl->device);
  cudaStream_t s = as_stream(stream);
  int rc;
  cudaError_t e = cudaSuccess;
  for (cudaEvent_t& ev : pl->host_ev)
    if (!ev && e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess) e = cudaEventRecord(pl->host_ev[0], s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  if (h_psf) {
    if ((rc = clean_set_psf(pl, h_psf, 1, stream)) != CLEAN_OK) return rc;
  }
  if ((rc = common_checks(pl)) != CLEAN_OK) return rc;
  const size_t img = sizeof(float) * (size_t)pl->d.ny * pl->d.nx;
  // the dirty image lands in the residual buffer; set-up copies it in place
  e = cudaMemcpyAsync(pl->d.R, h_dirty, img, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(pl->host_ev[1], s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  if ((rc = start_run(pl, pl->d.R, s)) != CLEAN_OK) return rc;
  if ((rc = run_rounds(pl, -1, s)) != CLEAN_OK) return rc;
  e = cudaEventRecord(pl->host_ev[2], s);
  if (e == cudaSuccess && h_residual)
    e = cudaMemcpyAsync(h_residual, pl->d.R, img, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && h_model)
    e = cudaMemcpyAsync(h_model, pl->d.model, img, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(pl, e);
  const int64_t n = pl->h_st->total;  // read by run_rounds' last status read
  if (n_comps) *n_comps = n;
  if (h_comps && comps_cap > 0 && n > 0) {
    e = cudaMemcpyAsync(h_comps, pl->d.list,
                        sizeof(clean_component) * (size_t)std::min(n, comps_cap),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(pl, e);
  }
  e = cudaEventRecord(pl->host_ev[3], s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pl->host_ev[i], pl->host_ev[i + 1]);
    pl->host_ms[i] = ms;
  }
  if (e != cudaSuccess) return cuda_fail(pl, e);
  return CLEAN_OK;
}

int clean_stats(clean_plan_t pl, clean_stats_t* out, void* stream) {
  if (!pl || !out) return CLEAN_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  const bool pipe = use_pipe(pl);
  out->group_ctas = pl->mc.G;
  out->group_sync = pl->mc.sync;
  out->resident = pipe ? pl->mc_pipe.resident : pl->mc.resident;
  out->minor_pipe = pipe ? 1 : 0;
  out->minor_tmem = (pipe && tmem_in_use(pl)) ? 1 : 0;
  out->minor_pairs = (pipe && pl->mc_pipe.pair) ? 1 : 0;
  out->feedback_mode = pl->fft ? CLEAN_FB_FFT : CLEAN_FB_GATHER;
  out->feedback_tma =
      (pl->psf_map_ok && pl->feedback_path != 1) ? 1 : 0;
  out->sm_count = pl->sm_count;
  out->rounds_launched = pl->rounds_launched;
  out->kernel_launches = pl->kernel_launches;
  out->host_in_ms = pl->host_ms[0];
  out->host_run_ms = pl->host_ms[1];
  out->host_out_ms = pl->host_ms[2];
  if (pl->poisoned != CLEAN_OK) return pl->poisoned;
  if (!pl->started) return CLEAN_OK;
  DeviceGuard g(pl->device);
  int rc = read_state(pl, as_stream(stream));
  if (rc != CLEAN_OK) return rc;
  out->n_components = pl->h_st->total;
  out->rounds = pl->h_st->n_rounds;
  out->minor_launches = pl->minor_launches;
  out->feedback_launches = pl->feedback_launches;
  out->minor_ms = pl->minor_ms;
  out->feedback_ms = pl->feedback_ms;
  out->graph_launches = pl->graph_launches;
  return CLEAN_OK;
}

int clean_debug_set(clean_plan_t pl, int32_t what, int64_t value) {
  if (!pl) return CLEAN_ERR_INVALID_ARG;
  switch (what) {
    case CLEAN_DEBUG_SPIN_LIMIT_NS:
      if (value < 1) return CLEAN_ERR_INVALID_ARG;
      pl->mc.spin_limit_ns = pl->mc_pipe.spin_limit_ns = value;
      return CLEAN_OK;
    case CLEAN_DEBUG_FORCE_TIMEOUT:
      pl->mc.force_timeout = pl->mc_pipe.force_timeout = value ? 1 : 0;
      return CLEAN_OK;
    case CLEAN_DEBUG_MINOR_PATH:
      if (value < 0 || value > 2) return CLEAN_ERR_INVALID_ARG;
      pl->minor_path = (int)value;
      return CLEAN_OK;
    case CLEAN_DEBUG_PIPE_CHUNK_PX:
    case CLEAN_DEBUG_PIPE_STAGES: {
      if (value < 0 || value > (1 << 20)) return CLEAN_ERR_INVALID_ARG;
      const int old_chunk = pl->pipe_chunk_px, old_stages = pl->pipe_stages;
      const MinorCfg old_cfg = pl->mc_pipe;
      if (what == CLEAN_DEBUG_PIPE_CHUNK_PX)
        pl->pipe_chunk_px = (int)value;
      else
        pl->pipe_stages = (int)value;
      DeviceGuard g(pl->device);
      bool ok = configure_pipe(pl);
      if (ok && pl->mc.sync == CLEAN_SYNC_CLUSTER)
        ok = minor_max_cluster_ctas(pl->mc_pipe.G, pl->mc_pipe.resident, pl->mc_pipe.smem,
                                    pl->mc_pipe.threads) >= 1;
      if (ok) ok = minor_prepare(pl->mc_pipe) == cudaSuccess;
      if (ok) refresh_pipe_maps(pl);
      if (!ok) {
        cudaGetLastError();
        pl->pipe_chunk_px = old_chunk;
        pl->pipe_stages = old_stages;
        pl->mc_pipe = old_cfg;
        return CLEAN_ERR_INVALID_ARG;
      }
      return CLEAN_OK;
    }
    case CLEAN_DEBUG_MINOR_PAIR: {
      if (value < 0 || value > 1) return CLEAN_ERR_INVALID_ARG;
      const bool old_allowed = pl->pair_allowed;
      pl->pair_allowed = value != 0;
      if (!pl->pipe_ok) return CLEAN_OK;
      const MinorCfg old_cfg = pl->mc_pipe;
      DeviceGuard g(pl->device);
      bool ok = configure_pipe(pl) && minor_prepare(pl->mc_pipe) == cudaSuccess;
      // pairs exchange over 2G slots a tile: a changed layout restarts the
      // exchange count with every slot marked (as at a run's start)
      if (ok && pl->mc_pipe.pair != old_cfg.pair)
        ok = cudaDeviceSynchronize() == cudaSuccess &&
             cudaMemset(pl->d.gkeys, 0x80, sizeof(uint64_t) * 4 * (size_t)pl->d.T * pl->mc.G) ==
                 cudaSuccess &&
             cudaMemset(pl->d.gbar, 0, sizeof(uint32_t) * (size_t)pl->d.T) == cudaSuccess &&
             cudaDeviceSynchronize() == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        pl->pair_allowed = old_allowed;
        pl->mc_pipe = old_cfg;
        return CLEAN_ERR_INVALID_ARG;
      }
      return CLEAN_OK;
    }
    case CLEAN_DEBUG_MINOR_TMEM: {
      if (value < 0 || value > 1) return CLEAN_ERR_INVALID_ARG;
      const bool old_allowed = pl->tmem_allowed;
      pl->tmem_allowed = value != 0;
      if (!pl->pipe_ok) return CLEAN_OK;
      const MinorCfg old_cfg = pl->mc_pipe;
      DeviceGuard g(pl->device);
      const bool ok = configure_pipe(pl) && minor_prepare(pl->mc_pipe) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        pl->tmem_allowed = old_allowed;
        pl->mc_pipe = old_cfg;
        return CLEAN_ERR_INVALID_ARG;
      }
      return CLEAN_OK;
    }
    case CLEAN_DEBUG_FEEDBACK_PATH:
      if (value < 0 || value > 2) return CLEAN_ERR_INVALID_ARG;
      pl->feedback_path = (int)value;
      return CLEAN_OK;
    case CLEAN_DEBUG_GRAPHS:
      if (value < 0 || value > 1) return CLEAN_ERR_INVALID_ARG;
      pl->use_graphs = value != 0;
      pl->graphs_refused = false;
      return CLEAN_OK;
    case CLEAN_DEBUG_TIMING:
      pl->timing = value != 0;
      pl->ev_kind.clear();
      pl->minor_launches = pl->feedback_launches = 0;
      pl->minor_ms = pl->feedback_ms = 0.0;
      return CLEAN_OK;
    default:
      return CLEAN_ERR_INVALID_ARG;
  }
}

const char* clean_strerror(int status) {
  switch (status) {
    case CLEAN_OK: return "ok";
    case CLEAN_ERR_INVALID_ARG: return "invalid argument";
    case CLEAN_ERR_NONFINITE: return "non-finite value in the dirty image or PSF";
    case CLEAN_ERR_OOM: return "out of device memory";
    case CLEAN_ERR_CUDA: return "CUDA error";
    case CLEAN_ERR_TIMEOUT: return "bounded device wait expired";
    case CLEAN_ERR_UNSUPPORTED: return "unsupported by the library";
    default: return "unknown status";
  }
}

}  // extern "C"
