// Many deconvolutions on one GPU at once: fixed batches (clean_batch_*) and
// continuous batching for serving (clean_server_*).
//
// Every resident image's round runs in shared launches.  The minor loops of
// all images whose residual and PSF allow 2-D TMA boxes run in ONE
// persistent launch (one CTA per SM working through a schedule of waves:
// each tile of each image is a unit of G CTAs in one wave, exchanging its
// peaks through the bounded grid exchange; largest tiles first); the other
// images' minor loops run in launches grouped by CTAs per tile and residual
// placement (plain loads, one CTA per small tile, a thread-block cluster per
// large one).  Then one feedback launch covers every image's blocks (two if
// some images need the plain-load feedback).  Each image
// keeps its own round phase (it may have joined later), its own budgets,
// peaks and component list, so its results are bit for bit those of its own
// clean_plan + clean_run.  Images that finish leave the work lists; new ones
// join between rounds.
//
// Rounds are replayed from CUDA graphs: after each rebuild of the work lists
// the launches of two consecutive rounds are captured once per starting
// round parity (kernels only use the round's parity relative to each image's
// first round), and a run of n rounds becomes n / 2 graph launches plus at
// most one directly launched round.  Rounds past an image's end are no-ops,
// so the host can launch an upper bound of rounds between reads.  If the
// capture is refused the engine launches the kernels directly.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "cleangb_internal.cuh"

using namespace cleangb;

namespace {

constexpr int64_t kGroupSmemMax = 200 * 1024;  // resident rows per CTA
constexpr int kMaxUnitG = 32;                   // exchange slots per tile (a pair's 2G CTAs)
// dynamic shared memory floor of the persistent launch: above half an SM, so
// each SM holds one CTA (units that keep residual chunks in tensor memory
// take all of its columns)
constexpr int kPersistSmemMin = 116 * 1024;

struct Job {
  clean_plan_t plan = nullptr;
  PlanDev dev{};
  CUtensorMap map{};
  bool tma = false;
  // residual and PSF box maps of the batched minor-loop pipeline
  CUtensorMap rmap{}, pmap{};
  bool pipe = false;
  // grid-exchange slots of the persistent minor loop: 2 sets x T tiles x
  // kMaxUnitG CTAs, owned by the engine
  uint64_t* bkeys = nullptr;
  // CTAs per tile in the persistent minor loop, fixed from the run's first
  // schedule to its end: the exchange slots of tile t are t G .. t G + G - 1,
  // and the exchange count runs on across rounds (0: not chosen yet)
  int unit_G = 0;
  bool unit_pair = false;  // tile pairs (fixed with unit_G: the slots are laid out by 2G)
  bool fft = false;  // feedback by FFT convolution (the job's own launches)
  int64_t id = 0;
  int slot = 0;
  bool finished = false;
};

struct Group {
  int offset = 0, count = 0;  // into the item array
  int G = 1, resident = 0, smem = 0;
  int pipe = 0;               // 1: TMA pipeline (cfg), 0: plain loads
  int max_rows = 0, max_w = 0;
  MinorCfg cfg{};
};

}  // namespace

// Shared engine behind both APIs.
struct clean_engine_s {
  int device = 0;
  int cap = 0;                          // state slots
  std::vector<Job> jobs;                // resident jobs (finished ones until removed)
  std::vector<int> free_slots;
  DevState* d_states = nullptr;         // [cap] control blocks
  DevState* h_states = nullptr;         // pinned mirror
  PlanDev* d_plans = nullptr;           // [cap] device copies, indexed by work position
  BatchItem* d_items = nullptr;
  int items_cap = 0;
  BatchImage* d_imgs = nullptr;         // [cap] feedback geometry (TMA images first)
  CUtensorMap* d_maps = nullptr;        // [cap]
  CUtensorMap* d_rmaps = nullptr;       // [cap] minor-loop residual boxes
  CUtensorMap* d_pmaps = nullptr;       // [cap] minor-loop PSF boxes
  std::vector<Group> groups;
  int n_work = 0, n_tma = 0, n_gather = 0, blocks_tma = 0, blocks_plain = 0, max_T = 1;
  std::vector<int> fft_work;            // work positions of FFT-feedback jobs
  // persistent minor loop of the pipelined images (n_waves = 0: none)
  BatchUnitItem* d_uitems = nullptr;
  int uitems_cap = 0;
  int2* d_units = nullptr;
  int units_cap = 0;
  int n_waves = 0, p_grid = 0, p_smem = 0;
  std::vector<int> work_jobs;           // job index of each work position
  bool dirty = true;                    // work lists need a rebuild
  int round = 0;                        // rounds launched so far (global)
  int64_t next_id = 1;
  int poisoned = CLEAN_OK;
  int64_t rounds_launched = 0, kernel_launches = 0;
  // CUDA graphs of two rounds, indexed by the parity of the first round
  cudaStream_t cap_stream = nullptr;    // private stream used only for capture
  cudaGraphExec_t pair[2] = {nullptr, nullptr};
  int pair_kernels = 0;                 // kernels in one pair graph
  bool use_graphs = true;
  bool graphs_refused = false;
  int64_t graph_launches = 0;
};

namespace {

int eng_fail(clean_engine_s* e, int code) {
  cudaGetLastError();
  if (e->poisoned == CLEAN_OK) e->poisoned = code;
  return e->poisoned;
}

void drop_graphs(clean_engine_s* e) {
  for (cudaGraphExec_t& g : e->pair)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void engine_free(clean_engine_s* e) {
  if (!e) return;
  cudaDeviceSynchronize();
  drop_graphs(e);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  for (Job& j : e->jobs) {
    clean_destroy(j.plan);
    cudaFree(j.bkeys);
  }
  cudaFree(e->d_uitems);
  cudaFree(e->d_units);
  cudaFree(e->d_states);
  cudaFree(e->d_plans);
  cudaFree(e->d_items);
  cudaFree(e->d_imgs);
  cudaFree(e->d_maps);
  cudaFree(e->d_rmaps);
  cudaFree(e->d_pmaps);
  if (e->h_states) cudaFreeHost(e->h_states);
  cudaGetLastError();
  delete e;
}

int engine_create(clean_engine_s** out, int cap) {
  clean_engine_s* e = new (std::nothrow) clean_engine_s();
  if (!e) return CLEAN_ERR_OOM;
  e->cap = cap;
  cudaGetDevice(&e->device);
  if (cudaMalloc(&e->d_states, sizeof(DevState) * cap) != cudaSuccess ||
      cudaMallocHost(&e->h_states, sizeof(DevState) * cap) != cudaSuccess ||
      cudaMalloc(&e->d_plans, sizeof(PlanDev) * cap) != cudaSuccess ||
      cudaMalloc(&e->d_imgs, sizeof(BatchImage) * cap) != cudaSuccess ||
      cudaMalloc(&e->d_maps, sizeof(CUtensorMap) * cap) != cudaSuccess ||
      cudaMalloc(&e->d_rmaps, sizeof(CUtensorMap) * cap) != cudaSuccess ||
      cudaMalloc(&e->d_pmaps, sizeof(CUtensorMap) * cap) != cudaSuccess) {
    engine_free(e);
    return CLEAN_ERR_OOM;
  }
  std::memset(e->h_states, 0, sizeof(DevState) * cap);
  for (int i = cap - 1; i >= 0; --i) e->free_slots.push_back(i);
  *out = e;
  return CLEAN_OK;
}

// Starts (or restarts) a job's run from a dirty image: control block and
// peaks cleared, set-up kernel on `s`; the job's rounds count from now.
int engine_start(clean_engine_s* e, Job& j, const float* d_dirty, cudaStream_t s) {
  j.dev.round0 = e->round;
  j.finished = false;
  j.unit_G = 0;
  j.unit_pair = false;
  cudaError_t err = cudaMemsetAsync(j.dev.st, 0, sizeof(DevState), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(j.dev.peak, 0, sizeof(uint64_t) * 2 * j.dev.T, s);
  if (err == cudaSuccess) err = launch_init(j.dev, d_dirty, plan_niter(j.plan), s);
  ++e->kernel_launches;
  if (err == cudaSuccess) err = launch_first_level(j.dev, s);
  if (err == cudaSuccess && j.fft) err = plan_fft_start(j.plan, j.dev, s);
  // the persistent minor loop's exchange slots start marked (bit 63 set), as
  // in a single plan's run; set-up zeroed the exchange counts
  if (err == cudaSuccess && j.bkeys)
    err = cudaMemsetAsync(j.bkeys, 0x80, sizeof(uint64_t) * 2 * (size_t)j.dev.T * kMaxUnitG, s);
  if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
  std::memset(&e->h_states[j.slot], 0, sizeof(DevState));
  e->h_states[j.slot].active = 1;  // refreshed at the next status read
  e->dirty = true;
  return CLEAN_OK;
}

// Creates a job's plan (its device state) in a free slot.
int engine_register(clean_engine_s* e, const clean_params* p, const float* d_psf, Job** out,
                    cudaStream_t s) {
  if (e->free_slots.empty()) return CLEAN_ERR_OOM;
  int rc = clean_params_check(p);
  if (rc != CLEAN_OK) return rc;
  if (!d_psf || p->mode != CLEAN_TILED) return CLEAN_ERR_INVALID_ARG;
  Job j;
  rc = clean_plan(&j.plan, p, d_psf, s);
  if (rc != CLEAN_OK) return rc;
  j.fft = plan_uses_fft(j.plan);
  j.slot = e->free_slots.back();
  e->free_slots.pop_back();
  j.dev = plan_device_state(j.plan);
  j.dev.st = e->d_states + j.slot;
  j.tma = plan_psf_tensor_map(j.plan, &j.map);
  // the minor-loop pipeline needs box maps over the residual and the PSF
  j.pipe = p->ny >= kBatchBoxRows && p->psf_ny >= kBatchBoxRows && p->nx >= kBatchBoxW &&
           p->psf_nx >= kBatchBoxW &&
           make_box_tensor_map(&j.pmap, d_psf, p->psf_ny, p->psf_nx, kBatchBoxW, kBatchBoxRows) &&
           make_box_tensor_map(&j.rmap, j.dev.R, p->ny, p->nx, kBatchBoxW, kBatchBoxRows);
  if (j.pipe) {
    if (cudaMalloc(&j.bkeys, sizeof(uint64_t) * 2 * (size_t)j.dev.T * kMaxUnitG) != cudaSuccess) {
      cudaGetLastError();
      e->free_slots.push_back(j.slot);
      clean_destroy(j.plan);
      return CLEAN_ERR_OOM;
    }
    j.dev.gkeys = j.bkeys;
  }
  j.id = e->next_id++;
  j.finished = true;  // not running until started
  e->jobs.push_back(j);
  *out = &e->jobs.back();
  return CLEAN_OK;
}

// CTAs per tile for a tile of h x w pixels: the fewest (a power of two up to
// 16) whose row slabs fit in shared memory; 16 streamed CTAs if none does.
void tile_group(int h, int w, int* G, int* resident, int* smem) {
  for (int g = 1; g <= 16; g *= 2) {
    const int64_t slab = (int64_t)((h + g - 1) / g) * w * 4;
    if (slab <= kGroupSmemMax) {
      *G = g;
      *resident = 1;
      *smem = (int)slab;
      return;
    }
  }
  *G = 16;
  *resident = 0;
  *smem = 0;
}

// CTAs per tile for the batched pipeline: the fewest power-of-two CTAs
// (<= 16) whose row slabs fit in shared memory beside a ring of at least two
// PSF boxes, and, when `fast`, at least one CTA per 8192 pixels (each
// iteration's pass stays short, as in the single-plan choice); else 16 CTAs
// streaming their rows.  The group's geometry is checked once the group's
// largest slab is known.
void pipe_tile_group(int h, int w, bool fast, int* G, int* resident, int* rows) {
  int g0 = 1;
  while (fast && g0 < 16 && (int64_t)g0 * 8192 < (int64_t)h * w) g0 *= 2;
  for (int g = g0; g <= 16; g *= 2) {
    MinorCfg c;
    const int r = (h + g - 1) / g;
    if (minor_pipe_batch_geometry(c, g, 1, r, w)) {
      *G = g;
      *resident = 1;
      *rows = r;
      return;
    }
  }
  *G = 16;
  *resident = 0;
  *rows = (h + 15) / 16;
}

// Rebuilds the device work lists from the unfinished jobs.
int engine_rebuild(clean_engine_s* e, cudaStream_t s) {
  std::vector<int> work;
  for (int i = 0; i < (int)e->jobs.size(); ++i)
    if (!e->jobs[i].finished) work.push_back(i);
  // gather images fed by TMA first, then gather images with plain loads (each
  // feedback launch covers a contiguous range), FFT-feedback images last
  std::stable_partition(work.begin(), work.end(), [&](int i) { return !e->jobs[i].fft; });
  std::stable_partition(work.begin(), work.end(),
                        [&](int i) { return !e->jobs[i].fft && e->jobs[i].tma; });
  e->n_work = (int)work.size();
  e->n_tma = 0;
  e->n_gather = 0;
  e->fft_work.clear();
  e->work_jobs = work;
  e->max_T = 1;
  std::vector<PlanDev> plans;
  std::vector<CUtensorMap> maps, rmaps, pmaps;
  std::vector<BatchImage> imgs;
  struct Sized {
    int64_t px;
    int pipe, G, resident, smem, rows, w;
    BatchItem it;
  };
  std::vector<Sized> all;
  int block0 = 0;
  // latency or throughput: when the tiles of every resident image fit on the
  // SMs even with one CTA per 8192 pixels, use that many (short iterations);
  // otherwise the fewest CTAs that hold each tile (the launches run in waves
  // anyway, and fewer, larger CTAs lose less to exchanges)
  bool fast = true;
  {
    int64_t ctas = 0;
    for (int i : work) {
      const Job& j = e->jobs[i];
      for (int t = 0; t < j.dev.T; ++t) {
        const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
        int g = 1, res = 0, rows = 0, sm = 0;
        if (j.pipe)
          pipe_tile_group(r.y1 - r.y0, r.x1 - r.x0, true, &g, &res, &rows);
        else
          tile_group(r.y1 - r.y0, r.x1 - r.x0, &g, &res, &sm);
        ctas += g;
      }
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
    fast = ctas <= sms;
  }
  // the pipelined images' minor loops go to the persistent launch when it can
  // be resident
  const int p_grid = minor_batch_persistent_grid(kPersistSmemMin);
  std::vector<BatchUnitItem> uitems;
  std::vector<int64_t> upx;  // pixels of each unit item's tile (scheduling order)
  int p_smem = kPersistSmemMin;
  e->blocks_tma = e->blocks_plain = 0;
  for (int w = 0; w < (int)work.size(); ++w) {
    Job& j = e->jobs[work[w]];
    if (p_grid > 0 && j.pipe) {
      // one G for the whole image (its tiles share the exchange slots), the
      // largest any of its tiles asks for, kept while the run lasts
      if (j.unit_G == 0) {
        // tile pairs when the tile count is even and every tile is two chunks
        // wide: G row bands per tile, each band short enough that a CTA's
        // full chunks of both tiles sit in tensor memory (4 chunks a tile)
        int min_w = 1 << 30, max_h = 0, half_w = 0;
        for (int t = 0; t < j.dev.T; ++t) {
          const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
          min_w = std::min(min_w, r.x1 - r.x0);
          max_h = std::max(max_h, r.y1 - r.y0);
          half_w = std::max(half_w, ((r.x1 - r.x0) / 2 + 127) / 128 * 128);
        }
        const int per_band = kBatchBoxRows * std::max(1, 4 / std::max(1, half_w / 128));
        const int Gp = (max_h + per_band - 1) / per_band;
        if (j.dev.T % 2 == 0 && min_w >= 2 * 128 && 2 * Gp <= kMaxUnitG) {
          j.unit_pair = true;
          j.unit_G = Gp;
        } else {
          int Gi = 1;
          for (int t = 0; t < j.dev.T; ++t) {
            const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
            int g = 1, res = 0, rows = 0;
            pipe_tile_group(r.y1 - r.y0, r.x1 - r.x0, fast, &g, &res, &rows);
            Gi = std::max(Gi, g);
          }
          j.unit_G = Gi;
        }
      }
      const int Gi = j.unit_G;
      if (j.unit_pair) {
        for (int pr = 0; pr < j.dev.T / 2; ++pr) {
          int rows = 0, wd = 0;
          int64_t px = 0;
          for (int t = 2 * pr; t <= 2 * pr + 1; ++t) {
            const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
            rows = std::max(rows, (r.y1 - r.y0 + Gi - 1) / Gi);
            wd = std::max(wd, r.x1 - r.x0);
            px += (int64_t)(r.y1 - r.y0) * (r.x1 - r.x0);
          }
          BatchUnitItem u{};
          if (!minor_pipe_batch_geometry(u.cfg, Gi, 0, rows, wd)) return CLEAN_ERR_UNSUPPORTED;
          u.cfg.sync = CLEAN_SYNC_GRID;
          u.cfg.G = Gi;
          u.cfg.pair = 1;
          u.kind = kUnitPair;
          u.image = w;
          u.tile = pr;
          u.ranks = 2 * Gi;
          p_smem = std::max(p_smem, u.cfg.smem);
          uitems.push_back(u);
          upx.push_back(px);
        }
      }
      for (int t = 0; t < j.dev.T && !j.unit_pair; ++t) {
        const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
        const int rows = (r.y1 - r.y0 + Gi - 1) / Gi, wd = r.x1 - r.x0;
        BatchUnitItem u{};
        if (minor_pipe_batch_geometry(u.cfg, Gi, 1, rows, wd)) {
          u.kind = kUnitResident;
        } else if (minor_pipe_batch_geometry(u.cfg, Gi, 0, rows, wd)) {
          u.kind = u.cfg.tmem ? kUnitTmem : kUnitStreamed;
        } else {
          return CLEAN_ERR_UNSUPPORTED;
        }
        u.cfg.sync = CLEAN_SYNC_GRID;
        u.cfg.G = Gi;
        u.image = w;
        u.tile = t;
        u.ranks = Gi;
        p_smem = std::max(p_smem, u.cfg.smem);
        uitems.push_back(u);
        upx.push_back((int64_t)(r.y1 - r.y0) * wd);
      }
    }
    plans.push_back(j.dev);
    maps.push_back(j.map);
    rmaps.push_back(j.rmap);
    pmaps.push_back(j.pmap);
    if (j.fft)
      e->fft_work.push_back(w);
    else
      ++e->n_gather;
    if (j.tma && !j.fft) ++e->n_tma;
    e->max_T = std::max(e->max_T, j.dev.T);
    for (int t = 0; t < j.dev.T && !(p_grid > 0 && j.pipe); ++t) {
      const Rect r = tile_rect(t, j.dev.ny, j.dev.nx, j.dev.ty, j.dev.tx);
      Sized z;
      z.px = (int64_t)(r.y1 - r.y0) * (r.x1 - r.x0);
      z.pipe = j.pipe ? 1 : 0;
      z.w = r.x1 - r.x0;
      if (z.pipe) {
        pipe_tile_group(r.y1 - r.y0, z.w, fast, &z.G, &z.resident, &z.rows);
        z.smem = 0;
      } else {
        tile_group(r.y1 - r.y0, z.w, &z.G, &z.resident, &z.smem);
        z.rows = (r.y1 - r.y0 + z.G - 1) / z.G;
      }
      z.it = BatchItem{w, t};
      all.push_back(z);
    }
    int bx = 0, by = 0;
    feedback_blocks(j.dev, j.tma, &bx, &by);
    if (!j.tma && w == e->n_tma) block0 = 0;  // plain images restart the block count
    BatchImage im;
    im.block0 = block0;
    im.bx = bx;
    im.by = by;
    im.nblocks = bx * by * j.dev.T;
    if (!j.fft) {
      block0 += im.nblocks;
      (j.tma ? e->blocks_tma : e->blocks_plain) += im.nblocks;
    }
    imgs.push_back(im);
  }
  // groups of equal (kernel, G, resident), biggest tiles first within each
  std::stable_sort(all.begin(), all.end(), [](const Sized& a, const Sized& b) {
    if (a.pipe != b.pipe) return a.pipe > b.pipe;
    if (a.G != b.G) return a.G > b.G;
    if (a.resident != b.resident) return a.resident < b.resident;
    return a.px > b.px;
  });
  e->groups.clear();
  std::vector<BatchItem> items;
  for (size_t k = 0; k < all.size(); ++k) {
    if (e->groups.empty() || e->groups.back().pipe != all[k].pipe ||
        e->groups.back().G != all[k].G || e->groups.back().resident != all[k].resident) {
      Group g;
      g.offset = (int)items.size();
      g.pipe = all[k].pipe;
      g.G = all[k].G;
      g.resident = all[k].resident;
      e->groups.push_back(g);
    }
    Group& g = e->groups.back();
    g.smem = std::max(g.smem, all[k].smem);
    g.max_rows = std::max(g.max_rows, all[k].rows);
    g.max_w = std::max(g.max_w, all[k].w);
    ++g.count;
    items.push_back(all[k].it);
  }
  for (Group& g : e->groups) {
    if (g.pipe) {
      // every tile fits alone, so the group's largest slab fits too
      if (!minor_pipe_batch_geometry(g.cfg, g.G, g.resident, g.max_rows, g.max_w))
        return CLEAN_ERR_UNSUPPORTED;
      g.smem = g.cfg.smem;
      if (g.G > 1 && minor_pipe_batch_cluster(g.G, g.resident, g.smem) != g.G)
        return CLEAN_ERR_UNSUPPORTED;
    } else if (g.G > 1) {
      // a cluster size the device cannot schedule
      const int ok = minor_batch_cluster(g.G, g.resident, g.smem);
      if (ok != g.G) return CLEAN_ERR_UNSUPPORTED;
    }
  }
  if ((int)items.size() > e->items_cap) {
    cudaFree(e->d_items);
    e->items_cap = std::max<int>((int)items.size(), 2 * e->items_cap);
    if (cudaMalloc(&e->d_items, sizeof(BatchItem) * e->items_cap) != cudaSuccess)
      return eng_fail(e, CLEAN_ERR_OOM);
  }
  cudaError_t err = cudaSuccess;
  if (!plans.empty()) {
    err = cudaMemcpyAsync(e->d_plans, plans.data(), sizeof(PlanDev) * plans.size(),
                          cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                            cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_rmaps, rmaps.data(), sizeof(CUtensorMap) * rmaps.size(),
                            cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_pmaps, pmaps.data(), sizeof(CUtensorMap) * pmaps.size(),
                            cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_imgs, imgs.data(), sizeof(BatchImage) * imgs.size(),
                            cudaMemcpyHostToDevice, s);
  }
  if (err == cudaSuccess && !items.empty())
    err = cudaMemcpyAsync(e->d_items, items.data(), sizeof(BatchItem) * items.size(),
                          cudaMemcpyHostToDevice, s);
  // the persistent schedule: items largest first, each item's G ranks into
  // the first wave with G idle CTAs (first fit)
  std::vector<int2> units;
  e->n_waves = 0;
  if (!uitems.empty()) {
    std::vector<int> order(uitems.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return upx[a] > upx[b]; });
    std::vector<int> used;  // CTAs taken in each wave
    for (int i : order) {
      const int G = uitems[i].ranks;
      size_t w = 0;
      while (w < used.size() && used[w] + G > p_grid) ++w;
      if (w == used.size()) {
        used.push_back(0);
        units.resize(units.size() + p_grid, make_int2(-1, 0));
      }
      for (int r = 0; r < G; ++r) units[w * p_grid + used[w] + r] = make_int2(i, r);
      used[w] += G;
    }
    e->n_waves = (int)used.size();
    if ((int)uitems.size() > e->uitems_cap) {
      cudaFree(e->d_uitems);
      e->uitems_cap = std::max<int>((int)uitems.size(), 2 * e->uitems_cap);
      if (cudaMalloc(&e->d_uitems, sizeof(BatchUnitItem) * e->uitems_cap) != cudaSuccess)
        return eng_fail(e, CLEAN_ERR_OOM);
    }
    if ((int)units.size() > e->units_cap) {
      cudaFree(e->d_units);
      e->units_cap = std::max<int>((int)units.size(), 2 * e->units_cap);
      if (cudaMalloc(&e->d_units, sizeof(int2) * e->units_cap) != cudaSuccess)
        return eng_fail(e, CLEAN_ERR_OOM);
    }
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_uitems, uitems.data(), sizeof(BatchUnitItem) * uitems.size(),
                            cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e->d_units, units.data(), sizeof(int2) * units.size(),
                            cudaMemcpyHostToDevice, s);
  }
  e->p_grid = p_grid;
  e->p_smem = p_smem;
  // the host vectors die here: make the copies complete first
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
  drop_graphs(e);  // the captured launches name the old work lists
  e->dirty = false;
  return CLEAN_OK;
}

int engine_read(clean_engine_s* e, cudaStream_t s) {
  cudaError_t err = cudaMemcpyAsync(e->h_states, e->d_states, sizeof(DevState) * e->cap,
                                    cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
  bool timeout = false;
  for (const Job& j : e->jobs) {
    const DevState& st = e->h_states[j.slot];
    if (!(st.status & ST_TIMEOUT)) continue;
    timeout = true;
    // CLEANGB_REPORT_TIMEOUT: which job, tile and exchange gave up (stderr)
    if (std::getenv("CLEANGB_REPORT_TIMEOUT"))
      std::fprintf(stderr,
                   "cleangb: timeout in job %lld (%d x %d, %d tiles, %s G %d): tile %lld, "
                   "iteration %lld\n",
                   (long long)j.id, j.dev.ny, j.dev.nx, j.dev.T, j.unit_pair ? "pairs" : "units",
                   j.unit_G, (long long)(st.timeout_where >> 32),
                   (long long)(st.timeout_where & 0xffffffffll));
  }
  if (timeout) return eng_fail(e, CLEAN_ERR_TIMEOUT);
  return CLEAN_OK;
}

// Marks jobs whose runs are over; returns how many are still running.
int engine_mark(clean_engine_s* e) {
  int running = 0;
  for (Job& j : e->jobs) {
    if (j.finished) continue;
    const DevState& st = e->h_states[j.slot];
    if (!st.active || (st.status & ST_NONFINITE_DIRTY)) {
      j.finished = true;
      e->dirty = true;
    } else {
      ++running;
    }
  }
  return running;
}

// Launches `rounds` rounds of every unfinished job.
// The kernels of one round (round index `round`) on stream s; *n counts them.
cudaError_t launch_round(clean_engine_s* e, int round, cudaStream_t s, int* n) {
  cudaError_t err = cudaSuccess;
  if (e->n_waves > 0) {
    err = launch_minor_batch_persistent(e->d_plans, e->d_uitems, e->d_units, e->n_waves,
                                        e->p_grid, e->p_smem, e->d_rmaps, e->d_pmaps, round, s);
    ++*n;
    if (err != cudaSuccess) return err;
  }
  for (const Group& g : e->groups) {
    err = g.pipe ? launch_minor_pipe_batch(e->d_plans, e->d_items + g.offset, g.count, g.cfg,
                                           e->d_rmaps, e->d_pmaps, round, s)
                 : launch_minor_batch(e->d_plans, e->d_items + g.offset, g.count, g.G,
                                      g.resident, g.smem, round, s);
    ++*n;
    if (err != cudaSuccess) return err;
  }
  if (e->blocks_tma > 0) {
    err = launch_feedback_batch(e->d_plans, e->d_imgs, e->n_tma, e->blocks_tma, e->max_T,
                                e->d_maps, round, 1, 2000000000ull, s);
    ++*n;
    if (err != cudaSuccess) return err;
  }
  if (e->blocks_plain > 0) {
    err = launch_feedback_batch(e->d_plans + e->n_tma, e->d_imgs + e->n_tma,
                                e->n_gather - e->n_tma, e->blocks_plain, e->max_T, nullptr,
                                round, 1, 2000000000ull, s);
    ++*n;
    if (err != cudaSuccess) return err;
  }
  // FFT-feedback images: each its own transform kernels
  for (int w : e->fft_work) {
    const Job& j = e->jobs[e->work_jobs[w]];
    err = plan_fft_round(j.plan, j.dev, (round - j.dev.round0) & 1, s);
    *n += 3;
    if (err != cudaSuccess) return err;
  }
  return err;
}

// Captures two rounds starting at a round of parity `par` into e->pair[par].
// Returns false (and leaves no capture open) if the runtime refuses.
bool capture_pair(clean_engine_s* e, int par) {
  if (!e->cap_stream &&
      cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaGraph_t graph = nullptr;
  int n = 0;
  cudaError_t err = cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeRelaxed);
  if (err == cudaSuccess) {
    cudaError_t l = launch_round(e, par, e->cap_stream, &n);
    if (l == cudaSuccess) l = launch_round(e, par + 1, e->cap_stream, &n);
    err = cudaStreamEndCapture(e->cap_stream, &graph);
    if (l != cudaSuccess) err = l;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->pair[par], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    e->pair[par] = nullptr;
    cudaGetLastError();
    return false;
  }
  e->pair_kernels = n;
  return true;
}

int engine_rounds(clean_engine_s* e, int64_t rounds, cudaStream_t s) {
  int rc;
  if (e->dirty && (rc = engine_rebuild(e, s)) != CLEAN_OK) return rc;
  if (e->n_work == 0) return CLEAN_OK;
  while (rounds >= 2 && e->use_graphs && !e->graphs_refused) {
    const int par = e->round & 1;
    if (!e->pair[par] && !capture_pair(e, par)) {
      e->graphs_refused = true;
      break;
    }
    if (cudaGraphLaunch(e->pair[par], s) != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
    e->kernel_launches += e->pair_kernels;
    ++e->graph_launches;
    e->round += 2;
    e->rounds_launched += 2;
    rounds -= 2;
  }
  for (int64_t r = 0; r < rounds; ++r) {
    int n = 0;
    const cudaError_t err = launch_round(e, e->round, s, &n);
    e->kernel_launches += n;
    if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
    ++e->round;
    ++e->rounds_launched;
  }
  return CLEAN_OK;
}

Job* engine_find(clean_engine_s* e, int64_t id) {
  for (Job& j : e->jobs)
    if (j.id == id) return &j;
  return nullptr;
}

int engine_get(clean_engine_s* e, const Job& j, float* d_residual, float* d_model,
               clean_component* d_comps, int64_t comps_cap, int64_t* n_comps, cudaStream_t s) {
  const size_t img = sizeof(float) * (size_t)j.dev.ny * j.dev.nx;
  cudaError_t err = cudaSuccess;
  if (d_residual) err = cudaMemcpyAsync(d_residual, j.dev.R, img, cudaMemcpyDeviceToDevice, s);
  if (err == cudaSuccess && d_model)
    err = cudaMemcpyAsync(d_model, j.dev.model, img, cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
  if (d_comps || n_comps) {
    DevState st;
    err = cudaMemcpyAsync(&st, j.dev.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
    if (n_comps) *n_comps = st.total;
    const int64_t m = std::min(st.total, comps_cap);
    if (d_comps && m > 0) {
      err = cudaMemcpyAsync(d_comps, j.dev.list, sizeof(clean_component) * (size_t)m,
                            cudaMemcpyDeviceToDevice, s);
      if (err != cudaSuccess) return eng_fail(e, CLEAN_ERR_CUDA);
    }
  }
  return CLEAN_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Fixed batches
// ---------------------------------------------------------------------------
struct clean_batch_s {
  clean_engine_s* eng = nullptr;
  std::vector<int64_t> ids;  // job i of the batch is eng->jobs[i]
  bool started = false;
};

extern "C" {

void clean_batch_destroy(clean_batch_t b) {
  if (!b) return;
  engine_free(b->eng);
  delete b;
}

int clean_batch_create(clean_batch_t* out, int32_t n, const clean_params* params,
                       const float* const* d_psfs, void* stream) {
  if (!out) return CLEAN_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || !params || !d_psfs) return CLEAN_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int rc = clean_params_check(&params[i]);
    if (rc != CLEAN_OK) return rc;
    if (!d_psfs[i] || params[i].mode != CLEAN_TILED) return CLEAN_ERR_INVALID_ARG;
  }
  clean_batch_s* b = new (std::nothrow) clean_batch_s();
  if (!b) return CLEAN_ERR_OOM;
  int rc = engine_create(&b->eng, n);
  if (rc != CLEAN_OK) {
    delete b;
    return rc;
  }
  b->eng->jobs.reserve(n);  // Job pointers stay valid while registering
  for (int i = 0; i < n; ++i) {
    Job* j = nullptr;
    rc = engine_register(b->eng, &params[i], d_psfs[i], &j, reinterpret_cast<cudaStream_t>(stream));
    if (rc != CLEAN_OK) {
      clean_batch_destroy(b);
      return rc;
    }
    b->ids.push_back(j->id);
  }
  *out = b;
  return CLEAN_OK;
}

int clean_batch_run(clean_batch_t b, const float* const* d_dirties, int32_t max_rounds,
                    void* stream) {
  if (!b) return CLEAN_ERR_INVALID_ARG;
  clean_engine_s* e = b->eng;
  if (e->poisoned != CLEAN_OK) return e->poisoned;
  if (max_rounds < -1) return CLEAN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc;
  if (d_dirties) {
    for (size_t i = 0; i < b->ids.size(); ++i)
      if (!d_dirties[i]) return CLEAN_ERR_INVALID_ARG;
    // new runs, every image starting at the same round
    for (size_t i = 0; i < b->ids.size(); ++i)
      if ((rc = engine_start(e, e->jobs[i], d_dirties[i], s)) != CLEAN_OK) return rc;
    b->started = true;
  } else if (!b->started) {
    return CLEAN_ERR_INVALID_ARG;
  }
  if ((rc = engine_read(e, s)) != CLEAN_OK) return rc;
  for (const Job& j : e->jobs)
    if (e->h_states[j.slot].status & ST_NONFINITE_DIRTY) {
      b->started = false;
      return CLEAN_ERR_NONFINITE;
    }
  int64_t done = 0;
  while (max_rounds < 0 || done < max_rounds) {
    if (engine_mark(e) == 0) break;
    int64_t chunk = 1;
    for (const Job& j : e->jobs) {
      if (j.finished) continue;
      const int K = j.dev.K;
      const int64_t need = K > 0 ? (e->h_states[j.slot].max_budget + K - 1) / K : 1;
      chunk = std::max<int64_t>(chunk, need);
    }
    if (max_rounds >= 0) chunk = std::min<int64_t>(chunk, max_rounds - done);
    if ((rc = engine_rounds(e, chunk, s)) != CLEAN_OK) return rc;
    done += chunk;
    if ((rc = engine_read(e, s)) != CLEAN_OK) return rc;
  }
  return CLEAN_OK;
}

int clean_batch_get(clean_batch_t b, int32_t i, float* d_residual, float* d_model,
                    clean_component* d_comps, int64_t comps_cap, int64_t* n_comps, void* stream) {
  if (!b || i < 0 || i >= (int32_t)b->ids.size()) return CLEAN_ERR_INVALID_ARG;
  clean_engine_s* e = b->eng;
  if (e->poisoned != CLEAN_OK) return e->poisoned;
  Job* j = engine_find(e, b->ids[i]);
  if (!j) return CLEAN_ERR_INVALID_ARG;
  return engine_get(e, *j, d_residual, d_model, d_comps, comps_cap, n_comps,
                    reinterpret_cast<cudaStream_t>(stream));
}

int clean_batch_stats(clean_batch_t b, int64_t* rounds_launched, int64_t* kernel_launches,
                      int64_t* n_components) {
  if (!b) return CLEAN_ERR_INVALID_ARG;
  clean_engine_s* e = b->eng;
  if (rounds_launched) *rounds_launched = e->rounds_launched;
  if (kernel_launches) *kernel_launches = e->kernel_launches;
  if (n_components) {
    int64_t t = 0;
    for (const Job& j : e->jobs) t += e->h_states[j.slot].total;
    *n_components = t;
  }
  return CLEAN_OK;
}

int clean_batch_graphs(clean_batch_t b, int32_t enable, int64_t* graph_launches) {
  if (!b || enable < -1 || enable > 1) return CLEAN_ERR_INVALID_ARG;
  clean_engine_s* e = b->eng;
  if (enable >= 0) {
    e->use_graphs = enable != 0;
    e->graphs_refused = false;
  }
  if (graph_launches) *graph_launches = e->graph_launches;
  return CLEAN_OK;
}

// ---------------------------------------------------------------------------
// Continuous batching
// ---------------------------------------------------------------------------
int clean_server_create(clean_server_t* out, int32_t max_jobs, void* stream) {
  (void)stream;
  if (!out || max_jobs < 1 || max_jobs > (1 << 16)) return CLEAN_ERR_INVALID_ARG;
  *out = nullptr;
  clean_engine_s* e = nullptr;
  const int rc = engine_create(&e, max_jobs);
  if (rc != CLEAN_OK) return rc;
  *out = reinterpret_cast<clean_server_t>(e);
  return CLEAN_OK;
}

void clean_server_destroy(clean_server_t sv) { engine_free(reinterpret_cast<clean_engine_s*>(sv)); }

int clean_server_add(clean_server_t sv, const clean_params* p, const float* d_psf,
                     const float* d_dirty, int64_t* job_id, void* stream) {
  clean_engine_s* e = reinterpret_cast<clean_engine_s*>(sv);
  if (!e || !p || !d_dirty) return CLEAN_ERR_INVALID_ARG;
  if (e->poisoned != CLEAN_OK) return e->poisoned;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Job* j = nullptr;
  int rc = engine_register(e, p, d_psf, &j, s);
  if (rc != CLEAN_OK) return rc;
  if ((rc = engine_start(e, *j, d_dirty, s)) != CLEAN_OK) return rc;
  if (job_id) *job_id = j->id;
  return CLEAN_OK;
}

int clean_server_step(clean_server_t sv, int32_t rounds, int32_t* n_running, void* stream) {
  clean_engine_s* e = reinterpret_cast<clean_engine_s*>(sv);
  if (!e || rounds < 0) return CLEAN_ERR_INVALID_ARG;
  if (e->poisoned != CLEAN_OK) return e->poisoned;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = engine_read(e, s);
  if (rc != CLEAN_OK) return rc;
  if (engine_mark(e) > 0 && rounds > 0) {
    if ((rc = engine_rounds(e, rounds, s)) != CLEAN_OK) return rc;
    if ((rc = engine_read(e, s)) != CLEAN_OK) return rc;
  }
  const int running = engine_mark(e);
  if (n_running) *n_running = running;
  return CLEAN_OK;
}

int clean_server_done(clean_server_t sv, int64_t* ids, int32_t cap, int32_t* n_done) {
  clean_engine_s* e = reinterpret_cast<clean_engine_s*>(sv);
  if (!e || (cap > 0 && !ids)) return CLEAN_ERR_INVALID_ARG;
  int n = 0;
  for (const Job& j : e->jobs)
    if (j.finished) {
      if (n < cap) ids[n] = j.id;
      ++n;
    }
  if (n_done) *n_done = n;
  return CLEAN_OK;
}

int clean_server_get(clean_server_t sv, int64_t job_id, float* d_residual, float* d_model,
                     clean_component* d_comps, int64_t comps_cap, int64_t* n_comps,
                     void* stream) {
  clean_engine_s* e = reinterpret_cast<clean_engine_s*>(sv);
  if (!e) return CLEAN_ERR_INVALID_ARG;
  if (e->poisoned != CLEAN_OK) return e->poisoned;
  Job* j = engine_find(e, job_id);
  if (!j) return CLEAN_ERR_INVALID_ARG;
  return engine_get(e, *j, d_residual, d_model, d_comps, comps_cap, n_comps,
                    reinterpret_cast<cudaStream_t>(stream));
}

int clean_server_remove(clean_server_t sv, int64_t job_id) {
  clean_engine_s* e = reinterpret_cast<clean_engine_s*>(sv);
  if (!e) return CLEAN_ERR_INVALID_ARG;
  for (size_t k = 0; k < e->jobs.size(); ++k)
    if (e->jobs[k].id == job_id) {
      cudaDeviceSynchronize();
      clean_destroy(e->jobs[k].plan);
      cudaFree(e->jobs[k].bkeys);
      e->free_slots.push_back(e->jobs[k].slot);
      e->jobs.erase(e->jobs.begin() + (long)k);
      e->dirty = true;
      return CLEAN_OK;
    }
  return CLEAN_ERR_INVALID_ARG;
}

}  // extern "C"
