// Batched tiled CLEAN: many dirty images of uneven sizes deconvolved
// together, every round of every image in the same launches (one minor-loop
// launch per residual placement and one feedback launch), so small images
// fill the GPU together instead of one after another.  Each image's
// arithmetic is exactly that of its own plan (clean_plan + clean_run): the
// batch only changes which CTA serves which tile, so each image's results
// are identical to its solo run.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "cleangb_internal.cuh"

using namespace cleangb;

namespace {
constexpr int64_t kBatchResidentMax = 200 * 1024;  // one CTA's tile in shared memory
}

struct clean_batch_s {
  int device = 0;
  int n = 0;
  std::vector<clean_plan_t> plans;
  std::vector<PlanDev> dev;        // host copies of the images' plan state
  PlanDev* d_plans = nullptr;      // device array of PlanDev
  BatchItem* d_items = nullptr;    // resident items then streamed items
  int n_res = 0, n_str = 0, res_smem = 0;
  BatchImage* d_imgs = nullptr;
  int total_blocks = 0, max_T = 1;
  CUtensorMap* d_maps = nullptr;   // one PSF tensor map per image (TMA feedback)
  bool tma = false;
  DevState* d_states = nullptr;    // contiguous control blocks of all images
  DevState* h_states = nullptr;    // pinned mirror
  int parity = 0;
  bool started = false;
  int poisoned = CLEAN_OK;
  int64_t rounds_launched = 0, kernel_launches = 0;
};

namespace {

int batch_fail(clean_batch_s* b, int code) {
  cudaGetLastError();
  if (b->poisoned == CLEAN_OK) b->poisoned = code;
  return b->poisoned;
}

int read_states(clean_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->h_states, b->d_states, sizeof(DevState) * b->n,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return batch_fail(b, CLEAN_ERR_CUDA);
  for (int i = 0; i < b->n; ++i)
    if (b->h_states[i].status & ST_TIMEOUT) return batch_fail(b, CLEAN_ERR_TIMEOUT);
  return CLEAN_OK;
}

}  // namespace

extern "C" {

void clean_batch_destroy(clean_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (clean_plan_t p : b->plans) clean_destroy(p);
  cudaFree(b->d_plans);
  cudaFree(b->d_items);
  cudaFree(b->d_imgs);
  cudaFree(b->d_maps);
  cudaFree(b->d_states);
  if (b->h_states) cudaFreeHost(b->h_states);
  cudaGetLastError();
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
    if (!d_psfs[i] || params[i].mode != CLEAN_TILED || params[i].feedback_mode == CLEAN_FB_FFT)
      return CLEAN_ERR_INVALID_ARG;
  }
  clean_batch_s* b = new (std::nothrow) clean_batch_s();
  if (!b) return CLEAN_ERR_OOM;
  b->n = n;
  cudaGetDevice(&b->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) {
    clean_params p = params[i];
    p.feedback_mode = CLEAN_FB_GATHER;
    clean_plan_t pl = nullptr;
    const int rc = clean_plan(&pl, &p, d_psfs[i], stream);
    if (rc != CLEAN_OK) {
      clean_batch_destroy(b);
      return rc;
    }
    b->plans.push_back(pl);
  }
  // contiguous control blocks, read back with one copy per batch of rounds
  if (cudaMalloc(&b->d_states, sizeof(DevState) * n) != cudaSuccess ||
      cudaMallocHost(&b->h_states, sizeof(DevState) * n) != cudaSuccess) {
    clean_batch_destroy(b);
    return CLEAN_ERR_OOM;
  }
  b->tma = true;
  std::vector<BatchItem> res, str;
  std::vector<std::pair<int64_t, BatchItem>> res_sized, str_sized;
  std::vector<BatchImage> imgs(n);
  std::vector<CUtensorMap> maps(n);
  int block0 = 0;
  for (int i = 0; i < n; ++i) {
    PlanDev d = plan_device_state(b->plans[i]);
    d.st = b->d_states + i;
    b->dev.push_back(d);
    b->tma = b->tma && plan_psf_tensor_map(b->plans[i], &maps[i]);
    b->max_T = std::max(b->max_T, d.T);
    for (int t = 0; t < d.T; ++t) {
      const Rect r = tile_rect(t, d.ny, d.nx, d.ty, d.tx);
      const int64_t bytes = (int64_t)(r.y1 - r.y0) * (r.x1 - r.x0) * 4;
      const BatchItem it{i, t};
      if (bytes <= kBatchResidentMax) {
        res_sized.push_back({bytes, it});
        b->res_smem = (int)std::max<int64_t>(b->res_smem, bytes);
      } else {
        str_sized.push_back({bytes, it});
      }
    }
  }
  // largest tiles first, so the last wave is made of the short ones
  auto by_size = [](const std::pair<int64_t, BatchItem>& a, const std::pair<int64_t, BatchItem>& c) {
    return a.first > c.first;
  };
  std::stable_sort(res_sized.begin(), res_sized.end(), by_size);
  std::stable_sort(str_sized.begin(), str_sized.end(), by_size);
  for (auto& x : res_sized) res.push_back(x.second);
  for (auto& x : str_sized) str.push_back(x.second);
  b->n_res = (int)res.size();
  b->n_str = (int)str.size();
  for (int i = 0; i < n; ++i) {
    int bx = 0, by = 0;
    feedback_blocks(b->dev[i], b->tma, &bx, &by);
    imgs[i].block0 = block0;
    imgs[i].bx = bx;
    imgs[i].by = by;
    imgs[i].nblocks = bx * by * b->dev[i].T;
    block0 += imgs[i].nblocks;
  }
  b->total_blocks = block0;
  std::vector<BatchItem> items = res;
  items.insert(items.end(), str.begin(), str.end());
  if (cudaMalloc(&b->d_plans, sizeof(PlanDev) * n) != cudaSuccess ||
      cudaMalloc(&b->d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)) != cudaSuccess ||
      cudaMalloc(&b->d_imgs, sizeof(BatchImage) * n) != cudaSuccess ||
      cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * n) != cudaSuccess) {
    clean_batch_destroy(b);
    return CLEAN_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_plans, b->dev.data(), sizeof(PlanDev) * n,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_imgs, imgs.data(), sizeof(BatchImage) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b->tma)
    e = cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_states, 0, sizeof(DevState) * n, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    clean_batch_destroy(b);
    return CLEAN_ERR_CUDA;
  }
  *out = b;
  return CLEAN_OK;
}

int clean_batch_run(clean_batch_t b, const float* const* d_dirties, int32_t max_rounds,
                    void* stream) {
  if (!b) return CLEAN_ERR_INVALID_ARG;
  if (b->poisoned != CLEAN_OK) return b->poisoned;
  if (max_rounds < -1) return CLEAN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (d_dirties) {
    for (int i = 0; i < b->n; ++i)
      if (!d_dirties[i]) return CLEAN_ERR_INVALID_ARG;
    cudaError_t e = cudaMemsetAsync(b->d_states, 0, sizeof(DevState) * b->n, s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
      const PlanDev& d = b->dev[i];
      e = cudaMemsetAsync(d.peak, 0, sizeof(uint64_t) * 2 * d.T, s);
      if (e == cudaSuccess) e = launch_init(d, d_dirties[i], plan_niter(b->plans[i]), s);
      ++b->kernel_launches;
    }
    if (e != cudaSuccess) return batch_fail(b, CLEAN_ERR_CUDA);
    b->parity = 0;
    b->rounds_launched = 0;
    b->started = true;
  } else if (!b->started) {
    return CLEAN_ERR_INVALID_ARG;
  }
  int rc = read_states(b, s);
  if (rc != CLEAN_OK) return rc;
  for (int i = 0; i < b->n; ++i)
    if (b->h_states[i].status & ST_NONFINITE_DIRTY) {
      b->started = false;
      return CLEAN_ERR_NONFINITE;
    }
  int64_t done = 0;
  while (max_rounds < 0 || done < max_rounds) {
    int64_t chunk = 0;
    for (int i = 0; i < b->n; ++i) {
      if (!b->h_states[i].active) continue;
      const int K = b->dev[i].K;
      const int64_t need = K > 0 ? (b->h_states[i].max_budget + K - 1) / K : 1;
      chunk = std::max<int64_t>(chunk, std::max<int64_t>(need, 1));
    }
    if (chunk == 0) break;
    if (max_rounds >= 0) chunk = std::min<int64_t>(chunk, max_rounds - done);
    for (int64_t r = 0; r < chunk; ++r) {
      cudaError_t e = launch_minor_batch(b->d_plans, b->d_items, b->n_res, 1, b->res_smem,
                                         b->parity, s);
      if (e == cudaSuccess)
        e = launch_minor_batch(b->d_plans, b->d_items + b->n_res, b->n_str, 0, 0, b->parity, s);
      if (e == cudaSuccess)
        e = launch_feedback_batch(b->d_plans, b->d_imgs, b->n, b->total_blocks, b->max_T,
                                  b->tma ? b->d_maps : nullptr, b->parity, 1, 2000000000ull, s);
      b->kernel_launches += 3;
      if (e != cudaSuccess) return batch_fail(b, CLEAN_ERR_CUDA);
      b->parity ^= 1;
      ++b->rounds_launched;
    }
    done += chunk;
    if ((rc = read_states(b, s)) != CLEAN_OK) return rc;
  }
  return CLEAN_OK;
}

int clean_batch_get(clean_batch_t b, int32_t i, float* d_residual, float* d_model,
                    clean_component* d_comps, int64_t comps_cap, int64_t* n_comps, void* stream) {
  if (!b || i < 0 || i >= b->n) return CLEAN_ERR_INVALID_ARG;
  if (b->poisoned != CLEAN_OK) return b->poisoned;
  if (!b->started) return CLEAN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const PlanDev& d = b->dev[i];
  const size_t img = sizeof(float) * (size_t)d.ny * d.nx;
  cudaError_t e = cudaSuccess;
  if (d_residual) e = cudaMemcpyAsync(d_residual, d.R, img, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_model) e = cudaMemcpyAsync(d_model, d.model, img, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return batch_fail(b, CLEAN_ERR_CUDA);
  if (d_comps || n_comps) {
    const int rc = read_states(b, s);
    if (rc != CLEAN_OK) return rc;
    const int64_t total = b->h_states[i].total;
    if (n_comps) *n_comps = total;
    const int64_t m = std::min(total, comps_cap);
    if (d_comps && m > 0) {
      e = cudaMemcpyAsync(d_comps, d.list, sizeof(clean_component) * (size_t)m,
                          cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return batch_fail(b, CLEAN_ERR_CUDA);
    }
  }
  return CLEAN_OK;
}

int clean_batch_stats(clean_batch_t b, int64_t* rounds_launched, int64_t* kernel_launches,
                      int64_t* n_components) {
  if (!b) return CLEAN_ERR_INVALID_ARG;
  if (rounds_launched) *rounds_launched = b->rounds_launched;
  if (kernel_launches) *kernel_launches = b->kernel_launches;
  if (n_components) {
    int64_t t = 0;
    for (int i = 0; i < b->n; ++i) t += b->h_states[i].total;
    *n_components = t;
  }
  return CLEAN_OK;
}

}  // extern "C"
