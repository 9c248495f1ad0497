// clean_hogbom_noalloc: plain (untiled) Hogbom CLEAN on the whole GPU that
// allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// streaming imaging pipeline that reserves all of its device memory in one
// pool at start-up (cudaMalloc can block, synchronise the device or fail on
// a fragmented heap, which such a pipeline cannot afford mid-observation),
// or code embedded in a host framework that owns every device allocation.
// This entry point serves them: the caller passes the inputs and the outputs,
// and the only other memory the kernels need -- the grid-barrier counters,
// the per-CTA partial peak keys and a few control words -- lives in a
// file-scope __device__ array of fixed size.  Every GPU that loads the
// library holds that array until the process exits.
//
// The arithmetic is that of clean_plan/clean_run with CLEAN_UNTILED_GRID:
// the same set-up kernel and the same grid-synchronised minor-loop kernel.
#include <cstring>

#include "cleangb_internal.cuh"

namespace cleangb {
namespace {

// Scratch layout (bytes): control block, two peak keys, the budget, the
// component count, the grid-barrier counter, then two parity slots of
// per-CTA partial keys (kNoAllocMaxCtas each).
constexpr int kNoAllocMaxCtas = 1024;
constexpr size_t kOffState = 0;
constexpr size_t kOffPeak = 256;
constexpr size_t kOffBudget = kOffPeak + 2 * sizeof(uint64_t);
constexpr size_t kOffCount = kOffBudget + sizeof(int64_t);
constexpr size_t kOffBar = kOffCount + sizeof(int32_t);
constexpr size_t kOffKeys = 512;
constexpr size_t kScratchBytes = kOffKeys + 2 * kNoAllocMaxCtas * sizeof(uint64_t);  // 16.5 KiB
static_assert(sizeof(DevState) <= kOffPeak, "control block overlaps the peak keys");
static_assert(kOffBar + sizeof(uint32_t) <= kOffKeys, "counters overlap the key slots");

// The scratch.  In host code this name is only a stand-in for the symbol,
// never a device address: the device address comes from
// cudaGetSymbolAddress with the device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch in the current device's context.  Looked up
// on every call rather than cached: after cudaDeviceReset, or from another
// context on the same device, the module is loaded again and the array may
// sit at another address.  The lookup allocates nothing.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace cleangb

using namespace cleangb;

extern "C" CLEAN_API int clean_hogbom_noalloc(const float* d_dirty, const float* d_psf,
                                              int32_t ny, int32_t nx, int32_t psf_ny,
                                              int32_t psf_nx, float gain, int64_t niter,
                                              float threshold, float* d_residual,
                                              float* d_model, clean_component* d_comps,
                                              int64_t* n_comps, void* stream) {
  clean_params p;
  clean_params_default(&p);
  p.ny = ny;
  p.nx = nx;
  p.psf_ny = psf_ny;
  p.psf_nx = psf_nx;
  p.gain = gain;
  p.threshold = threshold;
  p.niter = niter;
  p.mode = CLEAN_UNTILED_GRID;
  if (clean_params_check(&p) != CLEAN_OK) return CLEAN_ERR_INVALID_ARG;
  if (!d_dirty || !d_psf || !d_residual || !d_model || (niter > 0 && !d_comps))
    return CLEAN_ERR_INVALID_ARG;
  if (niter > 0x7fffffffll) return CLEAN_ERR_INVALID_ARG;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  // one CTA per SM in the grid-synchronised group; the key slots hold at
  // most kNoAllocMaxCtas of them
  const int G = sms < ny ? sms : ny;
  if (G > kNoAllocMaxCtas) return CLEAN_ERR_UNSUPPORTED;

  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  PlanDev d{};
  d.R = d_residual;
  d.model = d_model;
  d.P = d_psf;
  d.ny = ny;
  d.nx = nx;
  d.pny = psf_ny;
  d.pnx = psf_nx;
  d.cy = psf_ny / 2;
  d.cx = psf_nx / 2;
  d.ty = d.tx = d.T = 1;
  d.gain = gain;
  d.thr = threshold;
  d.K = 0;
  d.trigger = 0.f;
  d.cap_round = (int32_t)(niter > 0 ? niter : 1);
  d.budget = reinterpret_cast<int64_t*>(base + kOffBudget);
  d.peak = reinterpret_cast<uint64_t*>(base + kOffPeak);
  d.rcount = reinterpret_cast<int32_t*>(base + kOffCount);
  d.rcomps = d_comps;  // one tile, one round: the round list is the output list
  d.list = nullptr;
  d.round_off = nullptr;
  d.gkeys = reinterpret_cast<uint64_t*>(base + kOffKeys);
  d.gbar = reinterpret_cast<uint32_t*>(base + kOffBar);
  d.st = reinterpret_cast<DevState*>(base + kOffState);

  MinorCfg mc{};
  mc.G = G;
  mc.sync = CLEAN_SYNC_GRID;
  mc.threads = minor_threads();
  mc.spin_limit_ns = 2000000000ll;
  const int64_t slab = (int64_t)((ny + G - 1) / G) * nx * 4;
  mc.resident = slab <= 200 * 1024 ? 1 : 0;
  mc.smem = mc.resident ? (int)slab : 0;

  // the peak keys are atomic-max targets and the control block collects
  // status bits: both must start at zero (the array keeps the last call's
  // contents); set-up zeroes the exchange count and sets the budget
  cudaError_t e = cudaMemsetAsync(d.st, 0, sizeof(DevState), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.peak, 0, 2 * sizeof(uint64_t), s);
  // grid-barrier key slots start with mark bit 63 set (see the minor loop)
  if (e == cudaSuccess) e = cudaMemsetAsync(d.gkeys, 0x80, 2 * sizeof(uint64_t) * (size_t)G, s);
  if (e == cudaSuccess) e = minor_prepare(mc);
  if (e == cudaSuccess) e = launch_validate_psf(d, s);
  if (e == cudaSuccess) e = launch_init(d, d_dirty, niter, s);
  DevState hs;
  int32_t count = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hs, d.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  if (hs.status & (ST_NONFINITE_DIRTY | ST_NONFINITE_PSF)) return CLEAN_ERR_NONFINITE;
  if (hs.status & ST_PSF_OFFCENTRE) return CLEAN_ERR_INVALID_ARG;
  e = launch_minor(d, mc, 0, nullptr, nullptr, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hs, d.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&count, d.rcount, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CLEAN_ERR_CUDA;
  }
  if (hs.status & ST_TIMEOUT) return CLEAN_ERR_TIMEOUT;
  if (n_comps) *n_comps = count;
  return CLEAN_OK;
}
