// k_noalloc.cu -- ts_l1_loss_noalloc: the L1 colour + depth loss without a caller workspace.
//
// Some callers cannot hand this library any device memory beyond the images they pass in: a
// host application that owns the whole device budget and only lends out its input and output
// buffers, or a loop that must not call cudaMalloc because the allocation would synchronise the
// device or fail under a fixed memory pool.  For them this entry point keeps the loss's
// per-block partial sums in a file-scope static device array instead of the plan's workspace.
//
// The array holds TS_NOALLOC_LOSS_SLOTS (view, block) pairs of two floats (512 KiB); every GPU
// that loads the library keeps it until the process exits.  Every call overwrites the slots it
// reads, so no state carries over from the previous call and nothing needs clearing; two calls
// that run at the same time on the GPU (different streams, or different host threads) share the
// array and race.  The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (with that device current); make that first call before any stream
// capture.  The cached address is valid for the life of the device's context: after a
// cudaDeviceReset it is stale and the entry point must not be called on that device again.
// It allocates nothing and calls no allocating routine.
#include <atomic>
#include <cmath>
#include <mutex>

#include "ts_internal.cuh"

#define TS_NOALLOC_LOSS_SLOTS 65536  // (view, 2048-pixel block) pairs
#define TS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_noalloc_loss_partials[2 * TS_NOALLOC_LOSS_SLOTS];

namespace {

constexpr int NA_T = 256;
constexpr int NA_PER = 8;  // 2048 pixels per block

struct NaViews {  // image sizes and packing offsets of the views
  int32_t W[TS_MAX_VIEWS], H[TS_MAX_VIEWS];
  long long pix_off[TS_MAX_VIEWS];
};

// The loss body is the one ts_l1_loss runs (ts_l1_loss_block / ts_l1_loss_final); only the
// partial sums' home differs.
__global__ void __launch_bounds__(NA_T) k_na_loss_partial(NaViews tab, const float* __restrict__ C,
                                                          const float* __restrict__ D, const float* __restrict__ tC,
                                                          const float* __restrict__ tD, float lambda_dep,
                                                          float* __restrict__ dC, float* __restrict__ dD,
                                                          float* __restrict__ part, int nblk) {
  const int v = blockIdx.y;
  ts_l1_loss_block<NA_T, NA_PER>((long long)tab.W[v] * tab.H[v], tab.pix_off[v],
                                 (long long)blockIdx.x * NA_T * NA_PER, C, D, tC, tD, lambda_dep, dC, dD,
                                 part + ((long long)v * nblk + blockIdx.x) * 2);
}

__global__ void __launch_bounds__(NA_T) k_na_loss_final(NaViews tab, const float* __restrict__ part, int nblk,
                                                        float lambda_dep, float* __restrict__ loss) {
  const int v = blockIdx.x;
  ts_l1_loss_final<NA_T>((long long)tab.W[v] * tab.H[v], part + (long long)v * nblk * 2, nblk, lambda_dep, loss + v);
}

std::mutex g_setup_mutex;
std::atomic<float*> g_partials_ptr[TS_NOALLOC_MAX_DEVICES];

// Device address of the static scratch array on the current device.  It is looked up once per
// device (under a lock) and then read without one.  The address belongs to the CUDA context that
// loaded the module: after cudaDeviceReset the cached address is stale, so a process that resets a
// device must not call ts_l1_loss_noalloc on it again.
ts_status scratch_on_current_device(float** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TS_NOALLOC_MAX_DEVICES) return TS_ERR_CUDA;
  float* p = g_partials_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    p = g_partials_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
      void* q = nullptr;
      if (cudaGetSymbolAddress(&q, g_noalloc_loss_partials) != cudaSuccess || !q) return TS_ERR_CUDA;
      p = static_cast<float*>(q);
      g_partials_ptr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return TS_OK;
}

}  // namespace

extern "C" ts_status ts_l1_loss_noalloc(const ts_camera* cams, int32_t n_views, const float* color, const float* depth,
                                        const float* tgt_color, const float* tgt_depth, float lambda_dep,
                                        float* loss, float* dC, float* dD, ts_stream stream) {
  if (!cams || n_views < 1 || n_views > TS_MAX_VIEWS) return TS_ERR_INVALID_ARG;
  if (!color || !depth || !tgt_color || !tgt_depth || !loss || !dC || !dD || !(lambda_dep >= 0.0f) ||
      !std::isfinite(lambda_dep))
    return TS_ERR_INVALID_ARG;
  NaViews tab;
  long long off = 0, max_hw = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width < 1 || cams[v].height < 1 || cams[v].width > 16384 || cams[v].height > 16384)
      return TS_ERR_INVALID_ARG;
    tab.W[v] = cams[v].width;
    tab.H[v] = cams[v].height;
    tab.pix_off[v] = off;
    const long long hw = (long long)cams[v].width * cams[v].height;
    off += hw;
    if (hw > max_hw) max_hw = hw;
  }
  const long long nblk = (max_hw + NA_T * NA_PER - 1) / (NA_T * NA_PER);
  if ((long long)n_views * nblk > TS_NOALLOC_LOSS_SLOTS) return TS_ERR_INVALID_ARG;  // beyond the static scratch
  float* part = nullptr;
  const ts_status st = scratch_on_current_device(&part);
  if (st != TS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid((unsigned)nblk, (unsigned)n_views);
  k_na_loss_partial<<<grid, NA_T, 0, s>>>(tab, color, depth, tgt_color, tgt_depth, lambda_dep, dC, dD, part, (int)nblk);
  k_na_loss_final<<<n_views, NA_T, 0, s>>>(tab, part, (int)nblk, lambda_dep, loss);
  return cudaGetLastError() == cudaSuccess ? TS_OK : TS_ERR_CUDA;
}
