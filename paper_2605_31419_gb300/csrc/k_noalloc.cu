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
// capture.  It allocates nothing and calls no allocating routine.
#include <mutex>

#include "ts_internal.cuh"

#define TS_NOALLOC_LOSS_SLOTS 65536  // (view, 2048-pixel block) pairs
#define TS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_noalloc_loss_partials[2 * TS_NOALLOC_LOSS_SLOTS];

namespace {

constexpr int NA_T = 256;
constexpr int NA_PER = 8;  // 2048 pixels per block

struct NaViews {
  int32_t W[TS_MAX_VIEWS], H[TS_MAX_VIEWS];
  long long pix_off[TS_MAX_VIEWS];
};

__global__ void __launch_bounds__(NA_T) k_na_loss_partial(NaViews tab, const float* __restrict__ C,
                                                          const float* __restrict__ D, const float* __restrict__ tC,
                                                          const float* __restrict__ tD, float lambda_dep,
                                                          float* __restrict__ dC, float* __restrict__ dD,
                                                          float* __restrict__ part, int nblk) {
  __shared__ float red[NA_T / 32][2];
  const int v = blockIdx.y;
  const long long HW = (long long)tab.W[v] * tab.H[v];
  const long long po = tab.pix_off[v];
  const long long base = (long long)blockIdx.x * NA_T * NA_PER;
  float lc = 0.f, ld = 0.f;
  if (base < HW) {
    const float ic = 1.0f / (3.0f * (float)HW), id = lambda_dep / (float)HW;
    for (int k = 0; k < NA_PER; ++k) {
      const long long i = base + (long long)k * NA_T + threadIdx.x;
      if (i >= HW) break;
      for (int ch = 0; ch < 3; ++ch) {
        const long long o = 3 * po + ch * HW + i;
        const float r = C[o] - tC[o];
        lc += fabsf(r);
        dC[o] = r > 0.f ? ic : (r < 0.f ? -ic : 0.f);
      }
      const long long o = po + i;
      const float t = tD[o];
      const float r = D[o] - t;
      const bool valid = t > 0.f;
      if (valid) ld += fabsf(r);
      dD[o] = valid ? (r > 0.f ? id : (r < 0.f ? -id : 0.f)) : 0.f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lc += __shfl_xor_sync(0xffffffffu, lc, o);
    ld += __shfl_xor_sync(0xffffffffu, ld, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = lc;
    red[threadIdx.x >> 5][1] = ld;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float s = 0.f;
    for (int w = 0; w < NA_T / 32; ++w) s += red[w][threadIdx.x];
    part[((long long)v * nblk + blockIdx.x) * 2 + threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(NA_T) k_na_loss_final(NaViews tab, const float* __restrict__ part, int nblk,
                                                        float lambda_dep, float* __restrict__ loss) {
  __shared__ float red[NA_T][2];
  const int v = blockIdx.x;
  float a = 0.f, b = 0.f;
  for (int k = threadIdx.x; k < nblk; k += NA_T) {
    a += part[((long long)v * nblk + k) * 2];
    b += part[((long long)v * nblk + k) * 2 + 1];
  }
  red[threadIdx.x][0] = a;
  red[threadIdx.x][1] = b;
  __syncthreads();
  for (int o = NA_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x][0] += red[threadIdx.x + o][0];
      red[threadIdx.x][1] += red[threadIdx.x + o][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double HW = (double)tab.W[v] * tab.H[v];
    loss[v] = (float)((double)red[0][0] / (3.0 * HW) + (double)lambda_dep * (double)red[0][1] / HW);
  }
}

std::mutex g_setup_mutex;
float* g_partials_ptr[TS_NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the static scratch array on the current device (looked up once per device).
ts_status scratch_on_current_device(float** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TS_NOALLOC_MAX_DEVICES) return TS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_loss_partials) != cudaSuccess || !p) return TS_ERR_CUDA;
    g_partials_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_partials_ptr[dev];
  return TS_OK;
}

}  // namespace

extern "C" ts_status ts_l1_loss_noalloc(const ts_camera* cams, int32_t n_views, const float* color, const float* depth,
                                        const float* tgt_color, const float* tgt_depth, float lambda_dep,
                                        float* loss, float* dC, float* dD, ts_stream stream) {
  if (!cams || n_views < 1 || n_views > TS_MAX_VIEWS) return TS_ERR_INVALID_ARG;
  if (!color || !depth || !tgt_color || !tgt_depth || !loss || !dC || !dD || !(lambda_dep >= 0.0f))
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
