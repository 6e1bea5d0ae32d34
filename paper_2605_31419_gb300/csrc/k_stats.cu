// k_stats.cu -- the map statistics that Sec. 3.4's map management reads from a render:
//   * pixel coverage per (view, face), counted by the forward blend (TS_FLAG_STATS): the number of
//     pixels at which the face was blended; densification splits faces whose coverage exceeds
//     theta_blur * H * W;
//   * projected area per (view, face): |D2| / 2 of the projected triangle, recomputed from the
//     record's vertices in the projection's fixed FP32 operation order (bit-identical to the
//     value culling saw); pruning removes faces above epsilon_a pixels;
//   * per-view visible-face bitsets and counts, and the co-visibility IoU between views that
//     keyframe selection compares.
#include "ts_internal.cuh"

namespace {

constexpr int ST_T = 256;

struct StatsArgs {
  const float4* frec;
  const uint32_t* count;
  const uint32_t* cov_in;
  long long M;
  int words;  // ceil(M / 32)
  uint32_t* coverage;
  float* area;
  uint32_t* visible;
  uint32_t* n_visible;
};

// grid (ceil(M / 256), V): thread = face m of view v; a warp covers 32 faces of one view, so its
// ballot is one word of the view's bitset
__global__ void __launch_bounds__(ST_T) k_face_stats(StatsArgs a) {
  const int v = blockIdx.y;
  const long long m = (long long)blockIdx.x * ST_T + threadIdx.x;
  const long long idx = (long long)v * a.M + m;
  const bool in = m < a.M;
  const bool proj = in && a.count[idx] > 0;
  const uint32_t cov = (proj && a.cov_in) ? a.cov_in[idx] : 0u;
  if (in && a.coverage) a.coverage[idx] = cov;
  if (in && a.area) {
    float ar = 0.f;
    if (proj) {
      const float* r = reinterpret_cast<const float*>(a.frec + idx * (TS_REC_WORDS / 4));
      const float du1 = __fsub_rn(r[R_U1], r[R_U0]), dv1 = __fsub_rn(r[R_V1], r[R_V0]);
      const float du2 = __fsub_rn(r[R_U2], r[R_U0]), dv2 = __fsub_rn(r[R_V2], r[R_V0]);
      ar = 0.5f * fabsf(__fsub_rn(__fmul_rn(du1, dv2), __fmul_rn(du2, dv1)));
    }
    a.area[idx] = ar;
  }
  if (a.visible || a.n_visible) {
    const unsigned bal = __ballot_sync(0xffffffffu, cov > 0);
    if ((threadIdx.x & 31) == 0 && m < a.M) {
      if (a.visible) a.visible[(long long)v * a.words + (m >> 5)] = bal;
      if (a.n_visible && bal) atomicAdd(a.n_visible + v, (unsigned)__popc(bal));
    }
  }
}

// iou[i][j] = |S_i & S_j| / |S_i | S_j| over the views' bitsets (0 when both sets are empty)
__global__ void __launch_bounds__(ST_T) k_covis(const uint32_t* __restrict__ bits, int words, int V,
                                                float* __restrict__ iou) {
  __shared__ unsigned long long red[2][ST_T / 32];
  const int i = blockIdx.y, j = blockIdx.x;
  const uint32_t* a = bits + (long long)i * words;
  const uint32_t* b = bits + (long long)j * words;
  unsigned long long in = 0, un = 0;
  for (int k = threadIdx.x; k < words; k += ST_T) {
    const uint32_t x = a[k], y = b[k];
    in += __popc(x & y);
    un += __popc(x | y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    in += __shfl_xor_sync(0xffffffffu, in, o);
    un += __shfl_xor_sync(0xffffffffu, un, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = in;
    red[1][threadIdx.x >> 5] = un;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long si = 0, su = 0;
#pragma unroll
    for (int w = 0; w < ST_T / 32; ++w) {
      si += red[0][w];
      su += red[1][w];
    }
    iou[(long long)i * V + j] = su ? (float)((double)si / (double)su) : 0.f;
  }
}

}  // namespace

cudaError_t ts_launch_face_stats(const TsPlanImpl* p, const TsWs& w, uint32_t* coverage, float* area,
                                 uint32_t* visible, uint32_t* n_visible, cudaStream_t s) {
  if (n_visible) {
    cudaError_t e = cudaMemsetAsync(n_visible, 0, sizeof(uint32_t) * p->V, s);
    if (e != cudaSuccess) return e;
  }
  if (p->M == 0) return cudaSuccess;
  StatsArgs a;
  a.frec = w.frec;
  a.count = w.count;
  a.cov_in = w.cov;
  a.M = p->M;
  a.words = (int)((p->M + 31) / 32);
  a.coverage = coverage;
  a.area = area;
  a.visible = visible;
  a.n_visible = n_visible;
  k_face_stats<<<dim3((unsigned)((p->M + ST_T - 1) / ST_T), (unsigned)p->V), ST_T, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t ts_launch_covisibility(const TsPlanImpl* p, const uint32_t* visible, float* iou, cudaStream_t s) {
  const int words = (int)((p->M + 31) / 32);
  k_covis<<<dim3((unsigned)p->V, (unsigned)p->V), ST_T, 0, s>>>(visible, words, p->V, iou);
  return cudaGetLastError();
}
