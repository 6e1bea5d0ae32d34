// k_loss.cu -- the tracking/mapping loss of the raster path and the pose update.
//
// Loss (Eq. 8 L1 part and Eq. 9, per view): sum |C - Cbar| / (3HW) + lambda_dep *
// sum_{Dbar > 0} |D - Dbar| / (HW), with its gradient written in the same pass; partial sums
// per block are reduced in a fixed order so the loss is deterministic.  The normal loss of
// Eq. 12 follows the same pattern.
// Pose update: T <- Exp(-step) o T with the closed-form SE(3) exponential (left perturbation,
// step = (rho, theta)), used by gradient-descent tracking (Sec. 3.3).
#include <algorithm>

#include "ts_internal.cuh"

namespace {

constexpr int LOSS_T = 256;
constexpr int LOSS_PER = 8;  // pixels per thread; 2048 per block

__global__ void __launch_bounds__(LOSS_T) k_loss_partial(const TsImageTable tab, const float* __restrict__ C,
                                                         const float* __restrict__ D, const float* __restrict__ tC,
                                                         const float* __restrict__ tD, float lambda_dep,
                                                         float* __restrict__ dC, float* __restrict__ dD,
                                                         float* __restrict__ part, int nblk) {
  const int v = blockIdx.y;
  ts_l1_loss_block<LOSS_T, LOSS_PER>((long long)tab.W[v] * tab.H[v], tab.pix_off[v],
                                     (long long)blockIdx.x * LOSS_T * LOSS_PER, C, D, tC, tD, lambda_dep, dC, dD,
                                     part + ((long long)v * nblk + blockIdx.x) * 2);
}

__global__ void __launch_bounds__(LOSS_T) k_loss_final(const TsImageTable tab, const float* __restrict__ part,
                                                       int nblk, float lambda_dep, float* __restrict__ loss) {
  const int v = blockIdx.x;
  ts_l1_loss_final<LOSS_T>((long long)tab.W[v] * tab.H[v], part + (long long)v * nblk * 2, nblk, lambda_dep, loss + v);
}

// Normal loss of Eq. 12 per view: sum over pixels with a sensor normal (Nbar != 0) of
// (1 - N . Nbar) / HW, with dN = weight * dloss/dN = -weight Nbar / HW there and 0 elsewhere.
__global__ void __launch_bounds__(LOSS_T) k_nloss_partial(const TsImageTable tab, const float* __restrict__ N,
                                                          const float* __restrict__ tN, float weight,
                                                          float* __restrict__ dN, float* __restrict__ part, int nblk) {
  __shared__ float red[LOSS_T / 32];
  const int v = blockIdx.y;
  const long long HW = (long long)tab.W[v] * tab.H[v];
  const long long pix_off = tab.pix_off[v];
  const long long base = (long long)blockIdx.x * LOSS_T * LOSS_PER;
  float l = 0.f;
  if (base < HW) {
    const float sc = -weight / (float)HW;
#pragma unroll
    for (int k = 0; k < LOSS_PER; ++k) {
      const long long i = base + (long long)k * LOSS_T + threadIdx.x;
      if (i >= HW) break;
      float nb[3], dot = 0.f;
      bool valid = false;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const long long o = 3 * pix_off + ch * HW + i;
        nb[ch] = tN[o];
        valid = valid || nb[ch] != 0.f;
        dot += N[o] * nb[ch];
      }
      if (valid) l += 1.f - dot;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) dN[3 * pix_off + ch * HW + i] = valid ? sc * nb[ch] : 0.f;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < LOSS_T / 32; ++w) s += red[w];
    part[(long long)v * nblk + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(LOSS_T) k_nloss_final(const TsImageTable tab, const float* __restrict__ part,
                                                        int nblk, float* __restrict__ loss) {
  __shared__ double red[LOSS_T];
  const int v = blockIdx.x;
  double a = 0;
  for (int k = threadIdx.x; k < nblk; k += LOSS_T) a += part[(long long)v * nblk + k];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = LOSS_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[v] = (float)(red[0] / ((double)tab.W[v] * tab.H[v]));
}

// T <- Exp(-st) o T for one view (closed-form SE(3) exponential, st = (rho, theta)).
__device__ void pose_left_step(ts_pose* poses, int v, const float st[6]) {
  const float rho[3] = {-st[0], -st[1], -st[2]};
  const float w0 = -st[3], w1 = -st[4], w2 = -st[5];
  const float a2 = w0 * w0 + w1 * w1 + w2 * w2;
  const float a = sqrtf(a2);
  float A, B, Cc;  // sin a / a, (1 - cos a) / a^2, (a - sin a) / a^3
  if (a < 1e-3f) {
    A = 1.f - a2 / 6.f;
    B = 0.5f - a2 / 24.f;
    Cc = 1.f / 6.f - a2 / 120.f;
  } else {
    const float sa = sinf(a), ca = cosf(a);
    A = sa / a;
    B = (1.f - ca) / a2;
    Cc = (a - sa) / (a2 * a);
  }
  const float K[9] = {0.f, -w2, w1, w2, 0.f, -w0, -w1, w0, 0.f};
  float K2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  float R[9], Vm[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float I3 = (i % 4 == 0) ? 1.f : 0.f;
    R[i] = I3 + A * K[i] + B * K2[i];
    Vm[i] = I3 + B * K[i] + Cc * K2[i];
  }
  float te[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) te[i] = Vm[3 * i] * rho[0] + Vm[3 * i + 1] * rho[1] + Vm[3 * i + 2] * rho[2];
  ts_pose P = poses[v];
  ts_pose Q;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.R[3 * i + j] = R[3 * i] * P.R[j] + R[3 * i + 1] * P.R[3 + j] + R[3 * i + 2] * P.R[6 + j];
    Q.t[i] = R[3 * i] * P.t[0] + R[3 * i + 1] * P.t[1] + R[3 * i + 2] * P.t[2] + te[i];
  }
  poses[v] = Q;
}

__global__ void k_pose_apply(ts_pose* poses, const float* __restrict__ step, int V) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float st[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) st[i] = step[6 * v + i];
  pose_left_step(poses, v, st);
}

// Adam on the manifold gradient dL/dtau of each view (Sec. 3.3 tracking; learning rates per
// block: rho (translation) and theta (rotation), Table S5), then T <- Exp(-step) o T.
// state[v] = first moments (6), second moments (6), step count (1); updated in place so the
// iteration can be replayed from a CUDA graph.
__global__ void k_pose_adam(ts_pose* poses, const float* __restrict__ dtau, float* __restrict__ state, int V,
                            float lr_rho, float lr_theta, float b1, float b2, float eps) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float* s = state + 13 * v;
  const float t = s[12] + 1.0f;
  s[12] = t;
  const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
  float st[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float g = dtau[6 * v + i];
    const float m = b1 * s[i] + (1.0f - b1) * g;
    const float q = b2 * s[6 + i] + (1.0f - b2) * g * g;
    s[i] = m;
    s[6 + i] = q;
    st[i] = (i < 3 ? lr_rho : lr_theta) * (m / c1) / (sqrtf(q / c2) + eps);
  }
  pose_left_step(poses, v, st);
}

// Failure-detection probe: one thread waits on an mbarrier phase that nothing completes (no
// arrival, no copy in flight) with the library's bounded wait, and latches the timeout bit when
// the limit passes.
__global__ void k_timeout_probe(TsDevHeader* hdr, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  ts_mbar_init(&bar, 1);
  ts_fence_mbar_init();
  if (!ts_mbar_wait(&bar, 0u, limit_ns)) atomicOr(&hdr->error_bits, TS_ERRBIT_TIMEOUT);
}

}  // namespace

cudaError_t ts_launch_timeout_probe(const TsWs& w, unsigned long long limit_ns, cudaStream_t s) {
  k_timeout_probe<<<1, 32, 0, s>>>(w.hdr, limit_ns);
  return cudaGetLastError();
}

cudaError_t ts_launch_l1_loss(const TsPlanImpl* p, const TsWs& w, const float* color, const float* depth,
                              const float* tc, const float* td, float lambda_dep, float* loss, float* dC, float* dD,
                              cudaStream_t s) {
  const int nblk = (int)p->n_loss_blocks;
  dim3 grid((unsigned)nblk, (unsigned)p->V);
  const TsImageTable tab = ts_image_table(p);
  k_loss_partial<<<grid, LOSS_T, 0, s>>>(tab, color, depth, tc, td, lambda_dep, dC, dD, w.loss, nblk);
  k_loss_final<<<p->V, LOSS_T, 0, s>>>(tab, w.loss, nblk, lambda_dep, loss);
  return cudaGetLastError();
}

cudaError_t ts_launch_normal_loss(const TsPlanImpl* p, const TsWs& w, const float* normal, const float* tgt,
                                  float weight, float* loss, float* dN, cudaStream_t s) {
  const int nblk = (int)p->n_loss_blocks;
  const TsImageTable tab = ts_image_table(p);
  k_nloss_partial<<<dim3((unsigned)nblk, (unsigned)p->V), LOSS_T, 0, s>>>(tab, normal, tgt, weight, dN, w.nloss, nblk);
  k_nloss_final<<<p->V, LOSS_T, 0, s>>>(tab, w.nloss, nblk, loss);
  return cudaGetLastError();
}

cudaError_t ts_launch_pose_apply(const TsPlanImpl* p, ts_pose* poses, const float* step, cudaStream_t s) {
  k_pose_apply<<<(p->V + 63) / 64, 64, 0, s>>>(poses, step, p->V);
  return cudaGetLastError();
}

cudaError_t ts_launch_pose_adam(const TsPlanImpl* p, ts_pose* poses, const float* dtau, float* state, float lr_rho,
                                float lr_theta, float b1, float b2, float eps, cudaStream_t s) {
  k_pose_adam<<<(p->V + 63) / 64, 64, 0, s>>>(poses, dtau, state, p->V, lr_rho, lr_theta, b1, b2, eps);
  return cudaGetLastError();
}
