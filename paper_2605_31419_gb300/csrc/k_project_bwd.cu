// k_project_bwd.cu -- chain rule from the per-face screen-space sums to the map and the pose.
//
// One thread per face loops over the views.  For each view where the face was visible it reads
// (and clears, so the accumulator is zero for the next call) the 24 sums written by the raster
// backward, recomputes the projection in the same fixed FP32 order as the forward pass, and
// applies, in closed form:
//   * interpolants with vertex values w (colour channels, camera depth): dL/dw_k is the sum
//     itself, and moving vertex k moves the interpolant's plane: dL/dq_k -= dL/dw_k * grad f;
//   * edge functions E_i = s_i lambda_{i+2} with s_i = perimeter / |e_i| (Eq. 2-3 normalised
//     by phi(s), the inradius): the same plane term plus the chain through the edge lengths;
//   * o_F = (o_i + o_j + o_k) / 3 (Sec. 3.1): each vertex opacity gets a third;
//   * the pinhole (Eq. 1) to camera space, R^T to world space, and the left-perturbation pose
//     Jacobian [I, -[v_C]x] (Eq. 7): dL/dtau += [g_C ; v_C x g_C].
// The per-view pose terms are reduced over the block (fixed order) into per-block partials; a
// second kernel sums the partials of each view in a fixed order, so dtau is deterministic.
#include "ts_internal.cuh"

namespace {

struct PBArgs {
  const TsView* views;
  const ts_pose* poses;
  int V;
  long long M;
  const uint32_t* count;
  float* grad;
  const TsDevHeader* hdr;
  float *gpx, *gpy, *gpz, *gcr, *gcg, *gcb, *gop;
  float* part;
  int nblocks;
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void __launch_bounds__(256) k_project_bwd(PBArgs a) {
  __shared__ float red[8][6];
  const long long m = (long long)blockIdx.x * 256 + threadIdx.x;
  const bool valid = m < a.M;
  const TsDevHeader* h = a.hdr;
  long long vi[3] = {0, 0, 0};
  float X[3][3], col[3][3];
  if (valid) {
    if (h->faces) {
      vi[0] = h->faces[3 * m]; vi[1] = h->faces[3 * m + 1]; vi[2] = h->faces[3 * m + 2];
    } else {
      vi[0] = 3 * m; vi[1] = 3 * m + 1; vi[2] = 3 * m + 2;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long j = (vi[k] >= 0 && vi[k] < h->n_vertices) ? vi[k] : 0;
      X[k][0] = h->px[j]; X[k][1] = h->py[j]; X[k][2] = h->pz[j];
      col[k][0] = h->cr[j]; col[k][1] = h->cg[j]; col[k][2] = h->cb[j];
    }
  }
  float dpos[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  float dcol[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  float dop = 0.f;  // same for all three vertices
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < a.V; ++v) {
    float tau[6] = {0, 0, 0, 0, 0, 0};
    const long long slot = (long long)v * a.M + m;
    if (valid && a.count[slot] > 0) {
      float G[24];
      float4* gp = reinterpret_cast<float4*>(a.grad + slot * TS_GRAD_WORDS);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float4 q = gp[i];
        G[4 * i] = q.x; G[4 * i + 1] = q.y; G[4 * i + 2] = q.z; G[4 * i + 3] = q.w;
        gp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const TsView vw = a.views[v];
      const ts_pose P = a.poses[v];
      float xc[3], yc[3], zc[3], u[3], w[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ts_rigid_f32(P, X[k][0], X[k][1], X[k][2], xc[k], yc[k], zc[k]);
        ts_pinhole_f32(vw, xc[k], yc[k], zc[k], u[k], w[k]);
      }
      float ex[3], ey[3], len[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3;
        ex[i] = u[j] - u[i];
        ey[i] = w[j] - w[i];
        len[i] = sqrtf(ex[i] * ex[i] + ey[i] * ey[i]);
      }
      const float per = len[0] + len[1] + len[2];
      const float D2 = (u[1] - u[0]) * (w[2] - w[0]) - (u[2] - u[0]) * (w[1] - w[0]);
      const float invD = 1.0f / D2;
      float A[3], B[3];  // gradient of the barycentric lambda_k
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        A[k] = (w[k1] - w[k2]) * invD;
        B[k] = (u[k2] - u[k1]) * invD;
      }
      float s[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) s[i] = per / len[i];
      float fa[3], fb[3];  // colour-field gradients
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        fa[ch] = col[0][ch] * A[0] + col[1][ch] * A[1] + col[2][ch] * A[2];
        fb[ch] = col[0][ch] * B[0] + col[1][ch] * B[1] + col[2][ch] * B[2];
      }
      const float za = zc[0] * A[0] + zc[1] * A[1] + zc[2] * A[2];
      const float zb = zc[0] * B[0] + zc[1] * B[1] + zc[2] * B[2];
      float gu[3], gv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float su = G[G_Z + k] * za, sv = G[G_Z + k] * zb;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          su += G[G_C + 3 * ch + k] * fa[ch];
          sv += G[G_C + 3 * ch + k] * fb[ch];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int o = (i + 2) % 3;
          su += G[G_E + 3 * i + k] * s[i] * A[o];
          sv += G[G_E + 3 * i + k] * s[i] * B[o];
        }
        gu[k] = -su;
        gv[k] = -sv;
      }
      // edge lengths through s_i = per / len_i
      float ds[3], sum_ds_len = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ds[i] = G[G_E + 3 * i + (i + 2) % 3];
        sum_ds_len += ds[i] / len[i];
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float dlen = sum_ds_len - ds[j] * per / (len[j] * len[j]);
        const float cx = dlen * ex[j] / len[j], cy = dlen * ey[j] / len[j];
        const int j1 = (j + 1) % 3;
        gu[j1] += cx; gv[j1] += cy;
        gu[j] -= cx; gv[j] -= cy;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float iz = 1.0f / zc[k];
        const float gx = gu[k] * vw.fx * iz;
        const float gy = gv[k] * vw.fy * iz;
        const float gz = -(gx * xc[k] + gy * yc[k]) * iz + G[G_Z + k];  // pinhole + interpolated depth
        // world-space gradient R^T g_C
        dpos[k][0] += P.R[0] * gx + P.R[3] * gy + P.R[6] * gz;
        dpos[k][1] += P.R[1] * gx + P.R[4] * gy + P.R[7] * gz;
        dpos[k][2] += P.R[2] * gx + P.R[5] * gy + P.R[8] * gz;
        tau[0] += gx; tau[1] += gy; tau[2] += gz;
        tau[3] += yc[k] * gz - zc[k] * gy;
        tau[4] += zc[k] * gx - xc[k] * gz;
        tau[5] += xc[k] * gy - yc[k] * gx;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) dcol[k][ch] += G[G_C + 3 * ch + k];
      }
      dop += G[G_O] * (1.0f / 3.0f);
    }
    // fixed-order block reduction of the pose terms of view v
#pragma unroll
    for (int i = 0; i < 6; ++i) tau[i] = warp_sum(tau[i]);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) red[warp][i] = tau[i];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
      a.part[((long long)v * a.nblocks + blockIdx.x) * 6 + threadIdx.x] = s;
    }
    __syncthreads();
  }
  if (!valid) return;
  float* gp3[3] = {a.gpx, a.gpy, a.gpz};
  float* gc3[3] = {a.gcr, a.gcg, a.gcb};
  const bool indexed = h->faces != nullptr;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long j = vi[k];
    if (j < 0 || j >= h->n_vertices) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (gp3[c]) {
        if (indexed) atomicAdd(gp3[c] + j, dpos[k][c]); else gp3[c][j] += dpos[k][c];
      }
      if (gc3[c]) {
        if (indexed) atomicAdd(gc3[c] + j, dcol[k][c]); else gc3[c][j] += dcol[k][c];
      }
    }
    if (a.gop) {
      if (indexed) atomicAdd(a.gop + j, dop); else a.gop[j] += dop;
    }
  }
}

__global__ void __launch_bounds__(256) k_pose_reduce(const float* __restrict__ part, int nblocks, float* dtau) {
  __shared__ float red[256][6];
  const int v = blockIdx.x;
  float s[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += 256) {
    const float* p = part + ((long long)v * nblocks + b) * 6;
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] += p[i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) red[threadIdx.x][i] = s[i];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int i = 0; i < 6; ++i) red[threadIdx.x][i] += red[threadIdx.x + o][i];
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) dtau[v * 6 + threadIdx.x] = red[0][threadIdx.x];
}

}  // namespace

cudaError_t ts_launch_project_bwd(const TsPlanImpl* p, const TsWs& w, const ts_map_grad* g, cudaStream_t s) {
  if (p->M == 0) {
    return cudaMemsetAsync(w.pose, 0, (size_t)p->V * p->n_pose_blocks * 6 * 4, s);
  }
  PBArgs a;
  a.views = w.views;
  a.poses = w.poses;
  a.V = p->V;
  a.M = p->M;
  a.count = w.count;
  a.grad = w.grad;
  a.hdr = w.hdr;
  a.gpx = g->gpx; a.gpy = g->gpy; a.gpz = g->gpz;
  a.gcr = g->gcr; a.gcg = g->gcg; a.gcb = g->gcb;
  a.gop = g->gop;
  a.part = w.pose;
  a.nblocks = (int)p->n_pose_blocks;
  k_project_bwd<<<(unsigned)p->n_pose_blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t ts_launch_pose_reduce(const TsPlanImpl* p, const TsWs& w, float* dtau, cudaStream_t s) {
  k_pose_reduce<<<p->V, 256, 0, s>>>(w.pose, (int)p->n_pose_blocks, dtau);
  return cudaGetLastError();
}
