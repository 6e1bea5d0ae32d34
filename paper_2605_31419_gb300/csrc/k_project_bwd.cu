// k_project_bwd.cu -- chain rule from the per-face screen-space sums to the map and the pose.
//
// Closed form per visible (view, face), from the 24 sums the raster backward accumulated:
//   * interpolants with vertex values w (colour channels, camera depth): dL/dw_k is the sum
//     itself, and moving vertex k moves the interpolant's plane: dL/dq_k -= dL/dw_k * grad f;
//   * edge functions E_i = s_i lambda_{i+2} with s_i = perimeter / |e_i| (Eq. 2-3 normalised
//     by phi(s), the inradius): the same plane term plus the chain through the edge lengths;
//   * o_F = (o_i + o_j + o_k) / 3 (Sec. 3.1): each vertex opacity gets a third;
//   * with TS_FLAG_NORMALS, the face normal of the normal map (Eq. 12) through the cross product
//     of the camera-space edge vectors; with TS_FLAG_FACE_SIGMA, dL/dsigma_F (a sum the raster
//     backward already formed, word 24) is summed over views;
//   * the pinhole (Eq. 1) to camera space, R^T to world space, and the left-perturbation pose
//     Jacobian [I, -[v_C]x] (Eq. 7): dL/dtau += [g_C ; v_C x g_C].
//
// Gradient slots are face-major (slot = face * V + view) and cleared by the projection pass for
// the visible ones.  Persistent warps take 4 faces at a time; one ballot per face and 32 views
// gives the face's visible views.  Lanes 0..20 each own one output word (3 positions x 3 vertices,
// 3 colours x 3 vertices, the opacity; lane 21 sigma_F), sum it over the face's visible views in
// view order and add it to the map gradient.  Each view's pose terms are added to the warp's
// per-view sums in shared memory in face order; at the end the warps' sums are added in a fixed
// order into per-block partials, which a last kernel adds in a fixed order.  Two forms, with the
// same arithmetic and the same summation orders (so the same results):
//   * one pass (8 or more views): the 4 faces' (face, view) entries, numbered face by face with
//     views in order, run the chain rule one per lane (batches of 32), each lane leaving its
//     entry's 20 map words in a shared-memory row that the word lanes sum; each slot is read
//     once and nothing is written back;
//   * two passes (fewer views, where 4 faces fill few lanes): A. persistent warps scan the
//     visibility counts, queue the visible slots with ballots and run the chain rule on full warps,
//     writing each slot's results back into it; B. the word lanes sum the written-back words,
//     with up to 8 loads in flight.

#include <algorithm>

#include "ts_internal.cuh"

namespace {

struct PBArgs {
  const TsView* views;
  const ts_pose* poses;
  int V;
  long long M, VM;
  const uint32_t* count;
  float* grad;
  const float4* aux;  // per (view, face) normal and sigma_F (TS_FLAG_NORMALS / TS_FLAG_FACE_SIGMA)
  bool normals, face_sigma;
  float* dst_sigma;  // dL/dsigma_F per face (TS_FLAG_FACE_SIGMA), may be null
  const TsDevHeader* hdr;
  float* dst[7];  // gpx, gpy, gpz, gcr, gcg, gcb, gop
  bool min_opacity;  // o_F = min of the vertex opacities: dL/do_F to the first minimal vertex
  float* part;
  int nblocks;
};

__device__ __forceinline__ long long face_vertex(const TsDevHeader* h, long long m, int k) {
  long long j = h->faces ? (long long)h->faces[3 * m + k] : 3 * m + k;
  return (j >= 0 && j < h->n_vertices) ? j : 0;
}

// One 32-byte load (eight floats) from a 32-byte aligned global address.
__device__ __forceinline__ void ld_v8(const float* p, float* o) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
               : "l"(p)
               : "memory");
}

// What the chain rule of one visible (view, face) gives: the world-space vertex-position
// gradients, the pose terms, and the slot's colour, opacity and sigma_F sums passed through.
struct SlotTerms {
  float out[9];  // dL/dp of vertex k, coordinate c at 3k + c
  float tau[6];  // [g_C ; v_C x g_C] summed over the vertices
  float gc[9];   // dL/dc of vertex k, channel ch at 3 ch + k (the raster sums)
  float go;      // dL/do_F
  float gsig;    // dL/dsigma_F (TS_FLAG_FACE_SIGMA)
};

// The chain rule of one visible (view, face).
__device__ __forceinline__ void chain_terms(const PBArgs& a, int v, long long m, SlotTerms& t) {
  const TsDevHeader* h = a.hdr;
  const long long slot = m * a.V + v;
  const float* gw = a.grad + slot * TS_GRAD_WORDS;
  float G[24];
  ld_v8(gw, G);
  ld_v8(gw + 8, G + 8);
  ld_v8(gw + 16, G + 16);
  const float gsig = a.face_sigma ? gw[24] : 0.f;  // word 24
  const TsView vw = a.views[v];
  const ts_pose P = a.poses[v];
  // The projection, edge vectors, lengths and area are recomputed in the forward record's fixed
  // operation order, so the chain rule sees bit-identical values; for slivers the area is a
  // cancelling difference and a one-ulp change of a vertex would move the gradient visibly.
  float xc[3], yc[3], zc[3], u[3], w[3], col[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long j = face_vertex(h, m, k);
    ts_rigid_f32(P, __ldg(h->px + j), __ldg(h->py + j), __ldg(h->pz + j), xc[k], yc[k], zc[k]);
    ts_pinhole_f32(vw, xc[k], yc[k], zc[k], u[k], w[k]);
    col[k][0] = __ldg(h->cr + j); col[k][1] = __ldg(h->cg + j); col[k][2] = __ldg(h->cb + j);
  }
  float ex[3], ey[3], len[3], il[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3;
    ex[i] = u[j] - u[i];
    ey[i] = w[j] - w[i];
    len[i] = __fsqrt_rn(__fadd_rn(__fmul_rn(ex[i], ex[i]), __fmul_rn(ey[i], ey[i])));
    il[i] = 1.0f / len[i];
  }
  const float per = __fadd_rn(__fadd_rn(len[0], len[1]), len[2]);
  const float D2 = __fsub_rn(__fmul_rn(__fsub_rn(u[1], u[0]), __fsub_rn(w[2], w[0])),
                             __fmul_rn(__fsub_rn(u[2], u[0]), __fsub_rn(w[1], w[0])));
  const float invD = 1.0f / D2;
  float A[3], B[3];  // gradient of the barycentric lambda_k
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    A[k] = (w[k1] - w[k2]) * invD;
    B[k] = (u[k2] - u[k1]) * invD;
  }
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
      const float si = per * il[i];
      su += G[G_E + 3 * i + k] * si * A[o];
      sv += G[G_E + 3 * i + k] * si * B[o];
    }
    gu[k] = -su;
    gv[k] = -sv;
  }
  // edge lengths through s_i = per / len_i: dL/dlen_j = sum_i dL/ds_i / len_i - dL/ds_j per / len_j^2
  float ds[3], sum_ds_len = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ds[i] = G[G_E + 3 * i + (i + 2) % 3];
    sum_ds_len += ds[i] * il[i];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float dlen = sum_ds_len - ds[j] * per * il[j] * il[j];
    const float cx = dlen * ex[j] * il[j], cy = dlen * ey[j] * il[j];
    const int j1 = (j + 1) % 3;
    gu[j1] += cx; gv[j1] += cy;
    gu[j] -= cx; gv[j] -= cy;
  }
  // normal map (Eq. 12): dL/dn_F from words 23, 30, 31 through n = s u / |u|, u = e1 x e2 with
  // e1 = v1 - v0, e2 = v2 - v0 in camera space and s = +-1 the camera-facing turn of the forward:
  // dL/du = s (g - n (n . g)) / |u|, dL/de1 = e2 x dL/du, dL/de2 = dL/du x e1
  float ng[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (a.normals) {
    const float gn[3] = {G[23], a.grad[slot * TS_GRAD_WORDS + 30], a.grad[slot * TS_GRAD_WORDS + 31]};
    if (gn[0] != 0.f || gn[1] != 0.f || gn[2] != 0.f) {
      const float4 nn = a.aux[(long long)v * a.M + m];
      const float e1[3] = {xc[1] - xc[0], yc[1] - yc[0], zc[1] - zc[0]};
      const float e2[3] = {xc[2] - xc[0], yc[2] - yc[0], zc[2] - zc[0]};
      const float uu[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      const float il2 = rsqrtf(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
      const float sg = (nn.x * uu[0] + nn.y * uu[1] + nn.z * uu[2]) < 0.f ? -1.f : 1.f;
      const float n[3] = {sg * uu[0] * il2, sg * uu[1] * il2, sg * uu[2] * il2};
      const float ndg = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];
      float du[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) du[r] = sg * il2 * (gn[r] - n[r] * ndg);
      const float d1[3] = {e2[1] * du[2] - e2[2] * du[1], e2[2] * du[0] - e2[0] * du[2], e2[0] * du[1] - e2[1] * du[0]};
      const float d2[3] = {du[1] * e1[2] - du[2] * e1[1], du[2] * e1[0] - du[0] * e1[2], du[0] * e1[1] - du[1] * e1[0]};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ng[1][r] = d1[r];
        ng[2][r] = d2[r];
        ng[0][r] = -(d1[r] + d2[r]);
      }
    }
  }
  float* out = t.out;
  float* tau = t.tau;
#pragma unroll
  for (int i = 0; i < 6; ++i) tau[i] = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float iz = 1.0f / zc[k];
    const float gxp = gu[k] * vw.fx * iz;
    const float gyp = gv[k] * vw.fy * iz;
    const float gz = -(gxp * xc[k] + gyp * yc[k]) * iz + G[G_Z + k] + ng[k][2];  // pinhole + depth + normal
    const float gx = gxp + ng[k][0], gy = gyp + ng[k][1];
    out[3 * k + 0] = P.R[0] * gx + P.R[3] * gy + P.R[6] * gz;  // R^T g_C
    out[3 * k + 1] = P.R[1] * gx + P.R[4] * gy + P.R[7] * gz;
    out[3 * k + 2] = P.R[2] * gx + P.R[5] * gy + P.R[8] * gz;
    tau[0] += gx; tau[1] += gy; tau[2] += gz;
    tau[3] += yc[k] * gz - zc[k] * gy;
    tau[4] += zc[k] * gx - xc[k] * gz;
    tau[5] += xc[k] * gy - yc[k] * gx;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) t.gc[i] = G[G_C + i];
  t.go = G[G_O];
  t.gsig = gsig;
}

// Two-pass form, pass A: the chain rule of one visible (view, face), written back into its slot:
// positions into words 0..8 (the edge sums, now consumed), pose terms into 24..29, sigma_F into 23.
__device__ __forceinline__ void chain_slot(const PBArgs& a, int v, long long m) {
  SlotTerms t;
  chain_terms(a, v, m, t);
  float* gs = a.grad + (m * a.V + v) * TS_GRAD_WORDS;
  float4* gp = reinterpret_cast<float4*>(gs);
  gp[0] = make_float4(t.out[0], t.out[1], t.out[2], t.out[3]);
  gp[1] = make_float4(t.out[4], t.out[5], t.out[6], t.out[7]);
  gs[8] = t.out[8];
  gp[6] = make_float4(t.tau[0], t.tau[1], t.tau[2], t.tau[3]);
  gs[28] = t.tau[4];
  gs[29] = t.tau[5];
  if (a.face_sigma) gs[23] = t.gsig;
}

constexpr int PA_T = 256;
constexpr int PA_WARPS = PA_T / 32;

__global__ void __launch_bounds__(PA_T) k_pbwd_chain(PBArgs a) {
  __shared__ long long q[PA_WARPS][64];  // queued view-major indices v * M + m
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * PA_WARPS + warp, nw = (long long)gridDim.x * PA_WARPS;
  const unsigned lt = (1u << lane) - 1u;
  int qn = 0;
  for (long long c = gw; c * 32 < a.VM; c += nw) {
    const long long idx = c * 32 + lane;
    const bool vis = idx < a.VM && a.count[idx] > 0;
    const unsigned bal = __ballot_sync(0xffffffffu, vis);
    if (vis) q[warp][qn + __popc(bal & lt)] = idx;
    qn += __popc(bal);
    __syncwarp();
    if (qn >= 32) {
      const long long e = q[warp][lane];
      const int v = (int)(e / a.M);
      chain_slot(a, v, e - (long long)v * a.M);
      __syncwarp();
      if (lane < qn - 32) q[warp][lane] = q[warp][lane + 32];
      qn -= 32;
      __syncwarp();
    }
  }
  if (lane < qn) {
    const long long e = q[warp][lane];
    const int v = (int)(e / a.M);
    chain_slot(a, v, e - (long long)v * a.M);
  }
}

constexpr int PG_WARPS = 4;
constexpr int PG_T = 32 * PG_WARPS;
constexpr int PG_F = 4;    // faces per warp iteration
constexpr int PG_RS = 21;  // floats per entry row (out 9, colour 9, opacity, sigma; odd: no bank conflicts)
constexpr int PG_RMAX = (TS_MAX_VIEWS + 31) / 32;
constexpr int PBWD_ONE_PASS_VIEWS = 8;  // from here on the one-pass form is faster (room scene, 300k faces)

// Shared memory of one block: per-warp per-view pose sums, per-warp entry rows, per-warp view masks.
size_t pbwd_smem(int V) {
  return (size_t)PG_WARPS * V * 8 * sizeof(float) + (size_t)PG_WARPS * 32 * PG_RS * sizeof(float) +
         (size_t)PG_WARPS * PG_F * PG_RMAX * sizeof(uint32_t);
}

// Two-pass form, pass B.
__global__ void __launch_bounds__(PG_T) k_pbwd_gather(PBArgs a) {
  extern __shared__ float pv[];  // [PG_WARPS][V][8] per-warp per-view pose sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TsDevHeader* h = a.hdr;
  float* my = pv + (size_t)warp * a.V * 8;
  for (int i = lane; i < a.V * 8; i += 32) my[i] = 0.f;
  __syncwarp();
  // lanes 0..20 each own one output word: array c (gpx..gop), vertex k; with per-face sigma,
  // lane 21 owns the face's dL/dsigma_F (word 23 after the chain pass)
  const int c = lane / 3, k = lane - 3 * (lane / 3);
  const bool face_word = lane == 21;
  const bool owner = lane < 21 || (face_word && a.face_sigma);
  const int word = c < 3 ? G_DPOS + 3 * k + c : (c < 6 ? G_C + 3 * (c - 3) + k : (c == 6 ? G_O : 23));
  const float mean_scale = c == 6 ? (1.0f / 3.0f) : 1.0f;
  float* dst = owner ? (face_word ? a.dst_sigma : a.dst[c]) : nullptr;
  const bool indexed = h->faces != nullptr;
  const long long stride = (long long)gridDim.x * PG_WARPS * PG_F;
  for (long long m0 = ((long long)blockIdx.x * PG_WARPS + warp) * PG_F; m0 < a.M; m0 += stride) {
    long long j[PG_F];
    float old[PG_F], s[PG_F];
#pragma unroll
    for (int f = 0; f < PG_F; ++f) {
      const long long m = m0 + f;
      j[f] = (m < a.M && dst) ? (face_word ? m : face_vertex(h, m, k)) : 0;
      old[f] = (m < a.M && dst && (!indexed || face_word)) ? dst[j[f]] : 0.f;  // issued early
      s[f] = 0.f;
    }
    for (int r = 0; r * 32 < a.V; ++r) {
      const int vl = r * 32 + lane;
      unsigned msk[PG_F];
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        const long long m = m0 + f;
        const uint32_t cnt = (m < a.M && vl < a.V) ? a.count[(long long)vl * a.M + m] : 0u;
        msk[f] = __ballot_sync(0xffffffffu, cnt > 0);
      }
      // pose terms: the lane owning view vl adds each face's terms to the warp's sums (face order)
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        if ((msk[f] >> lane) & 1u) {
          const float* t = a.grad + ((m0 + f) * a.V + vl) * TS_GRAD_WORDS + G_TAU;
#pragma unroll
          for (int i = 0; i < 6; ++i) my[vl * 8 + i] += t[i];
        }
      }
      // output words: sum over the visible views in view order, up to 8 loads in flight
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        unsigned bits = msk[f];
        const float* base = a.grad + (m0 + f) * a.V * TS_GRAD_WORDS + word;
        while (bits) {
          float vals[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            vals[u] = 0.f;
            if (bits) {
              const int v = r * 32 + __ffs(bits) - 1;
              bits &= bits - 1;
              if (dst) vals[u] = base[(long long)v * TS_GRAD_WORDS];  // only for a requested output
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) s[f] += vals[u];
        }
      }
    }
#pragma unroll
    for (int f = 0; f < PG_F; ++f) {
      if (m0 + f < a.M && dst) {
        float scale = mean_scale;
        if (c == 6 && a.min_opacity) {  // the first vertex, in face order, attaining the minimum
          const long long m = m0 + f;
          const float o0 = __ldg(h->op + face_vertex(h, m, 0)), o1 = __ldg(h->op + face_vertex(h, m, 1));
          const float o2 = __ldg(h->op + face_vertex(h, m, 2));
          const int km = (o0 <= o1 && o0 <= o2) ? 0 : (o1 <= o2 ? 1 : 2);
          scale = k == km ? 1.0f : 0.0f;
        }
        if (indexed && !face_word) atomicAdd(dst + j[f], s[f] * scale);
        else dst[j[f]] = old[f] + s[f] * scale;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < a.V * 6; t += PG_T) {
    const int v = t / 6, i = t - 6 * (t / 6);
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < PG_WARPS; ++w) sum += pv[((size_t)w * a.V + v) * 8 + i];
    a.part[((long long)v * a.nblocks + blockIdx.x) * 6 + i] = sum;
  }
}

// One-pass form.
__global__ void __launch_bounds__(PG_T) k_pbwd_face(PBArgs a) {
  extern __shared__ float pv[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TsDevHeader* h = a.hdr;
  float* my = pv + (size_t)warp * a.V * 8;  // this warp's pose sums [V][8]
  float* rows = pv + (size_t)PG_WARPS * a.V * 8 + (size_t)warp * 32 * PG_RS;
  uint32_t* vm = reinterpret_cast<uint32_t*>(pv + (size_t)PG_WARPS * a.V * 8 + (size_t)PG_WARPS * 32 * PG_RS) +
                 warp * PG_F * PG_RMAX;  // [f][r]: the face's visible views r * 32 + bit
  for (int i = lane; i < a.V * 8; i += 32) my[i] = 0.f;
  __syncwarp();
  // lanes 0..20 each own one output word: array c (gpx..gop), vertex k; with per-face sigma,
  // lane 21 owns the face's dL/dsigma_F
  const int c = lane / 3, k = lane - 3 * (lane / 3);
  const bool face_word = lane == 21;
  const bool owner = lane < 21 || (face_word && a.face_sigma);
  const int ridx = c < 3 ? 3 * k + c : (c < 6 ? 9 + 3 * (c - 3) + k : (c == 6 ? 18 : 19));
  const float mean_scale = c == 6 ? (1.0f / 3.0f) : 1.0f;
  float* dst = owner ? (face_word ? a.dst_sigma : a.dst[c]) : nullptr;
  const bool indexed = h->faces != nullptr;
  const int R = (a.V + 31) >> 5;
  const long long stride = (long long)gridDim.x * PG_WARPS * PG_F;
  for (long long m0 = ((long long)blockIdx.x * PG_WARPS + warp) * PG_F; m0 < a.M; m0 += stride) {
    long long j[PG_F];
    float old[PG_F], s[PG_F];
    int nf[PG_F];
#pragma unroll
    for (int f = 0; f < PG_F; ++f) {
      const long long m = m0 + f;
      j[f] = (m < a.M && dst) ? (face_word ? m : face_vertex(h, m, k)) : 0;
      old[f] = (m < a.M && dst && (!indexed || face_word)) ? dst[j[f]] : 0.f;  // issued early
      s[f] = 0.f;
      nf[f] = 0;
    }
    // the faces' visible views, 32 at a time
    for (int r = 0; r < R; ++r) {
      const int vl = r * 32 + lane;
      uint32_t cnt[PG_F];
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        const long long m = m0 + f;
        cnt[f] = (m < a.M && vl < a.V) ? a.count[(long long)vl * a.M + m] : 0u;
      }
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        const unsigned msk = __ballot_sync(0xffffffffu, cnt[f] > 0);
        if (lane == 0) vm[f * PG_RMAX + r] = msk;
        nf[f] += __popc(msk);
      }
    }
    __syncwarp();
    int total = 0, st[PG_F];
#pragma unroll
    for (int f = 0; f < PG_F; ++f) {
      st[f] = total;
      total += nf[f];
    }
    // the (face, view) entries, face by face and views in order, one per lane
    for (int b0 = 0; b0 < total; b0 += 32) {
      const int ee = b0 + lane;
      const bool act = ee < total;
      int fe = 0, kk = ee;
      bool found = false;
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        if (!found) {
          if (kk < nf[f]) {
            fe = f;
            found = true;
          } else {
            kk -= nf[f];
          }
        }
      }
      int v = 0;
      SlotTerms t;
      if (act) {
        int r = 0;
        uint32_t mr = vm[fe * PG_RMAX];
        while (kk >= __popc(mr)) {  // the entry is in a later round of the face's views
          kk -= __popc(mr);
          mr = vm[fe * PG_RMAX + ++r];
        }
        int pb = 0;
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) {  // the kk-th set bit of mr
          const int cl = __popc(mr & ((1u << w) - 1u));
          if (kk >= cl) {
            kk -= cl;
            pb += w;
            mr >>= w;
          }
        }
        v = r * 32 + pb;
        chain_terms(a, v, m0 + fe, t);
        float* row = rows + lane * PG_RS;
#pragma unroll
        for (int i = 0; i < 9; ++i) row[i] = t.out[i];
#pragma unroll
        for (int i = 0; i < 9; ++i) row[9 + i] = t.gc[i];
        row[18] = t.go;
        row[19] = t.gsig;
      }
      // pose terms: face by face (a face's views are distinct), so each view's sum runs in face order
#pragma unroll
      for (int f = 0; f < PG_F; ++f) {
        if (act && fe == f) {
#pragma unroll
          for (int i = 0; i < 6; ++i) my[v * 8 + i] += t.tau[i];
        }
        __syncwarp();
      }
      // output words: each face's entries of this batch, views in order
      if (dst) {
#pragma unroll
        for (int f = 0; f < PG_F; ++f) {
          const int lo = max(st[f] - b0, 0), hi = min(st[f] + nf[f] - b0, 32);
          for (int e = lo; e < hi; ++e) s[f] += rows[e * PG_RS + ridx];
        }
      }
      __syncwarp();  // every lane has read the rows before the next batch writes them
    }
#pragma unroll
    for (int f = 0; f < PG_F; ++f) {
      if (m0 + f < a.M && dst) {
        float scale = mean_scale;
        if (c == 6 && a.min_opacity) {  // the first vertex, in face order, attaining the minimum
          const long long m = m0 + f;
          const float o0 = __ldg(h->op + face_vertex(h, m, 0)), o1 = __ldg(h->op + face_vertex(h, m, 1));
          const float o2 = __ldg(h->op + face_vertex(h, m, 2));
          const int km = (o0 <= o1 && o0 <= o2) ? 0 : (o1 <= o2 ? 1 : 2);
          scale = k == km ? 1.0f : 0.0f;
        }
        if (indexed && !face_word) atomicAdd(dst + j[f], s[f] * scale);
        else dst[j[f]] = old[f] + s[f] * scale;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < a.V * 6; t += PG_T) {
    const int v = t / 6, i = t - 6 * (t / 6);
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < PG_WARPS; ++w) sum += pv[((size_t)w * a.V + v) * 8 + i];
    a.part[((long long)v * a.nblocks + blockIdx.x) * 6 + i] = sum;
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

// The chain-rule pass's block count fixes the partial-sum layout of the pose gradient and so its summation
// order: a constant cap (not the device's SM count) keeps dtau's rounding the same on every GPU.
constexpr long long POSE_BLOCKS_MAX = 2432;
int ts_pose_blocks(long long M) {
  const long long want = (M + PG_WARPS * PG_F - 1) / (PG_WARPS * PG_F);
  return (int)std::max<long long>(1, std::min<long long>(want, POSE_BLOCKS_MAX));
}

cudaError_t ts_launch_project_bwd(const TsPlanImpl* p, const TsWs& w, const ts_map_grad* g, cudaStream_t s) {
  if (p->M == 0) {
    return cudaMemsetAsync(w.pose, 0, (size_t)p->V * p->n_pose_blocks * 6 * 4, s);
  }
  PBArgs a;
  a.views = w.views;
  a.poses = w.poses;
  a.V = p->V;
  a.M = p->M;
  a.VM = (long long)p->V * p->M;
  a.count = w.count;
  a.grad = w.grad;
  a.aux = w.aux;
  a.normals = p->normals;
  a.face_sigma = p->face_sigma;
  a.dst_sigma = p->face_sigma ? g->gsigma : nullptr;
  a.hdr = w.hdr;
  a.dst[0] = g->gpx; a.dst[1] = g->gpy; a.dst[2] = g->gpz;
  a.dst[3] = g->gcr; a.dst[4] = g->gcg; a.dst[5] = g->gcb;
  a.dst[6] = g->gop;
  a.min_opacity = p->min_opacity;
  a.part = w.pose;
  a.nblocks = (int)p->n_pose_blocks;
  if (p->V >= PBWD_ONE_PASS_VIEWS) {
    k_pbwd_face<<<(unsigned)p->n_pose_blocks, PG_T, pbwd_smem(p->V), s>>>(a);  // < 44 KiB for 256 views
  } else {
    const long long chunks = (a.VM + 31) / 32;
    const long long grid_a = std::min<long long>((chunks + PA_WARPS - 1) / PA_WARPS, (long long)ts_sm_count() * 8);
    k_pbwd_chain<<<(unsigned)grid_a, PA_T, 0, s>>>(a);
    k_pbwd_gather<<<(unsigned)p->n_pose_blocks, PG_T, (size_t)PG_WARPS * p->V * 8 * sizeof(float), s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t ts_launch_pose_reduce(const TsPlanImpl* p, const TsWs& w, float* dtau, cudaStream_t s) {
  k_pose_reduce<<<p->V, 256, 0, s>>>(w.pose, (int)p->n_pose_blocks, dtau);
  return cudaGetLastError();
}
