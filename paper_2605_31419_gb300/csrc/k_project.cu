// k_project.cu -- Eq. 1-3 per (view, face): projection, culling and the screen-space record.
//
// One thread per face and block of views: the thread loads its face's vertex data once (a warp
// reads 32 consecutive faces: coalesced structure-of-arrays loads) and projects it into each view
// of its block, writing the (view, face) outputs view-major, so that every store of a warp is to
// 32 consecutive (view, face) entries.  A block holds up to 4 views, so a map is read from memory
// once per 4 views instead of once per view.  The projection, area, perimeter, inradius, face
// opacity, pixel box and depth key follow one fixed FP32 operation order (no FMA contraction, IEEE
// division and square root), so culling, tiles and depth keys are reproducible bit for bit.
#include <algorithm>

#include "ts_internal.cuh"

namespace {

struct MapArgs {
  const float *px, *py, *pz, *cr, *cg, *cb, *op;
  const int32_t* faces;
  long long n_vertices;
};

__global__ void k_setup(TsViewTable tab, int V, MapArgs map, const ts_pose* __restrict__ poses, TsDevHeader* hdr,
                        TsView* views, ts_pose* ws_poses, unsigned long long* ctr) {
  const int t = threadIdx.x;
  for (int v = t; v < V; v += blockDim.x) {
    views[v] = tab.v[v];
    ws_poses[v] = poses[v];
  }
  for (int i = t; i < TS_N_CTR * TS_CTR_SLOTS; i += blockDim.x) ctr[(size_t)i * TS_CTR_STRIDE] = 0ull;
  if (t == 0) {
    hdr->n_pairs = 0;
    hdr->n_visible = 0;
    hdr->fwd_contrib = 0;
    hdr->bwd_contrib = 0;
    hdr->indexed = map.faces ? 1u : 0u;
    hdr->px = map.px; hdr->py = map.py; hdr->pz = map.pz;
    hdr->cr = map.cr; hdr->cg = map.cg; hdr->cb = map.cb;
    hdr->op = map.op;
    hdr->faces = map.faces;
    hdr->n_vertices = map.n_vertices;
  }
}

// One 32-byte store (eight floats) to a 32-byte aligned global address.
__device__ __forceinline__ void st_v8(float* p, float a0, float a1, float a2, float a3, float a4, float a5, float a6,
                                      float a7) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a0), "f"(a1), "f"(a2),
               "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
               : "memory");
}

struct ProjArgs {
  MapArgs map;
  const TsView* views;
  const ts_pose* poses;
  long long M;
  long long VM;
  int V;
  float z_near, r_min, alpha_min;
  bool min_opacity;
  int tile_w, tile_h;
  float4* frec;
  float4* aux;  // camera-space unit normal (TS_FLAG_NORMALS) and sigma_F in .w (TS_FLAG_FACE_SIGMA)
  bool normals;
  const float* sigma;  // per-face window exponents (TS_FLAG_FACE_SIGMA), else null
  uint32_t* cov;  // per (view, face) forward pixel coverage (TS_FLAG_STATS), else null
  float* grad;
  short4* rect;
  uint32_t* zbits;
  uint32_t* count;
  TsDevHeader* hdr;
  unsigned long long* ctr;
};

__global__ void __launch_bounds__(256, 3) k_project(ProjArgs a, int views_per_block) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v0 = (int)blockIdx.y * views_per_block;
  const int v1 = min(a.V, v0 + views_per_block);
  // the face's vertex data, loaded once for the block of views (all loads up front, so that their
  // latencies overlap)
  float o[3], wp[3][3], col[3][3];
  bool face_ok = m < a.M;
  if (face_ok) {
    long long vi[3];
    if (a.map.faces) {
      vi[0] = a.map.faces[3 * m]; vi[1] = a.map.faces[3 * m + 1]; vi[2] = a.map.faces[3 * m + 2];
    } else {
      vi[0] = 3 * m; vi[1] = 3 * m + 1; vi[2] = 3 * m + 2;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (vi[k] < 0 || vi[k] >= a.map.n_vertices) face_ok = false;
    if (face_ok) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const long long j = vi[k];
        wp[k][0] = __ldg(a.map.px + j);
        wp[k][1] = __ldg(a.map.py + j);
        wp[k][2] = __ldg(a.map.pz + j);
        o[k] = __ldg(a.map.op + j);
        col[k][0] = __ldg(a.map.cr + j);
        col[k][1] = __ldg(a.map.cg + j);
        col[k][2] = __ldg(a.map.cb + j);
      }
    }
  }
  const float sig_m = (face_ok && a.sigma) ? __ldg(a.sigma + m) : 0.f;
  for (int view = v0; view < v1; ++view) {
    const long long idx = (long long)view * a.M + m;
    bool vis = face_ok;
    if (m < a.M) {
      const TsView vw = a.views[view];
      const ts_pose P = a.poses[view];
      float u[3], v[3], z[3], xv[3], yv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (!vis) break;
        float xc, yc, zc;
        ts_rigid_f32(P, wp[k][0], wp[k][1], wp[k][2], xc, yc, zc);
        if (!(zc > a.z_near)) { vis = false; break; }
        ts_pinhole_f32(vw, xc, yc, zc, u[k], v[k]);
        z[k] = zc;
        xv[k] = xc;
        yv[k] = yc;
      }
      float area2 = 0.f, len[3] = {0.f, 0.f, 0.f}, per = 0.f, oF = 0.f;
      if (vis) {
        const float du1 = __fsub_rn(u[1], u[0]), dv1 = __fsub_rn(v[1], v[0]);
        const float du2 = __fsub_rn(u[2], u[0]), dv2 = __fsub_rn(v[2], v[0]);
        area2 = __fsub_rn(__fmul_rn(du1, dv2), __fmul_rn(du2, dv1));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int j = (i + 1) % 3;
          const float ex = __fsub_rn(u[j], u[i]), ey = __fsub_rn(v[j], v[i]);
          len[i] = __fsqrt_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)));
        }
        per = __fadd_rn(__fadd_rn(len[0], len[1]), len[2]);
        const float r = __fdiv_rn(fabsf(area2), per);
        if (!(r >= a.r_min)) vis = false;
        oF = a.min_opacity ? fminf(o[0], fminf(o[1], o[2])) : __fdiv_rn(__fadd_rn(__fadd_rn(o[0], o[1]), o[2]), 3.0f);
        if (oF < a.alpha_min) vis = false;
      }
      int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
      if (vis) {
        const float umin = fminf(u[0], fminf(u[1], u[2])), umax = fmaxf(u[0], fmaxf(u[1], u[2]));
        const float vmin = fminf(v[0], fminf(v[1], v[2])), vmax = fmaxf(v[0], fmaxf(v[1], v[2]));
        const float fx0 = ceilf(__fsub_rn(umin, 0.5f)), fx1 = floorf(__fsub_rn(umax, 0.5f));
        const float fy0 = ceilf(__fsub_rn(vmin, 0.5f)), fy1 = floorf(__fsub_rn(vmax, 0.5f));
        const float Wm = (float)(vw.W - 1), Hm = (float)(vw.H - 1);
        if (!(fx0 <= fx1) || fx1 < 0.0f || fx0 > Wm) vis = false;
        if (!(fy0 <= fy1) || fy1 < 0.0f || fy0 > Hm) vis = false;
        if (vis) {
          x0 = fx0 < 0.0f ? 0 : (int)fx0;
          x1 = fx1 > Wm ? vw.W - 1 : (int)fx1;
          y0 = fy0 < 0.0f ? 0 : (int)fy0;
          y1 = fy1 > Hm ? vw.H - 1 : (int)fy1;
        }
      }
      if (vis) {
        const float zk = __fdiv_rn(__fadd_rn(__fadd_rn(z[0], z[1]), z[2]), 3.0f);
        a.zbits[idx] = __float_as_uint(zk);
        // record: edge vectors, normalised edge-function scales s_i / D2, barycentric scale 1 / D2
        const float e0x = u[1] - u[0], e0y = v[1] - v[0];
        const float e1x = u[2] - u[1], e1y = v[2] - v[1];
        const float e2x = u[0] - u[2], e2y = v[0] - v[2];
        const float invD = 1.0f / area2;
        const float k0 = (per / len[0]) * invD, k1 = (per / len[1]) * invD, k2 = (per / len[2]) * invD;
        float* rec = reinterpret_cast<float*>(a.frec + idx * (TS_REC_WORDS / 4));
        st_v8(rec, u[0], u[1], u[2], v[0], v[1], v[2], e0x, e0y);
        st_v8(rec + 8, e1x, e1y, e2x, e2y, k0, k1, k2, invD);
        st_v8(rec + 16, oF, col[0][0], col[0][1], col[0][2], col[1][0], col[1][1], col[1][2], col[2][0]);
        // gradient slot of this (view, face), face-major so that a face's views are adjacent;
        // cleared here for the raster backward's atomics
        const long long slot = m * a.V + view;
        st_v8(rec + 24, col[2][1], col[2][2], z[0], z[1], z[2], __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)),
              __uint_as_float((uint32_t)y0 | ((uint32_t)y1 << 16)), __uint_as_float((uint32_t)slot));
        if (a.grad) {  // null for a forward-only plan
          // the raster backward adds into words 0..22, and with the side array (normals, sigma_F)
          // also into 23, 24, 30, 31; words 25..29 are not used
          float* gs = a.grad + slot * TS_GRAD_WORDS;
          const int nz = a.aux ? TS_GRAD_WORDS / 8 : 3;
          for (int i = 0; i < nz; ++i) st_v8(gs + 8 * i, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        }
        const int tx0 = x0 / a.tile_w, tx1 = x1 / a.tile_w, ty0 = y0 / a.tile_h, ty1 = y1 / a.tile_h;
        a.rect[idx] = make_short4((short)tx0, (short)ty0, (short)tx1, (short)ty1);
        a.count[idx] = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        if (a.cov) a.cov[idx] = 0u;
        float4 ax = make_float4(0.f, 0.f, 0.f, sig_m);
        if (a.normals) {
          // unit normal (v1 - v0) x (v2 - v0), turned towards the camera.  The edge vectors are
          // taken in world space, where nearby float32 positions subtract almost exactly, and the
          // unit normal is then rotated by R: camera-space edges would be differences of
          // metre-sized coordinates and lose ~1e-5 of the normal for centimetre faces.
          float e1[3], e2[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            e1[c] = wp[1][c] - wp[0][c];
            e2[c] = wp[2][c] - wp[0][c];
          }
          const float wx = e1[1] * e2[2] - e1[2] * e2[1], wy = e1[2] * e2[0] - e1[0] * e2[2];
          const float wz = e1[0] * e2[1] - e1[1] * e2[0];
          const float inv = rsqrtf(wx * wx + wy * wy + wz * wz);
          float nc[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) nc[r] = (P.R[3 * r] * wx + P.R[3 * r + 1] * wy + P.R[3 * r + 2] * wz) * inv;
          const float facing =
              nc[0] * (xv[0] + xv[1] + xv[2]) + nc[1] * (yv[0] + yv[1] + yv[2]) + nc[2] * (z[0] + z[1] + z[2]);
          const float sg = facing > 0.f ? -1.f : 1.f;
          ax.x = sg * nc[0];
          ax.y = sg * nc[1];
          ax.z = sg * nc[2];
        }
        if (a.aux) a.aux[idx] = ax;
      } else {
        a.rect[idx] = make_short4(-1, -1, -1, -1);
        a.count[idx] = 0u;
      }
    }
    ts_count_add(a.ctr, TS_CTR_VISIBLE, vis ? 1u : 0u);
  }
}

}  // namespace

cudaError_t ts_launch_setup(const TsPlanImpl* p, const TsWs& w, const ts_map* map, const ts_pose* poses,
                            cudaStream_t s) {
  TsViewTable local;  // passed by value: capture-safe, no host-to-device copy
  for (int v = 0; v < p->V; ++v) local.v[v] = p->views[v];
  MapArgs m{map->px, map->py, map->pz, map->cr, map->cg, map->cb, map->op, map->faces, map->n_vertices};
  k_setup<<<1, 256, 0, s>>>(local, p->V, m, poses, w.hdr, w.views, w.poses, w.ctr);
  return cudaGetLastError();
}

cudaError_t ts_launch_project(const TsPlanImpl* p, const TsWs& w, const ts_map* map, cudaStream_t s) {
  const long long VM = (long long)p->V * p->M;
  if (VM == 0) return cudaSuccess;
  ProjArgs a;
  a.map = MapArgs{map->px, map->py, map->pz, map->cr, map->cg, map->cb, map->op, map->faces, map->n_vertices};
  a.views = w.views;
  a.poses = w.poses;
  a.M = p->M;
  a.VM = VM;
  a.z_near = p->prm.z_near;
  a.r_min = p->prm.r_min;
  a.alpha_min = p->prm.alpha_min;
  a.min_opacity = p->min_opacity;
  a.tile_w = p->prm.tile_w;
  a.tile_h = p->prm.tile_h;
  a.V = p->V;
  a.grad = w.grad;
  a.frec = w.frec;
  a.aux = w.aux;
  a.normals = p->normals;
  a.sigma = p->face_sigma ? map->sigma : nullptr;
  a.cov = w.cov;
  a.rect = w.rect;
  a.zbits = w.zbits;
  a.count = w.count;
  a.hdr = w.hdr;
  a.ctr = w.ctr;
  // up to 4 views per thread: measured on the 300k-face, 20-view room and the 1M-face, 12-view
  // mapping window against 1, 2 and all views per thread, it is within 0.01 ms of the best of both
  const long long face_blocks = (p->M + 255) / 256;
  const int per = std::min(p->V, 4);
  k_project<<<dim3((unsigned)face_blocks, (unsigned)((p->V + per - 1) / per)), 256, 0, s>>>(a, per);
  return cudaGetLastError();
}

// The counters' slots summed into the header (read by ts_sync_status).
__global__ void __launch_bounds__(256) k_sum_counters(const unsigned long long* __restrict__ ctr, TsDevHeader* hdr) {
  __shared__ unsigned long long red[TS_N_CTR][256];
  for (int c = 0; c < TS_N_CTR; ++c) {
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < TS_CTR_SLOTS; i += 256) s += ctr[((size_t)c * TS_CTR_SLOTS + i) * TS_CTR_STRIDE];
    red[c][threadIdx.x] = s;
  }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < TS_N_CTR; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    hdr->n_visible = red[TS_CTR_VISIBLE][0];
    hdr->fwd_contrib = red[TS_CTR_FWD][0];
    hdr->bwd_contrib = red[TS_CTR_BWD][0];
  }
}

cudaError_t ts_launch_sum_counters(const TsWs& w, cudaStream_t s) {
  k_sum_counters<<<1, 256, 0, s>>>(w.ctr, w.hdr);
  return cudaGetLastError();
}
