// k_render.cu -- Eq. 3-4 forward blend and its adjoint, one CTA per (view, tile) at a time.
//
// Staging: the tile's depth-sorted face ids select 128-byte records that one warp copies into
// shared memory with TMA bulk copies (cp.async.bulk, one per record) completing on an mbarrier;
// two buffers alternate so the next stage streams in while the current one is blended.  Each
// warp owns an 8 x 4 pixel sub-block of the tile; per stage, a mask per record says which
// sub-blocks can contain one of the face's covered pixel centres, and each warp walks only the
// set bits of its own ballot over the stage.
//
// Forward: per pixel, front to back: window (Eq. 3) from cancellation-free edge functions,
// alpha = min(alpha_max, o_F I), skip below alpha_min, stop before the face that would take T
// below T_min, accumulate colour, depth and opacity (Eq. 4).  Writes C + T bg, D, A = 1 - T, and
// per pixel T_final and the list position after the last contribution, and per sorted pair the
// mask of warps that blended the face at one of their pixels.
//
// Backward: per pixel, back to front from that position: recover T_n = T_{n+1} / (1 - alpha_n),
// keep the suffix sum S of later contributions (including the background term), form
// dL/dalpha_n = T_n v_n - S / (1 - alpha_n) with v_n = gC . c_n + gD z_n + gA, and chain into 22
// per-face sums (barycentric-weighted gradients of the edge, colour and depth interpolants, and
// of o_F).  A warp reduces the 24-word vector with a 27-shuffle reduce-scatter, leaving one sum
// per lane, and issues a single 24-lane atomic add into the face's accumulator.  A warp visits
// only the faces whose forward mask holds its bit.
//
// Launch forms: one CTA per tile, or persistent CTAs (as many as fit on the GPU) that take tiles
// from a device counter, keeping their mbarriers across tiles.
#include <algorithm>

#include "ts_internal.cuh"

namespace {

struct RenderArgs {
  const TsView* views;
  int V;
  long long M, VM;
  long long n_tiles;
  const float4* frec;
  const uint32_t* ids;
  const uint2* ranges;
  float* color;
  float* depth;
  float* alpha;
  float* tfin;
  int32_t* nlast;
  const float* dC;
  const float* dD;
  const float* dA;
  float* grad;
  float sigma, alpha_min, alpha_max, T_min;
  float bg0, bg1, bg2;
  int S;
  unsigned int* counter;
  uint16_t* cmask;
  const float4* aux;   // per (view, face): camera-space normal and, in .w, sigma_F; else null
  bool normals;        // TS_FLAG_NORMALS: composite the normal map
  bool face_sigma;     // TS_FLAG_FACE_SIGMA: each face's own window exponent
  float* normal;       // normal map output (may be null)
  const float* dN;     // gradient w.r.t. the normal map (may be null)
  uint32_t* cov;       // per (view, face) pixels blended by the forward (TS_FLAG_STATS), else null
  TsDevHeader* hdr;
};

constexpr unsigned FULL = 0xffffffffu;

// Register budget of the raster kernels per thread (0: the compiler's choice), expressed as the
// minimum number of resident CTAs in the launch bounds.  Both kernels are latency-bound: on the
// room workload (tile 16x8) 56 registers beat the compiler's unconstrained 87-104 by 20 % and
// 64 or 72 registers by 1-4 %, small spills included.
#ifndef TS_RASTER_REGS
#define TS_RASTER_REGS 56
#endif
constexpr int raster_min_blocks(int threads) {
  return TS_RASTER_REGS > 0 ? (65536 / (threads * TS_RASTER_REGS) > 0 ? 65536 / (threads * TS_RASTER_REGS) : 1) : 1;
}

// Shared state of a render CTA.
struct RenderSmem {
  uint64_t bar[2];
  uint32_t smask[2][128];
  uint32_t cm[2][128];  // forward: warps of the tile that blended each staged face
  uint32_t cv[2][128];  // forward, TS_FLAG_STATS: pixels of the tile that blended each staged face
  int view;
  int nmax;
  int next_tile;
  int fail;
};

template <int TW, int TH>
struct TileGeom {
  static constexpr int NSBX = TW / 8;
  int view, X0, Y0, x, y;
  bool inimg;
  float px, py;
  TsView vw;
};

template <int TW, int TH>
__device__ __forceinline__ TileGeom<TW, TH> tile_geom(const RenderArgs& a, long long tile, RenderSmem& sm) {
  TileGeom<TW, TH> g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {  // the view owning the tile: one coalesced load and a ballot per 32 views
    int below = 0;
    for (int base = 0; base < a.V; base += 32) {
      const int v = base + lane;
      const unsigned b = __ballot_sync(FULL, v < a.V && a.views[v].tile_off <= tile);
      below += __popc(b);
      if (b != FULL) break;
    }
    if (lane == 0) sm.view = below - 1;
  }
  __syncthreads();
  g.view = sm.view;
  g.vw = a.views[g.view];
  const long long lt = tile - g.vw.tile_off;
  const int ty = (int)(lt / g.vw.TX), tx = (int)(lt - (long long)ty * g.vw.TX);
  g.X0 = tx * TW;
  g.Y0 = ty * TH;
  g.x = g.X0 + (warp % TileGeom<TW, TH>::NSBX) * 8 + (lane & 7);
  g.y = g.Y0 + (warp / TileGeom<TW, TH>::NSBX) * 4 + (lane >> 3);
  g.inimg = g.x < g.vw.W && g.y < g.vw.H;
  g.px = (float)g.x + 0.5f;
  g.py = (float)g.y + 0.5f;
  return g;
}

// Warp 0 issues the bulk copies of stage `st` (records [st*S, st*S + cnt) of the tile's list)
// into buffer `b`; with AUX also each record's 16-byte side entry (normal, sigma_F), after both
// record buffers.
template <bool AUX>
__device__ __forceinline__ void issue_stage(const RenderArgs& a, float4* smrec, uint64_t* bar, int b, int st,
                                            uint32_t start, int n, const float4* vbase, const float4* nbase) {
  const int lane = threadIdx.x & 31;
  const int S = a.S;
  const int cnt = min(S, n - st * S);
  if (lane == 0) ts_mbar_arrive_expect_tx(&bar[b], (uint32_t)cnt * (AUX ? 144u : 128u));
  __syncwarp();
  for (int j = lane; j < cnt; j += 32) {
    uint32_t id = __ldg(a.ids + start + (uint32_t)(st * S + j));
    if ((long long)id >= a.M) {  // never expected: record the fault and stage an in-bounds record
      atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
      id = 0;
    }
    ts_bulk_g2s(smrec + ((size_t)b * S + j) * 8, vbase + (size_t)id * 8, 128u, &bar[b]);
    if (AUX) ts_bulk_g2s(smrec + (size_t)2 * S * 8 + (size_t)b * S + j, nbase + id, 16u, &bar[b]);
  }
}

// For each staged record, the mask of warp sub-blocks (8 x 4 pixels) that can contain one of its
// covered pixel centres: sub-blocks inside the face's pixel box whose pixel-centre rectangle,
// widened by 0.01 px, is not entirely outside one of the three edges.  Conservative: a pixel with
// a positive window always keeps its sub-block's bit.
template <int TW, int TH>
__device__ __forceinline__ void stage_masks(const float* rb, uint32_t* smask, int cnt, int X0, int Y0) {
  constexpr int NSBX = TW / 8;
  for (int j = threadIdx.x; j < cnt; j += TW * TH) {
    const float* r = rb + j * TS_REC_WORDS;
    const uint32_t bx = __float_as_uint(r[R_BOXX]), by = __float_as_uint(r[R_BOXY]);
    const int x0 = (int)(bx & 0xffffu) - X0, x1 = (int)(bx >> 16) - X0;
    const int y0 = (int)(by & 0xffffu) - Y0, y1 = (int)(by >> 16) - Y0;
    uint32_t mask = 0;
    if (x1 >= 0 && x0 < TW && y1 >= 0 && y0 < TH) {
      const int c0 = max(x0, 0) >> 3, c1 = min(x1, TW - 1) >> 3;
      const int r0 = max(y0, 0) >> 2, r1 = min(y1, TH - 1) >> 2;
      const float sgn = r[R_INVD] > 0.f ? 1.f : -1.f;
      const float qx[3] = {r[R_U0], r[R_U1], r[R_U2]}, qy[3] = {r[R_V0], r[R_V1], r[R_V2]};
      const float ex[3] = {r[R_E0X], r[R_E1X], r[R_E2X]}, ey[3] = {r[R_E0Y], r[R_E1Y], r[R_E2Y]};
      for (int rr = r0; rr <= r1; ++rr) {
        const float cy = (float)(Y0 + rr * 4) + 2.0f;  // centre of the sub-block's pixel centres
        for (int cc = c0; cc <= c1; ++cc) {
          const float cx = (float)(X0 + cc * 8) + 4.0f;
          bool in = true;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float f = sgn * (ex[i] * (cy - qy[i]) - ey[i] * (cx - qx[i])) + fabsf(ey[i]) * 3.51f +
                            fabsf(ex[i]) * 1.51f;
            in = in && f > 0.f;
          }
          if (in) mask |= 1u << (rr * NSBX + cc);
        }
      }
    }
    smask[j] = mask;
  }
}

__device__ __forceinline__ void count_add(unsigned long long* ctr, unsigned v) {
  const unsigned s = __reduce_add_sync(FULL, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// Wait for stage sequence number `seq` (buffer seq & 1, phase (seq >> 1) & 1) in every thread.
// Returns false on timeout (after latching the error and letting the late copies land).
__device__ __forceinline__ bool wait_stage(const RenderArgs& a, RenderSmem& sm, int seq) {
  const bool ok = ts_mbar_wait(&sm.bar[seq & 1], (uint32_t)(seq >> 1) & 1u);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(&a.hdr->error_bits, TS_ERRBIT_TIMEOUT);
      ts_mbar_wait(&sm.bar[seq & 1], (uint32_t)(seq >> 1) & 1u);
    }
    return false;
  }
  return true;
}

// Forward of one tile; seq counts the stages this CTA has waited for so far (mbarrier phases).
template <int TW, int TH, bool AUX>
__device__ __forceinline__ bool fwd_tile(const RenderArgs& a, long long tile, float4* smrec, RenderSmem& sm,
                                         int& seq) {
  const TileGeom<TW, TH> g = tile_geom<TW, TH>(a, tile, sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 rg = a.ranges[tile];
  const int n = (int)(rg.y - rg.x);
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  float N0 = 0.f, N1 = 0.f, N2 = 0.f;
  int nl = 0;
  bool done = !g.inimg;
  unsigned contrib = 0;
  bool ok = true;
  if (n > 0) {
    const int S = a.S;
    const int nst = (n + S - 1) / S;
    const float4* vbase = a.frec + (size_t)g.view * (size_t)a.M * 8;
    const float4* nbase = AUX ? a.aux + (size_t)g.view * (size_t)a.M : nullptr;
    if (warp == 0) issue_stage<AUX>(a, smrec, sm.bar, seq & 1, 0, rg.x, n, vbase, nbase);
    for (int st = 0; st < nst; ++st) {
      const int b = seq & 1;
      const int cnt = min(S, n - st * S);
      if (!wait_stage(a, sm, seq)) { ok = false; break; }
      ++seq;
      const float* rb = reinterpret_cast<const float*>(smrec + (size_t)b * S * 8);
      const float4* nb = smrec + (size_t)2 * S * 8 + (size_t)b * S;
      stage_masks<TW, TH>(rb, sm.smask[b], cnt, g.X0, g.Y0);
      for (int j = threadIdx.x; j < cnt; j += TW * TH) {
        sm.cm[b][j] = 0u;
        sm.cv[b][j] = 0u;
      }
      __syncthreads();
      if (warp == 0 && st + 1 < nst) issue_stage<AUX>(a, smrec, sm.bar, b ^ 1, st + 1, rg.x, n, vbase, nbase);
      for (int q = 0; q * 32 < cnt; ++q) {
        const int jq = q * 32 + lane;
        unsigned bits = __ballot_sync(FULL, jq < cnt && ((sm.smask[b][min(jq, cnt - 1)] >> warp) & 1u));
        while (bits) {
          const int j = q * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          bool blended = false;
          if (!done) {
            const float* r = rb + j * TS_REC_WORDS;
            const TsPix e = ts_eval_edges(r, g.px, g.py);
            if (e.m > 0.f) {
              const float sig = (AUX && a.face_sigma) ? nb[j].w : a.sigma;
              const float I = ts_window(e.m, sig);
              const float al = fminf(r[R_OF] * I, a.alpha_max);
              if (al >= a.alpha_min) {
                const float Tn = T * (1.f - al);
                if (Tn < a.T_min) {
                  done = true;
                } else {
                  const float invD = r[R_INVD];
                  const float l0 = e.cr1 * invD, l1 = e.cr2 * invD, l2 = e.cr0 * invD;
                  const float w = al * T;
                  C0 += w * (l0 * r[R_C0] + l1 * r[R_C1] + l2 * r[R_C2]);
                  C1 += w * (l0 * r[R_C0 + 1] + l1 * r[R_C1 + 1] + l2 * r[R_C2 + 1]);
                  C2 += w * (l0 * r[R_C0 + 2] + l1 * r[R_C1 + 2] + l2 * r[R_C2 + 2]);
                  D += w * (l0 * r[R_Z0] + l1 * r[R_Z1] + l2 * r[R_Z2]);
                  if (AUX && a.normals) {
                    const float4 nn = nb[j];
                    N0 += w * nn.x;
                    N1 += w * nn.y;
                    N2 += w * nn.z;
                  }
                  T = Tn;
                  nl = st * S + j + 1;
                  ++contrib;
                  blended = true;
                }
              }
            }
          }
          // the backward revisits exactly the (warp, face) pairs that blended somewhere
          const unsigned bl = __ballot_sync(FULL, blended);
          if (bl && lane == 0) {
            atomicOr(&sm.cm[b][j], 1u << warp);
            if (a.cov) atomicAdd(&sm.cv[b][j], (unsigned)__popc(bl));
          }
        }
      }
      const int alive = __syncthreads_count(!done);
      for (int j = threadIdx.x; j < cnt; j += TW * TH) {
        a.cmask[rg.x + st * S + j] = (uint16_t)sm.cm[b][j];
        if (a.cov && sm.cv[b][j]) {  // face m of the record's slot m * V + view
          const uint32_t slot = __float_as_uint(rb[j * TS_REC_WORDS + R_SLOT]);
          const long long m = (long long)(slot / (uint32_t)a.V);
          if (m < a.M) atomicAdd(a.cov + (long long)g.view * a.M + m, sm.cv[b][j]);
        }
      }
      if (alive == 0) {
        if (st + 1 < nst) {  // a prefetched stage is in flight: consume its phase before leaving
          if (!wait_stage(a, sm, seq)) { ok = false; break; }
          ++seq;
        }
        break;
      }
    }
  }
  count_add(&a.hdr->fwd_contrib, contrib);
  if (ok && g.inimg) {
    const long long HW = (long long)g.vw.W * g.vw.H;
    const long long pi = (long long)g.y * g.vw.W + g.x;
    const long long o = g.vw.pix_off + pi;
    if (a.color) {
      float* c = a.color + 3 * g.vw.pix_off + pi;
      c[0] = C0 + T * a.bg0;
      c[HW] = C1 + T * a.bg1;
      c[2 * HW] = C2 + T * a.bg2;
    }
    if (a.depth) a.depth[o] = D;
    if (a.alpha) a.alpha[o] = 1.f - T;
    if (AUX && a.normal) {
      float* q = a.normal + 3 * g.vw.pix_off + pi;
      q[0] = N0;
      q[HW] = N1;
      q[2 * HW] = N2;
    }
    a.tfin[o] = T;
    a.nlast[o] = nl;
  }
  return ok;
}

template <int TW, int TH, bool AUX>
__device__ __forceinline__ bool bwd_tile(const RenderArgs& a, long long tile, float4* smrec, RenderSmem& sm,
                                         int& seq) {
  const TileGeom<TW, TH> g = tile_geom<TW, TH>(a, tile, sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 rg = a.ranges[tile];
  float T = 0.f, Sacc = 0.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f;
  float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
  int nl = 0;
  if (g.inimg) {
    const long long HW = (long long)g.vw.W * g.vw.H;
    const long long pi = (long long)g.y * g.vw.W + g.x;
    const long long o = g.vw.pix_off + pi;
    T = a.tfin[o];
    nl = a.nlast[o];
    const float* dc = a.dC + 3 * g.vw.pix_off + pi;
    gC0 = dc[0];
    gC1 = dc[HW];
    gC2 = dc[2 * HW];
    gD = a.dD ? a.dD[o] : 0.f;
    gA = a.dA ? a.dA[o] : 0.f;
    if (AUX && a.dN) {
      const float* dn = a.dN + 3 * g.vw.pix_off + pi;
      gN0 = dn[0];
      gN1 = dn[HW];
      gN2 = dn[2 * HW];
    }
    Sacc = T * (gC0 * a.bg0 + gC1 * a.bg1 + gC2 * a.bg2);
  }
  if (threadIdx.x == 0) sm.nmax = 0;
  __syncthreads();
  {
    const int m = __reduce_max_sync(FULL, (unsigned)nl);
    if (lane == 0 && m) atomicMax(&sm.nmax, m);
  }
  __syncthreads();
  // positions come from the forward pass over the same lists; clamp in case the caller did not
  // run it after the last ts_bin
  const int n = min(sm.nmax, (int)(rg.y - rg.x));
  unsigned contrib = 0;
  bool ok = true;
  if (n > 0) {
    const int S = a.S;
    const int nst = (n + S - 1) / S;
    const float4* vbase = a.frec + (size_t)g.view * (size_t)a.M * 8;
    const float4* nbase = AUX ? a.aux + (size_t)g.view * (size_t)a.M : nullptr;
    if (warp == 0) issue_stage<AUX>(a, smrec, sm.bar, seq & 1, nst - 1, rg.x, n, vbase, nbase);
    const bool hi16 = lane & 16, hi8 = lane & 8, hi4 = lane & 4;
    const int q = lane & 3;
    const int widx = (hi16 ? 12 : 0) + (hi8 ? 6 : 0) + (hi4 ? 3 : 0) + q;
    for (int k = 0; k < nst; ++k) {
      const int st = nst - 1 - k;
      const int b = seq & 1;
      const int cnt = min(S, n - st * S);
      if (!wait_stage(a, sm, seq)) { ok = false; break; }
      ++seq;
      const float* rb = reinterpret_cast<const float*>(smrec + (size_t)b * S * 8);
      const float4* nb = smrec + (size_t)2 * S * 8 + (size_t)b * S;
      // the forward's record of which warps blended each face (positions below the tile's
      // largest list position after a contribution were all written by the forward)
      for (int j = threadIdx.x; j < cnt; j += TW * TH) sm.smask[b][j] = a.cmask[rg.x + st * S + j];
      __syncthreads();
      if (warp == 0 && k + 1 < nst) issue_stage<AUX>(a, smrec, sm.bar, b ^ 1, st - 1, rg.x, n, vbase, nbase);
      // this warp visits only the stage's faces it blended in the forward (back to front)
      for (int qq = (cnt - 1) >> 5; qq >= 0; --qq) {
        const int jq = qq * 32 + lane;
        unsigned bits = __ballot_sync(FULL, jq < cnt && ((sm.smask[b][min(jq, cnt - 1)] >> warp) & 1u));
        while (bits) {
          const int hb = 31 - __clz(bits);
          bits &= ~(1u << hb);
          const int j = qq * 32 + hb;
          const float* r = rb + j * TS_REC_WORDS;
          const int pos = st * S + j;
          bool cb = false;
          TsPix e;
          float I = 0.f, al = 0.f;
          const float sig = (AUX && a.face_sigma) ? nb[j].w : a.sigma;
          if (pos < nl) {
            e = ts_eval_edges(r, g.px, g.py);
            if (e.m > 0.f) {
              I = ts_window(e.m, sig);
              al = fminf(r[R_OF] * I, a.alpha_max);
              cb = al >= a.alpha_min;
            }
          }
          if (!__any_sync(FULL, cb)) continue;
          // per-face sums: words 0..22, and with the side array dL/dn_F in words 23, 30, 31 and
          // dL/dsigma_F in word 24 (the chain pass moves it to 23 before it writes the pose terms)
          constexpr int NVAL = AUX ? 32 : 24;
          float v[NVAL];
#pragma unroll
          for (int i = 0; i < NVAL; ++i) v[i] = 0.f;
          if (cb) {
            const float oma = 1.f - al;  // >= 1 - alpha_max
            const float ro = ts_rcp_approx(oma);
            const float Tn = T * ro;
            const float invD = r[R_INVD];
            const float l0 = e.cr1 * invD, l1 = e.cr2 * invD, l2 = e.cr0 * invD;
            const float c0 = l0 * r[R_C0] + l1 * r[R_C1] + l2 * r[R_C2];
            const float c1 = l0 * r[R_C0 + 1] + l1 * r[R_C1 + 1] + l2 * r[R_C2 + 1];
            const float c2 = l0 * r[R_C0 + 2] + l1 * r[R_C1 + 2] + l2 * r[R_C2 + 2];
            const float z = l0 * r[R_Z0] + l1 * r[R_Z1] + l2 * r[R_Z2];
            float val = gC0 * c0 + gC1 * c1 + gC2 * c2 + gD * z + gA;
            float4 nn = make_float4(0.f, 0.f, 0.f, 0.f);
            if (AUX && a.normals) {
              nn = nb[j];
              val += gN0 * nn.x + gN1 * nn.y + gN2 * nn.z;
            }
            const float dal = val * Tn - Sacc * ro;
            Sacc += val * al * Tn;
            T = Tn;
            const float w = al * Tn;
            const float w0 = gC0 * w, w1 = gC1 * w, w2 = gC2 * w, wz = gD * w;
            v[G_C + 0] = w0 * l0; v[G_C + 1] = w0 * l1; v[G_C + 2] = w0 * l2;
            v[G_C + 3] = w1 * l0; v[G_C + 4] = w1 * l1; v[G_C + 5] = w1 * l2;
            v[G_C + 6] = w2 * l0; v[G_C + 7] = w2 * l1; v[G_C + 8] = w2 * l2;
            v[G_Z + 0] = wz * l0; v[G_Z + 1] = wz * l1; v[G_Z + 2] = wz * l2;
            v[G_CNT] = 1.f;
            if constexpr (AUX) {
              v[23] = gN0 * w;
              v[30] = gN1 * w;
              v[31] = gN2 * w;
            }
            const float oF = r[R_OF];
            if (!(oF * I > a.alpha_max)) {
              v[G_O] = dal * I;
              const float dI = dal * oF;
              // I >= alpha_min / o_F here, far from zero
              const float dm = (sig == 0.5f) ? dI * 0.5f * ts_rcp_approx(I) : dI * sig * I / e.m;
              if constexpr (AUX) {  // dL/dsigma_F = dL/dalpha o_F I ln(ratio)
                if (a.face_sigma) v[24] = dI * I * logf(e.m);
              }
              const float d0 = dm * l0, d1 = dm * l1, d2 = dm * l2;
              v[G_E + 0] = e.arg == 0 ? d0 : 0.f; v[G_E + 1] = e.arg == 0 ? d1 : 0.f; v[G_E + 2] = e.arg == 0 ? d2 : 0.f;
              v[G_E + 3] = e.arg == 1 ? d0 : 0.f; v[G_E + 4] = e.arg == 1 ? d1 : 0.f; v[G_E + 5] = e.arg == 1 ? d2 : 0.f;
              v[G_E + 6] = e.arg == 2 ? d0 : 0.f; v[G_E + 7] = e.arg == 2 ? d1 : 0.f; v[G_E + 8] = e.arg == 2 ? d2 : 0.f;
            }
            ++contrib;
          }
          if constexpr (AUX) {
            // reduce-scatter 32 -> 16 -> 8 -> 4 -> 2 -> 1: lane L ends with the sum of value L
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
              const bool hi = lane & o;
#pragma unroll
              for (int i = 0; i < o; ++i) {
                const float send = hi ? v[i] : v[i + o];
                const float keep = hi ? v[i + o] : v[i];
                v[i] = keep + __shfl_xor_sync(FULL, send, o);
              }
            }
            if (v[0] != 0.f) {
              const uint32_t slot = __float_as_uint(r[R_SLOT]);
              if ((long long)slot < a.VM) {
                atomicAdd(a.grad + (size_t)slot * TS_GRAD_WORDS + lane, v[0]);
              } else {
                atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
              }
            }
            continue;
          }
          // reduce-scatter: 24 -> 12 -> 6 -> 3 values per lane, then a butterfly over 4 lanes
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            const float send = hi16 ? v[i] : v[i + 12];
            const float keep = hi16 ? v[i + 12] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 16);
          }
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const float send = hi8 ? v[i] : v[i + 6];
            const float keep = hi8 ? v[i + 6] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 8);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float send = hi4 ? v[i] : v[i + 3];
            const float keep = hi4 ? v[i + 3] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 4);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            v[i] += __shfl_xor_sync(FULL, v[i], 2);
            v[i] += __shfl_xor_sync(FULL, v[i], 1);
          }
          const float mine = q == 0 ? v[0] : (q == 1 ? v[1] : v[2]);
          if (q < 3 && mine != 0.f) {
            const uint32_t slot = __float_as_uint(r[R_SLOT]);
            if ((long long)slot < a.VM) {
              atomicAdd(a.grad + (size_t)slot * TS_GRAD_WORDS + widx, mine);
            } else {
              atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
            }
          }
        }
      }
    }
  }
  count_add(&a.hdr->bwd_contrib, contrib);
  return ok;
}

__device__ __forceinline__ void init_bars(RenderSmem& sm) {
  if (threadIdx.x == 0) {
    ts_mbar_init(&sm.bar[0], 1);
    ts_mbar_init(&sm.bar[1], 1);
    ts_fence_mbar_init();
  }
  __syncthreads();
}

// Next tile of a persistent CTA (the same value in every thread), or -1 when none is left.
__device__ __forceinline__ long long next_tile(const RenderArgs& a, RenderSmem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) sm.next_tile = (int)atomicAdd(a.counter, 1u);
  __syncthreads();
  return sm.next_tile < a.n_tiles ? (long long)sm.next_tile : -1;
}

template <int TW, int TH, bool PERSIST, bool AUX>
__global__ void __launch_bounds__(TW * TH, raster_min_blocks(TW * TH)) k_render_fwd(RenderArgs a) {
  extern __shared__ __align__(128) float4 smrec[];
  __shared__ RenderSmem sm;
  init_bars(sm);
  int seq = 0;
  if (!PERSIST) {
    fwd_tile<TW, TH, AUX>(a, blockIdx.x, smrec, sm, seq);
    return;
  }
  for (long long t = next_tile(a, sm); t >= 0; t = next_tile(a, sm))
    if (!fwd_tile<TW, TH, AUX>(a, t, smrec, sm, seq)) return;
}

template <int TW, int TH, bool PERSIST, bool AUX>
__global__ void __launch_bounds__(TW * TH, raster_min_blocks(TW * TH)) k_render_bwd(RenderArgs a) {
  extern __shared__ __align__(128) float4 smrec[];
  __shared__ RenderSmem sm;
  init_bars(sm);
  int seq = 0;
  if (!PERSIST) {
    bwd_tile<TW, TH, AUX>(a, blockIdx.x, smrec, sm, seq);
    return;
  }
  for (long long t = next_tile(a, sm); t >= 0; t = next_tile(a, sm))
    if (!bwd_tile<TW, TH, AUX>(a, t, smrec, sm, seq)) return;
}

// Dynamic shared memory: two stage buffers of S 128-byte records, then (with the side array) two
// of S 16-byte side entries.
template <int TW, int TH, bool AUX>
cudaError_t launch_pair(bool fwd, bool persist, const RenderArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)2 * a.S * (AUX ? 144 : 128);
  if (a.n_tiles == 0) return cudaSuccess;
  if (!persist) {
    if (fwd) k_render_fwd<TW, TH, false, AUX><<<(unsigned)a.n_tiles, TW * TH, smem, s>>>(a);
    else k_render_bwd<TW, TH, false, AUX><<<(unsigned)a.n_tiles, TW * TH, smem, s>>>(a);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fwd) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_fwd<TW, TH, true, AUX>, TW * TH, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd<TW, TH, true, AUX>, TW * TH, smem);
  const long long grid = std::max(1LL, std::min<long long>(a.n_tiles, (long long)sms * std::max(per_sm, 1)));
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (fwd) k_render_fwd<TW, TH, true, AUX><<<(unsigned)grid, TW * TH, smem, s>>>(a);
  else k_render_bwd<TW, TH, true, AUX><<<(unsigned)grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool AUX>
cudaError_t dispatch_tiles(bool fwd, const TsPlanImpl* p, const RenderArgs& a, cudaStream_t s) {
  const int tw = p->prm.tile_w, th = p->prm.tile_h;
  const bool persist = (p->prm.flags & TS_FLAG_PERSISTENT) != 0;
  if (tw == 16 && th == 8) return launch_pair<16, 8, AUX>(fwd, persist, a, s);
  if (tw == 16 && th == 16) return launch_pair<16, 16, AUX>(fwd, persist, a, s);
  if (tw == 8 && th == 8) return launch_pair<8, 8, AUX>(fwd, persist, a, s);
  if (tw == 32 && th == 8) return launch_pair<32, 8, AUX>(fwd, persist, a, s);
  if (tw == 16 && th == 32) return launch_pair<16, 32, AUX>(fwd, persist, a, s);
  if (tw == 32 && th == 16) return launch_pair<32, 16, AUX>(fwd, persist, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t dispatch(bool fwd, const TsPlanImpl* p, const RenderArgs& a, cudaStream_t s) {
  return (p->normals || p->face_sigma) ? dispatch_tiles<true>(fwd, p, a, s) : dispatch_tiles<false>(fwd, p, a, s);
}

RenderArgs base_args(const TsPlanImpl* p, const TsWs& w) {
  RenderArgs a;
  a.views = w.views;
  a.V = p->V;
  a.M = p->M;
  a.VM = (long long)p->V * p->M;
  a.n_tiles = p->n_tiles;
  a.frec = w.frec;
  a.ids = w.vals[ts_sort_final_buffer(p)];
  a.ranges = w.ranges;
  a.color = a.depth = a.alpha = nullptr;
  a.tfin = w.tfin;
  a.nlast = w.nlast;
  a.dC = a.dD = a.dA = nullptr;
  a.grad = w.grad;
  a.sigma = p->prm.sigma;
  a.alpha_min = p->prm.alpha_min;
  a.alpha_max = p->prm.alpha_max;
  a.T_min = p->prm.T_min;
  a.bg0 = p->prm.bg[0];
  a.bg1 = p->prm.bg[1];
  a.bg2 = p->prm.bg[2];
  a.S = p->prm.tris_per_stage;
  a.hdr = w.hdr;
  a.counter = &w.hdr->tile_counter;
  a.cmask = w.cmask;
  a.aux = w.aux;
  a.normals = p->normals;
  a.face_sigma = p->face_sigma;
  a.cov = w.cov;
  a.normal = nullptr;
  a.dN = nullptr;
  return a;
}

}  // namespace

cudaError_t ts_launch_render_fwd(const TsPlanImpl* p, const TsWs& w, float* color, float* depth, float* alpha,
                                 float* normal, cudaStream_t s) {
  RenderArgs a = base_args(p, w);
  a.color = color;
  a.depth = depth;
  a.alpha = alpha;
  a.normal = normal;
  return dispatch(true, p, a, s);
}

cudaError_t ts_launch_render_bwd(const TsPlanImpl* p, const TsWs& w, const float* dC, const float* dD,
                                 const float* dA, const float* dN, cudaStream_t s) {
  RenderArgs a = base_args(p, w);
  a.dC = dC;
  a.dD = dD;
  a.dA = dA;
  a.dN = dN;
  return dispatch(false, p, a, s);
}
