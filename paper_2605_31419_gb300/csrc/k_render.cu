// k_render.cu -- Eq. 3-4 forward blend and its adjoint, one CTA per (view, tile) at a time.
//
// Staging: the tile's depth-sorted face ids select 128-byte records that the CTA copies into
// shared memory with 16-byte cp.async copies (a warp moves four records per instruction; one
// bulk copy per record was bound by its per-request cost); two buffers alternate so the next
// stage streams in while the current one is blended.  Each warp owns an 8 x 4 pixel sub-block of
// the tile; per stage, a mask per record says which sub-blocks can contain one of the face's
// covered pixel centres, and each warp walks only the set bits of its own ballot over the stage.
//
// Forward: per pixel, front to back: window (Eq. 3) from cancellation-free edge functions,
// alpha = min(alpha_max, o_F I), skip below alpha_min, stop before the face that would take T
// below T_min, accumulate colour, depth and opacity (Eq. 4).  Writes C + T bg, D, A = 1 - T, and
// per pixel T_final and the list position after the last contribution, and per sorted pair and
// warp the mask of the warp's pixels that blended the face.
//
// Backward: per pixel, back to front from that position: recover T_n = T_{n+1} / (1 - alpha_n),
// keep the suffix sum S of later contributions (including the background term), form
// dL/dalpha_n = T_n v_n - S / (1 - alpha_n) with v_n = gC . c_n + gD z_n + gA, and chain into 23
// per-face sums (barycentric-weighted gradients of the edge, colour and depth interpolants, of
// o_F, and the contribution count).  The forward stores, per sorted pair and warp, the 32-bit
// mask of the warp's pixels that blended the face; the backward numbers those (face, pixel)
// entries back to front (a warp-wide scan of the masks' bit counts) and processes them 32 at a
// time, one per lane, so that no lane idles on a pixel the face does not cover.  Lanes holding
// entries of the same pixel replay its recurrence in entry order (the same products and sums, in
// the same order, as a per-pixel loop).  Every
// per-face sum is over products of two per-entry factors (a weighted gradient times a
// barycentric coordinate, or a scalar times one); each lane writes its factors to a ring row in
// shared memory, and lane L then sums word L's products over each face's run of rows and adds it
// into the face's accumulator with one atomic.
//
// Launch forms: one CTA per tile, or persistent CTAs (as many as fit on the GPU) that take tiles
// from a device counter.  The fused L1 step (ts_render_step_l1) runs a tile's forward, its loss
// and its backward in one CTA.
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
  uint32_t* lmask;
  const float4* aux;   // per (view, face): camera-space normal and, in .w, sigma_F; else null
  bool normals;        // TS_FLAG_NORMALS: composite the normal map
  bool face_sigma;     // TS_FLAG_FACE_SIGMA: each face's own window exponent
  float* normal;       // normal map output (may be null)
  const float* dN;     // gradient w.r.t. the normal map (may be null)
  uint32_t* cov;       // per (view, face) pixels blended by the forward (TS_FLAG_STATS), else null
  // fused L1 step (ts_render_step_l1): targets, depth weight, optional loss-gradient images and
  // the per-tile loss partials
  const float* tC;
  const float* tD;
  float lambda_dep;
  float* dC_out;
  float* dD_out;
  float* tloss;
  TsDevHeader* hdr;
  unsigned long long* ctr;  // counter slots (contributions)
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
  uint16_t smask[2][128];  // per staged face, the warps (sub-blocks) that visit it
  float lred[16][2];       // fused step: the warps' loss sums
  int lmax[16];            // fused step: the warps' largest last positions
  int view;
  int nmax;
  int next_tile;
  int fail;
};

// Forward only, TS_FLAG_STATS: per staged face, the number of the tile's pixels that blended it.
struct FwdMasks {
  uint32_t cv[2][128];
};

// What a tile's forward leaves for the backward of the fused step, per pixel (thread) and for the
// stage buffers: the last stage processed, its buffer, and whether the stage before it is still in
// the other buffer.
struct TileCarry {
  float T, C0, C1, C2, D;
  int nl;
  int st_last, b_last;
  bool prev_in;
};

// The backward's per-pixel inputs in the fused step: T_final and the loss gradients.
struct PixIn {
  float T, gC0, gC1, gC2, gD;
  int nl;
  int nmax;  // the same in every thread: the tile's largest nl
};

// Backward scratch per warp: the pixels' back-to-front state and the ring of one batch's rows.  A ring row holds the
// factors of one entry; row words: 0-2 barycentrics l_k; 3-5 w gC_c; 6 w gD; 7-9 dm routed to
// the nearest edge (zero for the other two); 10 dL/do_F; 11 one; with the side array 12-14 w gN_c
// and 15 dL/dsigma_F.
constexpr int RING_CAP = 32;   // rows: one batch of entries, one per lane
constexpr int FMAX = 4;        // faces per lane when the backward numbers a stage's entries (128 / 32)
template <bool AUX>
struct Ring {
  static constexpr int EW = AUX ? 16 : 12;
  static constexpr int BYTES_PER_WARP = RING_CAP * EW * 4 + 32 * 8;
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

// Every thread of the CTA copies 16-byte chunks of stage `st` (records [st*S, st*S + cnt) of the
// tile's list) into buffer `b` with cp.async, eight chunks per record and, with the side array,
// one more for the record's side entry (normal, sigma_F) after both record buffers; one commit
// group per stage.  A warp moves four records per instruction, and no copy engine request is
// made per record.
template <bool AUX>
__device__ __forceinline__ void issue_stage(const RenderArgs& a, float4* smrec, int b, int st, uint32_t start, int n,
                                            const float4* vbase, const float4* nbase, int nthreads) {
  const int S = a.S;
  const int cnt = min(S, n - st * S);
  constexpr int PER = AUX ? 9 : 8;
  for (int i = threadIdx.x; i < cnt * PER; i += nthreads) {
    const int j = i / PER, c = i - j * PER;
    uint32_t id = __ldg(a.ids + start + (uint32_t)(st * S + j));
    if ((long long)id >= a.M) {  // never expected: record the fault and stage an in-bounds record
      atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
      id = 0;
    }
    if (!AUX || c < 8) {
      ts_cp_async16(smrec + ((size_t)b * S + j) * 8 + c, vbase + (size_t)id * 8 + c);
    } else {
      ts_cp_async16(smrec + (size_t)2 * S * 8 + (size_t)b * S + j, nbase + id);
    }
  }
  ts_cp_async_commit();
}

// For each staged record, the mask of warp sub-blocks (8 x 4 pixels) that can contain one of its
// covered pixel centres: sub-blocks inside the face's pixel box whose pixel-centre rectangle,
// widened by 0.01 px, is not entirely outside one of the three edges.  Conservative: a pixel with
// a positive window always keeps its sub-block's bit.
template <int TW, int TH>
__device__ __forceinline__ void stage_masks(const float* rb, uint16_t* smask, int cnt, int X0, int Y0) {
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
    smask[j] = (uint16_t)mask;
  }
}


// Wait for the stage issued last: each thread's copies (they always complete), then a barrier.
__device__ __forceinline__ void wait_stage() {
  ts_cp_async_wait_all();
  __syncthreads();
}

// Forward of one tile; seq counts the stages this CTA has staged so far (buffer seq & 1 is next).
template <int TW, int TH, bool AUX, bool FUSED = false>
__device__ __forceinline__ void fwd_tile(const RenderArgs& a, long long tile, float4* smrec, RenderSmem& sm,
                                         FwdMasks& fm, int& seq, TileCarry* carry = nullptr,
                                         const TileGeom<TW, TH>* gin = nullptr) {
  const TileGeom<TW, TH> g = FUSED ? *gin : tile_geom<TW, TH>(a, tile, sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 rg = a.ranges[tile];
  const int n = (int)(rg.y - rg.x);
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  float N0 = 0.f, N1 = 0.f, N2 = 0.f;
  int nl = 0;
  bool done = !g.inimg;
  unsigned contrib = 0;
  int st_last = -1, b_last = 0;
  bool prefetched = false;
  if (n > 0) {
    const int S = a.S;
    const int nst = (n + S - 1) / S;
    const float4* vbase = a.frec + (size_t)g.view * (size_t)a.M * 8;
    const float4* nbase = AUX ? a.aux + (size_t)g.view * (size_t)a.M : nullptr;
    issue_stage<AUX>(a, smrec, seq & 1, 0, rg.x, n, vbase, nbase, TW * TH);
    for (int st = 0; st < nst; ++st) {
      const int b = seq & 1;
      const int cnt = min(S, n - st * S);
      wait_stage();
      ++seq;
      st_last = st;
      b_last = b;
      const float* rb = reinterpret_cast<const float*>(smrec + (size_t)b * S * 8);
      const float4* nb = smrec + (size_t)2 * S * 8 + (size_t)b * S;
      stage_masks<TW, TH>(rb, sm.smask[b], cnt, g.X0, g.Y0);
      if (a.cov)
        for (int j = threadIdx.x; j < cnt; j += TW * TH) fm.cv[b][j] = 0u;
      __syncthreads();
      if (st + 1 < nst) issue_stage<AUX>(a, smrec, b ^ 1, st + 1, rg.x, n, vbase, nbase, TW * TH);
      for (int q = 0; q * 32 < cnt; ++q) {
        const int jq = q * 32 + lane;
        unsigned lm = 0;  // lane L: this warp's pixels that blended face q * 32 + L
        unsigned bits = __ballot_sync(FULL, jq < cnt && ((sm.smask[b][min(jq, cnt - 1)] >> warp) & 1u));
        while (bits) {
          const int j0 = q * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const bool two = bits != 0;
          const int j1 = two ? q * 32 + __ffs(bits) - 1 : j0;
          if (two) bits &= bits - 1;
          // two faces per pass: both edge functions first (independent work the scheduler can overlap),
          // then the compositing in list order, exactly as one face at a time
          const float* r0 = rb + j0 * TS_REC_WORDS;
          const float* r1 = rb + j1 * TS_REC_WORDS;
          const TsPix e0 = ts_eval_edges(r0, g.px, g.py);
          const TsPix e1 = ts_eval_edges(r1, g.px, g.py);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int j = h ? j1 : j0;
            const float* r = h ? r1 : r0;
            const TsPix e = h ? e1 : e0;
            bool blended = false;
            if (!done && e.m > 0.f) {
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
            // the backward takes exactly these (face, pixel) contributions
            const unsigned bl = __ballot_sync(FULL, blended);
            if (lane == (j & 31)) lm = bl;
            if (bl && lane == 0 && a.cov) atomicAdd(&fm.cv[b][j], (unsigned)__popc(bl));
          }
        }
        if (a.lmask && jq < cnt) a.lmask[(size_t)(rg.x + (uint32_t)(st * S + jq)) * (TW * TH / 32) + warp] = lm;
      }
      const int alive = __syncthreads_count(!done);
      if (a.cov) {
        for (int j = threadIdx.x; j < cnt; j += TW * TH) {
          if (fm.cv[b][j]) {  // face m of the record's slot m * V + view
            const uint32_t slot = __float_as_uint(rb[j * TS_REC_WORDS + R_SLOT]);
            const long long m = (long long)(slot / (uint32_t)a.V);
            if (m < a.M) atomicAdd(a.cov + (long long)g.view * a.M + m, fm.cv[b][j]);
          }
        }
      }
      if (alive == 0) {
        if (st + 1 < nst) {  // a prefetched stage is in flight: let it land before leaving
          wait_stage();
          ++seq;
          prefetched = true;
        }
        break;
      }
    }
  }
  ts_count_add(a.ctr, TS_CTR_FWD, contrib);
  if constexpr (FUSED) {
    carry->T = T;
    carry->C0 = C0;
    carry->C1 = C1;
    carry->C2 = C2;
    carry->D = D;
    carry->nl = nl;
    carry->st_last = st_last;
    carry->b_last = b_last;
    carry->prev_in = st_last >= 1 && !prefetched;
  }
  if (g.inimg) {
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
    if (!FUSED) {  // what ts_render_bwd needs; the fused step keeps them in registers
      a.tfin[o] = T;
      a.nlast[o] = nl;
    }
  }
}

// Lane `lane`'s gradient word as a product of two ring-row words (ia x ib); false for a lane with
// no word of its own (it multiplies one by one and adds nothing).
template <bool AUX>
__device__ __forceinline__ bool ring_word(int lane, int& ia, int& ib) {
  ia = 11;
  ib = 11;
  if (lane < G_C) {  // G_E[i][k]: dm routed to edge i, times l_k
    ia = 7 + lane / 3;
    ib = lane % 3;
  } else if (lane < G_Z) {  // G_C[c][k]: w gC_c times l_k
    ia = 3 + (lane - G_C) / 3;
    ib = (lane - G_C) % 3;
  } else if (lane < G_O) {  // G_Z[k]: w gD times l_k
    ia = 6;
    ib = lane - G_Z;
  } else if (lane == G_O) {
    ia = 10;
  } else if (lane == G_CNT) {
  } else if (AUX && lane == 23) {
    ia = 12;
  } else if (AUX && lane == 24) {
    ia = 15;
  } else if (AUX && lane == 30) {
    ia = 13;
  } else if (AUX && lane == 31) {
    ia = 14;
  } else {
    return false;
  }
  return true;
}

// The edge evaluation of ts_eval_edges from the record's first four 16-byte groups (one vector
// load each; lanes holding different faces then conflict only within a quarter warp).
static_assert(R_U0 == 0 && R_V0 == 3 && R_V1 == 4 && R_E0X == 6 && R_E1X == 8 && R_E2X == 10 && R_K0 == 12 &&
                  R_INVD == 15 && R_OF == 16 && R_C0 == 17 && R_C1 == 20 && R_C2 == 23 && R_Z0 == 26 && R_Z2 == 28,
              "record layout assumed by the vector loads");
__device__ __forceinline__ TsPix eval_edges_v(float4 q0, float4 q1, float4 q2, float4 q3, float px, float py) {
  TsPix o;
  o.cr0 = ts_det2(q1.z, q1.w, px - q0.x, py - q0.w);
  o.cr1 = ts_det2(q2.x, q2.y, px - q0.y, py - q1.x);
  o.cr2 = ts_det2(q2.z, q2.w, px - q0.z, py - q1.y);
  const float e0 = o.cr0 * q3.x, e1 = o.cr1 * q3.y, e2 = o.cr2 * q3.z;
  o.m = e0;
  o.arg = 0;
  if (e1 < o.m) { o.m = e1; o.arg = 1; }
  if (e2 < o.m) { o.m = e2; o.arg = 2; }
  return o;
}

template <int TW, int TH, bool AUX, bool FUSED = false>
__device__ __forceinline__ void bwd_tile(const RenderArgs& a, long long tile, float4* smrec, RenderSmem& sm,
                                         int& seq, const PixIn* pin = nullptr, const TileCarry* carry = nullptr,
                                         const TileGeom<TW, TH>* gin = nullptr) {
  const TileGeom<TW, TH> g = FUSED ? *gin : tile_geom<TW, TH>(a, tile, sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 rg = a.ranges[tile];
  float T = 0.f, Sacc = 0.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f;
  float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
  int nl = 0;
  if (FUSED) {  // the forward's state and the loss gradients, still in registers
    if (g.inimg) {
      T = pin->T;
      nl = pin->nl;
      gC0 = pin->gC0;
      gC1 = pin->gC1;
      gC2 = pin->gC2;
      gD = pin->gD;
      Sacc = T * (gC0 * a.bg0 + gC1 * a.bg1 + gC2 * a.bg2);
    }
  } else if (g.inimg) {
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
  int nmax;
  if (FUSED) {
    nmax = pin->nmax;  // the tile's largest last position, reduced with the loss sums
  } else {
    if (threadIdx.x == 0) sm.nmax = 0;
    __syncthreads();
    {
      const int m = __reduce_max_sync(FULL, (unsigned)nl);
      if (lane == 0 && m) atomicMax(&sm.nmax, m);
    }
    __syncthreads();
    nmax = sm.nmax;
  }
  // positions come from the forward pass over the same lists; clamp in case the caller did not
  // run it after the last ts_bin
  const int n = min(nmax, (int)(rg.y - rg.x));
  unsigned contrib = 0;
  if (n > 0) {
    const int S = a.S;
    const int nst = (n + S - 1) / S;
    const float4* vbase = a.frec + (size_t)g.view * (size_t)a.M * 8;
    const float4* nbase = AUX ? a.aux + (size_t)g.view * (size_t)a.M : nullptr;
    if (!FUSED) issue_stage<AUX>(a, smrec, seq & 1, nst - 1, rg.x, n, vbase, nbase, TW * TH);
    constexpr int EW = Ring<AUX>::EW;
    unsigned char* wbase = reinterpret_cast<unsigned char*>(smrec + (size_t)2 * S * (AUX ? 9 : 8)) +
                           (size_t)warp * Ring<AUX>::BYTES_PER_WARP;
    float* ring = reinterpret_cast<float*>(wbase);
    float2* pst = reinterpret_cast<float2*>(wbase + RING_CAP * EW * 4);  // per pixel lane: (T, S)
    pst[lane] = make_float2(T, Sacc);
    int ia, ib;
    const bool has = ring_word<AUX>(lane, ia, ib);
    const int xw = g.x - (lane & 7), yw = g.y - (lane >> 3);  // the warp's first pixel
    for (int k = 0; k < nst; ++k) {
      const int st = nst - 1 - k;
      int b = seq & 1;
      const int cnt = min(S, n - st * S);
      // The forward's lane masks (positions below the tile's largest list position after a
      // contribution were all written by it) give, per face, the pixels of this warp that blended
      // it.  Lane L holds the masks of F = ceil(cnt / 32) faces, lane 0 the backmost; the stage's
      // (face, pixel) entries are numbered back to front, face by face, pixels in lane order, and
      // each batch of 32 consecutive numbers gives every lane one entry.  The masks load while
      // the stage's copies land.
      constexpr int NW = TW * TH / 32;
      const uint32_t* lmrow = a.lmask + (size_t)(rg.x + (uint32_t)(st * S)) * NW + warp;
      const int F = (cnt + 31) >> 5;  // faces per lane: lane L holds faces F * (32 - L) - 1 - i, i < F
      unsigned lmk[FMAX];
#pragma unroll
      for (int i = 0; i < FMAX; ++i) {
        const int jf = F * (32 - lane) - 1 - i;
        lmk[i] = (i < F && jf < cnt) ? lmrow[(size_t)jf * NW] : 0u;
      }
      if (FUSED) {
        // the forward's last stage, and the one before it unless a prefetch replaced it, are
        // still staged; other stages are staged again (all warps are done with both buffers)
        if (st == carry->st_last) {
          b = carry->b_last;
        } else if (st == carry->st_last - 1 && carry->prev_in) {
          b = carry->b_last ^ 1;
        } else {
          __syncthreads();
          b = 0;
          issue_stage<AUX>(a, smrec, b, st, rg.x, n, vbase, nbase, TW * TH);
          wait_stage();
        }
      } else {
        wait_stage();
        ++seq;
        if (k + 1 < nst) issue_stage<AUX>(a, smrec, b ^ 1, st - 1, rg.x, n, vbase, nbase, TW * TH);
      }
      const float* rb = reinterpret_cast<const float*>(smrec + (size_t)b * S * 8);
      const float4* nb = smrec + (size_t)2 * S * 8 + (size_t)b * S;
      {
        // lane L's faces have popc of their masks entries; their numbers start at the exclusive
        // scan over the lanes, face by face within a lane
        int c = 0;
#pragma unroll
        for (int i = 0; i < FMAX; ++i) c += __popc(lmk[i]);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - c;
        for (int e0 = 0; e0 < total; e0 += 32) {
          const int ne = min(total - e0, 32);
          const bool act = lane < ne;
          const int ee = e0 + lane;
          // the entry's lane: the last lane whose first number is at most ee (binary search)
          int ow = 0;
#pragma unroll
          for (int w = 16; w > 0; w >>= 1) {
            const int ex = __shfl_sync(FULL, excl, (ow + w) & 31);
            if (ow + w < 32 && ex <= ee) ow += w;
          }
          int kk = ee - __shfl_sync(FULL, excl, ow);  // the entry's rank among that lane's pixels
          // the face among the lane's F faces, then its pixel: the kk-th set bit of its mask
          unsigned om = 0u;
          int fi = 0;
          bool found = false;
#pragma unroll
          for (int i = 0; i < FMAX; ++i) {
            const unsigned mi = __shfl_sync(FULL, lmk[i], ow);
            const int ci = __popc(mi);
            if (!found && i < F) {
              if (kk < ci) {
                om = mi;
                fi = i;
                found = true;
              } else {
                kk -= ci;
              }
            }
          }
          int pb = 0;
          unsigned mm = om;
#pragma unroll
          for (int w = 16; w > 0; w >>= 1) {
            const int cl = __popc(mm & ((1u << w) - 1u));
            if (kk >= cl) {
              kk -= cl;
              pb += w;
              mm >>= w;
            }
          }
          const int j = act ? F * (32 - ow) - 1 - fi : 0;
          const int p = act ? pb : lane;
          // -- one entry per lane: face j at pixel lane p ---------------------------------------
          const float4* r4 = reinterpret_cast<const float4*>(rb + j * TS_REC_WORDS);
          const float px = (float)(xw + (p & 7)) + 0.5f, py = (float)(yw + (p >> 3)) + 0.5f;
          const float sig = (AUX && a.face_sigma) ? nb[j].w : a.sigma;
          const float4 q3 = r4[3];  // k_0, k_1, k_2, invD
          const TsPix e = eval_edges_v(r4[0], r4[1], r4[2], q3, px, py);
          const float4 q4 = r4[4];  // o_F, colour of vertex 0
          const float oF = q4.x;
          const float I = act ? ts_window(e.m, sig) : 0.f;
          const float al = fminf(oF * I, a.alpha_max);
          const float ro = ts_rcp_approx(1.f - al);  // 1 - al >= 1 - alpha_max
          // entries of the same pixel, in entry (back-to-front) order; each lane replays its
          // pixel's recurrence T <- T / (1 - alpha) over the earlier ones and itself, in order
          const unsigned peers = __match_any_sync(FULL, act ? p : 32 + lane);
          const int K = (int)__reduce_max_sync(FULL, (unsigned)__popc(peers));
          const float2 st0 = pst[p];
          float Tn = st0.x;
          {
            unsigned rem = peers;
            for (int i = 0; i < K; ++i) {
              const int src = rem ? __ffs(rem) - 1 : 31;
              const bool use = rem != 0 && src <= lane;
              rem &= rem - 1;
              const float f = __shfl_sync(FULL, ro, src);
              if (use) Tn *= f;
            }
          }
          const float qC0 = __shfl_sync(FULL, gC0, p), qC1 = __shfl_sync(FULL, gC1, p);
          const float qC2 = __shfl_sync(FULL, gC2, p), qD = __shfl_sync(FULL, gD, p);
          const float qA = __shfl_sync(FULL, gA, p);
          float qN0 = 0.f, qN1 = 0.f, qN2 = 0.f;
          if constexpr (AUX) {
            qN0 = __shfl_sync(FULL, gN0, p);
            qN1 = __shfl_sync(FULL, gN1, p);
            qN2 = __shfl_sync(FULL, gN2, p);
          }
          const float invD = q3.w;
          const float l0 = e.cr1 * invD, l1 = e.cr2 * invD, l2 = e.cr0 * invD;
          const float4 q5 = r4[5], q6 = r4[6];  // colours of vertices 1 and 2, depths z_0, z_1
          const float4 q7 = r4[7];
          const float z2 = q7.x;
          const uint32_t slot = __float_as_uint(q7.w);
          const float c0 = l0 * q4.y + l1 * q5.x + l2 * q5.w;
          const float c1 = l0 * q4.z + l1 * q5.y + l2 * q6.x;
          const float c2 = l0 * q4.w + l1 * q5.z + l2 * q6.y;
          const float z = l0 * q6.z + l1 * q6.w + l2 * z2;
          float val = qC0 * c0 + qC1 * c1 + qC2 * c2 + qD * z + qA;
          if (AUX && a.normals) {
            const float4 nn = nb[j];
            val += qN0 * nn.x + qN1 * nn.y + qN2 * nn.z;
          }
          const float w = al * Tn;
          const float add = val * al * Tn;  // this face's term of the suffix sum S seen by earlier faces
          float Sn = st0.y;
          {
            unsigned rem = peers;
            for (int i = 0; i < K; ++i) {
              const int src = rem ? __ffs(rem) - 1 : 31;
              const bool use = rem != 0 && src < lane;
              rem &= rem - 1;
              const float f = __shfl_sync(FULL, add, src);
              if (use) Sn += f;
            }
          }
          __syncwarp();  // every lane has read its pixel's state before the last entries replace it
          if (act && (peers >> lane) == 1u) pst[p] = make_float2(Tn, Sn + add);
          const float dal = val * Tn - Sn * ro;
          float go = 0.f, dm = 0.f, gs = 0.f;
          if (!(oF * I > a.alpha_max)) {
            go = dal * I;
            const float dI = dal * oF;
            // I >= alpha_min / o_F for a contributing entry, far from zero
            dm = (sig == 0.5f) ? dI * 0.5f * ts_rcp_approx(I) : dI * sig * I / e.m;
            if constexpr (AUX) {  // dL/dsigma_F = dL/dalpha o_F I ln(ratio)
              if (a.face_sigma) gs = dI * I * logf(e.m);
            }
          }
          if (act) {
            float4* row = reinterpret_cast<float4*>(ring + lane * EW);
            row[0] = make_float4(l0, l1, l2, qC0 * w);
            row[1] = make_float4(qC1 * w, qC2 * w, qD * w, e.arg == 0 ? dm : 0.f);
            row[2] = make_float4(e.arg == 1 ? dm : 0.f, e.arg == 2 ? dm : 0.f, go, 1.f);
            if constexpr (AUX) row[3] = make_float4(qN0 * w, qN1 * w, qN2 * w, gs);
            ++contrib;
          }
          // the batch's faces are runs of consecutive entries; lane L sums word L over each run
          const int jprev = __shfl_up_sync(FULL, j, 1);  // in every lane, outside any condition
          const unsigned starts = __ballot_sync(FULL, act && (lane == 0 || j != jprev));
          __syncwarp();
          unsigned rem = starts;
          while (rem) {
            const int s0 = __ffs(rem) - 1;
            rem &= rem - 1;
            const int s1 = rem ? __ffs(rem) - 1 : ne;
            const uint32_t sl = __shfl_sync(FULL, slot, s0);
            float sum = 0.f;
#pragma unroll 4
            for (int q = s0; q < s1; ++q) sum = fmaf(ring[q * EW + ia], ring[q * EW + ib], sum);
            if (has && sum != 0.f) {
              if ((long long)sl < a.VM) {
                atomicAdd(a.grad + (size_t)sl * TS_GRAD_WORDS + lane, sum);
              } else {
                atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }
  ts_count_add(a.ctr, TS_CTR_BWD, contrib);
}

// The fused L1 step of one tile: the forward, the mean-L1 loss of its pixels (Eq. 8 L1 part with
// the depth term of Eq. 9: per pixel dL/dC = sign(C - Cbar) / (3HW) on the colour image with its
// background term, dL/dD = lambda_dep sign(D - Dbar) / (HW) where Dbar > 0), the tile's loss sums
// in a fixed order, and the backward from those gradients -- the same values ts_render_fwd,
// ts_l1_loss and ts_render_bwd give, without the images' round trip through memory.
template <int TW, int TH>
__device__ __forceinline__ void step_tile(const RenderArgs& a, long long tile, float4* smrec, RenderSmem& sm,
                                          FwdMasks& fm, int& seq) {
  TileCarry c;
  const TileGeom<TW, TH> g = tile_geom<TW, TH>(a, tile, sm);
  fwd_tile<TW, TH, false, true>(a, tile, smrec, sm, fm, seq, &c, &g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PixIn pin{c.T, 0.f, 0.f, 0.f, 0.f, c.nl, 0};
  float lc = 0.f, ld = 0.f;
  if (g.inimg) {
    const long long HW = (long long)g.vw.W * g.vw.H;
    const long long pi = (long long)g.y * g.vw.W + g.x;
    const long long o = g.vw.pix_off + pi;
    const float ic = 1.0f / (3.0f * (float)HW), id = a.lambda_dep / (float)HW;
    const float col[3] = {c.C0 + c.T * a.bg0, c.C1 + c.T * a.bg1, c.C2 + c.T * a.bg2};  // the colour image
    float gc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const long long q = 3 * g.vw.pix_off + ch * HW + pi;
      const float r = col[ch] - a.tC[q];
      lc += fabsf(r);
      gc[ch] = r > 0.f ? ic : (r < 0.f ? -ic : 0.f);
      if (a.dC_out) a.dC_out[q] = gc[ch];
    }
    const float t = a.tD[o];
    const float r = c.D - t;
    const bool valid = t > 0.f;
    if (valid) ld += fabsf(r);
    pin.gD = valid ? (r > 0.f ? id : (r < 0.f ? -id : 0.f)) : 0.f;
    if (a.dD_out) a.dD_out[o] = pin.gD;
    pin.gC0 = gc[0];
    pin.gC1 = gc[1];
    pin.gC2 = gc[2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lc += __shfl_xor_sync(FULL, lc, o);
    ld += __shfl_xor_sync(FULL, ld, o);
  }
  const int wmax = (int)__reduce_max_sync(FULL, (unsigned)c.nl);
  if (lane == 0) {
    sm.lred[warp][0] = lc;
    sm.lred[warp][1] = ld;
    sm.lmax[warp] = wmax;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < TW * TH / 32; ++w) sum += sm.lred[w][threadIdx.x];
    a.tloss[2 * tile + threadIdx.x] = sum;
  }
#pragma unroll
  for (int w = 0; w < TW * TH / 32; ++w) pin.nmax = max(pin.nmax, sm.lmax[w]);
  bwd_tile<TW, TH, false, true>(a, tile, smrec, sm, seq, &pin, &c, &g);
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
  __shared__ FwdMasks fm;
  int seq = 0;
  if constexpr (!PERSIST) {
    fwd_tile<TW, TH, AUX>(a, blockIdx.x, smrec, sm, fm, seq);
  } else {
    for (long long t = next_tile(a, sm); t >= 0; t = next_tile(a, sm))
      fwd_tile<TW, TH, AUX>(a, t, smrec, sm, fm, seq);
  }
}

template <int TW, int TH, bool PERSIST, bool AUX>
__global__ void __launch_bounds__(TW * TH, raster_min_blocks(TW * TH)) k_render_bwd(RenderArgs a) {
  extern __shared__ __align__(128) float4 smrec[];
  __shared__ RenderSmem sm;
  int seq = 0;
  if constexpr (!PERSIST) {
    bwd_tile<TW, TH, AUX>(a, blockIdx.x, smrec, sm, seq);
  } else {
    for (long long t = next_tile(a, sm); t >= 0; t = next_tile(a, sm))
      bwd_tile<TW, TH, AUX>(a, t, smrec, sm, seq);
  }
}

// The fused step kernel.  Its forward's coverage counts (TS_FLAG_STATS) live in the space of the
// backward's rings, which the forward does not use.
template <int TW, int TH, bool PERSIST>
__global__ void __launch_bounds__(TW * TH, raster_min_blocks(TW * TH)) k_render_step(RenderArgs a) {
  extern __shared__ __align__(128) float4 smrec[];
  __shared__ RenderSmem sm;
  static_assert(sizeof(FwdMasks) <= (TW * TH / 32) * Ring<false>::BYTES_PER_WARP, "coverage counts fit the rings");
  FwdMasks& fm = *reinterpret_cast<FwdMasks*>(smrec + (size_t)2 * a.S * 8);
  int seq = 0;
  if constexpr (!PERSIST) {
    step_tile<TW, TH>(a, blockIdx.x, smrec, sm, fm, seq);
  } else {
    for (long long t = next_tile(a, sm); t >= 0; t = next_tile(a, sm)) step_tile<TW, TH>(a, t, smrec, sm, fm, seq);
  }
}

// Per view, the sum of its tiles' loss partials in a fixed order.
__global__ void __launch_bounds__(256) k_loss_tiles(const TsView* __restrict__ views, const float* __restrict__ tloss,
                                                    float lambda_dep, float* __restrict__ loss) {
  __shared__ float red[256][2];
  const TsView& vw = views[blockIdx.x];
  const long long t0 = vw.tile_off, nt = (long long)vw.TX * vw.TY;
  float x = 0.f, y = 0.f;
  for (long long t = threadIdx.x; t < nt; t += 256) {
    x += tloss[2 * (t0 + t)];
    y += tloss[2 * (t0 + t) + 1];
  }
  red[threadIdx.x][0] = x;
  red[threadIdx.x][1] = y;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x][0] += red[threadIdx.x + o][0];
      red[threadIdx.x][1] += red[threadIdx.x + o][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double HW = (double)vw.W * vw.H;
    loss[blockIdx.x] = (float)((double)red[0][0] / (3.0 * HW) + (double)lambda_dep * (double)red[0][1] / HW);
  }
}

template <int TW, int TH>
cudaError_t launch_step(bool persist, const RenderArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)2 * a.S * 128 + (size_t)(TW * TH / 32) * Ring<false>::BYTES_PER_WARP;
  if (a.n_tiles == 0) return cudaSuccess;
  const void* f = persist ? (const void*)k_render_step<TW, TH, true> : (const void*)k_render_step<TW, TH, false>;
  cudaError_t e = ts_smem_limit(f, (int)smem);
  if (e != cudaSuccess) return e;
  if (!persist) {
    k_render_step<TW, TH, false><<<(unsigned)a.n_tiles, TW * TH, smem, s>>>(a);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_step<TW, TH, true>, TW * TH, smem);
  const long long grid = std::max(1LL, std::min<long long>(a.n_tiles, (long long)sms * std::max(per_sm, 1)));
  e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  k_render_step<TW, TH, true><<<(unsigned)grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

// Dynamic shared memory: two stage buffers of S 128-byte records, then (with the side array) two
// of S 16-byte side entries, then in the backward the warps' rings and their headers.
template <int TW, int TH, bool AUX>
cudaError_t launch_pair(bool fwd, bool persist, const RenderArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)2 * a.S * (AUX ? 144 : 128) + (fwd ? 0 : (size_t)(TW * TH / 32) * Ring<AUX>::BYTES_PER_WARP);
  if (a.n_tiles == 0) return cudaSuccess;
  {
    const void* f = fwd ? (persist ? (const void*)k_render_fwd<TW, TH, true, AUX> : (const void*)k_render_fwd<TW, TH, false, AUX>)
                        : (persist ? (const void*)k_render_bwd<TW, TH, true, AUX> : (const void*)k_render_bwd<TW, TH, false, AUX>);
    const cudaError_t e = ts_smem_limit(f, (int)smem);
    if (e != cudaSuccess) return e;
  }
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
  a.ids = w.vals[0];
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
  a.ctr = w.ctr;
  a.counter = &w.hdr->tile_counter;
  a.lmask = w.lmask;
  a.aux = w.aux;
  a.normals = p->normals;
  a.face_sigma = p->face_sigma;
  a.cov = w.cov;
  a.normal = nullptr;
  a.dN = nullptr;
  a.tC = a.tD = nullptr;
  a.lambda_dep = 0.f;
  a.dC_out = a.dD_out = nullptr;
  a.tloss = nullptr;
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

cudaError_t ts_launch_render_step(const TsPlanImpl* p, const TsWs& w, const float* tgt_color, const float* tgt_depth,
                                  float lambda_dep, float* color, float* depth, float* alpha, float* loss, float* dC,
                                  float* dD, cudaStream_t s) {
  RenderArgs a = base_args(p, w);
  a.color = color;
  a.depth = depth;
  a.alpha = alpha;
  a.tC = tgt_color;
  a.tD = tgt_depth;
  a.lambda_dep = lambda_dep;
  a.dC_out = dC;
  a.dD_out = dD;
  a.tloss = w.tloss;
  const int tw = p->prm.tile_w, th = p->prm.tile_h;
  const bool persist = (p->prm.flags & TS_FLAG_PERSISTENT) != 0;
  cudaError_t e;
  if (tw == 16 && th == 8) e = launch_step<16, 8>(persist, a, s);
  else if (tw == 16 && th == 16) e = launch_step<16, 16>(persist, a, s);
  else if (tw == 8 && th == 8) e = launch_step<8, 8>(persist, a, s);
  else if (tw == 32 && th == 8) e = launch_step<32, 8>(persist, a, s);
  else if (tw == 16 && th == 32) e = launch_step<16, 32>(persist, a, s);
  else if (tw == 32 && th == 16) e = launch_step<32, 16>(persist, a, s);
  else e = cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  k_loss_tiles<<<p->V, 256, 0, s>>>(w.views, w.tloss, lambda_dep, loss);
  return cudaGetLastError();
}
