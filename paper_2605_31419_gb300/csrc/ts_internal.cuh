// ts_internal.cuh -- internal declarations shared by libts translation units (sm_103a).
//
// Layout of the device workspace, the per-(view, face) screen-space record, the host plan, and
// the device helpers the kernels use: the fixed-order FP32 projection (Eq. 1), the
// cancellation-free edge functions (Eq. 2-3), 16-byte cp.async staging, and an mbarrier wait
// that reports a timeout instead of hanging (the failure-detection probe).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ts_api.h"

#define TS_PLAN_MAGIC 0x54535031u  // "TSP1"
#define TS_REC_WORDS 32            // 128-byte record, a multiple of 16 B for cp.async.bulk
#define TS_GRAD_WORDS 32           // per-(view, face) gradient slot: 24 accumulators + chain outputs
#define TS_SCAN_ITEMS 4096         // items per scan block (1024 threads x 4)
#define TS_BIN_FACES 8192          // faces per block of the shared-memory tile counts
#define TS_BIN_MAX_TILES 40960     // the most tiles of a view those counts hold (160 KB)
#define TS_ERRBIT_CAPACITY 1u
#define TS_ERRBIT_TIMEOUT 2u
#define TS_ERRBIT_BOUNDS 4u  // an index failed its bounds check (the access was skipped)
// Device counters (visible records, forward and backward contributions) are kept in TS_CTR_SLOTS
// slots each, one 32-byte sector apart, chosen by the adding warp, so that the adds of all warps
// do not queue on one address; ts_sync_status sums the slots.
#define TS_CTR_SLOTS 1024
#define TS_CTR_STRIDE 4  // unsigned long long words between slots (32 bytes)
enum { TS_CTR_VISIBLE = 0, TS_CTR_FWD = 1, TS_CTR_BWD = 2, TS_N_CTR = 3 };

// Record word indices.  u, v: projected vertices (pixels, FP32 as produced by Eq. 1 in the fixed
// op order); e_i = q_{i+1} - q_i; k_i = s_i / D2 with s_i = perimeter / |e_i| and D2 twice the
// signed area, so that E_i(p) = k_i * cross(e_i, p - q_i) = s_i * lambda_{i+2}(p) is the edge
// function normalised to 1 at the incentre (E_i = phi-ratio of Eq. 3 where edge i is nearest);
// invD = 1 / D2 gives the barycentrics lambda_{i+2} = cross_i * invD; oF the face opacity;
// c the vertex colours; z the camera-space vertex depths; box the pixel box (x0 | x1 << 16,
// y0 | y1 << 16); slot = view * M + face.
enum {
  R_U0 = 0, R_U1, R_U2, R_V0, R_V1, R_V2,
  R_E0X, R_E0Y, R_E1X, R_E1Y, R_E2X, R_E2Y,
  R_K0, R_K1, R_K2, R_INVD,
  R_OF, R_C0 = 17, R_C1 = 20, R_C2 = 23, R_Z0 = 26, R_Z1, R_Z2,
  R_BOXX = 29, R_BOXY = 30, R_SLOT = 31
};
// In shared memory the render kernels overwrite R_BOXY with the per-warp sub-block mask.
#define R_MASK R_BOXY

// Gradient word indices: G_E[i][k] = sum_p dL/dE_i * lambda_k (edge i nearest), G_c[ch][k] =
// sum_p dL/dc_ch * lambda_k, G_z[k] = sum_p dL/dz * lambda_k, G_o = dL/do_F, count = pixels.
// The raster backward accumulates words 0..23; the chain-rule pass then overwrites words
// G_DPOS.. with the face's world-space vertex-position gradients and G_TAU.. with its pose terms.
enum { G_E = 0, G_C = 9, G_Z = 18, G_O = 21, G_CNT = 22, G_DPOS = 0, G_TAU = 24 };

struct TsView {
  float fx, fy, cx, cy;
  int32_t W, H, TX, TY;
  int64_t tile_off, pix_off;
};  // 48 bytes

struct TsViewTable {
  TsView v[TS_MAX_VIEWS];
};

// Image sizes and packing offsets of the views, handed to the loss kernels by value so that a
// loss call needs no earlier call on the workspace.
struct TsImageTable {
  int32_t W[TS_MAX_VIEWS], H[TS_MAX_VIEWS];
  long long pix_off[TS_MAX_VIEWS];
};

// Device-side header at the start of the workspace.
struct TsDevHeader {
  unsigned long long n_pairs;
  unsigned long long n_visible;
  unsigned long long fwd_contrib;
  unsigned long long bwd_contrib;
  unsigned int error_bits;
  unsigned int indexed;
  const float *px, *py, *pz, *cr, *cg, *cb, *op;
  const int32_t* faces;
  long long n_vertices;
  unsigned int tile_counter;  // work counter of the persistent raster launches
  unsigned int n_large;       // tiles listed for the CTA-wide pair sort
  unsigned int pad[12];
};

struct TsPlanImpl {
  uint32_t magic;
  int32_t V;
  int64_t M;
  int64_t cap;
  ts_raster_params prm;
  int64_t n_tiles, n_pix;
  int64_t n_tile_scan_blocks, n_pose_blocks, n_loss_blocks, n_pho_blocks;
  int64_t bin_blocks;       // face blocks per view of the shared-memory tile counts (0: global counts)
  int64_t max_view_tiles;   // the most tiles of one view
  bool normals;  // TS_FLAG_NORMALS
  bool stats;    // TS_FLAG_STATS
  bool min_opacity;  // TS_FLAG_MIN_OPACITY
  bool face_sigma;   // TS_FLAG_FACE_SIGMA
  bool fwd_only;     // TS_FLAG_FORWARD_ONLY: no gradient slots, no lane masks
  // workspace layout (byte offsets)
  size_t o_hdr, o_views, o_poses, o_frec, o_rect, o_zbits, o_count, o_tcnt, o_bsums, o_tlarge, o_tmat, o_tloss, o_keys0, o_keys1,
      o_vals0, o_ranges, o_tfin, o_nlast, o_grad, o_pose, o_loss, o_lmask, o_pho, o_equi, o_aux, o_nloss,
      o_cov, o_ctr, total;
  void* events[2 * TS_N_STAGES];
  int32_t timing;
  TsView views[TS_MAX_VIEWS];
};
static_assert(sizeof(TsPlanImpl) <= TS_PLAN_BYTES, "plan too large");

// Pointers into one workspace.
struct TsWs {
  TsDevHeader* hdr;
  TsView* views;
  ts_pose* poses;
  float4* frec;
  short4* rect;
  uint32_t* zbits;
  uint32_t* count;
  uint32_t* tcnt;    // per tile: pairs (binning)
  uint32_t* tlarge;  // tiles whose pair lists the CTA-wide sort takes
  uint32_t* tmat;    // [tile][face block] pair counts, then their exclusive scan
  float* tloss;      // fused L1 step: per tile, the colour and depth L1 sums
  uint32_t* bsums;
  unsigned long long* keys[2];  // [0]: the sorted pair keys; [1]: the tile segments before their sort
  uint32_t* vals[1];            // the sorted pairs' face ids
  uint2* ranges;
  float* tfin;
  int32_t* nlast;
  float* grad;
  float* pose;
  float* loss;
  float* pho;  // per (view, 32 x 32 tile): L1, SSIM and depth partial sums of the photometric loss
  float* equi;  // per block of 256 faces: partial sums of the equilateral regulariser
  float4* aux;  // per (view, face): camera-space unit normal (TS_FLAG_NORMALS) and the face's sigma
               // (TS_FLAG_FACE_SIGMA) in .w; null without either flag
  float* nloss;  // per (view, 2048-pixel block): partial sums of the normal loss
  uint32_t* cov;  // per (view, face): pixels blended by the forward (TS_FLAG_STATS), else null
  uint32_t* lmask;  // per sorted pair and warp of its tile: the lanes (pixels) that blended the face in the forward
  unsigned long long* ctr;  // [TS_N_CTR][TS_CTR_SLOTS] counters, TS_CTR_STRIDE words apart
};

inline TsWs ts_ws(const TsPlanImpl* p, void* ws) {
  char* b = (char*)ws;
  TsWs w;
  w.hdr = (TsDevHeader*)(b + p->o_hdr);
  w.views = (TsView*)(b + p->o_views);
  w.poses = (ts_pose*)(b + p->o_poses);
  w.frec = (float4*)(b + p->o_frec);
  w.rect = (short4*)(b + p->o_rect);
  w.zbits = (uint32_t*)(b + p->o_zbits);
  w.count = (uint32_t*)(b + p->o_count);
  w.tcnt = (uint32_t*)(b + p->o_tcnt);
  w.tlarge = (uint32_t*)(b + p->o_tlarge);
  w.tmat = (uint32_t*)(b + p->o_tmat);
  w.tloss = (float*)(b + p->o_tloss);
  w.bsums = (uint32_t*)(b + p->o_bsums);
  w.keys[0] = (unsigned long long*)(b + p->o_keys0);
  w.keys[1] = (unsigned long long*)(b + p->o_keys1);
  w.vals[0] = (uint32_t*)(b + p->o_vals0);
  w.ranges = (uint2*)(b + p->o_ranges);
  w.tfin = (float*)(b + p->o_tfin);
  w.nlast = (int32_t*)(b + p->o_nlast);
  w.grad = p->fwd_only ? nullptr : (float*)(b + p->o_grad);
  w.pose = (float*)(b + p->o_pose);
  w.loss = (float*)(b + p->o_loss);
  w.pho = (float*)(b + p->o_pho);
  w.equi = (float*)(b + p->o_equi);
  w.aux = (p->normals || p->face_sigma) ? (float4*)(b + p->o_aux) : nullptr;
  w.nloss = (float*)(b + p->o_nloss);
  w.cov = p->stats ? (uint32_t*)(b + p->o_cov) : nullptr;
  w.lmask = p->fwd_only ? nullptr : (uint32_t*)(b + p->o_lmask);
  w.ctr = (unsigned long long*)(b + p->o_ctr);
  return w;
}

// ------------------------------------------------------------------------------------------
// Launchers (one per translation unit); each returns cudaGetLastError() of its launches.
// ------------------------------------------------------------------------------------------
cudaError_t ts_launch_setup(const TsPlanImpl* p, const TsWs& w, const ts_map* map, const ts_pose* poses,
                            cudaStream_t s);
cudaError_t ts_launch_project(const TsPlanImpl* p, const TsWs& w, const ts_map* map, cudaStream_t s);
cudaError_t ts_launch_bin(const TsPlanImpl* p, const TsWs& w, cudaStream_t s);
cudaError_t ts_launch_face_stats(const TsPlanImpl* p, const TsWs& w, uint32_t* coverage, float* area,
                                 uint32_t* visible, uint32_t* n_visible, cudaStream_t s);
cudaError_t ts_launch_covisibility(const TsPlanImpl* p, const uint32_t* visible, float* iou, cudaStream_t s);
cudaError_t ts_launch_normal_loss(const TsPlanImpl* p, const TsWs& w, const float* normal, const float* tgt,
                                  float weight, float* loss, float* dN, cudaStream_t s);
cudaError_t ts_launch_render_fwd(const TsPlanImpl* p, const TsWs& w, float* color, float* depth, float* alpha,
                                 float* normal, cudaStream_t s);
cudaError_t ts_launch_render_step(const TsPlanImpl* p, const TsWs& w, const float* tgt_color, const float* tgt_depth,
                                  float lambda_dep, float* color, float* depth, float* alpha, float* loss, float* dC,
                                  float* dD, cudaStream_t s);
cudaError_t ts_launch_render_bwd(const TsPlanImpl* p, const TsWs& w, const float* dC, const float* dD,
                                 const float* dA, const float* dN, cudaStream_t s);
cudaError_t ts_launch_project_bwd(const TsPlanImpl* p, const TsWs& w, const ts_map_grad* g, cudaStream_t s);
cudaError_t ts_launch_pose_reduce(const TsPlanImpl* p, const TsWs& w, float* dtau, cudaStream_t s);
inline TsImageTable ts_image_table(const TsPlanImpl* p) {
  TsImageTable t;
  for (int v = 0; v < p->V; ++v) {
    t.W[v] = p->views[v].W;
    t.H[v] = p->views[v].H;
    t.pix_off[v] = p->views[v].pix_off;
  }
  return t;
}
// Raise a kernel's dynamic shared-memory limit on the current device to at least `bytes`.  The
// attribute call runs only when the limit grows (a host call that must not run per launch: the
// launches of concurrent streams would wait on it); a failed call is remembered and reported again.
cudaError_t ts_smem_limit(const void* func, int bytes);
int64_t ts_pho_blocks(const TsView* views, int V);
int64_t ts_equi_blocks(int64_t M);
cudaError_t ts_launch_equilateral(const TsPlanImpl* p, const TsWs& w, const ts_map* map, float weight, float* loss,
                                  const ts_map_grad* grad, cudaStream_t s);
cudaError_t ts_launch_pho_loss(const TsPlanImpl* p, const TsWs& w, const float* color, const float* depth,
                               const float* tc, const float* td, float lambda, float lambda_dep, float* loss,
                               float* dC, float* dD, cudaStream_t s);
cudaError_t ts_launch_l1_loss(const TsPlanImpl* p, const TsWs& w, const float* color, const float* depth,
                              const float* tc, const float* td, float lambda_dep, float* loss, float* dC,
                              float* dD, cudaStream_t s);
cudaError_t ts_launch_pose_apply(const TsPlanImpl* p, ts_pose* poses, const float* step, cudaStream_t s);
cudaError_t ts_launch_pose_adam(const TsPlanImpl* p, ts_pose* poses, const float* dtau, float* state, float lr_rho,
                                float lr_theta, float b1, float b2, float eps, cudaStream_t s);
cudaError_t ts_launch_timeout_probe(const TsWs& w, unsigned long long limit_ns, cudaStream_t s);
int ts_pose_blocks(long long M);                 // blocks of the projection-backward kernel
// Streaming multiprocessors of the current device (queried once per device; 1 if the query fails).
int ts_sm_count();
cudaError_t ts_launch_sum_counters(const TsWs& w, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__

// Add v (summed over the calling warp) to counter c: one add by lane 0 into the slot of the warp.
__device__ __forceinline__ void ts_count_add(unsigned long long* ctr, int c, unsigned v) {
  const unsigned s = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && s) {
    const unsigned slot = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (TS_CTR_SLOTS - 1);
    atomicAdd(ctr + ((size_t)c * TS_CTR_SLOTS + slot) * TS_CTR_STRIDE, (unsigned long long)s);
  }
}

__device__ __forceinline__ int ts_find_view(const TsView* views, int V, long long tile) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Camera-space vertex in the fixed FP32 operation order (Eq. 1, one rounding per operation,
// no FMA): x_c = ((R0 x + R1 y) + R2 z) + t0, likewise y_c, z_c.
__device__ __forceinline__ void ts_rigid_f32(const ts_pose& P, float x, float y, float z, float& xc, float& yc,
                                             float& zc) {
  xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P.R[0], x), __fmul_rn(P.R[1], y)), __fmul_rn(P.R[2], z)), P.t[0]);
  yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P.R[3], x), __fmul_rn(P.R[4], y)), __fmul_rn(P.R[5], z)), P.t[1]);
  zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P.R[6], x), __fmul_rn(P.R[7], y)), __fmul_rn(P.R[8], z)), P.t[2]);
}

// Pinhole projection in the fixed order: u = (fx * (x_c / z_c)) + cx.
__device__ __forceinline__ void ts_pinhole_f32(const TsView& v, float xc, float yc, float zc, float& u, float& w) {
  u = __fadd_rn(__fmul_rn(v.fx, __fdiv_rn(xc, zc)), v.cx);
  w = __fadd_rn(__fmul_rn(v.fy, __fdiv_rn(yc, zc)), v.cy);
}

// a*d - b*c with a single rounding error (Kahan's FMA algorithm).  With exact inputs the
// edge cross products keep full relative accuracy near the edge, where the window's slope
// is largest (sigma = 0.5 gives an infinite derivative at the boundary).
__device__ __forceinline__ float ts_det2(float a, float b, float c, float d) {
  const float w = b * c;
  const float e = fmaf(-b, c, w);
  const float f = fmaf(a, d, -w);
  return f + e;
}

// Per-pixel evaluation of one staged record: barycentric cross products, normalised edge
// functions and their minimum (the ratio phi(p) / phi(s) of Eq. 3).
struct TsPix {
  float cr0, cr1, cr2;  // cross(e_i, p - q_i)
  float m;              // min_i E_i
  int arg;              // argmin
};

__device__ __forceinline__ TsPix ts_eval_edges(const float* r, float px, float py) {
  TsPix o;
  o.cr0 = ts_det2(r[R_E0X], r[R_E0Y], px - r[R_U0], py - r[R_V0]);
  o.cr1 = ts_det2(r[R_E1X], r[R_E1Y], px - r[R_U1], py - r[R_V1]);
  o.cr2 = ts_det2(r[R_E2X], r[R_E2Y], px - r[R_U2], py - r[R_V2]);
  const float e0 = o.cr0 * r[R_K0], e1 = o.cr1 * r[R_K1], e2 = o.cr2 * r[R_K2];
  o.m = e0;
  o.arg = 0;
  if (e1 < o.m) { o.m = e1; o.arg = 1; }
  if (e2 < o.m) { o.m = e2; o.arg = 2; }
  return o;
}

__device__ __forceinline__ float ts_sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float ts_rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Eq. 3 window: I = ratio^sigma for ratio > 0 (hardware square root / exp2-log2, ~1-2 ulp; the
// forward and backward passes share this function, so they see identical values).
__device__ __forceinline__ float ts_window(float m, float sigma) {
  if (sigma == 0.5f) return ts_sqrt_approx(m);
  return exp2f(sigma * __log2f(m));
}

__device__ __forceinline__ uint32_t ts_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ts_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ts_smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void ts_fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}


// 16-byte asynchronous copy global -> shared through the load path (cp.async, cache-global), and
// its group commit and wait (a thread waits for its own copies; a barrier then publishes them).
__device__ __forceinline__ void ts_cp_async16(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ts_smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void ts_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void ts_cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint64_t ts_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after ~limit_ns nanoseconds.  Returns
// false on timeout (the caller latches TS_ERRBIT_TIMEOUT and leaves).
__device__ __forceinline__ bool ts_mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
  const uint32_t a = ts_smem_u32(bar);
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = ts_globaltimer();
    else if ((it & 63) == 0 && ts_globaltimer() - t0 > limit_ns) return false;
  }
}

// Mean-L1 colour + depth loss (Eq. 8 L1 part, Eq. 9), one block of NT * PER pixels of one view
// (W x H pixels at pix_off in the packed images): writes dC = sign(C - Cbar) / (3HW) and
// dD = lambda_dep sign(D - Dbar) / (HW) where Dbar > 0 (else 0), and the block's colour and depth
// L1 sums, reduced in a fixed order, to part[0..1].  Every thread of the block must call it.
template <int NT, int PER>
__device__ __forceinline__ void ts_l1_loss_block(long long HW, long long pix_off, long long base, const float* C,
                                                 const float* D, const float* tC, const float* tD, float lambda_dep,
                                                 float* dC, float* dD, float* part) {
  __shared__ float red[NT / 32][2];
  float lc = 0.f, ld = 0.f;
  if (base < HW) {
    const float ic = 1.0f / (3.0f * (float)HW), id = lambda_dep / (float)HW;
#pragma unroll
    for (int k = 0; k < PER; ++k) {  // a guard, not an exit: all pixels' loads can be in flight
      const long long i = base + (long long)k * NT + threadIdx.x;
      if (i < HW) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const long long o = 3 * pix_off + ch * HW + i;
          const float r = C[o] - tC[o];
          lc += fabsf(r);
          dC[o] = r > 0.f ? ic : (r < 0.f ? -ic : 0.f);
        }
        const long long o = pix_off + i;
        const float t = tD[o];
        const float r = D[o] - t;
        const bool valid = t > 0.f;
        if (valid) ld += fabsf(r);
        dD[o] = valid ? (r > 0.f ? id : (r < 0.f ? -id : 0.f)) : 0.f;
      }
    }
  }
#pragma unroll
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
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) sum += red[w][threadIdx.x];
    part[threadIdx.x] = sum;
  }
}

// The view's loss from its nblk block partials part[2k], part[2k + 1], summed in a fixed order:
// colour sum / (3HW) + lambda_dep * depth sum / (HW).  Every thread of the block must call it.
template <int NT>
__device__ __forceinline__ void ts_l1_loss_final(long long HW, const float* part, int nblk, float lambda_dep,
                                                 float* loss) {
  __shared__ float red[NT][2];
  float a = 0.f, b = 0.f;
  for (int k = threadIdx.x; k < nblk; k += NT) {
    a += part[2 * (long long)k];
    b += part[2 * (long long)k + 1];
  }
  red[threadIdx.x][0] = a;
  red[threadIdx.x][1] = b;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x][0] += red[threadIdx.x + o][0];
      red[threadIdx.x][1] += red[threadIdx.x + o][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    *loss = (float)((double)red[0][0] / (3.0 * (double)HW) + (double)lambda_dep * (double)red[0][1] / (double)HW);
}

#endif  // __CUDACC__
