// ts_api.cu -- the C ABI of libts: plan, workspace layout, argument checks and stage launches.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ts_internal.cuh"

namespace {

const TsPlanImpl* impl(const ts_plan* p) {
  const TsPlanImpl* q = reinterpret_cast<const TsPlanImpl*>(p);
  return (p && q->magic == TS_PLAN_MAGIC) ? q : nullptr;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool valid_tile(int tw, int th) {
  return (tw == 8 || tw == 16 || tw == 32) && (th == 4 || th == 8 || th == 16 || th == 32) && tw * th <= 512 &&
         (tw / 8) * (th / 4) <= 16;
}

ts_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TS_OK : TS_ERR_CUDA; }

bool ws_ok(const TsPlanImpl* p, void* ws, size_t ws_bytes) {
  return ws && ws_bytes >= p->total && (reinterpret_cast<uintptr_t>(ws) & 255) == 0;
}

struct StageTimer {
  const TsPlanImpl* p;
  int stage;
  cudaStream_t s;
  StageTimer(const TsPlanImpl* p_, int st, cudaStream_t s_) : p(p_), stage(st), s(s_) {
    if (p->timing && p->events[2 * stage]) cudaEventRecord((cudaEvent_t)p->events[2 * stage], s);
  }
  ~StageTimer() {
    if (p->timing && p->events[2 * stage + 1]) cudaEventRecord((cudaEvent_t)p->events[2 * stage + 1], s);
  }
};

}  // namespace

cudaError_t ts_smem_limit(const void* func, int bytes) {
  struct Entry {
    int dev;
    const void* func;
    int bytes;   // the largest limit set so far
    bool failed;
  };
  static std::mutex mu;
  static std::vector<Entry> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  Entry* hit = nullptr;
  for (Entry& x : set)
    if (x.dev == dev && x.func == func) hit = &x;
  if (hit && hit->failed) return cudaErrorInvalidValue;
  if (hit && hit->bytes >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (!hit) {
    set.push_back(Entry{dev, func, 0, false});
    hit = &set.back();
  }
  if (e == cudaSuccess) hit->bytes = bytes;
  else hit->failed = true;
  return e;
}

int ts_sm_count() {
  static std::mutex mu;
  static std::vector<std::pair<int, int>> seen;  // (device, SMs)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& x : seen)
    if (x.first == dev) return x.second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  seen.emplace_back(dev, sms);
  return sms;
}

extern "C" {

void ts_default_params(ts_raster_params* o) {
  if (!o) return;
  o->sigma = 0.5f;
  o->alpha_min = 1.0f / 255.0f;
  o->alpha_max = 0.99f;
  o->T_min = 1e-4f;
  o->z_near = 0.01f;
  o->r_min = 0.01f;
  o->bg[0] = o->bg[1] = o->bg[2] = 0.0f;
  o->tile_w = 16;
  o->tile_h = 8;
  o->tris_per_stage = 64;
  o->flags = 0;
}

ts_status ts_plan_init(ts_plan* plan, const ts_camera* cams, int32_t n_views, int64_t n_faces,
                       const ts_raster_params* prm, int64_t pair_capacity) {
  if (!plan || !cams || !prm) return TS_ERR_INVALID_ARG;
  if (n_views < 1 || n_views > TS_MAX_VIEWS || n_faces < 0) return TS_ERR_INVALID_ARG;
  if ((int64_t)n_views * n_faces >= (int64_t)1 << 31) return TS_ERR_INVALID_ARG;
  if (!valid_tile(prm->tile_w, prm->tile_h)) return TS_ERR_INVALID_ARG;
  if (prm->tris_per_stage != 32 && prm->tris_per_stage != 64 && prm->tris_per_stage != 128) return TS_ERR_INVALID_ARG;
  if (!(prm->sigma > 0.0f) || !(prm->alpha_max > 0.0f && prm->alpha_max < 1.0f) || !(prm->alpha_min >= 0.0f) ||
      !(prm->T_min >= 0.0f && prm->T_min < 1.0f) || !(prm->z_near > 0.0f) || !(prm->r_min >= 0.0f) ||
      (prm->flags & ~(TS_FLAG_PERSISTENT | TS_FLAG_NORMALS | TS_FLAG_STATS | TS_FLAG_MIN_OPACITY |
                       TS_FLAG_FACE_SIGMA | TS_FLAG_FORWARD_ONLY)) != 0)
    return TS_ERR_INVALID_ARG;
  if (pair_capacity < 0) return TS_ERR_INVALID_ARG;
  memset(plan, 0, sizeof(ts_plan));
  TsPlanImpl* p = reinterpret_cast<TsPlanImpl*>(plan);
  p->V = n_views;
  p->M = n_faces;
  p->prm = *prm;
  int64_t toff = 0, poff = 0, max_tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    const ts_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return TS_ERR_INVALID_ARG;
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !std::isfinite(c.cx) || !std::isfinite(c.cy)) return TS_ERR_INVALID_ARG;
    TsView& w = p->views[v];
    w.fx = c.fx; w.fy = c.fy; w.cx = c.cx; w.cy = c.cy;
    w.W = c.width; w.H = c.height;
    w.TX = (c.width + prm->tile_w - 1) / prm->tile_w;
    w.TY = (c.height + prm->tile_h - 1) / prm->tile_h;
    w.tile_off = toff;
    w.pix_off = poff;
    toff += (int64_t)w.TX * w.TY;
    poff += (int64_t)c.width * c.height;
    max_tiles = std::max<int64_t>(max_tiles, (int64_t)w.TX * w.TY);
  }
  if (toff >= ((int64_t)1 << 31)) return TS_ERR_INVALID_ARG;
  p->n_tiles = toff;
  p->n_pix = poff;
  const int64_t VM = (int64_t)n_views * n_faces;
  int64_t cap = pair_capacity ? pair_capacity : std::max<int64_t>(1024, 4 * VM);
  if (cap >= ((int64_t)1 << 32) - 4096) return TS_ERR_INVALID_ARG;
  p->cap = cap;
  p->max_view_tiles = max_tiles;
  p->bin_blocks = max_tiles <= TS_BIN_MAX_TILES ? std::max<int64_t>(1, (n_faces + TS_BIN_FACES - 1) / TS_BIN_FACES) : 0;
  {
    const int64_t scanned = p->bin_blocks ? toff * p->bin_blocks : toff;
    p->n_tile_scan_blocks = std::max<int64_t>(1, (scanned + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS);
  }
  p->n_pose_blocks = std::max(1, ts_pose_blocks(n_faces));
  int64_t max_hw = 0;
  for (int v = 0; v < n_views; ++v) max_hw = std::max<int64_t>(max_hw, (int64_t)p->views[v].W * p->views[v].H);
  p->n_loss_blocks = (max_hw + 2047) / 2048;
  p->n_pho_blocks = ts_pho_blocks(p->views, n_views);
  p->normals = (prm->flags & TS_FLAG_NORMALS) != 0;
  p->stats = (prm->flags & TS_FLAG_STATS) != 0;
  p->min_opacity = (prm->flags & TS_FLAG_MIN_OPACITY) != 0;
  p->face_sigma = (prm->flags & TS_FLAG_FACE_SIGMA) != 0;
  p->fwd_only = (prm->flags & TS_FLAG_FORWARD_ONLY) != 0;
  // layout
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  p->o_hdr = take(sizeof(TsDevHeader));
  p->o_views = take(sizeof(TsView) * n_views);
  p->o_poses = take(sizeof(ts_pose) * n_views);
  p->o_frec = take((size_t)VM * TS_REC_WORDS * 4);
  p->o_rect = take((size_t)VM * 8);
  p->o_zbits = take((size_t)VM * 4);
  p->o_count = take((size_t)VM * 4);
  p->o_tcnt = take((size_t)toff * 4);
  p->o_bsums = take((size_t)(p->n_tile_scan_blocks + 1) * 4);
  p->o_tlarge = take((size_t)toff * 4);
  p->o_tmat = take((size_t)toff * (size_t)p->bin_blocks * 4);
  p->o_tloss = take((size_t)toff * 2 * 4);
  p->o_keys0 = take((size_t)cap * 8);
  p->o_keys1 = take((size_t)cap * 8);
  p->o_vals0 = take((size_t)cap * 4);
  p->o_ranges = take((size_t)toff * 8);
  p->o_tfin = take((size_t)poff * 4);
  p->o_nlast = take((size_t)poff * 4);
  p->o_grad = take(p->fwd_only ? 0 : (size_t)VM * TS_GRAD_WORDS * 4);
  p->o_pose = take((size_t)n_views * p->n_pose_blocks * 6 * 4);
  p->o_loss = take((size_t)n_views * p->n_loss_blocks * 2 * 4);
  p->o_lmask = take(p->fwd_only ? 0 : (size_t)cap * (size_t)(prm->tile_w * prm->tile_h / 32) * 4);
  p->o_pho = take((size_t)n_views * p->n_pho_blocks * 3 * 4);
  p->o_equi = take((size_t)ts_equi_blocks(n_faces) * 4);
  p->o_aux = take((p->normals || p->face_sigma) ? (size_t)VM * 16 : 0);
  p->o_nloss = take((size_t)n_views * p->n_loss_blocks * 4);
  p->o_cov = take(p->stats ? (size_t)VM * 4 : 0);
  p->o_ctr = take((size_t)TS_N_CTR * TS_CTR_SLOTS * TS_CTR_STRIDE * 8);
  p->total = o;
  p->magic = TS_PLAN_MAGIC;
  return TS_OK;
}

size_t ts_workspace_size(const ts_plan* plan) {
  const TsPlanImpl* p = impl(plan);
  return p ? p->total : 0;
}

ts_status ts_plan_layout(const ts_plan* plan, int64_t* pix_off, int64_t* tile_off, int32_t* tiles_x,
                         int32_t* tiles_y) {
  const TsPlanImpl* p = impl(plan);
  if (!p) return TS_ERR_INVALID_ARG;
  for (int v = 0; v <= p->V; ++v) {
    if (pix_off) pix_off[v] = v < p->V ? p->views[v].pix_off : p->n_pix;
    if (tile_off) tile_off[v] = v < p->V ? p->views[v].tile_off : p->n_tiles;
    if (v < p->V) {
      if (tiles_x) tiles_x[v] = p->views[v].TX;
      if (tiles_y) tiles_y[v] = p->views[v].TY;
    }
  }
  return TS_OK;
}

ts_status ts_set_stage_events(ts_plan* plan, void* const* events) {
  TsPlanImpl* p = const_cast<TsPlanImpl*>(impl(plan));
  if (!p) return TS_ERR_INVALID_ARG;
  if (!events) {
    p->timing = 0;
    memset(p->events, 0, sizeof(p->events));
    return TS_OK;
  }
  for (int i = 0; i < 2 * TS_N_STAGES; ++i) p->events[i] = events[i];
  p->timing = 1;
  return TS_OK;
}

ts_status ts_workspace_init(const ts_plan* plan, void* ws, size_t ws_bytes, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws_ok(p, ws, ws_bytes)) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the header (counters, error word) and the per-pixel state the backward reads; every other
  // region is written before it is read within a call sequence (the projection clears the
  // gradient slots of the visible faces)
  cudaError_t e = cudaMemsetAsync((char*)ws + p->o_hdr, 0, sizeof(TsDevHeader), s);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)ws + p->o_tfin, 0, p->o_grad - p->o_tfin, s);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)ws + p->o_ctr, 0, (size_t)TS_N_CTR * TS_CTR_SLOTS * TS_CTR_STRIDE * 8, s);
  return cuda_status(e);
}

ts_status ts_project(const ts_plan* plan, const ts_map* map, const ts_pose* poses, void* ws, size_t ws_bytes,
                     ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !map || !poses || !ws_ok(p, ws, ws_bytes)) return TS_ERR_INVALID_ARG;
  if (map->n_faces != p->M) return TS_ERR_INVALID_ARG;
  if (p->M > 0) {
    if (!map->px || !map->py || !map->pz || !map->cr || !map->cg || !map->cb || !map->op) return TS_ERR_INVALID_ARG;
    if (!map->faces && map->n_vertices != 3 * map->n_faces) return TS_ERR_INVALID_ARG;
    if (map->faces && map->n_vertices < 1) return TS_ERR_INVALID_ARG;
    if (p->face_sigma && !map->sigma) return TS_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  TsWs w = ts_ws(p, ws);
  StageTimer t(p, TS_STAGE_PROJECT, s);
  cudaError_t e = ts_launch_setup(p, w, map, poses, s);
  if (e == cudaSuccess) e = ts_launch_project(p, w, map, s);
  return cuda_status(e);
}

ts_status ts_bin(const ts_plan* plan, void* ws, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_BIN, s);
  return cuda_status(ts_launch_bin(p, ts_ws(p, ws), s));
}

ts_status ts_render_fwd_n(const ts_plan* plan, void* ws, float* color, float* depth, float* alpha, float* normal,
                          ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return TS_ERR_INVALID_ARG;
  if (color && ((void*)color == (void*)depth || (void*)color == (void*)alpha)) return TS_ERR_INVALID_ARG;
  if (normal && (!p->normals || (void*)normal == (void*)color || (void*)normal == (void*)depth ||
                 (void*)normal == (void*)alpha))
    return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_FWD, s);
  return cuda_status(ts_launch_render_fwd(p, ts_ws(p, ws), color, depth, alpha, normal, s));
}

ts_status ts_render_fwd(const ts_plan* plan, void* ws, float* color, float* depth, float* alpha, ts_stream stream) {
  return ts_render_fwd_n(plan, ws, color, depth, alpha, nullptr, stream);
}

ts_status ts_render_bwd(const ts_plan* plan, void* ws, const float* dC, const float* dD, const float* dA,
                        const ts_map_grad* grad, ts_stream stream) {
  return ts_render_bwd_n(plan, ws, dC, dD, dA, nullptr, grad, stream);
}

ts_status ts_render_bwd_n(const ts_plan* plan, void* ws, const float* dC, const float* dD, const float* dA,
                          const float* dN, const ts_map_grad* grad, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) || !dC || p->fwd_only) return TS_ERR_INVALID_ARG;
  if (dN && !p->normals) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TsWs w = ts_ws(p, ws);
  cudaError_t e;
  {
    StageTimer t(p, TS_STAGE_BWD_RASTER, s);
    e = ts_launch_render_bwd(p, w, dC, dD, dA, dN, s);
  }
  if (e != cudaSuccess) return TS_ERR_CUDA;
  StageTimer t(p, TS_STAGE_BWD_PROJECT, s);
  ts_map_grad none;
  memset(&none, 0, sizeof(none));
  return cuda_status(ts_launch_project_bwd(p, w, grad ? grad : &none, s));
}

ts_status ts_render_step_l1(const ts_plan* plan, void* ws, const float* tgt_color, const float* tgt_depth,
                           float lambda_dep, float* color, float* depth, float* alpha, float* loss, float* dC,
                           float* dD, const ts_map_grad* grad, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) || !tgt_color || !tgt_depth || !color || !loss ||
      p->fwd_only)
    return TS_ERR_INVALID_ARG;
  if (!(lambda_dep >= 0.0f) || !std::isfinite(lambda_dep)) return TS_ERR_INVALID_ARG;
  if (p->normals || p->face_sigma) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TsWs w = ts_ws(p, ws);
  cudaError_t e;
  {
    StageTimer t(p, TS_STAGE_FWD, s);
    e = ts_launch_render_step(p, w, tgt_color, tgt_depth, lambda_dep, color, depth, alpha, loss, dC, dD, s);
  }
  if (e != cudaSuccess) return TS_ERR_CUDA;
  StageTimer t(p, TS_STAGE_BWD_PROJECT, s);
  ts_map_grad none;
  memset(&none, 0, sizeof(none));
  return cuda_status(ts_launch_project_bwd(p, w, grad ? grad : &none, s));
}

ts_status ts_pose_grad(const ts_plan* plan, void* ws, float* dtau, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || !dtau || (reinterpret_cast<uintptr_t>(ws) & 255) || p->fwd_only) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_POSE, s);
  return cuda_status(ts_launch_pose_reduce(p, ts_ws(p, ws), dtau, s));
}

ts_status ts_l1_loss(const ts_plan* plan, void* ws, const float* color, const float* depth, const float* tgt_color,
                     const float* tgt_depth, float lambda_dep, float* loss, float* dC, float* dD, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || !color || !depth || !tgt_color || !tgt_depth || !loss || !dC || !dD) return TS_ERR_INVALID_ARG;
  if (!(lambda_dep >= 0.0f) || !std::isfinite(lambda_dep)) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_LOSS, s);
  return cuda_status(ts_launch_l1_loss(p, ts_ws(p, ws), color, depth, tgt_color, tgt_depth, lambda_dep, loss, dC, dD, s));
}

ts_status ts_pho_loss(const ts_plan* plan, void* ws, const float* color, const float* depth, const float* tgt_color,
                      const float* tgt_depth, float lambda_ssim, float lambda_dep, float* loss, float* dC, float* dD,
                      ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || !color || !depth || !tgt_color || !tgt_depth || !loss || !dC || !dD) return TS_ERR_INVALID_ARG;
  if (!(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f) || !(lambda_dep >= 0.0f) || !std::isfinite(lambda_dep))
    return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_LOSS, s);
  return cuda_status(ts_launch_pho_loss(p, ts_ws(p, ws), color, depth, tgt_color, tgt_depth, lambda_ssim, lambda_dep,
                                        loss, dC, dD, s));
}

ts_status ts_face_stats(const ts_plan* plan, void* ws, uint32_t* coverage, float* area, uint32_t* visible,
                        uint32_t* n_visible, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return TS_ERR_INVALID_ARG;
  if ((coverage || visible || n_visible) && !p->stats) return TS_ERR_INVALID_ARG;
  return cuda_status(ts_launch_face_stats(p, ts_ws(p, ws), coverage, area, visible, n_visible, (cudaStream_t)stream));
}

ts_status ts_covisibility(const ts_plan* plan, const uint32_t* visible, float* iou, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !visible || !iou) return TS_ERR_INVALID_ARG;
  return cuda_status(ts_launch_covisibility(p, visible, iou, (cudaStream_t)stream));
}

ts_status ts_normal_loss(const ts_plan* plan, void* ws, const float* normal, const float* tgt_normal, float weight,
                         float* loss, float* dN, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || !normal || !tgt_normal || !loss || !dN || !std::isfinite(weight)) return TS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StageTimer t(p, TS_STAGE_LOSS, s);
  return cuda_status(ts_launch_normal_loss(p, ts_ws(p, ws), normal, tgt_normal, weight, loss, dN, s));
}

ts_status ts_equilateral(const ts_plan* plan, const ts_map* map, void* ws, size_t ws_bytes, float weight, float* loss,
                         const ts_map_grad* grad, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !map || !loss || !ws_ok(p, ws, ws_bytes) || !std::isfinite(weight)) return TS_ERR_INVALID_ARG;
  if (map->n_faces != p->M) return TS_ERR_INVALID_ARG;
  if (p->M > 0) {
    if (!map->px || !map->py || !map->pz) return TS_ERR_INVALID_ARG;
    if (!map->faces && map->n_vertices != 3 * map->n_faces) return TS_ERR_INVALID_ARG;
    if (map->faces && map->n_vertices < 1) return TS_ERR_INVALID_ARG;
  }
  return cuda_status(ts_launch_equilateral(p, ts_ws(p, ws), map, weight, loss, grad, (cudaStream_t)stream));
}

ts_status ts_pose_apply(const ts_plan* plan, ts_pose* poses, const float* step, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !poses || !step) return TS_ERR_INVALID_ARG;
  return cuda_status(ts_launch_pose_apply(p, poses, step, (cudaStream_t)stream));
}

ts_status ts_pose_adam(const ts_plan* plan, ts_pose* poses, const float* dtau, float* state, float lr_rho,
                       float lr_theta, float beta1, float beta2, float eps, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !poses || !dtau || !state) return TS_ERR_INVALID_ARG;
  if (!(lr_rho >= 0.f) || !(lr_theta >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return TS_ERR_INVALID_ARG;
  return cuda_status(ts_launch_pose_adam(p, poses, dtau, state, lr_rho, lr_theta, beta1, beta2, eps,
                                         (cudaStream_t)stream));
}

ts_status ts_sync_status(const ts_plan* plan, void* ws, ts_stream stream, ts_counters* out) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws) return TS_ERR_INVALID_ARG;
  TsDevHeader h;
  cudaError_t e = ts_launch_sum_counters(ts_ws(p, ws), (cudaStream_t)stream);  // the slots into the header
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, (char*)ws + p->o_hdr, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return TS_ERR_CUDA;
  if (out) {
    out->n_pairs = h.n_pairs;
    out->pair_capacity = (uint64_t)p->cap;
    out->n_visible = h.n_visible;
    out->fwd_contrib = h.fwd_contrib;
    out->bwd_contrib = h.bwd_contrib;
    out->error_bits = h.error_bits;
    out->reserved = 0;
  }
  if (h.error_bits & TS_ERRBIT_BOUNDS) return TS_ERR_CUDA;
  if (h.error_bits & TS_ERRBIT_TIMEOUT) return TS_ERR_TIMEOUT;
  if (h.error_bits & TS_ERRBIT_CAPACITY) return TS_ERR_CAPACITY;
  return TS_OK;
}

ts_status ts_debug_copy(const ts_plan* plan, void* ws, int32_t what, void* dst, size_t bytes, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || !dst) return TS_ERR_INVALID_ARG;
  const int64_t VM = (int64_t)p->V * p->M;
  size_t off, avail;
  switch (what) {
    case 0: off = p->o_keys0; avail = (size_t)p->cap * 8; break;
    case 1: off = p->o_vals0; avail = (size_t)p->cap * 4; break;
    case 2: off = p->o_ranges; avail = (size_t)p->n_tiles * 8; break;
    case 3: off = p->o_rect; avail = (size_t)VM * 8; break;
    case 4: off = p->o_zbits; avail = (size_t)VM * 4; break;
    case 5: off = p->o_count; avail = (size_t)VM * 4; break;
    case 6: off = p->o_tfin; avail = (size_t)p->n_pix * 4; break;
    case 7: off = p->o_nlast; avail = (size_t)p->n_pix * 4; break;
    case 8: off = p->o_frec; avail = (size_t)VM * TS_REC_WORDS * 4; break;
    default: return TS_ERR_INVALID_ARG;
  }
  if (bytes > avail) return TS_ERR_INVALID_ARG;
  if (bytes == 0) return TS_OK;
  return cuda_status(cudaMemcpyAsync(dst, (char*)ws + off, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
}

ts_status ts_debug_timeout_probe(const ts_plan* plan, void* ws, uint32_t limit_us, ts_stream stream) {
  const TsPlanImpl* p = impl(plan);
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) || limit_us == 0 || limit_us > 5000000u)
    return TS_ERR_INVALID_ARG;
  return cuda_status(ts_launch_timeout_probe(ts_ws(p, ws), (unsigned long long)limit_us * 1000ull, (cudaStream_t)stream));
}

const char* ts_status_string(ts_status s) {
  switch (s) {
    case TS_OK: return "ok";
    case TS_ERR_INVALID_ARG: return "invalid argument";
    case TS_ERR_CUDA: return "CUDA error";
    case TS_ERR_CAPACITY: return "pair capacity exceeded";
    case TS_ERR_TIMEOUT: return "device wait timed out";
    case TS_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

}  // extern "C"
