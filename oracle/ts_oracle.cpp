// ts_oracle.cpp -- CPU oracle for the differentiable triangle-splatting rasterizer.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA path is checked against.  Only the test-suite, the package smoke check
// and the benchmark's CPU-baseline leg may load it; the product path never
// calls it and shares no code, header, table or helper with it.
//
// What it computes (Triangle Splatting SLAM, Sec. 3.1-3.3):
//   * Eq. 1   projection v_I = pi(T_CW v_W) of every face vertex;
//   * Eq. 2   2D signed distance phi(p) = max_i (n_i . p + d_i) with outward
//             unit edge normals n_i;
//   * Eq. 3   window I(p) = ReLU(phi(p) / phi(s))^sigma, s the incentre;
//   * Sec 3.1 face colour by barycentric interpolation of vertex colours and
//             face opacity o_F = (o_i + o_j + o_k) / 3;
//   * Eq. 4   front-to-back alpha compositing over the depth-sorted faces,
//             with depth and opacity images composited the same way;
//   * the adjoint of all of the above w.r.t. vertex positions, colours,
//     opacities, and the pose through the left perturbation Exp(tau) o T
//     (Eq. 5-7, tau = (rho, theta), translation first);
//   * Eq. 8-10 the tracking loss: L1 and D-SSIM photometric terms and the L1
//     depth term, with their gradients w.r.t. the rendered images;
//   * Eq. 12 the rendered normal map and the normal loss, with the normal's
//     gradient folded into the adjoint above;
//   * Eq. 14 the equilateral regulariser of the mapping loss and its gradient
//     w.r.t. vertex positions.
//
// How: the forward pass walks each pixel's depth-sorted list literally.  The
// backward pass stores every contribution of a pixel front to back, forms the
// suffix sums from the back (no division by 1 - alpha), and differentiates
// each (pixel, face) term with forward-mode dual numbers over the face's 21
// vertex parameters and the view's 6 pose parameters.  All blending runs in
// double precision.
//
// Readings of the paper that this file fixes (the paper is silent on them):
//   R1 edge i runs from vertex i to vertex i+1; its unit normal points away
//      from the opposite vertex (either winding works; no back-face culling);
//   R3 the exponent applies after the ReLU; sigma = 0.5 (Table S5);
//   R4 pixel (x, y) samples the point (x + 0.5, y + 0.5);
//   R5 colour and camera-space depth are interpolated with screen-space
//      barycentrics of the projected vertices;
//   R6 depth order: key z = ((z0 + z1) + z2) / 3 of camera-space vertex depth,
//      ascending, ties by ascending face id;
//   R7 D = sum z(p) alpha_n T_n (unnormalised), A = sum alpha_n T_n;
//   R8 background colour bg is added with weight T_final; depth has none;
//   R9 alpha = min(alpha_max, o_F I); contributions with alpha < alpha_min are
//      skipped; a pixel stops before the face that would take T below T_min;
//   R10 a face is culled if a vertex has z <= z_near, if its inradius is below
//      r_min, if o_F < alpha_min, or if its pixel box is empty; the pixel box is
//      ceil(min - 0.5) .. floor(max - 0.5) clamped to the image;
//   R11 loss = mean |C - Cbar| over 3HW + lambda_dep * sum_{Dbar>0} |D - Dbar| / HW
//      per view, summed over views; sign(0) = 0;
//   R16 the D-SSIM term of Eq. 8 is 1 - SSIM, SSIM the mean over the 3HW channel pixels of the
//      per-pixel structural similarity (Wang et al. 2004) with the common defaults: 11 x 11
//      Gaussian window, sigma 1.5, normalised to sum 1; C1 = 0.01^2, C2 = 0.03^2 (colours in
//      [0, 1]);
//   R17 the window sums see zeros outside the image ("same"-size output, zero padding), and
//      every image pixel carries one SSIM value;
//   R18 E_pho weights the same mean L1 colour term as R11 by (1 - lambda), lambda = 0.2
//      (Table S5); the depth term is that of R11;
//   R19 Eq. 14 averages over all M faces; a face with a zero-length edge has no defined angle
//      and adds 0 (no gradient);
//   R20 the rendered normal map of Eq. 12 is composited like colour, N = sum alpha_n T_n n_F,
//      with the face's unit normal n_F in camera space and no background term;
//   R21 n_F is turned towards the camera: the normalised (v1 - v0) x (v2 - v0) of the
//      camera-space vertices, negated when it has a positive dot product with v0 + v1 + v2
//      (triangles are two-sided, so the winding carries no orientation);
//   R22 Eq. 12 sums 1 - N . Nbar over the pixels with a sensor normal (Nbar != 0), divided by
//      HW like the depth term of R11; N is used as rendered (not renormalised);
//   R23 Sec. 3.4's map statistics: a face's pixel coverage in a view counts the pixels at which
//      it was blended (its alpha passed alpha_min before termination); its projected area is
//      that of the projected triangle; a face is visible in a view when its coverage is > 0;
//   R24 the Mesh Splatting variant (Sec. 3.1 contrasts it) takes o_F = min of the three vertex
//      opacities; its derivative goes to the first vertex (in face order) attaining the minimum;
//   R25 the learnable-sigma variant (Triangle Splatting, which Eq. 3 follows) gives each face its
//      own exponent sigma_F in I = ReLU(phi / phi(s))^sigma_F, differentiated like the other
//      face parameters; dI/dsigma_F = I ln(phi / phi(s));
//   R14 in FP32 mode the projection follows one fixed operation order with
//      no fused multiply-add (build with -ffp-contract=off), so that culling,
//      pixel boxes, tiles and depth keys are bit-identical to any other
//      implementation that follows the same order.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
// Optional -DORACLE_MUTANT=k plants the k-th deliberate mistake (tests only).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

extern "C" {

typedef struct {
  double sigma, alpha_min, alpha_max, T_min, z_near, r_min;
  double bg[3];
  int32_t tile_w, tile_h;
  int32_t fp64;       // 0: projection in FP32 with the fixed op order (R14); 1: FP64 throughout
  int32_t n_threads;  // OpenMP threads (<= 0: library default)
  int32_t min_opacity;  // 1: o_F = min of the vertex opacities (Mesh Splatting variant, R24)
} or_params;

typedef struct {
  const double* pos;     // [N][3] world positions
  const double* col;     // [N][3] vertex colours
  const double* opa;     // [N]    vertex opacities
  const int32_t* faces;  // [M][3] or NULL: face m = vertices 3m, 3m+1, 3m+2
  int64_t n_vertices, n_faces;
  const double* cams;    // [V][6] fx, fy, cx, cy, W, H
  const double* poses;   // [V][12] row-major R, then t: v_C = R v_W + t
  int32_t n_views;
  const double* sigma_face;  // [M] per-face window exponent (learnable-sigma variant, R25), or NULL
} or_scene;

}  // extern "C"

namespace {

// ---------------------------------------------------------------- dual numbers
constexpr int NT = 28;  // 3 vertices x (x, y, z, r, g, b, o) + 6 pose (rho, theta) + the face's sigma

struct Dual {
  double v;
  double d[NT];
  Dual() : v(0) { std::memset(d, 0, sizeof(d)); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }  // NOLINT: implicit constant
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < NT; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  const double ib = 1.0 / b.v;
  for (int i = 0; i < NT; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
inline Dual sqrt_(const Dual& a) { Dual r(std::sqrt(a.v)); const double k = 0.5 / r.v; for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * k; return r; }
inline Dual pow_(const Dual& a, double e) {
  Dual r(std::pow(a.v, e));
  const double k = e * std::pow(a.v, e - 1.0);
  for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * k;
  return r;
}
// a^e with a dual exponent: d(a^e) = e a^(e-1) da + a^e ln(a) de
inline Dual pow_(const Dual& a, const Dual& e) {
  Dual r(std::pow(a.v, e.v));
  const double ka = e.v * std::pow(a.v, e.v - 1.0);
#if ORACLE_MUTANT == 22
  const double ke = r.v;  // the logarithm dropped
#else
  const double ke = r.v * std::log(a.v);
#endif
  for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * ka + e.d[i] * ke;
  return r;
}
inline double val(const Dual& a) { return a.v; }
inline double sqrt_(double a) { return std::sqrt(a); }
inline double pow_(double a, double e) { return std::pow(a, e); }
inline double val(double a) { return a; }
template <class S> inline S max_(const S& a, const S& b) { return val(a) >= val(b) ? a : b; }
template <class S> inline S min_(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }

// ---------------------------------------------------------------- scene access
struct View {
  double fx, fy, cx, cy;
  int W, H, TX, TY;
  int64_t tile_off, pix_off;
};

struct Ctx {
  const or_scene* sc;
  or_params p;
  std::vector<View> views;
  int64_t n_tiles = 0, n_pix = 0;
};

Ctx make_ctx(const or_scene* sc, const or_params* p) {
  Ctx c;
  c.sc = sc;
  c.p = *p;
  int64_t toff = 0, poff = 0;
  for (int v = 0; v < sc->n_views; ++v) {
    const double* cm = sc->cams + 6 * v;
    View w;
    w.fx = cm[0]; w.fy = cm[1]; w.cx = cm[2]; w.cy = cm[3];
    w.W = (int)cm[4]; w.H = (int)cm[5];
    w.TX = (w.W + p->tile_w - 1) / p->tile_w;
    w.TY = (w.H + p->tile_h - 1) / p->tile_h;
    w.tile_off = toff; w.pix_off = poff;
    toff += (int64_t)w.TX * w.TY;
    poff += (int64_t)w.W * w.H;
    c.views.push_back(w);
  }
  c.n_tiles = toff;
  c.n_pix = poff;
  return c;
}

inline int64_t vidx(const or_scene* sc, int64_t m, int k) {
  return sc->faces ? (int64_t)sc->faces[3 * m + k] : 3 * m + k;
}

// ---------------------------------------------------------------- Eq. 1 projection (+ culling, R10, R14)
struct Proj {
  bool visible = false;
  int x0, x1, y0, y1;        // pixel box (inclusive)
  int tx0, tx1, ty0, ty1;    // tile box (inclusive)
  uint32_t zbits = 0;        // depth key bits (R6)
  double u[3], v[3], z[3];   // projected vertices and camera-space depth
  double oF;                 // face opacity (Sec. 3.1)
};

// FP32 projection in the fixed operation order (R14).  Every line is one
// rounded IEEE single operation; the build disables contraction into FMA.
Proj project_f32(const Ctx& c, int view, int64_t m) {
  const or_scene* sc = c.sc;
  const View& w = c.views[view];
  const double* P = sc->poses + 12 * view;
  float R[9], t[3];
  for (int i = 0; i < 9; ++i) R[i] = (float)P[i];
  for (int i = 0; i < 3; ++i) t[i] = (float)P[9 + i];
#if ORACLE_MUTANT == 3
  { float Rt[9]; for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Rt[3 * a + b] = R[3 * b + a]; std::memcpy(R, Rt, sizeof(R)); }
#endif
  const float fx = (float)w.fx, fy = (float)w.fy, cx = (float)w.cx, cy = (float)w.cy;
  Proj pr;
  float u[3], v[3], z[3], o[3];
  for (int k = 0; k < 3; ++k) {
    const int64_t vi = vidx(sc, m, k);
    const float x = (float)sc->pos[3 * vi], y = (float)sc->pos[3 * vi + 1], zz = (float)sc->pos[3 * vi + 2];
    float a, b;
    a = R[0] * x; b = R[1] * y; float xc = a + b; a = R[2] * zz; xc = xc + a; xc = xc + t[0];
    a = R[3] * x; b = R[4] * y; float yc = a + b; a = R[5] * zz; yc = yc + a; yc = yc + t[1];
    a = R[6] * x; b = R[7] * y; float zc = a + b; a = R[8] * zz; zc = zc + a; zc = zc + t[2];
    if (!(zc > (float)c.p.z_near)) return pr;  // culled (also catches NaN)
    float q = xc / zc; q = fx * q; u[k] = q + cx;
    q = yc / zc; q = fy * q; v[k] = q + cy;
    z[k] = zc;
    o[k] = (float)sc->opa[vi];
  }
  // inradius r = |2A| / perimeter
  float du1 = u[1] - u[0], dv1 = v[1] - v[0], du2 = u[2] - u[0], dv2 = v[2] - v[0];
  float a1 = du1 * dv2, a2 = du2 * dv1;
  float area2 = a1 - a2;
  float len[3];
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3;
    float ex = u[j] - u[i], ey = v[j] - v[i];
    float s1 = ex * ex, s2 = ey * ey;
    len[i] = std::sqrt(s1 + s2);
  }
  float per = len[0] + len[1];
  per = per + len[2];
  float r = std::fabs(area2) / per;
  if (!(r >= (float)c.p.r_min)) return pr;
  float oF;
  if (c.p.min_opacity) {
    oF = std::min(o[0], std::min(o[1], o[2]));
  } else {
    oF = o[0] + o[1];
    oF = oF + o[2];
    oF = oF / 3.0f;
  }
  if (oF < (float)c.p.alpha_min) return pr;
  float umin = std::min(u[0], std::min(u[1], u[2])), umax = std::max(u[0], std::max(u[1], u[2]));
  float vmin = std::min(v[0], std::min(v[1], v[2])), vmax = std::max(v[0], std::max(v[1], v[2]));
  float fx0 = std::ceil(umin - 0.5f), fx1 = std::floor(umax - 0.5f);
  float fy0 = std::ceil(vmin - 0.5f), fy1 = std::floor(vmax - 0.5f);
  if (!(fx0 <= fx1) || fx1 < 0.0f || fx0 > (float)(w.W - 1)) return pr;
  if (!(fy0 <= fy1) || fy1 < 0.0f || fy0 > (float)(w.H - 1)) return pr;
  pr.x0 = fx0 < 0.0f ? 0 : (int)fx0;
  pr.x1 = fx1 > (float)(w.W - 1) ? w.W - 1 : (int)fx1;
  pr.y0 = fy0 < 0.0f ? 0 : (int)fy0;
  pr.y1 = fy1 > (float)(w.H - 1) ? w.H - 1 : (int)fy1;
  float zk = z[0] + z[1];
  zk = zk + z[2];
  zk = zk / 3.0f;
  std::memcpy(&pr.zbits, &zk, 4);
  for (int k = 0; k < 3; ++k) { pr.u[k] = u[k]; pr.v[k] = v[k]; pr.z[k] = z[k]; }
  pr.oF = oF;
  pr.visible = true;
  return pr;
}

// The same projection and culling in double precision (finite-difference mode).
Proj project_f64(const Ctx& c, int view, int64_t m) {
  const or_scene* sc = c.sc;
  const View& w = c.views[view];
  const double* P = sc->poses + 12 * view;
  Proj pr;
  double o[3];
  for (int k = 0; k < 3; ++k) {
    const int64_t vi = vidx(sc, m, k);
    const double* X = sc->pos + 3 * vi;
    double xc = P[0] * X[0] + P[1] * X[1] + P[2] * X[2] + P[9];
    double yc = P[3] * X[0] + P[4] * X[1] + P[5] * X[2] + P[10];
    double zc = P[6] * X[0] + P[7] * X[1] + P[8] * X[2] + P[11];
    if (!(zc > c.p.z_near)) return pr;
    pr.u[k] = w.fx * (xc / zc) + w.cx;
    pr.v[k] = w.fy * (yc / zc) + w.cy;
    pr.z[k] = zc;
    o[k] = sc->opa[vi];
  }
  double area2 = (pr.u[1] - pr.u[0]) * (pr.v[2] - pr.v[0]) - (pr.u[2] - pr.u[0]) * (pr.v[1] - pr.v[0]);
  double per = 0;
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3;
    per += std::hypot(pr.u[j] - pr.u[i], pr.v[j] - pr.v[i]);
  }
  if (!(std::fabs(area2) / per >= c.p.r_min)) return pr;
  double oF = c.p.min_opacity ? std::min(o[0], std::min(o[1], o[2])) : (o[0] + o[1] + o[2]) / 3.0;
  if (oF < c.p.alpha_min) return pr;
  double umin = std::min({pr.u[0], pr.u[1], pr.u[2]}), umax = std::max({pr.u[0], pr.u[1], pr.u[2]});
  double vmin = std::min({pr.v[0], pr.v[1], pr.v[2]}), vmax = std::max({pr.v[0], pr.v[1], pr.v[2]});
  double fx0 = std::ceil(umin - 0.5), fx1 = std::floor(umax - 0.5);
  double fy0 = std::ceil(vmin - 0.5), fy1 = std::floor(vmax - 0.5);
  if (!(fx0 <= fx1) || fx1 < 0 || fx0 > w.W - 1) return pr;
  if (!(fy0 <= fy1) || fy1 < 0 || fy0 > w.H - 1) return pr;
  pr.x0 = fx0 < 0 ? 0 : (int)fx0;
  pr.x1 = fx1 > w.W - 1 ? w.W - 1 : (int)fx1;
  pr.y0 = fy0 < 0 ? 0 : (int)fy0;
  pr.y1 = fy1 > w.H - 1 ? w.H - 1 : (int)fy1;
  float zk = (float)((pr.z[0] + pr.z[1] + pr.z[2]) / 3.0);
  std::memcpy(&pr.zbits, &zk, 4);
  pr.oF = oF;
  pr.visible = true;
  return pr;
}

Proj project(const Ctx& c, int view, int64_t m) {
  Proj pr = c.p.fp64 ? project_f64(c, view, m) : project_f32(c, view, m);
  if (pr.visible) {
    const View& w = c.views[view];
    pr.tx0 = pr.x0 / c.p.tile_w;
    pr.tx1 = pr.x1 / c.p.tile_w;
    pr.ty0 = pr.y0 / c.p.tile_h;
    pr.ty1 = pr.y1 / c.p.tile_h;
#if ORACLE_MUTANT == 11
    pr.tx1 = std::min(pr.tx1 + 1, w.TX - 1);
#endif
    (void)w;
  }
  return pr;
}

// ---------------------------------------------------------------- Eq. 2-3 window and Sec. 3.1 interpolation
// Evaluates, at pixel sample point (px, py), the window I of the 2D triangle
// (qx, qy) and its screen-space barycentrics lam.  Returns I; ratio gets
// phi(p) / phi(s).
template <class S>
S window_and_bary(const S qx[3], const S qy[3], double px, double py, const S& sigma, S lam[3], double* ratio_out) {
  S nx[3], ny[3], d[3], len[3];
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    S ex = qx[j] - qx[i], ey = qy[j] - qy[i];
    len[i] = sqrt_(ex * ex + ey * ey);
    nx[i] = ey / len[i];
    ny[i] = -ex / len[i];
    // outward: the opposite vertex lies on the negative side (R1)
#if ORACLE_MUTANT == 2
    if (val(nx[i] * (qx[k] - qx[i]) + ny[i] * (qy[k] - qy[i])) < 0) { nx[i] = -nx[i]; ny[i] = -ny[i]; }
#else
    if (val(nx[i] * (qx[k] - qx[i]) + ny[i] * (qy[k] - qy[i])) > 0) { nx[i] = -nx[i]; ny[i] = -ny[i]; }
#endif
    d[i] = -(nx[i] * qx[i] + ny[i] * qy[i]);
  }
  // Eq. 2 at p
  S phi_p = nx[0] * S(px) + ny[0] * S(py) + d[0];
  for (int i = 1; i < 3; ++i) phi_p = max_(phi_p, nx[i] * S(px) + ny[i] * S(py) + d[i]);
  // incentre: vertices weighted by the length of the opposite side
  S per = len[0] + len[1] + len[2];
  S sx = (len[1] * qx[0] + len[2] * qx[1] + len[0] * qx[2]) / per;
  S sy = (len[1] * qy[0] + len[2] * qy[1] + len[0] * qy[2]) / per;
  S phi_s = nx[0] * sx + ny[0] * sy + d[0];
  for (int i = 1; i < 3; ++i) phi_s = max_(phi_s, nx[i] * sx + ny[i] * sy + d[i]);
  S ratio = phi_p / phi_s;
  *ratio_out = val(ratio);
  // Eq. 3: ReLU first, then the exponent (R3)
  S I = val(ratio) > 0 ? pow_(ratio, sigma) : S(0.0);
  // screen-space barycentrics (R5): signed sub-areas over the full signed area
  S area = (qx[1] - qx[0]) * (qy[2] - qy[0]) - (qx[2] - qx[0]) * (qy[1] - qy[0]);
  S PX(px), PY(py);
  lam[0] = ((qx[1] - PX) * (qy[2] - PY) - (qx[2] - PX) * (qy[1] - PY)) / area;
  lam[1] = ((qx[2] - PX) * (qy[0] - PY) - (qx[0] - PX) * (qy[2] - PY)) / area;
  lam[2] = ((qx[0] - PX) * (qy[1] - PY) - (qx[1] - PX) * (qy[0] - PY)) / area;
  return I;
}

inline double face_opacity(double o0, double o1, double o2, bool min_variant) {
#if ORACLE_MUTANT == 1
  min_variant = true;
#endif
  return min_variant ? std::min(o0, std::min(o1, o2)) : (o0 + o1 + o2) / 3.0;
}

// Per (pixel, face) quantities used by the compositing.
struct Term {
  double alpha, I, ratio, col[3], z, nrm[3];
  bool clamped;
};

// Unit normal of face m in camera space, turned towards the camera (R20, R21): the normalised
// cross product (v1 - v0) x (v2 - v0) of the camera-space vertices, negated when it points away
// from the camera (positive dot product with the vertex sum).  S is double or Dual; vc [3][3].
template <class S>
void face_normal(const S vc[3][3], S n[3]) {
  S e1[3], e2[3];
  for (int r = 0; r < 3; ++r) { e1[r] = vc[1][r] - vc[0][r]; e2[r] = vc[2][r] - vc[0][r]; }
  S u[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const S len = sqrt_(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double facing = 0;
  for (int r = 0; r < 3; ++r) facing += val(u[r]) * (val(vc[0][r]) + val(vc[1][r]) + val(vc[2][r]));
#if ORACLE_MUTANT == 17
  facing = -1.0;  // never turned: the winding decides
#endif
  const S sgn(facing > 0 ? -1.0 : 1.0);
  for (int r = 0; r < 3; ++r) n[r] = sgn * u[r] / len;
}

Term eval_term(const Ctx& c, int view, int64_t m, const Proj& pr, double px, double py) {
  const or_scene* sc = c.sc;
  double lam[3], ratio;
  const double sig = sc->sigma_face ? sc->sigma_face[m] : c.p.sigma;
  double I = window_and_bary<double>(pr.u, pr.v, px, py, sig, lam, &ratio);
  Term t;
  double o[3];
  for (int k = 0; k < 3; ++k) o[k] = sc->opa[vidx(sc, m, k)];
  const double oF = face_opacity(o[0], o[1], o[2], c.p.min_opacity != 0);
  t.I = I;
  t.ratio = ratio;
#if ORACLE_MUTANT == 23
  t.clamped = false;  // no alpha_max clamp
#else
  t.clamped = oF * I > c.p.alpha_max;
#endif
  t.alpha = t.clamped ? c.p.alpha_max : oF * I;
  for (int ch = 0; ch < 3; ++ch) {
    t.col[ch] = 0;
    for (int k = 0; k < 3; ++k) t.col[ch] += lam[k] * sc->col[3 * vidx(sc, m, k) + ch];
  }
#if ORACLE_MUTANT == 7
  t.z = lam[1] * pr.z[0] + lam[2] * pr.z[1] + lam[0] * pr.z[2];
#else
  t.z = lam[0] * pr.z[0] + lam[1] * pr.z[1] + lam[2] * pr.z[2];
#endif
  const double* P = sc->poses + 12 * view;
  double vc[3][3];
  for (int k = 0; k < 3; ++k) {
    const double* X = sc->pos + 3 * vidx(sc, m, k);
    for (int r = 0; r < 3; ++r)
#if ORACLE_MUTANT == 18
      vc[k][r] = X[r];  // world instead of camera space
#else
      vc[k][r] = P[3 * r] * X[0] + P[3 * r + 1] * X[1] + P[3 * r + 2] * X[2] + P[9 + r];
#endif
  }
  face_normal<double>(vc, t.nrm);
  return t;
}

// ---------------------------------------------------------------- binning (depth order, Eq. 4 "sorted in depth order")
struct Bins {
  std::vector<uint64_t> keys;
  std::vector<uint32_t> ids;
  std::vector<int64_t> start, end;  // per global tile
  std::vector<Proj> proj;           // [V * M]
};

Bins make_bins(const Ctx& c) {
  Bins b;
  const int64_t M = c.sc->n_faces;
  const int V = c.sc->n_views;
  b.proj.resize((size_t)V * M);
  for (int v = 0; v < V; ++v)
    for (int64_t m = 0; m < M; ++m) b.proj[(size_t)v * M + m] = project(c, v, m);
  std::vector<std::pair<uint64_t, uint32_t>> pairs;
  for (int v = 0; v < V; ++v) {
    const View& w = c.views[v];
    for (int64_t m = 0; m < M; ++m) {
      const Proj& pr = b.proj[(size_t)v * M + m];
      if (!pr.visible) continue;
      for (int ty = pr.ty0; ty <= pr.ty1; ++ty)
        for (int tx = pr.tx0; tx <= pr.tx1; ++tx) {
          const uint64_t tile = (uint64_t)(w.tile_off + (int64_t)ty * w.TX + tx);
          uint32_t zb = pr.zbits;
#if ORACLE_MUTANT == 10
          zb = ~zb;
#endif
          pairs.emplace_back((tile << 32) | zb, (uint32_t)m);
        }
    }
  }
  std::stable_sort(pairs.begin(), pairs.end(),
                   [](const std::pair<uint64_t, uint32_t>& a, const std::pair<uint64_t, uint32_t>& b2) { return a.first < b2.first; });
  b.keys.resize(pairs.size());
  b.ids.resize(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) { b.keys[i] = pairs[i].first; b.ids[i] = pairs[i].second; }
  b.start.assign(c.n_tiles, 0);
  b.end.assign(c.n_tiles, 0);
  for (size_t i = 0; i < pairs.size(); ++i) {
    const int64_t tile = (int64_t)(b.keys[i] >> 32);
    if (i == 0 || (int64_t)(b.keys[i - 1] >> 32) != tile) b.start[tile] = (int64_t)i;
    b.end[tile] = (int64_t)i + 1;
  }
  return b;
}

inline void pixel_centre(int x, int y, double* px, double* py) {
#if ORACLE_MUTANT == 6
  *px = x; *py = y;
#else
  *px = x + 0.5; *py = y + 0.5;
#endif
}

// One contribution of a pixel's front-to-back walk.
struct Contrib {
  int64_t pos;    // position in the tile's sorted list
  uint32_t face;
  double alpha, T;  // alpha_n and T_n (transmittance in front of face n)
  Term term;
};

// Eq. 4 for one pixel: returns the contributions in order and the final
// transmittance; *n_last = list position after the last contribution.
double walk_pixel(const Ctx& c, const Bins& b, int view, int x, int y, std::vector<Contrib>* out, int64_t* n_last) {
  const View& w = c.views[view];
  const int64_t M = c.sc->n_faces;
  const int64_t tile = w.tile_off + (int64_t)(y / c.p.tile_h) * w.TX + (x / c.p.tile_w);
  double px, py;
  pixel_centre(x, y, &px, &py);
  double T = 1.0;
  *n_last = 0;
  if (out) out->clear();
  for (int64_t i = b.start[tile]; i < b.end[tile]; ++i) {
    const uint32_t m = b.ids[i];
    const Proj& pr = b.proj[(size_t)view * M + m];
    Term t = eval_term(c, view, m, pr, px, py);
    if (!(t.ratio > 0)) continue;           // outside the face: window is 0
    if (t.alpha < c.p.alpha_min) continue;  // R9 skip
    const double Tn = T * (1.0 - t.alpha);
#if ORACLE_MUTANT == 24
    if (Tn < c.p.T_min) continue;           // skip the face and keep walking
#else
    if (Tn < c.p.T_min) break;              // R9 stop before this face
#endif
    if (out) out->push_back(Contrib{i, m, t.alpha, T, t});
#if ORACLE_MUTANT == 4
    T = Tn;
    if (out) out->back().T = T;
#else
    T = Tn;
#endif
    *n_last = i - b.start[tile] + 1;
  }
  return T;
}

// ---------------------------------------------------------------- dual evaluation for the adjoint
struct DualTerm {
  Dual alpha, col[3], z, nrm[3];
};

// alpha, colour and depth of face m at pixel (px, py) as functions of the
// face's 21 vertex parameters (tangent slots 7k + 0..6) and the view's pose
// perturbation tau = (rho, theta) (slots 21..26), evaluated at tau = 0.
// Left perturbation Exp(tau) o T_CW moves a camera-space point v_C to
// v_C + rho + theta x v_C to first order (Eq. 6-7).
// The projected vertices carry the VALUES of the walk's projection pr (the
// FP32 fixed-order values in FP32 mode, R14) and the derivatives of the
// projection evaluated in double: the term is differentiated at the same
// point the forward walk evaluated it, which matters near edges where the
// window's slope grows like 1/sqrt(ratio).
DualTerm dual_term(const Ctx& c, int view, int64_t m, const Proj& pr, double px, double py) {
  const or_scene* sc = c.sc;
  const View& w = c.views[view];
  const double* P = sc->poses + 12 * view;
  Dual qx[3], qy[3], zc[3], col[3][3], op[3], vcs[3][3];
  Dual rho[3], th[3];
  for (int i = 0; i < 3; ++i) {
    rho[i] = Dual(0.0); rho[i].d[21 + i] = 1.0;
    th[i] = Dual(0.0); th[i].d[24 + i] = 1.0;
  }
  for (int k = 0; k < 3; ++k) {
    const int64_t vi = vidx(sc, m, k);
    Dual X[3];
    for (int a = 0; a < 3; ++a) { X[a] = Dual(sc->pos[3 * vi + a]); X[a].d[7 * k + a] = 1.0; }
    for (int a = 0; a < 3; ++a) { col[k][a] = Dual(sc->col[3 * vi + a]); col[k][a].d[7 * k + 3 + a] = 1.0; }
    op[k] = Dual(sc->opa[vi]); op[k].d[7 * k + 6] = 1.0;
    Dual vc[3];
    for (int r = 0; r < 3; ++r) vc[r] = Dual(P[3 * r]) * X[0] + Dual(P[3 * r + 1]) * X[1] + Dual(P[3 * r + 2]) * X[2] + Dual(P[9 + r]);
    // theta x v_C
    Dual cr[3];
#if ORACLE_MUTANT == 8
    cr[0] = vc[1] * th[2] - vc[2] * th[1];
    cr[1] = vc[2] * th[0] - vc[0] * th[2];
    cr[2] = vc[0] * th[1] - vc[1] * th[0];
#else
    cr[0] = th[1] * vc[2] - th[2] * vc[1];
    cr[1] = th[2] * vc[0] - th[0] * vc[2];
    cr[2] = th[0] * vc[1] - th[1] * vc[0];
#endif
    for (int r = 0; r < 3; ++r) vc[r] = vc[r] + rho[r] + cr[r];
    for (int r = 0; r < 3; ++r) vcs[k][r] = vc[r];
    qx[k] = Dual(w.fx) * (vc[0] / vc[2]) + Dual(w.cx);
    qy[k] = Dual(w.fy) * (vc[1] / vc[2]) + Dual(w.cy);
    zc[k] = vc[2];
    qx[k].v = pr.u[k];
    qy[k].v = pr.v[k];
    zc[k].v = pr.z[k];
  }
  Dual lam[3];
  double ratio;
  Dual sig(sc->sigma_face ? sc->sigma_face[m] : c.p.sigma);
  if (sc->sigma_face) sig.d[27] = 1.0;
  Dual I = window_and_bary<Dual>(qx, qy, px, py, sig, lam, &ratio);
#if ORACLE_MUTANT == 1
  const bool min_variant = true;
#else
  const bool min_variant = c.p.min_opacity != 0;
#endif
  // the minimum passes its derivative to the first vertex that attains it (R24)
  Dual oF = min_variant ? min_(op[0], min_(op[1], op[2])) : (op[0] + op[1] + op[2]) / Dual(3.0);
#if ORACLE_MUTANT == 21
  if (min_variant) {  // the minimum's value with the mean's derivative
    const double mv = oF.v;
    oF = (op[0] + op[1] + op[2]) / Dual(3.0);
    oF.v = mv;
  }
#endif
  DualTerm t;
  Dual a = oF * I;
#if ORACLE_MUTANT == 23
  t.alpha = a;
#else
  t.alpha = a.v > c.p.alpha_max ? Dual(c.p.alpha_max) : a;
#endif
  for (int ch = 0; ch < 3; ++ch) t.col[ch] = lam[0] * col[0][ch] + lam[1] * col[1][ch] + lam[2] * col[2][ch];
#if ORACLE_MUTANT == 7
  t.z = lam[1] * zc[0] + lam[2] * zc[1] + lam[0] * zc[2];
#else
  t.z = lam[0] * zc[0] + lam[1] * zc[1] + lam[2] * zc[2];
#endif
  face_normal<Dual>(vcs, t.nrm);
  return t;
}

int threads_of(const or_params* p) {
#ifdef _OPENMP
  return p->n_threads > 0 ? p->n_threads : omp_get_max_threads();
#else
  (void)p;
  return 1;
#endif
}

}  // namespace

extern "C" {

// Eq. 1 + culling for every (view, face).  rect: [V*M][4] tile box tx0,ty0,tx1,ty1
// (-1 when culled); pix: [V*M][4] pixel box; zbits: depth key bits; count:
// tiles touched; uvz: [V*M][9] u0,u1,u2,v0,v1,v2,z0,z1,z2 (NaN when culled).
int oracle_project(const or_scene* sc, const or_params* p, int32_t* rect, int32_t* pix, uint32_t* zbits,
                   uint32_t* count, double* uvz) {
  Ctx c = make_ctx(sc, p);
  const int64_t M = sc->n_faces;
  for (int v = 0; v < sc->n_views; ++v)
    for (int64_t m = 0; m < M; ++m) {
      const int64_t s = (int64_t)v * M + m;
      Proj pr = project(c, v, m);
      if (rect) { rect[4 * s] = pr.visible ? pr.tx0 : -1; rect[4 * s + 1] = pr.visible ? pr.ty0 : -1; rect[4 * s + 2] = pr.visible ? pr.tx1 : -1; rect[4 * s + 3] = pr.visible ? pr.ty1 : -1; }
      if (pix) { pix[4 * s] = pr.visible ? pr.x0 : -1; pix[4 * s + 1] = pr.visible ? pr.y0 : -1; pix[4 * s + 2] = pr.visible ? pr.x1 : -1; pix[4 * s + 3] = pr.visible ? pr.y1 : -1; }
      if (zbits) zbits[s] = pr.visible ? pr.zbits : 0u;
      if (count) count[s] = pr.visible ? (uint32_t)((pr.tx1 - pr.tx0 + 1) * (pr.ty1 - pr.ty0 + 1)) : 0u;
      if (uvz) for (int k = 0; k < 3; ++k) {
        uvz[9 * s + k] = pr.visible ? pr.u[k] : NAN;
        uvz[9 * s + 3 + k] = pr.visible ? pr.v[k] : NAN;
        uvz[9 * s + 6 + k] = pr.visible ? pr.z[k] : NAN;
      }
    }
  return 0;
}

// Depth-sorted tile lists.  Writes up to cap (key, id) pairs and, when
// ranges != NULL, [n_tiles][2] start/end.  Returns the number of pairs.
int64_t oracle_bin(const or_scene* sc, const or_params* p, uint64_t* keys, uint32_t* ids, int64_t cap,
                   int64_t* ranges) {
  Ctx c = make_ctx(sc, p);
  Bins b = make_bins(c);
  const int64_t n = (int64_t)b.keys.size();
  for (int64_t i = 0; i < n && i < cap; ++i) { if (keys) keys[i] = b.keys[i]; if (ids) ids[i] = b.ids[i]; }
  if (ranges)
    for (int64_t t = 0; t < c.n_tiles; ++t) { ranges[2 * t] = b.start[t]; ranges[2 * t + 1] = b.end[t]; }
  return n;
}

int64_t oracle_total_tiles(const or_scene* sc, const or_params* p) { return make_ctx(sc, p).n_tiles; }

// Eq. 4 forward.  Images are packed per view: colour and normal [3][H][W], the others [H][W].
// normal (optional): the rendered normal map of Eq. 12, sum_n alpha_n T_n n_F (R20), no background.
int oracle_forward(const or_scene* sc, const or_params* p, double* color, double* depth, double* alpha,
                   double* T_final, int32_t* n_last, double* normal) {
  Ctx c = make_ctx(sc, p);
  Bins b = make_bins(c);
  const int nt = threads_of(p);
  for (int v = 0; v < sc->n_views; ++v) {
    const View& w = c.views[v];
    const int64_t HW = (int64_t)w.W * w.H;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int y = 0; y < w.H; ++y) {
      std::vector<Contrib> list;
      for (int x = 0; x < w.W; ++x) {
        int64_t nl;
        const double T = walk_pixel(c, b, v, x, y, &list, &nl);
        double C[3] = {0, 0, 0}, D = 0, A = 0, N[3] = {0, 0, 0};
        for (const Contrib& k : list) {
          const double wgt = k.alpha * k.T;
          for (int ch = 0; ch < 3; ++ch) C[ch] += wgt * k.term.col[ch];
          for (int ch = 0; ch < 3; ++ch) N[ch] += wgt * k.term.nrm[ch];
          D += wgt * k.term.z;
          A += wgt;
        }
#if ORACLE_MUTANT != 5
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * p->bg[ch];
#endif
        const int64_t pi = (int64_t)y * w.W + x;
        if (color) for (int ch = 0; ch < 3; ++ch) color[3 * w.pix_off + ch * HW + pi] = C[ch];
        if (depth) depth[w.pix_off + pi] = D;
        if (alpha) alpha[w.pix_off + pi] = A;
        if (T_final) T_final[w.pix_off + pi] = T;
        if (n_last) n_last[w.pix_off + pi] = (int32_t)nl;
        if (normal) for (int ch = 0; ch < 3; ++ch) normal[3 * w.pix_off + ch * HW + pi] = N[ch];
      }
    }
  }
  return 0;
}

// Mapping-support statistics per (view, face) (Sec. 3.4, R23): coverage [V*M] = pixels at which
// the face was blended in the forward walk; area [V*M] = projected area |D2| / 2 in pixels^2 of a
// face that passed culling (0 otherwise), D2 = (u1 - u0)(v2 - v0) - (u2 - u0)(v1 - v0) in the
// projection's precision (R14).  Either output may be NULL.
int oracle_face_stats(const or_scene* sc, const or_params* p, uint32_t* coverage, double* area) {
  Ctx c = make_ctx(sc, p);
  Bins b = make_bins(c);
  const int64_t M = sc->n_faces;
  if (area)
    for (int v = 0; v < sc->n_views; ++v)
      for (int64_t m = 0; m < M; ++m) {
        const Proj& pr = b.proj[(size_t)v * M + m];
        double a = 0;
        if (pr.visible) {
          if (p->fp64) {
            a = 0.5 * std::fabs((pr.u[1] - pr.u[0]) * (pr.v[2] - pr.v[0]) - (pr.u[2] - pr.u[0]) * (pr.v[1] - pr.v[0]));
          } else {
            const float u0 = (float)pr.u[0], u1 = (float)pr.u[1], u2 = (float)pr.u[2];
            const float v0 = (float)pr.v[0], v1 = (float)pr.v[1], v2 = (float)pr.v[2];
            float du1 = u1 - u0, dv1 = v1 - v0, du2 = u2 - u0, dv2 = v2 - v0;
            float a1 = du1 * dv2, a2 = du2 * dv1;
            float d2 = a1 - a2;
#if ORACLE_MUTANT == 19
            a = (double)std::fabs(d2);  // twice the area
#else
            a = 0.5 * (double)std::fabs(d2);
#endif
          }
        }
        area[(size_t)v * M + m] = a;
      }
  if (coverage) {
    std::memset(coverage, 0, sizeof(uint32_t) * (size_t)sc->n_views * M);
    for (int v = 0; v < sc->n_views; ++v) {
      const View& w = c.views[v];
      std::vector<Contrib> list;
      for (int y = 0; y < w.H; ++y)
        for (int x = 0; x < w.W; ++x) {
          int64_t nl;
          walk_pixel(c, b, v, x, y, &list, &nl);
          for (const Contrib& k : list) coverage[(size_t)v * M + k.face] += 1;
#if ORACLE_MUTANT == 20
          {  // also counts faces whose window is positive but whose alpha was skipped
            double px, py;
            pixel_centre(x, y, &px, &py);
            const int64_t tile = w.tile_off + (int64_t)(y / c.p.tile_h) * w.TX + (x / c.p.tile_w);
            for (int64_t i = b.start[tile]; i < b.end[tile]; ++i) {
              const Term t = eval_term(c, v, b.ids[i], b.proj[(size_t)v * M + b.ids[i]], px, py);
              if (t.ratio > 0 && t.alpha < c.p.alpha_min) coverage[(size_t)v * M + b.ids[i]] += 1;
            }
          }
#endif
        }
    }
  }
  return 0;
}

// The faces of one pixel's walk (front to back) with alpha_n and T_n.
int oracle_pixel_trace(const or_scene* sc, const or_params* p, int view, int x, int y, int32_t* faces,
                       double* alphas, double* T_before, int cap, double* T_final) {
  Ctx c = make_ctx(sc, p);
  Bins b = make_bins(c);
  std::vector<Contrib> list;
  int64_t nl;
  const double T = walk_pixel(c, b, view, x, y, &list, &nl);
  if (T_final) *T_final = T;
  int n = 0;
  for (const Contrib& k : list) {
    if (n < cap) { faces[n] = (int32_t)k.face; alphas[n] = k.alpha; T_before[n] = k.T; }
    ++n;
  }
  return n;
}

// Adjoint of Eq. 4 and Eq. 1-3 for the loss gradients dC, dD, dA, dN (same packing
// as the images; dN, the gradient w.r.t. the normal map, may be NULL).  Gradients are ADDED to dpos [N][3], dcol [N][3], dopa [N],
// dtau [V][6] (rho then theta).  dtau_abs (optional, [V][6]) receives the sum of the absolute
// values of the per-(pixel, face) pose terms: the scale against which the cancelling sum dtau is
// compared.
int oracle_backward_ex(const or_scene* sc, const or_params* p, const double* dC, const double* dD, const double* dA,
                       const double* dN, double* dpos, double* dcol, double* dopa, double* dtau, double* dtau_abs,
                       double* dsigma) {
  Ctx c = make_ctx(sc, p);
  Bins b = make_bins(c);
  const int nt = threads_of(p);
  for (int v = 0; v < sc->n_views; ++v) {
    const View& w = c.views[v];
    const int64_t HW = (int64_t)w.W * w.H;
    double tau_acc[6] = {0, 0, 0, 0, 0, 0}, tau_abs[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) reduction(+ : tau_acc[:6], tau_abs[:6])
    for (int y = 0; y < w.H; ++y) {
      std::vector<Contrib> list;
      for (int x = 0; x < w.W; ++x) {
        int64_t nl;
        const double Tf = walk_pixel(c, b, v, x, y, &list, &nl);
        const int64_t pi = (int64_t)y * w.W + x;
        double gC[3], gD, gA, gN[3];
        for (int ch = 0; ch < 3; ++ch) gC[ch] = dC ? dC[3 * w.pix_off + ch * HW + pi] : 0.0;
        for (int ch = 0; ch < 3; ++ch) gN[ch] = dN ? dN[3 * w.pix_off + ch * HW + pi] : 0.0;
        gD = dD ? dD[w.pix_off + pi] : 0.0;
        gA = dA ? dA[w.pix_off + pi] : 0.0;
        const size_t n = list.size();
        if (n == 0) continue;
        // suffix sums S_n = sum_{k > n} val_k alpha_k T_k + (gC . bg) T_final
        std::vector<double> suffix(n + 1);
        suffix[n] = (gC[0] * p->bg[0] + gC[1] * p->bg[1] + gC[2] * p->bg[2]) * Tf;
#if ORACLE_MUTANT == 5
        suffix[n] = 0;
#endif
        for (size_t k = n; k-- > 0;) {
          const Contrib& q = list[k];
          const double valk = gC[0] * q.term.col[0] + gC[1] * q.term.col[1] + gC[2] * q.term.col[2] + gD * q.term.z + gA +
                              gN[0] * q.term.nrm[0] + gN[1] * q.term.nrm[1] + gN[2] * q.term.nrm[2];
          suffix[k] = suffix[k + 1] + valk * q.alpha * q.T;
        }
        double px, py;
        pixel_centre(x, y, &px, &py);
        for (size_t k = 0; k < n; ++k) {
          const Contrib& q = list[k];
          const double valk = gC[0] * q.term.col[0] + gC[1] * q.term.col[1] + gC[2] * q.term.col[2] + gD * q.term.z + gA +
                              gN[0] * q.term.nrm[0] + gN[1] * q.term.nrm[1] + gN[2] * q.term.nrm[2];
#if ORACLE_MUTANT == 9
          const double dalpha = valk * q.T - suffix[k + 1];
#else
          const double dalpha = valk * q.T - suffix[k + 1] / (1.0 - q.alpha);
#endif
          const double wgt = q.alpha * q.T;
          DualTerm dt = dual_term(c, v, q.face, b.proj[(size_t)v * sc->n_faces + q.face], px, py);
          double g[NT];
          for (int i = 0; i < NT; ++i) {
            g[i] = dalpha * dt.alpha.d[i] + gD * wgt * dt.z.d[i];
            for (int ch = 0; ch < 3; ++ch) g[i] += gC[ch] * wgt * dt.col[ch].d[i] + gN[ch] * wgt * dt.nrm[ch].d[i];
          }
          for (int kk = 0; kk < 3; ++kk) {
            const int64_t vi = vidx(sc, q.face, kk);
            for (int a = 0; a < 3; ++a) {
              if (dpos) {
#pragma omp atomic
                dpos[3 * vi + a] += g[7 * kk + a];
              }
              if (dcol) {
#pragma omp atomic
                dcol[3 * vi + a] += g[7 * kk + 3 + a];
              }
            }
            if (dopa) {
#pragma omp atomic
              dopa[vi] += g[7 * kk + 6];
            }
          }
          if (dsigma && sc->sigma_face) {
#pragma omp atomic
            dsigma[q.face] += g[27];
          }
          for (int i = 0; i < 6; ++i) {
            tau_acc[i] += g[21 + i];
            tau_abs[i] += std::fabs(g[21 + i]);
          }
        }
      }
    }
    if (dtau) for (int i = 0; i < 6; ++i) dtau[6 * v + i] += tau_acc[i];
    if (dtau_abs) for (int i = 0; i < 6; ++i) dtau_abs[6 * v + i] += tau_abs[i];
  }
  return 0;
}

int oracle_backward(const or_scene* sc, const or_params* p, const double* dC, const double* dD, const double* dA,
                    double* dpos, double* dcol, double* dopa, double* dtau) {
  return oracle_backward_ex(sc, p, dC, dD, dA, nullptr, dpos, dcol, dopa, dtau, nullptr, nullptr);
}

// L1 colour + depth loss (R11).  Returns the total over views; loss_v [V];
// gradients dC, dD written (not accumulated) in the image packing.
double oracle_l1_loss(const or_scene* sc, const double* color, const double* depth, const double* tC,
                      const double* tD, double lambda_dep, double* loss_v, double* dC, double* dD) {
  double total = 0;
  int64_t off = 0;
  for (int v = 0; v < sc->n_views; ++v) {
    const int W = (int)sc->cams[6 * v + 4], H = (int)sc->cams[6 * v + 5];
    const int64_t HW = (int64_t)W * H;
#if ORACLE_MUTANT == 12
    const double nc = (double)HW;
#else
    const double nc = 3.0 * (double)HW;
#endif
    double lc = 0, ld = 0;
    for (int64_t i = 0; i < 3 * HW; ++i) {
      const double r = color[3 * off + i] - tC[3 * off + i];
      lc += std::fabs(r);
      if (dC) dC[3 * off + i] = (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / nc;
    }
    for (int64_t i = 0; i < HW; ++i) {
      const bool valid = tD[off + i] > 0;
      const double r = depth[off + i] - tD[off + i];
      if (valid) ld += std::fabs(r);
      if (dD) dD[off + i] = valid ? lambda_dep * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)HW : 0.0;
    }
    const double l = lc / nc + lambda_dep * ld / (double)HW;
    if (loss_v) loss_v[v] = l;
    total += l;
    off += HW;
  }
  return total;
}

// Photometric loss of Eq. 8 with the depth term of Eq. 9 (R16-R18), per view:
//   loss_v = (1 - lambda) mean_{3HW} |C - Cbar| + lambda (1 - mean_{3HW} SSIM(C, Cbar))
//            + lambda_dep sum_{Dbar > 0} |D - Dbar| / HW.
// SSIM at a pixel p of one channel is the structural similarity of Wang et al. (2004) with local
// statistics taken under the 11 x 11 Gaussian window w (sigma 1.5, normalised), centred on p, with
// zeros outside the image:
//   mu_x = sum w x,  e_xx = sum w x^2,  e_xy = sum w x y  (and likewise for y),
//   SSIM = (2 mu_x mu_y + C1)(2 (e_xy - mu_x mu_y) + C2) / ((mu_x^2 + mu_y^2 + C1)(e_xx - mu_x^2 + e_yy - mu_y^2 + C2)),
// C1 = 0.01^2, C2 = 0.03^2.  The gradient w.r.t. C follows the chain rule through the three
// moments that depend on x: dSSIM(p)/dx(q) = w(q - p) (dS/dmu_x + 2 x(q) dS/de_xx + y(q) dS/de_xy).
// Every sum is the plain 121-term window sum (no separable filtering).  ssim_map [3P] optional.
// dC_abs [3P] (optional) receives the scale of the rounding error of an evaluation of dC in
// finite precision: the sum for dC with every term replaced by its absolute value (and dS/dmu_x
// by the sum of the absolute values of its parts), each term p weighted by 1 + kappa_p, kappa_p = (e_xx + e_yy + mu_x^2 + mu_y^2 + 2|e_xy| + 2|mu_x mu_y|) /
// (sigma_x^2 + sigma_y^2 + C2): the factor by which rounding of the window sums is amplified
// when the variances are formed as differences of second moments and means.
double oracle_pho_loss(const or_scene* sc, const double* color, const double* depth, const double* tC,
                       const double* tD, double lambda, double lambda_dep, double* loss_v, double* dC, double* dD,
                       double* ssim_map, double* dC_abs) {
  const int R = 5;
  double g1[2 * R + 1], gs = 0;
  for (int k = -R; k <= R; ++k) gs += (g1[k + R] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
  for (int k = 0; k <= 2 * R; ++k) g1[k] /= gs;
  double w[2 * R + 1][2 * R + 1];
  for (int i = 0; i <= 2 * R; ++i)
    for (int j = 0; j <= 2 * R; ++j) w[i][j] = g1[i] * g1[j];
#if ORACLE_MUTANT == 13
  const double C1 = 0.01 * 0.01, C2 = C1;
#else
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
#endif
  double total = 0;
  int64_t off = 0;
  for (int v = 0; v < sc->n_views; ++v) {
    const int W = (int)sc->cams[6 * v + 4], H = (int)sc->cams[6 * v + 5];
    const int64_t HW = (int64_t)W * H;
    const double nc = 3.0 * (double)HW;
    double lc = 0, ls = 0, ld = 0;
    std::vector<double> m0(HW), m1(HW), m2(HW), S(HW), kap(HW), m0a(HW);
    for (int ch = 0; ch < 3; ++ch) {
      const double* x = color + 3 * off + ch * HW;
      const double* y = tC + 3 * off + ch * HW;
      auto inside = [&](int px, int py) { return px >= 0 && px < W && py >= 0 && py < H; };
#if ORACLE_MUTANT == 15
      auto at = [&](const double* a, int px, int py) {  // clamp to the edge instead of zeros
        px = std::min(std::max(px, 0), W - 1);
        py = std::min(std::max(py, 0), H - 1);
        return a[(int64_t)py * W + px];
      };
#else
      auto at = [&](const double* a, int px, int py) { return inside(px, py) ? a[(int64_t)py * W + px] : 0.0; };
#endif
#pragma omp parallel for schedule(static) reduction(+ : ls)
      for (int py = 0; py < H; ++py) {
        for (int px = 0; px < W; ++px) {
          double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
          for (int i = -R; i <= R; ++i) {
            for (int j = -R; j <= R; ++j) {
              const double ww = w[i + R][j + R];
              const double a = at(x, px + j, py + i), b = at(y, px + j, py + i);
              mx += ww * a;
              my += ww * b;
              exx += ww * a * a;
              eyy += ww * b * b;
              exy += ww * a * b;
            }
          }
          const double A1 = 2 * mx * my + C1, A2 = 2 * (exy - mx * my) + C2;
          const double B1 = mx * mx + my * my + C1, B2 = (exx - mx * mx) + (eyy - my * my) + C2;
          const double s = A1 * A2 / (B1 * B2);
          const int64_t p = (int64_t)py * W + px;
          S[p] = s;
          // partial derivatives of s w.r.t. mu_x, e_xx, e_xy
          m0[p] = (2 * my * (A2 - A1) - 2 * mx * s * (B2 - B1)) / (B1 * B2);
          m1[p] = -s / B2;
          m2[p] = 2 * A1 / (B1 * B2);
          kap[p] = (exx + eyy + mx * mx + my * my + 2 * std::fabs(exy) + 2 * std::fabs(mx * my)) / B2;
          m0a[p] = 2 * (std::fabs(my) * (std::fabs(A2) + A1) + std::fabs(mx * s) * (B2 + B1)) / (B1 * B2);
          ls += s;
        }
      }
      if (ssim_map)
        for (int64_t p = 0; p < HW; ++p) ssim_map[3 * off + ch * HW + p] = S[p];
      for (int64_t q = 0; q < HW; ++q) lc += std::fabs(x[q] - y[q]);
      if (!dC) continue;
#pragma omp parallel for schedule(static)
      for (int qy = 0; qy < H; ++qy) {
        for (int qx = 0; qx < W; ++qx) {
          const int64_t q = (int64_t)qy * W + qx;
          double gsum = 0, gabs = 0;  // sums over the pixels p whose window holds q
          for (int i = -R; i <= R; ++i) {
            for (int j = -R; j <= R; ++j) {
              const int px = qx + j, py = qy + i;
              if (!inside(px, py)) continue;
              const int64_t p = (int64_t)py * W + px;
#if ORACLE_MUTANT == 14
              gsum += w[i + R][j + R] * (m0[p] + x[q] * m1[p] + y[q] * m2[p]);
#else
              gsum += w[i + R][j + R] * (m0[p] + 2 * x[q] * m1[p] + y[q] * m2[p]);
#endif
              gabs += w[i + R][j + R] * (m0a[p] + std::fabs(2 * x[q] * m1[p]) + std::fabs(y[q] * m2[p])) * (1 + kap[p]);
            }
          }
          const double r = x[q] - y[q];
          dC[3 * off + ch * HW + q] = (1 - lambda) * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / nc - lambda * gsum / nc;
          if (dC_abs) dC_abs[3 * off + ch * HW + q] = ((1 - lambda) * (r != 0 ? 1.0 : 0.0) + lambda * gabs) / nc;
        }
      }
    }
    for (int64_t i = 0; i < HW; ++i) {
      const bool valid = tD[off + i] > 0;
      const double r = depth[off + i] - tD[off + i];
      if (valid) ld += std::fabs(r);
      if (dD) dD[off + i] = valid ? lambda_dep * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)HW : 0.0;
    }
    const double l = (1 - lambda) * lc / nc + lambda * (1 - ls / nc) + lambda_dep * ld / (double)HW;
    if (loss_v) loss_v[v] = l;
    total += l;
    off += HW;
  }
  return total;
}

// Eq. 3 window of a 2D triangle q = (x0, y0, x1, y1, x2, y2) at point (px, py).
double oracle_window(const double* q, double sigma, double px, double py, double* lam_out) {
  double qx[3] = {q[0], q[2], q[4]}, qy[3] = {q[1], q[3], q[5]}, lam[3], ratio;
  const double I = window_and_bary<double>(qx, qy, px, py, sigma, lam, &ratio);
  if (lam_out) for (int k = 0; k < 3; ++k) lam_out[k] = lam[k];
  return I;
}

// Normal loss of Eq. 12 (R22), per view: loss_v = sum_{p valid} (1 - N_p . Nbar_p) / HW, a pixel
// valid where the sensor normal Nbar_p is not the zero vector; dN = weight * dloss_v/dN (written;
// the weight is lambda_norm of Eq. 15).
double oracle_normal_loss(const or_scene* sc, const double* normal, const double* tgt_normal, double weight,
                          double* loss_v, double* dN) {
  double total = 0;
  int64_t off = 0;
  for (int v = 0; v < sc->n_views; ++v) {
    const int W = (int)sc->cams[6 * v + 4], H = (int)sc->cams[6 * v + 5];
    const int64_t HW = (int64_t)W * H;
    double l = 0;
    for (int64_t i = 0; i < HW; ++i) {
      double nb[3], dot = 0;
      bool valid = false;
      for (int ch = 0; ch < 3; ++ch) {
        nb[ch] = tgt_normal[3 * off + ch * HW + i];
        valid = valid || nb[ch] != 0.0;
        dot += normal[3 * off + ch * HW + i] * nb[ch];
      }
      if (valid) l += 1.0 - dot;
      if (dN)
        for (int ch = 0; ch < 3; ++ch) dN[3 * off + ch * HW + i] = valid ? -weight * nb[ch] / (double)HW : 0.0;
    }
    l /= (double)HW;
    if (loss_v) loss_v[v] = l;
    total += l;
    off += HW;
  }
  return total;
}

// Equilateral regulariser of Eq. 14 (R19): E = (1/M) sum_faces (1/3) sum_n (cos theta_n - 0.5)^2,
// theta_n the internal angle at vertex n, cos theta_n from the normalised edge vectors leaving
// vertex n.  A face with a zero-length edge adds 0 (it still counts in M).  dpos [N][3]
// (optional) receives dE/dpos, added over the faces that share a vertex; each face is
// differentiated with forward-mode dual numbers over its 9 vertex coordinates.
double oracle_equilateral(const or_scene* sc, double* dpos) {
  const int64_t M = sc->n_faces;
  if (dpos) std::memset(dpos, 0, sizeof(double) * 3 * sc->n_vertices);
  if (M == 0) return 0.0;
  double total = 0;
  for (int64_t m = 0; m < M; ++m) {
    Dual P[3][3];
    int64_t vi[3];
    for (int k = 0; k < 3; ++k) {
      vi[k] = vidx(sc, m, k);
      for (int c = 0; c < 3; ++c) {
        P[k][c] = Dual(sc->pos[3 * vi[k] + c]);
        P[k][c].d[3 * k + c] = 1.0;
      }
    }
    bool degenerate = false;
    Dual e(0.0);
    for (int n = 0; n < 3; ++n) {
#if ORACLE_MUTANT == 16
      const int i1 = (n + 1) % 3, i2 = (n + 2) % 3, i0 = i1;  // second edge leaves the wrong vertex
#else
      const int i1 = (n + 1) % 3, i2 = (n + 2) % 3, i0 = n;
#endif
      Dual a[3], b[3];
      for (int c = 0; c < 3; ++c) {
        a[c] = P[i1][c] - P[n][c];
        b[c] = P[i2][c] - P[i0][c];
      }
      const Dual aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
      const Dual bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
      if (!(aa.v > 0) || !(bb.v > 0)) {
        degenerate = true;
        break;
      }
      const Dual cs = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (sqrt_(aa) * sqrt_(bb));
      const Dual d = cs - Dual(0.5);
      e = e + d * d;
    }
    if (degenerate) continue;
    total += e.v / 3.0;
    if (dpos)
      for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) dpos[3 * vi[k] + c] += e.d[3 * k + c] / (3.0 * (double)M);
  }
  return total / (double)M;
}

// SE(3) exponential (closed form of Sola et al., "A micro Lie theory"):
// tau = (rho, theta) -> T = [R | t], R = Exp_SO3(theta), t = V(theta) rho.
void oracle_se3_exp(const double* tau, double* T) {
  const double* rho = tau;
  const double* th = tau + 3;
  const double a2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
  const double a = std::sqrt(a2);
  double A, B, Cc;  // sin a / a, (1 - cos a) / a^2, (a - sin a) / a^3
  if (a < 1e-6) {
    A = 1 - a2 / 6; B = 0.5 - a2 / 24; Cc = 1.0 / 6 - a2 / 120;
  } else {
    A = std::sin(a) / a; B = (1 - std::cos(a)) / a2; Cc = (a - std::sin(a)) / (a2 * a);
  }
  const double K[9] = {0, -th[2], th[1], th[2], 0, -th[0], -th[1], th[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      K2[3 * i + j] = 0;
      for (int l = 0; l < 3; ++l) K2[3 * i + j] += K[3 * i + l] * K[3 * l + j];
    }
  double R[9], Vm[9];
  for (int i = 0; i < 9; ++i) {
    const double I3 = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I3 + A * K[i] + B * K2[i];
    Vm[i] = I3 + B * K[i] + Cc * K2[i];
  }
  for (int i = 0; i < 9; ++i) T[i] = R[i];
  for (int i = 0; i < 3; ++i) T[9 + i] = Vm[3 * i] * rho[0] + Vm[3 * i + 1] * rho[1] + Vm[3 * i + 2] * rho[2];
}

// Left perturbation Exp(tau) o T_CW of a pose [12].
void oracle_pose_left_update(const double* tau, const double* pose, double* out) {
  double E[12];
  oracle_se3_exp(tau, E);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) out[3 * i + j] = E[3 * i] * pose[j] + E[3 * i + 1] * pose[3 + j] + E[3 * i + 2] * pose[6 + j];
    out[9 + i] = E[3 * i] * pose[9] + E[3 * i + 1] * pose[10] + E[3 * i + 2] * pose[11] + E[9 + i];
  }
}

int oracle_mutant(void) { return ORACLE_MUTANT; }

}  // extern "C"
