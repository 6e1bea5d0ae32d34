// k_pho.cu -- photometric loss of Eq. 8 (L1 + D-SSIM) with the depth term of Eq. 9-10, fused
// with its gradient w.r.t. the rendered colour and depth images.
//
// Per view:  loss = (1 - lambda) sum|C - Cbar| / 3HW + lambda (1 - sum SSIM / 3HW)
//                   + lambda_dep sum_{Dbar > 0} |D - Dbar| / HW.
// SSIM (Wang et al. 2004) of one channel at pixel p uses the local statistics mu_x, mu_y,
// e_xx, e_yy, e_xy: sums of x, y, x^2, y^2, xy under the 11 x 11 Gaussian window (sigma 1.5,
// normalised) centred on p, with zeros outside the image; C1 = 0.01^2, C2 = 0.03^2.  Its gradient
// is dSSIM_sum/dx(q) = (G * m0)(q) + 2 x(q) (G * m1)(q) + y(q) (G * m2)(q), where m0, m1, m2 are
// the partials of SSIM(p) w.r.t. mu_x, e_xx and e_xy (zero outside the image) and G * the same
// symmetric window sum.  In FP32 the variances formed as e_xx - mu_x^2 lose digits where the
// window is nearly constant at a non-zero value; the error of dL/dC stays below ~1e-7 of the
// magnitude of its terms weighted by (moments) / (sigma_x^2 + sigma_y^2 + C2).  (A shift of the
// data by one constant per tile does not help: it moves the cancellation to flat regions at other
// values, such as the zeros of a clamped or black background.)
//
// One CTA owns a 32 x 32 output tile of one view and walks the three channels.  It stages x and y
// over the tile widened by 10 pixels (the window of a window) with asynchronous copies, the next
// channel's while the current one is processed, filters the five moment maps along
// rows and then columns over the tile widened by 5, evaluates SSIM and m0..m2 there, filters those
// three maps back over the tile, and writes dL/dC.  Every filter pass is register-blocked: a
// thread produces R consecutive outputs along the filter direction from R + 10 shared-memory
// loads.  Shared-memory row strides are odd, so lanes that walk consecutive rows hit distinct
// banks.  Loss partial sums go to one slot per CTA and are reduced per view in a fixed order:
// the loss is deterministic.
#include <algorithm>
#include <cmath>

#include "ts_internal.cuh"

namespace {

constexpr int PT = 256;          // threads per CTA
constexpr int OT = 32;           // output tile side
constexpr int RAD = 5;           // window radius
constexpr int NT = 2 * RAD + 1;  // taps
constexpr int IN = OT + 4 * RAD, IS = IN + 1;   // staged x, y: 52 x 52, stride 53
constexpr int MO = OT + 2 * RAD, MS = MO + 1;   // moment / partial maps: 42 x 42, stride 43
constexpr int OS = OT + 1;                      // column-filtered partials: 42 rows x 32, stride 33
constexpr int R_H1 = 7, R_V1 = 7, R_H2 = 8, R_V2 = 4;
static_assert(MO % R_H1 == 0 && MO % R_V1 == 0 && OT % R_H2 == 0 && OT % R_V2 == 0, "blocking");
// two staging buffers (x, y) so that the next channel streams in while this one is filtered
constexpr int SM_XY = 0, SM_H = SM_XY + 4 * IN * IS, SM_M = SM_H + 5 * IN * MS, SM_FLOATS = SM_M + 3 * MO * MS;
static_assert(3 * MO * OS <= 5 * IN * MS, "column-filtered partials alias the moment rows");
constexpr size_t PHO_SMEM = (size_t)SM_FLOATS * 4;

struct Taps {
  float w[NT];
};

// 4-byte asynchronous global-to-shared copy; valid == false writes a zero and reads nothing.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Issue the copies of x and y over image rows Y0-10 .. Y0+41 and columns X0-10 .. X0+41 (zeros
// outside the image) into one staging buffer.
__device__ __forceinline__ void stage_channel(float* sx, float* sy, const float* xc, const float* yc, int X0, int Y0,
                                              int W, int H) {
  for (int i = threadIdx.x; i < IN * IN; i += PT) {
    const int r = i / IN, c = i - r * IN;
    const int gy = Y0 - 2 * RAD + r, gx = X0 - 2 * RAD + c;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const long long o = in ? (long long)gy * W + gx : 0;
    cp_async4(sx + r * IS + c, xc + o, in);
    cp_async4(sy + r * IS + c, yc + o, in);
  }
  cp_async_commit();
}

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PT / 32; ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(PT, 2)
    k_pho_tile(const TsImageTable tab, const float* __restrict__ C, const float* __restrict__ D,
               const float* __restrict__ tC, const float* __restrict__ tD, float lambda, float lambda_dep, Taps tp,
               float* __restrict__ dC, float* __restrict__ dD, float* __restrict__ part, int nblk) {
  extern __shared__ float sm[];
  __shared__ float red[PT / 32];
  const int v = blockIdx.y;
  const int W = tab.W[v], H = tab.H[v];
  const long long pix_off = tab.pix_off[v];
  const int TXo = (W + OT - 1) / OT, TYo = (H + OT - 1) / OT;
  if ((int)blockIdx.x >= TXo * TYo) return;  // uniform over the CTA
  const int X0 = (blockIdx.x % TXo) * OT, Y0 = (blockIdx.x / TXo) * OT;
  const long long HW = (long long)W * H;
  const float inv3 = 1.0f / (3.0f * (float)HW);
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  float* hmo = sm + SM_H;  // 5 maps [IN][MS]: row-filtered moments
  float* mp = sm + SM_M;   // 3 maps [MO][MS]: partials m0, m1, m2
  float* hm = sm + SM_H;   // 3 maps [MO][OS]: column-filtered partials (aliases hmo)
  float l1 = 0.f, ss = 0.f, dep = 0.f;

  stage_channel(sm + SM_XY, sm + SM_XY + IN * IS, C + 3 * pix_off, tC + 3 * pix_off, X0, Y0, W, H);
  for (int ch = 0; ch < 3; ++ch) {
    if (ch + 1 < 3) {
      float* nb = sm + SM_XY + ((ch + 1) & 1) * 2 * IN * IS;
      stage_channel(nb, nb + IN * IS, C + 3 * pix_off + (ch + 1) * HW, tC + 3 * pix_off + (ch + 1) * HW, X0, Y0, W,
                    H);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* sx = sm + SM_XY + (ch & 1) * 2 * IN * IS;
    const float* sy = sx + IN * IS;
    // rows: moments at staged row r, columns cm in [0, MO) (image column X0 - 5 + cm)
    for (int it = threadIdx.x; it < IN * (MO / R_H1); it += PT) {
      const int r = it % IN, c0 = (it / IN) * R_H1;
      float a[5][R_H1];
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int j = 0; j < R_H1; ++j) a[m][j] = 0.f;
#pragma unroll
      for (int k = 0; k < R_H1 + 2 * RAD; ++k) {
        const float x = sx[r * IS + c0 + k], y = sy[r * IS + c0 + k];
        const float xx = x * x, yy = y * y, xy = x * y;
#pragma unroll
        for (int j = 0; j < R_H1; ++j) {
          const int t = k - j;
          if (t >= 0 && t < NT) {
            a[0][j] = fmaf(tp.w[t], x, a[0][j]);
            a[1][j] = fmaf(tp.w[t], y, a[1][j]);
            a[2][j] = fmaf(tp.w[t], xx, a[2][j]);
            a[3][j] = fmaf(tp.w[t], yy, a[3][j]);
            a[4][j] = fmaf(tp.w[t], xy, a[4][j]);
          }
        }
      }
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int j = 0; j < R_H1; ++j) hmo[m * IN * MS + r * MS + c0 + j] = a[m][j];
    }
    __syncthreads();
    // columns: statistics at moment-map pixel (rm, cm) = image (Y0 - 5 + rm, X0 - 5 + cm)
    for (int it = threadIdx.x; it < MO * (MO / R_V1); it += PT) {
      const int cm = it % MO, r0 = (it / MO) * R_V1;
      float a[5][R_V1];
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int j = 0; j < R_V1; ++j) a[m][j] = 0.f;
#pragma unroll
      for (int k = 0; k < R_V1 + 2 * RAD; ++k) {
        float u[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) u[m] = hmo[m * IN * MS + (r0 + k) * MS + cm];
#pragma unroll
        for (int j = 0; j < R_V1; ++j) {
          const int t = k - j;
          if (t >= 0 && t < NT) {
#pragma unroll
            for (int m = 0; m < 5; ++m) a[m][j] = fmaf(tp.w[t], u[m], a[m][j]);
          }
        }
      }
      const int gx = X0 - RAD + cm;
      const bool colin = gx >= 0 && gx < W, colinner = cm >= RAD && cm < RAD + OT;
#pragma unroll
      for (int j = 0; j < R_V1; ++j) {
        const int rm = r0 + j, gy = Y0 - RAD + rm;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
        if (colin && gy >= 0 && gy < H) {
          const float mx = a[0][j], my = a[1][j];
          const float A1 = 2.f * mx * my + C1, A2 = 2.f * (a[4][j] - mx * my) + C2;
          const float B1 = mx * mx + my * my + C1, B2 = (a[2][j] - mx * mx) + (a[3][j] - my * my) + C2;
          const float iB = 1.f / (B1 * B2);
          const float s = A1 * A2 * iB;
          // partials w.r.t. mu_x, e_xx and e_xy
          m0 = 2.f * (my * (A2 - A1) - mx * s * (B2 - B1)) * iB;
          m1 = -s * B1 * iB;
          m2 = 2.f * A1 * iB;
          if (colinner && rm >= RAD && rm < RAD + OT) ss += s;
        }
        mp[0 * MO * MS + rm * MS + cm] = m0;
        mp[1 * MO * MS + rm * MS + cm] = m1;
        mp[2 * MO * MS + rm * MS + cm] = m2;
      }
    }
    __syncthreads();
    // rows: partials filtered to output columns co (image X0 + co), at moment rows rm
    for (int it = threadIdx.x; it < MO * (OT / R_H2); it += PT) {
      const int rm = it % MO, c0 = (it / MO) * R_H2;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float a[R_H2];
#pragma unroll
        for (int j = 0; j < R_H2; ++j) a[j] = 0.f;
#pragma unroll
        for (int k = 0; k < R_H2 + 2 * RAD; ++k) {
          const float u = mp[m * MO * MS + rm * MS + c0 + k];
#pragma unroll
          for (int j = 0; j < R_H2; ++j) {
            const int t = k - j;
            if (t >= 0 && t < NT) a[j] = fmaf(tp.w[t], u, a[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < R_H2; ++j) hm[m * MO * OS + rm * OS + c0 + j] = a[j];
      }
    }
    __syncthreads();
    // columns: output pixel (ro, co) = image (Y0 + ro, X0 + co)
    for (int it = threadIdx.x; it < OT * (OT / R_V2); it += PT) {
      const int co = it % OT, r0 = (it / OT) * R_V2;
      float g[3][R_V2];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int j = 0; j < R_V2; ++j) g[m][j] = 0.f;
#pragma unroll
      for (int k = 0; k < R_V2 + 2 * RAD; ++k) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const float u = hm[m * MO * OS + (r0 + k) * OS + co];
#pragma unroll
          for (int j = 0; j < R_V2; ++j) {
            const int t = k - j;
            if (t >= 0 && t < NT) g[m][j] = fmaf(tp.w[t], u, g[m][j]);
          }
        }
      }
      const int gx = X0 + co;
#pragma unroll
      for (int j = 0; j < R_V2; ++j) {
        const int gy = Y0 + r0 + j;
        if (gx < W && gy < H) {
          const float x = sx[(r0 + j + 2 * RAD) * IS + co + 2 * RAD], y = sy[(r0 + j + 2 * RAD) * IS + co + 2 * RAD];
          const float r = x - y;
          l1 += fabsf(r);
          const float sg = r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f);
          const float gs = g[0][j] + 2.f * x * g[1][j] + y * g[2][j];
          dC[3 * pix_off + ch * HW + (long long)gy * W + gx] = ((1.f - lambda) * sg - lambda * gs) * inv3;
        }
      }
    }
    __syncthreads();  // the channel after next restages into this buffer; every map is reused
  }
  // depth term of Eq. 9 over the tile's own pixels
  {
    const float id = lambda_dep / (float)HW;
#pragma unroll
    for (int i = threadIdx.x; i < OT * OT; i += PT) {
      const int gy = Y0 + i / OT, gx = X0 + i % OT;
      if (gx < W && gy < H) {
        const long long o = pix_off + (long long)gy * W + gx;
        const float t = tD[o];
        const float r = D[o] - t;
        const bool valid = t > 0.f;
        if (valid) dep += fabsf(r);
        dD[o] = valid ? (r > 0.f ? id : (r < 0.f ? -id : 0.f)) : 0.f;
      }
    }
  }
  l1 = block_sum(l1, red);
  ss = block_sum(ss, red);
  dep = block_sum(dep, red);
  if (threadIdx.x == 0) {
    float* o = part + ((long long)v * nblk + blockIdx.x) * 3;
    o[0] = l1;
    o[1] = ss;
    o[2] = dep;
  }
}

__global__ void __launch_bounds__(PT) k_pho_final(const TsImageTable tab, const float* __restrict__ part, int nblk,
                                                   float lambda, float lambda_dep, float* __restrict__ loss) {
  __shared__ double red[PT][3];
  const int v = blockIdx.x;
  const int n = ((tab.W[v] + OT - 1) / OT) * ((tab.H[v] + OT - 1) / OT);
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < n; k += PT) {
    const float* o = part + ((long long)v * nblk + k) * 3;
    a += o[0];
    b += o[1];
    c += o[2];
  }
  red[threadIdx.x][0] = a;
  red[threadIdx.x][1] = b;
  red[threadIdx.x][2] = c;
  __syncthreads();
  for (int o = PT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int i = 0; i < 3; ++i) red[threadIdx.x][i] += red[threadIdx.x + o][i];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double HW = (double)tab.W[v] * tab.H[v];
    loss[v] = (float)((1.0 - lambda) * red[0][0] / (3.0 * HW) + lambda * (1.0 - red[0][1] / (3.0 * HW)) +
                      (double)lambda_dep * red[0][2] / HW);
  }
}

Taps gaussian_taps() {
  double g[NT], s = 0;
  for (int k = 0; k < NT; ++k) s += (g[k] = std::exp(-(double)((k - RAD) * (k - RAD)) / (2.0 * 1.5 * 1.5)));
  Taps t;
  for (int k = 0; k < NT; ++k) t.w[k] = (float)(g[k] / s);
  return t;
}

}  // namespace

int64_t ts_pho_blocks(const TsView* views, int V) {
  int64_t n = 1;
  for (int v = 0; v < V; ++v)
    n = std::max<int64_t>(n, (int64_t)((views[v].W + OT - 1) / OT) * ((views[v].H + OT - 1) / OT));
  return n;
}

cudaError_t ts_launch_pho_loss(const TsPlanImpl* p, const TsWs& w, const float* color, const float* depth,
                               const float* tc, const float* td, float lambda, float lambda_dep, float* loss,
                               float* dC, float* dD, cudaStream_t s) {
  cudaError_t e = ts_smem_limit((const void*)k_pho_tile, (int)PHO_SMEM);
  if (e != cudaSuccess) return e;
  const int nblk = (int)p->n_pho_blocks;
  const TsImageTable tab = ts_image_table(p);
  k_pho_tile<<<dim3((unsigned)nblk, (unsigned)p->V), PT, PHO_SMEM, s>>>(tab, color, depth, tc, td, lambda,
                                                                      lambda_dep, gaussian_taps(), dC, dD, w.pho,
                                                                      nblk);
  k_pho_final<<<p->V, PT, 0, s>>>(tab, w.pho, nblk, lambda, lambda_dep, loss);
  return cudaGetLastError();
}
