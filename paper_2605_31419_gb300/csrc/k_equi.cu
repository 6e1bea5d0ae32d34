// k_equi.cu -- the equilateral regulariser of the mapping loss (Eq. 14) and its gradient w.r.t.
// vertex positions.
//
// E = (1/M) sum_faces (1/3) sum_n (cos theta_n - 0.5)^2, theta_n the internal angle at vertex n:
// with a = v_{n+1} - v_n and b = v_{n+2} - v_n, cos theta_n = a.b / (|a||b|), and
//   dcos/da = b / (|a||b|) - cos a / |a|^2,   dcos/db = a / (|a||b|) - cos b / |b|^2,
// moving v_{n+1} by dcos/da, v_{n+2} by dcos/db and v_n by minus their sum.  One thread per face;
// a face with a zero-length edge adds nothing.  Per-block partial sums are reduced in a fixed
// order, so the value is deterministic; so are the gradients of a soup map, whose vertices belong
// to one face each (plain read-modify-write), while an indexed mesh adds with atomics.
#include "ts_internal.cuh"

namespace {

constexpr int EQ_T = 256;

struct EquiArgs {
  const float *px, *py, *pz;
  const int32_t* faces;
  long long n_vertices, M;
  float* gx;
  float* gy;
  float* gz;
  float gscale;  // weight / M
  float* part;
  TsDevHeader* hdr;
};

__global__ void __launch_bounds__(EQ_T) k_equi_partial(EquiArgs a) {
  __shared__ float red[EQ_T / 32];
  const long long m = (long long)blockIdx.x * EQ_T + threadIdx.x;
  float e = 0.f;
  if (m < a.M) {
    long long j[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      j[k] = a.faces ? (long long)a.faces[3 * m + k] : 3 * m + k;
      if (j[k] < 0 || j[k] >= a.n_vertices) ok = false;
    }
    if (!ok) {
      atomicOr(&a.hdr->error_bits, TS_ERRBIT_BOUNDS);
    } else {
      float p[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        p[k][0] = a.px[j[k]];
        p[k][1] = a.py[j[k]];
        p[k][2] = a.pz[j[k]];
      }
      float g[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      bool degenerate = false;
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        const int n1 = (n + 1) % 3, n2 = (n + 2) % 3;
        float av[3], bv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          av[c] = p[n1][c] - p[n][c];
          bv[c] = p[n2][c] - p[n][c];
        }
        const float aa = av[0] * av[0] + av[1] * av[1] + av[2] * av[2];
        const float bb = bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2];
        if (!(aa > 0.f) || !(bb > 0.f)) degenerate = true;
        const float ia = rsqrtf(aa), ib = rsqrtf(bb);
        const float cs = (av[0] * bv[0] + av[1] * bv[1] + av[2] * bv[2]) * ia * ib;
        const float d = cs - 0.5f;
        e += d * d;
        const float gd = (2.f / 3.f) * d * a.gscale;  // dE_weighted / dcos
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float da = gd * (bv[c] * ia * ib - cs * av[c] * ia * ia);
          const float db = gd * (av[c] * ia * ib - cs * bv[c] * ib * ib);
          g[n1][c] += da;
          g[n2][c] += db;
          g[n][c] -= da + db;
        }
      }
      if (degenerate) {
        e = 0.f;
      } else {
        e *= 1.f / 3.f;
        float* dst[3] = {a.gx, a.gy, a.gz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!dst[c]) continue;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (a.faces)
              atomicAdd(dst[c] + j[k], g[k][c]);
            else
              dst[c][j[k]] += g[k][c];
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < EQ_T / 32; ++w) s += red[w];
    a.part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(EQ_T) k_equi_final(const float* __restrict__ part, int nblk, long long M,
                                                      float* __restrict__ loss) {
  __shared__ double red[EQ_T];
  double s = 0;
  for (int k = threadIdx.x; k < nblk; k += EQ_T) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = EQ_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = M > 0 ? (float)(red[0] / (double)M) : 0.f;
}

}  // namespace

int64_t ts_equi_blocks(int64_t M) { return M > 0 ? (M + EQ_T - 1) / EQ_T : 1; }

cudaError_t ts_launch_equilateral(const TsPlanImpl* p, const TsWs& w, const ts_map* map, float weight, float* loss,
                                  const ts_map_grad* grad, cudaStream_t s) {
  EquiArgs a;
  a.px = map->px;
  a.py = map->py;
  a.pz = map->pz;
  a.faces = map->faces;
  a.n_vertices = map->n_vertices;
  a.M = p->M;
  a.gx = grad ? grad->gpx : nullptr;
  a.gy = grad ? grad->gpy : nullptr;
  a.gz = grad ? grad->gpz : nullptr;
  a.gscale = p->M > 0 ? weight / (float)p->M : 0.f;
  a.part = w.equi;
  a.hdr = w.hdr;
  const int nblk = (int)ts_equi_blocks(p->M);
  if (p->M > 0) k_equi_partial<<<nblk, EQ_T, 0, s>>>(a);
  k_equi_final<<<1, EQ_T, 0, s>>>(w.equi, p->M > 0 ? nblk : 0, p->M, loss);
  return cudaGetLastError();
}
