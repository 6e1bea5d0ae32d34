// k_bin.cu -- depth ordering per tile (Eq. 4: faces are composited in depth order).
//
//  1. per tile, the number of (view, face) pairs whose tile rectangle covers it.  When every
//     view's tiles fit in shared memory (TS_BIN_MAX_TILES), one block per (TS_BIN_FACES faces,
//     view) counts its pairs per tile there and writes a [tile][face block] count matrix; else
//     global atomic counts per tile;
//  2. an exclusive scan of the counts (two-level, 4096 items per block; tile-major for the
//     matrix) gives each tile's segment [start, end) of the pair list -- and with the matrix each
//     block's first place in it -- the pair total and the capacity check;
//  3. each pair is placed in its tile's segment (shared-memory atomics on the block's places, or
//     global atomic cursors) as the 64-bit key (float bits of the depth key << 32 | face id),
//     unique within a tile;
//  4. each segment is sorted by that key (bitonic networks: one warp in registers up to 64 pairs,
//     one warp in shared memory up to 512, one CTA beyond), and written out as the pair list:
//     key (global tile id << 32 | depth bits) and face id, ascending depth with ties in ascending
//     face id -- the order a stable sort of the (view, face)-ordered pairs by (tile, depth) gives.
// Every kernel reads the pair count from the device, so nothing here synchronises the host.
#include <algorithm>

#include "ts_internal.cuh"

namespace {

constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = TS_SCAN_ITEMS / SCAN_T;  // 4

// length of a scanned array
struct Len {
  long long n;
  __device__ __forceinline__ long long get() const { return n; }
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block scan of one value per thread (1024 threads); returns the block total in *tot.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* sm, uint32_t* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(x);
  if (lane == 31) sm[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = sm[lane];
    const uint32_t wi = warp_incl_scan(w);
    sm[lane] = wi - w;
    if (lane == 31) sm[32] = wi;
  }
  __syncthreads();
  const uint32_t r = sm[warp] + inc - x;
  *tot = sm[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t* __restrict__ in, Len len,
                                                        uint32_t* __restrict__ bsums) {
  __shared__ uint32_t sm[33];
  const long long n = len.get();
  const long long base = (long long)blockIdx.x * TS_SCAN_ITEMS;
  if (base >= n) return;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    const long long i = base + (long long)k * SCAN_T + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint32_t tot;
  block_excl_scan(s, sm, &tot);
  if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in place (one block); writes the grand total, and zeroes
// *zero_out (the sort's count of long lists) for the launches that follow.
__global__ void __launch_bounds__(SCAN_T) k_scan_bsums(uint32_t* bsums, Len len, unsigned long long* total_out,
                                                       unsigned int* err, long long cap, unsigned int* zero_out) {
  __shared__ uint32_t sm[33];
  __shared__ unsigned long long wsum[SCAN_T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n = len.get();
  const long long nb = (n + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS;
  const long long per = (nb + SCAN_T - 1) / SCAN_T;
  const long long b0 = (long long)threadIdx.x * per;
  unsigned long long s = 0;
  for (long long i = b0; i < b0 + per && i < nb; ++i) s += bsums[i];
  uint32_t tot;
  uint32_t run = block_excl_scan((uint32_t)s, sm, &tot);
  // the 64-bit total guards against overflow of the 32-bit running offsets: a warp reduction,
  // then the warps' sums in order
  unsigned long long ws = s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if (lane == 0) wsum[warp] = ws;
  for (long long i = b0; i < b0 + per && i < nb; ++i) {
    const uint32_t v = bsums[i];
    bsums[i] = run;
    run += v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot64 = 0;
    for (int w = 0; w < SCAN_T / 32; ++w) tot64 += wsum[w];
    if (total_out) {
      *total_out = tot64;
      if ((long long)tot64 > cap) atomicOr(err, TS_ERRBIT_CAPACITY);
    }
    if (zero_out) *zero_out = 0u;
  }
}


// Second level of a plain in-place exclusive scan (blocked: 4 consecutive items per thread).
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(uint32_t* __restrict__ data, Len len,
                                                       const uint32_t* __restrict__ bsums) {
  __shared__ uint32_t sm[33];
  const long long n = len.get();
  const long long base = (long long)blockIdx.x * TS_SCAN_ITEMS;
  if (base >= n) return;
  const long long i0 = base + (long long)threadIdx.x * SCAN_PER;
  uint32_t c[SCAN_PER];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    c[k] = (i0 + k < n) ? data[i0 + k] : 0u;
    s += c[k];
  }
  uint32_t tot;
  uint32_t off = block_excl_scan(s, sm, &tot) + bsums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    if (i0 + k < n) data[i0 + k] = off;
    off += c[k];
  }
}

// ---------------------------------------------------------------------------- tile segments
struct TileArgs {
  const uint32_t* count;
  const short4* rect;
  const uint32_t* zbits;
  const TsView* views;
  long long VM, M, cap, n_tiles;
  uint32_t* tcnt;                  // per tile: pair count (step 1)
  uint2* ranges;                   // per tile: [start, cursor) (steps 2-3), then [start, end)
  unsigned long long* seg;         // the segments' unsorted keys (cap entries)
  unsigned int* err;
};

// Step 1: one thread per (view, face); a face adds one to each tile of its rectangle.
__global__ void __launch_bounds__(256) k_tile_count(TileArgs a) {
  const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
  if (idx >= a.VM || a.count[idx] == 0) return;
  const int view = (int)(idx / a.M);
  const TsView& vw = a.views[view];
  const short4 r = a.rect[idx];
  for (int ty = r.y; ty <= r.w; ++ty) {
    const long long trow = vw.tile_off + (long long)ty * vw.TX;
    for (int tx = r.x; tx <= r.z; ++tx) atomicAdd(a.tcnt + trow + tx, 1u);
  }
}

// Step 2, second level: the exclusive scan of the counts, written as empty ranges [start, start).
__global__ void __launch_bounds__(SCAN_T) k_tile_starts(TileArgs a, const uint32_t* __restrict__ bsums) {
  __shared__ uint32_t sm[33];
  const long long n = a.n_tiles;
  const long long base = (long long)blockIdx.x * TS_SCAN_ITEMS;
  if (base >= n) return;
  const long long i0 = base + (long long)threadIdx.x * SCAN_PER;
  uint32_t c[SCAN_PER];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    c[k] = (i0 + k < n) ? a.tcnt[i0 + k] : 0u;
    s += c[k];
  }
  uint32_t tot;
  uint32_t off = block_excl_scan(s, sm, &tot) + bsums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    if (i0 + k < n) a.ranges[i0 + k] = make_uint2(off, off);
    off += c[k];
  }
}

// Step 3: one thread per (view, face); each of its tiles takes the next place of its segment.
// The places of up to four tiles are requested together (independent atomics in flight at
// once), and only then written.
__global__ void __launch_bounds__(256) k_tile_scatter(TileArgs a) {
  const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
  if (idx >= a.VM || a.count[idx] == 0) return;
  const int view = (int)(idx / a.M);
  const uint32_t face = (uint32_t)(idx - (long long)view * a.M);
  const TsView& vw = a.views[view];
  const short4 r = a.rect[idx];
  const unsigned long long key = ((unsigned long long)a.zbits[idx] << 32) | face;
  const int w = r.z - r.x + 1, h = r.w - r.y + 1;
  const long long t0 = vw.tile_off + (long long)r.y * vw.TX + r.x;
  if (w * h <= 4) {
    uint32_t pos[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int dy = k / w, dx = k - dy * w;  // w >= 1
      if (k < w * h) pos[k] = atomicAdd(&a.ranges[t0 + (long long)dy * vw.TX + dx].y, 1u);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < w * h && (long long)pos[k] < a.cap) a.seg[pos[k]] = key;  // beyond: capacity bit latched
    return;
  }
  for (int ty = r.y; ty <= r.w; ++ty) {
    const long long trow = vw.tile_off + (long long)ty * vw.TX;
    for (int tx = r.x; tx <= r.z; ++tx) {
      const uint32_t pos = atomicAdd(&a.ranges[trow + tx].y, 1u);
      if ((long long)pos < a.cap) a.seg[pos] = key;
    }
  }
}

// Steps 1-3 when every view's tiles fit in shared memory: one block per (block of TS_BIN_FACES
// faces, view) counts its pairs per tile in shared memory, and the exclusive scan of the
// [tile][face block] count matrix (tile-major) gives each block its first place in every tile's
// segment; the block then places its pairs with shared-memory atomics.
struct MatArgs {
  const uint32_t* count;
  const short4* rect;
  const uint32_t* zbits;
  const TsView* views;
  long long M, B, cap, n_tiles;
  uint32_t* mat;
  unsigned long long* seg;
  uint2* ranges;
  const unsigned long long* n_pairs;
};

constexpr int BIN_T = 1024;
constexpr int BIN_PER = TS_BIN_FACES / BIN_T;  // faces per thread
static_assert(TS_BIN_FACES % BIN_T == 0, "whole faces per thread");

__global__ void __launch_bounds__(BIN_T) k_bin_counts(MatArgs a) {
  extern __shared__ uint32_t hcnt[];
  const int v = blockIdx.y;
  const long long blk = blockIdx.x;
  const TsView& vw = a.views[v];
  const int T = vw.TX * vw.TY;
  for (int t = threadIdx.x; t < T; t += BIN_T) hcnt[t] = 0u;
  __syncthreads();
  const long long m0 = blk * TS_BIN_FACES + threadIdx.x;
  uint32_t cnt[BIN_PER];
  short4 rc[BIN_PER];
#pragma unroll
  for (int k = 0; k < BIN_PER; ++k) {  // all loads first, so that their latencies overlap
    const long long m = m0 + (long long)k * BIN_T;
    const long long idx = (long long)v * a.M + m;
    cnt[k] = m < a.M ? a.count[idx] : 0u;
    rc[k] = m < a.M ? a.rect[idx] : make_short4(0, 0, -1, -1);
  }
#pragma unroll
  for (int k = 0; k < BIN_PER; ++k) {
    if (cnt[k] == 0) continue;  // (an invisible face's rectangle is -1)
    const short4 r = rc[k];
    for (int ty = r.y; ty <= r.w; ++ty)
      for (int tx = r.x; tx <= r.z; ++tx) atomicAdd(&hcnt[ty * vw.TX + tx], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += BIN_T) a.mat[(vw.tile_off + t) * a.B + blk] = hcnt[t];
}

__global__ void __launch_bounds__(BIN_T) k_bin_place(MatArgs a) {
  extern __shared__ uint32_t place[];
  const int v = blockIdx.y;
  const long long blk = blockIdx.x;
  const TsView& vw = a.views[v];
  const int T = vw.TX * vw.TY;
  for (int t = threadIdx.x; t < T; t += BIN_T) place[t] = a.mat[(vw.tile_off + t) * a.B + blk];
  __syncthreads();
  const long long m0 = blk * TS_BIN_FACES + threadIdx.x;
  uint32_t cnt[BIN_PER], zb[BIN_PER];
  short4 rc[BIN_PER];
#pragma unroll
  for (int k = 0; k < BIN_PER; ++k) {  // all loads first, so that their latencies overlap
    const long long m = m0 + (long long)k * BIN_T;
    const long long idx = (long long)v * a.M + m;
    cnt[k] = m < a.M ? a.count[idx] : 0u;
    rc[k] = m < a.M ? a.rect[idx] : make_short4(0, 0, -1, -1);
    zb[k] = m < a.M ? a.zbits[idx] : 0u;
  }
#pragma unroll
  for (int k = 0; k < BIN_PER; ++k) {
    if (cnt[k] == 0) continue;  // (an invisible face's rectangle is -1)
    const short4 r = rc[k];
    const unsigned long long key = ((unsigned long long)zb[k] << 32) | (uint32_t)(m0 + (long long)k * BIN_T);
    for (int ty = r.y; ty <= r.w; ++ty)
      for (int tx = r.x; tx <= r.z; ++tx) {
        const uint32_t pos = atomicAdd(&place[ty * vw.TX + tx], 1u);
        if ((long long)pos < a.cap) a.seg[pos] = key;  // beyond: the scan has latched the capacity bit
      }
  }
}

// Step 4.  Bitonic networks in the form whose every compare-exchange moves the smaller key to the
// lower index (each merge starts by comparing mirrored positions), so that the positions past a
// segment's end can stand for +infinity without being stored: a pair with one of them never moves.
struct SortOut {
  const unsigned long long* seg;
  unsigned long long* keys;
  uint32_t* vals;
  uint2* ranges;           // cut to the capacity here
  long long n_tiles, cap;
  uint32_t* large;         // tiles left to the CTA-wide sort
  unsigned int* n_large;
  const uint32_t* mat;     // the scanned [tile][face block] count matrix, or null: ranges from the scatter
  long long B;             // face blocks per tile row of the matrix
  const unsigned long long* n_pairs;
};

__device__ __forceinline__ void put_pair(const SortOut& o, long long t, long long pos, unsigned long long k) {
  o.keys[pos] = ((unsigned long long)t << 32) | (k >> 32);
  o.vals[pos] = (uint32_t)k;
}

constexpr int WARP_SORT_MAX = 512;  // pairs a warp sorts in its shared memory (32 KB per block)
constexpr int SORT_WARPS_PER_BLOCK = 8;

// One warp per tile: up to 32 pairs in registers, up to WARP_SORT_MAX in shared memory; longer
// segments are listed for the CTA-wide kernel.
__global__ void __launch_bounds__(32 * SORT_WARPS_PER_BLOCK) k_tile_sort(SortOut o) {
  __shared__ unsigned long long sbuf[SORT_WARPS_PER_BLOCK][WARP_SORT_MAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long t = (long long)blockIdx.x * SORT_WARPS_PER_BLOCK + warp;
  if (t >= o.n_tiles) return;
  // the segment: from the scanned matrix (its first block's place, the next tile's, the pair total
  // after the last tile), else as the scatter left it in ranges
  uint2 rg;
  if (o.mat) {
    rg.x = o.mat[t * o.B];
    rg.y = t + 1 < o.n_tiles ? o.mat[(t + 1) * o.B] : (uint32_t)min(*o.n_pairs, 0xffffffffull);
  } else {
    rg = o.ranges[t];
  }
  const long long start = min((long long)rg.x, o.cap);
  const long long end = min((long long)rg.y, o.cap);
  // the tile's range for the passes that follow; past the capacity (its bit is latched) the lists
  // are cut, and the ranges with them, so that no later pass reads outside the pair list
  if (lane == 0 && (o.mat || (long long)rg.y > o.cap)) o.ranges[t] = make_uint2((uint32_t)start, (uint32_t)end);
  const int n = (int)max(0LL, end - start);
  if (n == 0) return;
  if (n <= 32) {
    unsigned long long x = lane < n ? o.seg[start + lane] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
      {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, k - 1);
        const bool lower = (lane & (k >> 1)) == 0;
        x = lower ? min(x, y) : max(x, y);
      }
#pragma unroll
      for (int j = k >> 2; j > 0; j >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
        const bool lower = (lane & j) == 0;
        x = lower ? min(x, y) : max(x, y);
      }
    }
    if (lane < n) put_pair(o, t, start + lane, x);
    return;
  }
  if (n <= 64) {  // two keys per lane: x0 at position lane, x1 at position 32 + lane
    unsigned long long x0 = o.seg[start + lane];
    unsigned long long x1 = 32 + lane < n ? o.seg[start + 32 + lane] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {  // each half sorted as in the 32-key network
      {
        const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, x0, k - 1);
        const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, x1, k - 1);
        const bool lower = (lane & (k >> 1)) == 0;
        x0 = lower ? min(x0, y0) : max(x0, y0);
        x1 = lower ? min(x1, y1) : max(x1, y1);
      }
#pragma unroll
      for (int j = k >> 2; j > 0; j >>= 1) {
        const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, x0, j);
        const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, x1, j);
        const bool lower = (lane & j) == 0;
        x0 = lower ? min(x0, y0) : max(x0, y0);
        x1 = lower ? min(x1, y1) : max(x1, y1);
      }
    }
    {  // merge of 64: position lane pairs with 63 - lane, i.e. x1 of lane 31 - lane
      const unsigned long long y0 = __shfl_sync(0xffffffffu, x1, 31 - lane);
      const unsigned long long y1 = __shfl_sync(0xffffffffu, x0, 31 - lane);
      x0 = min(x0, y0);
      x1 = max(x1, y1);
    }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
      const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, x0, j);
      const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, x1, j);
      const bool lower = (lane & j) == 0;
      x0 = lower ? min(x0, y0) : max(x0, y0);
      x1 = lower ? min(x1, y1) : max(x1, y1);
    }
    put_pair(o, t, start + lane, x0);
    if (32 + lane < n) put_pair(o, t, start + 32 + lane, x1);
    return;
  }
  if (n > WARP_SORT_MAX) {
    if (lane == 0) {
      const unsigned slot = atomicAdd(o.n_large, 1u);
      if ((long long)slot < o.n_tiles) o.large[slot] = (uint32_t)t;
    }
    return;
  }
  unsigned long long* s = sbuf[warp];
  for (int i = lane; i < n; i += 32) s[i] = o.seg[start + i];
  __syncwarp();
  int P = 64;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = lane; q < P / 2; q += 32) {
        const int blk = q / j, off = q - blk * j;
        const int i = blk * 2 * j + off;
        // the merge's first step pairs mirrored positions of its block of k, then half-cleaners
        const int l = (j == (k >> 1)) ? (i / k) * k + k - 1 - (i % k) : i + j;
        if (l < n) {
          const unsigned long long u = s[i], v = s[l];
          if (v < u) {
            s[i] = v;
            s[l] = u;
          }
        }
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < n; i += 32) put_pair(o, t, start + i, s[i]);
}

constexpr int LARGE_T = 1024;
constexpr int LARGE_SMEM_ITEMS = 16384;  // 128 KB of keys

// The listed long segments, one CTA each (grid-stride over the list): in shared memory up to
// LARGE_SMEM_ITEMS pairs, else in place in the segment buffer.
__global__ void __launch_bounds__(LARGE_T) k_tile_sort_large(SortOut o, unsigned long long* seg) {
  extern __shared__ __align__(16) unsigned long long lbuf[];
  const unsigned nl = min(*o.n_large, (unsigned)o.n_tiles);
  for (unsigned w = blockIdx.x; w < nl; w += gridDim.x) {
    const long long t = o.large[w];
    const uint2 rg = o.ranges[t];  // already cut to the capacity
    const long long start = rg.x;
    const long long end = rg.y;
    const long long n = end - start;
    const bool in_smem = n <= LARGE_SMEM_ITEMS;
    unsigned long long* s = in_smem ? lbuf : seg + start;
    if (in_smem)
      for (long long i = threadIdx.x; i < n; i += LARGE_T) s[i] = seg[start + i];
    __syncthreads();
    long long P = 1;
    while (P < n) P <<= 1;
    for (long long k = 2; k <= P; k <<= 1) {
      for (long long j = k >> 1; j > 0; j >>= 1) {
        for (long long q = threadIdx.x; q < P / 2; q += LARGE_T) {
          const long long blk = q / j, off = q - blk * j;
          const long long i = blk * 2 * j + off;
          const long long l = (j == (k >> 1)) ? (i / k) * k + k - 1 - (i % k) : i + j;
          if (l < n) {
            const unsigned long long u = s[i], v = s[l];
            if (v < u) {
              s[i] = v;
              s[l] = u;
            }
          }
        }
        __syncthreads();
      }
    }
    for (long long i = threadIdx.x; i < n; i += LARGE_T) put_pair(o, t, start + i, s[i]);
    __syncthreads();
  }
}

}  // namespace

cudaError_t ts_launch_bin(const TsPlanImpl* p, const TsWs& w, cudaStream_t s) {
  const long long VM = (long long)p->V * p->M;
  cudaError_t e = cudaSuccess;
  if (VM == 0) {  // no records: empty ranges and no pairs (otherwise the kernels below write them)
    e = cudaMemsetAsync(w.ranges, 0, (size_t)p->n_tiles * sizeof(uint2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&w.hdr->n_large, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&w.hdr->n_pairs, 0, sizeof(unsigned long long), s);
    return e;
  }
  if (p->bin_blocks > 0) {
    // 1-3 with shared-memory counts: counts, their scan (the total is the pair count; above the
    // capacity latches its bit), places, ranges
    MatArgs ma{w.count, w.rect, w.zbits, w.views, p->M, p->bin_blocks, p->cap, p->n_tiles, w.tmat, w.keys[1],
               w.ranges, &w.hdr->n_pairs};
    const int smem = (int)(p->max_view_tiles * sizeof(uint32_t));
    e = ts_smem_limit((const void*)k_bin_counts, smem);
    if (e == cudaSuccess) e = ts_smem_limit((const void*)k_bin_place, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)p->bin_blocks, (unsigned)p->V);
    k_bin_counts<<<grid, BIN_T, smem, s>>>(ma);
    Len lm{p->n_tiles * p->bin_blocks};
    const unsigned nb = (unsigned)((lm.n + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS);
    k_scan_reduce<<<nb, SCAN_T, 0, s>>>(w.tmat, lm, w.bsums);
    k_scan_bsums<<<1, SCAN_T, 0, s>>>(w.bsums, lm, &w.hdr->n_pairs, &w.hdr->error_bits, p->cap, &w.hdr->n_large);
    k_scan_apply<<<nb, SCAN_T, 0, s>>>(w.tmat, lm, w.bsums);
    k_bin_place<<<grid, BIN_T, smem, s>>>(ma);
  } else {
    // 1-3 with global counts: counts, their scan, starts, places
    e = cudaMemsetAsync(w.tcnt, 0, (size_t)p->n_tiles * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    TileArgs ta{w.count, w.rect, w.zbits, w.views, VM, p->M, p->cap, p->n_tiles, w.tcnt, w.ranges, w.keys[1],
                &w.hdr->error_bits};
    const unsigned nf = (unsigned)((VM + 255) / 256);
    k_tile_count<<<nf, 256, 0, s>>>(ta);
    Len lt{p->n_tiles};
    const unsigned nb = (unsigned)((p->n_tiles + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS);
    k_scan_reduce<<<nb, SCAN_T, 0, s>>>(w.tcnt, lt, w.bsums);
    k_scan_bsums<<<1, SCAN_T, 0, s>>>(w.bsums, lt, &w.hdr->n_pairs, &w.hdr->error_bits, p->cap, &w.hdr->n_large);
    k_tile_starts<<<nb, SCAN_T, 0, s>>>(ta, w.bsums);
    k_tile_scatter<<<nf, 256, 0, s>>>(ta);
  }
  // 4: the segments' sorts
  // (with the matrix, the sort also writes each tile's range)
  SortOut so{w.keys[1], w.keys[0], w.vals[0], w.ranges, p->n_tiles, p->cap, w.tlarge, &w.hdr->n_large,
             p->bin_blocks > 0 ? w.tmat : nullptr, p->bin_blocks, &w.hdr->n_pairs};
  k_tile_sort<<<(unsigned)((p->n_tiles + SORT_WARPS_PER_BLOCK - 1) / SORT_WARPS_PER_BLOCK), 32 * SORT_WARPS_PER_BLOCK,
                0, s>>>(so);
  e = ts_smem_limit((const void*)k_tile_sort_large, (int)(LARGE_SMEM_ITEMS * sizeof(unsigned long long)));
  if (e != cudaSuccess) return e;
  k_tile_sort_large<<<(unsigned)ts_sm_count(), LARGE_T, LARGE_SMEM_ITEMS * sizeof(unsigned long long), s>>>(so, w.keys[1]);
  return cudaGetLastError();
}
