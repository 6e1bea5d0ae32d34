// k_bin.cu -- depth ordering per tile (Eq. 4: faces are composited in depth order).
//
//  1. exclusive scan of the tiles each (view, face) touches (two-level, 4096 items per block);
//  2. emission of one 64-bit key (global tile id << 32 | float bits of the depth key) and a
//     face-id value per touched tile, in (view, face) order;
//  3. a stable LSD radix sort over the key bits in use (31 depth bits -- a positive depth's sign
//     bit is 0 -- and ceil(log2 tiles) tile bits, 8 bits per pass): per-block digit histograms,
//     a scan of the digit-major histogram, and a scatter whose in-block ranks come from
//     warp-level match masks, so that equal keys keep emission order (ascending face id); the
//     block first reorders its keys by digit in shared memory so that each digit's run is
//     written to global memory contiguously;
//  4. per-tile [start, end) ranges.
// Every kernel reads the pair count from the device, so nothing here synchronises the host.
#include <algorithm>

#include "ts_internal.cuh"

namespace {

// Digit of a (tile << 32 | depth bits) key for an LSD pass starting at bit `shift` of the key with
// bit 31 removed: visible faces have positive depth, so that bit is always 0 and 31 + ceil(log2
// tiles) bits order the keys exactly as all 64 do.
__device__ __forceinline__ uint32_t key_digit(unsigned long long key, int shift) {
  const unsigned long long packed = ((key >> 32) << 31) | (key & 0x7fffffffull);
  return (uint32_t)(packed >> shift) & 255u;
}

constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = TS_SCAN_ITEMS / SCAN_T;  // 4

// length of a scanned array: a constant, or the digit-major histogram of the current sort
struct Len {
  long long n;                         // used when pairs == nullptr
  const unsigned long long* pairs;     // device pair counter
  long long cap;
  __device__ __forceinline__ long long get() const {
    if (!pairs) return n;
    const long long np = (long long)min(*pairs, (unsigned long long)cap);
    return 256LL * ((np + TS_SORT_ITEMS - 1) / TS_SORT_ITEMS);
  }
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

// Exclusive scan of the block sums in place (one block); writes the grand total.
__global__ void __launch_bounds__(SCAN_T) k_scan_bsums(uint32_t* bsums, Len len, unsigned long long* total_out,
                                                       unsigned int* err, long long cap) {
  __shared__ uint32_t sm[33];
  const long long n = len.get();
  const long long nb = (n + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS;
  const long long per = (nb + SCAN_T - 1) / SCAN_T;
  const long long b0 = (long long)threadIdx.x * per;
  unsigned long long s = 0;
  for (long long i = b0; i < b0 + per && i < nb; ++i) s += bsums[i];
  uint32_t tot;
  uint32_t run = block_excl_scan((uint32_t)s, sm, &tot);
  // the 64-bit total guards against overflow of the 32-bit running offsets
  __shared__ unsigned long long tot64;
  if (threadIdx.x == 0) tot64 = 0;
  __syncthreads();
  atomicAdd(&tot64, s);
  __syncthreads();
  for (long long i = b0; i < b0 + per && i < nb; ++i) {
    const uint32_t v = bsums[i];
    bsums[i] = run;
    run += v;
  }
  if (threadIdx.x == 0 && total_out) {
    *total_out = tot64;
    if ((long long)tot64 > cap) atomicOr(err, TS_ERRBIT_CAPACITY);
  }
}

// Second level of the scan of tiles touched, fused with key emission.
struct EmitArgs {
  const uint32_t* count;
  const short4* rect;
  const uint32_t* zbits;
  const uint32_t* bsums;
  const TsView* views;
  long long VM, M, cap;
  unsigned long long* keys;
  uint32_t* vals;
  uint32_t* offs;
};

__global__ void __launch_bounds__(SCAN_T) k_scan_emit(EmitArgs a) {
  __shared__ uint32_t sm[33];
  const long long base = (long long)blockIdx.x * TS_SCAN_ITEMS;
  if (base >= a.VM) return;
  // blocked layout: thread t owns items base + 4t .. base + 4t + 3 (consecutive faces)
  const long long i0 = base + (long long)threadIdx.x * SCAN_PER;
  uint32_t c[SCAN_PER];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    c[k] = (i0 + k < a.VM) ? a.count[i0 + k] : 0u;
    s += c[k];
  }
  uint32_t tot;
  uint32_t off = block_excl_scan(s, sm, &tot) + a.bsums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    const long long idx = i0 + k;
    if (idx < a.VM) a.offs[idx] = off;
    if (c[k]) {
      const int view = (int)(idx / a.M);
      const uint32_t face = (uint32_t)(idx - (long long)view * a.M);
      const TsView& vw = a.views[view];
      const short4 r = a.rect[idx];
      const unsigned long long zb = a.zbits[idx];
      long long pos = off;
      for (int ty = r.y; ty <= r.w; ++ty) {
        const long long trow = vw.tile_off + (long long)ty * vw.TX;
        for (int tx = r.x; tx <= r.z; ++tx, ++pos) {
          if (pos < a.cap) {
            a.keys[pos] = ((unsigned long long)(trow + tx) << 32) | zb;
            a.vals[pos] = face;
          }
        }
      }
    }
    off += c[k];
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

// ------------------------------------------------------------------------------ radix sort
struct SortArgs {
  const unsigned long long* keys_in;
  const uint32_t* vals_in;
  unsigned long long* keys_out;
  uint32_t* vals_out;
  const unsigned long long* n_pairs;
  long long cap;
  int shift;
  uint32_t* hist;  // digit-major [256][nbs]
  unsigned int* err;
};

__device__ __forceinline__ void sort_sizes(const SortArgs& a, long long* n, long long* nbs) {
  *n = (long long)min(*a.n_pairs, (unsigned long long)a.cap);
  *nbs = (*n + TS_SORT_ITEMS - 1) / TS_SORT_ITEMS;
}

__global__ void __launch_bounds__(TS_SORT_THREADS) k_radix_upsweep(SortArgs a) {
  __shared__ uint32_t h[256];
  long long n, nbs;
  sort_sizes(a, &n, &nbs);
  if (blockIdx.x >= nbs) return;
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * TS_SORT_ITEMS;
  const int lane = threadIdx.x & 31;
#pragma unroll 4
  for (int j = 0; j < TS_SORT_ITEMS / TS_SORT_THREADS; ++j) {
    const long long i = base + (long long)j * TS_SORT_THREADS + threadIdx.x;
    const bool ok = i < n;
    const uint32_t d = ok ? key_digit(a.keys_in[i], a.shift) : 256u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  a.hist[(long long)threadIdx.x * nbs + blockIdx.x] = h[threadIdx.x];
}

constexpr int SORT_WARPS = TS_SORT_THREADS / 32;         // 8
constexpr int SORT_ROUNDS = TS_SORT_ITEMS / TS_SORT_THREADS;  // 16: items per lane

// Dynamic shared memory of the downsweep: the block's keys and values reordered by digit.
constexpr size_t DOWNSWEEP_SMEM = (size_t)TS_SORT_ITEMS * (sizeof(unsigned long long) + sizeof(uint32_t));

__global__ void __launch_bounds__(TS_SORT_THREADS) k_radix_downsweep(SortArgs a) {
  extern __shared__ __align__(16) unsigned char sbuf[];
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(sbuf);
  uint32_t* sval = reinterpret_cast<uint32_t*>(sbuf + (size_t)TS_SORT_ITEMS * sizeof(unsigned long long));
  __shared__ uint32_t wc[SORT_WARPS][256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t doff[256];       // start of each digit's run in the block's reordered keys
  __shared__ uint32_t wsum[SORT_WARPS];
  long long n, nbs;
  sort_sizes(a, &n, &nbs);
  if (blockIdx.x >= nbs) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < SORT_WARPS * 256; i += TS_SORT_THREADS) (&wc[0][0])[i] = 0;
  gbase[threadIdx.x] = a.hist[(long long)threadIdx.x * nbs + blockIdx.x];
  __syncthreads();
  // each warp ranks a contiguous chunk of 512 keys in 16 rounds of 32
  const long long bbase = (long long)blockIdx.x * TS_SORT_ITEMS;
  const long long wbase = bbase + (long long)warp * (32 * SORT_ROUNDS);
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long key[SORT_ROUNDS];
  uint32_t val[SORT_ROUNDS];
  uint32_t rank[SORT_ROUNDS];
#pragma unroll
  for (int r = 0; r < SORT_ROUNDS; ++r) {
    const long long i = wbase + r * 32 + lane;
    const bool ok = i < n;
    key[r] = ok ? a.keys_in[i] : 0ull;
    val[r] = ok ? a.vals_in[i] : 0u;
    const uint32_t d = ok ? key_digit(key[r], a.shift) : 256u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = ok ? wc[warp][d] : 0u;
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wc[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = ok ? before + __popc(peers & lt) : 0xffffffffu;
  }
  __syncthreads();
  // digit-wise exclusive prefix over warps (in warp order = index order), and the block's count
  // of each digit
  uint32_t total;
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
      const uint32_t c = wc[w][d];
      wc[w][d] = run;
      run += c;
    }
    total = run;
  }
  // exclusive scan of the digit counts over the 256 digits (thread d = digit d)
  {
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w)
      if (w < warp) wpre += wsum[w];
    doff[threadIdx.x] = wpre + x - total;
  }
  __syncthreads();
  // reorder by digit in shared memory
#pragma unroll
  for (int r = 0; r < SORT_ROUNDS; ++r) {
    if (rank[r] == 0xffffffffu) continue;
    const uint32_t d = key_digit(key[r], a.shift);
    const uint32_t lp = doff[d] + wc[warp][d] + rank[r];
    skey[lp] = key[r];
    sval[lp] = val[r];
  }
  __syncthreads();
  // write each digit's run to its place: consecutive threads write consecutive addresses
  const int nb = (int)min((long long)TS_SORT_ITEMS, n - bbase);
  for (int i = threadIdx.x; i < nb; i += TS_SORT_THREADS) {
    const unsigned long long k = skey[i];
    const uint32_t d = key_digit(k, a.shift);
    const long long dst = (long long)gbase[d] + (i - (long long)doff[d]);
    if (dst < n) {
      a.keys_out[dst] = k;
      a.vals_out[dst] = sval[i];
    } else {
      atomicOr(a.err, TS_ERRBIT_BOUNDS);
    }
  }
}

__global__ void k_ranges(const unsigned long long* __restrict__ keys, const unsigned long long* n_pairs, long long cap,
                         uint2* __restrict__ ranges, long long n_tiles, unsigned int* err) {
  const long long n = (long long)min(*n_pairs, (unsigned long long)cap);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if ((long long)t >= n_tiles) {
      atomicOr(err, TS_ERRBIT_BOUNDS);
      continue;
    }
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

}  // namespace

int ts_sort_final_buffer(const TsPlanImpl* p) { return p->sort_passes & 1; }

cudaError_t ts_launch_bin(const TsPlanImpl* p, const TsWs& w, cudaStream_t s) {
  const long long VM = (long long)p->V * p->M;
  cudaError_t e = cudaMemsetAsync(w.ranges, 0, (size_t)p->n_tiles * sizeof(uint2), s);
  if (e != cudaSuccess || VM == 0) return e;
  // 1-2: scan of tiles touched, fused emission
  Len lvm{VM, nullptr, 0};
  const unsigned nb = (unsigned)p->n_scan_blocks;
  k_scan_reduce<<<nb, SCAN_T, 0, s>>>(w.count, lvm, w.bsums);
  k_scan_bsums<<<1, SCAN_T, 0, s>>>(w.bsums, lvm, &w.hdr->n_pairs, &w.hdr->error_bits, p->cap);
  EmitArgs ea{w.count, w.rect, w.zbits, w.bsums, w.views, VM, p->M, p->cap, w.keys[0], w.vals[0], w.offs};
  k_scan_emit<<<nb, SCAN_T, 0, s>>>(ea);
  // 3: radix sort over the key bits in use
  const unsigned nbs = (unsigned)p->n_sort_blocks_cap;
  const long long hist_len = 256LL * p->n_sort_blocks_cap;
  const unsigned nbh = (unsigned)((hist_len + TS_SCAN_ITEMS - 1) / TS_SCAN_ITEMS);
  Len lh{0, &w.hdr->n_pairs, p->cap};
  {
    const cudaError_t e = ts_smem_limit((const void*)k_radix_downsweep, (int)DOWNSWEEP_SMEM);
    if (e != cudaSuccess) return e;
  }
  for (int pass = 0; pass < p->sort_passes; ++pass) {
    const int in = pass & 1;
    SortArgs sa{w.keys[in], w.vals[in], w.keys[in ^ 1], w.vals[in ^ 1], &w.hdr->n_pairs, p->cap, 8 * pass, w.hist,
                &w.hdr->error_bits};
    k_radix_upsweep<<<nbs, TS_SORT_THREADS, 0, s>>>(sa);
    k_scan_reduce<<<nbh, SCAN_T, 0, s>>>(w.hist, lh, w.hsums);
    k_scan_bsums<<<1, SCAN_T, 0, s>>>(w.hsums, lh, nullptr, nullptr, 0);
    k_scan_apply<<<nbh, SCAN_T, 0, s>>>(w.hist, lh, w.hsums);
    k_radix_downsweep<<<nbs, TS_SORT_THREADS, DOWNSWEEP_SMEM, s>>>(sa);
  }
  // 4: tile ranges over the sorted keys
  const int fb = ts_sort_final_buffer(p);
  const long long grid = std::min<long long>((p->cap + 255) / 256, 152LL * 16);
  k_ranges<<<(unsigned)grid, 256, 0, s>>>(w.keys[fb], &w.hdr->n_pairs, p->cap, w.ranges, p->n_tiles,
                                          &w.hdr->error_bits);
  return cudaGetLastError();
}
