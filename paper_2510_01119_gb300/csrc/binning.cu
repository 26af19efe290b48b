// Tile binning: exclusive scan of per-record tile counts, key emission, a stable LSD radix sort of
// (tile << 32 | depth bits, Gaussian id) pairs, and per-tile [start, end) ranges.
//
// Every kernel reads the pair count from device memory (never from the host), so the whole
// binning step can sit inside a captured CUDA graph; grids are sized for the capacity and blocks
// beyond the live count return at once.
#include <algorithm>

#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;                       // per thread per round
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096
constexpr int kScanMaxBlocks = 1024;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// block-wide exclusive scan of one value per thread (blockDim.x == 1024); returns the block total
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t x, uint64_t& excl) {
  __shared__ uint64_t wsum[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t inc = warp_incl_scan(x);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint64_t s = wsum[lane];
    const uint64_t si = warp_incl_scan(s);
    wsum[lane] = si - s;
    if (lane == 31) wsum[32] = si;
  }
  __syncthreads();
  excl = wsum[warp] + inc - x;
  const uint64_t total = wsum[32];
  __syncthreads();
  return total;
}

// Element loaders of the scan: the value itself, or 1 for a nonzero value.
struct LoadPlain {
  const uint32_t* p;
  __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct LoadNonzero {
  const uint32_t* p;
  __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i] != 0u ? 1u : 0u; }
};

template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(Load in, const int64_t* __restrict__ n_dev,
                                                                   int64_t n_max, int64_t chunk,
                                                                   uint64_t* __restrict__ bsum) {
  const int64_t n = n_dev ? min(*n_dev, n_max) : n_max;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(lo + chunk, n);
  uint64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += in(i);
  __shared__ uint64_t red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t t = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(Load in, uint32_t* __restrict__ out,
                                                                 const int64_t* __restrict__ n_dev, int64_t n_max,
                                                                 int64_t chunk, const uint64_t* __restrict__ bsum,
                                                                 int64_t* __restrict__ total_out) {
  const int64_t n = n_dev ? min(*n_dev, n_max) : n_max;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(lo + chunk, n);
  uint64_t carry;
  {
    __shared__ uint64_t red[32];
    uint64_t x = (threadIdx.x < blockIdx.x) ? bsum[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    x = red[threadIdx.x & 31];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    carry = x;
    __syncthreads();
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = (int64_t)(carry + bsum[blockIdx.x]);
  for (int64_t base = lo; base < hi; base += kScanTile) {
    uint32_t v[kScanItems];
    uint64_t s = 0;
    const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (i0 + k < hi) ? in(i0 + k) : 0u;
      s += v[k];
    }
    uint64_t ex;
    const uint64_t tot = block_excl_scan(s, ex);
    uint64_t run = carry + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (i0 + k < hi) out[i0 + k] = (uint32_t)run;
      run += v[k];
    }
    carry += tot;
  }
}

void scan_geometry(int64_t n, int& nb, int64_t& chunk) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  nb = (int)(tiles < kScanMaxBlocks ? tiles : kScanMaxBlocks);
  const int64_t tiles_per_block = (tiles + nb - 1) / nb;
  chunk = tiles_per_block * kScanTile;
  nb = (int)((n + chunk - 1) / chunk);
  if (nb < 1) nb = 1;
}

// ---- visible records, emission in depth order ----------------------------------------------------
// keys[k] = float bits of the depth of the k-th visible record (records in index order), vals[k] = r
__global__ void __launch_bounds__(256) visible_compact_kernel(int64_t VN, const float4* __restrict__ proj,
                                                              const uint32_t* __restrict__ touched,
                                                              const uint32_t* __restrict__ offs,
                                                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= VN || touched[r] == 0) return;
  const uint32_t k = offs[r];
  keys[k] = __float_as_uint(proj[4 * r + 3].z);  // positive depths: float bits order as the values
  vals[k] = (uint32_t)r;
}

// Every (tile, Gaussian) pair of the k-th depth-ordered record's rectangle, at offs[k]: key = global
// tile index, value = Gaussian id.  A warp emits its 32 records' pairs together, 32 consecutive
// outputs per round: each lane finds the record that owns its output by a binary search over the
// warp's inclusive prefix of the records' pair counts, so long and short rectangles cost the same
// and every store is coalesced.
__global__ void __launch_bounds__(256) emit_sorted_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                          const int64_t* __restrict__ R_dev,
                                                          const uint32_t* __restrict__ rec,
                                                          const uint32_t* __restrict__ offs, int64_t capacity,
                                                          uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t R = *R_dev;
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k - lane >= R) return;  // the whole warp is past the last record
  int cnt = 0, x0 = 0, y0 = 0, w = 1, txs = 0;
  uint32_t id = 0, tbase = 0;
  int64_t o = 0;
  if (k < R) {
    const uint32_t r = rec[k];
    const int v = (int)(r / (uint32_t)n);
    id = r - (uint32_t)v * (uint32_t)n;
    int x1, y1;
    box_rect(proj[4 * (size_t)r], vt.width[v], vt.height[v], vt.tile_w, vt.tile_h, vt.tiles_x[v], vt.tiles_y[v], x0,
             y0, x1, y1);
    if (x1 > x0 && y1 > y0) {
      w = x1 - x0;
      cnt = w * (y1 - y0);
    }
    o = offs[k];
    tbase = (uint32_t)vt.tile_off[v];
    txs = vt.tiles_x[v];
  }
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int excl = incl - cnt;
  for (int s0 = 0; s0 < total; s0 += 32) {  // warp-uniform
    const int s = s0 + lane;
    // owner: the number of lanes whose inclusive count is <= s (counts are nonnegative)
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int t = __shfl_sync(0xffffffffu, incl, j + step - 1);
      if (t <= s) j += step;
    }
    const int loc = s - __shfl_sync(0xffffffffu, excl, j);
    const int wj = __shfl_sync(0xffffffffu, w, j);
    const int x0j = __shfl_sync(0xffffffffu, x0, j), y0j = __shfl_sync(0xffffffffu, y0, j);
    const int txj = __shfl_sync(0xffffffffu, txs, j);
    const uint32_t tbj = __shfl_sync(0xffffffffu, tbase, j), idj = __shfl_sync(0xffffffffu, id, j);
    const int64_t oj = __shfl_sync(0xffffffffu, o, j);
    if (s < total) {
      const int dy = loc / wj, dx = loc - dy * wj;
      const int64_t out = oj + loc;
      if (out < capacity) {
        keys[out] = tbj + (uint32_t)((y0j + dy) * txj + x0j + dx);
        vals[out] = idj;
      }
    }
  }
}

// ---- radix sort ---------------------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsBins = 256;
static_assert(kRsThreads == kRsBins, "one thread per digit in the scatter's digit scan");

// Keys per thread and per block: the scatter stages a block's keys and values in shared memory,
// 8 KB + 8 KB for 32-bit keys, 16 KB + 8 KB for 64-bit ones.  Eight keys per thread rather than
// sixteen: twice the blocks, and the scatter's 0.75 ms per training step on the 1.13M-Gaussian
// workload falls to 0.60 ms for 0.06 ms more in the histograms and their scans.
template <class K>
struct RsCfg {
  static constexpr int kItems = 8;
  static constexpr int kTile = kRsThreads * kItems;
};
constexpr int kRsMinTile = RsCfg<uint64_t>::kTile;  // workspace sizes hold for either key width

__device__ __forceinline__ int64_t live_count(const int64_t* n_dev, int64_t capacity) {
  const int64_t n = *n_dev;
  return n < capacity ? n : capacity;
}

template <class K>
__global__ void __launch_bounds__(kRsThreads) radix_hist_kernel(const K* __restrict__ keys,
                                                                const int64_t* __restrict__ n_dev, int64_t capacity,
                                                                int shift, int nblocks, uint32_t* __restrict__ hist) {
  constexpr int kTile = RsCfg<K>::kTile;
  __shared__ uint32_t h[kRsWarps][kRsBins];
  for (int k = threadIdx.x; k < kRsWarps * kRsBins; k += kRsThreads) (&h[0][0])[k] = 0;
  __syncthreads();
  const int64_t n = live_count(n_dev, capacity);
  const int64_t lo = (int64_t)blockIdx.x * kTile;
  const int warp = threadIdx.x >> 5;
  if (lo < n) {
    const int64_t hi = min(lo + (int64_t)kTile, n);
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRsThreads) {
      const uint32_t d = (uint32_t)(keys[i] >> shift) & 0xffu;
      atomicAdd(&h[warp][d], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRsBins; d += kRsThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) s += h[w][d];
    hist[(int64_t)d * nblocks + blockIdx.x] = s;
  }
}

// Stable scatter: warp w ranks the keys of its contiguous segment in order, using warp-private digit
// counters; per digit, an exclusive scan over the warps places each warp's keys after those of the
// earlier warps.  The block's keys and values are then laid out digit-major in shared memory and
// written out by consecutive threads, so each digit's run of the block goes to consecutive
// addresses (after the scanned histogram's offset for the block).
// Compiled for 4 resident blocks per SM (at most 64 registers): the kernel waits on memory, and 32
// warps hide more of it than 24 (0.60 against 0.69 ms per step with 8 keys per thread).
// kgather (nullable): write kgather[value] in place of each key (the last pass of a sort whose
// sorted keys are not needed but a per-value quantity is, in sorted order).
template <class K>
__global__ void __launch_bounds__(kRsThreads, 4) radix_scatter_kernel(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, const int64_t* __restrict__ n_dev, int64_t capacity, int shift, int nblocks,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ kgather) {
  constexpr int kItems = RsCfg<K>::kItems, kTile = RsCfg<K>::kTile;
  __shared__ uint32_t cnt[kRsWarps][kRsBins];
  __shared__ uint32_t dstart[kRsBins];  // first slot of each digit in the block's digit-major layout
  __shared__ uint32_t gbase[kRsBins];   // output position of that slot
  __shared__ uint32_t wtot[kRsWarps];
  __shared__ K skey[kTile];
  __shared__ uint32_t sval[kTile];
  const int64_t n = live_count(n_dev, capacity);
  const int64_t lo = (int64_t)blockIdx.x * kTile;
  if (lo >= n) return;  // uniform per block
  for (int k = threadIdx.x; k < kRsWarps * kRsBins; k += kRsThreads) (&cnt[0][0])[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t seg = lo + (int64_t)warp * (32 * kItems);
  K key[kItems];
  uint32_t val[kItems];
  uint32_t rank[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = seg + j * 32 + lane;
    const bool ok = i < n;
    key[j] = ok ? kin[i] : (K)0;
    val[j] = ok ? vin[i] : 0u;
    const uint32_t d = ok ? ((uint32_t)(key[j] >> shift) & 0xffu) : 0x100u;  // 256 = padding
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = (d < 256u) ? cnt[warp][d] : 0u;
    __syncwarp();
    rank[j] = before + __popc(peers & lt_mask);
    if (d < 256u && (peers & lt_mask) == 0) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread d: exclusive scan of digit d over the warps, then of the block's digit totals over d
    const int d = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = tot;
      tot += c;
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    gbase[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) before += (w < warp) ? wtot[w] : 0u;
    dstart[d] = before + incl - tot;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = seg + j * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(key[j] >> shift) & 0xffu;
      const uint32_t s = dstart[d] + cnt[warp][d] + rank[j];
      skey[s] = key[j];
      sval[s] = val[j];
    }
  }
  __syncthreads();
  const int count = (int)min((int64_t)kTile, n - lo);
  for (int s = threadIdx.x; s < count; s += kRsThreads) {
    const K k = skey[s];
    const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
    const uint32_t pos = gbase[d] + ((uint32_t)s - dstart[d]);
    const uint32_t v = sval[s];
    kout[pos] = kgather ? (K)kgather[v] : k;
    vout[pos] = v;
  }
}

// ---- tile ranges ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint32_t* __restrict__ keys,
                                                          const int64_t* __restrict__ n_dev, int64_t capacity,
                                                          uint32_t* __restrict__ ranges, int32_t* __restrict__ status) {
  const int64_t total = *n_dev;
  const int64_t n = total < capacity ? total : capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > capacity) set_status(status, I4D_ERR_CAPACITY);
  // four keys per thread (one 16-byte load), their neighbours one load each
  const int64_t n4 = (n + 3) / 4;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * g;
    uint32_t k[4];
    if (i0 + 4 <= n) {
      const uint4 v = reinterpret_cast<const uint4*>(keys)[g];
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = (i0 + j < n) ? keys[i0 + j] : 0u;
    }
    const uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0u;
    const uint32_t next = i0 + 4 < n ? keys[i0 + 4] : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i >= n) break;
      const uint32_t t = k[j];
      const uint32_t left = j ? k[j - 1] : prev;
      const uint32_t right = j < 3 ? k[j + 1] : next;
      if (i == 0 || left != t) ranges[2 * (int64_t)t] = (uint32_t)i;
      if (i == n - 1 || right != t) ranges[2 * (int64_t)t + 1] = (uint32_t)(i + 1);
    }
  }
}

// Tiles ordered longest first by octave of list length; inside an octave the tiles keep their index
// order (view by view, row-major), so that the CTAs in flight at one time work on neighbouring tiles
// and share the records they gather in L2 (on the 1.13M-Gaussian, 8-view training batch the
// backward's DRAM traffic falls from 2.26 to 1.80 GB against quarter-octave buckets, for 0.6% more
// time in the two compositing kernels).  The order only decides which CTA starts first, never a
// result.  One CTA of 32 warps: a stable counting sort over 32 buckets, each chunk of 1024 tiles
// ranked per warp with match_any, and per bucket by warp k scanning bucket k's counts over the
// warps.
constexpr int kOrderBuckets = 32;  // octaves; lists of 2^31 entries or more share the first bucket

__device__ __forceinline__ int order_bucket(uint32_t len) {
  return kOrderBuckets - 1 - min((int)floorf(log2f((float)len + 1.0f)), kOrderBuckets - 1);
}

__global__ void __launch_bounds__(1024) tile_order_kernel(const uint32_t* __restrict__ ranges, int T,
                                                          uint32_t* __restrict__ order) {
  __shared__ uint32_t base[kOrderBuckets];
  __shared__ uint32_t warp_pos[32][kOrderBuckets + 1];  // [warp][bucket], padded row
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  if (threadIdx.x < kOrderBuckets) base[threadIdx.x] = 0;
  warp_pos[warp][lane] = 0;
  __syncthreads();
  // bucket sizes (warp-aggregated), then their exclusive scan by warp 0
  for (int t0 = 0; t0 < T; t0 += blockDim.x) {
    const int t = t0 + (int)threadIdx.x;
    const int b = t < T ? order_bucket(ranges[2 * t + 1] - ranges[2 * t]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && (peers & lt_mask) == 0) atomicAdd(&base[b], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t c = base[lane];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    base[lane] = incl - c;
  }
  __syncthreads();
  for (int t0 = 0; t0 < T; t0 += blockDim.x) {
    const int t = t0 + (int)threadIdx.x;
    const int b = t < T ? order_bucket(ranges[2 * t + 1] - ranges[2 * t]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const uint32_t rank = __popc(peers & lt_mask);
    if (b >= 0 && rank == 0) warp_pos[warp][b] = __popc(peers);
    __syncthreads();
    {
      // warp k: bucket k's counts over the warps (lane = warp index) -> each warp's first position
      const int k = warp;
      const uint32_t c = warp_pos[lane][k];
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t b0 = base[k];
      warp_pos[lane][k] = b0 + incl - c;
      __syncwarp();
      if (lane == 31) base[k] = b0 + incl;
    }
    __syncthreads();
    if (b >= 0) order[warp_pos[warp][b] + rank] = (uint32_t)t;
    __syncthreads();
    warp_pos[warp][lane] = 0;
    __syncthreads();
  }
}

}  // namespace

size_t scan_workspace_bytes(int64_t) { return sizeof(uint64_t) * kScanMaxBlocks; }

namespace {
template <class Load>
cudaError_t scan_impl(Load in, uint32_t* out, int64_t n_max, const int64_t* n_dev, int64_t* total, void* ws,
                      cudaStream_t st) {
  uint64_t* bsum = reinterpret_cast<uint64_t*>(ws);
  int nb;
  int64_t chunk;
  scan_geometry(n_max, nb, chunk);
  if (n_max == 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
    return cudaSuccess;
  }
  I4D_PROF("scan", st);
  scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, n_dev, n_max, chunk, bsum);
  scan_down_kernel<<<nb, kScanThreads, 0, st>>>(in, out, n_dev, n_max, chunk, bsum, total);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, int64_t* total, void* ws, cudaStream_t st) {
  return scan_impl(LoadPlain{in}, out, n, nullptr, total, ws, st);
}

size_t radix_workspace_bytes(int64_t capacity) {
  const int64_t nblocks = (capacity + kRsMinTile - 1) / kRsMinTile;
  const int64_t hist = (int64_t)kRsBins * (nblocks > 0 ? nblocks : 1);
  size_t b = sizeof(uint32_t) * (size_t)hist;  // histogram, scanned in place
  b = (b + 255) & ~(size_t)255;
  b += scan_workspace_bytes(hist);
  return b;
}

// vals_out must be a buffer of its own (neither vals nor vals_alt): the last pass reads one of those.
// key_gather (nullable): the last pass writes key_gather[value] in place of the sorted keys.
template <class K>
cudaError_t launch_radix_sort(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, uint32_t* vals_out,
                              int64_t capacity, const int64_t* n_dev, int bits, void* ws, K** keys_result,
                              cudaStream_t st, const uint32_t* key_gather) {
  const int64_t nb64 = (capacity + RsCfg<K>::kTile - 1) / RsCfg<K>::kTile;
  const int nblocks = (int)(nb64 > 0 ? nb64 : 1);
  const int64_t hist_n = (int64_t)kRsBins * nblocks;
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws);
  size_t off = (sizeof(uint32_t) * (size_t)hist_n + 255) & ~(size_t)255;
  void* scan_ws = reinterpret_cast<char*>(ws) + off;
  const int passes = bits > 0 ? (bits + 7) / 8 : 1;
  K* kb[2] = {keys, keys_alt};
  uint32_t* vb[2] = {vals, vals_alt};
  for (int p = 0; p < passes; ++p) {
    const K* kin = kb[p & 1];
    const uint32_t* vin = (p == 0) ? vals : vb[p & 1];
    K* kout = kb[(p + 1) & 1];
    uint32_t* vout = (p == passes - 1) ? vals_out : vb[(p + 1) & 1];
    {
      I4D_PROF("radix_hist", st);
      radix_hist_kernel<K><<<nblocks, kRsThreads, 0, st>>>(kin, n_dev, capacity, 8 * p, nblocks, hist);
    }
    cudaError_t e = launch_scan_u32(hist, hist, hist_n, nullptr, scan_ws, st);
    if (e != cudaSuccess) return e;
    I4D_PROF("radix_scatter", st);
    radix_scatter_kernel<K><<<nblocks, kRsThreads, 0, st>>>(kin, vin, kout, vout, n_dev, capacity, 8 * p, nblocks,
                                                            hist, p == passes - 1 ? key_gather : nullptr);
  }
  if (keys_result) *keys_result = kb[passes & 1];
  return cudaGetLastError();
}

template cudaError_t launch_radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t,
                                                 const int64_t*, int, void*, uint32_t**, cudaStream_t,
                                                 const uint32_t*);
template cudaError_t launch_radix_sort<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, uint32_t*, int64_t,
                                                 const int64_t*, int, void*, uint64_t**, cudaStream_t,
                                                 const uint32_t*);

size_t bin_workspace_bytes(int64_t VN, int64_t capacity) {
  const size_t vn = (size_t)(VN > 0 ? VN : 1), cap = (size_t)(capacity > 0 ? capacity : 1);
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t b = 0;
  b += 7 * a(4 * vn);                   // flag offsets, depth keys x2, record values x3, emit offsets
  b += a(8);                            // visible-record count
  b += a(scan_workspace_bytes(VN));
  b += 4 * a(4 * cap);                  // tile keys x2, id values x2 (the sorted ids go to the output)
  b += a(radix_workspace_bytes(VN > capacity ? VN : capacity));
  return b;
}

cudaError_t launch_bin_tiles(const ViewTable& vt, int n, const float* proj_f, const uint32_t* touched,
                             int64_t capacity, uint32_t* ids, uint32_t* ranges, int64_t* n_inst, int32_t* status,
                             void* ws, cudaStream_t st) {
  const int64_t VN = (int64_t)vt.n_views * n;
  const int64_t T = vt.tile_off[vt.n_views];
  const float4* proj = reinterpret_cast<const float4*>(proj_f);
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = reinterpret_cast<char*>(ws);
  const size_t vn = (size_t)(VN > 0 ? VN : 1), cap = (size_t)(capacity > 0 ? capacity : 1);
  uint32_t* offs1 = (uint32_t*)p; p += a(4 * vn);
  uint32_t* dkA = (uint32_t*)p; p += a(4 * vn);
  uint32_t* dkB = (uint32_t*)p; p += a(4 * vn);
  uint32_t* dvA = (uint32_t*)p; p += a(4 * vn);
  uint32_t* dvB = (uint32_t*)p; p += a(4 * vn);
  uint32_t* dvOut = (uint32_t*)p; p += a(4 * vn);
  uint32_t* offs2 = (uint32_t*)p; p += a(4 * vn);
  int64_t* R_dev = (int64_t*)p; p += a(8);
  void* scan_ws = p; p += a(scan_workspace_bytes(VN));
  uint32_t* tkA = (uint32_t*)p; p += a(4 * cap);
  uint32_t* tkB = (uint32_t*)p; p += a(4 * cap);
  uint32_t* tvA = (uint32_t*)p; p += a(4 * cap);
  uint32_t* tvB = (uint32_t*)p; p += a(4 * cap);
  void* radix_ws = p;

  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  // 1. visible records (touched > 0) in index order, keyed by depth
  e = scan_impl(LoadNonzero{touched}, offs1, VN, nullptr, R_dev, scan_ws, st);
  if (e != cudaSuccess) return e;
  if (VN > 0) {
    I4D_PROF("visible_compact", st);
    visible_compact_kernel<<<(unsigned)((VN + 255) / 256), 256, 0, st>>>(VN, proj, touched, offs1, dkA, dvA);
  }
  // 2. stable sort of the visible records by depth (equal depths keep index order); the last pass
  //    writes each record's tile count where its key would go
  uint32_t* cnt_sorted = nullptr;
  e = launch_radix_sort<uint32_t>(dkA, dvA, dkB, dvB, dvOut, VN, R_dev, 32, radix_ws, &cnt_sorted, st, touched);
  if (e != cudaSuccess) return e;
  uint32_t* rec_sorted = dvOut;
  // 3. tile counts in depth order -> output offsets; the total is the instance count
  e = scan_impl(LoadPlain{cnt_sorted}, offs2, VN, R_dev, n_inst, scan_ws, st);
  if (e != cudaSuccess) return e;
  if (VN > 0) {
    I4D_PROF("emit_keys", st);
    emit_sorted_kernel<<<(unsigned)((VN + 255) / 256), 256, 0, st>>>(vt, n, proj, R_dev, rec_sorted, offs2, capacity,
                                                                     tkA, tvA);
  }
  // 4. stable sort of the pairs by tile: within a tile they stay in (depth, id) order
  int bits = 0;
  while ((1ll << bits) < T) ++bits;
  uint32_t* sorted_tiles = nullptr;
  e = launch_radix_sort<uint32_t>(tkA, tvA, tkB, tvB, ids, capacity, n_inst, bits, radix_ws, &sorted_tiles, st);
  if (e != cudaSuccess) return e;
  // 5. per-tile ranges and the longest-first tile order
  return launch_tile_ranges(sorted_tiles, n_inst, capacity, ranges, T, status, st);
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const int64_t* n_dev, int64_t capacity, uint32_t* ranges,
                               int64_t total_tiles, int32_t* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles, st);
  if (e != cudaSuccess) return e;
  I4D_PROF("tile_ranges", st);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((capacity / 4 + threads) / threads, 152 * 16);
  tile_ranges_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), threads, 0, st>>>(keys, n_dev, capacity, ranges, status);
  {
    I4D_PROF("tile_order", st);
    tile_order_kernel<<<1, 1024, 0, st>>>(ranges, (int)total_tiles, ranges + 2 * total_tiles);
  }
  return cudaGetLastError();
}

}  // namespace i4d
