// Voxel-grid pruning of the back-projected depth point cloud (Eq. 5, Sec. 3.2 "Grid Pruning").
//
//   1. insert: per pixel (or per point), back-project, compute the integer voxel key and aggregate
//      into an open-addressing device hash table: count, minimum point index, and the sums of
//      x, y, z, r, g, b, t in 64-bit fixed point (order-independent, so results do not depend on
//      atomic ordering).  Lanes of a warp that hit the same voxel are merged before the atomics.
//   2. compact: occupied slots with count >= min_support get an output position (scan).
//   3. order: a radix sort by representative (minimum) point index makes the output order the
//      point order, independent of the hash layout.
//   4. gather: centroid = sum / count and the averaged attributes.
// The point cloud itself is never written to HBM when starting from depth maps.
#include "kernels.cuh"

namespace i4d {

namespace {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kCoordBits = 21;
constexpr int64_t kCoordHalf = 1ll << (kCoordBits - 1);
constexpr double kFix = 4294967296.0;  // 2^32
constexpr int kSums = 7;
constexpr int kMaxProbes = 4096;

struct Table {
  uint64_t* keys;
  uint32_t* cnt;
  uint32_t* minidx;
  unsigned long long* sums;  // kSums planes of `slots`
  int64_t slots;
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// floor of one correctly rounded float32 product (no contraction, no fast-math)
__device__ __forceinline__ int64_t voxel_coord(float x, float inv) { return (int64_t)floorf(__fmul_rn(x, inv)); }

__device__ __forceinline__ bool make_key(float x, float y, float z, int flag, float inv, uint64_t& key) {
  const int64_t ix = voxel_coord(x, inv), iy = voxel_coord(y, inv), iz = voxel_coord(z, inv);
  // (iz stops one short of the top so that no key can equal the all-ones empty marker; ix too, so
  // that the x field's top value is free for the keys of unpruned points)
  if (ix < -kCoordHalf || ix >= kCoordHalf - 1 || iy < -kCoordHalf || iy >= kCoordHalf || iz < -kCoordHalf ||
      iz >= kCoordHalf - 1)
    return false;
  const uint64_t m = (1ull << kCoordBits) - 1;
  key = ((uint64_t)flag << 63) | ((uint64_t)(ix + kCoordHalf) & m) << 42 | ((uint64_t)(iy + kCoordHalf) & m) << 21 |
        ((uint64_t)(iz + kCoordHalf) & m);
  return true;
}

// A dynamic point that is not pruned (voxel_dynamic = 0, the Full model of Sec. 4.1) forms a voxel
// of its own: dynamic flag, the x field's top value (no voxel key has it) and its index.
constexpr uint64_t kUnprunedTag = (1ull << 22) - 1;  // flag bit + 21 ones, in bits 42..63
__device__ __forceinline__ uint64_t unpruned_key(uint32_t idx) { return (kUnprunedTag << 42) | (uint64_t)idx; }
__device__ __forceinline__ bool is_unpruned(uint64_t key) { return (key >> 42) == kUnprunedTag; }

__device__ __forceinline__ unsigned long long to_fix(float x) {
  return (unsigned long long)(long long)llrint((double)x * kFix);
}

// Insert one (possibly warp-merged) contribution.  Returns false if the probe bound was hit.
__device__ __forceinline__ bool table_add(const Table& T, uint64_t key, uint32_t count, uint32_t minidx,
                                          const unsigned long long* s) {
  const int64_t mask = T.slots - 1;
  int64_t h = (int64_t)(mix64(key) & (uint64_t)mask);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    uint64_t cur = __ldcg(reinterpret_cast<const unsigned long long*>(&T.keys[h]));
    if (cur == kEmpty) cur = atomicCAS(reinterpret_cast<unsigned long long*>(&T.keys[h]), kEmpty, key);
    if (cur == kEmpty || cur == key) {
      atomicAdd(&T.cnt[h], count);
      atomicMin(&T.minidx[h], minidx);
#pragma unroll
      for (int k = 0; k < kSums; ++k) atomicAdd(&T.sums[(int64_t)k * T.slots + h], s[k]);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

// All 32 lanes call this (valid or not).  Lanes with equal keys are merged by their lowest lane.
__device__ __forceinline__ void warp_insert(const Table& T, bool valid, uint64_t key, uint32_t idx,
                                            const unsigned long long* s, int32_t* status) {
  __shared__ unsigned long long buf[8][32][kSums];
  __shared__ uint32_t ibuf[8][32];
  const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) & 7;
  const uint64_t k = valid ? key : kEmpty;
  const unsigned peers = __match_any_sync(0xffffffffu, k);
#pragma unroll
  for (int j = 0; j < kSums; ++j) buf[warp][lane][j] = s[j];
  ibuf[warp][lane] = idx;
  __syncwarp();
  const int leader = __ffs(peers) - 1;
  if (valid && lane == leader) {
    unsigned long long acc[kSums];
#pragma unroll
    for (int j = 0; j < kSums; ++j) acc[j] = 0ull;
    uint32_t mn = 0xffffffffu;
    unsigned m = peers;
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
#pragma unroll
      for (int j = 0; j < kSums; ++j) acc[j] += buf[warp][l][j];
      mn = min(mn, ibuf[warp][l]);
    }
    if (!table_add(T, key, (uint32_t)__popc(peers), mn, acc)) set_status(status, I4D_ERR_CAPACITY);
  }
  __syncwarp();
}

// K1 + K2: one thread per pixel, warps cover 8x4 pixel patches (neighbouring pixels share voxels).
__global__ void __launch_bounds__(256) insert_depth_kernel(const float* __restrict__ depth,
                                                           const uint8_t* __restrict__ rgb8,
                                                           const uint8_t* __restrict__ dyn,
                                                           const i4d_camera* __restrict__ cams, int W, int H,
                                                           int tiles_x, float inv_s, float inv_d, Table T,
                                                           int32_t* status) {
  const int f = blockIdx.y;
  const int tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // block = 32 x 8 pixels = 4 x 2 warps of 8 x 4
  const int px = (tile % tiles_x) * 32 + (warp & 3) * 8 + (lane & 7);
  const int py = (tile / tiles_x) * 8 + (warp >> 2) * 4 + (lane >> 3);
  const bool inside = px < W && py < H;
  const i4d_camera& c = cams[f];
  bool valid = false;
  uint64_t key = 0;
  unsigned long long s[kSums] = {0, 0, 0, 0, 0, 0, 0};
  uint32_t idx = 0;
  if (inside) {
    const int64_t pi = ((int64_t)f * H + py) * W + px;
    idx = (uint32_t)pi;
    const float D = depth[pi];
    // Eq. 5: camera-space point D K^-1 (px + 0.5, py + 0.5, 1), world point R^T (X_c - t), as a
    // fixed sequence of correctly rounded float32 operations (no FMA contraction), so that every
    // IEEE-754 machine computes the same cloud and hence the same voxel keys
    const float xc = __fmul_rn(D, __fdiv_rn(__fsub_rn((float)px + 0.5f, c.cx), c.fx));
    const float yc = __fmul_rn(D, __fdiv_rn(__fsub_rn((float)py + 0.5f, c.cy), c.fy));
    const float dx = __fsub_rn(xc, c.t[0]), dy = __fsub_rn(yc, c.t[1]), dz = __fsub_rn(D, c.t[2]);
    const float x = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], dx), __fmul_rn(c.R[3], dy)), __fmul_rn(c.R[6], dz));
    const float y = __fadd_rn(__fadd_rn(__fmul_rn(c.R[1], dx), __fmul_rn(c.R[4], dy)), __fmul_rn(c.R[7], dz));
    const float z = __fadd_rn(__fadd_rn(__fmul_rn(c.R[2], dx), __fmul_rn(c.R[5], dy)), __fmul_rn(c.R[8], dz));
    const int flag = dyn ? (dyn[pi] != 0) : 0;
    if (flag && inv_d == 0.0f) {
      key = unpruned_key(idx);
      valid = true;
    } else {
      valid = make_key(x, y, z, flag, flag ? inv_d : inv_s, key);
      if (!valid) set_status(status, I4D_ERR_CAPACITY);
    }
    s[0] = to_fix(x);
    s[1] = to_fix(y);
    s[2] = to_fix(z);
    if (rgb8) {
      s[3] = to_fix((float)rgb8[3 * pi] * (1.0f / 255.0f));
      s[4] = to_fix((float)rgb8[3 * pi + 1] * (1.0f / 255.0f));
      s[5] = to_fix((float)rgb8[3 * pi + 2] * (1.0f / 255.0f));
    }
    s[6] = to_fix(c.time);
  }
  warp_insert(T, valid, key, idx, s, status);
}

__global__ void __launch_bounds__(256) insert_xyz_kernel(const float* __restrict__ xyz, const float* __restrict__ rgb,
                                                         const float* __restrict__ tpt,
                                                         const uint8_t* __restrict__ dyn, int64_t n, float inv_s,
                                                         float inv_d, Table T, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = false;
  uint64_t key = 0;
  unsigned long long s[kSums] = {0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const int flag = dyn ? (dyn[i] != 0) : 0;
    if (flag && inv_d == 0.0f) {
      key = unpruned_key((uint32_t)i);
      valid = true;
    } else {
      valid = make_key(x, y, z, flag, flag ? inv_d : inv_s, key);
      if (!valid) set_status(status, I4D_ERR_CAPACITY);
    }
    s[0] = to_fix(x);
    s[1] = to_fix(y);
    s[2] = to_fix(z);
    if (rgb) {
      s[3] = to_fix(rgb[3 * i]);
      s[4] = to_fix(rgb[3 * i + 1]);
      s[5] = to_fix(rgb[3 * i + 2]);
    }
    if (tpt) s[6] = to_fix(tpt[i]);
  }
  warp_insert(T, valid, key, (uint32_t)i, s, status);
}

__global__ void table_flags_kernel(Table T, int min_support, uint32_t* __restrict__ flags) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T.slots) return;
  const uint64_t k = T.keys[s];
  flags[s] = (k != kEmpty && (T.cnt[s] >= (uint32_t)min_support || is_unpruned(k))) ? 1u : 0u;
}

__global__ void table_compact_kernel(Table T, const uint32_t* __restrict__ flags, const uint32_t* __restrict__ offs,
                                     int64_t capacity, uint64_t* __restrict__ skeys, uint32_t* __restrict__ svals) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T.slots || !flags[s]) return;
  const int64_t o = offs[s];
  if (o < capacity) {
    skeys[o] = (uint64_t)T.minidx[s];
    svals[o] = (uint32_t)s;
  }
}

__global__ void gather_kernel(Table T, const uint32_t* __restrict__ slot_sorted, const int64_t* __restrict__ n_dev,
                              int64_t capacity, PruneOut out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = *n_dev;
  if (j == 0) {
    *out.n_kept = total;
    if (total > capacity) set_status(out.status, I4D_ERR_CAPACITY);
  }
  const int64_t n = total < capacity ? total : capacity;
  if (j >= n) return;
  const int64_t s = slot_sorted[j];
  const uint32_t c = T.cnt[s];
  const double inv = 1.0 / ((double)c * kFix);
  float v[kSums];
#pragma unroll
  for (int k = 0; k < kSums; ++k) v[k] = (float)((double)(long long)T.sums[(int64_t)k * T.slots + s] * inv);
  out.rep[j] = T.minidx[s];
  out.count[j] = (int32_t)c;
  out.xyz[3 * j] = v[0];
  out.xyz[3 * j + 1] = v[1];
  out.xyz[3 * j + 2] = v[2];
  out.rgb[3 * j] = v[3];
  out.rgb[3 * j + 1] = v[4];
  out.rgb[3 * j + 2] = v[5];
  out.t[j] = v[6];
  out.flag[j] = (uint8_t)(T.keys[s] >> 63);
}

__global__ void table_init_kernel(Table T) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T.slots) return;
  T.keys[s] = kEmpty;
  T.cnt[s] = 0;
  T.minidx[s] = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < kSums; ++k) T.sums[(int64_t)k * T.slots + s] = 0ull;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct PruneWs {
  Table T;
  uint32_t* flags;
  uint32_t* offs;
  int64_t* total;
  void* scan_ws;
  uint64_t* sk[2];
  uint32_t* sv[2];
  uint32_t* sorted_slots;
  void* radix_ws;
};

PruneWs carve(void* ws, int64_t slots, int64_t capacity) {
  PruneWs w;
  char* p = reinterpret_cast<char*>(ws);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += align256(bytes);
    return r;
  };
  w.T.slots = slots;
  w.T.keys = (uint64_t*)take(8 * (size_t)slots);
  w.T.cnt = (uint32_t*)take(4 * (size_t)slots);
  w.T.minidx = (uint32_t*)take(4 * (size_t)slots);
  w.T.sums = (unsigned long long*)take(8 * (size_t)kSums * slots);
  w.flags = (uint32_t*)take(4 * (size_t)slots);
  w.offs = (uint32_t*)take(4 * (size_t)slots);
  w.total = (int64_t*)take(8);
  w.scan_ws = take(scan_workspace_bytes(slots));
  w.sk[0] = (uint64_t*)take(8 * (size_t)capacity);
  w.sk[1] = (uint64_t*)take(8 * (size_t)capacity);
  w.sv[0] = (uint32_t*)take(4 * (size_t)capacity);
  w.sv[1] = (uint32_t*)take(4 * (size_t)capacity);
  w.sorted_slots = (uint32_t*)take(4 * (size_t)capacity);
  w.radix_ws = take(radix_workspace_bytes(capacity));
  return w;
}

}  // namespace

size_t prune_workspace_bytes(int64_t n_points, int64_t table_slots) {
  (void)n_points;
  const int64_t capacity = table_slots;  // never more kept voxels than slots
  size_t b = 0;
  b += align256(8 * (size_t)table_slots) + 2 * align256(4 * (size_t)table_slots);
  b += align256(8 * (size_t)kSums * table_slots);
  b += 2 * align256(4 * (size_t)table_slots) + align256(8) + align256(scan_workspace_bytes(table_slots));
  b += 2 * align256(8 * (size_t)capacity) + 3 * align256(4 * (size_t)capacity);
  b += align256(radix_workspace_bytes(capacity));
  return b;
}

cudaError_t launch_prune(const float* depth, const uint8_t* rgb8, const uint8_t* dyn, const i4d_camera* cams, int F,
                         int W, int H, const float* xyz, const float* rgbf, const float* tpt, int64_t n_points,
                         float inv_static, float inv_dynamic, int min_support, int64_t table_slots, int64_t capacity,
                         const PruneOut& out, void* ws, cudaStream_t st) {
  (void)capacity;
  const int64_t cap_int = table_slots;  // internal sort capacity
  PruneWs w = carve(ws, table_slots, cap_int);
  const int threads = 256;
  const int64_t sblocks = (table_slots + threads - 1) / threads;
  {
    I4D_PROF("prune_table_init", st);
    table_init_kernel<<<(unsigned)sblocks, threads, 0, st>>>(w.T);
  }
  if (depth) {
    I4D_PROF("prune_insert", st);
    const int tiles_x = (W + 31) / 32, tiles_y = (H + 7) / 8;
    dim3 grid((unsigned)(tiles_x * tiles_y), (unsigned)F);
    if (F > 0 && W > 0 && H > 0)
      insert_depth_kernel<<<grid, threads, 0, st>>>(depth, rgb8, dyn, cams, W, H, tiles_x, inv_static, inv_dynamic,
                                                    w.T, out.status);
  } else if (n_points > 0) {
    I4D_PROF("prune_insert", st);
    const int64_t blocks = (n_points + threads - 1) / threads;
    insert_xyz_kernel<<<(unsigned)blocks, threads, 0, st>>>(xyz, rgbf, tpt, dyn, n_points, inv_static, inv_dynamic,
                                                           w.T, out.status);
  }
  {
    I4D_PROF("prune_compact", st);
    table_flags_kernel<<<(unsigned)sblocks, threads, 0, st>>>(w.T, min_support, w.flags);
  }
  cudaError_t e = launch_scan_u32(w.flags, w.offs, table_slots, w.total, w.scan_ws, st);
  if (e != cudaSuccess) return e;
  {
    I4D_PROF("prune_compact", st);
    table_compact_kernel<<<(unsigned)sblocks, threads, 0, st>>>(w.T, w.flags, w.offs, cap_int, w.sk[0], w.sv[0]);
  }
  e = launch_radix_sort<uint64_t>(w.sk[0], w.sv[0], w.sk[1], w.sv[1], w.sorted_slots, cap_int, w.total, 32,
                                  w.radix_ws, nullptr, st);
  if (e != cudaSuccess) return e;
  const int64_t oblocks = (capacity + threads - 1) / threads;
  I4D_PROF("prune_gather", st);
  gather_kernel<<<(unsigned)(oblocks > 0 ? oblocks : 1), threads, 0, st>>>(w.T, w.sorted_slots, w.total, capacity,
                                                                            out);
  return cudaGetLastError();
}

}  // namespace i4d
