// Voxel-neighbourhood features of the pruned points (inputs of the learned initialisation) and the
// mean distance to the 3 nearest neighbours (the spatial scale of the heuristic initialisation).
//
// A device hash table maps each occupied voxel cell to a linked list of its points (built with one
// atomicCAS per new cell and one atomicExch per point); a query walks the (2R+1)^3 cells around a
// point's cell and keeps the 16 nearest other points, ordered by (squared distance, index), in a
// register-resident sorted list.  Results do not depend on list order.
#include "kernels.cuh"

namespace i4d {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kEnd = 0xffffffffu;
constexpr int kProbeLimit = 4096;
constexpr int kK = 16;

__device__ __forceinline__ uint64_t cell_key(int64_t cx, int64_t cy, int64_t cz) {
  const int64_t half = 1ll << 20;
  const uint64_t m = (1ull << 21) - 1;
  return ((uint64_t)(cx + half) & m) << 42 | ((uint64_t)(cy + half) & m) << 21 | ((uint64_t)(cz + half) & m);
}

__device__ __forceinline__ uint64_t mix(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ void cell_of(const float* p, float inv, int64_t& cx, int64_t& cy, int64_t& cz) {
  cx = (int64_t)floorf(__fmul_rn(p[0], inv));
  cy = (int64_t)floorf(__fmul_rn(p[1], inv));
  cz = (int64_t)floorf(__fmul_rn(p[2], inv));
}

__global__ void knn_table_init(uint64_t* keys, uint32_t* head, int64_t slots) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < slots) {
    keys[s] = kEmptyKey;
    head[s] = kEnd;
  }
}

__global__ void knn_insert(const float* __restrict__ xyz, int64_t n, float inv, uint64_t* keys, uint32_t* head,
                           uint32_t* next, int64_t slots, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t cx, cy, cz;
  cell_of(xyz + 3 * i, inv, cx, cy, cz);
  const uint64_t key = cell_key(cx, cy, cz);
  const int64_t mask = slots - 1;
  int64_t h = (int64_t)(mix(key) & (uint64_t)mask);
  for (int probe = 0; probe < kProbeLimit; ++probe) {
    uint64_t cur = __ldcg(reinterpret_cast<const unsigned long long*>(&keys[h]));
    if (cur == kEmptyKey) cur = atomicCAS(reinterpret_cast<unsigned long long*>(&keys[h]), kEmptyKey, key);
    if (cur == kEmptyKey || cur == key) {
      next[i] = atomicExch(&head[h], (uint32_t)i);
      return;
    }
    h = (h + 1) & mask;
  }
  set_status(status, I4D_ERR_CAPACITY);
  next[i] = kEnd;
}

__device__ __forceinline__ bool before(float d, uint32_t j, float d2, uint32_t j2) {
  return d < d2 || (d == d2 && j < j2);
}

__global__ void __launch_bounds__(128) knn_query(const float* __restrict__ xyz, const float* __restrict__ rgb,
                                                 const float* __restrict__ t, const uint8_t* __restrict__ flag,
                                                 int64_t n, float voxel, float inv, int radius, float rx, float ry,
                                                 float rz, const uint64_t* __restrict__ keys,
                                                 const uint32_t* __restrict__ head, const uint32_t* __restrict__ next,
                                                 int64_t slots, float* __restrict__ feat, float* __restrict__ knn3) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2];
  int64_t cx, cy, cz;
  cell_of(xyz + 3 * i, inv, cx, cy, cz);
  float bd[kK];
  uint32_t bj[kK];
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    bd[k] = INFINITY;
    bj[k] = kEnd;
  }
  const int64_t mask = slots - 1;
  for (int dz = -radius; dz <= radius; ++dz)
    for (int dy = -radius; dy <= radius; ++dy)
      for (int dx = -radius; dx <= radius; ++dx) {
        const uint64_t key = cell_key(cx + dx, cy + dy, cz + dz);
        int64_t h = (int64_t)(mix(key) & (uint64_t)mask);
        uint32_t j = kEnd;
        for (int probe = 0; probe < kProbeLimit; ++probe) {
          const uint64_t cur = keys[h];
          if (cur == key) {
            j = head[h];
            break;
          }
          if (cur == kEmptyKey) break;
          h = (h + 1) & mask;
        }
        for (int guard = 0; j != kEnd && guard < (1 << 20); ++guard) {
          if (j != (uint32_t)i) {
            const float ex = xyz[3 * (int64_t)j] - px, ey = xyz[3 * (int64_t)j + 1] - py,
                        ez = xyz[3 * (int64_t)j + 2] - pz;
            const float d = ex * ex + ey * ey + ez * ez;
            if (before(d, j, bd[kK - 1], bj[kK - 1])) {
              bd[kK - 1] = d;
              bj[kK - 1] = j;
#pragma unroll
              for (int k = kK - 1; k > 0; --k) {
                if (before(bd[k], bj[k], bd[k - 1], bj[k - 1])) {
                  const float td = bd[k];
                  bd[k] = bd[k - 1];
                  bd[k - 1] = td;
                  const uint32_t tj = bj[k];
                  bj[k] = bj[k - 1];
                  bj[k - 1] = tj;
                }
              }
            }
          }
          j = next[j];
        }
      }
  float* f = feat + 64 * i;
  int found = 0;
  const float iv = 1.0f / voxel;
  const float ti = t ? t[i] : 0.0f;
  float vx = 0.f, vy = 0.f, vz = 0.f, dtt = 0.f;  // least-squares velocity of the neighbourhood
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    const bool ok = bj[k] != kEnd;
    found += ok ? 1 : 0;
    const int64_t j = ok ? (int64_t)bj[k] : i;
    const float ox = ok ? (xyz[3 * j] - px) * iv : 0.0f;
    const float oy = ok ? (xyz[3 * j + 1] - py) * iv : 0.0f;
    const float oz = ok ? (xyz[3 * j + 2] - pz) * iv : 0.0f;
    f[3 * k] = ox;
    f[3 * k + 1] = oy;
    f[3 * k + 2] = oz;
    const float dt = (ok && t) ? t[j] - ti : 0.0f;
    vx += dt * ox;
    vy += dt * oy;
    vz += dt * oz;
    dtt += dt * dt;
  }
  const float ex = px - rx, ey = py - ry, ez = pz - rz;
  f[48] = sqrtf(ex * ex + ey * ey + ez * ez);
  f[49] = rgb ? rgb[3 * i] : 0.0f;
  f[50] = rgb ? rgb[3 * i + 1] : 0.0f;
  f[51] = rgb ? rgb[3 * i + 2] : 0.0f;
  f[52] = t ? t[i] : 0.0f;
  f[53] = (float)found / (float)kK;
  f[54] = flag ? (float)(flag[i] != 0) : 0.0f;
  const float iv16 = 1.0f / (16.0f * (dtt + 1e-6f));
  f[55] = vx * iv16;
  f[56] = vy * iv16;
  f[57] = vz * iv16;
  f[58] = found ? sqrtf(dtt / (float)found) : 0.0f;
#pragma unroll
  for (int k = 59; k < 64; ++k) f[k] = 0.0f;
  if (knn3) knn3[i] = found >= 3 ? (sqrtf(bd[0]) + sqrtf(bd[1]) + sqrtf(bd[2])) * (1.0f / 3.0f) : voxel;
}

}  // namespace

size_t knn_workspace_bytes(int64_t n, int64_t slots) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return a(8 * (size_t)slots) + a(4 * (size_t)slots) + a(4 * (size_t)(n > 0 ? n : 1));
}

cudaError_t launch_knn_features(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int64_t n,
                                float voxel, int radius, const float* ref, float* feat, float* knn3, int64_t slots,
                                int32_t* status, void* ws, cudaStream_t st) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = reinterpret_cast<char*>(ws);
  uint64_t* keys = (uint64_t*)p;
  p += a(8 * (size_t)slots);
  uint32_t* head = (uint32_t*)p;
  p += a(4 * (size_t)slots);
  uint32_t* next = (uint32_t*)p;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess || n == 0) return e;
  I4D_PROF("knn_features", st);
  const float inv = 1.0f / voxel;
  knn_table_init<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(keys, head, slots);
  knn_insert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xyz, n, inv, keys, head, next, slots, status);
  knn_query<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(xyz, rgb, t, flag, n, voxel, inv, radius, ref[0], ref[1],
                                                         ref[2], keys, head, next, slots, feat, knn3);
  return cudaGetLastError();
}

}  // namespace i4d
