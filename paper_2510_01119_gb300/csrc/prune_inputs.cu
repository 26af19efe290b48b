// The two inputs of grid pruning derived from the video (Sec. 3.2): the adaptive voxel edge of
// Eq. 6 and the static / dynamic masks from Otsu's thresholding of motion-probability maps.
//
// Eq. 6: per-frame depth sums in exact 64-bit fixed point (2^-32 units, warp-reduced, one atomic
// per block), then S_v = lambda_s * mean_i (D_i / f_i) in float64 in frame order, so the result
// does not depend on the summation order.  Motion masks: each low-resolution map is upsampled
// bilinearly (pixel-centre alignment, every step an explicitly rounded float32 operation), binned
// into a per-frame 256-bin histogram (shared-memory atomics), Otsu's threshold is found by one
// 256-thread block per frame from exact integer prefix sums, and a second pass writes the masks.
#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) depth_sum_kernel(const float* __restrict__ depth, int64_t HW,
                                                             unsigned long long* __restrict__ sums,
                                                             unsigned int* __restrict__ counts) {
  const int f = blockIdx.y;
  const float* d = depth + (int64_t)f * HW;
  unsigned long long s = 0;
  unsigned int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < HW; i += (int64_t)gridDim.x * kThreads) {
    const float v = d[i];
    if (v > 0.0f) {
      s += __double2ull_rn((double)v * 4294967296.0);
      ++c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0 && c) {
    atomicAdd(&sums[f], s);
    atomicAdd(&counts[f], c);
  }
}

__global__ void adaptive_voxel_finish_kernel(const unsigned long long* __restrict__ sums,
                                             const unsigned int* __restrict__ counts,
                                             const i4d_camera* __restrict__ cams, int F, float lambda_s,
                                             float* __restrict__ out) {
  double acc = 0.0;
  for (int i = 0; i < F; ++i) {
    const double mean = counts[i] ? __ddiv_rn(__ddiv_rn(__ull2double_rn(sums[i]), 4294967296.0), (double)counts[i])
                                  : 0.0;
    acc = __dadd_rn(acc, __ddiv_rn(mean, (double)cams[i].fx));
  }
  *out = (float)__dmul_rn((double)lambda_s, __ddiv_rn(acc, (double)F));
}

// bilinear sample of an (h, w) map at output pixel (x, y) of an (H, W) frame, pixel-centre aligned
__device__ __forceinline__ float upsample_at(const float* __restrict__ m, int h, int w, float sx_scale,
                                             float sy_scale, int x, int y) {
  const float sx = fmaxf(__fsub_rn(__fmul_rn(__fadd_rn((float)x, 0.5f), sx_scale), 0.5f), 0.0f);
  const float sy = fmaxf(__fsub_rn(__fmul_rn(__fadd_rn((float)y, 0.5f), sy_scale), 0.5f), 0.0f);
  const int x0 = (int)floorf(sx), y0 = (int)floorf(sy);
  const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
  const float wx = __fsub_rn(sx, (float)x0), wy = __fsub_rn(sy, (float)y0);
  const float ox = __fsub_rn(1.0f, wx), oy = __fsub_rn(1.0f, wy);
  const float a = m[y0 * w + x0], b = m[y0 * w + x1], c = m[y1 * w + x0], d = m[y1 * w + x1];
  const float top = __fadd_rn(__fmul_rn(ox, a), __fmul_rn(wx, b));
  const float bot = __fadd_rn(__fmul_rn(ox, c), __fmul_rn(wx, d));
  return __fadd_rn(__fmul_rn(oy, top), __fmul_rn(wy, bot));
}

__device__ __forceinline__ int bin_of(float p) {
  const int b = (int)floorf(__fmul_rn(p, 256.0f));
  return min(max(b, 0), 255);
}

__global__ void __launch_bounds__(kThreads) motion_hist_kernel(const float* __restrict__ prob, int h, int w, int H,
                                                               int W, float sx_scale, float sy_scale,
                                                               unsigned int* __restrict__ hist) {
  __shared__ unsigned int sh[256];
  const int f = blockIdx.y;
  sh[threadIdx.x] = 0;
  __syncthreads();
  const float* m = prob + (int64_t)f * h * w;
  const int64_t HW = (int64_t)H * W;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < HW; i += (int64_t)gridDim.x * kThreads) {
    const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
    atomicAdd(&sh[bin_of(upsample_at(m, h, w, sx_scale, sy_scale, x, y))], 1u);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&hist[f * 256 + threadIdx.x], sh[threadIdx.x]);
}

// One block per frame, thread t = candidate threshold t: exact prefix sums of counts and of
// level-weighted counts (integers below 2^53 in float64), then the between-class variance
// (mu_T w0 - m)^2 / (w0 (1 - w0)) and its first maximum.
__global__ void __launch_bounds__(256) otsu_threshold_kernel(const unsigned int* __restrict__ hist,
                                                             int* __restrict__ thresh) {
  __shared__ double wc[8], wm[8];
  __shared__ double best_v[8];
  __shared__ int best_t[8];
  const int f = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const double cnt = (double)hist[f * 256 + t];
  double C = cnt, M = cnt * (double)t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double c2 = __shfl_up_sync(0xffffffffu, C, o), m2 = __shfl_up_sync(0xffffffffu, M, o);
    if (lane >= o) {
      C += c2;
      M += m2;
    }
  }
  if (lane == 31) {
    wc[warp] = C;
    wm[warp] = M;
  }
  __syncthreads();
  double totC = 0.0, totM = 0.0;
  for (int k = 0; k < 8; ++k) {
    if (k < warp) {
      C += wc[k];
      M += wm[k];
    }
    totC += wc[k];
    totM += wm[k];
  }
  double sb = 0.0;
  if (C > 0.0 && C < totC) {
    const double w0 = __ddiv_rn(C, totC), m = __ddiv_rn(M, totC), muT = __ddiv_rn(totM, totC);
    const double e = __dsub_rn(__dmul_rn(muT, w0), m);
    sb = __ddiv_rn(__dmul_rn(e, e), __dmul_rn(w0, __dsub_rn(1.0, w0)));
  }
  // first maximum: larger value wins, equal values keep the smaller t
  double v = sb;
  int bt = t;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int t2 = __shfl_xor_sync(0xffffffffu, bt, o);
    if (v2 > v || (v2 == v && t2 < bt)) {
      v = v2;
      bt = t2;
    }
  }
  if (lane == 0) {
    best_v[warp] = v;
    best_t[warp] = bt;
  }
  __syncthreads();
  if (t == 0) {
    double bv = best_v[0];
    int b = best_t[0];
    for (int k = 1; k < 8; ++k)
      if (best_v[k] > bv || (best_v[k] == bv && best_t[k] < b)) {
        bv = best_v[k];
        b = best_t[k];
      }
    thresh[f] = b;
  }
}

__global__ void __launch_bounds__(kThreads) motion_mask_kernel(const float* __restrict__ prob, int h, int w, int H,
                                                               int W, float sx_scale, float sy_scale,
                                                               const int* __restrict__ thresh,
                                                               uint8_t* __restrict__ mask) {
  const int f = blockIdx.y;
  const float* m = prob + (int64_t)f * h * w;
  const int64_t HW = (int64_t)H * W;
  const int t = thresh[f];
  uint8_t* out = mask + (int64_t)f * HW;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < HW; i += (int64_t)gridDim.x * kThreads) {
    const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
    out[i] = bin_of(upsample_at(m, h, w, sx_scale, sy_scale, x, y)) > t ? 1 : 0;
  }
}

int blocks_per_frame(int64_t HW) {
  const int64_t b = (HW + kThreads * 8 - 1) / (kThreads * 8);
  return (int)(b < 64 ? (b > 0 ? b : 1) : 64);
}

}  // namespace

size_t adaptive_voxel_workspace_bytes(int F) { return (size_t)(F > 0 ? F : 1) * (8 + 4) + 256; }

cudaError_t launch_adaptive_voxel(const float* depth, int F, int H, int W, const i4d_camera* cams, float lambda_s,
                                  float* out, void* ws, cudaStream_t st) {
  unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws);
  unsigned int* counts = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(ws) + 8 * (size_t)F);
  cudaError_t e = cudaMemsetAsync(ws, 0, (size_t)F * 12, st);
  if (e != cudaSuccess) return e;
  const int64_t HW = (int64_t)H * W;
  {
    I4D_PROF("adaptive_voxel", st);
    depth_sum_kernel<<<dim3(blocks_per_frame(HW), F), kThreads, 0, st>>>(depth, HW, sums, counts);
    adaptive_voxel_finish_kernel<<<1, 1, 0, st>>>(sums, counts, cams, F, lambda_s, out);
  }
  return cudaGetLastError();
}

size_t motion_mask_workspace_bytes(int F) { return (size_t)(F > 0 ? F : 1) * (256 * 4 + 4) + 256; }

cudaError_t launch_motion_masks(const float* prob, int F, int h, int w, int H, int W, uint8_t* mask, int32_t* thresh,
                                void* ws, cudaStream_t st) {
  unsigned int* hist = reinterpret_cast<unsigned int*>(ws);
  int* th = thresh ? thresh : reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + 1024 * (size_t)F);
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)F * 1024, st);
  if (e != cudaSuccess) return e;
  const float sxs = (float)w / (float)W, sys = (float)h / (float)H;  // IEEE single division on the host
  const int64_t HW = (int64_t)H * W;
  I4D_PROF("motion_masks", st);
  const dim3 grid(blocks_per_frame(HW), F);
  motion_hist_kernel<<<grid, kThreads, 0, st>>>(prob, h, w, H, W, sxs, sys, hist);
  otsu_threshold_kernel<<<F, 256, 0, st>>>(hist, th);
  motion_mask_kernel<<<grid, kThreads, 0, st>>>(prob, h, w, H, W, sxs, sys, th, mask);
  return cudaGetLastError();
}

}  // namespace i4d
