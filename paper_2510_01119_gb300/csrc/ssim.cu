// The photometric loss of the training step: (1 - lambda) L1 + lambda (1 - SSIM) (the loss weights
// of standard 3D Gaussian splatting that Sec. 4.1 adopts), over all views of a batch.
//
// SSIM per channel with an 11x11 Gaussian window (sigma 1.5, separable), zero padding, C1 = 0.01^2,
// C2 = 0.03^2.  The forward kernel stages a 42x26 halo tile of image and target in shared memory,
// blurs the five products (x, y, x^2, y^2, x y) horizontally then vertically for a 32x16 output
// tile, and writes per pixel the three partial derivatives of S with respect to the moments
// (a = dS/dmu_x, b = dS/ds_xx, c = dS/ds_xy) plus block sums of S and |x - y| (FP32 within a block,
// FP64 across blocks).  The backward kernel
// blurs a, b, c the same way (the window is symmetric) and writes
// dL/dx = ((1 - lambda) sign(x - y) - lambda (w*a + 2 x w*b + y w*c)) / count.
#include <math.h>

#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int kR = 5;                 // window radius
constexpr int kSW = 32, kSH = 16;     // output tile
constexpr int kHW = kSW + 2 * kR, kHH = kSH + 2 * kR;
constexpr int kThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Win {
  float g[2 * kR + 1];
};

// per view: first block of the view in the flattened (view, channel, tile) grid, tiles per row
struct SsimTiles {
  int off[kMaxViews + 1];
  int tx[kMaxViews];
};

__device__ __forceinline__ void decode(const ViewTable& vt, const SsimTiles& tt, int b, int& v, int& ch, int& tx,
                                       int& ty) {
  v = 0;
  while (v + 1 < vt.n_views && b >= tt.off[v + 1]) ++v;
  const int local = b - tt.off[v];
  const int per_ch = (tt.off[v + 1] - tt.off[v]) / 3;
  ch = local / per_ch;
  const int t = local - ch * per_ch;
  tx = t % tt.tx[v];
  ty = t / tt.tx[v];
}

// Block sum by a shuffle tree (a block covers at most 512 pixels, so FP32 loses nothing that
// matters; the totals over blocks accumulate in FP64).
__device__ __forceinline__ float block_sum(float x, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  x = (threadIdx.x < kThreads / 32) ? red[lane] : 0.0f;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  return x;  // valid in thread 0
}

// Work split of the blur passes: the horizontal pass gives each of kHH x 8 threads four adjacent
// outputs of a row (14 inputs in registers for 4 x 11 taps), the vertical pass gives each of the
// 256 threads two vertically adjacent outputs of a column (12 inputs for 2 x 11 taps).
constexpr int kHCols = 4;
constexpr int kHItems = kHH * (kSW / kHCols);
static_assert(kHItems <= kThreads, "one horizontal item per thread");
static_assert(kSW * (kSH / 2) == kThreads, "one vertical pair per thread");

__global__ void __launch_bounds__(kThreads) ssim_fwd_kernel(ViewTable vt, SsimTiles tt, const float* __restrict__ img,
                                                            const float* __restrict__ tgt, Win w,
                                                            float* __restrict__ abc, int64_t plane,
                                                            double* __restrict__ acc) {
  __shared__ float sx[kHH][kHW], sy[kHH][kHW];
  __shared__ float hs[5][kHH][kSW];
  __shared__ float red[kThreads / 32];
  int v, ch, tx, ty;
  decode(vt, tt, blockIdx.x, v, ch, tx, ty);
  const int W = vt.width[v], H = vt.height[v];
  const int64_t base = 3 * vt.pix_off[v] + (int64_t)ch * W * H;
  const int x0 = tx * kSW - kR, y0 = ty * kSH - kR;
  for (int i = threadIdx.x; i < kHH * kHW; i += kThreads) {
    const int r = i / kHW, c = i - r * kHW;
    const int gy = y0 + r, gx = x0 + c;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const int64_t o = base + (int64_t)gy * W + gx;
    sx[r][c] = in ? img[o] : 0.0f;
    sy[r][c] = in ? tgt[o] : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x < kHItems) {
    const int r = threadIdx.x / (kSW / kHCols), c0 = kHCols * (threadIdx.x % (kSW / kHCols));
    float m[5][kHCols];
#pragma unroll
    for (int j = 0; j < kHCols; ++j) m[0][j] = m[1][j] = m[2][j] = m[3][j] = m[4][j] = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + kHCols; ++k) {
      const float x = sx[r][c0 + k], y = sy[r][c0 + k];
      const float xx = x * x, yy = y * y, xy = x * y;
#pragma unroll
      for (int j = 0; j < kHCols; ++j) {
        if (k - j < 0 || k - j > 2 * kR) continue;
        const float g = w.g[k - j];
        m[0][j] = fmaf(g, x, m[0][j]);
        m[1][j] = fmaf(g, y, m[1][j]);
        m[2][j] = fmaf(g, xx, m[2][j]);
        m[3][j] = fmaf(g, yy, m[3][j]);
        m[4][j] = fmaf(g, xy, m[4][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kHCols; ++j) {
#pragma unroll
      for (int q = 0; q < 5; ++q) hs[q][r][c0 + j] = m[q][j];
    }
  }
  __syncthreads();
  float s_sum = 0.0f, l1_sum = 0.0f;
  {
    const int c = threadIdx.x % kSW, r0 = 2 * (threadIdx.x / kSW);
    float mo[2][5];
#pragma unroll
    for (int j = 0; j < 2; ++j) mo[j][0] = mo[j][1] = mo[j][2] = mo[j][3] = mo[j][4] = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + 2; ++k) {
      float hv[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) hv[q] = hs[q][r0 + k][c];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (k - j < 0 || k - j > 2 * kR) continue;
        const float g = w.g[k - j];
#pragma unroll
        for (int q = 0; q < 5; ++q) mo[j][q] = fmaf(g, hv[q], mo[j][q]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + j;
      const int gy = ty * kSH + r, gx = tx * kSW + c;
      if (gy >= H || gx >= W) continue;
      const float mx = mo[j][0], my = mo[j][1], sxx = mo[j][2], syy = mo[j][3], sxy = mo[j][4];
      const float vx = sxx - mx * mx, vy = syy - my * my, cov = sxy - mx * my;
      const float A1 = 2.0f * mx * my + kC1, A2 = 2.0f * cov + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
      const float iB1 = 1.0f / B1, iB2 = 1.0f / B2;
      const float S = A1 * A2 * iB1 * iB2;
      // S as a function of (mu_x, s_xx, s_xy), mu_y and s_yy held fixed
      const float da = 2.0f * my * (A2 - A1) * iB1 * iB2 - 2.0f * mx * S * (iB1 - iB2);
      const float db = -S * iB2;
      const float dc = 2.0f * A1 * iB1 * iB2;
      const int64_t o = base + (int64_t)gy * W + gx;
      abc[o] = da;
      abc[plane + o] = db;
      abc[2 * plane + o] = dc;
      s_sum += S;
      l1_sum += fabsf(sx[r + kR][c + kR] - sy[r + kR][c + kR]);
    }
  }
  s_sum = block_sum(s_sum, red);
  __syncthreads();
  l1_sum = block_sum(l1_sum, red);
  if (threadIdx.x == 0) {
    atomicAdd(&acc[0], (double)s_sum);
    atomicAdd(&acc[1], (double)l1_sum);
  }
}

__global__ void __launch_bounds__(kThreads) ssim_bwd_kernel(ViewTable vt, SsimTiles tt, const float* __restrict__ img,
                                                            const float* __restrict__ tgt, Win w,
                                                            const float* __restrict__ abc, int64_t plane, float lam,
                                                            float inv_count, float* __restrict__ dimg) {
  __shared__ float sa[3][kHH][kHW];
  __shared__ float hs[3][kHH][kSW];
  int v, ch, tx, ty;
  decode(vt, tt, blockIdx.x, v, ch, tx, ty);
  const int W = vt.width[v], H = vt.height[v];
  const int64_t base = 3 * vt.pix_off[v] + (int64_t)ch * W * H;
  const int x0 = tx * kSW - kR, y0 = ty * kSH - kR;
  for (int i = threadIdx.x; i < kHH * kHW; i += kThreads) {
    const int r = i / kHW, c = i - r * kHW;
    const int gy = y0 + r, gx = x0 + c;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const int64_t o = base + (int64_t)gy * W + gx;
    sa[0][r][c] = in ? abc[o] : 0.0f;
    sa[1][r][c] = in ? abc[plane + o] : 0.0f;
    sa[2][r][c] = in ? abc[2 * plane + o] : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x < kHItems) {
    const int r = threadIdx.x / (kSW / kHCols), c0 = kHCols * (threadIdx.x % (kSW / kHCols));
    float m[3][kHCols];
#pragma unroll
    for (int j = 0; j < kHCols; ++j) m[0][j] = m[1][j] = m[2][j] = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + kHCols; ++k) {
      const float a0 = sa[0][r][c0 + k], a1 = sa[1][r][c0 + k], a2 = sa[2][r][c0 + k];
#pragma unroll
      for (int j = 0; j < kHCols; ++j) {
        if (k - j < 0 || k - j > 2 * kR) continue;
        const float g = w.g[k - j];
        m[0][j] = fmaf(g, a0, m[0][j]);
        m[1][j] = fmaf(g, a1, m[1][j]);
        m[2][j] = fmaf(g, a2, m[2][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kHCols; ++j) {
      hs[0][r][c0 + j] = m[0][j];
      hs[1][r][c0 + j] = m[1][j];
      hs[2][r][c0 + j] = m[2][j];
    }
  }
  __syncthreads();
  {
    const int c = threadIdx.x % kSW, r0 = 2 * (threadIdx.x / kSW);
    float go[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) go[j][0] = go[j][1] = go[j][2] = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + 2; ++k) {
      const float h0 = hs[0][r0 + k][c], h1 = hs[1][r0 + k][c], h2 = hs[2][r0 + k][c];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (k - j < 0 || k - j > 2 * kR) continue;
        const float g = w.g[k - j];
        go[j][0] = fmaf(g, h0, go[j][0]);
        go[j][1] = fmaf(g, h1, go[j][1]);
        go[j][2] = fmaf(g, h2, go[j][2]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gy = ty * kSH + r0 + j, gx = tx * kSW + c;
      if (gy >= H || gx >= W) continue;
      const int64_t o = base + (int64_t)gy * W + gx;
      const float x = img[o], y = tgt[o], d = x - y;
      const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
      const float dS = go[j][0] + 2.0f * x * go[j][1] + y * go[j][2];
      dimg[o] = ((1.0f - lam) * sgn - lam * dS) * inv_count;
    }
  }
}

__global__ void photometric_finish_kernel(const double* __restrict__ acc, double inv_count, float lam,
                                          float* __restrict__ loss, float* __restrict__ ssim_mean) {
  const double s = acc[0] * inv_count, l1 = acc[1] * inv_count;
  *loss = (float)((1.0 - lam) * l1 + lam * (1.0 - s));
  if (ssim_mean) *ssim_mean = (float)s;
}

SsimTiles ssim_tiles(const ViewTable& vt) {
  SsimTiles t;
  t.off[0] = 0;
  for (int v = 0; v < vt.n_views; ++v) {
    t.tx[v] = (vt.width[v] + kSW - 1) / kSW;
    const int ty = (vt.height[v] + kSH - 1) / kSH;
    t.off[v + 1] = t.off[v] + 3 * t.tx[v] * ty;
  }
  return t;
}

Win gaussian_window() {
  double g[2 * kR + 1], s = 0.0;
  for (int k = 0; k <= 2 * kR; ++k) {
    const double x = (double)(k - kR);
    g[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
    s += g[k];
  }
  Win w;
  for (int k = 0; k <= 2 * kR; ++k) w.g[k] = (float)(g[k] / s);
  return w;
}

}  // namespace

size_t photometric_workspace_bytes(const ViewTable& vt) {
  const int64_t P = vt.pix_off[vt.n_views];
  return 256 + sizeof(float) * (size_t)(9 * (P > 0 ? P : 1));
}

cudaError_t launch_photometric_loss(const ViewTable& vt, const float* img, const float* target, float lam,
                                    float* dL_dimg, float* loss_out, float* ssim_out, void* ws, cudaStream_t st) {
  const int64_t P = vt.pix_off[vt.n_views];
  double* acc = reinterpret_cast<double*>(ws);
  float* abc = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + 256);
  cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (P > 0) {
    const SsimTiles tt = ssim_tiles(vt);
    const Win w = gaussian_window();
    const int64_t plane = 3 * P;
    const float inv_count = (float)(1.0 / (double)plane);
    {
      I4D_PROF("ssim_fwd", st);
      ssim_fwd_kernel<<<tt.off[vt.n_views], kThreads, 0, st>>>(vt, tt, img, target, w, abc, plane, acc);
    }
    {
      I4D_PROF("ssim_bwd", st);
      ssim_bwd_kernel<<<tt.off[vt.n_views], kThreads, 0, st>>>(vt, tt, img, target, w, abc, plane, lam, inv_count,
                                                               dL_dimg);
    }
  }
  photometric_finish_kernel<<<1, 1, 0, st>>>(acc, P > 0 ? 1.0 / (3.0 * (double)P) : 0.0, lam, loss_out, ssim_out);
  return cudaGetLastError();
}

}  // namespace i4d
