// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile); one thread per pixel.  Records of the tile's depth-sorted list are
// staged in shared memory in batches; the forward leaves the batch loop as soon as every pixel
// of the tile is saturated (block-wide vote), and the backward walks the list back to front from
// each pixel's last blended fragment, recovering the transmittance from T_final by division (no
// per-fragment state is stored).  Per-Gaussian 2D gradients are summed over the warp with
// shuffles, and lane 0 issues float4 atomics, only when some lane of the warp contributed.
#include "kernels.cuh"

namespace i4d {

namespace {

struct TileCoord {
  int v, tx, ty, W, H;
};

__device__ __forceinline__ TileCoord tile_coord(const ViewTable& vt, int tile) {
  TileCoord c;
  c.v = view_of_tile(vt, tile);
  const int lt = tile - vt.tile_off[c.v];
  c.tx = lt % vt.tiles_x[c.v];
  c.ty = lt / vt.tiles_x[c.v];
  c.W = vt.width[c.v];
  c.H = vt.height[c.v];
  return c;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_fwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                             const uint32_t* __restrict__ ids,
                                                             const uint2* __restrict__ ranges, Settings S,
                                                             float* __restrict__ img, float* __restrict__ T_final,
                                                             uint32_t* __restrict__ last_out,
                                                             uint32_t* __restrict__ ncon) {
  constexpr int B = TW * TH;
  __shared__ float4 s0[B];
  __shared__ float4 s1[B];
  __shared__ float s2[B];
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const int px = tc.tx * TW + (int)(threadIdx.x % TW);
  const int py = tc.ty * TH + (int)(threadIdx.x / TW);
  const bool inside = px < tc.W && py < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const size_t base = (size_t)tc.v * n;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  uint32_t last = 0, cnt = 0;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += B) {
    if (__syncthreads_count(done) == B) break;
    const uint32_t idx = start + threadIdx.x;
    if (idx < rg.y) {
      const size_t r = base + __ldg(&ids[idx]);
      s0[threadIdx.x] = __ldg(&proj[r]);
      s1[threadIdx.x] = __ldg(&proj[VN + r]);
      s2[threadIdx.x] = __ldg(&proj[2 * VN + r]).x;
    }
    __syncthreads();
    const int m = min((int)B, (int)(rg.y - start));
    if (!done) {
      for (int j = 0; j < m; ++j) {
        const float4 a = s0[j];
        const float4 b = s1[j];
        float q, G, ar, al;
        if (!eval_fragment(__fsub_rn(fx, a.x), __fsub_rn(fy, a.y), a.z, a.w, b.x, b.y, S, q, G, ar, al)) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
        if (Tn < S.T_min) {
          done = true;
          break;
        }
        const float w = al * T;
        C0 += w * b.z;
        C1 += w * b.w;
        C2 += w * s2[j];
        T = Tn;
        last = start + (uint32_t)j - rg.x + 1u;
        ++cnt;
      }
    }
  }
  if (inside) {
    const int64_t HW = (int64_t)tc.W * tc.H;
    const int64_t p = vt.pix_off[tc.v] + (int64_t)py * tc.W + px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)py * tc.W + px;
    img[pimg] = C0 + T * S.bg[0];
    img[pimg + HW] = C1 + T * S.bg[1];
    img[pimg + 2 * HW] = C2 + T * S.bg[2];
    T_final[p] = T;
    last_out[p] = last;
    ncon[p] = cnt;
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_bwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                             const uint32_t* __restrict__ ids,
                                                             const uint2* __restrict__ ranges, Settings S,
                                                             const float* __restrict__ T_final,
                                                             const uint32_t* __restrict__ last_in,
                                                             const float* __restrict__ dimg,
                                                             float4* __restrict__ grad2d) {
  constexpr int B = TW * TH;
  __shared__ float4 s0[B];
  __shared__ float4 s1[B];
  __shared__ float s2[B];
  __shared__ uint32_t sid[B];
  __shared__ uint32_t smax;
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const int px = tc.tx * TW + (int)(threadIdx.x % TW);
  const int py = tc.ty * TH + (int)(threadIdx.x / TW);
  const bool inside = px < tc.W && py < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const size_t base = (size_t)tc.v * n;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  float T = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
  uint32_t L = 0;
  if (inside) {
    const int64_t HW = (int64_t)tc.W * tc.H;
    const int64_t p = vt.pix_off[tc.v] + (int64_t)py * tc.W + px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)py * tc.W + px;
    T = T_final[p];
    L = last_in[p];
    g0 = dimg[pimg];
    g1 = dimg[pimg + HW];
    g2 = dimg[pimg + 2 * HW];
  }
  // colour composited behind the current fragment: starts with the background
  float S0 = T * S.bg[0], S1 = T * S.bg[1], S2 = T * S.bg[2];
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, wmax);
  __syncthreads();
  const uint32_t end = rg.x + min(smax, rg.y - rg.x);  // never past the tile's range
  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = (hi - rg.x > (uint32_t)B) ? hi - B : rg.x;
    __syncthreads();
    const uint32_t idx = lo + threadIdx.x;
    if (idx < hi) {
      const uint32_t id = __ldg(&ids[idx]);
      const size_t r = base + id;
      s0[threadIdx.x] = __ldg(&proj[r]);
      s1[threadIdx.x] = __ldg(&proj[VN + r]);
      s2[threadIdx.x] = __ldg(&proj[2 * VN + r]).x;
      sid[threadIdx.x] = id;
    }
    __syncthreads();
    for (int j = (int)(hi - lo) - 1; j >= 0; --j) {
      const uint32_t pos = lo + (uint32_t)j - rg.x;  // 0-based position in the tile list
      const float4 a = s0[j];
      const float4 b = s1[j];
      float gu = 0.f, gv = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, got = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
      bool valid = inside && pos < L;
      if (valid) {
        const float dx = __fsub_rn(fx, a.x), dy = __fsub_rn(fy, a.y);
        float q, G, ar, al;
        valid = eval_fragment(dx, dy, a.z, a.w, b.x, b.y, S, q, G, ar, al);
        if (valid) {
          const float om = 1.0f - al;
          const float Tk = T / om;  // transmittance in front of this fragment
          const float w = al * Tk;
          const float c2 = s2[j];
          gr = w * g0;
          gg = w * g1;
          gb = w * g2;
          const float iom = 1.0f / om;
          const float dA = g0 * (Tk * b.z - S0 * iom) + g1 * (Tk * b.w - S1 * iom) + g2 * (Tk * c2 - S2 * iom);
          S0 += w * b.z;
          S1 += w * b.w;
          S2 += w * c2;
          T = Tk;
          if (ar < S.alpha_max) {
            got = dA * G;
            const float dq = -0.5f * ar * dA;
            gu = -2.0f * dq * (a.z * dx + a.w * dy);
            gv = -2.0f * dq * (a.w * dx + b.x * dy);
            gca = dq * dx * dx;
            gcb = 2.0f * dq * dx * dy;
            gcc = dq * dy * dy;
          }
        }
      }
      if (__any_sync(0xffffffffu, valid)) {
        gu = warp_sum(gu);
        gv = warp_sum(gv);
        gca = warp_sum(gca);
        gcb = warp_sum(gcb);
        gcc = warp_sum(gcc);
        got = warp_sum(got);
        gr = warp_sum(gr);
        gg = warp_sum(gg);
        gb = warp_sum(gb);
        if ((threadIdx.x & 31) == 0) {
          const size_t r = base + sid[j];
          atomicAdd(&grad2d[r], make_float4(gu, gv, gca, gcb));
          atomicAdd(&grad2d[VN + r], make_float4(gcc, got, gr, gg));
          atomicAdd(reinterpret_cast<float*>(&grad2d[2 * VN + r]), gb);
        }
      }
    }
    hi = lo;
  }
}

template <int TW, int TH>
cudaError_t launch_fwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, float* img, float* T_final, uint32_t* last, uint32_t* n_contrib,
                         cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_fwd", st);
  render_fwd_kernel<TW, TH><<<tiles, TW * TH, 0, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
                                                        reinterpret_cast<const uint2*>(ranges), S, img, T_final, last,
                                                        n_contrib);
  return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_bwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, const float* T_final, const uint32_t* last, const float* dL_dimg,
                         float* grad2d, cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_bwd", st);
  render_bwd_kernel<TW, TH><<<tiles, TW * TH, 0, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
                                                        reinterpret_cast<const uint2*>(ranges), S, T_final, last,
                                                        dL_dimg, reinterpret_cast<float4*>(grad2d));
  return cudaGetLastError();
}

}  // namespace

#define I4D_TILE_DISPATCH(FN, ...)                                          \
  do {                                                                      \
    if (vt.tile_w == 16 && vt.tile_h == 16) return FN<16, 16>(__VA_ARGS__); \
    if (vt.tile_w == 8 && vt.tile_h == 8) return FN<8, 8>(__VA_ARGS__);     \
    if (vt.tile_w == 16 && vt.tile_h == 8) return FN<16, 8>(__VA_ARGS__);   \
    if (vt.tile_w == 32 && vt.tile_h == 8) return FN<32, 8>(__VA_ARGS__);   \
    if (vt.tile_w == 32 && vt.tile_h == 16) return FN<32, 16>(__VA_ARGS__); \
    return cudaErrorInvalidValue;                                           \
  } while (0)

cudaError_t launch_render_fwd(const ViewTable& vt, int n, const float* proj, const uint32_t* ids,
                              const uint32_t* ranges, const Settings& S, int batch, float* img, float* T_final,
                              uint32_t* last, uint32_t* n_contrib, cudaStream_t st) {
  (void)batch;
  if (vt.tile_off[vt.n_views] == 0) return cudaSuccess;
  I4D_TILE_DISPATCH(launch_fwd_t, vt, n, proj, ids, ranges, S, img, T_final, last, n_contrib, st);
}

cudaError_t launch_render_bwd(const ViewTable& vt, int n, const float* proj, const uint32_t* ids,
                              const uint32_t* ranges, const Settings& S, const float* T_final, const uint32_t* last,
                              const float* dL_dimg, float* grad2d, cudaStream_t st) {
  const size_t VN = (size_t)vt.n_views * n;
  cudaError_t e;
  {
    I4D_PROF("grad2d_clear", st);
    e = cudaMemsetAsync(grad2d, 0, sizeof(float) * I4D_GRAD2D_FLOATS * VN, st);
  }
  if (e != cudaSuccess) return e;
  if (vt.tile_off[vt.n_views] == 0) return cudaSuccess;
  I4D_TILE_DISPATCH(launch_bwd_t, vt, n, proj, ids, ranges, S, T_final, last, dL_dimg, grad2d, st);
}

}  // namespace i4d
