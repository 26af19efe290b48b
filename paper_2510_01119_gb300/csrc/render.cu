// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile); each warp owns an 8x8 pixel block of the tile and each thread two
// vertically adjacent pixels.  The warps of a CTA do not synchronise with one another: each warp
// streams its tile's depth-sorted list in chunks of 32 entries, one entry per lane, tests the
// entry's ellipse box (precomputed by slice_project) against its own 8x8 block, and stages only the
// hits -- compacted in list order by a ballot and a prefix count -- in its private shared-memory
// slots; its pixels then visit those hits.  The test is exact: the box holds every pixel centre
// with q <= q_max.  A warp stops as soon as all its pixels are saturated (forward) or when it has
// passed its pixels' last blended fragments (backward), independently of the other warps.
// The backward walks the list back to front, recovering the transmittance from T_final by division
// (no per-fragment state), and sums each Gaussian's nine 2D-gradient components over the warp with
// a transposed shuffle reduction (14 shuffles) before nine lanes issue one atomic each.
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

// Per-warp geometry: the warp's 8x8 block and the thread's two pixels.
template <int TW>
struct WarpPix {
  int px, py0;
  float wx0, wx1, wy0, wy1;  // pixel-centre extent of the warp's block
  __device__ __forceinline__ WarpPix(const TileCoord& tc, int TH) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = tc.tx * TW + (warp % (TW / 8)) * 8;
    const int by = tc.ty * TH + (warp / (TW / 8)) * 8;
    px = bx + (lane & 7);
    py0 = by + (lane >> 3) * 2;
    wx0 = (float)bx + 0.5f;
    wx1 = (float)bx + 7.5f;
    wy0 = (float)by + 0.5f;
    wy1 = (float)by + 7.5f;
  }
  __device__ __forceinline__ bool misses(const float4 b) const {
    return b.y < wx0 || b.x > wx1 || b.w < wy0 || b.z > wy1;
  }
};

// A warp's staged hits of one chunk.
struct WarpStage {
  float4 a[32];
  float4 b[32];
  float c2[32];
  uint32_t pos[32];
  uint32_t rec[32];
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) render_fwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint2* __restrict__ ranges, Settings S,
                                                                 float* __restrict__ img, float* __restrict__ T_final,
                                                                 uint32_t* __restrict__ last_out,
                                                                 uint32_t* __restrict__ ncon) {
  __shared__ WarpStage stage[TW * TH / 64];
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31;
  WarpStage& st = stage[threadIdx.x >> 5];
  const unsigned lt = (1u << lane) - 1u;
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const uint32_t vbase = (uint32_t)tc.v * (uint32_t)n;
  const float fx = (float)wp.px + 0.5f, fy0 = (float)wp.py0 + 0.5f, fy1 = fy0 + 1.0f;
  float T0 = 1.0f, T1 = 1.0f;
  float C00 = 0.f, C01 = 0.f, C02 = 0.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
  uint32_t last0 = 0, last1 = 0, cnt0 = 0, cnt1 = 0;
  bool done0 = !in0, done1 = !in1;
  for (uint32_t base = rg.x; base < rg.y; base += 32) {
    if (__all_sync(0xffffffffu, done0 && done1)) break;
    const uint32_t idx = base + lane;
    uint32_t r = 0;
    bool hit = false;
    if (idx < rg.y) {
      r = vbase + __ldg(&ids[idx]);
      hit = !wp.misses(__ldg(&proj[3 * VN + r]));
    }
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int k = __popc(mask & lt);
      st.a[k] = __ldg(&proj[r]);
      st.b[k] = __ldg(&proj[VN + r]);
      st.c2[k] = __ldg(&proj[2 * VN + r]).x;
      st.pos[k] = idx - rg.x;
    }
    __syncwarp();
    const int cnt = __popc(mask);
    for (int t = 0; t < cnt && !(done0 && done1); ++t) {
      const float4 a = st.a[t];
      const float4 b = st.b[t];
      const float dx = __fsub_rn(fx, a.x);
      float q, G, ar, al;
      if (!done0 && eval_fragment(dx, __fsub_rn(fy0, a.y), a.z, a.w, b.x, b.y, S, q, G, ar, al)) {
        const float Tn = __fmul_rn(T0, __fsub_rn(1.0f, al));
        if (Tn < S.T_min) {
          done0 = true;
        } else {
          const float w = al * T0;
          C00 += w * b.z;
          C01 += w * b.w;
          C02 += w * st.c2[t];
          T0 = Tn;
          last0 = st.pos[t] + 1u;
          ++cnt0;
        }
      }
      if (!done1 && eval_fragment(dx, __fsub_rn(fy1, a.y), a.z, a.w, b.x, b.y, S, q, G, ar, al)) {
        const float Tn = __fmul_rn(T1, __fsub_rn(1.0f, al));
        if (Tn < S.T_min) {
          done1 = true;
        } else {
          const float w = al * T1;
          C10 += w * b.z;
          C11 += w * b.w;
          C12 += w * st.c2[t];
          T1 = Tn;
          last1 = st.pos[t] + 1u;
          ++cnt1;
        }
      }
    }
    __syncwarp();
  }
  const int64_t HW = (int64_t)tc.W * tc.H;
  if (in0) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    img[pimg] = C00 + T0 * S.bg[0];
    img[pimg + HW] = C01 + T0 * S.bg[1];
    img[pimg + 2 * HW] = C02 + T0 * S.bg[2];
    T_final[p] = T0;
    last_out[p] = last0;
    ncon[p] = cnt0;
  }
  if (in1) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    img[pimg] = C10 + T1 * S.bg[0];
    img[pimg + HW] = C11 + T1 * S.bg[1];
    img[pimg + 2 * HW] = C12 + T1 * S.bg[2];
    T_final[p] = T1;
    last_out[p] = last1;
    ncon[p] = cnt1;
  }
}

// Backward state of one pixel: transmittance in front of the next (nearer) fragment, colour
// composited behind it, upstream gradient and the position of its last blended fragment.
struct PixBwd {
  float T, S0, S1, S2, g0, g1, g2;
  uint32_t L;
};

// Gradient contribution of one fragment at one pixel (accumulated into g[9]).
__device__ __forceinline__ bool pixel_grad(PixBwd& P, float dx, float dy, const float4& a, const float4& b, float c2,
                                           const Settings& S, float* g) {
  float q, G, ar, al;
  if (!eval_fragment(dx, dy, a.z, a.w, b.x, b.y, S, q, G, ar, al)) return false;
  const float om = 1.0f - al;
  const float iom = __fdividef(1.0f, om);
  const float Tk = P.T * iom;  // transmittance in front of this fragment
  const float w = al * Tk;
  g[6] += w * P.g0;
  g[7] += w * P.g1;
  g[8] += w * P.g2;
  const float dA = P.g0 * (Tk * b.z - P.S0 * iom) + P.g1 * (Tk * b.w - P.S1 * iom) + P.g2 * (Tk * c2 - P.S2 * iom);
  P.S0 += w * b.z;
  P.S1 += w * b.w;
  P.S2 += w * c2;
  P.T = Tk;
  if (ar < S.alpha_max) {
    g[5] += dA * G;
    const float dq = -0.5f * ar * dA;
    g[0] += -2.0f * dq * (a.z * dx + a.w * dy);
    g[1] += -2.0f * dq * (a.w * dx + b.x * dy);
    g[2] += dq * dx * dx;
    g[3] += 2.0f * dq * dx * dy;
    g[4] += dq * dy * dy;
  }
  return true;
}

// Sum g[0..7] over the warp so that lane l ends up with the total of component l >> 2 (every lane
// of a group of four holds it): 4 + 2 + 1 + 1 + 1 = 9 shuffles instead of 8 x 5.
__device__ __forceinline__ float warp_transpose_sum8(const float* g, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b4 ? g[k] : g[k + 4];
    const float keep = b4 ? g[k + 4] : g[k];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b3 ? w[k] : w[k + 2];
    const float keep = b3 ? w[k + 2] : w[k];
    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? x[0] : x[1];
  const float keep = b2 ? x[1] : x[0];
  float y = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return y;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) render_bwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint2* __restrict__ ranges, Settings S,
                                                                 const float* __restrict__ T_final,
                                                                 const uint32_t* __restrict__ last_in,
                                                                 const float* __restrict__ dimg,
                                                                 float* __restrict__ grad2d) {
  __shared__ WarpStage stage[TW * TH / 64];
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31;
  WarpStage& st = stage[threadIdx.x >> 5];
  const unsigned lt = (1u << lane) - 1u;
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const uint32_t vbase = (uint32_t)tc.v * (uint32_t)n;
  const float fx = (float)wp.px + 0.5f, fy0 = (float)wp.py0 + 0.5f, fy1 = fy0 + 1.0f;
  const int64_t HW = (int64_t)tc.W * tc.H;
  PixBwd P0{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}, P1{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
  if (in0) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    P0.T = T_final[p];
    P0.L = last_in[p];
    P0.g0 = dimg[pimg];
    P0.g1 = dimg[pimg + HW];
    P0.g2 = dimg[pimg + 2 * HW];
    P0.S0 = P0.T * S.bg[0];
    P0.S1 = P0.T * S.bg[1];
    P0.S2 = P0.T * S.bg[2];
  }
  if (in1) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    P1.T = T_final[p];
    P1.L = last_in[p];
    P1.g0 = dimg[pimg];
    P1.g1 = dimg[pimg + HW];
    P1.g2 = dimg[pimg + 2 * HW];
    P1.S0 = P1.T * S.bg[0];
    P1.S1 = P1.T * S.bg[1];
    P1.S2 = P1.T * S.bg[2];
  }
  // this warp never needs entries past its pixels' last blended fragments
  const uint32_t wL = __reduce_max_sync(0xffffffffu, max(P0.L, P1.L));
  const uint32_t end = rg.x + min(wL, rg.y - rg.x);
  // component c of a 2D-gradient record lives in plane c / 4, lane c % 4 (c = 8: plane 2, lane 0)
  const int comp = lane >> 2;
  const size_t comp_off = (size_t)(comp >> 2) * VN * 4 + (comp & 3);
  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = (hi - rg.x > 32u) ? hi - 32u : rg.x;
    const uint32_t idx = lo + lane;
    uint32_t r = 0;
    bool hit = false;
    if (idx < hi) {
      r = vbase + __ldg(&ids[idx]);
      hit = !wp.misses(__ldg(&proj[3 * VN + r]));
    }
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int k = __popc(mask & lt);
      st.a[k] = __ldg(&proj[r]);
      st.b[k] = __ldg(&proj[VN + r]);
      st.c2[k] = __ldg(&proj[2 * VN + r]).x;
      st.pos[k] = idx - rg.x;
      st.rec[k] = r;
    }
    __syncwarp();
    for (int t = __popc(mask) - 1; t >= 0; --t) {  // warp-uniform trip count
      const float4 a = st.a[t];
      const float4 b = st.b[t];
      const float c2 = st.c2[t];
      const uint32_t pos = st.pos[t];
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float dx = __fsub_rn(fx, a.x);
      bool any = false;
      if (in0 && pos < P0.L) any |= pixel_grad(P0, dx, __fsub_rn(fy0, a.y), a, b, c2, S, g);
      if (in1 && pos < P1.L) any |= pixel_grad(P1, dx, __fsub_rn(fy1, a.y), a, b, c2, S, g);
      if (__any_sync(0xffffffffu, any)) {
        const float tot = warp_transpose_sum8(g, lane);
        const float gb = warp_sum(g[8]);
        const size_t rr = st.rec[t];
        if ((lane & 3) == 0) atomicAdd(&grad2d[comp_off + rr * 4], tot);
        if (lane == 1) atomicAdd(&grad2d[2 * VN * 4 + rr * 4], gb);
      }
    }
    __syncwarp();
    hi = lo;
  }
}

template <int TW, int TH>
cudaError_t launch_fwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, float* img, float* T_final, uint32_t* last, uint32_t* n_contrib,
                         cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_fwd", st);
  render_fwd_kernel<TW, TH><<<tiles, TW * TH / 2, 0, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
                                                            reinterpret_cast<const uint2*>(ranges), S, img, T_final,
                                                            last, n_contrib);
  return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_bwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, const float* T_final, const uint32_t* last, const float* dL_dimg,
                         float* grad2d, cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_bwd", st);
  render_bwd_kernel<TW, TH><<<tiles, TW * TH / 2, 0, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
                                                            reinterpret_cast<const uint2*>(ranges), S, T_final, last,
                                                            dL_dimg, grad2d);
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
