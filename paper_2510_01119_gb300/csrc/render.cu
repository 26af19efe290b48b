// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile), taken longest list first.  Each 16-lane half-warp owns an 8x4 pixel
// block of the tile and each thread two vertically adjacent pixels.  The warps of a CTA never
// synchronise with one another: each warp streams its tile's depth-sorted list in chunks of 32
// entries, one entry per lane, tests the entry's ellipse box (precomputed by slice_project) against
// the blocks of its two halves, and stages the hits of each half -- compacted in list order by a
// ballot and a prefix count -- in that half's shared-memory slots; each half's pixels then visit
// only those hits, the two halves side by side.  The test is exact: the box holds every pixel
// centre where the fragment can be blended (q <= q_max and alpha >= alpha_min).  A warp stops as soon as all its pixels are saturated (forward) or when
// it has passed its pixels' last blended fragments (backward).
// The backward walks the list back to front, recovering the transmittance from T_final by division
// (no per-fragment state), and sums each Gaussian's nine 2D-gradient components over its half-warp
// with a transposed shuffle reduction (12 shuffles serve the two halves' Gaussians at once) before
// nine lanes of the half issue one atomic each.
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

// Geometry of a warp: its two half-warps' 8x4 blocks and the thread's two pixels.
template <int TW>
struct WarpPix {
  int px, py0;
  int half;                       // 0: lanes 0-15, 1: lanes 16-31
  float hx0, hx1, hy0[2], hy1[2];  // pixel-centre extents of the two halves' blocks
  __device__ __forceinline__ WarpPix(const TileCoord& tc, int TH) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = tc.tx * TW + (warp % (TW / 8)) * 8;
    const int by = tc.ty * TH + (warp / (TW / 8)) * 8;
    half = lane >> 4;
    px = bx + (lane & 7);
    py0 = by + half * 4 + ((lane >> 3) & 1) * 2;
    hx0 = (float)bx + 0.5f;
    hx1 = (float)bx + 7.5f;
    hy0[0] = (float)by + 0.5f;
    hy1[0] = (float)by + 3.5f;
    hy0[1] = (float)by + 4.5f;
    hy1[1] = (float)by + 7.5f;
  }
  __device__ __forceinline__ bool misses(const float4 b, int h) const {
    return b.y < hx0 || b.x > hx1 || b.w < hy0[h] || b.z > hy1[h];
  }
};

// A half-warp's staged hits of one chunk.
struct HalfStage {
  float4 a[32];
  float4 b[32];
  float c2[32];
  uint32_t pos[32];
  uint32_t rec[32];
};

// Stage the chunk [lo, hi) of the tile list: every lane tests one entry against both halves' blocks
// and writes a hit into the list of each half it meets, in list order.  Returns this half's count.
template <class WP>
__device__ __forceinline__ int stage_chunk(const WP& wp, HalfStage* st, const float4* __restrict__ proj, size_t VN,
                                           const uint32_t* __restrict__ ids, uint32_t vbase, uint32_t lo, uint32_t hi,
                                           uint32_t tile_start, int lane, int& other) {
  const uint32_t idx = lo + lane;
  uint32_t r = 0;
  bool hit0 = false, hit1 = false;
  if (idx < hi) {
    r = vbase + __ldg(&ids[idx]);
    const float4 box = __ldg(&proj[3 * VN + r]);
    hit0 = !wp.misses(box, 0);
    hit1 = !wp.misses(box, 1);
  }
  const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
  const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
  if (hit0 || hit1) {
    const unsigned lt = (1u << lane) - 1u;
    const float4 a = __ldg(&proj[r]);
    const float4 b = __ldg(&proj[VN + r]);
    const float c2 = __ldg(&proj[2 * VN + r]).x;
    const uint32_t pos = idx - tile_start;
    if (hit0) {
      const int k = __popc(m0 & lt);
      st[0].a[k] = a; st[0].b[k] = b; st[0].c2[k] = c2; st[0].pos[k] = pos; st[0].rec[k] = r;
    }
    if (hit1) {
      const int k = __popc(m1 & lt);
      st[1].a[k] = a; st[1].b[k] = b; st[1].c2[k] = c2; st[1].pos[k] = pos; st[1].rec[k] = r;
    }
  }
  __syncwarp();
  other = __popc(wp.half ? m0 : m1);
  return __popc(wp.half ? m1 : m0);
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) render_fwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ ranges, Settings S,
                                                                 float* __restrict__ img, float* __restrict__ T_final,
                                                                 uint32_t* __restrict__ last_out,
                                                                 uint32_t* __restrict__ ncon) {
  __shared__ HalfStage stage[TW * TH / 64][2];
  const int T_all = vt.tile_off[vt.n_views];
  const int tile = (int)ranges[2 * T_all + blockIdx.x];
  const TileCoord tc = tile_coord(vt, tile);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31;
  HalfStage* st = stage[threadIdx.x >> 5];
  const HalfStage& mine = st[wp.half];
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];
  const size_t VN = (size_t)vt.n_views * n;
  const uint32_t vbase = (uint32_t)tc.v * (uint32_t)n;
  const float fx = (float)wp.px + 0.5f, fy0 = (float)wp.py0 + 0.5f, fy1 = fy0 + 1.0f;
  float T0 = 1.0f, T1 = 1.0f;
  float C00 = 0.f, C01 = 0.f, C02 = 0.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
  uint32_t last0 = 0, last1 = 0, cnt0 = 0, cnt1 = 0;
  bool done0 = !in0, done1 = !in1;
  for (uint32_t base = rs; base < re; base += 32) {
    if (__all_sync(0xffffffffu, done0 && done1)) break;
    int other;
    const int cnt = stage_chunk(wp, st, proj, VN, ids, vbase, base, min(base + 32u, re), rs, lane, other);
    for (int t = 0; t < cnt && !(done0 && done1); ++t) {
      const float4 a = mine.a[t];
      const float4 b = mine.b[t];
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
          C02 += w * mine.c2[t];
          T0 = Tn;
          last0 = mine.pos[t] + 1u;
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
          C12 += w * mine.c2[t];
          T1 = Tn;
          last1 = mine.pos[t] + 1u;
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

// Sum g[0..7] over each 16-lane half so that lane l of a half ends up with the half's total of
// component (l >> 1) & 7 (both lanes of a pair hold it): 4 + 2 + 1 + 1 = 8 shuffles.
__device__ __forceinline__ float half_transpose_sum8(const float* g, int lane) {
  const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b3 ? g[k] : g[k + 4];
    const float keep = b3 ? g[k + 4] : g[k];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float x[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b2 ? w[k] : w[k + 2];
    const float keep = b2 ? w[k + 2] : w[k];
    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = b1 ? x[0] : x[1];
  const float keep = b1 ? x[1] : x[0];
  float y = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return y;
}

__device__ __forceinline__ float half_sum(float x) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) render_bwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ ranges, Settings S,
                                                                 const float* __restrict__ T_final,
                                                                 const uint32_t* __restrict__ last_in,
                                                                 const float* __restrict__ dimg,
                                                                 float* __restrict__ grad2d) {
  __shared__ HalfStage stage[TW * TH / 64][2];
  const int T_all = vt.tile_off[vt.n_views];
  const int tile = (int)ranges[2 * T_all + blockIdx.x];
  const TileCoord tc = tile_coord(vt, tile);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31;
  HalfStage* st = stage[threadIdx.x >> 5];
  const HalfStage& mine = st[wp.half];
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];
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
  const uint32_t end = rs + min(wL, re - rs);
  // component c of a 2D-gradient record lives in plane c / 4, lane c % 4 (c = 8: plane 2, lane 0)
  const int comp = (lane >> 1) & 7;
  const size_t comp_off = (size_t)(comp >> 2) * VN * 4 + (comp & 3);
  const bool comp_lane = (lane & 1) == 0;
  const bool gb_lane = (lane & 15) == 1;
  for (uint32_t hi = end; hi > rs;) {
    const uint32_t lo = (hi - rs > 32u) ? hi - 32u : rs;
    int other;
    const int cnt = stage_chunk(wp, st, proj, VN, ids, vbase, lo, hi, rs, lane, other);
    const int trips = max(cnt, other);  // warp-uniform
    for (int t = trips - 1; t >= 0; --t) {
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool any = false;
      uint32_t rr = 0;
      if (t < cnt) {
        const float4 a = mine.a[t];
        const float4 b = mine.b[t];
        const float c2 = mine.c2[t];
        const uint32_t pos = mine.pos[t];
        rr = mine.rec[t];
        const float dx = __fsub_rn(fx, a.x);
        if (in0 && pos < P0.L) any |= pixel_grad(P0, dx, __fsub_rn(fy0, a.y), a, b, c2, S, g);
        if (in1 && pos < P1.L) any |= pixel_grad(P1, dx, __fsub_rn(fy1, a.y), a, b, c2, S, g);
      }
      const unsigned vm = __ballot_sync(0xffffffffu, any);
      if (vm) {
        const float tot = half_transpose_sum8(g, lane);
        const float gb = half_sum(g[8]);
        if ((vm >> (16 * wp.half)) & 0xffffu) {  // this half has a contribution
          if (comp_lane) atomicAdd(&grad2d[comp_off + (size_t)rr * 4], tot);
          if (gb_lane) atomicAdd(&grad2d[2 * VN * 4 + (size_t)rr * 4], gb);
        }
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
                                                            ranges, S, img, T_final, last, n_contrib);
  return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_bwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, const float* T_final, const uint32_t* last, const float* dL_dimg,
                         float* grad2d, cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_bwd", st);
  render_bwd_kernel<TW, TH><<<tiles, TW * TH / 2, 0, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
                                                            ranges, S, T_final, last, dL_dimg, grad2d);
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
