// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile).  Each warp owns an 8x8 pixel block of the tile and each thread two
// vertically adjacent pixels, so a record fetched from shared memory serves two pixels.  Records of
// the tile's depth-sorted list are staged in shared memory in batches, together with the bounding
// box of each Gaussian's 3-sigma ellipse.  Each warp then compacts, in list order, the batch
// entries whose box meets its 8x8 block (one test per entry spread over the lanes, a ballot and a
// prefix count), and its pixels visit only those: exact, because the box contains every pixel
// centre with q <= q_max, and about 40% of a 16x16 tile's list survives for a block.
// The forward leaves the batch loop once every pixel of the tile is saturated (block vote); the
// backward walks the list back to front from each pixel's last blended fragment, recovering the
// transmittance from T_final by division (no per-fragment state), and sums each Gaussian's nine 2D
// gradient components over the warp with a transposed shuffle reduction (14 shuffles) before nine
// lanes issue one atomic each.
#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int kBatch = 256;  // records staged per round

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

// Bounding box (xmin, xmax, ymin, ymax) of the ellipse q <= q_max, widened by 1% + 0.01 px so that
// float rounding can never exclude a pixel centre the per-pixel test would accept.
__device__ __forceinline__ float4 ellipse_box(float u, float v, float ca, float cb, float cc, float q_max) {
  const float det = ca * cc - cb * cb;
  if (!(det > 0.0f)) return make_float4(-1e30f, 1e30f, -1e30f, 1e30f);
  const float hx = sqrtf(q_max * cc / det) * 1.01f + 0.01f;
  const float hy = sqrtf(q_max * ca / det) * 1.01f + 0.01f;
  return make_float4(u - hx, u + hx, v - hy, v + hy);
}

// Compact, in order, the indices j < m of the batch whose boxes meet the warp's block into list;
// returns the count (warp-uniform).
template <class WP>
__device__ __forceinline__ int warp_candidates(const WP& wp, const float4* sbox, int m, uint8_t* list, int lane) {
  int cnt = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < m; r += 32) {
    const int j = r + lane;
    const bool hit = j < m && !wp.misses(sbox[j]);
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (hit) list[cnt + __popc(mask & lt)] = (uint8_t)j;
    cnt += __popc(mask);
  }
  __syncwarp();
  return cnt;
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

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) render_fwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint2* __restrict__ ranges, Settings S,
                                                                 float* __restrict__ img, float* __restrict__ T_final,
                                                                 uint32_t* __restrict__ last_out,
                                                                 uint32_t* __restrict__ ncon) {
  constexpr int NT = TW * TH / 2;
  __shared__ float4 s0[kBatch];
  __shared__ float4 s1[kBatch];
  __shared__ float4 sbox[kBatch];
  __shared__ float s2[kBatch];
  __shared__ uint8_t wlist[NT / 32][kBatch];
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const size_t base = (size_t)tc.v * n;
  const float fx = (float)wp.px + 0.5f, fy0 = (float)wp.py0 + 0.5f, fy1 = fy0 + 1.0f;
  float T0 = 1.0f, T1 = 1.0f;
  float C00 = 0.f, C01 = 0.f, C02 = 0.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
  uint32_t last0 = 0, last1 = 0, cnt0 = 0, cnt1 = 0;
  bool done0 = !in0, done1 = !in1;
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(done0 && done1) == NT) break;
    for (int k = threadIdx.x; k < kBatch; k += NT) {
      const uint32_t idx = start + k;
      if (idx < rg.y) {
        const size_t r = base + __ldg(&ids[idx]);
        const float4 a = __ldg(&proj[r]);
        const float4 b = __ldg(&proj[VN + r]);
        s0[k] = a;
        s1[k] = b;
        s2[k] = __ldg(&proj[2 * VN + r]).x;
        sbox[k] = ellipse_box(a.x, a.y, a.z, a.w, b.x, S.q_max);
      }
    }
    __syncthreads();
    const int m = min(kBatch, (int)(rg.y - start));
    const int cand = warp_candidates(wp, sbox, m, wlist[warp], lane);
    for (int t = 0; t < cand && !(done0 && done1); ++t) {
      const int j = wlist[warp][t];
      const float4 a = s0[j];
      const float4 b = s1[j];
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
          C02 += w * s2[j];
          T0 = Tn;
          last0 = start + (uint32_t)j - rg.x + 1u;
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
          C12 += w * s2[j];
          T1 = Tn;
          last1 = start + (uint32_t)j - rg.x + 1u;
          ++cnt1;
        }
      }
    }
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
  constexpr int NT = TW * TH / 2;
  __shared__ float4 s0[kBatch];
  __shared__ float4 s1[kBatch];
  __shared__ float4 sbox[kBatch];
  __shared__ float s2[kBatch];
  __shared__ uint32_t sid[kBatch];
  __shared__ uint8_t wlist[NT / 32][kBatch];
  __shared__ uint32_t smax;
  const TileCoord tc = tile_coord(vt, blockIdx.x);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint2 rg = ranges[blockIdx.x];
  const size_t VN = (size_t)vt.n_views * n;
  const size_t base = (size_t)tc.v * n;
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
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(P0.L, P1.L));
  if (lane == 0) atomicMax(&smax, wmax);
  __syncthreads();
  const uint32_t end = rg.x + min(smax, rg.y - rg.x);  // never past the tile's range
  // component c of a 2D-gradient record lives in plane c / 4, lane c % 4 (c = 8: plane 2, lane 0)
  const int comp = lane >> 2;
  const size_t comp_off = (size_t)(comp >> 2) * VN * 4 + (comp & 3);
  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = (hi - rg.x > (uint32_t)kBatch) ? hi - kBatch : rg.x;
    __syncthreads();
    for (int k = threadIdx.x; k < kBatch; k += NT) {
      const uint32_t idx = lo + k;
      if (idx < hi) {
        const uint32_t id = __ldg(&ids[idx]);
        const size_t r = base + id;
        const float4 a = __ldg(&proj[r]);
        const float4 b = __ldg(&proj[VN + r]);
        s0[k] = a;
        s1[k] = b;
        s2[k] = __ldg(&proj[2 * VN + r]).x;
        sid[k] = id;
        sbox[k] = ellipse_box(a.x, a.y, a.z, a.w, b.x, S.q_max);
      }
    }
    __syncthreads();
    const int cand = warp_candidates(wp, sbox, (int)(hi - lo), wlist[warp], lane);
    for (int t = cand - 1; t >= 0; --t) {  // warp-uniform trip count
      const int j = wlist[warp][t];
      const uint32_t pos = lo + (uint32_t)j - rg.x;  // 0-based position in the tile list
      const float4 a = s0[j];
      const float4 b = s1[j];
      const float c2 = s2[j];
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float dx = __fsub_rn(fx, a.x);
      bool any = false;
      if (in0 && pos < P0.L) any |= pixel_grad(P0, dx, __fsub_rn(fy0, a.y), a, b, c2, S, g);
      if (in1 && pos < P1.L) any |= pixel_grad(P1, dx, __fsub_rn(fy1, a.y), a, b, c2, S, g);
      if (__any_sync(0xffffffffu, any)) {
        const float tot = warp_transpose_sum8(g, lane);
        const float gb = warp_sum(g[8]);
        const size_t r = base + sid[j];
        if ((lane & 3) == 0) atomicAdd(&grad2d[comp_off + r * 4], tot);
        if (lane == 1) atomicAdd(&grad2d[2 * VN * 4 + r * 4], gb);
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
