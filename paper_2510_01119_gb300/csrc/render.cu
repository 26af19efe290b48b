// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile), taken longest list first.  Each 16-lane half-warp owns an 8x4 pixel
// block of the tile and each thread two vertically adjacent pixels, whose arithmetic runs side by
// side on the packed FP32x2 instructions (one instruction per operation for both pixels).  The warps of a CTA never
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
  uint4 x[32];  // (colour b bits, list position, record, q threshold bits)
};

// Stage the chunk [lo, hi) of the tile list: every lane tests one entry against both halves' blocks
// and writes a hit into the list of each half it meets, in list order.  Returns this half's count.
template <class WP>
__device__ __forceinline__ int stage_chunk(const WP& wp, HalfStage* st, const float4* __restrict__ proj, size_t VN,
                                           const uint32_t* __restrict__ ids, uint32_t vbase, uint32_t lo, uint32_t hi,
                                           uint32_t tile_start, int lane, int& other, const Settings& S) {
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
    const float q_thr = fminf(S.q_max, 2.0f * logf(b.y / S.alpha_min));
    const uint4 x = make_uint4(__float_as_uint(c2), pos, r, __float_as_uint(q_thr));
    if (hit0) {
      const int k = __popc(m0 & lt);
      st[0].a[k] = a; st[0].b[k] = b; st[0].x[k] = x;
    }
    if (hit1) {
      const int k = __popc(m1 & lt);
      st[1].a[k] = a; st[1].b[k] = b; st[1].x[k] = x;
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
  const float fx = (float)wp.px + 0.5f;
  const float2 fy = make_float2((float)wp.py0 + 0.5f, (float)wp.py0 + 1.5f);
  // the thread's two pixels side by side in float2 lanes: transmittance and colour
  float2 T = make_float2(1.0f, 1.0f);
  float2 Cr = make_float2(0.0f, 0.0f), Cg = Cr, Cb = Cr;
  uint32_t last0 = 0, last1 = 0, cnt0 = 0, cnt1 = 0;
  bool done0 = !in0, done1 = !in1;
  for (uint32_t base = rs; base < re; base += 32) {
    if (__all_sync(0xffffffffu, done0 && done1)) break;
    int other;
    const int cnt = stage_chunk(wp, st, proj, VN, ids, vbase, base, min(base + 32u, re), rs, lane, other, S);
    for (int t = 0; t < cnt; ++t) {
      const float4 a = mine.a[t];
      const float4 b = mine.b[t];
      const uint4 x = mine.x[t];
      const float dx = __fsub_rn(fx, a.x);
      FragPair f;
      eval_pair(dx, __fadd2_rn(fy, make_float2(-a.y, -a.y)), a.z, a.w, b.x, b.y, __uint_as_float(x.w), S, f);
      const bool k0 = f.k0 && !done0, k1 = f.k1 && !done1;
      // a kept fragment that would take T below T_min stops the pixel without being blended;
      // T (1 - alpha) is formed as T - alpha T, so a pixel with weight 0 keeps T exactly
      const float2 wk = __fmul2_rn(f.alpha, T);
      const float2 Tn = __fadd2_rn(T, make_float2(-wk.x, -wk.y));
      const bool s0 = k0 && Tn.x < S.T_min, s1 = k1 && Tn.y < S.T_min;
      done0 = done0 || s0;
      done1 = done1 || s1;
      const bool b0 = k0 && !s0, b1 = k1 && !s1;
      // a pixel that does not blend gets weight 0, which leaves its colour and T unchanged exactly
      const float2 w = make_float2(b0 ? wk.x : 0.0f, b1 ? wk.y : 0.0f);
      const float c2 = __uint_as_float(x.x);
      Cr = __ffma2_rn(w, make_float2(b.z, b.z), Cr);
      Cg = __ffma2_rn(w, make_float2(b.w, b.w), Cg);
      Cb = __ffma2_rn(w, make_float2(c2, c2), Cb);
      T = __fadd2_rn(T, make_float2(-w.x, -w.y));
      const uint32_t p1 = x.y + 1u;
      last0 = b0 ? p1 : last0;
      last1 = b1 ? p1 : last1;
      cnt0 += b0 ? 1u : 0u;
      cnt1 += b1 ? 1u : 0u;
    }
    __syncwarp();
  }
  const int64_t HW = (int64_t)tc.W * tc.H;
  if (in0) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    img[pimg] = Cr.x + T.x * S.bg[0];
    img[pimg + HW] = Cg.x + T.x * S.bg[1];
    img[pimg + 2 * HW] = Cb.x + T.x * S.bg[2];
    T_final[p] = T.x;
    last_out[p] = last0;
    ncon[p] = cnt0;
  }
  if (in1) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    img[pimg] = Cr.y + T.y * S.bg[0];
    img[pimg + HW] = Cg.y + T.y * S.bg[1];
    img[pimg + 2 * HW] = Cb.y + T.y * S.bg[2];
    T_final[p] = T.y;
    last_out[p] = last1;
    ncon[p] = cnt1;
  }
}

// Backward state of the thread's two pixels (float2 lanes): transmittance in front of the next
// (nearer) fragment, colour composited behind it, upstream gradient, and the positions of the
// pixels' last blended fragments.
struct PairBwd {
  float2 T, Sr, Sg, Sb, ur, ug, ub;
  uint32_t L0, L1;
};

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// Gradient of one fragment at the thread's two pixels, summed over the pixels into g[9] (the 2D
// record components du, dv, dconic_a, dconic_b, dconic_c, do_t, dr, dg, db).  k0 / k1 say which
// pixel blended this fragment in the forward; the other lane gets weight 0 and stays unchanged.
__device__ __forceinline__ void pair_grad(PairBwd& P, float dx, float2 dy, const FragPair& f, bool k0, bool k1,
                                          const float4& a, const float4& b, float c2, const Settings& S, float* g) {
  const float2 om = __ffma2_rn(f.alpha, f2(-1.0f), f2(1.0f));
  const float2 iom = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
  const float2 niom = __fmul2_rn(iom, f2(-1.0f));
  const float2 Tk = __fmul2_rn(P.T, iom);  // transmittance in front of this fragment
  const float2 w = __fmul2_rn(make_float2(k0 ? f.alpha.x : 0.0f, k1 ? f.alpha.y : 0.0f), Tk);
  // dL/dalpha = sum_c u_c (T_k c_k - S_c / (1 - alpha)), S_c the colour composited behind
  const float2 xr = __ffma2_rn(Tk, f2(b.z), __fmul2_rn(P.Sr, niom));
  const float2 xg = __ffma2_rn(Tk, f2(b.w), __fmul2_rn(P.Sg, niom));
  const float2 xb = __ffma2_rn(Tk, f2(c2), __fmul2_rn(P.Sb, niom));
  const float2 dA = __ffma2_rn(P.ub, xb, __ffma2_rn(P.ug, xg, __fmul2_rn(P.ur, xr)));
  const float2 s6 = __fmul2_rn(w, P.ur), s7 = __fmul2_rn(w, P.ug), s8 = __fmul2_rn(w, P.ub);
  P.Sr = __ffma2_rn(w, f2(b.z), P.Sr);
  P.Sg = __ffma2_rn(w, f2(b.w), P.Sg);
  P.Sb = __ffma2_rn(w, f2(c2), P.Sb);
  P.T = make_float2(k0 ? Tk.x : P.T.x, k1 ? Tk.y : P.T.y);
  // through alpha = o_t G (zero where the 0.99 cap binds): do_t = dA G, and with
  // dq = -dA o_t G / 2 = -p / 2: du = p (ca dx + cb dy), dv = p (cb dx + cc dy),
  // dconic = (dq dx^2, 2 dq dx dy, dq dy^2)
  const bool a0 = k0 && f.a_raw.x < S.alpha_max, a1 = k1 && f.a_raw.y < S.alpha_max;
  const float2 dAe = make_float2(a0 ? dA.x : 0.0f, a1 ? dA.y : 0.0f);
  const float2 s5 = __fmul2_rn(dAe, f.G);
  const float2 p = __fmul2_rn(f.a_raw, dAe);
  const float2 s0 = __fmul2_rn(p, __ffma2_rn(f2(a.w), dy, f2(__fmul_rn(a.z, dx))));
  const float2 s1 = __fmul2_rn(p, __ffma2_rn(f2(b.x), dy, f2(__fmul_rn(a.w, dx))));
  const float2 s2 = __fmul2_rn(p, f2(__fmul_rn(-0.5f, __fmul_rn(dx, dx))));
  const float2 s3 = __fmul2_rn(__fmul2_rn(p, f2(-1.0f)), f.dxdy);
  const float2 s4 = __fmul2_rn(p, __fmul2_rn(f2(-0.5f), f.dydy));
  g[0] = s0.x + s0.y;
  g[1] = s1.x + s1.y;
  g[2] = s2.x + s2.y;
  g[3] = s3.x + s3.y;
  g[4] = s4.x + s4.y;
  g[5] = s5.x + s5.y;
  g[6] = s6.x + s6.y;
  g[7] = s7.x + s7.y;
  g[8] = s8.x + s8.y;
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
  const float fx = (float)wp.px + 0.5f;
  const float2 fy = make_float2((float)wp.py0 + 0.5f, (float)wp.py0 + 1.5f);
  const int64_t HW = (int64_t)tc.W * tc.H;
  PairBwd P;
  P.T = P.Sr = P.Sg = P.Sb = P.ur = P.ug = P.ub = f2(0.0f);
  P.L0 = P.L1 = 0u;
  if (in0) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    P.T.x = T_final[p];
    P.L0 = last_in[p];
    P.ur.x = dimg[pimg];
    P.ug.x = dimg[pimg + HW];
    P.ub.x = dimg[pimg + 2 * HW];
  }
  if (in1) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    P.T.y = T_final[p];
    P.L1 = last_in[p];
    P.ur.y = dimg[pimg];
    P.ug.y = dimg[pimg + HW];
    P.ub.y = dimg[pimg + 2 * HW];
  }
  P.Sr = __fmul2_rn(P.T, f2(S.bg[0]));
  P.Sg = __fmul2_rn(P.T, f2(S.bg[1]));
  P.Sb = __fmul2_rn(P.T, f2(S.bg[2]));
  // this warp never needs entries past its pixels' last blended fragments
  const uint32_t wL = __reduce_max_sync(0xffffffffu, max(P.L0, P.L1));
  const uint32_t end = rs + min(wL, re - rs);
  // component c of a 2D-gradient record lives in plane c / 4, lane c % 4 (c = 8: plane 2, lane 0)
  const int comp = (lane >> 1) & 7;
  const size_t comp_off = (size_t)(comp >> 2) * VN * 4 + (comp & 3);
  const bool comp_lane = (lane & 1) == 0;
  const bool gb_lane = (lane & 15) == 1;
  for (uint32_t hi = end; hi > rs;) {
    const uint32_t lo = (hi - rs > 32u) ? hi - 32u : rs;
    int other;
    const int cnt = stage_chunk(wp, st, proj, VN, ids, vbase, lo, hi, rs, lane, other, S);
    const int trips = max(cnt, other);  // warp-uniform
    for (int t = trips - 1; t >= 0; --t) {
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool any = false;
      uint32_t rr = 0;
      if (t < cnt) {
        const float4 a = mine.a[t];
        const float4 b = mine.b[t];
        const uint4 x = mine.x[t];
        const float c2 = __uint_as_float(x.x);
        const uint32_t pos = x.y;
        rr = x.z;
        const float dx = __fsub_rn(fx, a.x);
        const float2 dy = __fadd2_rn(fy, make_float2(-a.y, -a.y));
        FragPair f;
        eval_pair(dx, dy, a.z, a.w, b.x, b.y, __uint_as_float(x.w), S, f);
        // the fragments a pixel blended are the kept ones before its last (out-of-view pixels: L = 0)
        const bool k0 = f.k0 && pos < P.L0, k1 = f.k1 && pos < P.L1;
        any = k0 || k1;
        if (any) pair_grad(P, dx, dy, f, k0, k1, a, b, c2, S, g);
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
