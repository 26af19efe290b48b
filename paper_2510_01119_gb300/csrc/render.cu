// Front-to-back compositing of all views' tiles in one launch, and its backward.
//
// One CTA per (view, tile), taken longest list first.  Each 16-lane half-warp owns an 8x4 pixel
// block of the tile and each thread two vertically adjacent pixels, whose arithmetic runs side by
// side on the packed FP32x2 instructions (one instruction per operation for both pixels).  The
// warps of a CTA never synchronise with one another: each warp streams its tile's depth-sorted list
// in chunks of 32 entries, one entry per lane, tests the entry's ellipse box (precomputed by
// slice_project) against the blocks of its two halves, and stages the hits of each half --
// compacted in list order by a ballot and a prefix count -- in shared memory (the forward keeps a
// copy per half, the backward stores each entry once with per-half index lists); each half's pixels
// then visit only those hits, the two halves side by side.  The test is exact: the box holds every pixel
// centre where the fragment can be blended (q <= q_max and alpha >= alpha_min).  A warp stops as
// soon as all its pixels are saturated (forward) or when it has passed its pixels' last blended
// fragments (backward).
// The backward walks the list back to front, recovering the transmittance from T_final by division
// (no per-fragment state).  Per group of up to 16 staged hits of each half it runs two phases: the
// pixel lanes carry the recurrence and leave two numbers per (pixel, hit) in shared memory, then
// one to four lanes per hit sum its gradient over the block's 32 pixels in registers and add the
// nine components with three vector reductions -- no reduction across the pixel lanes.
#include "kernels.cuh"

namespace i4d {

namespace {

// Fire-and-forget global float adds: one component, or four consecutive components at a 16-byte
// aligned address (every record of the 2D-gradient planes starts on 16 bytes; i4d_render_bwd
// rejects a plane base that does not).
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.v4.f32.add [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

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
  // Whether a staged record (a = (u, v, sa, sb2), b = (sc, o_t, m_thr, r)) can be kept at some pixel
  // centre of half h's block: the largest exponent m = sa dx^2 + sb2 dx dy + sc dy^2 over the block's
  // rectangle of pixel centres reaches m_thr.  m is concave, so its maximum over the rectangle is 0
  // at the projected mean when that lies inside, else it lies on one of the (at most two) edges facing
  // the mean, where m is a 1D quadratic maximised at its stationary point clamped to the edge.  The
  // test keeps a slack of 1e-4 (relative and absolute) so that rounding never drops a pixel the
  // per-pixel test keeps.
  __device__ __forceinline__ bool meets(const float4 a, const float4 b, int h) const {
    const float u = a.x, v = a.y, sa = a.z, sb2 = a.w, sc = b.x, mthr = b.z;
    const float y0 = hy0[h], y1 = hy1[h];
    const float dxc = fminf(fmaxf(u, hx0), hx1) - u;
    const float dyc = fminf(fmaxf(v, y0), y1) - v;
    const float dy1 = fminf(fmaxf(v - __fdividef(0.5f * sb2, sc) * dxc, y0), y1) - v;
    const float dx2 = fminf(fmaxf(u - __fdividef(0.5f * sb2, sa) * dyc, hx0), hx1) - u;
    const float m1 = dxc != 0.0f ? fmaf(sa * dxc, dxc, fmaf(sb2 * dxc, dy1, sc * dy1 * dy1)) : -INFINITY;
    const float m2 = dyc != 0.0f ? fmaf(sa * dx2, dx2, fmaf(sb2 * dx2, dyc, sc * dyc * dyc)) : -INFINITY;
    const float m = (dxc == 0.0f && dyc == 0.0f) ? 0.0f : fmaxf(m1, m2);
    return m >= mthr - (1e-4f * fabsf(mthr) + 1e-4f);
  }
};

// The staged form of a record (slice_project writes it ready: 64 bytes, the box first): a = (u, v,
// sa, sb2), b = (sc, o_t, m_thr, r), c = (g, b, list position bits, record index bits), with the
// conic pre-scaled by kFalloff and m_thr the exponent threshold of the kept test (see eval_pair).
// The box was read to test the entry; the other 48 bytes sit in the same 64-byte segment.
__device__ __forceinline__ void stage_entry(const float4* __restrict__ proj, uint32_t r, uint32_t pos, float4& a,
                                            float4& b, float4& c) {
  a = __ldg(&proj[4 * (size_t)r + 1]);
  b = __ldg(&proj[4 * (size_t)r + 2]);
  const float4 t = __ldg(&proj[4 * (size_t)r + 3]);
  c = make_float4(t.x, t.y, __uint_as_float(pos), __uint_as_float(r));
}

// A half-warp's staged hits of one batch of B list entries.
// One staged entry (48 bytes: one address per entry, the three parts at fixed offsets).
struct Staged {
  float4 a, b, c;
};

template <int B>
struct HalfStage {
  Staged e[B];
};

// Stage the batch [lo, hi) of the tile list (hi - lo <= B): 32 entries at a time, every lane tests
// one entry against both halves' blocks and writes a hit into the list of each half it meets, in
// list order (B = 16 leaves the upper lanes idle).  Returns this half's count.
template <int B, class WP>
__device__ __forceinline__ int stage_batch(const WP& wp, HalfStage<B>* st, const float4* __restrict__ proj,
                                           const uint32_t* __restrict__ ids, uint32_t vbase, uint32_t lo, uint32_t hi,
                                           uint32_t tile_start, int lane, int& other) {
  int c0 = 0, c1 = 0;
#pragma unroll
  for (int sub = 0; sub < (B + 31) / 32; ++sub) {
    const uint32_t idx = lo + 32u * sub + lane;
    uint32_t r = 0;
    bool hit0 = false, hit1 = false;
    if ((B >= 32 || lane < B) && idx < hi) {
      r = vbase + __ldg(&ids[idx]);
      const float4 box = __ldg(&proj[4 * (size_t)r]);
      hit0 = !wp.misses(box, 0);
      hit1 = !wp.misses(box, 1);
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
    const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
    if (hit0 || hit1) {
      const unsigned lt = (1u << lane) - 1u;
      float4 a, b, c;
      stage_entry(proj, r, idx - tile_start, a, b, c);
      if (hit0) {
        const int k = c0 + __popc(m0 & lt);
        st[0].e[k] = Staged{a, b, c};
      }
      if (hit1) {
        const int k = c1 + __popc(m1 & lt);
        st[1].e[k] = Staged{a, b, c};
      }
    }
    c0 += __popc(m0);
    c1 += __popc(m1);
  }
  // the half with fewer hits gets null entries up to the other's count (never kept, colour 0, all
  // values finite), so that both halves run the same number of iterations
  const int lo_c = min(c0, c1), hi_c = max(c0, c1);
  for (int k = lo_c + lane; k < hi_c; k += 32) {
    const float inf = __int_as_float(0x7f800000);
    st[c0 < c1 ? 0 : 1].e[k] =
        Staged{make_float4(0.0f, 0.0f, 0.0f, 0.0f), make_float4(0.0f, 0.0f, inf, 0.0f), make_float4(0.0f, 0.0f, 0.0f, 0.0f)};
  }
  __syncwarp();
  other = wp.half ? c0 : c1;
  return wp.half ? c1 : c0;
}

// The backward's staging: the chunk's entries that hit either half, stored once in list order, and
// per half the positions of its hits among them (a hit of both halves is staged once).
struct SharedStage {
  Staged e[32];
  uint8_t idx[2][32];
};

template <class WP>
__device__ __forceinline__ int stage_chunk_shared(const WP& wp, SharedStage& st, const float4* __restrict__ proj,
                                                  const uint32_t* __restrict__ ids, uint32_t vbase, uint32_t lo,
                                                  uint32_t hi, uint32_t tile_start, int lane, int& other) {
  const uint32_t idx = lo + lane;
  uint32_t r = 0;
  bool hit0 = false, hit1 = false;
  float4 a, b, c;
  if (idx < hi) {
    r = vbase + __ldg(&ids[idx]);
    const float4 box = __ldg(&proj[4 * (size_t)r]);
    hit0 = !wp.misses(box, 0);
    hit1 = !wp.misses(box, 1);
    if (hit0 || hit1) {
      stage_entry(proj, r, idx - tile_start, a, b, c);
      hit0 = hit0 && wp.meets(a, b, 0);
      hit1 = hit1 && wp.meets(a, b, 1);
    }
  }
  const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
  const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
  if (hit0 || hit1) {
    const unsigned lt = (1u << lane) - 1u;
    const int k = __popc((m0 | m1) & lt);
    st.e[k] = Staged{a, b, c};
    if (hit0) st.idx[0][__popc(m0 & lt)] = (uint8_t)k;
    if (hit1) st.idx[1][__popc(m1 & lt)] = (uint8_t)k;
  }
  __syncwarp();
  other = __popc(wp.half ? m0 : m1);
  return __popc(wp.half ? m1 : m0);
}

// Resident CTAs per SM the forward is compiled for: 36 warps, which caps the registers at 56 per
// thread (the kernel needs 63 unbounded, which allows 32 warps).
template <int TW, int TH>
constexpr int fwd_min_blocks() {
  return (TW * TH / 64) >= 36 ? 1 : (36 / (TW * TH / 64) > 32 ? 32 : 36 / (TW * TH / 64));
}

// COUNT: also write n_contrib, the number of fragments each pixel blended (an extra add per pixel and
// fragment; the training step does not need it).  B: list entries each warp stages per round.
template <int TW, int TH, bool COUNT, int B>
__global__ void __launch_bounds__(TW * TH / 2, fwd_min_blocks<TW, TH>()) render_fwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ ranges, Settings S,
                                                                 float* __restrict__ img, float* __restrict__ T_final,
                                                                 uint32_t* __restrict__ stop_out,
                                                                 uint32_t* __restrict__ ncon) {
  __shared__ HalfStage<B> stage[TW * TH / 64][2];
  const int T_all = vt.tile_off[vt.n_views];
  const int tile = (int)ranges[2 * T_all + blockIdx.x];
  const TileCoord tc = tile_coord(vt, tile);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31;
  HalfStage<B>* st = stage[threadIdx.x >> 5];
  const HalfStage<B>& mine = st[wp.half];
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];
  const uint32_t vbase = (uint32_t)tc.v * (uint32_t)n;
  const float fx = (float)wp.px + 0.5f;
  const float2 fy = make_float2((float)wp.py0 + 0.5f, (float)wp.py0 + 1.5f);
  // The thread's two pixels side by side in float2 lanes: transmittance and colour.  A pixel that
  // stops keeps its final transmittance in Tf and goes on with T = 0 and a stop threshold of -1:
  // every later fragment then has weight alpha * 0 = 0 (colour and T unchanged exactly) and cannot
  // stop it again, so the hot loop needs no per-pixel "done" logic.  Pixels outside the view start
  // stopped.
  float2 T = make_float2(in0 ? 1.0f : 0.0f, in1 ? 1.0f : 0.0f);
  float2 thr = make_float2(in0 ? S.T_min : -1.0f, in1 ? S.T_min : -1.0f);
  float2 Tf = T;
  float2 Cr = make_float2(0.0f, 0.0f), Cg = Cr, Cb = Cr;
  uint32_t stop0 = in0 ? re - rs : 0u, stop1 = in1 ? re - rs : 0u;
  uint32_t cnt0 = 0, cnt1 = 0;
  for (uint32_t base = rs; base < re; base += B) {
    if (__all_sync(0xffffffffu, thr.x < 0.0f && thr.y < 0.0f)) break;
    int other;
    const int cnt = stage_batch<B>(wp, st, proj, ids, vbase, base, min(base + (uint32_t)B, re), rs, lane, other);
    // both halves run max(cnt, other) iterations (the shorter list is padded with null entries), so
    // the warp-wide vote below is reached by all 32 lanes together
    const int tmax = max(cnt, other);
#pragma unroll 2
    for (int t = 0; t < tmax; ++t) {
      const Staged& se = mine.e[t];
      const float4 a = se.a;
      const float4 b = se.b;
      const float4 c = se.c;
      const float dx = __fsub_rn(fx, a.x);
      FragPair f;
      eval_pair(dx, __fadd2_rn(fy, make_float2(-a.y, -a.y)), a.z, a.w, b.x, b.y, b.z, S, f);
      // weight alpha T of a kept fragment (T (1 - alpha) is formed as T - alpha T, so a weight of 0
      // keeps T exactly)
      const float2 wk = __fmul2_rn(f.alpha, T);
      float2 w = make_float2(f.k0 ? wk.x : 0.0f, f.k1 ? wk.y : 0.0f);
      float2 Tn = __fadd2_rn(T, make_float2(-w.x, -w.y));
      if (__any_sync(0xffffffffu, Tn.x < thr.x || Tn.y < thr.y)) {
        // a kept fragment that would take T below T_min stops the pixel without being blended
        if (Tn.x < thr.x) {
          Tf.x = T.x;
          stop0 = __float_as_uint(c.z);
          thr.x = -1.0f;
          w.x = 0.0f;
          Tn.x = 0.0f;
        }
        if (Tn.y < thr.y) {
          Tf.y = T.y;
          stop1 = __float_as_uint(c.z);
          thr.y = -1.0f;
          w.y = 0.0f;
          Tn.y = 0.0f;
        }
      }
      Cr = __ffma2_rn(w, make_float2(b.w, b.w), Cr);
      Cg = __ffma2_rn(w, make_float2(c.x, c.x), Cg);
      Cb = __ffma2_rn(w, make_float2(c.y, c.y), Cb);
      T = Tn;
      if (COUNT) {
        // a blended fragment has weight >= alpha_min T_min > 0
        cnt0 += w.x != 0.0f ? 1u : 0u;
        cnt1 += w.y != 0.0f ? 1u : 0u;
      }
    }
    __syncwarp();
  }
  if (thr.x >= 0.0f) Tf.x = T.x;
  if (thr.y >= 0.0f) Tf.y = T.y;
  const int64_t HW = (int64_t)tc.W * tc.H;
  if (in0) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)wp.py0 * tc.W + wp.px;
    img[pimg] = Cr.x + Tf.x * S.bg[0];
    img[pimg + HW] = Cg.x + Tf.x * S.bg[1];
    img[pimg + 2 * HW] = Cb.x + Tf.x * S.bg[2];
    T_final[p] = Tf.x;
    stop_out[p] = stop0;
    if (COUNT) ncon[p] = cnt0;
  }
  if (in1) {
    const int64_t p = vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    const int64_t pimg = 3 * vt.pix_off[tc.v] + (int64_t)(wp.py0 + 1) * tc.W + wp.px;
    img[pimg] = Cr.y + Tf.y * S.bg[0];
    img[pimg + HW] = Cg.y + Tf.y * S.bg[1];
    img[pimg + 2 * HW] = Cb.y + Tf.y * S.bg[2];
    T_final[p] = Tf.y;
    stop_out[p] = stop1;
    if (COUNT) ncon[p] = cnt1;
  }
}

// Backward state of the thread's two pixels (float2 lanes): transmittance in front of the next
// (nearer) fragment, uNS = -sum_c u_c S_c with S_c the colour composited behind it (the only form of
// S the gradient needs), the upstream gradient u, and the pixels' stop positions.
struct PairBwd {
  float2 T, uNS, ur, ug, ub;
  uint32_t L0, L1;
};

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// The backward runs in two phases per group of up to kGroup = 16 hits of each half.  Phase A (lanes =
// pixel pairs, hits back to front) carries the per-pixel recurrence -- the transmittance in front
// of the fragment, the colour composited behind it -- and leaves, for every (pixel, hit) slot, the
// two numbers the hit's gradient is linear in: s = dL/dalpha G (zero where the fragment was not
// blended or the 0.99 cap binds) and -w = -alpha T.  Phase B (lanes = hits) sums them over the
// block's 32 pixels in registers (1, 2 or 4 lanes per hit by the group's size):
//   do_t = sum s,  dc = sum w u_c,
//   du = o_t (ca sum s dx + cb sum s dy),  dv = o_t (cb sum s dx + cc sum s dy),
//   dconic = -o_t (sum s dx^2 / 2, sum s dx dy, sum s dy^2 / 2)
// (dL/dq = -dL/dalpha o_t G / 2 = -o_t s / 2), then adds the nine totals to the record's three
// 2D-gradient planes (components 0-3, 4-7, 8).  Phase A carries S negated and stores -w, which
// saves the negations in dL/dalpha; phase B flips the colour totals back.
constexpr int kGroup = 16;

// Placement of pixel pair q's entries: with z(q) = (q & 7) ^ 6 (q >> 3), the 16-byte slots that one
// quarter-warp touches fall in distinct bank groups for every access pattern of the two phases --
// phase A (fixed hit, q = 0..7 or 8..15) and phase B with 1, 2 or 4 lanes per hit (hits k and pairs
// q = i; q = i, 8 + i; q = i, 4 + i, 8 + i, 12 + i).
__device__ __forceinline__ int pair_swz(int q) { return (q & 7) ^ (6 * (q >> 3)); }

struct BwdWarp {
  SharedStage st;
  // (s_upper, s_lower, -w_upper, -w_lower) of pixel pair q for hit slot k, at [q][k ^ pair_swz(q)]
  float4 sw[2][16][kGroup];
  float4 urg[2][16];  // upstream gradient of pair q at [(q & 8) | pair_swz(q)]: (r_up, r_low, g_up, g_low)
  float2 ub[2][16];   // (b_upper, b_lower) of pair q
};

template <int TW, int TH>
constexpr size_t bwd_smem_bytes() {
  return sizeof(BwdWarp) * (TW * TH / 64);
}

// One hit's nine sums over (part of) its block: sum s, sum s dx, sum s dy, sum s dx^2, sum s dx dy,
// sum s dy^2 and sum_c (-w) u_c, with (dx, dy) the pixel centre minus the projected mean.
struct HitSums {
  float s0, sx, sy, sxx, sxy, syy, cr, cg, cb;
};

// Adds to h the sums of hit slot k over NK consecutive pixel pairs q = qb .. qb + NK - 1 of one row
// pair.  The pairs' columns are c0 + i (i = 0 .. NK - 1) and their rows r0 and r0 + 1, so with
// cx = x(c0) - u and cy = y(r0) - v the offsets are dx = i + cx, dy = {0, 1} + cy: the loop only
// accumulates sum s, sum i s and sum i^2 s (per row, packed) with i a compile-time constant, and the
// offsets enter once at the end.
template <int NK>
__device__ __forceinline__ void seg_sums(const float4 (*sw)[kGroup], const float4* urg, const float2* ub, int qb,
                                         int k, float cx, float cy, HitSums& h) {
  float2 A = f2(0.0f), B = A, C = A, ur = A, ug = A, uB = A;
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int q = qb + i;
    const int z = pair_swz(q);
    const float4 v = sw[q][k ^ z];
    const float4 u = urg[(q & 8) | z];
    const float2 u3 = ub[q];
    const float2 sv = make_float2(v.x, v.y), nwv = make_float2(v.z, v.w);
    A = __fadd2_rn(A, sv);
    if (i == 1) {
      B = __fadd2_rn(B, sv);
      C = __fadd2_rn(C, sv);
    } else if (i > 1) {
      B = __ffma2_rn(sv, f2((float)i), B);
      C = __ffma2_rn(sv, f2((float)(i * i)), C);
    }
    ur = __ffma2_rn(nwv, make_float2(u.x, u.y), ur);
    ug = __ffma2_rn(nwv, make_float2(u.z, u.w), ug);
    uB = __ffma2_rn(nwv, u3, uB);
  }
  // sum s (i + cx)^j (r + cy)^l with r in {0, 1} the row within the pair (r^2 = r)
  const float a = A.x + A.y, ay = A.y, b = B.x + B.y, by = B.y, c = C.x + C.y;
  h.s0 += a;
  h.sx += fmaf(cx, a, b);
  h.sy += fmaf(cy, a, ay);
  h.sxx += fmaf(cx, fmaf(cx, a, 2.0f * b), c);
  h.sxy += fmaf(cx, fmaf(cy, a, ay), fmaf(cy, b, by));
  h.syy += fmaf(cy, fmaf(cy, a, 2.0f * ay), ay);
  h.cr += ur.x + ur.y;
  h.cg += ug.x + ug.y;
  h.cb += uB.x + uB.y;
}

__device__ __forceinline__ void hit_sums_xor(HitSums& h, int m) {
  h.s0 += __shfl_xor_sync(0xffffffffu, h.s0, m);
  h.sx += __shfl_xor_sync(0xffffffffu, h.sx, m);
  h.sy += __shfl_xor_sync(0xffffffffu, h.sy, m);
  h.sxx += __shfl_xor_sync(0xffffffffu, h.sxx, m);
  h.sxy += __shfl_xor_sync(0xffffffffu, h.sxy, m);
  h.syy += __shfl_xor_sync(0xffffffffu, h.syy, m);
  h.cr += __shfl_xor_sync(0xffffffffu, h.cr, m);
  h.cg += __shfl_xor_sync(0xffffffffu, h.cg, m);
  h.cb += __shfl_xor_sync(0xffffffffu, h.cb, m);
}

// Phase B with S lanes per hit (S = 1, 2 or 4; 16 / S hits of each half at most): lane l of a half
// takes hit slot l / S and the S-th part l % S of the block's 16 pixel pairs (S = 1: both row
// pairs; S = 2: row pair l % 2; S = 4: half a row pair), then the S lanes of a hit add their sums
// and the first issues the hit's three reductions.
template <int S>
__device__ __forceinline__ void phase_b(const BwdWarp& W, int half, int l16, int hc, int glo, const uint8_t* my_idx,
                                        float bx0, float by0, size_t VN, float* __restrict__ grad2d) {
  const int k = l16 / S, part = l16 % S;
  const bool valid = k < hc;
  HitSums h = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
  uint32_t rr = 0;
  if (valid) {
    const int e = my_idx[glo + k];
    a = W.st.e[e].a;
    b = W.st.e[e].b;
    rr = __float_as_uint(W.st.e[e].c.w);
    const float4(*sw)[kGroup] = W.sw[half];
    if (S == 1) {
      const float cx = __fsub_rn(bx0, a.x);
      seg_sums<8>(sw, W.urg[half], W.ub[half], 0, k, cx, __fsub_rn(by0, a.y), h);
      seg_sums<8>(sw, W.urg[half], W.ub[half], 8, k, cx, __fsub_rn(by0 + 2.0f, a.y), h);
    } else if (S == 2) {
      seg_sums<8>(sw, W.urg[half], W.ub[half], 8 * part, k, __fsub_rn(bx0, a.x),
                  __fsub_rn(by0 + (float)(2 * part), a.y), h);
    } else {
      seg_sums<4>(sw, W.urg[half], W.ub[half], 4 * part, k, __fsub_rn(bx0 + (float)(4 * (part & 1)), a.x),
                  __fsub_rn(by0 + (float)(2 * (part >> 1)), a.y), h);
    }
  }
  if (S >= 2) hit_sums_xor(h, 1);
  if (S >= 4) hit_sums_xor(h, 2);
  if (valid && part == 0) {
    // the staged conic is scaled by kFalloff (see eval_pair); the gradients need it plain
    const float o = b.y, ca = kFalloffInv * a.z, cb = 0.5f * kFalloffInv * a.w, cc = kFalloffInv * b.x;
    const float g[9] = {o * (ca * h.sx + cb * h.sy), o * (cb * h.sx + cc * h.sy), -0.5f * o * h.sxx, -o * h.sxy,
                        -0.5f * o * h.syy, h.s0, -h.cr, -h.cg, -h.cb};
    // a hit that blended none of the block's pixels has all nine totals zero; adding zeros changes
    // nothing, so such hits issue no reductions
    bool nz = false;
#pragma unroll
    for (int c = 0; c < 9; ++c) nz = nz || g[c] != 0.0f;
    if (nz) {
      // planes: float4 (g0..g3), float4 (g4..g7), float (g8), each VN long
      red_add4(grad2d + (size_t)rr * 4, g[0], g[1], g[2], g[3]);
      red_add4(grad2d + (VN + rr) * 4, g[4], g[5], g[6], g[7]);
      red_add(grad2d + VN * 8 + rr, g[8]);
    }
  }
}

// Phase A over this half's hits t = thi - 1 .. glo of a group, back to front.  A fragment the pixel
// did not blend (not kept, or at or after its stop position) enters with alpha 0, which leaves T
// and the colour behind unchanged exactly (T_k = T + T alpha / (1 - alpha)) and makes its (s, -w)
// slot zero.  CHECK: compare the hits' list positions with the pixels' stop positions; a chunk that
// lies wholly below every stop position of the warp needs no comparison.
template <bool CHECK>
__device__ __forceinline__ void phase_a(const SharedStage& stg, const uint8_t* my_idx, int thi, int glo, float fx,
                                        float2 fy, const Settings& S, PairBwd& P, float4* sw_mine, int zl) {
  for (int t = thi - 1; t >= glo; --t) {
    const int e = my_idx[t];
    const Staged& se = stg.e[e];
    const float4 a = se.a;
    const float4 b = se.b;
    const float4 c = se.c;
    const float dx = __fsub_rn(fx, a.x);
    const float2 dy = __fadd2_rn(fy, make_float2(-a.y, -a.y));
    FragPair f;
    eval_pair(dx, dy, a.z, a.w, b.x, b.y, b.z, S, f);
    bool k0 = f.k0, k1 = f.k1;
    if (CHECK) {
      const uint32_t pos = __float_as_uint(c.z);
      k0 = k0 && pos < P.L0;
      k1 = k1 && pos < P.L1;
    }
    const float2 ae = make_float2(k0 ? f.alpha.x : 0.0f, k1 ? f.alpha.y : 0.0f);
    const float2 om = __fadd2_rn(f2(1.0f), make_float2(-ae.x, -ae.y));
    const float2 iom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    // transmittance in front of this fragment
    const float2 Tk = __ffma2_rn(P.T, __fmul2_rn(ae, iom), P.T);
    const float2 nw = __fmul2_rn(make_float2(-ae.x, -ae.y), Tk);  // -alpha T_k
    // dL/dalpha = sum_c u_c (T_k c_k - S_c / (1 - alpha)) = (T (u . c_k) + uNS) / (1 - alpha), T the
    // transmittance behind; the colour behind grows by alpha T_k c_k, so uNS by -alpha T_k (u . c_k)
    const float2 uc = __ffma2_rn(P.ub, f2(c.y), __ffma2_rn(P.ug, f2(c.x), __fmul2_rn(P.ur, f2(b.w))));
    const float2 dA = __fmul2_rn(iom, __ffma2_rn(P.T, uc, P.uNS));
    P.uNS = __ffma2_rn(nw, uc, P.uNS);
    P.T = Tk;
    // alpha = o_t G carries the gradient only below the alpha_max cap
    const float2 Ge = make_float2(k0 && f.a_raw.x < S.alpha_max ? f.G.x : 0.0f,
                                  k1 && f.a_raw.y < S.alpha_max ? f.G.y : 0.0f);
    const float2 sv = __fmul2_rn(dA, Ge);
    sw_mine[(t - glo) ^ zl] = make_float4(sv.x, sv.y, nw.x, nw.y);
  }
}

// Resident CTAs per SM the backward is compiled for: 20 warps (10.3 KB of shared memory each),
// which caps the registers at 102 per thread.
template <int TW, int TH>
constexpr int bwd_min_blocks() {
  return (TW * TH / 64) >= 20 ? 1 : 20 / (TW * TH / 64);
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2, bwd_min_blocks<TW, TH>()) render_bwd_kernel(ViewTable vt, int n, const float4* __restrict__ proj,
                                                                 const uint32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ ranges, Settings S,
                                                                 const float* __restrict__ T_final,
                                                                 const uint32_t* __restrict__ last_in,
                                                                 const float* __restrict__ dimg,
                                                                 float* __restrict__ grad2d) {
  extern __shared__ float4 bwd_smem[];
  BwdWarp& W = reinterpret_cast<BwdWarp*>(bwd_smem)[threadIdx.x >> 5];
  const int T_all = vt.tile_off[vt.n_views];
  const int tile = (int)ranges[2 * T_all + blockIdx.x];
  const TileCoord tc = tile_coord(vt, tile);
  const WarpPix<TW> wp(tc, TH);
  const int lane = threadIdx.x & 31, l16 = lane & 15;
  const SharedStage& stg = W.st;
  const uint8_t* my_idx = W.st.idx[wp.half];
  const bool in0 = wp.px < tc.W && wp.py0 < tc.H;
  const bool in1 = wp.px < tc.W && wp.py0 + 1 < tc.H;
  const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];
  const size_t VN = (size_t)vt.n_views * n;
  const uint32_t vbase = (uint32_t)tc.v * (uint32_t)n;
  const float fx = (float)wp.px + 0.5f;
  const float2 fy = make_float2((float)wp.py0 + 0.5f, (float)wp.py0 + 1.5f);
  const int64_t HW = (int64_t)tc.W * tc.H;
  PairBwd P;
  P.T = P.uNS = P.ur = P.ug = P.ub = f2(0.0f);
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
  const int zl = pair_swz(l16);
  W.urg[wp.half][(l16 & 8) | zl] = make_float4(P.ur.x, P.ur.y, P.ug.x, P.ug.y);
  W.ub[wp.half][l16] = P.ub;
  // behind the last fragment: the background, weighted by T_final
  P.uNS = __fmul2_rn(P.T, __ffma2_rn(P.ub, f2(-S.bg[2]), __ffma2_rn(P.ug, f2(-S.bg[1]), __fmul2_rn(P.ur, f2(-S.bg[0])))));
  // this warp never needs entries at or past its pixels' stop positions, and below the smallest stop
  // position of its pixels in the view every kept fragment was blended (pixels outside the view have
  // T = 0 and no upstream gradient: whatever they take contributes exactly zero)
  const uint32_t wL = __reduce_max_sync(0xffffffffu, max(P.L0, P.L1));
  const uint32_t wLmin = __reduce_min_sync(0xffffffffu, min(in0 ? P.L0 : 0xffffffffu, in1 ? P.L1 : 0xffffffffu));
  const uint32_t end = rs + min(wL, re - rs);
  // pixel-centre offsets of this half's block: lane j's pair sits in column j & 7, rows 2 (j >> 3) + {0, 1}
  const float bx0 = wp.hx0, by0 = wp.hy0[wp.half];
  float4* sw_mine = &W.sw[wp.half][l16][0];
  for (uint32_t hi = end; hi > rs;) {
    const uint32_t lo = (hi - rs > 32u) ? hi - 32u : rs;
    int other;
    const int cnt = stage_chunk_shared(wp, W.st, proj, ids, vbase, lo, hi, rs, lane, other);
    for (int ghi = max(cnt, other); ghi > 0; ghi -= kGroup) {  // warp-uniform
      const int glo = max(ghi - kGroup, 0);
      // ---- phase A: the recurrence, hits back to front ----
      if (hi - rs <= wLmin)  // warp-uniform
        phase_a<false>(stg, my_idx, min(ghi, cnt), glo, fx, fy, S, P, sw_mine, zl);
      else
        phase_a<true>(stg, my_idx, min(ghi, cnt), glo, fx, fy, S, P, sw_mine, zl);
      __syncwarp();
      // ---- phase B: per hit, its sums over the block; 1, 2 or 4 lanes per hit by the group's size ----
      const int hc = max(min(ghi, cnt) - glo, 0);
      const int hmax = max(hc, min(ghi, other) - glo);  // warp-uniform
      if (hmax <= 4)
        phase_b<4>(W, wp.half, l16, hc, glo, my_idx, bx0, by0, VN, grad2d);
      else if (hmax <= 8)
        phase_b<2>(W, wp.half, l16, hc, glo, my_idx, bx0, by0, VN, grad2d);
      else
        phase_b<1>(W, wp.half, l16, hc, glo, my_idx, bx0, by0, VN, grad2d);
      __syncwarp();
    }
    __syncwarp();
    hi = lo;
  }
}

template <int TW, int TH, int B>
cudaError_t launch_fwd_tb(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                          const Settings& S, float* img, float* T_final, uint32_t* last, uint32_t* n_contrib,
                          cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  I4D_PROF("render_fwd", st);
  const float4* pr = reinterpret_cast<const float4*>(proj);
  if (n_contrib)
    render_fwd_kernel<TW, TH, true, B><<<tiles, TW * TH / 2, 0, st>>>(vt, n, pr, ids, ranges, S, img, T_final, last,
                                                                       n_contrib);
  else
    render_fwd_kernel<TW, TH, false, B><<<tiles, TW * TH / 2, 0, st>>>(vt, n, pr, ids, ranges, S, img, T_final,
                                                                        last, nullptr);
  return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_fwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, int batch, float* img, float* T_final, uint32_t* last,
                         uint32_t* n_contrib, cudaStream_t st) {
  if (batch == 16) return launch_fwd_tb<TW, TH, 16>(vt, n, proj, ids, ranges, S, img, T_final, last, n_contrib, st);
  if (batch == 64) return launch_fwd_tb<TW, TH, 64>(vt, n, proj, ids, ranges, S, img, T_final, last, n_contrib, st);
  return launch_fwd_tb<TW, TH, 32>(vt, n, proj, ids, ranges, S, img, T_final, last, n_contrib, st);
}

template <int TW, int TH>
cudaError_t launch_bwd_t(const ViewTable& vt, int n, const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         const Settings& S, const float* T_final, const uint32_t* last, const float* dL_dimg,
                         float* grad2d, cudaStream_t st) {
  const int tiles = vt.tile_off[vt.n_views];
  constexpr size_t smem = bwd_smem_bytes<TW, TH>();
  cudaError_t e = cudaFuncSetAttribute(render_bwd_kernel<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  I4D_PROF("render_bwd", st);
  render_bwd_kernel<TW, TH><<<tiles, TW * TH / 2, smem, st>>>(vt, n, reinterpret_cast<const float4*>(proj), ids,
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
  if (vt.tile_off[vt.n_views] == 0) return cudaSuccess;
  I4D_TILE_DISPATCH(launch_fwd_t, vt, n, proj, ids, ranges, S, batch, img, T_final, last, n_contrib, st);
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
