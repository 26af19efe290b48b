// Shared device-side definitions of the sm_103a kernels (no host-visible ABI here; see i4d.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/i4d.h"

#define I4D_HD __host__ __device__ __forceinline__
#define I4D_D __device__ __forceinline__

namespace i4d {

constexpr int kMaxViews = I4D_MAX_VIEWS;

// Per-launch table of the batch of views, passed by value as a kernel parameter.
struct ViewTable {
  int n_views;
  int tile_w, tile_h;
  int width[kMaxViews], height[kMaxViews];
  int tiles_x[kMaxViews], tiles_y[kMaxViews];
  int tile_off[kMaxViews + 1];   // cumulative tiles over views
  int64_t pix_off[kMaxViews + 1];  // cumulative pixels over views
};

struct Settings {
  float alpha_max, alpha_min, T_min, q_max, ot_min, z_near, dilation, fov_clamp;
  float bg[3];
};

// Camera as loaded into registers / shared memory
struct Cam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float time;
  float pad[3];
};
static_assert(sizeof(Cam) == sizeof(i4d_camera), "camera layout");

I4D_HD int sh_planes(int deg) { return deg == 0 ? 0 : (deg == 1 ? 3 : (deg == 2 ? 6 : 12)); }
I4D_HD int sh_coeffs(int deg) { return (deg + 1) * (deg + 1) - 1; }
// SCH variant: (nt - 1) temporal terms x (deg + 1)^2 harmonics x 3 channels, in planes of 4 floats
I4D_HD int sch_floats(int deg, int nt) { return nt > 1 ? (nt - 1) * (deg + 1) * (deg + 1) * 3 : 0; }
I4D_HD int sch_planes(int deg, int nt) { return (sch_floats(deg, nt) + 3) / 4; }

// Which view owns a global tile index (linear scan: at most 64 views, uniform across a block).
I4D_D int view_of_tile(const ViewTable& vt, int tile) {
  int v = 0;
  while (v + 1 < vt.n_views && tile >= vt.tile_off[v + 1]) ++v;
  return v;
}

// Tile rectangle [x0, x1) x [y0, y1) of the square of half-width `radius` around (u, v).
// The same function is used when counting and when emitting, so both agree bit for bit.
I4D_D void box_rect(float4 b, int W, int H, int tile_w, int tile_h, int tiles_x, int tiles_y, int& x0, int& y0,
                    int& x1, int& y1) {
  // tiles [x0,x1) x [y0,y1) holding the pixels of the W x H view whose centres (p + 0.5) lie in the
  // box: the box is first clipped to the view's pixel centres [0.5, W - 0.5] x [0.5, H - 0.5], so a
  // box beyond the view's edge gets no tile even where the edge tiles reach past it
  const float bx0 = fmaxf(b.x, 0.5f), bx1 = fminf(b.y, (float)W - 0.5f);
  const float by0 = fmaxf(b.z, 0.5f), by1 = fminf(b.w, (float)H - 0.5f);
  if (!(bx0 <= bx1 && by0 <= by1)) {
    x0 = x1 = y0 = y1 = 0;
    return;
  }
  const float fx0 = floorf((bx0 + 0.5f) / (float)tile_w);
  const float fx1 = floorf((bx1 - 0.5f) / (float)tile_w) + 1.0f;
  const float fy0 = floorf((by0 + 0.5f) / (float)tile_h);
  const float fy1 = floorf((by1 - 0.5f) / (float)tile_h) + 1.0f;
  x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)tiles_x);
  x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)tiles_x);
  y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)tiles_y);
  y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)tiles_y);
  x1 = max(x1, x0);
  y1 = max(y1, y0);
}

// Largest q at which a fragment of temporal opacity ot can be blended: coverage ends at q_max, and
// alpha = ot exp(-q/2) reaches alpha_min only while q <= 2 ln(ot / alpha_min).  The 1e-3 slack
// covers the rounding of the fast exponential and of the product in eval_pair (relative errors of a
// few 1e-7), so every fragment that eval_pair keeps lies inside the resulting ellipse.
I4D_D float blend_q(float ot, const Settings& s) {
  const float qa = 2.0f * logf(ot / s.alpha_min);
  return fminf(s.q_max, fmaxf(qa, 0.0f) + 1e-3f);
}

// G = exp(-q/2) = 2^(kFalloff q): the compositing kernels stage each conic multiplied by kFalloff so
// that a fragment's exponent comes straight out of the quadratic form.
constexpr float kFalloff = -0.72134752044448170368f;  // -log2(e) / 2
constexpr float kFalloffInv = -1.38629436111989061883f;  // 1 / kFalloff = -2 ln 2

I4D_D float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / x by the hardware's approximate reciprocal (one instruction; relative error below 2^-22)
I4D_D float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One Gaussian evaluated at a thread's two pixels (same column, offsets dx and dy.x / dy.y from the
// projected mean), given its conic pre-scaled by kFalloff (sa = kFalloff ca, sb2 = 2 kFalloff cb,
// sc = kFalloff cc): the exponent m = kFalloff q = sa dx^2 + sb2 dx dy + sc dy^2, the falloff
// G = 2^m = exp(-q/2), the raw alpha o_t G and the clamped alpha.  A fragment is kept where
// q <= q_max and o_t exp(-q/2) >= alpha_min, i.e. where m >= m_thr = kFalloff min(q_max, 2 ln(o_t / alpha_min)),
// a per-Gaussian threshold computed once when the entry is staged (one compare per pixel; the forms
// differ only by rounding, well inside the 1e-4 relative margin the parity protocol gives threshold
// decisions).  The pixel pair runs on the packed FP32x2 instructions of sm_100 and later
// (__fmul2_rn / __ffma2_rn round each lane exactly as __fmul_rn / __fmaf_rn).  The forward and the
// backward compositing kernels call exactly this code on the same staged values, so they take the
// same decisions.
struct FragPair {
  float2 G, a_raw, alpha;
  bool k0, k1;
};

I4D_D void eval_pair(float dx, float2 dy, float sa, float sb2, float sc, float ot, float m_thr, const Settings& s,
                     FragPair& f) {
  const float t0 = __fmul_rn(sa, __fmul_rn(dx, dx));
  const float2 dxdy = __fmul2_rn(make_float2(dx, dx), dy);
  const float2 dydy = __fmul2_rn(dy, dy);
  const float2 m = __ffma2_rn(make_float2(sc, sc), dydy, __ffma2_rn(make_float2(sb2, sb2), dxdy, make_float2(t0, t0)));
  f.G = make_float2(ex2_approx(m.x), ex2_approx(m.y));
  f.a_raw = __fmul2_rn(make_float2(ot, ot), f.G);
  f.alpha = make_float2(fminf(s.alpha_max, f.a_raw.x), fminf(s.alpha_max, f.a_raw.y));
  f.k0 = m.x >= m_thr;
  f.k1 = m.y >= m_thr;
}

// Pixel-space box (xmin, xmax, ymin, ymax) of the ellipse q <= q_max of a conic, widened by
// 1% + 0.01 px so that float rounding can never exclude a pixel centre that the per-pixel test
// accepts (the half-widths are sqrt(q_max) times the square roots of the inverse conic's diagonal).
I4D_D float4 ellipse_box(float u, float v, float ca, float cb, float cc, float q_max) {
  // ca cc - cb^2 by Kahan's difference of products: accurate to a few ulp however thin the ellipse
  const float w = __fmul_rn(cb, cb);
  const float det = __fadd_rn(__fmaf_rn(ca, cc, -w), __fmaf_rn(-cb, cb, w));
  if (!(det > 0.0f)) return make_float4(-1e30f, 1e30f, -1e30f, 1e30f);
  const float hx = sqrtf(q_max * cc / det) * 1.01f + 0.01f;
  const float hy = sqrtf(q_max * ca / det) * 1.01f + 0.01f;
  return make_float4(u - hx, u + hx, v - hy, v + hy);
}

// device status / error word helpers
I4D_D void set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace i4d
