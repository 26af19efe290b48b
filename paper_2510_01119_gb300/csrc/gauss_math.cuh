// Per-Gaussian float32 math of slicing (Eq. 7-8), temporal opacity (Eq. 9), EWA projection and
// SH colour, and its reverse mode.  Used by the slice/project kernel and by the backward chain.
#pragma once

#include "i4d_common.cuh"

namespace i4d {

// ---- real SH of degree 1..3 (textbook real form without the Condon-Shortley phase) --------------
// Y index k = l*l + l + m - 1.  Constants: sqrt(3/4pi), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4,
// sqrt(35/2pi)/4, sqrt(105/pi)/2, sqrt(21/2pi)/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f;
constexpr float kSH20 = 0.31539156525252005f;
constexpr float kSH22 = 0.5462742152960396f;
constexpr float kSH33 = 0.5900435899266435f;
constexpr float kSH32 = 2.890611442640554f;
constexpr float kSH31 = 0.4570457994644658f;
constexpr float kSH30 = 0.3731763325901154f;
constexpr float kSH322 = 1.445305721320277f;

template <int DEG>
I4D_D void sh_basis(float x, float y, float z, float* Y) {
  if (DEG >= 1) {
    Y[0] = kSH1 * y;
    Y[1] = kSH1 * z;
    Y[2] = kSH1 * x;
  }
  if (DEG >= 2) {
    Y[3] = kSH2a * x * y;
    Y[4] = kSH2a * y * z;
    Y[5] = kSH20 * (3.0f * z * z - 1.0f);
    Y[6] = kSH2a * x * z;
    Y[7] = kSH22 * (x * x - y * y);
  }
  if (DEG >= 3) {
    Y[8] = kSH33 * y * (3.0f * x * x - y * y);
    Y[9] = kSH32 * x * y * z;
    Y[10] = kSH31 * y * (5.0f * z * z - 1.0f);
    Y[11] = kSH30 * z * (5.0f * z * z - 3.0f);
    Y[12] = kSH31 * x * (5.0f * z * z - 1.0f);
    Y[13] = kSH322 * z * (x * x - y * y);
    Y[14] = kSH33 * x * (x * x - 3.0f * y * y);
  }
}

// gradient of sum_k w_k Y_k(x, y, z) with respect to (x, y, z) (polynomial extension)
template <int DEG>
I4D_D void sh_basis_grad(float x, float y, float z, const float* w, float& gx, float& gy, float& gz) {
  gx = gy = gz = 0.0f;
  if (DEG >= 1) {
    gy += kSH1 * w[0];
    gz += kSH1 * w[1];
    gx += kSH1 * w[2];
  }
  if (DEG >= 2) {
    gx += kSH2a * y * w[3];
    gy += kSH2a * x * w[3];
    gy += kSH2a * z * w[4];
    gz += kSH2a * y * w[4];
    gz += kSH20 * 6.0f * z * w[5];
    gx += kSH2a * z * w[6];
    gz += kSH2a * x * w[6];
    gx += 2.0f * kSH22 * x * w[7];
    gy += -2.0f * kSH22 * y * w[7];
  }
  if (DEG >= 3) {
    gx += kSH33 * 6.0f * x * y * w[8];
    gy += kSH33 * 3.0f * (x * x - y * y) * w[8];
    gx += kSH32 * y * z * w[9];
    gy += kSH32 * x * z * w[9];
    gz += kSH32 * x * y * w[9];
    gy += kSH31 * (5.0f * z * z - 1.0f) * w[10];
    gz += kSH31 * 10.0f * y * z * w[10];
    gz += kSH30 * (15.0f * z * z - 3.0f) * w[11];
    gx += kSH31 * (5.0f * z * z - 1.0f) * w[12];
    gz += kSH31 * 10.0f * x * z * w[12];
    gx += kSH322 * 2.0f * x * z * w[13];
    gy += -kSH322 * 2.0f * y * z * w[13];
    gz += kSH322 * (x * x - y * y) * w[13];
    gx += kSH33 * 3.0f * (x * x - y * y) * w[14];
    gy += -kSH33 * 6.0f * x * y * w[14];
  }
}

// ---- view-independent state of one Gaussian --------------------------------------------------------
struct GaussState {
  float mu[4];
  float s[4];           // scales after the isotropic tying
  float ql[4], qr[4];   // normalised quaternions
  float nl, nr;         // their norms before normalisation
  float R[4][4];        // R = L(q_l) Rr(q_r)
  float A[6];           // Sigma_{1:3,1:3} as xx xy xz yy yz zz
  float b[3];           // Sigma_{1:3,4}
  float c;              // Sigma_44
  float sig;            // sigmoid(opacity logit)
  float base[3];        // base colour
};

// Left multiplication by p = (a, b, c, d) on 4-vectors (x, y, z, t) <-> t + xi + yj + zk:
//   [[a,-d, c, b], [d, a,-b, c], [-c, b, a, d], [-b,-c,-d, a]]
// Right multiplication by q = (e, f, g, h):
//   [[e, h,-g, f], [-h, e, f, g], [g,-f, e, h], [-f,-g,-h, e]]
I4D_D void left_mat(const float* p, float L[4][4]) {
  const float a = p[0], b = p[1], c = p[2], d = p[3];
  L[0][0] = a;  L[0][1] = -d; L[0][2] = c;  L[0][3] = b;
  L[1][0] = d;  L[1][1] = a;  L[1][2] = -b; L[1][3] = c;
  L[2][0] = -c; L[2][1] = b;  L[2][2] = a;  L[2][3] = d;
  L[3][0] = -b; L[3][1] = -c; L[3][2] = -d; L[3][3] = a;
}
I4D_D void right_mat(const float* q, float M[4][4]) {
  const float e = q[0], f = q[1], g = q[2], h = q[3];
  M[0][0] = e;  M[0][1] = h;  M[0][2] = -g; M[0][3] = f;
  M[1][0] = -h; M[1][1] = e;  M[1][2] = f;  M[1][3] = g;
  M[2][0] = g;  M[2][1] = -f; M[2][2] = e;  M[2][3] = h;
  M[3][0] = -f; M[3][1] = -g; M[3][2] = -h; M[3][3] = e;
}

I4D_D void gauss_setup(const float4 m4, const float4 ls, const float4 ql, const float4 qr, const float4 orgb, int mode,
                       GaussState& G) {
  G.mu[0] = m4.x; G.mu[1] = m4.y; G.mu[2] = m4.z; G.mu[3] = m4.w;
  if (mode == I4D_MODE_FULL) {
    G.s[0] = expf(ls.x); G.s[1] = expf(ls.y); G.s[2] = expf(ls.z);
  } else {
    G.s[0] = G.s[1] = G.s[2] = expf(ls.x);
  }
  G.s[3] = expf(ls.w);
  if (mode == I4D_MODE_ISO_IDENTITY) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) G.R[i][j] = (i == j) ? 1.0f : 0.0f;
      G.ql[i] = G.qr[i] = (i == 0) ? 1.0f : 0.0f;
    }
    G.nl = G.nr = 1.0f;
  } else {
    G.nl = sqrtf(ql.x * ql.x + ql.y * ql.y + ql.z * ql.z + ql.w * ql.w);
    G.nr = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float il = 1.0f / G.nl, ir = 1.0f / G.nr;
    G.ql[0] = ql.x * il; G.ql[1] = ql.y * il; G.ql[2] = ql.z * il; G.ql[3] = ql.w * il;
    G.qr[0] = qr.x * ir; G.qr[1] = qr.y * ir; G.qr[2] = qr.z * ir; G.qr[3] = qr.w * ir;
    float L[4][4], M[4][4];
    left_mat(G.ql, L);
    right_mat(G.qr, M);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += L[i][k] * M[k][j];
        G.R[i][j] = acc;
      }
  }
  // Sigma = (R S)(R S)^T
  float RS[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) RS[i][k] = G.R[i][k] * G.s[k];
  auto dot4 = [&](int i, int j) {
    return RS[i][0] * RS[j][0] + RS[i][1] * RS[j][1] + RS[i][2] * RS[j][2] + RS[i][3] * RS[j][3];
  };
  G.A[0] = dot4(0, 0); G.A[1] = dot4(0, 1); G.A[2] = dot4(0, 2);
  G.A[3] = dot4(1, 1); G.A[4] = dot4(1, 2); G.A[5] = dot4(2, 2);
  G.b[0] = dot4(0, 3); G.b[1] = dot4(1, 3); G.b[2] = dot4(2, 3);
  G.c = dot4(3, 3);
  G.sig = 1.0f / (1.0f + expf(-orgb.x));
  G.base[0] = orgb.y; G.base[1] = orgb.z; G.base[2] = orgb.w;
}

// ---- per-view forward -------------------------------------------------------------------------------
struct ViewFwd {
  float dt, k;          // t - mu_t, dt / c
  float mean3[3];
  float cov3[6];
  float ot;
  float m[3];
  float rx, ry;
  bool clx, cly;
  float J00, J02, J11, J12;
  float Mc[6];          // W cov3 W^T
  float cov2[3];        // incl. dilation: xx, xy, yy
  float det;
  float conic[3];
  float radius, u, v;
  float dhat[3], dirn;
  float raw[3];
  bool visible;
};

// sym3 index helper: (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5
I4D_HD int s3(int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// Coefficient c of the SCH variant's term m (1..nt-1), harmonic k (0 = the constant, 1.. = the SH
// basis of degree >= 1), channel ch: float (m - 1)((DEG + 1)^2) 3 + 3 k + ch of the Gaussian's SCH
// block, which follows its SH planes (plane = float / 4, lane = float % 4).
template <int DEG>
I4D_D int sch_index(int m, int k, int ch) {
  return ((m - 1) * (DEG + 1) * (DEG + 1) + k) * 3 + ch;
}

template <int DEG>
I4D_D void view_forward(const GaussState& G, const float4* __restrict__ sh, int n, int gi, const Cam& C,
                        const float* campos, float tanx, float tany, const Settings& S, ViewFwd& F, int nt = 0) {
  F.dt = C.time - G.mu[3];
  const float inv_c = 1.0f / G.c;
  F.k = F.dt * inv_c;
#pragma unroll
  for (int a = 0; a < 3; ++a) F.mean3[a] = G.mu[a] + G.b[a] * F.k;
  F.cov3[0] = G.A[0] - G.b[0] * G.b[0] * inv_c;
  F.cov3[1] = G.A[1] - G.b[0] * G.b[1] * inv_c;
  F.cov3[2] = G.A[2] - G.b[0] * G.b[2] * inv_c;
  F.cov3[3] = G.A[3] - G.b[1] * G.b[1] * inv_c;
  F.cov3[4] = G.A[4] - G.b[1] * G.b[2] * inv_c;
  F.cov3[5] = G.A[5] - G.b[2] * G.b[2] * inv_c;
  F.ot = G.sig * expf(-0.5f * F.dt * F.dt * inv_c);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    F.m[a] = C.R[3 * a] * F.mean3[0] + C.R[3 * a + 1] * F.mean3[1] + C.R[3 * a + 2] * F.mean3[2] + C.t[a];
  F.visible = (F.ot >= S.ot_min) && (F.m[2] > S.z_near);
  F.u = F.v = F.radius = 0.0f;
  F.conic[0] = F.conic[1] = F.conic[2] = 0.0f;
  if (F.visible) {
    const float mz = F.m[2], imz = 1.0f / mz;
    F.u = C.fx * F.m[0] * imz + C.cx;
    F.v = C.fy * F.m[1] * imz + C.cy;
    // tanx = W / (2 fx), tany = H / (2 fy): half-FOV tangents of the view
    const float limx = S.fov_clamp * tanx, limy = S.fov_clamp * tany;
    const float rx = F.m[0] * imz, ry = F.m[1] * imz;
    F.clx = (rx < -limx) || (rx > limx);
    F.cly = (ry < -limy) || (ry > limy);
    F.rx = fminf(fmaxf(rx, -limx), limx);
    F.ry = fminf(fmaxf(ry, -limy), limy);
    F.J00 = C.fx * imz;
    F.J02 = -C.fx * F.rx * imz;
    F.J11 = C.fy * imz;
    F.J12 = -C.fy * F.ry * imz;
    // Mc = W cov3 W^T
    float T[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2)
        T[a][b2] = C.R[3 * a] * F.cov3[s3(0, b2)] + C.R[3 * a + 1] * F.cov3[s3(1, b2)] +
                   C.R[3 * a + 2] * F.cov3[s3(2, b2)];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b2 = a; b2 < 3; ++b2)
        F.Mc[s3(a, b2)] = T[a][0] * C.R[3 * b2] + T[a][1] * C.R[3 * b2 + 1] + T[a][2] * C.R[3 * b2 + 2];
    // cov2 = J Mc J^T + dilation
    const float* M = F.Mc;
    const float jm00 = F.J00 * M[0] + F.J02 * M[2], jm01 = F.J00 * M[1] + F.J02 * M[4],
                jm02 = F.J00 * M[2] + F.J02 * M[5];
    const float jm11 = F.J11 * M[3] + F.J12 * M[4], jm12 = F.J11 * M[4] + F.J12 * M[5];
    F.cov2[0] = jm00 * F.J00 + jm02 * F.J02 + S.dilation;
    F.cov2[1] = jm01 * F.J11 + jm02 * F.J12;
    F.cov2[2] = jm11 * F.J11 + jm12 * F.J12 + S.dilation;
    F.det = F.cov2[0] * F.cov2[2] - F.cov2[1] * F.cov2[1];
    if (F.det > 0.0f) {
      const float idet = 1.0f / F.det;
      F.conic[0] = F.cov2[2] * idet;
      F.conic[1] = -F.cov2[1] * idet;
      F.conic[2] = F.cov2[0] * idet;
      const float mid = 0.5f * (F.cov2[0] + F.cov2[2]);
      const float lam = mid + sqrtf(fmaxf(mid * mid - F.det, 0.0f));
      F.radius = ceilf(3.0f * sqrtf(lam));
    } else {
      F.visible = false;
    }
  }
  // colour: base + sum_k Y_k(dir) c_k, clamped at 0
  const float dx = F.mean3[0] - campos[0], dy = F.mean3[1] - campos[1], dz = F.mean3[2] - campos[2];
  F.dirn = sqrtf(dx * dx + dy * dy + dz * dz);
  const float idn = 1.0f / F.dirn;
  F.dhat[0] = dx * idn; F.dhat[1] = dy * idn; F.dhat[2] = dz * idn;
  F.raw[0] = G.base[0]; F.raw[1] = G.base[1]; F.raw[2] = G.base[2];
  if constexpr (DEG > 0) {
    float Y[15];
    sh_basis<DEG>(F.dhat[0], F.dhat[1], F.dhat[2], Y);
    constexpr int K = (DEG + 1) * (DEG + 1) - 1;
    constexpr int NP = DEG == 1 ? 3 : (DEG == 2 ? 6 : 12);
    float c[NP * 4];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float4 q = __ldg(&sh[(size_t)p * n + gi]);
      c[4 * p] = q.x; c[4 * p + 1] = q.y; c[4 * p + 2] = q.z; c[4 * p + 3] = q.w;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      F.raw[0] += Y[k] * c[3 * k];
      F.raw[1] += Y[k] * c[3 * k + 1];
      F.raw[2] += Y[k] * c[3 * k + 2];
    }
  }
  if (nt > 1) {
    // SCH variant (Sec. 3.1): + sum_m cos(2 pi m t) (c_m0 + sum_k Y_k c_mk), t the view's frame time
    float Y1[16];
    Y1[0] = 1.0f;
    if constexpr (DEG > 0) sh_basis<DEG>(F.dhat[0], F.dhat[1], F.dhat[2], Y1 + 1);
    const float* sch = reinterpret_cast<const float*>(sh + (size_t)sh_planes(DEG) * n);
    for (int m = 1; m < nt; ++m) {
      const float cs = cospif(2.0f * (float)m * C.time);
#pragma unroll
      for (int k = 0; k < (DEG + 1) * (DEG + 1); ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const int idx = sch_index<DEG>(m, k, ch);
          F.raw[ch] += cs * Y1[k] * __ldg(&sch[((size_t)(idx >> 2) * n + gi) * 4 + (idx & 3)]);
        }
    }
  }
}

// ---- per-view reverse mode -----------------------------------------------------------------------------
struct ParamGrad {
  float mu[4], ls[4], ql[4], qr[4], orgb[4];
};

// Accumulate into P (and gsh: float [3*K] for SH) the gradients of one view.
// g = (du, dv, dca, dcb, dcc, dot, dr, dg, db).
template <int DEG>
I4D_D void view_backward(const GaussState& G, const ViewFwd& F, const float4* __restrict__ sh, int n, int gi,
                         const Cam& C, const float* g, ParamGrad& P, float* gsh, float* gA_acc,
                         float& gc_acc, float* gb_acc, int nt = 0, float4* gsch = nullptr) {
  const float fx = C.fx, fy = C.fy;
  const float mz = F.m[2], imz = 1.0f / mz, imz2 = imz * imz;
  float gm[3] = {0.0f, 0.0f, 0.0f};
  // uv
  gm[0] += g[0] * fx * imz;
  gm[2] -= g[0] * fx * F.m[0] * imz2;
  gm[1] += g[1] * fy * imz;
  gm[2] -= g[1] * fy * F.m[1] * imz2;
  // conic = cov2^{-1}: G2 = -Q GQ Q
  const float qa = F.conic[0], qb = F.conic[1], qc = F.conic[2];
  const float ga = g[2], gb = 0.5f * g[3], gcc = g[4];
  // X = Q GQ
  const float x00 = qa * ga + qb * gb, x01 = qa * gb + qb * gcc;
  const float x10 = qb * ga + qc * gb, x11 = qb * gb + qc * gcc;
  const float G00 = -(x00 * qa + x01 * qb), G01 = -(x00 * qb + x01 * qc), G11 = -(x10 * qb + x11 * qc);
  // H = G2 J (2x3), J rows (J00, 0, J02), (0, J11, J12)
  const float H00 = G00 * F.J00, H01 = G01 * F.J11, H02 = G00 * F.J02 + G01 * F.J12;
  const float H10 = G01 * F.J00, H11 = G00 * 0.0f + G11 * F.J11, H12 = G01 * F.J02 + G11 * F.J12;
  // G_M = J^T H (sym): G_M_ij = J0_i H0_j + J1_i H1_j with J0 = (J00, 0, J02), J1 = (0, J11, J12)
  float GM[6];
  GM[0] = F.J00 * H00;
  GM[1] = F.J00 * H01;
  GM[2] = F.J00 * H02;
  GM[3] = F.J11 * H11;
  GM[4] = F.J11 * H12;
  GM[5] = F.J02 * H02 + F.J12 * H12;
  // G_J = 2 H Mc
  const float* M = F.Mc;
  const float GJ00 = 2.0f * (H00 * M[0] + H01 * M[1] + H02 * M[2]);
  const float GJ02 = 2.0f * (H00 * M[2] + H01 * M[4] + H02 * M[5]);
  const float GJ11 = 2.0f * (H10 * M[1] + H11 * M[3] + H12 * M[4]);
  const float GJ12 = 2.0f * (H10 * M[2] + H11 * M[4] + H12 * M[5]);
  gm[2] -= GJ00 * fx * imz2;
  gm[2] -= GJ11 * fy * imz2;
  if (!F.clx) {
    gm[0] -= GJ02 * fx * imz2;
    gm[2] += GJ02 * 2.0f * fx * F.m[0] * imz2 * imz;
  } else {
    gm[2] += GJ02 * fx * F.rx * imz2;
  }
  if (!F.cly) {
    gm[1] -= GJ12 * fy * imz2;
    gm[2] += GJ12 * 2.0f * fy * F.m[1] * imz2 * imz;
  } else {
    gm[2] += GJ12 * fy * F.ry * imz2;
  }
  // mean3 from m = W mean3 + t
  float gmean3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gmean3[a] = C.R[a] * gm[0] + C.R[3 + a] * gm[1] + C.R[6 + a] * gm[2];
  // G_cov3 = W^T G_M W
  float T2[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 3; ++b2)
      T2[a][b2] = C.R[a] * GM[s3(0, b2)] + C.R[3 + a] * GM[s3(1, b2)] + C.R[6 + a] * GM[s3(2, b2)];
  float G3[6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b2 = a; b2 < 3; ++b2) G3[s3(a, b2)] = T2[a][0] * C.R[b2] + T2[a][1] * C.R[3 + b2] + T2[a][2] * C.R[6 + b2];

  // colour
  {
    const float gr[3] = {g[6], g[7], g[8]};
    float graw[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) graw[ch] = (F.raw[ch] < 0.0f) ? 0.0f : gr[ch];
    P.orgb[1] += graw[0];
    P.orgb[2] += graw[1];
    P.orgb[3] += graw[2];
    if constexpr (DEG > 0) {
      constexpr int K = (DEG + 1) * (DEG + 1) - 1;
      constexpr int NP = DEG == 1 ? 3 : (DEG == 2 ? 6 : 12);
      float c[NP * 4];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float4 q = __ldg(&sh[(size_t)p * n + gi]);
        c[4 * p] = q.x; c[4 * p + 1] = q.y; c[4 * p + 2] = q.z; c[4 * p + 3] = q.w;
      }
      float Y[15], w[15];
      sh_basis<DEG>(F.dhat[0], F.dhat[1], F.dhat[2], Y);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        gsh[3 * k] += Y[k] * graw[0];
        gsh[3 * k + 1] += Y[k] * graw[1];
        gsh[3 * k + 2] += Y[k] * graw[2];
        w[k] = c[3 * k] * graw[0] + c[3 * k + 1] * graw[1] + c[3 * k + 2] * graw[2];
      }
      if (nt > 1) {  // the SCH terms' harmonics also depend on the view direction
        const float* sch = reinterpret_cast<const float*>(sh + (size_t)NP * n);
        for (int m = 1; m < nt; ++m) {
          const float cs = cospif(2.0f * (float)m * C.time);
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
              const int idx = sch_index<DEG>(m, k + 1, ch);
              w[k] += cs * __ldg(&sch[((size_t)(idx >> 2) * n + gi) * 4 + (idx & 3)]) * graw[ch];
            }
        }
      }
      float gx, gy, gz;
      sh_basis_grad<DEG>(F.dhat[0], F.dhat[1], F.dhat[2], w, gx, gy, gz);
      const float dd = F.dhat[0] * gx + F.dhat[1] * gy + F.dhat[2] * gz;
      const float idn = 1.0f / F.dirn;
      gmean3[0] += (gx - F.dhat[0] * dd) * idn;
      gmean3[1] += (gy - F.dhat[1] * dd) * idn;
      gmean3[2] += (gz - F.dhat[2] * dd) * idn;
    }
    if (nt > 1) {  // SCH coefficients: d raw / d c_mk = cos(2 pi m t) Y_k, summed over views in place
      float Y1[16];
      Y1[0] = 1.0f;
      if constexpr (DEG > 0) sh_basis<DEG>(F.dhat[0], F.dhat[1], F.dhat[2], Y1 + 1);
      float* gs = reinterpret_cast<float*>(gsch);
      for (int m = 1; m < nt; ++m) {
        const float cs = cospif(2.0f * (float)m * C.time);
#pragma unroll
        for (int k = 0; k < (DEG + 1) * (DEG + 1); ++k)
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            const int idx = sch_index<DEG>(m, k, ch);
            gs[((size_t)(idx >> 2) * n + gi) * 4 + (idx & 3)] += cs * Y1[k] * graw[ch];
          }
      }
    }
  }

  // temporal opacity
  const float inv_c = 1.0f / G.c;
  const float got = g[5];
  P.orgb[0] += got * F.ot * (1.0f - G.sig);
  float gc = got * F.ot * 0.5f * F.dt * F.dt * inv_c * inv_c;
  float gmut = got * F.ot * F.dt * inv_c;
  // Eq. 7: mean3 = mu + b dt / c
  const float bg3 = G.b[0] * gmean3[0] + G.b[1] * gmean3[1] + G.b[2] * gmean3[2];
  P.mu[0] += gmean3[0];
  P.mu[1] += gmean3[1];
  P.mu[2] += gmean3[2];
  gmut -= bg3 * inv_c;
  gc -= F.dt * bg3 * inv_c * inv_c;
  float gbv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gbv[a] = gmean3[a] * F.k;
  // Eq. 8: cov3 = A - b b^T / c
  float G3b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) G3b[a] = G3[s3(a, 0)] * G.b[0] + G3[s3(a, 1)] * G.b[1] + G3[s3(a, 2)] * G.b[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) gbv[a] -= 2.0f * G3b[a] * inv_c;
  gc += (G.b[0] * G3b[0] + G.b[1] * G3b[1] + G.b[2] * G3b[2]) * inv_c * inv_c;
  P.mu[3] += gmut;
  // accumulate the symmetric Sigma gradient across views (chained to R and s once, after the loop)
#pragma unroll
  for (int a = 0; a < 6; ++a) gA_acc[a] += G3[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) gb_acc[a] += gbv[a];
  gc_acc += gc;
}

// Chain the accumulated Sigma gradient (G_A sym 6, g_b 3, g_c) to scales and quaternions.
I4D_D void sigma_backward(const GaussState& G, int mode, const float* GA, const float* gbv, float gc, ParamGrad& P) {
  float GS[4][4];
  GS[0][0] = GA[0]; GS[0][1] = GS[1][0] = GA[1]; GS[0][2] = GS[2][0] = GA[2];
  GS[1][1] = GA[3]; GS[1][2] = GS[2][1] = GA[4]; GS[2][2] = GA[5];
  GS[0][3] = GS[3][0] = 0.5f * gbv[0];
  GS[1][3] = GS[3][1] = 0.5f * gbv[1];
  GS[2][3] = GS[3][2] = 0.5f * gbv[2];
  GS[3][3] = gc;
  // GSR = GS R
  float GSR[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) GSR[a][k] = GS[a][0] * G.R[0][k] + GS[a][1] * G.R[1][k] + GS[a][2] * G.R[2][k] + GS[a][3] * G.R[3][k];
  // G_D_k = (R^T GS R)_kk
  float GD[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) GD[k] = G.R[0][k] * GSR[0][k] + G.R[1][k] * GSR[1][k] + G.R[2][k] * GSR[2][k] + G.R[3][k] * GSR[3][k];
  if (mode == I4D_MODE_FULL) {
#pragma unroll
    for (int k = 0; k < 4; ++k) P.ls[k] += GD[k] * 2.0f * G.s[k] * G.s[k];
  } else {
    P.ls[0] += (GD[0] + GD[1] + GD[2]) * 2.0f * G.s[0] * G.s[0];
    P.ls[3] += GD[3] * 2.0f * G.s[3] * G.s[3];
  }
  if (mode == I4D_MODE_ISO_IDENTITY) return;
  // G_R = 2 GS R D
  float GR[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) GR[a][k] = 2.0f * GSR[a][k] * G.s[k] * G.s[k];
  // R = L Mr: dL/dL = GR Mr^T, dL/dMr = L^T GR
  float L[4][4], Mr[4][4];
  left_mat(G.ql, L);
  right_mat(G.qr, Mr);
  float GL[4][4], GMr[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) {
      GL[a][b2] = GR[a][0] * Mr[b2][0] + GR[a][1] * Mr[b2][1] + GR[a][2] * Mr[b2][2] + GR[a][3] * Mr[b2][3];
      GMr[a][b2] = L[0][a] * GR[0][b2] + L[1][a] * GR[1][b2] + L[2][a] * GR[2][b2] + L[3][a] * GR[3][b2];
    }
  // pattern of L(p): a on the diagonal; b at (0,3)+ (1,2)- (2,1)+ (3,0)-; c at (0,2)+ (1,3)+ (2,0)- (3,1)-;
  // d at (0,1)- (1,0)+ (2,3)+ (3,2)-
  float gl[4];
  gl[0] = GL[0][0] + GL[1][1] + GL[2][2] + GL[3][3];
  gl[1] = GL[0][3] - GL[1][2] + GL[2][1] - GL[3][0];
  gl[2] = GL[0][2] + GL[1][3] - GL[2][0] - GL[3][1];
  gl[3] = -GL[0][1] + GL[1][0] + GL[2][3] - GL[3][2];
  // pattern of Rr(q): e on the diagonal; f at (0,3)+ (1,2)+ (2,1)- (3,0)-; g at (0,2)- (1,3)+ (2,0)+ (3,1)-;
  // h at (0,1)+ (1,0)- (2,3)+ (3,2)-
  float gr[4];
  gr[0] = GMr[0][0] + GMr[1][1] + GMr[2][2] + GMr[3][3];
  gr[1] = GMr[0][3] + GMr[1][2] - GMr[2][1] - GMr[3][0];
  gr[2] = -GMr[0][2] + GMr[1][3] + GMr[2][0] - GMr[3][1];
  gr[3] = GMr[0][1] - GMr[1][0] + GMr[2][3] - GMr[3][2];
  const float dl = gl[0] * G.ql[0] + gl[1] * G.ql[1] + gl[2] * G.ql[2] + gl[3] * G.ql[3];
  const float dr = gr[0] * G.qr[0] + gr[1] * G.qr[1] + gr[2] * G.qr[2] + gr[3] * G.qr[3];
  const float il = 1.0f / G.nl, ir = 1.0f / G.nr;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    P.ql[j] += (gl[j] - G.ql[j] * dl) * il;
    P.qr[j] += (gr[j] - G.qr[j] * dr) * ir;
  }
}

}  // namespace i4d
