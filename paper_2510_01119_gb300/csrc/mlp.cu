// Learned initialisation: a 64 -> 64 -> 64 -> 12 MLP with GELU, bfloat16 operands and float32
// accumulation, mapping a pruned point's neighbourhood features to (log s_t, velocity, q_l, q_r).
//
// Forward (inference and training): one warp per 16 points; the three layers run on the tensor
// cores with mma.sync m16n8k16 (bf16 x bf16 -> f32); the accumulators of one layer, biased and
// passed through GELU, are rounded to bf16 and become the next layer's A fragments in registers.
// Training: the same forward per 64-point chunk, the loss and its gradient per point (log s_t and
// velocity squared errors, rotation compared as the 16 entries of R(q_l, q_r)), and the backward on
// the tensor cores too: bfloat16 operands (the gradient entering each product rounded once, the
// weights and activations as the forward used them), float32 accumulation; per-block partial
// weight gradients held in the mma accumulators across chunks, summed afterwards by a reduction
// kernel.
#include <cuda_bf16.h>

#include "gauss_math.cuh"
#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int kIn = 64, kH = 64, kOut = 12, kOutPad = 16;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH, kWeights = kOffB3 + kOut;
static_assert(kWeights == 9100, "weight layout");

struct MlpSmem {
  __nv_bfloat16 w1[kH][kIn];
  __nv_bfloat16 w2[kH][kH];
  __nv_bfloat16 w3[kOutPad][kH];
  float b1[kH], b2[kH], b3[kOutPad];
};

__device__ __forceinline__ float gelu(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad(float z) {
  return normcdff(z) + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void load_weights(MlpSmem& s, const float* __restrict__ w) {
  for (int k = threadIdx.x; k < kH * kIn; k += blockDim.x) {
    (&s.w1[0][0])[k] = __float2bfloat16_rn(w[kOffW1 + k]);
    (&s.w2[0][0])[k] = __float2bfloat16_rn(w[kOffW2 + k]);
  }
  for (int k = threadIdx.x; k < kOutPad * kH; k += blockDim.x)
    (&s.w3[0][0])[k] = __float2bfloat16_rn(k < kOut * kH ? w[kOffW3 + k] : 0.0f);
  for (int k = threadIdx.x; k < kH; k += blockDim.x) {
    s.b1[k] = w[kOffB1 + k];
    s.b2[k] = w[kOffB2 + k];
  }
  for (int k = threadIdx.x; k < kOutPad; k += blockDim.x) s.b3[k] = k < kOut ? w[kOffB3 + k] : 0.0f;
}

// One hidden layer for a warp's 16 rows: a_in (4 k-blocks of A fragments) -> z (8 n-tiles of C
// fragments, bias added) and a_out (A fragments of bf16(gelu(z))).
__device__ __forceinline__ void hidden_layer(const __nv_bfloat16 (*w)[kIn], const float* b, const uint32_t (*a_in)[4],
                                             float (*z)[4], uint32_t (*a_out)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&w[8 * j + g][16 * s + 2 * t]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&w[8 * j + g][16 * s + 8 + 2 * t]);
      mma16816(c, a_in[s], b0, b1);
    }
    const float bb0 = b[8 * j + 2 * t], bb1 = b[8 * j + 2 * t + 1];
    z[j][0] = c[0] + bb0;
    z[j][1] = c[1] + bb1;
    z[j][2] = c[2] + bb0;
    z[j][3] = c[3] + bb1;
    const uint32_t lo = pack_bf16(gelu(z[j][0]), gelu(z[j][1]));
    const uint32_t hi = pack_bf16(gelu(z[j][2]), gelu(z[j][3]));
    a_out[j >> 1][(j & 1) * 2 + 0] = lo;  // rows g, cols of n-tile j
    a_out[j >> 1][(j & 1) * 2 + 1] = hi;  // rows g + 8
  }
}

// Forward of 16 rows; x_row(r) gives the (already bf16-rounded or float) input row r.
struct WarpForward {
  float z1[8][4], z2[8][4], y[2][4];
  uint32_t a2[4][4], a3[4][4];
};

// A fragments of the input rows (k-blocks of 16 features) for a warp's 16 rows
template <class XLoad>
__device__ __forceinline__ void input_fragments(XLoad xl, uint32_t (*a1)[4], int g, int t) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a1[k][0] = pack_bf16(xl(g, 16 * k + 2 * t), xl(g, 16 * k + 2 * t + 1));
    a1[k][1] = pack_bf16(xl(g + 8, 16 * k + 2 * t), xl(g + 8, 16 * k + 2 * t + 1));
    a1[k][2] = pack_bf16(xl(g, 16 * k + 8 + 2 * t), xl(g, 16 * k + 9 + 2 * t));
    a1[k][3] = pack_bf16(xl(g + 8, 16 * k + 8 + 2 * t), xl(g + 8, 16 * k + 9 + 2 * t));
  }
}

// Output layer: y (2 n-tiles of C fragments) = bf16(h2) W3^T + b3
__device__ __forceinline__ void output_layer(const MlpSmem& s, const uint32_t (*a3)[4], float (*y)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&s.w3[8 * j + g][16 * k + 2 * t]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&s.w3[8 * j + g][16 * k + 8 + 2 * t]);
      mma16816(c, a3[k], b0, b1);
    }
    const float bb0 = s.b3[8 * j + 2 * t], bb1 = s.b3[8 * j + 2 * t + 1];
    y[j][0] = c[0] + bb0;
    y[j][1] = c[1] + bb1;
    y[j][2] = c[2] + bb0;
    y[j][3] = c[3] + bb1;
  }
}

template <class XLoad>
__device__ __forceinline__ void warp_forward(const MlpSmem& s, XLoad xl, WarpForward& F, int g, int t) {
  uint32_t a1[4][4];
  input_fragments(xl, a1, g, t);
  // the A-fragment register order is (row g | row g+8 | row g, +8 cols | row g+8, +8 cols); the
  // hidden layers write (lo, hi) of n-tile 2s into slots 0, 1 and of n-tile 2s+1 into 2, 3
  hidden_layer(s.w1, s.b1, a1, F.z1, F.a2, g, t);
  hidden_layer(s.w2, s.b2, F.a2, F.z2, F.a3, g, t);
  output_layer(s, F.a3, F.y, g, t);
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ feat, int64_t n,
                                                          const float* __restrict__ w, float* __restrict__ out) {
  __shared__ MlpSmem s;
  load_weights(s, w);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int64_t base = (int64_t)blockIdx.x * 64 + warp * 16; base < n; base += (int64_t)gridDim.x * 64) {
    auto xl = [&](int r, int c) -> float {
      const int64_t p = base + r;
      return p < n ? feat[p * kIn + c] : 0.0f;
    };
    WarpForward F;
    warp_forward(s, xl, F, g, t);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int col = 8 * j + 2 * t;
      const int64_t p0 = base + g, p1 = base + g + 8;
      if (col < kOut) {
        if (p0 < n) {
          out[p0 * kOut + col] = F.y[j][0];
          out[p0 * kOut + col + 1] = F.y[j][1];
        }
        if (p1 < n) {
          out[p1 * kOut + col] = F.y[j][2];
          out[p1 * kOut + col + 1] = F.y[j][3];
        }
      }
    }
  }
}

// ---- training ------------------------------------------------------------------------------------------
// Per block, chunks of 64 points; warp w owns points [16 w, 16 w + 16) of the chunk in the forward and
// in the gradient of the pre-activations, and rows [16 w, 16 w + 16) of dW1 and dW2 (and columns
// [16 w, 16 w + 16) of dW3) in the weight gradient, whose m16n8k16 accumulators it keeps across
// chunks.  Every product takes bfloat16 operands: the gradient entering a layer's product
// (dL/dy, dz2, dz1) is rounded to bfloat16 once and used for both that layer's weight gradient and
// the gradient of the layer below; the bias gradients sum the float32 values.  Operands of the
// weight-gradient products (K = the chunk's points) are stored transposed, [feature][point], with a
// padded row so that the fragment loads are free of bank conflicts.
constexpr int kTS = 72;  // row stride (bf16) of the transposed tiles
constexpr int kW3S = 24;  // row stride of the transposed W3 (16 outputs + pad)

struct TrainSmem {
  MlpSmem w;                           // forward operands
  __nv_bfloat16 w2t[kH][kTS];          // w2t[i][o] = W2[o][i]
  __nv_bfloat16 w3t[kH][kW3S];         // w3t[i][o] = W3[o][i], outputs 12..15 zero
  __nv_bfloat16 x0t[kIn][kTS];         // bf16 inputs, [feature][point]
  __nv_bfloat16 h1t[kH][kTS];          // bf16 activations, [unit][point]
  __nv_bfloat16 h2t[kH][kTS];
  __nv_bfloat16 d1t[kH][kTS];          // bf16(dz1), [unit][point]
  __nv_bfloat16 d2t[kH][kTS];          // bf16(dz2)
  __nv_bfloat16 dyt[kOutPad][kTS];     // bf16(dL/dy), [output][point], outputs 12..15 zero
  float2 z1[64][kH / 2];               // first-layer pre-activations (float32), C-fragment pairs
  float y[64][kOutPad];                // outputs, overwritten by dL/dy (float32)
  float bsum[4][2 * kH];               // per warp: column sums of dz1 | dz2 over its 16 points
};

// Loss of one point and its gradient with respect to the 12 outputs (scaled by inv_n).
__device__ float point_loss(const float* y, const float* tg, float w_st, float w_v, float w_R, float inv_n,
                            float* dy) {
  const float e0 = y[0] - tg[0];
  float loss = w_st * e0 * e0;
  dy[0] = 2.0f * w_st * e0 * inv_n;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    const float e = y[k] - tg[k];
    loss += w_v * e * e;
    dy[k] = 2.0f * w_v * e * inv_n;
  }
  float ql[4], qr[4];
  const float nl = sqrtf(y[4] * y[4] + y[5] * y[5] + y[6] * y[6] + y[7] * y[7]);
  const float nr = sqrtf(y[8] * y[8] + y[9] * y[9] + y[10] * y[10] + y[11] * y[11]);
  const float il = 1.0f / fmaxf(nl, 1e-12f), ir = 1.0f / fmaxf(nr, 1e-12f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ql[k] = y[4 + k] * il;
    qr[k] = y[8 + k] * ir;
  }
  float L[4][4], M[4][4];
  left_mat(ql, L);
  right_mat(qr, M);
  float G[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float R = L[a][0] * M[0][b] + L[a][1] * M[1][b] + L[a][2] * M[2][b] + L[a][3] * M[3][b];
      const float e = R - tg[4 + 4 * a + b];
      loss += w_R * e * e;
      G[a][b] = 2.0f * w_R * e;
    }
  // R = L M: dL/dL = G M^T, dL/dM = L^T G; then the sign patterns of L(p) and Rr(q)
  float GL[4][4], GM[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      GL[a][b] = G[a][0] * M[b][0] + G[a][1] * M[b][1] + G[a][2] * M[b][2] + G[a][3] * M[b][3];
      GM[a][b] = L[0][a] * G[0][b] + L[1][a] * G[1][b] + L[2][a] * G[2][b] + L[3][a] * G[3][b];
    }
  float gl[4], gr[4];
  gl[0] = GL[0][0] + GL[1][1] + GL[2][2] + GL[3][3];
  gl[1] = GL[0][3] - GL[1][2] + GL[2][1] - GL[3][0];
  gl[2] = GL[0][2] + GL[1][3] - GL[2][0] - GL[3][1];
  gl[3] = -GL[0][1] + GL[1][0] + GL[2][3] - GL[3][2];
  gr[0] = GM[0][0] + GM[1][1] + GM[2][2] + GM[3][3];
  gr[1] = GM[0][3] + GM[1][2] - GM[2][1] - GM[3][0];
  gr[2] = -GM[0][2] + GM[1][3] + GM[2][0] - GM[3][1];
  gr[3] = GM[0][1] - GM[1][0] + GM[2][3] - GM[3][2];
  const float dl = gl[0] * ql[0] + gl[1] * ql[1] + gl[2] * ql[2] + gl[3] * ql[3];
  const float dr = gr[0] * qr[0] + gr[1] * qr[1] + gr[2] * qr[2] + gr[3] * qr[3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    dy[4 + k] = (gl[k] - ql[k] * dl) * il * inv_n;
    dy[8 + k] = (gr[k] - qr[k] * dr) * ir * inv_n;
  }
  return loss;
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragments of a warp's 16 rows (bf16 pairs along the row) -> transposed tile dst[col][row]
__device__ __forceinline__ void store_a_transposed(__nv_bfloat16 (*dst)[kTS], const uint32_t (*a)[4], int r0, int g,
                                                   int t) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int slot = 0; slot < 4; ++slot) {
      const int col = 16 * s + 8 * (slot >> 1) + 2 * t, row = r0 + g + 8 * (slot & 1);
      const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&a[s][slot]);
      dst[col][row] = v.x;
      dst[col + 1][row] = v.y;
    }
}

// Column sums of a C fragment over the warp's 16 rows (lanes of equal t hold the same columns)
__device__ __forceinline__ float2 column_sums(float d0, float d1, float d2, float d3) {
  float s0 = d0 + d2, s1 = d1 + d3;
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  return make_float2(s0, s1);
}

// d = c * gelu'(z) for n-tile j of a layer: column sums into bsum, bf16(d) into the transposed tile
// and into the A fragments a (k-block j / 2) of the next product
__device__ __forceinline__ void pre_activation_grad(const float* c, const float* z, int j, int r0, int g, int t,
                                                    float* bsum, __nv_bfloat16 (*dt)[kTS], uint32_t (*a)[4]) {
  const float d0 = c[0] * gelu_grad(z[0]), d1 = c[1] * gelu_grad(z[1]);
  const float d2 = c[2] * gelu_grad(z[2]), d3 = c[3] * gelu_grad(z[3]);
  const float2 cs = column_sums(d0, d1, d2, d3);
  const int col = 8 * j + 2 * t;
  if (g == 0) {
    bsum[col] = cs.x;
    bsum[col + 1] = cs.y;
  }
  const uint32_t lo = pack_bf16(d0, d1), hi = pack_bf16(d2, d3);
  if (a) {
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
  }
  const __nv_bfloat162 vl = *reinterpret_cast<const __nv_bfloat162*>(&lo);
  const __nv_bfloat162 vh = *reinterpret_cast<const __nv_bfloat162*>(&hi);
  dt[col][r0 + g] = vl.x;
  dt[col + 1][r0 + g] = vl.y;
  dt[col][r0 + g + 8] = vh.x;
  dt[col + 1][r0 + g + 8] = vh.y;
}

__global__ void __launch_bounds__(128) mlp_grad_kernel(const float* __restrict__ feat, const float* __restrict__ tgt,
                                                       int64_t n, const float* __restrict__ w, float w_st, float w_v,
                                                       float w_R, float* __restrict__ partial,
                                                       float* __restrict__ loss_partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  __shared__ float red[4];
  load_weights(S.w, w);
  for (int k = threadIdx.x; k < kH * kH; k += blockDim.x) S.w2t[k % kH][k / kH] = __float2bfloat16_rn(w[kOffW2 + k]);
  for (int k = threadIdx.x; k < kOutPad * kH; k += blockDim.x) {
    const int o = k / kH, i = k % kH;
    S.w3t[i][o] = __float2bfloat16_rn(o < kOut ? w[kOffW3 + o * kH + i] : 0.0f);
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  const float inv_n = 1.0f / (float)n;
  float gW1[8][4], gW2[8][4], gW3[2][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) gW1[j][e] = gW2[j][e] = 0.0f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) gW3[j][e] = 0.0f;
  float gb = 0.0f, gb3 = 0.0f, loss = 0.0f;
  for (int64_t base = (int64_t)blockIdx.x * 64; base < n; base += (int64_t)gridDim.x * 64) {
    __syncthreads();
    for (int k = tid; k < 64 * kIn; k += 128) {
      const int64_t p = base + k / kIn;
      S.x0t[k % kIn][k / kIn] = __float2bfloat16_rn(p < n ? feat[p * kIn + (k % kIn)] : 0.0f);
    }
    __syncthreads();
    // forward of the warp's 16 points; z1 goes to shared memory, z2 stays in registers
    float z2[8][4];
    {
      uint32_t a1[4][4], a2[4][4], a3[4][4];
      input_fragments([&](int r, int c) -> float { return __bfloat162float(S.x0t[c][r0 + r]); }, a1, g, t);
      {
        float z1[8][4];
        hidden_layer(S.w.w1, S.w.b1, a1, z1, a2, g, t);
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // read back by the same lanes in the gradient of z1
          S.z1[r0 + g][4 * j + t] = make_float2(z1[j][0], z1[j][1]);
          S.z1[r0 + g + 8][4 * j + t] = make_float2(z1[j][2], z1[j][3]);
        }
      }
      store_a_transposed(S.h1t, a2, r0, g, t);
      hidden_layer(S.w.w2, S.w.b2, a2, z2, a3, g, t);
      store_a_transposed(S.h2t, a3, r0, g, t);
      float y[2][4];
      output_layer(S.w, a3, y, g, t);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int col = 8 * j + 2 * t;
        S.y[r0 + g][col] = y[j][0];
        S.y[r0 + g][col + 1] = y[j][1];
        S.y[r0 + g + 8][col] = y[j][2];
        S.y[r0 + g + 8][col + 1] = y[j][3];
      }
    }
    __syncthreads();
    // loss and dL/dy per point (float32, and its bf16 rounding transposed)
    if (tid < 64) {
      const int64_t p = base + tid;
      float dy[kOut];
      if (p < n) {
        loss += point_loss(S.y[tid], tgt + p * 20, w_st, w_v, w_R, inv_n, dy);
      } else {
#pragma unroll
        for (int k = 0; k < kOut; ++k) dy[k] = 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kOutPad; ++k) {
        const float v = k < kOut ? dy[k] : 0.0f;
        S.y[tid][k] = v;
        S.dyt[k][tid] = __float2bfloat16_rn(v);
      }
    }
    __syncthreads();
    {
      // dz2 = (bf16(dy) W3) * gelu'(z2) for the warp's 16 points (K = 16 outputs)
      uint32_t ady[4];
      ady[0] = pack_bf16(S.y[r0 + g][2 * t], S.y[r0 + g][2 * t + 1]);
      ady[1] = pack_bf16(S.y[r0 + g + 8][2 * t], S.y[r0 + g + 8][2 * t + 1]);
      ady[2] = pack_bf16(S.y[r0 + g][2 * t + 8], S.y[r0 + g][2 * t + 9]);
      ady[3] = pack_bf16(S.y[r0 + g + 8][2 * t + 8], S.y[r0 + g + 8][2 * t + 9]);
      uint32_t ad2[4][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, ady, ld_pair(&S.w3t[8 * j + g][2 * t]), ld_pair(&S.w3t[8 * j + g][2 * t + 8]));
        pre_activation_grad(c, z2[j], j, r0, g, t, &S.bsum[warp][kH], S.d2t, ad2);
      }
      // dz1 = (bf16(dz2) W2) * gelu'(z1) (K = 64 units)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 0; s < 4; ++s)
          mma16816(c, ad2[s], ld_pair(&S.w2t[8 * j + g][16 * s + 2 * t]),
                   ld_pair(&S.w2t[8 * j + g][16 * s + 8 + 2 * t]));
        const float2 za = S.z1[r0 + g][4 * j + t], zb = S.z1[r0 + g + 8][4 * j + t];
        const float z[4] = {za.x, za.y, zb.x, zb.y};
        pre_activation_grad(c, z, j, r0, g, t, &S.bsum[warp][0], S.d1t, nullptr);
      }
    }
    __syncthreads();
    // weight gradients over the chunk's 64 points (K): dW1 += bf16(dz1)^T x0, dW2 += bf16(dz2)^T h1,
    // dW3 += bf16(dy)^T h2
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int k0 = 16 * s + 2 * t;
      uint32_t a1[4] = {ld_pair(&S.d1t[r0 + g][k0]), ld_pair(&S.d1t[r0 + g + 8][k0]), ld_pair(&S.d1t[r0 + g][k0 + 8]),
                        ld_pair(&S.d1t[r0 + g + 8][k0 + 8])};
      uint32_t a2[4] = {ld_pair(&S.d2t[r0 + g][k0]), ld_pair(&S.d2t[r0 + g + 8][k0]), ld_pair(&S.d2t[r0 + g][k0 + 8]),
                        ld_pair(&S.d2t[r0 + g + 8][k0 + 8])};
      uint32_t a3[4] = {ld_pair(&S.dyt[g][k0]), ld_pair(&S.dyt[g + 8][k0]), ld_pair(&S.dyt[g][k0 + 8]),
                        ld_pair(&S.dyt[g + 8][k0 + 8])};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        mma16816(gW1[j], a1, ld_pair(&S.x0t[8 * j + g][k0]), ld_pair(&S.x0t[8 * j + g][k0 + 8]));
        mma16816(gW2[j], a2, ld_pair(&S.h1t[8 * j + g][k0]), ld_pair(&S.h1t[8 * j + g][k0 + 8]));
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int j = 2 * warp + jj;
        mma16816(gW3[jj], a3, ld_pair(&S.h2t[8 * j + g][k0]), ld_pair(&S.h2t[8 * j + g][k0 + 8]));
      }
    }
    // bias gradients: float32 sums (thread tid < 64: b1 unit tid; else b2 unit tid - 64; tid < 12: b3)
    gb += S.bsum[0][tid] + S.bsum[1][tid] + S.bsum[2][tid] + S.bsum[3][tid];
    if (tid < kOut)
      for (int p = 0; p < 64; ++p) gb3 += S.y[p][tid];
  }
  float* P = partial + (int64_t)blockIdx.x * kWeights;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int o = r0 + g, i = 8 * j + 2 * t;
    P[kOffW1 + o * kIn + i] = gW1[j][0];
    P[kOffW1 + o * kIn + i + 1] = gW1[j][1];
    P[kOffW1 + (o + 8) * kIn + i] = gW1[j][2];
    P[kOffW1 + (o + 8) * kIn + i + 1] = gW1[j][3];
    P[kOffW2 + o * kH + i] = gW2[j][0];
    P[kOffW2 + o * kH + i + 1] = gW2[j][1];
    P[kOffW2 + (o + 8) * kH + i] = gW2[j][2];
    P[kOffW2 + (o + 8) * kH + i + 1] = gW2[j][3];
  }
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    const int h = 8 * (2 * warp + jj) + 2 * t;
    if (g < kOut) {
      P[kOffW3 + g * kH + h] = gW3[jj][0];
      P[kOffW3 + g * kH + h + 1] = gW3[jj][1];
    }
    if (g + 8 < kOut) {
      P[kOffW3 + (g + 8) * kH + h] = gW3[jj][2];
      P[kOffW3 + (g + 8) * kH + h + 1] = gW3[jj][3];
    }
  }
  if (tid < 64)
    P[kOffB1 + tid] = gb;
  else
    P[kOffB2 + tid - 64] = gb;
  if (tid < kOut) P[kOffB3 + tid] = gb3;
  // block loss
  float l = loss;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) red[warp] = l;
  __syncthreads();
  if (tid == 0) loss_partial[blockIdx.x] = (red[0] + red[1] + red[2] + red[3]) * inv_n;
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ loss_partial, int blocks,
                                  float* __restrict__ grads, float* __restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kWeights) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += partial[(int64_t)b * kWeights + k];
    grads[k] = s;
  }
  if (k == 0 && loss) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += loss_partial[b];
    *loss = s;
  }
}

int grad_blocks(int64_t n) {
  const int64_t chunks = (n + 63) / 64;
  return (int)(chunks < 304 ? (chunks > 0 ? chunks : 1) : 304);
}

}  // namespace

int64_t mlp_weight_count() { return kWeights; }

size_t mlp_grad_workspace_bytes(int64_t n) {
  const int b = grad_blocks(n);
  return ((size_t)b * kWeights * 4 + 255) / 256 * 256 + (size_t)b * 4;
}

cudaError_t launch_mlp_forward(const float* feat, int64_t n, const float* w, float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  I4D_PROF("mlp_forward", st);
  const int64_t chunks = (n + 63) / 64;
  const int blocks = (int)(chunks < 152 * 8 ? chunks : 152 * 8);
  mlp_forward_kernel<<<blocks, 128, 0, st>>>(feat, n, w, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* feat, const float* tgt, int64_t n, const float* w, float w_st, float w_v,
                            float w_R, float* grads, float* loss, void* ws, cudaStream_t st) {
  const int blocks = grad_blocks(n);
  float* partial = reinterpret_cast<float*>(ws);
  float* loss_partial = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) +
                                                 ((size_t)blocks * kWeights * 4 + 255) / 256 * 256);
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n == 0) {
    e = cudaMemsetAsync(grads, 0, sizeof(float) * kWeights, st);
    if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    return e;
  }
  I4D_PROF("mlp_grad", st);
  mlp_grad_kernel<<<blocks, 128, smem, st>>>(feat, tgt, n, w, w_st, w_v, w_R, partial, loss_partial);
  mlp_reduce_kernel<<<(kWeights + 255) / 256, 256, 0, st>>>(partial, loss_partial, blocks, grads, loss);
  return cudaGetLastError();
}

}  // namespace i4d
