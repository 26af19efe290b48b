// Fused Adam update over the flat parameter buffer, the photometric loss and PSNR.
#include "kernels.cuh"

namespace i4d {

namespace {

// One float4 of parameters per thread (grid-stride).  The update number comes from device memory so a
// captured graph replays with the right bias correction and learning-rate schedule.
__global__ void __launch_bounds__(256) adam_kernel(float4* __restrict__ p, const float4* __restrict__ g,
                                                   float4* __restrict__ m, float4* __restrict__ v, int64_t n4,
                                                   AdamGroups G, const int32_t* __restrict__ step, float b1, float b2,
                                                   float eps) {
  __shared__ float lr[I4D_MAX_ADAM_GROUPS][4];
  __shared__ float bc[2];
  const int s = *step + 1;
  if (threadIdx.x < G.n * 4) {
    const int k = threadIdx.x >> 2, lane = threadIdx.x & 3;
    float r = 0.0f;
    if (G.decay[k] > 0) r = fminf((float)s / (float)G.decay[k], 1.0f);
    const float l0 = G.lr0[k][lane], l1 = G.lr1[k][lane];
    // log-linear interpolation between lr_init and lr_final (zero stays zero)
    lr[k][lane] = (l0 > 0.0f && l1 > 0.0f) ? expf((1.0f - r) * logf(l0) + r * logf(l1)) : l0;
  }
  if (threadIdx.x == 0) {
    bc[0] = 1.0f - powf(b1, (float)s);
    bc[1] = 1.0f - powf(b2, (float)s);
  }
  __syncthreads();
  const float ibc1 = 1.0f / bc[0], isbc2 = 1.0f / sqrtf(bc[1]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = 4 * i;
    int k = -1;
    for (int j = 0; j < G.n; ++j)
      if (e >= G.begin[j] && e < G.end[j]) {
        k = j;
        break;
      }
    if (k < 0) continue;
    const float4 gg = g[i];
    float4 mm = m[i], vv = v[i], pp = p[i];
    const float gs[4] = {gg.x, gg.y, gg.z, gg.w};
    float ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w}, ps[4] = {pp.x, pp.y, pp.z, pp.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      ms[l] = b1 * ms[l] + (1.0f - b1) * gs[l];
      vs[l] = b2 * vs[l] + (1.0f - b2) * gs[l] * gs[l];
      const float denom = sqrtf(vs[l]) * isbc2 + eps;
      ps[l] -= lr[k][l] * (ms[l] * ibc1) / denom;
    }
    p[i] = make_float4(ps[0], ps[1], ps[2], ps[3]);
    m[i] = make_float4(ms[0], ms[1], ms[2], ms[3]);
    v[i] = make_float4(vs[0], vs[1], vs[2], vs[3]);
  }
}

__global__ void step_increment_kernel(int32_t* step) { *step += 1; }

__device__ __forceinline__ float block_sum(float x) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  x = (threadIdx.x < (blockDim.x >> 5)) ? red[lane] : 0.0f;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  return x;  // valid in thread 0
}

__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                   int64_t count, int kind, float inv_count,
                                                   float* __restrict__ dimg, float* __restrict__ loss) {
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    if (kind == I4D_LOSS_L1) {
      acc += fabsf(d);
      dimg[i] = (d > 0.0f ? inv_count : (d < 0.0f ? -inv_count : 0.0f));
    } else {
      acc += d * d;
      dimg[i] = 2.0f * d * inv_count;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(loss, acc * inv_count);
}

__global__ void __launch_bounds__(256) sqerr_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                    int64_t count, float* __restrict__ out) {
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    acc += d * d;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

__global__ void psnr_finish_kernel(float* out, float count) {
  const float mse = *out / count;
  *out = 10.0f * log10f(1.0f / fmaxf(mse, 1e-30f));
}

int reduce_blocks(int64_t count) {
  int64_t b = (count + 255) / 256;
  return (int)(b < 1216 ? (b > 0 ? b : 1) : 1216);
}

}  // namespace

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, const AdamGroups& groups,
                        int32_t* step, float b1, float b2, float eps, cudaStream_t st) {
  const int64_t n4 = count / 4;
  if (n4 > 0) {
    I4D_PROF("adam", st);
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<float4*>(p), reinterpret_cast<const float4*>(g),
                                                  reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n4,
                                                  groups, step, b1, b2, eps);
  }
  step_increment_kernel<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* img, const float* target, int64_t count, int kind, float* dL_dimg,
                        float* loss_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss_out, 0, sizeof(float), st);
  if (e != cudaSuccess || count == 0) return e;
  I4D_PROF("loss", st);
  loss_kernel<<<reduce_blocks(count), 256, 0, st>>>(img, target, count, kind, 1.0f / (float)count, dL_dimg, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_psnr(const float* img, const float* target, int64_t count, float* psnr_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(psnr_out, 0, sizeof(float), st);
  if (e != cudaSuccess || count == 0) return e;
  sqerr_kernel<<<reduce_blocks(count), 256, 0, st>>>(img, target, count, psnr_out);
  psnr_finish_kernel<<<1, 1, 0, st>>>(psnr_out, (float)count);
  return cudaGetLastError();
}

}  // namespace i4d
