// Heuristic initialisation of 4D Gaussians from the pruned voxels (Sec. 4.1, Sec. 3.3
// "Motion-Aware Gaussian"): mean = (centroid, averaged frame time); temporal scale s_t = two
// frames for dynamic voxels and the whole video for static ones; isotropic spatial scale;
// identity rotation (R = I); averaged colour; one opacity for all.
#include "gauss_math.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace i4d {

namespace {

__global__ void __launch_bounds__(256) init_heuristic_kernel(const float* __restrict__ xyz,
                                                             const float* __restrict__ rgb,
                                                             const float* __restrict__ t,
                                                             const uint8_t* __restrict__ flag, int n, int nplanes,
                                                             float log_s, float log_st_dyn, float log_st_static,
                                                             float opac_logit, float4* __restrict__ P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t N = (size_t)n;
  const bool dyn = flag ? (flag[i] != 0) : false;
  P[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], t ? t[i] : 0.5f);
  P[N + i] = make_float4(log_s, log_s, log_s, dyn ? log_st_dyn : log_st_static);
  P[2 * N + i] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
  P[3 * N + i] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
  P[4 * N + i] = make_float4(opac_logit, rgb ? rgb[3 * i] : 0.5f, rgb ? rgb[3 * i + 1] : 0.5f,
                             rgb ? rgb[3 * i + 2] : 0.5f);
  for (int p = 5; p < nplanes; ++p) P[(size_t)p * N + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Initialisation from the learned proposal y = (log s_t, v, q_l, q_r) per point: spatial scale from
// the 3-NN distance, temporal log-scale and rotation from the MLP.  A point whose proposal is not
// finite or has a near-zero quaternion falls back to the heuristic (s_t by flag, R = I), counted.
__global__ void __launch_bounds__(256) init_learned_kernel(const float* __restrict__ xyz, const float* __restrict__ rgb,
                                                           const float* __restrict__ t,
                                                           const uint8_t* __restrict__ flag,
                                                           const float* __restrict__ spatial,
                                                           const float* __restrict__ y, int n, int nplanes,
                                                           float log_st_dyn, float log_st_static, float opac_logit,
                                                           float4* __restrict__ P, int32_t* __restrict__ fallbacks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t N = (size_t)n;
  const bool dyn = flag ? (flag[i] != 0) : false;
  const float* yi = y ? y + 12 * (size_t)i : nullptr;
  bool ok = false;
  if (yi) {
    float nl = 0.f, nr = 0.f;
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) finite = finite && isfinite(yi[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      nl += yi[4 + k] * yi[4 + k];
      nr += yi[8 + k] * yi[8 + k];
    }
    ok = finite && nl > 1e-8f && nr > 1e-8f && yi[0] > -20.0f && yi[0] < 5.0f;
    if (!ok && fallbacks) atomicAdd(fallbacks, 1);
  }
  const float ls = logf(spatial[i]);
  P[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], t ? t[i] : 0.5f);
  P[N + i] = make_float4(ls, ls, ls, ok ? yi[0] : (dyn ? log_st_dyn : log_st_static));
  P[2 * N + i] = ok ? make_float4(yi[4], yi[5], yi[6], yi[7]) : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
  P[3 * N + i] = ok ? make_float4(yi[8], yi[9], yi[10], yi[11]) : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
  P[4 * N + i] = make_float4(opac_logit, rgb ? rgb[3 * i] : 0.5f, rgb ? rgb[3 * i + 1] : 0.5f,
                             rgb ? rgb[3 * i + 2] : 0.5f);
  for (int p = 5; p < nplanes; ++p) P[(size_t)p * N + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Per Gaussian: (log s_t, velocity b / c of Eq. 7, R row-major) -- the quantities the learned
// initialisation is trained to propose.
__global__ void __launch_bounds__(256) motion_targets_kernel(const float4* __restrict__ P, int n, int mode,
                                                             float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t N = (size_t)n;
  GaussState G;
  gauss_setup(P[i], P[N + i], P[2 * N + i], P[3 * N + i], P[4 * N + i], mode, G);
  float* o = out + 20 * (size_t)i;
  o[0] = P[N + i].w;
  o[1] = G.b[0] / G.c;
  o[2] = G.b[1] / G.c;
  o[3] = G.b[2] / G.c;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) o[4 + 4 * a + b] = G.R[a][b];
}

}  // namespace

cudaError_t launch_motion_targets(const float* params, int n, int mode, float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  I4D_PROF("motion_targets", st);
  motion_targets_kernel<<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<const float4*>(params), n, mode, out);
  return cudaGetLastError();
}

cudaError_t launch_init_learned(const float* xyz, const float* rgb, const float* t, const uint8_t* flag,
                                const float* spatial, const float* y, int n, int sh_deg, float st_dynamic,
                                float st_static, float opacity, float* params, int32_t* fallbacks, cudaStream_t st) {
  cudaError_t e = fallbacks ? cudaMemsetAsync(fallbacks, 0, sizeof(int32_t), st) : cudaSuccess;
  if (e != cudaSuccess || n == 0) return e;
  I4D_PROF("init_learned", st);
  init_learned_kernel<<<(n + 255) / 256, 256, 0, st>>>(xyz, rgb, t, flag, spatial, y, n, 5 + sh_planes(sh_deg),
                                                        logf(st_dynamic), logf(st_static),
                                                        logf(opacity / (1.0f - opacity)),
                                                        reinterpret_cast<float4*>(params), fallbacks);
  return cudaGetLastError();
}

cudaError_t launch_init_heuristic(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int n,
                                  int sh_deg, float spatial_scale, float st_dynamic, float st_static, float opacity,
                                  float* params, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  I4D_PROF("init_heuristic", st);
  const float opac_logit = logf(opacity / (1.0f - opacity));
  init_heuristic_kernel<<<(n + 255) / 256, 256, 0, st>>>(xyz, rgb, t, flag, n, 5 + sh_planes(sh_deg),
                                                          logf(spatial_scale), logf(st_dynamic), logf(st_static),
                                                          opac_logit, reinterpret_cast<float4*>(params));
  return cudaGetLastError();
}

}  // namespace i4d
