// Slice + project (Eq. 7-9, EWA, SH colour, blendable extent and tile rectangle) and its backward
// chain.
//
// One thread per Gaussian loops over all views of the batch: the view-independent part (rotation,
// 4D covariance, sigmoid) is computed once and the parameters are read from HBM once per launch,
// not once per view.  Each (view, Gaussian) record is one 64-byte record (four float4), written only
// when the Gaussian covers a tile of the view.
#include "gauss_math.cuh"
#include "kernels.cuh"

namespace i4d {

namespace {

struct ViewExtra {
  float campos[3];
  float tanx, tany;
};

__device__ __forceinline__ void load_cameras(const ViewTable& vt, const i4d_camera* __restrict__ cams, Cam* sc,
                                             ViewExtra* sx) {
  const int V = vt.n_views;
  const float* src = reinterpret_cast<const float*>(cams);
  float* dst = reinterpret_cast<float*>(sc);
  for (int k = threadIdx.x; k < V * 20; k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const Cam& c = sc[v];
    sx[v].campos[0] = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
    sx[v].campos[1] = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
    sx[v].campos[2] = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
    sx[v].tanx = 0.5f * (float)vt.width[v] / c.fx;
    sx[v].tany = 0.5f * (float)vt.height[v] / c.fy;
  }
  __syncthreads();
}

template <int DEG>
__global__ void __launch_bounds__(256) slice_project_kernel(const float4* __restrict__ P, int n, int mode, ViewTable vt,
                                                            const i4d_camera* __restrict__ cams, Settings S,
                                                            float4* __restrict__ proj, uint32_t* __restrict__ touched,
                                                            int nt) {
  __shared__ Cam sc[kMaxViews];
  __shared__ ViewExtra sx[kMaxViews];
  load_cameras(vt, cams, sc, sx);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  GaussState G;
  gauss_setup(__ldg(&P[i]), __ldg(&P[(size_t)n + i]), __ldg(&P[2 * (size_t)n + i]), __ldg(&P[3 * (size_t)n + i]),
              __ldg(&P[4 * (size_t)n + i]), mode, G);
  for (int v = 0; v < vt.n_views; ++v) {
    ViewFwd F;
    view_forward<DEG>(G, P + 5 * (size_t)n, n, i, sc[v], sx[v].campos, sx[v].tanx, sx[v].tany, S, F, nt);
    uint32_t cnt = 0;
    float4 box = make_float4(1.0f, 0.0f, 1.0f, 0.0f);  // empty
    if (F.visible) {
      // screen extent where a fragment can be blended (q <= q_max and alpha >= alpha_min)
      box = ellipse_box(F.u, F.v, F.conic[0], F.conic[1], F.conic[2], blend_q(F.ot, S));
      int x0, y0, x1, y1;
      box_rect(box, vt.width[v], vt.height[v], vt.tile_w, vt.tile_h, vt.tiles_x[v], vt.tiles_y[v], x0, y0, x1, y1);
      cnt = (uint32_t)((x1 - x0) * (y1 - y0));
    }
    const size_t r = (size_t)v * n + i;
    if (cnt > 0) {
      // the record as the compositing kernels stage it: conic scaled by kFalloff (exp(-q/2) =
      // 2^(sa dx^2 + sb2 dx dy + sc dy^2)) and the exponent threshold of the kept test
      // m >= kFalloff min(q_max, 2 ln(o_t / alpha_min)), computed once here instead of at every
      // staging.  Records on no tile are never read, so they are not written.
      const float m_thr = __fmul_rn(kFalloff, fminf(S.q_max, 2.0f * logf(F.ot / S.alpha_min)));
      float4* rec = proj + 4 * r;
      rec[0] = box;
      rec[1] = make_float4(F.u, F.v, __fmul_rn(kFalloff, F.conic[0]), __fmul_rn(2.0f * kFalloff, F.conic[1]));
      rec[2] = make_float4(__fmul_rn(kFalloff, F.conic[2]), F.ot, m_thr, fmaxf(F.raw[0], 0.0f));
      rec[3] = make_float4(fmaxf(F.raw[1], 0.0f), fmaxf(F.raw[2], 0.0f), F.m[2], F.radius);
    }
    touched[r] = cnt;
  }
}

template <int DEG>
__global__ void __launch_bounds__(128) slice_project_bwd_kernel(const float4* __restrict__ P, int n, int mode,
                                                                ViewTable vt, const i4d_camera* __restrict__ cams,
                                                                Settings S, const uint32_t* __restrict__ touched,
                                                                const float4* __restrict__ grad2d,
                                                                float4* __restrict__ grads, int nt) {
  __shared__ Cam sc[kMaxViews];
  __shared__ ViewExtra sx[kMaxViews];
  load_cameras(vt, cams, sc, sx);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  GaussState G;
  gauss_setup(__ldg(&P[i]), __ldg(&P[(size_t)n + i]), __ldg(&P[2 * (size_t)n + i]), __ldg(&P[3 * (size_t)n + i]),
              __ldg(&P[4 * (size_t)n + i]), mode, G);
  constexpr int K = (DEG + 1) * (DEG + 1) - 1;
  constexpr int NP = DEG == 0 ? 0 : (DEG == 1 ? 3 : (DEG == 2 ? 6 : 12));
  ParamGrad PG;
#pragma unroll
  for (int a = 0; a < 4; ++a) PG.mu[a] = PG.ls[a] = PG.ql[a] = PG.qr[a] = PG.orgb[a] = 0.0f;
  float gsh[NP * 4 > 0 ? NP * 4 : 1];
#pragma unroll
  for (int a = 0; a < NP * 4; ++a) gsh[a] = 0.0f;
  float gA[6] = {0, 0, 0, 0, 0, 0}, gb[3] = {0, 0, 0}, gc = 0.0f;
  const size_t VN = (size_t)vt.n_views * n;
  // SCH variant: its coefficient gradients are summed over the views in place in this Gaussian's
  // own entries of the gradient planes (no other thread writes them)
  float4* gsch = grads + (size_t)(5 + NP) * n;
  for (int p = 0; p < sch_planes(DEG, nt); ++p) gsch[(size_t)p * n + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int v = 0; v < vt.n_views; ++v) {
    const size_t r = (size_t)v * n + i;
    if (__ldg(&touched[r]) == 0) continue;
    const float4 g0 = __ldg(&grad2d[r]), g1 = __ldg(&grad2d[VN + r]);
    const float g8 = __ldg(reinterpret_cast<const float*>(grad2d + 2 * VN) + r);
    const float g[9] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g8};
    ViewFwd F;
    view_forward<DEG>(G, P + 5 * (size_t)n, n, i, sc[v], sx[v].campos, sx[v].tanx, sx[v].tany, S, F, nt);
    view_backward<DEG>(G, F, P + 5 * (size_t)n, n, i, sc[v], g, PG, gsh, gA, gc, gb, nt, gsch);
  }
  sigma_backward(G, mode, gA, gb, gc, PG);
  grads[i] = make_float4(PG.mu[0], PG.mu[1], PG.mu[2], PG.mu[3]);
  grads[(size_t)n + i] = make_float4(PG.ls[0], PG.ls[1], PG.ls[2], PG.ls[3]);
  grads[2 * (size_t)n + i] = make_float4(PG.ql[0], PG.ql[1], PG.ql[2], PG.ql[3]);
  grads[3 * (size_t)n + i] = make_float4(PG.qr[0], PG.qr[1], PG.qr[2], PG.qr[3]);
  grads[4 * (size_t)n + i] = make_float4(PG.orgb[0], PG.orgb[1], PG.orgb[2], PG.orgb[3]);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    // lanes beyond 3K are padding
    float4 q;
    q.x = (4 * p + 0 < 3 * K) ? gsh[4 * p + 0] : 0.0f;
    q.y = (4 * p + 1 < 3 * K) ? gsh[4 * p + 1] : 0.0f;
    q.z = (4 * p + 2 < 3 * K) ? gsh[4 * p + 2] : 0.0f;
    q.w = (4 * p + 3 < 3 * K) ? gsh[4 * p + 3] : 0.0f;
    grads[(size_t)(5 + p) * n + i] = q;
  }
}

}  // namespace

cudaError_t launch_slice_project(const float* params, int n, int sh_deg, int mode, const ViewTable& vt,
                                 const i4d_camera* cams, const Settings& S, float* proj, uint32_t* touched,
                                 cudaStream_t st, int nt) {
  if (n == 0) return cudaSuccess;
  I4D_PROF("slice_project", st);
  const int threads = 256, blocks = (n + threads - 1) / threads;
  const float4* P = reinterpret_cast<const float4*>(params);
  float4* R = reinterpret_cast<float4*>(proj);
  switch (sh_deg) {
    case 0: slice_project_kernel<0><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, R, touched, nt); break;
    case 1: slice_project_kernel<1><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, R, touched, nt); break;
    case 2: slice_project_kernel<2><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, R, touched, nt); break;
    default: slice_project_kernel<3><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, R, touched, nt); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_project_bwd(const float* params, int n, int sh_deg, int mode, const ViewTable& vt,
                                     const i4d_camera* cams, const Settings& S, const uint32_t* touched,
                                     const float* grad2d, float* grads, cudaStream_t st, int nt) {
  if (n == 0) return cudaSuccess;
  I4D_PROF("slice_project_bwd", st);
  const int threads = 128, blocks = (n + threads - 1) / threads;
  const float4* P = reinterpret_cast<const float4*>(params);
  const float4* G2 = reinterpret_cast<const float4*>(grad2d);
  float4* GR = reinterpret_cast<float4*>(grads);
  switch (sh_deg) {
    case 0: slice_project_bwd_kernel<0><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, touched, G2, GR, nt); break;
    case 1: slice_project_bwd_kernel<1><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, touched, G2, GR, nt); break;
    case 2: slice_project_bwd_kernel<2><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, touched, G2, GR, nt); break;
    default: slice_project_bwd_kernel<3><<<blocks, threads, 0, st>>>(P, n, mode, vt, cams, S, touched, G2, GR, nt); break;
  }
  return cudaGetLastError();
}

}  // namespace i4d
