// extern "C" entry points of libi4d.so (declared and documented in include/i4d.h).
// Host-side argument checks happen here; every device buffer is caller-owned.
#include <string.h>

#include "kernels.cuh"

using namespace i4d;

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

Settings to_settings(const i4d_settings* s) {
  i4d_settings d;
  if (!s) {
    i4d_default_settings(&d);
    s = &d;
  }
  Settings r;
  r.alpha_max = s->alpha_max;
  r.alpha_min = s->alpha_min;
  r.T_min = s->T_min;
  r.q_max = s->q_max;
  r.ot_min = s->ot_min;
  r.z_near = s->z_near;
  r.dilation = s->dilation;
  r.fov_clamp = s->fov_clamp;
  r.bg[0] = s->bg[0];
  r.bg[1] = s->bg[1];
  r.bg[2] = s->bg[2];
  return r;
}

bool tile_supported(int w, int h) {
  return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 16 && h == 8) || (w == 32 && h == 8) ||
         (w == 32 && h == 16);
}

// Fill the per-launch view table; returns false on invalid views.
bool make_view_table(const i4d_views* v, ViewTable& vt) {
  if (!v || v->n_views < 1 || v->n_views > I4D_MAX_VIEWS || !tile_supported(v->tile_w, v->tile_h)) return false;
  memset(&vt, 0, sizeof(vt));
  vt.n_views = v->n_views;
  vt.tile_w = v->tile_w;
  vt.tile_h = v->tile_h;
  int64_t toff = 0, poff = 0;
  for (int k = 0; k < v->n_views; ++k) {
    const int W = v->width[k], H = v->height[k];
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return false;
    vt.width[k] = W;
    vt.height[k] = H;
    vt.tiles_x[k] = (W + v->tile_w - 1) / v->tile_w;
    vt.tiles_y[k] = (H + v->tile_h - 1) / v->tile_h;
    vt.tile_off[k] = (int)toff;
    vt.pix_off[k] = poff;
    toff += (int64_t)vt.tiles_x[k] * vt.tiles_y[k];
    poff += (int64_t)W * H;
  }
  if (toff >= (1ll << 31)) return false;
  vt.tile_off[v->n_views] = (int)toff;
  vt.pix_off[v->n_views] = poff;
  return true;
}

int32_t cuda_status(cudaError_t e) { return e == cudaSuccess ? I4D_OK : I4D_ERR_CUDA; }

int bits_for(int64_t x) {
  int b = 0;
  while ((1ll << b) < x) ++b;
  return b;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int32_t i4d_version(void) { return I4D_VERSION; }

const char* i4d_status_string(int32_t status) {
  switch (status) {
    case I4D_OK: return "ok";
    case I4D_ERR_ARG: return "invalid argument";
    case I4D_ERR_CAPACITY: return "capacity exceeded";
    case I4D_ERR_CUDA: return "CUDA error";
    case I4D_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown status";
  }
}

void i4d_default_settings(i4d_settings* out) {
  if (!out) return;
  out->alpha_max = 0.99f;
  out->alpha_min = 1.0f / 255.0f;
  out->T_min = 1e-4f;
  out->q_max = 9.0f;
  out->ot_min = 1.0f / 255.0f;
  out->z_near = 0.2f;
  out->dilation = 0.3f;
  out->fov_clamp = 1.3f;
  out->bg[0] = out->bg[1] = out->bg[2] = 0.0f;
  out->pad = 0.0f;
}

int64_t i4d_param_floats_sch(int32_t sh_deg, int32_t sch_terms) {
  if (sh_deg < 0 || sh_deg > 3 || sch_terms < 0 || sch_terms > I4D_MAX_SCH_TERMS) return -1;
  return 20 + 4 * sh_planes(sh_deg) + 4 * sch_planes(sh_deg, sch_terms);
}

int64_t i4d_param_floats(int32_t sh_deg) {
  if (sh_deg < 0 || sh_deg > 3) return -1;
  return 20 + 4 * sh_planes(sh_deg);
}

int64_t i4d_total_tiles(const i4d_views* views) {
  ViewTable vt;
  if (!make_view_table(views, vt)) return -1;
  return vt.tile_off[vt.n_views];
}

int64_t i4d_total_pixels(const i4d_views* views) {
  ViewTable vt;
  if (!make_view_table(views, vt)) return -1;
  return vt.pix_off[vt.n_views];
}

int32_t i4d_slice_project(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                          const i4d_settings* settings, float* proj, uint32_t* touched, void* stream) {
  ViewTable vt;
  if (!g || g->n < 0 || g->sh_deg < 0 || g->sh_deg > 3 || g->mode < 0 || g->mode > 2) return I4D_ERR_ARG;
  if (!make_view_table(views, vt)) return I4D_ERR_ARG;
  if (g->n == 0) return I4D_OK;
  if (!g->params || !cams || !proj || !touched || !aligned16(g->params) || !aligned16(proj)) return I4D_ERR_ARG;
  if (g->sch_terms < 0 || g->sch_terms > I4D_MAX_SCH_TERMS) return I4D_ERR_ARG;
  return cuda_status(launch_slice_project(g->params, g->n, g->sh_deg, g->mode, vt, cams, to_settings(settings), proj,
                                          touched, (cudaStream_t)stream, g->sch_terms));
}

size_t i4d_bin_tiles_workspace_size(const i4d_views* views, int32_t n, int64_t capacity) {
  ViewTable vt;
  if (!make_view_table(views, vt) || n < 0 || capacity < 0) return 0;
  return bin_workspace_bytes((int64_t)vt.n_views * n, capacity);
}

int32_t i4d_bin_tiles(const i4d_views* views, int32_t n, const float* proj, const uint32_t* touched,
                      int64_t capacity, uint32_t* ids, uint32_t* ranges, int64_t* n_inst, int32_t* status, void* ws,
                      size_t ws_bytes, void* stream) {
  ViewTable vt;
  if (!make_view_table(views, vt) || n < 0 || capacity < 1 || capacity >= (1ll << 32)) return I4D_ERR_ARG;
  if ((int64_t)vt.n_views * n >= (1ll << 32)) return I4D_ERR_ARG;
  if (!proj || !touched || !ids || !ranges || !n_inst || !status || !ws) return I4D_ERR_ARG;
  if (ws_bytes < i4d_bin_tiles_workspace_size(views, n, capacity)) return I4D_ERR_WORKSPACE;
  return cuda_status(
      launch_bin_tiles(vt, n, proj, touched, capacity, ids, ranges, n_inst, status, ws, (cudaStream_t)stream));
}

int32_t i4d_render_fwd(const i4d_views* views, int32_t n, const float* proj, const uint32_t* ids,
                       const uint32_t* ranges, const i4d_settings* settings, const i4d_tune* tune, float* img,
                       float* T_final, uint32_t* last, uint32_t* n_contrib, void* stream) {
  ViewTable vt;
  if (!make_view_table(views, vt) || n < 0) return I4D_ERR_ARG;
  if (!proj || !ids || !ranges || !img || !T_final || !last) return I4D_ERR_ARG;
  const int batch = tune ? tune->batch : 0;
  if (batch != 0 && batch != 16 && batch != 32 && batch != 64) return I4D_ERR_ARG;
  return cuda_status(launch_render_fwd(vt, n, proj, ids, ranges, to_settings(settings), batch ? batch : 32, img,
                                       T_final, last, n_contrib, (cudaStream_t)stream));
}

int32_t i4d_render_bwd(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                       const i4d_settings* settings, const float* proj, const uint32_t* touched,
                       const uint32_t* ids, const uint32_t* ranges, const float* T_final, const uint32_t* last,
                       const float* dL_dimg, float* grad2d, float* grads, void* stream) {
  ViewTable vt;
  if (!g || g->n < 0 || g->sh_deg < 0 || g->sh_deg > 3 || g->mode < 0 || g->mode > 2) return I4D_ERR_ARG;
  if (g->sch_terms < 0 || g->sch_terms > I4D_MAX_SCH_TERMS) return I4D_ERR_ARG;
  if (!make_view_table(views, vt)) return I4D_ERR_ARG;
  if (g->n == 0) return I4D_OK;
  if (!g->params || !cams || !proj || !touched || !ids || !ranges || !T_final || !last || !dL_dimg || !grad2d ||
      !grads || !aligned16(grad2d) || !aligned16(grads))
    return I4D_ERR_ARG;
  const Settings S = to_settings(settings);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_render_bwd(vt, g->n, proj, ids, ranges, S, T_final, last, dL_dimg, grad2d, st);
  if (e == cudaSuccess)
    e = launch_slice_project_bwd(g->params, g->n, g->sh_deg, g->mode, vt, cams, S, touched, grad2d, grads, st,
                                 g->sch_terms);
  return cuda_status(e);
}

int32_t i4d_loss(const float* img, const float* target, int64_t count, int32_t kind, float* dL_dimg,
                 float* loss_out, void* stream) {
  if (count < 0 || (kind != I4D_LOSS_L1 && kind != I4D_LOSS_MSE) || !loss_out) return I4D_ERR_ARG;
  if (count > 0 && (!img || !target || !dL_dimg)) return I4D_ERR_ARG;
  return cuda_status(launch_loss(img, target, count, kind, dL_dimg, loss_out, (cudaStream_t)stream));
}

size_t i4d_adaptive_voxel_workspace_size(int32_t F) { return F > 0 ? adaptive_voxel_workspace_bytes(F) : 0; }

int32_t i4d_adaptive_voxel(const float* depth, int32_t F, int32_t W, int32_t H, const i4d_camera* cams,
                           float lambda_s, float* voxel_out, void* ws, size_t ws_bytes, void* stream) {
  if (F < 1 || W < 1 || H < 1 || !depth || !cams || !voxel_out || !ws || !(lambda_s > 0.0f)) return I4D_ERR_ARG;
  if (ws_bytes < adaptive_voxel_workspace_bytes(F)) return I4D_ERR_WORKSPACE;
  return cuda_status(launch_adaptive_voxel(depth, F, H, W, cams, lambda_s, voxel_out, ws, (cudaStream_t)stream));
}

size_t i4d_motion_masks_workspace_size(int32_t F) { return F > 0 ? motion_mask_workspace_bytes(F) : 0; }

int32_t i4d_motion_masks(const float* prob, int32_t F, int32_t w, int32_t h, int32_t W, int32_t H, uint8_t* mask,
                         int32_t* thresholds, void* ws, size_t ws_bytes, void* stream) {
  if (F < 1 || w < 1 || h < 1 || W < 1 || H < 1 || (int64_t)W * H >= (1ll << 31) || !prob || !mask || !ws)
    return I4D_ERR_ARG;
  if (ws_bytes < motion_mask_workspace_bytes(F)) return I4D_ERR_WORKSPACE;
  return cuda_status(launch_motion_masks(prob, F, h, w, H, W, mask, thresholds, ws, (cudaStream_t)stream));
}

size_t i4d_photometric_loss_workspace_size(const i4d_views* views) {
  ViewTable vt;
  if (!make_view_table(views, vt)) return 0;
  return photometric_workspace_bytes(vt);
}

int32_t i4d_photometric_loss(const i4d_views* views, const float* img, const float* target, float lambda_dssim,
                             float* dL_dimg, float* loss_out, float* ssim_out, void* ws, size_t ws_bytes,
                             void* stream) {
  ViewTable vt;
  if (!make_view_table(views, vt)) return I4D_ERR_ARG;
  if (!(lambda_dssim >= 0.0f && lambda_dssim <= 1.0f) || !img || !target || !dL_dimg || !loss_out || !ws)
    return I4D_ERR_ARG;
  if (ws_bytes < photometric_workspace_bytes(vt)) return I4D_ERR_WORKSPACE;
  return cuda_status(launch_photometric_loss(vt, img, target, lambda_dssim, dL_dimg, loss_out, ssim_out, ws,
                                             (cudaStream_t)stream));
}

int32_t i4d_psnr(const float* img, const float* target, int64_t count, float* psnr_out, void* stream) {
  if (count < 0 || !psnr_out || (count > 0 && (!img || !target))) return I4D_ERR_ARG;
  return cuda_status(launch_psnr(img, target, count, psnr_out, (cudaStream_t)stream));
}

int32_t i4d_adam_step(float* params, const float* grads, float* m, float* v, int64_t count,
                      const i4d_adam_group* groups, int32_t n_groups, int32_t* step, float beta1, float beta2,
                      float eps, void* stream) {
  if (count < 0 || (count & 3) || n_groups < 0 || n_groups > I4D_MAX_ADAM_GROUPS || !step) return I4D_ERR_ARG;
  if (count > 0 && (!params || !grads || !m || !v || !aligned16(params) || !aligned16(grads) || !aligned16(m) ||
                    !aligned16(v)))
    return I4D_ERR_ARG;
  if (n_groups > 0 && !groups) return I4D_ERR_ARG;
  AdamGroups G;
  memset(&G, 0, sizeof(G));
  G.n = n_groups;
  for (int k = 0; k < n_groups; ++k) {
    if (groups[k].begin < 0 || groups[k].end > count || groups[k].begin > groups[k].end || (groups[k].begin & 3) ||
        (groups[k].end & 3))
      return I4D_ERR_ARG;
    G.begin[k] = groups[k].begin;
    G.end[k] = groups[k].end;
    for (int l = 0; l < 4; ++l) {
      G.lr0[k][l] = groups[k].lr_init[l];
      G.lr1[k][l] = groups[k].lr_final[l];
    }
    G.decay[k] = groups[k].decay_steps;
  }
  return cuda_status(launch_adam(params, grads, m, v, count, G, step, beta1, beta2, eps, (cudaStream_t)stream));
}

int32_t i4d_init_heuristic(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int32_t n,
                           int32_t sh_deg, float spatial_scale, float st_dynamic, float st_static, float opacity,
                           float* params, void* stream) {
  if (n < 0 || sh_deg < 0 || sh_deg > 3 || !(spatial_scale > 0.0f) || !(st_dynamic > 0.0f) || !(st_static > 0.0f) ||
      !(opacity > 0.0f && opacity < 1.0f))
    return I4D_ERR_ARG;
  if (n > 0 && (!xyz || !params || !aligned16(params))) return I4D_ERR_ARG;
  return cuda_status(launch_init_heuristic(xyz, rgb, t, flag, n, sh_deg, spatial_scale, st_dynamic, st_static,
                                           opacity, params, (cudaStream_t)stream));
}

int32_t i4d_init_learned(const float* xyz, const float* rgb, const float* t, const uint8_t* flag,
                         const float* spatial, const float* mlp_out, int32_t n, int32_t sh_deg, float st_dynamic,
                         float st_static, float opacity, float* params, int32_t* fallbacks, void* stream) {
  if (n < 0 || sh_deg < 0 || sh_deg > 3 || !(st_dynamic > 0.0f) || !(st_static > 0.0f) ||
      !(opacity > 0.0f && opacity < 1.0f))
    return I4D_ERR_ARG;
  if (n > 0 && (!xyz || !spatial || !params || !aligned16(params))) return I4D_ERR_ARG;
  return cuda_status(launch_init_learned(xyz, rgb, t, flag, spatial, mlp_out, n, sh_deg, st_dynamic, st_static,
                                         opacity, params, fallbacks, (cudaStream_t)stream));
}

size_t i4d_knn_workspace_size(int64_t n, int64_t table_slots) {
  if (n < 0 || table_slots < 1 || (table_slots & (table_slots - 1))) return 0;
  return knn_workspace_bytes(n, table_slots);
}

int32_t i4d_knn_features(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int64_t n,
                         float voxel, int32_t radius, const float* ref_center, float* features, float* knn3,
                         int64_t table_slots, int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || n >= (1ll << 32) - 1 || !(voxel > 0.0f) || radius < 0 || radius > 4 || !ref_center || !status ||
      table_slots < 1 || (table_slots & (table_slots - 1)))
    return I4D_ERR_ARG;
  if (n > 0 && (!xyz || !features || !ws)) return I4D_ERR_ARG;
  if (ws_bytes < knn_workspace_bytes(n, table_slots)) return I4D_ERR_WORKSPACE;
  return cuda_status(launch_knn_features(xyz, rgb, t, flag, n, voxel, radius, ref_center, features, knn3, table_slots,
                                         status, ws, (cudaStream_t)stream));
}

int32_t i4d_motion_targets(const i4d_gaussians* g, float* out, void* stream) {
  if (!g || g->n < 0 || g->sh_deg < 0 || g->sh_deg > 3 || g->mode < 0 || g->mode > 2) return I4D_ERR_ARG;
  if (g->n > 0 && (!g->params || !out || !aligned16(g->params))) return I4D_ERR_ARG;
  return cuda_status(launch_motion_targets(g->params, g->n, g->mode, out, (cudaStream_t)stream));
}

int64_t i4d_mlp_weight_count(void) { return mlp_weight_count(); }

int32_t i4d_mlp_forward(const float* features, int64_t n, const float* weights, float* out, void* stream) {
  if (n < 0 || (n > 0 && (!features || !weights || !out))) return I4D_ERR_ARG;
  return cuda_status(launch_mlp_forward(features, n, weights, out, (cudaStream_t)stream));
}

size_t i4d_mlp_grad_workspace_size(int64_t n) { return n < 0 ? 0 : mlp_grad_workspace_bytes(n); }

int32_t i4d_mlp_grad(const float* features, const float* targets, int64_t n, const float* weights, float w_st,
                     float w_v, float w_R, float* grads, float* loss_out, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || !weights || !grads || !ws) return I4D_ERR_ARG;
  if (n > 0 && (!features || !targets)) return I4D_ERR_ARG;
  if (ws_bytes < mlp_grad_workspace_bytes(n)) return I4D_ERR_WORKSPACE;
  return cuda_status(
      launch_mlp_grad(features, targets, n, weights, w_st, w_v, w_R, grads, loss_out, ws, (cudaStream_t)stream));
}

size_t i4d_prune_workspace_size(int64_t n_points, int64_t table_slots) {
  if (n_points < 0 || table_slots < 1 || (table_slots & (table_slots - 1))) return 0;
  return prune_workspace_bytes(n_points, table_slots);
}

static int32_t prune_common(const float* depth, const uint8_t* rgb8, const uint8_t* dyn, const i4d_camera* cams,
                            int32_t F, int32_t W, int32_t H, const float* xyz, const float* rgbf, const float* tpt,
                            int64_t n_points, float voxel_static, float voxel_dynamic, int32_t min_support,
                            int64_t table_slots, int64_t capacity, uint32_t* rep, int32_t* count, float* xyz_out,
                            float* rgb_out, float* t_out, uint8_t* flag, int64_t* n_kept, int32_t* status, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!(voxel_static > 0.0f) || !(voxel_dynamic >= 0.0f) || min_support < 1 || capacity < 1 || table_slots < 1 ||
      (table_slots & (table_slots - 1)) || table_slots >= (1ll << 32))
    return I4D_ERR_ARG;
  if (!rep || !count || !xyz_out || !rgb_out || !t_out || !flag || !n_kept || !status || !ws) return I4D_ERR_ARG;
  if (n_points >= (1ll << 32)) return I4D_ERR_ARG;
  if (ws_bytes < prune_workspace_bytes(n_points, table_slots)) return I4D_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  PruneOut out{rep, count, xyz_out, rgb_out, t_out, flag, n_kept, status};
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  // the voxel index is floor of x times the float32 reciprocal of the voxel size
  // voxel_dynamic = 0: dynamic points are not pruned (inv_d = 0 marks it for the kernels)
  const float inv_s = 1.0f / voxel_static, inv_d = voxel_dynamic > 0.0f ? 1.0f / voxel_dynamic : 0.0f;
  if (e == cudaSuccess)
    e = launch_prune(depth, rgb8, dyn, cams, F, W, H, xyz, rgbf, tpt, n_points, inv_s, inv_d, min_support,
                     table_slots, capacity, out, ws, st);
  return cuda_status(e);
}

int32_t i4d_prune_points(const float* depth, const uint8_t* rgb, const uint8_t* dyn, const i4d_camera* cams,
                         int32_t F, int32_t W, int32_t H, float voxel_static, float voxel_dynamic,
                         int32_t min_support, int64_t table_slots, int64_t capacity, uint32_t* rep, int32_t* count,
                         float* xyz, float* rgb_out, float* t_out, uint8_t* flag, int64_t* n_kept, int32_t* status,
                         void* ws, size_t ws_bytes, void* stream) {
  if (F < 0 || F > 65535 || W < 0 || H < 0 || !depth || !cams) return I4D_ERR_ARG;
  const int64_t np = (int64_t)F * W * H;
  return prune_common(depth, rgb, dyn, cams, F, W, H, nullptr, nullptr, nullptr, np, voxel_static, voxel_dynamic,
                      min_support, table_slots, capacity, rep, count, xyz, rgb_out, t_out, flag, n_kept, status, ws,
                      ws_bytes, stream);
}

int32_t i4d_prune_points_xyz(const float* xyz, const float* rgb, const float* t, const uint8_t* dyn,
                             int64_t n_points, float voxel_static, float voxel_dynamic, int32_t min_support,
                             int64_t table_slots, int64_t capacity, uint32_t* rep, int32_t* count, float* xyz_out,
                             float* rgb_out, float* t_out, uint8_t* flag, int64_t* n_kept, int32_t* status,
                             void* ws, size_t ws_bytes, void* stream) {
  if (n_points < 0 || (n_points > 0 && !xyz)) return I4D_ERR_ARG;
  return prune_common(nullptr, nullptr, dyn, nullptr, 0, 0, 0, xyz, rgb, t, n_points, voxel_static, voxel_dynamic,
                      min_support, table_slots, capacity, rep, count, xyz_out, rgb_out, t_out, flag, n_kept, status,
                      ws, ws_bytes, stream);
}

}  // extern "C"
