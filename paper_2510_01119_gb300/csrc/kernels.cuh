// Internal launchers of the sm_103a kernels (called by the C ABI in api.cu).
#pragma once

#include "i4d_common.cuh"
#include "profile.cuh"

namespace i4d {

// nt > 1: the SCH colour variant with nt - 1 temporal terms (its coefficients after the SH planes)
cudaError_t launch_slice_project(const float* params, int n, int sh_deg, int mode, const ViewTable& vt,
                                 const i4d_camera* cams, const Settings& S, float* proj, uint32_t* touched,
                                 cudaStream_t st, int nt = 0);
cudaError_t launch_slice_project_bwd(const float* params, int n, int sh_deg, int mode, const ViewTable& vt,
                                     const i4d_camera* cams, const Settings& S, const uint32_t* touched,
                                     const float* grad2d, float* grads, cudaStream_t st, int nt = 0);

// exclusive scan of n uint32 into out (may alias in); the total goes to *total (int64, device)
size_t scan_workspace_bytes(int64_t n);
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, int64_t* total, void* ws, cudaStream_t st);

// stable LSD radix sort of (key, value) pairs on bits [0, bits), 8 bits per pass; the count is
// min(*n_dev, capacity); the values of the last pass go to vals_out; with key_gather, the last pass
// writes key_gather[value] in place of each sorted key
size_t radix_workspace_bytes(int64_t capacity);
template <class K>
cudaError_t launch_radix_sort(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, uint32_t* vals_out,
                              int64_t capacity, const int64_t* n_dev, int bits, void* ws, K** keys_result,
                              cudaStream_t st, const uint32_t* key_gather = nullptr);

// tile binning (visible records sorted by depth, pairs emitted in that order, stable sort by tile)
size_t bin_workspace_bytes(int64_t VN, int64_t capacity);
cudaError_t launch_bin_tiles(const ViewTable& vt, int n, const float* proj, const uint32_t* touched,
                             int64_t capacity, uint32_t* ids, uint32_t* ranges, int64_t* n_inst, int32_t* status,
                             void* ws, cudaStream_t st);
cudaError_t launch_tile_ranges(const uint32_t* keys, const int64_t* n_dev, int64_t capacity, uint32_t* ranges,
                               int64_t total_tiles, int32_t* status, cudaStream_t st);

cudaError_t launch_render_fwd(const ViewTable& vt, int n, const float* proj, const uint32_t* ids,
                              const uint32_t* ranges, const Settings& S, int batch, float* img, float* T_final,
                              uint32_t* last, uint32_t* n_contrib, cudaStream_t st);
cudaError_t launch_render_bwd(const ViewTable& vt, int n, const float* proj, const uint32_t* ids,
                              const uint32_t* ranges, const Settings& S, const float* T_final, const uint32_t* last,
                              const float* dL_dimg, float* grad2d, cudaStream_t st);

cudaError_t launch_loss(const float* img, const float* target, int64_t count, int kind, float* dL_dimg,
                        float* loss_out, cudaStream_t st);
cudaError_t launch_psnr(const float* img, const float* target, int64_t count, float* psnr_out, cudaStream_t st);

// pruning inputs: adaptive voxel edge (Eq. 6) and Otsu motion masks
size_t adaptive_voxel_workspace_bytes(int F);
cudaError_t launch_adaptive_voxel(const float* depth, int F, int H, int W, const i4d_camera* cams, float lambda_s,
                                  float* out, void* ws, cudaStream_t st);
size_t motion_mask_workspace_bytes(int F);
cudaError_t launch_motion_masks(const float* prob, int F, int h, int w, int H, int W, uint8_t* mask, int32_t* thresh,
                                void* ws, cudaStream_t st);

// (1 - lambda) L1 + lambda (1 - SSIM) over all views, with its gradient
size_t photometric_workspace_bytes(const ViewTable& vt);
cudaError_t launch_photometric_loss(const ViewTable& vt, const float* img, const float* target, float lam,
                                    float* dL_dimg, float* loss_out, float* ssim_out, void* ws, cudaStream_t st);

struct AdamGroups {
  int n;
  int64_t begin[I4D_MAX_ADAM_GROUPS], end[I4D_MAX_ADAM_GROUPS];
  float lr0[I4D_MAX_ADAM_GROUPS][4], lr1[I4D_MAX_ADAM_GROUPS][4];
  int decay[I4D_MAX_ADAM_GROUPS];
};
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, const AdamGroups& groups,
                        int32_t* step, float b1, float b2, float eps, cudaStream_t st);

// grid pruning
size_t prune_workspace_bytes(int64_t n_points, int64_t table_slots);
struct PruneOut {
  uint32_t* rep;
  int32_t* count;
  float* xyz;
  float* rgb;
  float* t;
  uint8_t* flag;
  int64_t* n_kept;
  int32_t* status;
};
cudaError_t launch_prune(const float* depth, const uint8_t* rgb8, const uint8_t* dyn, const i4d_camera* cams, int F,
                         int W, int H, const float* xyz, const float* rgbf, const float* tpt, int64_t n_points,
                         float inv_static, float inv_dynamic, int min_support, int64_t table_slots, int64_t capacity,
                         const PruneOut& out, void* ws, cudaStream_t st);

cudaError_t launch_init_heuristic(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int n,
                                  int sh_deg, float spatial_scale, float st_dynamic, float st_static, float opacity,
                                  float* params, cudaStream_t st);

cudaError_t launch_init_learned(const float* xyz, const float* rgb, const float* t, const uint8_t* flag,
                                const float* spatial, const float* y, int n, int sh_deg, float st_dynamic,
                                float st_static, float opacity, float* params, int32_t* fallbacks, cudaStream_t st);

cudaError_t launch_motion_targets(const float* params, int n, int mode, float* out, cudaStream_t st);

// neighbourhood features and the learned-initialisation MLP
size_t knn_workspace_bytes(int64_t n, int64_t slots);
cudaError_t launch_knn_features(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int64_t n,
                                float voxel, int radius, const float* ref, float* feat, float* knn3, int64_t slots,
                                int32_t* status, void* ws, cudaStream_t st);
int64_t mlp_weight_count();
size_t mlp_grad_workspace_bytes(int64_t n);
cudaError_t launch_mlp_forward(const float* feat, int64_t n, const float* w, float* out, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* feat, const float* tgt, int64_t n, const float* w, float w_st, float w_v,
                            float w_R, float* grads, float* loss, void* ws, cudaStream_t st);

}  // namespace i4d
