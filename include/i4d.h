/*
 * i4d.h -- C ABI of the GB300 (sm_103a) 4D-Gaussian rasterizer of Instant4D (arXiv 2510.01119).
 *
 * The library (libi4d.so) runs the data-parallel hot path of the method's optimisation step:
 * slicing of native 4D Gaussians at the frame time, EWA projection, tile binning with a device
 * radix sort, front-to-back compositing, the analytic backward, a fused Adam update, the
 * photometric loss, and the voxel-grid pruning of the back-projected depth point cloud.
 *
 * Conventions for every entry point
 *   - Tensor arguments are DEVICE pointers owned by the caller, unless a comment says "host".
 *     The library never allocates device memory: calls that need scratch take a workspace
 *     pointer and size, with a *_workspace_size() query beside them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only enqueue work: none
 *     synchronises with the host, so a sequence of calls can be captured into a CUDA graph.
 *     Counts that the device computes (instances, kept voxels) stay in device memory and the
 *     kernels that consume them read them there.
 *   - Return value: I4D_OK, or a negative I4D_ERR_* code for argument errors detected on the
 *     host and for launch failures.  Conditions only the device can see (capacity overflow)
 *     are reported through a device status word that the caller reads after the stream work.
 *   - No call aborts, traps or spins without a bound.
 *
 * Data layouts
 *   Gaussian parameters are ONE flat float32 buffer of (5 + K) planes of N float4 each, where
 *   K = 0, 3, 6, 12 for SH degree 0..3 (plane p holds floats [4 N p, 4 N (p + 1))):
 *     plane 0  mean4      (x, y, z, t)                         Sec. 3.3: 4D mean
 *     plane 1  logscale4  (log s_x, log s_y, log s_z, log s_t) Sec. 3.3: diagonal 4D scale
 *     plane 2  q_l        (a, b, c, d) = a + bi + cj + dk      Sec. 3.3: 4x4 rotation R = L(q_l) R(q_r)
 *     plane 3  q_r                                             (two-quaternion form of 4DGS, Sec. 3.1)
 *     plane 4  (opacity logit, r, g, b)                        Sec. 3.3: opacity and RGB colour
 *     plane 5+ SH coefficients of degree 1..deg, coefficient k channel c at float 3k + c of the
 *              Gaussian's SH group, i.e. plane 5 + (3k + c) / 4, lane (3k + c) % 4.
 *   A 4-vector (x, y, z, t) is the quaternion t + xi + yj + zk; R v = q_l v q_r (normalised q).
 *   Gradients use the same flat layout.
 *   Projected records: V x N records of 64 bytes (view-major), each 4 float4: (xmin, xmax, ymin,
 *   ymax) the blendable box: the pixel-space box of the ellipse q <= q_b, with q_b = min(q_max,
 *   max(2 ln(o_t / alpha_min), 0) + 1e-3) the largest q at which alpha = o_t exp(-q/2) can reach
 *   alpha_min, widened by 1% + 0.01 px (empty (1, 0, 1, 0) when culled); (u, v, k conic_a,
 *   2 k conic_b); (k conic_c, o_t, m_thr, r); (g, b, depth, radius), with k = -log2(e) / 2 so that
 *   exp(-q/2) = 2^(k q), and m_thr = k min(q_max, 2 ln(o_t / alpha_min)) (a fragment is kept where
 *   k q >= m_thr).  The compositing kernels stage a record as it is: one 64-byte segment.
 *   2D gradients (scratch of the backward): 3 planes of V x N float4: (du, dv, dconic_a,
 *   dconic_b), (dconic_c, do_t, dr, dg), (db, 0, 0, 0).
 *   Images: per view, planar float32 [3][H][W]; views concatenated in order.  Per-pixel
 *   buffers (T_final, last, n_contrib): per view [H][W], concatenated.
 */
#ifndef I4D_H
#define I4D_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define I4D_API __attribute__((visibility("default")))
#else
#define I4D_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define I4D_VERSION 1

#define I4D_OK 0
#define I4D_ERR_ARG (-1)       /* invalid argument (null pointer, size, alignment, mode) */
#define I4D_ERR_CAPACITY (-2)  /* an output did not fit its capacity (device status word) */
#define I4D_ERR_CUDA (-3)      /* a CUDA launch or runtime call failed */
#define I4D_ERR_WORKSPACE (-4) /* workspace smaller than *_workspace_size() */

#define I4D_MAX_VIEWS 64
#define I4D_PROJ_FLOATS 16     /* floats per projected record (one 64-byte record) */
#define I4D_GRAD2D_FLOATS 9    /* floats per (view, Gaussian) 2D-gradient record: two float4 planes and one
                                  float plane, each n_views * n long */

enum { I4D_MODE_FULL = 0, I4D_MODE_ISO_ROT = 1, I4D_MODE_ISO_IDENTITY = 2 };
enum { I4D_LOSS_L1 = 0, I4D_LOSS_MSE = 1 };

/* One view's camera (DEVICE array of V entries, 80 bytes each).  World->camera pose (R, t) with
 * OpenCV axes (x right, y down, z forward); pixel centres at (px + 0.5, py + 0.5); time is the
 * frame time in the scene's normalised time axis. */
typedef struct {
  float R[9];   /* row-major */
  float t[3];
  float fx, fy, cx, cy;
  float time;
  float pad[3];
} i4d_camera;

/* Host description of a batch of views rendered in one launch. */
typedef struct {
  int32_t n_views;                   /* 1..I4D_MAX_VIEWS */
  int32_t tile_w, tile_h;            /* screen tile; supported: 16x16, 8x8, 16x8, 32x8, 32x16 */
  int32_t width[I4D_MAX_VIEWS];
  int32_t height[I4D_MAX_VIEWS];
} i4d_views;

/* Host struct naming the Gaussian parameters. */
typedef struct {
  const float* params;  /* DEVICE, flat layout above, 16-byte aligned */
  int32_t n;            /* number of Gaussians */
  int32_t sh_deg;       /* 0..3 */
  int32_t mode;         /* I4D_MODE_* (Sec. 3.3 "Isotropic Gaussian": ISO modes tie s_x = s_y = s_z
                           to logscale.x; ISO_IDENTITY also fixes R = I) */
  int32_t sch_terms;    /* 0 or 1: the colour of the method (base RGB + SH).  N_t in 2..I4D_MAX_SCH_TERMS:
                           the SCH appearance of the 4DGS it compares against (Sec. 3.1, Table 2 "SCH"):
                           colour += sum_{m=1}^{N_t-1} cos(2 pi m t) (c_m0 + sum_{k>=1} Y_k c_mk), t the
                           view's frame time (period = the normalised video length 1), Y_k the real SH of
                           the Gaussians' SH degree; the (N_t - 1)(deg + 1)^2 x 3 coefficients follow the
                           SH planes, coefficient (m, k, ch) at float (m - 1)(deg + 1)^2 3 + 3 k + ch of the
                           Gaussian's SCH block (plane = float / 4, lane = float % 4) */
} i4d_gaussians;

#define I4D_MAX_SCH_TERMS 8

/* Thresholds of the renderer (host).  The paper leaves them to the 3D splatting renderer it
 * builds on; i4d_default_settings() gives alpha_max 0.99, alpha_min 1/255, T_min 1e-4,
 * q_max 9 (3-sigma ellipse), ot_min 1/255 (temporal cull, Sec. 3.3), z_near 0.2,
 * dilation 0.3 px^2, fov_clamp 1.3. */
typedef struct {
  float alpha_max, alpha_min, T_min, q_max, ot_min, z_near, dilation, fov_clamp;
  float bg[3];          /* background colour composited behind the last fragment */
  float pad;
} i4d_settings;

/* Launch tuning of i4d_render_fwd (host); zeros select defaults.  The image does not depend on it. */
typedef struct {
  int32_t batch;        /* tile-list entries each warp tests and stages in shared memory per round:
                           16, 32 or 64 (0 = 32); any other value is rejected with I4D_ERR_ARG */
  int32_t reserved[7];
} i4d_tune;

/* One Adam parameter group: floats [begin, end) of the flat buffer; lane = index % 4 selects
 * lr_init/lr_final; the learning rate decays log-linearly from lr_init to lr_final over
 * decay_steps updates (constant if decay_steps <= 0). */
typedef struct {
  int64_t begin, end;
  float lr_init[4];
  float lr_final[4];
  int32_t decay_steps;
  int32_t pad;
} i4d_adam_group;

#define I4D_MAX_ADAM_GROUPS 16

I4D_API int32_t i4d_version(void);
I4D_API const char* i4d_status_string(int32_t status);
I4D_API void i4d_default_settings(i4d_settings* out /* host */);
/* Floats per Gaussian in the flat parameter layout: 20 + 4 K. */
I4D_API int64_t i4d_param_floats(int32_t sh_deg);
/* The same with the SCH variant's coefficients (sch_terms as in i4d_gaussians). */
I4D_API int64_t i4d_param_floats_sch(int32_t sh_deg, int32_t sch_terms);

/*
 * i4d_slice_project -- Eq. 7-8 (conditional mean mu_xyz|t and covariance Sigma_xyz|t of each 4D
 * Gaussian at each view's frame time), the temporal marginal opacity o_t = sigmoid(o) N(t; mu_t,
 * Sigma_44) with its cull below settings.ot_min (Sec. 3.3, Eq. 9), EWA projection to 2D, colour
 * (base RGB + real SH of degree 1..3 of the view direction), the blendable box and the tile
 * rectangle: the tiles [floor((xmin + 0.5) / tile_w), floor((xmax - 0.5) / tile_w) + 1) x (same in
 * y) that hold a pixel centre of the box, clipped to the view.  Every pixel where the Gaussian can
 * be blended lies in it, so the image equals that of the 3-sigma square of 3D splatting.
 *   g        host struct, params on the device
 *   views    host; cams: DEVICE array of views->n_views cameras
 *   settings host (NULL = defaults)
 *   proj     DEVICE out, n_views * n * I4D_PROJ_FLOATS floats in the 64-byte record layout; a
 *            record whose touched count is 0 is not written (its previous contents stay)
 *   touched  DEVICE out, n_views * n uint32: number of tiles of the record's rectangle
 *            (0 for culled or off-screen Gaussians)
 */
I4D_API int32_t i4d_slice_project(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                          const i4d_settings* settings, float* proj, uint32_t* touched, void* stream);

/*
 * i4d_bin_tiles -- the tile binning of the 3D splatting renderer (Sec. 3.1): every (tile,
 * Gaussian) pair of the touched rectangles gets key ((view tile offset + tile) << 32 | depth
 * bits), a stable LSD radix sort orders the pairs by (tile, depth, Gaussian id), and each tile's
 * [start, end) range in the sorted list is found.
 *   proj, touched  DEVICE in (from i4d_slice_project)
 *   capacity       size of ids (and of the key arrays in the workspace)
 *   ids            DEVICE out, capacity uint32: Gaussian id of each sorted pair
 *   ranges         DEVICE out, 3 * total_tiles uint32: [start, end) per tile (all views), then the
 *                  tile indices ordered by decreasing octave of list length, floor(log2(length +
 *                  1)), and by tile index within an octave (the order in which the compositing
 *                  kernels take tiles: the longest start first, and neighbouring tiles run
 *                  together so that they share the records they read in L2)
 *   n_inst         DEVICE out, 1 int64: number of pairs (may exceed capacity)
 *   status         DEVICE out, 1 int32: I4D_OK, or I4D_ERR_CAPACITY when n_inst > capacity
 *                  (the sorted output is then invalid; retry with capacity >= n_inst)
 *   ws, ws_bytes   DEVICE workspace, at least i4d_bin_tiles_workspace_size(views, n, capacity)
 */
I4D_API size_t i4d_bin_tiles_workspace_size(const i4d_views* views, int32_t n, int64_t capacity);
I4D_API int32_t i4d_bin_tiles(const i4d_views* views, int32_t n, const float* proj, const uint32_t* touched,
                      int64_t capacity, uint32_t* ids, uint32_t* ranges, int64_t* n_inst, int32_t* status,
                      void* ws, size_t ws_bytes, void* stream);
I4D_API int64_t i4d_total_tiles(const i4d_views* views);
I4D_API int64_t i4d_total_pixels(const i4d_views* views);

/*
 * i4d_render_fwd -- front-to-back alpha compositing (the 3D splatting renderer, Sec. 3.1, Eq. 3)
 * of every view in ONE launch: a Gaussian covers a pixel centre p when q = (p-uv)^T conic (p-uv)
 * <= q_max; alpha = min(alpha_max, o_t exp(-q/2)); fragments below alpha_min are skipped; the walk
 * ends before the fragment that would take T below T_min; C = sum T alpha rgb + T_final bg.
 *   img       DEVICE out, total_pixels * 3 floats (per view planar [3][H][W])
 *   T_final   DEVICE out, total_pixels floats
 *   last      DEVICE out, total_pixels uint32: the position (within the tile's range) where the
 *             pixel's walk ended -- the fragment that would have taken T below T_min, or the list
 *             length; the pixel blended exactly its kept fragments before it (the backward resumes
 *             from here)
 *   n_contrib DEVICE out, total_pixels uint32: fragments blended; NULL skips the count
 *   tune      host, nullable: i4d_tune.batch (I4D_ERR_ARG for an unsupported value)
 */
I4D_API int32_t i4d_render_fwd(const i4d_views* views, int32_t n, const float* proj, const uint32_t* ids,
                       const uint32_t* ranges, const i4d_settings* settings, const i4d_tune* tune, float* img,
                       float* T_final, uint32_t* last, uint32_t* n_contrib, void* stream);

/*
 * i4d_render_bwd -- analytic backward of i4d_render_fwd and i4d_slice_project: back-to-front
 * per pixel (transmittance recomputed from T_final, no per-fragment state), per-Gaussian 2D
 * gradients reduced over each warp before the atomics, then the chain through projection,
 * Eq. 7-8 slicing, the temporal opacity and the 4D parameterisation.
 *   dL_dimg  DEVICE in, same layout as img
 *   grad2d   DEVICE scratch, n_views * n * I4D_GRAD2D_FLOATS floats (contents undefined after)
 *   grads    DEVICE out, flat parameter layout (overwritten; views summed)
 */
I4D_API int32_t i4d_render_bwd(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                       const i4d_settings* settings, const float* proj, const uint32_t* touched,
                       const uint32_t* ids, const uint32_t* ranges, const float* T_final, const uint32_t* last,
                       const float* dL_dimg, float* grad2d, float* grads, void* stream);

/*
 * i4d_render_bwd_noalloc -- i4d_render_bwd for callers that may not allocate device memory when they
 * run the backward (a C/C++ host whose device heap belongs to its own memory manager, or a real-time
 * loop that must not stall on cudaMalloc).  The paper has no counterpart: this is a deployment
 * variant of the same computation.  The 2D-gradient scratch is a fixed array inside the library
 * (i4d_render_bwd_noalloc_max_records() records of 36 bytes, 18 MiB, held by every GPU that loads
 * the library until exit) instead of the grad2d argument; all other arguments are as for
 * i4d_render_bwd.  Returns I4D_ERR_CAPACITY, launching nothing, when n_views * n exceeds the maximum.
 * Every call shares the array: calls that overlap on the GPU race.  Each call looks up the array's
 * address with the caller's device current, except while `stream` is being captured, when the address
 * of the device's last uncaptured call is used: make the first call on a device before any stream
 * capture (a captured first call returns I4D_ERR_CUDA).
 */
I4D_API int64_t i4d_render_bwd_noalloc_max_records(void);
I4D_API int32_t i4d_render_bwd_noalloc(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                                       const i4d_settings* settings, const float* proj, const uint32_t* touched,
                                       const uint32_t* ids, const uint32_t* ranges, const float* T_final,
                                       const uint32_t* last, const float* dL_dimg, float* grads, void* stream);

/*
 * i4d_loss -- the single photometric loss of the method (supplementary "Discussion with previous
 * work": one photometric term; Sec. 4.1: the standard 3DGS loss), L1 or MSE over every pixel and
 * channel of all views, mean-reduced; writes dL/dimg and the loss value.
 *   loss_out DEVICE out, 1 float.  target: same layout as img.
 */
I4D_API int32_t i4d_loss(const float* img, const float* target, int64_t count, int32_t kind, float* dL_dimg,
                 float* loss_out, void* stream);

/*
 * i4d_photometric_loss -- the training loss with the loss weights of standard 3D Gaussian splatting
 * that Sec. 4.1 adopts: (1 - lambda_dssim) L1 + lambda_dssim (1 - SSIM), lambda_dssim = 0.2 there.
 * L1 is the mean absolute error over every pixel and channel of all views; SSIM is computed per
 * channel with an 11x11 Gaussian window (sigma 1.5, weights summing to 1) centred on every pixel,
 * zeros outside the image, C1 = 0.01^2, C2 = 0.03^2, and averaged over every pixel and channel of
 * all views (the SSIM of Tables 1-4, per view, when the batch holds one view).
 *   views     host; img, target DEVICE, the planar multi-view image layout
 *   dL_dimg   DEVICE out, same layout: the gradient of the loss (overwritten, not accumulated)
 *   loss_out  DEVICE out, 1 float; ssim_out DEVICE out, 1 float (nullable): the mean SSIM
 *   ws        DEVICE scratch of i4d_photometric_loss_workspace_size(views) bytes (9 floats per pixel)
 * Errors: I4D_ERR_ARG (bad views, lambda outside [0, 1], NULL pointers), I4D_ERR_WORKSPACE.
 */
I4D_API size_t i4d_photometric_loss_workspace_size(const i4d_views* views);
I4D_API int32_t i4d_photometric_loss(const i4d_views* views, const float* img, const float* target,
                                     float lambda_dssim, float* dL_dimg, float* loss_out, float* ssim_out, void* ws,
                                     size_t ws_bytes, void* stream);

/* i4d_psnr -- 10 log10(1 / MSE) over count floats in [0, 1] (the PSNR of Tables 1-4). */
I4D_API int32_t i4d_psnr(const float* img, const float* target, int64_t count, float* psnr_out, void* stream);

/*
 * i4d_adam_step -- fused Adam update over the flat buffer (Sec. 4.1: standard 3DGS optimiser
 * settings with per-group learning rates, position learning rate 1e-5, decayed over the run).
 * Reads the update number from *step (DEVICE int32, the count of updates already done), uses
 * step + 1 for the bias correction and the schedule, and increments *step, so a captured graph
 * replays correctly.  groups: host array of n_groups (<= I4D_MAX_ADAM_GROUPS).
 */
I4D_API int32_t i4d_adam_step(float* params, const float* grads, float* m, float* v, int64_t count,
                      const i4d_adam_group* groups, int32_t n_groups, int32_t* step, float beta1, float beta2,
                      float eps, void* stream);

/*
 * i4d_prune_points -- Eq. 5 back-projection of F depth maps (pixel centre, z-depth, camera-space
 * D K^-1 p, world R^T (X_c - t)) fused with the voxel-grid pruning of Sec. 3.2: voxel index =
 * floor(float32(x * (1 / S_v))) per axis, the dynamic flag is part of the key (static and dynamic
 * points never share a voxel, each flag with its own S_v), aggregation in a device hash table
 * (count, sums in 64-bit fixed point, minimum point index), voxels with fewer than min_support
 * points dropped, output ordered by representative (minimum) point index.  voxel_dynamic = 0
 * leaves the dynamic points unpruned (the Full model of Sec. 4.1): each is kept as its own voxel
 * whatever min_support (the table then needs a slot per dynamic point).  The Lite model is
 * voxel_static = voxel_dynamic = 4 units of Eq. 6 (see i4d_adaptive_voxel).
 *   depth    DEVICE F*H*W float32;  rgb: DEVICE F*H*W*3 uint8 or NULL;  dyn: F*H*W uint8 or NULL
 *   cams     DEVICE F cameras (time = frame time)
 *   outputs  DEVICE, capacity entries each: rep (uint32 point index f*H*W + py*W + px),
 *            count (int32), xyz (float32 x3 centroid), rgb_out (float32 x3 mean colour in [0,1]),
 *            t_out (float32 mean time), flag (uint8)
 *   n_kept   DEVICE out, 1 int64;  status: DEVICE out, 1 int32 (I4D_ERR_CAPACITY when the table or
 *            the output overflowed)
 */
I4D_API size_t i4d_prune_workspace_size(int64_t n_points, int64_t table_slots);
I4D_API int32_t i4d_prune_points(const float* depth, const uint8_t* rgb, const uint8_t* dyn, const i4d_camera* cams,
                         int32_t F, int32_t W, int32_t H, float voxel_static, float voxel_dynamic,
                         int32_t min_support, int64_t table_slots, int64_t capacity, uint32_t* rep, int32_t* count,
                         float* xyz, float* rgb_out, float* t_out, uint8_t* flag, int64_t* n_kept, int32_t* status,
                         void* ws, size_t ws_bytes, void* stream);
/*
 * i4d_adaptive_voxel -- Eq. 6: S_v = lambda_s * (1/F) sum_i D_i / f_i, D_i the mean depth of frame i
 * over its pixels with positive depth, f_i = cams[i].fx.  Per-frame depth sums are exact (64-bit
 * fixed point in 2^-32 units; depths are multiples of 2^-32 from 2^-9 up), the rest is float64 in
 * frame order, so the result does not depend on the launch.
 *   depth DEVICE F*H*W float32;  cams DEVICE F cameras;  voxel_out DEVICE 1 float
 *   ws    DEVICE scratch of i4d_adaptive_voxel_workspace_size(F) bytes
 * Errors: I4D_ERR_ARG (sizes < 1, NULL pointers, lambda_s <= 0), I4D_ERR_WORKSPACE.
 */
I4D_API size_t i4d_adaptive_voxel_workspace_size(int32_t F);
I4D_API int32_t i4d_adaptive_voxel(const float* depth, int32_t F, int32_t W, int32_t H, const i4d_camera* cams,
                                   float lambda_s, float* voxel_out, void* ws, size_t ws_bytes, void* stream);

/*
 * i4d_motion_masks -- the static / dynamic split of Sec. 3.2 ("Motion Probability Estimation"):
 * each frame's low-resolution motion-probability map (h x w, values in [0, 1]) is upsampled
 * bilinearly to W x H (source coordinate (x + 0.5) w / W - 0.5 clamped to the map, every step a
 * float32 operation), binned into 256 bins (bin = min(255, floor(256 p))), and Otsu's threshold t of
 * the frame's histogram (the bin maximising the between-class variance, first maximum on ties) splits
 * it: mask = 1 (dynamic) where bin > t.  The result feeds i4d_prune_points' dyn input.
 *   prob        DEVICE F*h*w float32;  mask DEVICE out F*H*W uint8
 *   thresholds  DEVICE out F int32 (nullable): the per-frame threshold bins
 *   ws          DEVICE scratch of i4d_motion_masks_workspace_size(F) bytes
 * Errors: I4D_ERR_ARG (sizes, NULL pointers), I4D_ERR_WORKSPACE.
 */
I4D_API size_t i4d_motion_masks_workspace_size(int32_t F);
I4D_API int32_t i4d_motion_masks(const float* prob, int32_t F, int32_t w, int32_t h, int32_t W, int32_t H,
                                 uint8_t* mask, int32_t* thresholds, void* ws, size_t ws_bytes, void* stream);

/* Same pruning on a ready float32 point cloud (xyz n x 3; rgb n x 3 float or NULL; t, dyn or NULL). */
I4D_API int32_t i4d_prune_points_xyz(const float* xyz, const float* rgb, const float* t, const uint8_t* dyn,
                             int64_t n_points, float voxel_static, float voxel_dynamic, int32_t min_support,
                             int64_t table_slots, int64_t capacity, uint32_t* rep, int32_t* count, float* xyz_out,
                             float* rgb_out, float* t_out, uint8_t* flag, int64_t* n_kept, int32_t* status,
                             void* ws, size_t ws_bytes, void* stream);

/*
 * i4d_init_heuristic -- 4D Gaussians from the pruned voxels (Sec. 4.1 and Sec. 3.3
 * "Motion-Aware Gaussian"): mean4 = (centroid, mean frame time); log-scales (log spatial_scale x3,
 * log s_t) with s_t = st_dynamic for dynamic voxels (two frames, 2/fps in the paper) and
 * st_static for static ones (the video length); q_l = q_r = 1 (R = I); opacity logit of
 * `opacity`; base colour = mean colour; SH coefficients zero.
 *   xyz (n x 3), rgb (n x 3, NULL = grey), t (n, NULL = 0.5), flag (n, NULL = static): DEVICE in
 *   params: DEVICE out, flat layout for sh_deg
 */
I4D_API int32_t i4d_init_heuristic(const float* xyz, const float* rgb, const float* t, const uint8_t* flag,
                                   int32_t n, int32_t sh_deg, float spatial_scale, float st_dynamic,
                                   float st_static, float opacity, float* params, void* stream);

/*
 * Learned initialisation (not in the paper: an addition that proposes the temporal scale, motion
 * and 4D rotation the paper sets by a heuristic in Sec. 4.1 / Sec. 3.3 "Motion-Aware Gaussian").
 *
 * i4d_knn_features -- per pruned point, the 16 nearest other points whose voxel cells lie within
 * +-radius cells on every axis, ordered by (squared distance, index), as features of 64 floats:
 * offsets / voxel (48, zeros for missing slots), distance to ref_center (host float[3]), colour (3),
 * time, neighbours found / 16, dynamic flag, the neighbourhood's least-squares velocity
 * sum dt o / (sum dt^2 + 1e-6) / 16 (3; dt = neighbour time - point time, o = offset in voxels), the
 * RMS of dt, zeros; knn3 (nullable): mean distance to the 3 nearest
 * (voxel when fewer exist).  xyz (n x 3), rgb (n x 3, NULL = 0), t, flag: DEVICE; features n x 64.
 * table_slots: power of two >= 2 n; status: I4D_ERR_CAPACITY if the table overflowed.
 */
I4D_API size_t i4d_knn_workspace_size(int64_t n, int64_t table_slots);
I4D_API int32_t i4d_knn_features(const float* xyz, const float* rgb, const float* t, const uint8_t* flag, int64_t n,
                                 float voxel, int32_t radius, const float* ref_center, float* features, float* knn3,
                                 int64_t table_slots, int32_t* status, void* ws, size_t ws_bytes, void* stream);
/*
 * MLP 64 -> 64 -> 64 -> 12, GELU (exact normal CDF), bfloat16 operands, float32 accumulation (tensor
 * cores in the forward).  weights: DEVICE float32, packed [W1 64x64 | b1 | W2 64x64 | b2 | W3 12x64 | b3]
 * (rows = outputs), i4d_mlp_weight_count() floats.  Outputs per point: log s_t, velocity (3), q_l, q_r.
 * i4d_mlp_grad: gradient of the mean loss w_st (log s_t - t0)^2 + w_v |v - t1:4|^2 + w_R ||R(q_l, q_r) -
 * t4:20||_F^2 over n points (targets n x 20: log s_t, velocity, R row-major) -> grads (overwritten),
 * loss_out (DEVICE float, nullable).
 */
/* i4d_motion_targets -- per Gaussian (log s_t, velocity b/c of Eq. 7, R row-major): n x 20 floats,
 * the training targets of the MLP when taken from Gaussians fitted by the plain method. */
I4D_API int32_t i4d_motion_targets(const i4d_gaussians* g, float* out, void* stream);
I4D_API int64_t i4d_mlp_weight_count(void);
I4D_API int32_t i4d_mlp_forward(const float* features, int64_t n, const float* weights, float* out, void* stream);
I4D_API size_t i4d_mlp_grad_workspace_size(int64_t n);
I4D_API int32_t i4d_mlp_grad(const float* features, const float* targets, int64_t n, const float* weights, float w_st,
                             float w_v, float w_R, float* grads, float* loss_out, void* ws, size_t ws_bytes,
                             void* stream);
/*
 * i4d_init_learned -- 4D Gaussians from the pruned voxels with per-point spatial scale `spatial`
 * (e.g. knn3), and temporal log-scale and quaternions from mlp_out (n x 12); points whose proposal is
 * not finite or degenerate fall back to the heuristic of i4d_init_heuristic (count in *fallbacks).
 * mlp_out NULL: the heuristic for every point (with the per-point spatial scale).
 */
I4D_API int32_t i4d_init_learned(const float* xyz, const float* rgb, const float* t, const uint8_t* flag,
                                 const float* spatial, const float* mlp_out, int32_t n, int32_t sh_deg,
                                 float st_dynamic, float st_static, float opacity, float* params, int32_t* fallbacks,
                                 void* stream);

/*
 * Kernel timing (host-side tracing): when enabled, every kernel the library launches is bracketed
 * by two CUDA events recorded on its stream; i4d_profile_read() waits for them and returns, per
 * kernel name, the summed device time and the launch count.  Off by default; costs two event
 * records per launch when on.  Not for use during CUDA-graph capture.
 */
I4D_API int32_t i4d_profile_enable(int32_t on);
I4D_API void i4d_profile_reset(void);
I4D_API int32_t i4d_profile_count(void);
I4D_API int32_t i4d_profile_read(int32_t k, char* name, int32_t name_len, double* total_ms, int64_t* launches);

/*
 * i4d_measure_fp32_peak -- the FP32 roofline's denominator, measured: a kernel of packed FP32x2
 * FMA chains (8 independent chains per thread, 256 threads per block, blocks_per_sm blocks per SM,
 * iters iterations) is timed with CUDA events on `stream`; *tflops = FLOPs (an FMA counts 2) per
 * second / 1e12.  Synchronises the stream.  The paper has no counterpart: it is the measured peak
 * that the compositing kernels' FP32 roofline divides by.  Errors: I4D_ERR_ARG (tflops NULL,
 * blocks_per_sm outside 1..64, iters < 1), I4D_ERR_CUDA.
 */
I4D_API int32_t i4d_measure_fp32_peak(int32_t blocks_per_sm, int32_t iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* I4D_H */
