/*
 * FP64 CPU oracle for the Instant4D 4D-Gaussian rasterizer (test infrastructure only).
 *
 * This file is the plain, slow, obviously-correct statement of what the GPU path computes.
 * Only tests, the smoke check and the bench's CPU-baseline leg load it; the product path never
 * does.  It shares no code, header or constant table with the CUDA library.
 *
 * What is computed, and where the paper defines it (Instant4D, arXiv 2510.01119):
 *   - 4D Gaussian primitive: 4D mean, diagonal 4D scale, opacity, 4x4 rotation (Sec. 3.3,
 *     "Motion Modeling").  The rotation is written as v -> q_l (x) v (x) q_r on quaternions
 *     (the two-quaternion form of the cited 4DGS work, Sec. 3.1).
 *   - Slicing at frame time t: conditional mean and covariance by Schur complement (Eq. 7-8).
 *   - Temporal marginal opacity o_t = o * N(t; mu_4, Sigma_44), unnormalised, and culling of
 *     Gaussians whose o_t falls below a threshold (Sec. 3.3, "Motion-Aware Gaussian", Eq. 9).
 *   - Isotropic variant with R = I and one shared spatial scale (Sec. 3.3, "Isotropic Gaussian").
 *   - EWA projection, per-pixel depth-sorted front-to-back alpha compositing and the analytic
 *     backward: the 3D Gaussian splatting renderer the paper builds on (Sec. 3.1, Eq. 3).
 *   - Back-projection of depth maps (Eq. 5), in float64 and as a fixed sequence of correctly
 *     rounded float32 operations, and voxel-grid pruning: points are assigned to voxels by
 *     division with S_v, aggregated per voxel into a centroid with averaged attributes, and
 *     voxels with too little support are dropped (Sec. 3.2, "Grid Pruning").
 *   - The tile lists of the binning step: the tiles that hold a pixel centre where a Gaussian can
 *     be blended, in (depth, id) order.
 *   - Every valid colour of a pixel whose threshold, T-stop or depth-order decisions sit within a
 *     margin of going the other way (the results a float32 pipeline may legitimately produce).
 *
 * Readings where the paper is silent (thresholds, pixel-centre convention, tie order, ...)
 * are the constants passed in `settings` and the conventions documented at each function.
 *
 * Layouts: all arrays are plain row-major float64 (or float32 where the input is a float32
 * point cloud).  Quaternions are (a, b, c, d) = a + b i + c j + d k.  A 4-vector (x, y, z, t)
 * is the quaternion t + x i + y j + z k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { MODE_FULL = 0, MODE_ISO_ROT = 1, MODE_ISO_IDENTITY = 2 };

/* settings[] indices */
enum { S_ALPHA_MAX = 0, S_ALPHA_MIN, S_T_MIN, S_Q_MAX, S_OT_MIN, S_Z_NEAR, S_DILATION, S_FOV_CLAMP, S_COUNT };

/* camera[] indices: world->camera rotation W (row-major 3x3), translation tau, intrinsics, size, time */
enum { C_R = 0, C_T = 9, C_FX = 12, C_FY, C_CX, C_CY, C_W, C_H, C_TIME, C_COUNT };

/* projected record columns */
enum {
  P_VISIBLE = 0, P_U, P_V, P_DEPTH, P_OT, P_CA, P_CB, P_CC, P_RADIUS, P_R, P_G, P_B,
  P_MARGIN, P_RADIUS_MARGIN,
  P_M3X, P_M3Y, P_M3Z, P_S3XX, P_S3XY, P_S3XZ, P_S3YY, P_S3YZ, P_S3ZZ, P_STRIDE
};

int orc_proj_stride(void) { return P_STRIDE; }

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Quaternion algebra                                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Hamilton product r = p q */
static void qmul(const double p[4], const double q[4], double r[4]) {
  r[0] = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
  r[1] = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
  r[2] = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
  r[3] = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
}

/* 4-vector (x,y,z,t) <-> quaternion t + x i + y j + z k */
static void vec_to_quat(const double v[4], double q[4]) { q[0] = v[3]; q[1] = v[0]; q[2] = v[1]; q[3] = v[2]; }
static void quat_to_vec(const double q[4], double v[4]) { v[0] = q[1]; v[1] = q[2]; v[2] = q[3]; v[3] = q[0]; }

/* y = ql (x) x (x) qr, on 4-vectors */
static void rot4_apply(const double ql[4], const double qr[4], const double x[4], double y[4]) {
  double xq[4], tmp[4], out[4];
  vec_to_quat(x, xq);
  qmul(ql, xq, tmp);
  qmul(tmp, qr, out);
  quat_to_vec(out, y);
}

/* R[:,k] = image of the k-th basis 4-vector */
static void rot4_matrix(const double ql[4], const double qr[4], double R[4][4]) {
  for (int k = 0; k < 4; ++k) {
    double e[4] = {0, 0, 0, 0}, col[4];
    e[k] = 1.0;
    rot4_apply(ql, qr, e, col);
    for (int i = 0; i < 4; ++i) R[i][k] = col[i];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Real orthonormal spherical harmonics of degree 1..3 (textbook real form, no Condon-Shortley */
/* phase), evaluated on a unit direction; index k = l*l + l + m - 1 for l >= 1.                */
/* The zero-degree term is the stored base colour itself (Sec. 3.3: plain RGB appearance).    */
/* ------------------------------------------------------------------------------------------ */
static void sh_eval(const double d[3], double Y[15], double dY[15][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k20 = 0.25 * sqrt(5.0 / PI);
  const double k22 = 0.25 * sqrt(15.0 / PI);
  const double k33 = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k32 = 0.5 * sqrt(105.0 / PI);
  const double k31 = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k30 = 0.25 * sqrt(7.0 / PI);
  const double k322 = 0.25 * sqrt(105.0 / PI);
  memset(dY, 0, sizeof(double) * 45);
  /* l = 1 */
  Y[0] = k1 * y;             dY[0][1] = k1;
  Y[1] = k1 * z;             dY[1][2] = k1;
  Y[2] = k1 * x;             dY[2][0] = k1;
  /* l = 2 */
  Y[3] = k2a * x * y;        dY[3][0] = k2a * y; dY[3][1] = k2a * x;
  Y[4] = k2a * y * z;        dY[4][1] = k2a * z; dY[4][2] = k2a * y;
  Y[5] = k20 * (3.0 * z * z - 1.0);  dY[5][2] = k20 * 6.0 * z;
  Y[6] = k2a * x * z;        dY[6][0] = k2a * z; dY[6][2] = k2a * x;
  Y[7] = k22 * (x * x - y * y);      dY[7][0] = 2.0 * k22 * x; dY[7][1] = -2.0 * k22 * y;
  /* l = 3 */
  Y[8] = k33 * y * (3.0 * x * x - y * y);
  dY[8][0] = k33 * 6.0 * x * y; dY[8][1] = k33 * (3.0 * x * x - 3.0 * y * y);
  Y[9] = k32 * x * y * z;
  dY[9][0] = k32 * y * z; dY[9][1] = k32 * x * z; dY[9][2] = k32 * x * y;
  Y[10] = k31 * y * (5.0 * z * z - 1.0);
  dY[10][1] = k31 * (5.0 * z * z - 1.0); dY[10][2] = k31 * 10.0 * y * z;
  Y[11] = k30 * (5.0 * z * z * z - 3.0 * z);
  dY[11][2] = k30 * (15.0 * z * z - 3.0);
  Y[12] = k31 * x * (5.0 * z * z - 1.0);
  dY[12][0] = k31 * (5.0 * z * z - 1.0); dY[12][2] = k31 * 10.0 * x * z;
  Y[13] = k322 * z * (x * x - y * y);
  dY[13][0] = k322 * 2.0 * x * z; dY[13][1] = -k322 * 2.0 * y * z; dY[13][2] = k322 * (x * x - y * y);
  Y[14] = k33 * x * (x * x - 3.0 * y * y);
  dY[14][0] = k33 * (3.0 * x * x - 3.0 * y * y); dY[14][1] = -k33 * 6.0 * x * y;
}

/* exported for the orthonormality pin */
void orc_sh_basis(const double* d, double* Y) {
  double dY[15][3];
  sh_eval(d, Y, dY);
}

static int sh_count(int deg) { return (deg + 1) * (deg + 1) - 1; }

/* ------------------------------------------------------------------------------------------ */
/* Forward of one Gaussian in one view, keeping every intermediate for the backward.          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double qln[4], qrn[4], nl, nr;     /* normalised quaternions and their norms */
  double R[4][4], s[4], Sig[4][4];   /* rotation, scales, 4D covariance */
  double dt, c, b[3];                /* t - mu_t, Sigma_44, Sigma_{1:3,4} */
  double mean3[3], cov3[3][3];       /* Eq. 7-8 */
  double sig, ot;                    /* sigmoid(opacity logit), temporal opacity */
  double m[3];                       /* camera-space mean */
  double rx, ry; int clx, cly;       /* clamped m_x/m_z, m_y/m_z and clamp flags */
  double J[2][3], Wm[3][3], M[3][3]; /* Jacobian, world->camera rotation, W cov3 W^T */
  double cov2[2][2], det, conic[3];
  double lam, radius, u, v;
  double dir[3], dirn, dhat[3], Y[15], dY[15][3], raw[3], rgb[3];
  int visible;
  double margin, radius_margin;
} gfwd;

static double rel_margin(double x, double thr) { return fabs(x - thr) / fabs(thr); }

static double frac_margin(double x) {
  double f = x - floor(x);
  return f < 1.0 - f ? f : 1.0 - f;
}

/*
 * SCH variant (Sec. 3.1, the 4DGS appearance model): nt temporal terms; for m = 1..nt-1 the colour
 * gains cos(2 pi m t) (c_m0 + sum_k Y_k c_mk) with t the camera's frame time.  Coefficient
 * (m, k, ch), k = 0 the constant harmonic, sits at ((m - 1)(K + 1) + k) 3 + ch of the Gaussian's
 * block of sch_stride(deg, nt) doubles.
 */
static const double kPi = 3.14159265358979323846;

static int sch_stride(int deg, int nt) { return nt > 1 ? (nt - 1) * (deg + 1) * (deg + 1) * 3 : 0; }

static void forward_one(int i, int sh_deg, int mode, const double* mean4, const double* logscale4,
                        const double* ql, const double* qr, const double* opac, const double* rgb,
                        const double* sh, int nt, const double* sch, const double* cam, const double* S, gfwd* f) {
  memset(f, 0, sizeof(*f));
  const double* mu = mean4 + 4 * i;
  const double* ls = logscale4 + 4 * i;
  f->margin = INFINITY;
  f->radius_margin = INFINITY;

  /* scales and rotation (Sec. 3.3: diagonal scale, 4x4 rotation; isotropic variant ties xyz) */
  if (mode == MODE_FULL) {
    for (int k = 0; k < 4; ++k) f->s[k] = exp(ls[k]);
  } else {
    f->s[0] = f->s[1] = f->s[2] = exp(ls[0]);
    f->s[3] = exp(ls[3]);
  }
  if (mode == MODE_ISO_IDENTITY) {
    for (int a = 0; a < 4; ++a)
      for (int b2 = 0; b2 < 4; ++b2) f->R[a][b2] = (a == b2) ? 1.0 : 0.0;
    f->nl = f->nr = 1.0;
  } else {
    f->nl = sqrt(ql[4 * i] * ql[4 * i] + ql[4 * i + 1] * ql[4 * i + 1] + ql[4 * i + 2] * ql[4 * i + 2] +
                 ql[4 * i + 3] * ql[4 * i + 3]);
    f->nr = sqrt(qr[4 * i] * qr[4 * i] + qr[4 * i + 1] * qr[4 * i + 1] + qr[4 * i + 2] * qr[4 * i + 2] +
                 qr[4 * i + 3] * qr[4 * i + 3]);
    for (int k = 0; k < 4; ++k) {
      f->qln[k] = ql[4 * i + k] / f->nl;
      f->qrn[k] = qr[4 * i + k] / f->nr;
    }
    rot4_matrix(f->qln, f->qrn, f->R);
  }
  /* Sigma = R diag(s^2) R^T */
  for (int a = 0; a < 4; ++a)
    for (int b2 = 0; b2 < 4; ++b2) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += f->R[a][k] * f->s[k] * f->s[k] * f->R[b2][k];
      f->Sig[a][b2] = acc;
    }

  /* Eq. 7-8: condition on time t */
  const double t = cam[C_TIME];
  f->c = f->Sig[3][3];
  for (int k = 0; k < 3; ++k) f->b[k] = f->Sig[k][3];
  f->dt = t - mu[3];
  for (int k = 0; k < 3; ++k) f->mean3[k] = mu[k] + f->b[k] * f->dt / f->c;
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) f->cov3[a][b2] = f->Sig[a][b2] - f->b[a] * f->b[b2] / f->c;

  /* temporal marginal opacity (unnormalised temporal Gaussian) */
  f->sig = 1.0 / (1.0 + exp(-opac[i]));
  f->ot = f->sig * exp(-0.5 * f->dt * f->dt / f->c);
  f->margin = fmin(f->margin, rel_margin(f->ot, S[S_OT_MIN]));

  /* camera space */
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) f->Wm[a][b2] = cam[C_R + 3 * a + b2];
  for (int a = 0; a < 3; ++a)
    f->m[a] = f->Wm[a][0] * f->mean3[0] + f->Wm[a][1] * f->mean3[1] + f->Wm[a][2] * f->mean3[2] + cam[C_T + a];
  f->margin = fmin(f->margin, rel_margin(f->m[2], S[S_Z_NEAR]));

  int vis = (f->ot >= S[S_OT_MIN]) && (f->m[2] > S[S_Z_NEAR]);

  const double fx = cam[C_FX], fy = cam[C_FY], cx = cam[C_CX], cy = cam[C_CY];
  const double Wd = cam[C_W], Hd = cam[C_H];
  const double mz = f->m[2];
  if (mz > 0.0) {
    f->u = fx * f->m[0] / mz + cx;
    f->v = fy * f->m[1] / mz + cy;
    const double limx = S[S_FOV_CLAMP] * 0.5 * Wd / fx;
    const double limy = S[S_FOV_CLAMP] * 0.5 * Hd / fy;
    double rx = f->m[0] / mz, ry = f->m[1] / mz;
    f->clx = (rx < -limx || rx > limx);
    f->cly = (ry < -limy || ry > limy);
    f->rx = rx < -limx ? -limx : (rx > limx ? limx : rx);
    f->ry = ry < -limy ? -limy : (ry > limy ? limy : ry);
    f->J[0][0] = fx / mz; f->J[0][1] = 0.0; f->J[0][2] = -fx * f->rx / mz;
    f->J[1][0] = 0.0; f->J[1][1] = fy / mz; f->J[1][2] = -fy * f->ry / mz;
    /* M = W cov3 W^T */
    double WC[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b2 = 0; b2 < 3; ++b2) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += f->Wm[a][k] * f->cov3[k][b2];
        WC[a][b2] = acc;
      }
    for (int a = 0; a < 3; ++a)
      for (int b2 = 0; b2 < 3; ++b2) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += WC[a][k] * f->Wm[b2][k];
        f->M[a][b2] = acc;
      }
    /* cov2 = J M J^T + dilation I */
    double JM[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b2 = 0; b2 < 3; ++b2) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += f->J[a][k] * f->M[k][b2];
        JM[a][b2] = acc;
      }
    for (int a = 0; a < 2; ++a)
      for (int b2 = 0; b2 < 2; ++b2) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += JM[a][k] * f->J[b2][k];
        f->cov2[a][b2] = acc + (a == b2 ? S[S_DILATION] : 0.0);
      }
    f->det = f->cov2[0][0] * f->cov2[1][1] - f->cov2[0][1] * f->cov2[1][0];
    if (f->det > 0.0) {
      f->conic[0] = f->cov2[1][1] / f->det;
      f->conic[1] = -f->cov2[0][1] / f->det;
      f->conic[2] = f->cov2[0][0] / f->det;
      const double mid = 0.5 * (f->cov2[0][0] + f->cov2[1][1]);
      const double disc = mid * mid - f->det;
      f->lam = mid + sqrt(disc > 0.0 ? disc : 0.0);
      const double r3 = 3.0 * sqrt(f->lam);
      f->radius = ceil(r3);
      f->radius_margin = frac_margin(r3) / fmax(r3, 1.0);
    } else {
      vis = 0;
    }
  } else {
    vis = 0;
  }

  /* colour: base RGB plus view-dependent real SH of the direction from the camera centre */
  {
    double cpos[3];
    for (int a = 0; a < 3; ++a)
      cpos[a] = -(f->Wm[0][a] * cam[C_T + 0] + f->Wm[1][a] * cam[C_T + 1] + f->Wm[2][a] * cam[C_T + 2]);
    for (int a = 0; a < 3; ++a) f->dir[a] = f->mean3[a] - cpos[a];
    f->dirn = sqrt(f->dir[0] * f->dir[0] + f->dir[1] * f->dir[1] + f->dir[2] * f->dir[2]);
    for (int a = 0; a < 3; ++a) f->dhat[a] = f->dir[a] / f->dirn;
    sh_eval(f->dhat, f->Y, f->dY);
    const int K = sh_count(sh_deg);
    for (int ch = 0; ch < 3; ++ch) {
      double acc = rgb[3 * i + ch];
      for (int k = 0; k < K; ++k) acc += f->Y[k] * sh[(size_t)i * 45 + 3 * k + ch];
      for (int m = 1; m < nt; ++m) {
        const double cs = cos(2.0 * kPi * m * cam[C_TIME]);
        for (int k = 0; k <= K; ++k) {
          const double Yk = k == 0 ? 1.0 : f->Y[k - 1];
          acc += cs * Yk * sch[(size_t)i * sch_stride(sh_deg, nt) + ((size_t)(m - 1) * (K + 1) + k) * 3 + ch];
        }
      }
      f->raw[ch] = acc;
      f->rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
  }

  f->visible = vis;
}

static void store_record(const gfwd* f, double* rec) {
  rec[P_VISIBLE] = f->visible;
  rec[P_U] = f->u; rec[P_V] = f->v; rec[P_DEPTH] = f->m[2]; rec[P_OT] = f->ot;
  rec[P_CA] = f->conic[0]; rec[P_CB] = f->conic[1]; rec[P_CC] = f->conic[2];
  rec[P_RADIUS] = f->radius;
  rec[P_R] = f->rgb[0]; rec[P_G] = f->rgb[1]; rec[P_B] = f->rgb[2];
  rec[P_MARGIN] = f->margin; rec[P_RADIUS_MARGIN] = f->radius_margin;
  rec[P_M3X] = f->mean3[0]; rec[P_M3Y] = f->mean3[1]; rec[P_M3Z] = f->mean3[2];
  rec[P_S3XX] = f->cov3[0][0]; rec[P_S3XY] = f->cov3[0][1]; rec[P_S3XZ] = f->cov3[0][2];
  rec[P_S3YY] = f->cov3[1][1]; rec[P_S3YZ] = f->cov3[1][2]; rec[P_S3ZZ] = f->cov3[2][2];
}

/*
 * Slice (Eq. 7-8), temporal opacity and cull (Eq. 9 and the threshold that follows it),
 * EWA projection and colour for every Gaussian in one camera.  out: n x P_STRIDE records.
 */
int orc_project(int n, int sh_deg, int mode, const double* mean4, const double* logscale4,
                const double* ql, const double* qr, const double* opac, const double* rgb,
                const double* sh, int nt, const double* sch, const double* cam, const double* S, double* out) {
  if (n < 0 || sh_deg < 0 || sh_deg > 3 || mode < 0 || mode > 2) return -1;
  if (nt > 1 && !sch) return -1;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    gfwd f;
    forward_one(i, sh_deg, mode, mean4, logscale4, ql, qr, opac, rgb, sh, nt, sch, cam, S, &f);
    store_record(&f, out + (size_t)i * P_STRIDE);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Per-pixel compositing                                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct { double depth; int id; double q, alpha, g, margin; int kept; } frag;

static int frag_cmp(const void* pa, const void* pb) {
  const frag* a = (const frag*)pa;
  const frag* b = (const frag*)pb;
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  return (a->id > b->id) - (a->id < b->id);
}

/* fragments closer than this (relative) to a threshold are reported as candidates for a flip */
#define NEAR_MARGIN 1e-3

/*
 * Collect the fragments of pixel (px, py), sorted by (depth, id): every visible Gaussian whose
 * 3-sigma ellipse covers the pixel centre (q <= q_max) and whose alpha = min(alpha_max,
 * o_t exp(-q/2)) reaches alpha_min (kept = 1), plus the Gaussians that miss one of these tests, or
 * the o_t cull or the near plane, by less than NEAR_MARGIN relative (kept = 0).  Each fragment
 * carries the smallest relative distance of its own decisions from their thresholds.
 */
static int gather_pixel(int n, const double* P, const double* S, int px, int py, frag* buf) {
  const double cxp = px + 0.5, cyp = py + 0.5;
  int cnt = 0;
  for (int i = 0; i < n; ++i) {
    const double* r = P + (size_t)i * P_STRIDE;
    const int vis = r[P_VISIBLE] != 0.0;
    if (!vis && !(r[P_MARGIN] < NEAR_MARGIN)) continue;
    if (r[P_DEPTH] <= 0.0 || !(r[P_CA] > 0.0)) continue;
    const double dx = cxp - r[P_U], dy = cyp - r[P_V];
    const double q = r[P_CA] * dx * dx + 2.0 * r[P_CB] * dx * dy + r[P_CC] * dy * dy;
    if (q > S[S_Q_MAX] * (1.0 + NEAR_MARGIN)) continue;
    const double g = exp(-0.5 * q);
    const double a_raw = r[P_OT] * g;
    const double alpha = a_raw < S[S_ALPHA_MAX] ? a_raw : S[S_ALPHA_MAX];
    double m = fmin(rel_margin(q, S[S_Q_MAX]), r[P_MARGIN]);
    m = fmin(m, rel_margin(a_raw, S[S_ALPHA_MIN]));
    const int kept = vis && q <= S[S_Q_MAX] && alpha >= S[S_ALPHA_MIN];
    if (!kept && !(m < NEAR_MARGIN)) continue;
    buf[cnt].depth = r[P_DEPTH];
    buf[cnt].id = i;
    buf[cnt].q = q;
    buf[cnt].alpha = alpha;
    buf[cnt].g = g;
    buf[cnt].margin = m;
    buf[cnt].kept = kept;
    ++cnt;
  }
  qsort(buf, cnt, sizeof(frag), frag_cmp);
  return cnt;
}

static double colour_scale(const double* r) {
  double c = 1.0;
  for (int ch = P_R; ch <= P_B; ++ch) c = fmax(c, fabs(r[ch]));
  return c;
}

/*
 * Walk the sorted fragments as the compositing does and report, for the decisions whose flip could
 * change the pixel by more than impact_min, the smallest relative distance from a threshold (*mg:
 * q, alpha, cull, near plane, the T stop) and the smallest relative depth gap between two
 * consecutive blended fragments (*dmg).  A fragment of weight T alpha moves the colour by at most
 * T alpha max(1, |c|) when it enters or leaves; swapping consecutive fragments j, k moves it by at
 * most T_j alpha_j alpha_k max(1, |c_j - c_k|).
 */
static void decision_margins(const double* P, const double* S, const frag* buf, int cnt, double impact_min,
                             double* mg, double* dmg) {
  double T = 1.0, Tprev = 0.0, aprev = 0.0;
  int prev = -1;
  for (int k = 0; k < cnt; ++k) {
    const frag* f = buf + k;
    const double* r = P + (size_t)f->id * P_STRIDE;
    const double w = T * fmin(S[S_ALPHA_MAX], r[P_OT] * f->g) * colour_scale(r);
    if (!f->kept) {
      if (w > impact_min) *mg = fmin(*mg, f->margin);
      continue;
    }
    const double a = f->alpha;
    const double Tn = T * (1.0 - a);
    if (w > impact_min) *mg = fmin(*mg, fmin(f->margin, rel_margin(Tn, S[S_T_MIN])));
    if (Tn < S[S_T_MIN]) break;
    if (prev >= 0) {
      const double* rp = P + (size_t)buf[prev].id * P_STRIDE;
      double dc = 1.0;
      for (int ch = P_R; ch <= P_B; ++ch) dc = fmax(dc, fabs(r[ch] - rp[ch]));
      if (Tprev * aprev * a * dc > impact_min)
        *dmg = fmin(*dmg, fabs(f->depth - buf[prev].depth) / buf[prev].depth);
    }
    prev = k;
    Tprev = T;
    aprev = a;
    T = Tn;
  }
}

/* drop the fragments that are not kept, preserving order; returns the new count */
static int compact_kept(frag* buf, int cnt) {
  int m = 0;
  for (int k = 0; k < cnt; ++k)
    if (buf[k].kept) buf[m++] = buf[k];
  return m;
}

/*
 * Front-to-back compositing of the sorted fragments: T = 1; a fragment whose blending would
 * take T(1 - alpha) below T_min ends the walk before it is blended; C += T alpha rgb,
 * T *= (1 - alpha); finally C += T bg.  Returns the number of fragments blended.
 */
static int composite(const double* P, const double* S, const frag* buf, int cnt, const double* bg,
                     double C[3], double* Tout) {
  double T = 1.0;
  C[0] = C[1] = C[2] = 0.0;
  int k = 0;
  for (; k < cnt; ++k) {
    const double a = buf[k].alpha;
    const double Tn = T * (1.0 - a);
    if (Tn < S[S_T_MIN]) break;
    const double* r = P + (size_t)buf[k].id * P_STRIDE;
    C[0] += T * a * r[P_R];
    C[1] += T * a * r[P_G];
    C[2] += T * a * r[P_B];
    T = Tn;
  }
  for (int ch = 0; ch < 3; ++ch) C[ch] += T * bg[ch];
  *Tout = T;
  return k;
}

/*
 * Render npix pixels (indices py*W + px; pix == NULL means all W*H in raster order) from the
 * records of orc_project.  img: npix x 3 (pixel-major), Tfinal, ncontrib, margin, dmargin: npix
 * (decision margins of decisions whose flip could move the pixel by more than impact_min).
 */
int orc_render(int n, const double* P, const double* cam, const double* bg, const double* S, int npix,
               const int* pix, double impact_min, double* img, double* Tfinal, int* ncontrib, double* margin,
               double* dmargin) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  if (pix == NULL && npix != W * H) return -1;
  int err = 0;
#pragma omp parallel
  {
    frag* buf = (frag*)malloc(sizeof(frag) * (size_t)(n > 0 ? n : 1));
    if (!buf) {
#pragma omp atomic write
      err = -2;
    }
#pragma omp for schedule(dynamic, 16)
    for (int j = 0; j < npix; ++j) {
      if (!buf) continue;
      const int p = pix ? pix[j] : j;
      const int px = p % W, py = p / W;
      double mg = INFINITY, dmg = INFINITY, C[3], T;
      int cnt = gather_pixel(n, P, S, px, py, buf);
      decision_margins(P, S, buf, cnt, impact_min, &mg, &dmg);
      cnt = compact_kept(buf, cnt);
      ncontrib[j] = composite(P, S, buf, cnt, bg, C, &T);
      img[3 * j + 0] = C[0];
      img[3 * j + 1] = C[1];
      img[3 * j + 2] = C[2];
      Tfinal[j] = T;
      margin[j] = mg;
      dmargin[j] = dmg;
    }
    free(buf);
  }
  return err;
}

/*
 * Every valid colour of a pixel whose compositing takes decisions that a float32 evaluation may
 * take the other way: (1) fragments whose depths differ by less than depth_margin (relative) have
 * no order a float32 sort can be held to, so every order of each maximal run of such consecutive
 * fragments (in (depth, id) order) is valid; (2) a fragment whose coverage, alpha, cull or
 * near-plane decision lies within `margin` (relative) of its threshold may be blended or not;
 * (3) a blend whose T(1 - alpha) lies within `margin` of T_min may stop the pixel or not.  A
 * decision is branched on only where its flip could move the colour by more than impact_min (the
 * fragment's weight T alpha max(1, |c|), as in decision_margins; a run is permuted only when two of
 * its fragments carry that much weight in the (depth, id) order).  The colours of all branches are
 * written; the first is the (depth, id) order with every decision taken as computed.
 */
static int factorial(int g) { int f = 1; for (int k = 2; k <= g; ++k) f *= k; return f; }

/* the idx-th permutation of 0..g-1 in lexicographic order (Lehmer code) */
static void nth_permutation(int g, int idx, int* perm) {
  int pool[8];
  for (int k = 0; k < g; ++k) pool[k] = k;
  for (int k = 0; k < g; ++k) {
    const int f = factorial(g - 1 - k);
    const int sel = idx / f;
    idx %= f;
    perm[k] = pool[sel];
    for (int m = sel; m < g - 1 - k; ++m) pool[m] = pool[m + 1];
  }
}

typedef struct {
  const double *P, *S, *bg;
  const frag* f;
  int cnt;
  const int* run_len;      /* > 1 at the first fragment of a permuted run, else 1 */
  double margin, impact_min;
  int max_alt, n_out;      /* n_out > max_alt: too many branches */
  double* out;
} alt_walk;

static void alt_leaf(alt_walk* w, const double C[3], double T) {
  if (w->n_out < w->max_alt)
    for (int ch = 0; ch < 3; ++ch) w->out[3 * w->n_out + ch] = C[ch] + T * w->bg[ch];
  w->n_out++;
}

/* outcomes of one fragment: (T after, colour after, stopped); returns their number (1..3) */
static int frag_outcomes(const alt_walk* w, const frag* fr, double T, const double C[3], double To[3],
                         double Co[3][3], int stop[3]) {
  const double* r = w->P + (size_t)fr->id * P_STRIDE;
  const double weight = T * fr->alpha * colour_scale(r);
  const int matters = weight > w->impact_min;
  int no = 0;
  const int blend_opts = (fr->margin < w->margin && matters) ? 2 : 1;
  for (int b = 0; b < blend_opts; ++b) {
    const int blend = blend_opts == 2 ? b : fr->kept;
    if (!blend) {
      To[no] = T; stop[no] = 0;
      for (int ch = 0; ch < 3; ++ch) Co[no][ch] = C[ch];
      ++no;
      continue;
    }
    const double Tn = T * (1.0 - fr->alpha);
    const int canon_stop = Tn < w->S[S_T_MIN];
    const int stop_opts = (rel_margin(Tn, w->S[S_T_MIN]) < w->margin && matters) ? 2 : 1;
    for (int q = 0; q < stop_opts; ++q) {
      const int st = stop_opts == 2 ? q : canon_stop;
      stop[no] = st;
      if (st) {
        To[no] = T;
        for (int ch = 0; ch < 3; ++ch) Co[no][ch] = C[ch];
      } else {
        To[no] = Tn;
        Co[no][0] = C[0] + T * fr->alpha * r[P_R];
        Co[no][1] = C[1] + T * fr->alpha * r[P_G];
        Co[no][2] = C[2] + T * fr->alpha * r[P_B];
      }
      ++no;
    }
  }
  return no;
}

static void alt_from(alt_walk* w, int k, double T, const double C[3]);

/* process the fragments seq[j..g) in that order, then continue in (depth, id) order from k_after */
static void alt_seq(alt_walk* w, const int* seq, int j, int g, int k_after, double T, const double C[3]) {
  if (w->n_out > w->max_alt) return;
  if (j == g) { alt_from(w, k_after, T, C); return; }
  double To[3], Co[3][3];
  int stop[3];
  const int no = frag_outcomes(w, &w->f[seq[j]], T, C, To, Co, stop);
  for (int o = 0; o < no; ++o) {
    if (stop[o]) alt_leaf(w, Co[o], To[o]);
    else alt_seq(w, seq, j + 1, g, k_after, To[o], Co[o]);
  }
}

static void alt_from(alt_walk* w, int k, double T, const double C[3]) {
  if (w->n_out > w->max_alt) return;
  if (k == w->cnt) { alt_leaf(w, C, T); return; }
  const int g = w->run_len[k];
  if (g > 1) {
    int perm[8], seq[8];
    for (int p = 0; p < factorial(g); ++p) {
      nth_permutation(g, p, perm);
      for (int m = 0; m < g; ++m) seq[m] = k + perm[m];
      alt_seq(w, seq, 0, g, k + g, T, C);
      if (w->n_out > w->max_alt) return;
    }
    return;
  }
  double To[3], Co[3][3];
  int stop[3];
  const int no = frag_outcomes(w, &w->f[k], T, C, To, Co, stop);
  for (int o = 0; o < no; ++o) {
    if (stop[o]) alt_leaf(w, Co[o], To[o]);
    else alt_from(w, k + 1, To[o], Co[o]);
  }
}

/*
 * alt: npix x max_alt x 3 colours; n_alt[j]: how many (>= 1), or -1 when the branches exceed
 * max_alt (alt then holds the first max_alt).  Runs longer than 7 fragments are not permuted and
 * make the pixel -1.
 */
int orc_render_alternatives(int n, const double* P, const double* cam, const double* bg, const double* S, int npix,
                            const int* pix, double margin, double depth_margin, double impact_min, int max_alt,
                            double* alt, int* n_alt) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  if ((pix == NULL && npix != W * H) || max_alt < 1) return -1;
  int err = 0;
#pragma omp parallel
  {
    frag* buf = (frag*)malloc(sizeof(frag) * (size_t)(n > 0 ? n : 1));
    int* run_len = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double* wgt = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!buf || !run_len || !wgt) {
#pragma omp atomic write
      err = -2;
    }
#pragma omp for schedule(dynamic, 4)
    for (int j = 0; j < npix; ++j) {
      if (err) continue;
      const int p = pix ? pix[j] : j;
      const int cnt = gather_pixel(n, P, S, p % W, p / W, buf);
      /* weights T alpha max(1, |c|) of the candidates in the (depth, id) walk (0 after its stop) */
      double T = 1.0;
      for (int k = 0; k < cnt; ++k) {
        const double* r = P + (size_t)buf[k].id * P_STRIDE;
        wgt[k] = T * buf[k].alpha * colour_scale(r);
        if (buf[k].kept && T > 0.0) {
          const double Tn = T * (1.0 - buf[k].alpha);
          T = Tn < S[S_T_MIN] ? 0.0 : Tn;
        }
      }
      int too_long = 0;
      for (int k = 0; k < cnt;) {
        int e = k + 1;
        while (e < cnt && fabs(buf[e].depth - buf[e - 1].depth) < depth_margin * fabs(buf[e - 1].depth)) ++e;
        int heavy = 0;
        for (int m = k; m < e; ++m) heavy += wgt[m] > impact_min;
        run_len[k] = (e - k > 1 && heavy > 1) ? e - k : 1;
        if (run_len[k] > 7) too_long = 1;
        for (int m = k + 1; m < e; ++m) run_len[m] = 1;
        if (run_len[k] == 1) e = k + 1;
        k = e;
      }
      alt_walk w = {P, S, bg, buf, cnt, run_len, margin, impact_min, max_alt, 0, alt + (size_t)j * max_alt * 3};
      if (too_long) {
        n_alt[j] = -1;
        continue;
      }
      const double C0[3] = {0.0, 0.0, 0.0};
      alt_from(&w, 0, 1.0, C0);
      n_alt[j] = w.n_out > max_alt ? -1 : w.n_out;
    }
    free(buf);
    free(run_len);
    free(wgt);
  }
  return err;
}

/* ------------------------------------------------------------------------------------------ */
/* Backward                                                                                     */
/* ------------------------------------------------------------------------------------------ */
/* 2D gradient columns per Gaussian */
enum { G_U = 0, G_V, G_CA, G_CB, G_CC, G_OT, G_R, G_G, G_B, G_STRIDE };

int orc_grad2d_stride(void) { return G_STRIDE; }

/*
 * Reverse mode of the compositing for one pixel.  With T_k the transmittance in front of
 * fragment k and S_k = sum_{j>k} T_j alpha_j c_j + T_final bg (everything behind it),
 *   dC/dc_k = T_k alpha_k,   dC/dalpha_k = T_k c_k - S_k / (1 - alpha_k).
 * alpha_k = o_t exp(-q/2) (zero derivative where it is clamped at alpha_max);
 * q = d^T Q d with d = p - uv and Q the conic [[a, b], [b, c]].
 */
static void pixel_backward(const double* P, const frag* buf, int nblend, double Tfinal, const double* bg,
                           const double* gC, int px, int py, const double* S, double* T, double* g2) {
  double t = 1.0;
  for (int k = 0; k < nblend; ++k) {
    T[k] = t;
    t *= (1.0 - buf[k].alpha);
  }
  double Sacc[3] = {Tfinal * bg[0], Tfinal * bg[1], Tfinal * bg[2]};
  for (int k = nblend - 1; k >= 0; --k) {
    const int id = buf[k].id;
    const double* r = P + (size_t)id * P_STRIDE;
    const double a = buf[k].alpha;
    const double c[3] = {r[P_R], r[P_G], r[P_B]};
    double* g = g2 + (size_t)id * G_STRIDE;
    g[G_R] += T[k] * a * gC[0];
    g[G_G] += T[k] * a * gC[1];
    g[G_B] += T[k] * a * gC[2];
    double dA = 0.0;
    for (int ch = 0; ch < 3; ++ch) dA += gC[ch] * (T[k] * c[ch] - Sacc[ch] / (1.0 - a));
    for (int ch = 0; ch < 3; ++ch) Sacc[ch] += T[k] * a * c[ch];
    const double a_raw = r[P_OT] * buf[k].g;
    if (a_raw >= S[S_ALPHA_MAX]) continue;
    g[G_OT] += dA * buf[k].g;
    const double dq = dA * (-0.5 * a_raw);
    const double dx = px + 0.5 - r[P_U], dy = py + 0.5 - r[P_V];
    g[G_U] += dq * (-2.0) * (r[P_CA] * dx + r[P_CB] * dy);
    g[G_V] += dq * (-2.0) * (r[P_CB] * dx + r[P_CC] * dy);
    g[G_CA] += dq * dx * dx;
    g[G_CB] += dq * 2.0 * dx * dy;
    g[G_CC] += dq * dy * dy;
  }
}

/*
 * Chain the 2D gradients of one Gaussian through projection, slicing and the 4D
 * parameterisation to the parameter gradients (accumulated into the g_* arrays).
 */
static void chain_to_params(int i, int sh_deg, int mode, const double* sh, int nt, const double* sch,
                            const double* cam, const gfwd* f, const double* g2, double* g_mean4,
                            double* g_logscale4, double* g_ql, double* g_qr, double* g_opac, double* g_rgb,
                            double* g_sh, double* g_sch) {
  const double fx = cam[C_FX], fy = cam[C_FY];
  const double mz = f->m[2], mx = f->m[0], my = f->m[1];
  double gm[3] = {0, 0, 0};
  double gmean3[3] = {0, 0, 0};

  /* uv = (fx mx/mz + cx, fy my/mz + cy) */
  gm[0] += g2[G_U] * fx / mz;
  gm[2] += g2[G_U] * (-fx * mx / (mz * mz));
  gm[1] += g2[G_V] * fy / mz;
  gm[2] += g2[G_V] * (-fy * my / (mz * mz));

  /* conic = cov2^{-1}: G_cov2 = -Q G_Q Q with G_Q the symmetric gradient of Q */
  const double Q[2][2] = {{f->conic[0], f->conic[1]}, {f->conic[1], f->conic[2]}};
  const double GQ[2][2] = {{g2[G_CA], 0.5 * g2[G_CB]}, {0.5 * g2[G_CB], g2[G_CC]}};
  double tmp[2][2], G2[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b2 = 0; b2 < 2; ++b2) tmp[a][b2] = Q[a][0] * GQ[0][b2] + Q[a][1] * GQ[1][b2];
  for (int a = 0; a < 2; ++a)
    for (int b2 = 0; b2 < 2; ++b2) G2[a][b2] = -(tmp[a][0] * Q[0][b2] + tmp[a][1] * Q[1][b2]);

  /* cov2 = J M J^T + dil I:  G_M = J^T G2 J,  G_J = 2 G2 J M */
  double GM[3][3], GJ[2][3];
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) {
      double acc = 0.0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) acc += f->J[k][a] * G2[k][l] * f->J[l][b2];
      GM[a][b2] = acc;
    }
  for (int a = 0; a < 2; ++a)
    for (int b2 = 0; b2 < 3; ++b2) {
      double acc = 0.0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 3; ++l) acc += G2[a][k] * f->J[k][l] * f->M[l][b2];
      GJ[a][b2] = 2.0 * acc;
    }
  /* J(m): J00 = fx/mz, J11 = fy/mz, J02 = -fx rx/mz, J12 = -fy ry/mz, rx = clamp(mx/mz) */
  gm[2] += GJ[0][0] * (-fx / (mz * mz));
  gm[2] += GJ[1][1] * (-fy / (mz * mz));
  if (!f->clx) {
    gm[0] += GJ[0][2] * (-fx / (mz * mz));
    gm[2] += GJ[0][2] * (2.0 * fx * mx / (mz * mz * mz));
  } else {
    gm[2] += GJ[0][2] * (fx * f->rx / (mz * mz));
  }
  if (!f->cly) {
    gm[1] += GJ[1][2] * (-fy / (mz * mz));
    gm[2] += GJ[1][2] * (2.0 * fy * my / (mz * mz * mz));
  } else {
    gm[2] += GJ[1][2] * (fy * f->ry / (mz * mz));
  }
  /* m = W mean3 + tau */
  for (int a = 0; a < 3; ++a) gmean3[a] += f->Wm[0][a] * gm[0] + f->Wm[1][a] * gm[1] + f->Wm[2][a] * gm[2];
  /* M = W cov3 W^T:  G_cov3 = W^T G_M W */
  double G3[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += f->Wm[k][a] * GM[k][l] * f->Wm[l][b2];
      G3[a][b2] = acc;
    }

  /* colour: rgb = max(0, base + sum_k Y_k(dhat) sh_k), dhat = dir/|dir|, dir = mean3 - campos */
  {
    double gdhat[3] = {0, 0, 0};
    const int K = sh_count(sh_deg);
    const double grgb[3] = {g2[G_R], g2[G_G], g2[G_B]};
    for (int ch = 0; ch < 3; ++ch) {
      if (f->raw[ch] < 0.0) continue;
      g_rgb[3 * i + ch] += grgb[ch];
      for (int k = 0; k < K; ++k) {
        g_sh[(size_t)i * 45 + 3 * k + ch] += f->Y[k] * grgb[ch];
        const double c = sh[(size_t)i * 45 + 3 * k + ch] * grgb[ch];
        for (int a = 0; a < 3; ++a) gdhat[a] += c * f->dY[k][a];
      }
      for (int m = 1; m < nt; ++m) {  /* SCH: d/dc_mk = cos(2 pi m t) Y_k; Y_k (k >= 1) depends on dhat */
        const double cs = cos(2.0 * kPi * m * cam[C_TIME]);
        for (int k = 0; k <= K; ++k) {
          const size_t o = (size_t)i * sch_stride(sh_deg, nt) + ((size_t)(m - 1) * (K + 1) + k) * 3 + ch;
          g_sch[o] += cs * (k == 0 ? 1.0 : f->Y[k - 1]) * grgb[ch];
          if (k > 0)
            for (int a = 0; a < 3; ++a) gdhat[a] += cs * sch[o] * grgb[ch] * f->dY[k - 1][a];
        }
      }
    }
    const double dd = f->dhat[0] * gdhat[0] + f->dhat[1] * gdhat[1] + f->dhat[2] * gdhat[2];
    for (int a = 0; a < 3; ++a) gmean3[a] += (gdhat[a] - f->dhat[a] * dd) / f->dirn;
  }

  /* temporal opacity o_t = sigmoid(o) exp(-dt^2 / (2c)) */
  double gc = 0.0, gmut = 0.0;
  const double got = g2[G_OT];
  g_opac[i] += got * f->ot * (1.0 - f->sig);
  gc += got * f->ot * 0.5 * f->dt * f->dt / (f->c * f->c);
  gmut += got * f->ot * f->dt / f->c;

  /* Eq. 7: mean3 = mu_xyz + b dt / c */
  double gb[3];
  const double bg3 = f->b[0] * gmean3[0] + f->b[1] * gmean3[1] + f->b[2] * gmean3[2];
  for (int a = 0; a < 3; ++a) {
    g_mean4[4 * i + a] += gmean3[a];
    gb[a] = gmean3[a] * f->dt / f->c;
  }
  gmut += -bg3 / f->c;
  gc += -f->dt * bg3 / (f->c * f->c);
  /* Eq. 8: cov3 = A - b b^T / c */
  double G3b[3];
  for (int a = 0; a < 3; ++a) G3b[a] = G3[a][0] * f->b[0] + G3[a][1] * f->b[1] + G3[a][2] * f->b[2];
  for (int a = 0; a < 3; ++a) gb[a] += -2.0 * G3b[a] / f->c;
  gc += (f->b[0] * G3b[0] + f->b[1] * G3b[1] + f->b[2] * G3b[2]) / (f->c * f->c);
  g_mean4[4 * i + 3] += gmut;

  /* symmetric gradient of the 4D covariance */
  double GS[4][4];
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) GS[a][b2] = G3[a][b2];
  for (int a = 0; a < 3; ++a) GS[a][3] = GS[3][a] = 0.5 * gb[a];
  GS[3][3] = gc;

  /* Sigma = R D R^T, D = diag(s^2):  G_R = 2 G R D,  G_D = diag(R^T G R) */
  double GR[4][4], GD[4];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) {
      double acc = 0.0;
      for (int l = 0; l < 4; ++l) acc += GS[a][l] * f->R[l][k];
      GR[a][k] = 2.0 * acc * f->s[k] * f->s[k];
    }
  for (int k = 0; k < 4; ++k) {
    double acc = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int l = 0; l < 4; ++l) acc += f->R[a][k] * GS[a][l] * f->R[l][k];
    GD[k] = acc;
  }
  /* D_kk = exp(2 logscale_k) */
  if (mode == MODE_FULL) {
    for (int k = 0; k < 4; ++k) g_logscale4[4 * i + k] += GD[k] * 2.0 * f->s[k] * f->s[k];
  } else {
    g_logscale4[4 * i + 0] += (GD[0] + GD[1] + GD[2]) * 2.0 * f->s[0] * f->s[0];
    g_logscale4[4 * i + 3] += GD[3] * 2.0 * f->s[3] * f->s[3];
  }

  if (mode == MODE_ISO_IDENTITY) return;
  /* R[:,k] = ql (x) e_k (x) qr is linear in ql and in qr:
     dR[:,k]/dql_j = E_j (x) e_k (x) qr,  dR[:,k]/dqr_j = ql (x) e_k (x) E_j. */
  double gqln[4] = {0, 0, 0, 0}, gqrn[4] = {0, 0, 0, 0};
  for (int j = 0; j < 4; ++j) {
    double Ej[4] = {0, 0, 0, 0};
    Ej[j] = 1.0;
    for (int k = 0; k < 4; ++k) {
      double e[4] = {0, 0, 0, 0}, col[4];
      e[k] = 1.0;
      rot4_apply(Ej, f->qrn, e, col);
      for (int a = 0; a < 4; ++a) gqln[j] += GR[a][k] * col[a];
      rot4_apply(f->qln, Ej, e, col);
      for (int a = 0; a < 4; ++a) gqrn[j] += GR[a][k] * col[a];
    }
  }
  /* q_hat = q / |q| */
  const double dl = gqln[0] * f->qln[0] + gqln[1] * f->qln[1] + gqln[2] * f->qln[2] + gqln[3] * f->qln[3];
  const double dr = gqrn[0] * f->qrn[0] + gqrn[1] * f->qrn[1] + gqrn[2] * f->qrn[2] + gqrn[3] * f->qrn[3];
  for (int j = 0; j < 4; ++j) {
    g_ql[4 * i + j] += (gqln[j] - f->qln[j] * dl) / f->nl;
    g_qr[4 * i + j] += (gqrn[j] - f->qrn[j] * dr) / f->nr;
  }
}

/*
 * Full backward for one camera: dL/dimg (npix x 3, pixel-major, for the pixels in pix or all
 * pixels) -> 2D gradients per Gaussian (n x G_STRIDE, overwritten) and parameter gradients
 * (accumulated into g_mean4 .. g_sh, so that several views can be summed by repeated calls).
 */
int orc_render_bwd(int n, int sh_deg, int mode, const double* mean4, const double* logscale4, const double* ql,
                   const double* qr, const double* opac, const double* rgb, const double* sh, int nt,
                   const double* sch, const double* cam, const double* bg, const double* S, int npix,
                   const int* pix, const double* dL_dimg, double* grad2d, double* g_mean4, double* g_logscale4,
                   double* g_ql, double* g_qr, double* g_opac, double* g_rgb, double* g_sh, double* g_sch) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  if (pix == NULL && npix != W * H) return -1;
  double* P = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * P_STRIDE);
  if (!P) return -2;
  if (orc_project(n, sh_deg, mode, mean4, logscale4, ql, qr, opac, rgb, sh, nt, sch, cam, S, P) != 0) {
    free(P);
    return -1;
  }
  memset(grad2d, 0, sizeof(double) * (size_t)n * G_STRIDE);
  int nthreads = orc_max_threads();
  double* part = (double*)calloc((size_t)nthreads * n * G_STRIDE + 1, sizeof(double));
  if (!part) { free(P); return -2; }
  int err = 0;
#pragma omp parallel
  {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    double* g2 = part + (size_t)tid * n * G_STRIDE;
    frag* buf = (frag*)malloc(sizeof(frag) * (size_t)(n > 0 ? n : 1));
    double* Tb = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!buf || !Tb) {
#pragma omp atomic write
      err = -2;
    }
#pragma omp for schedule(dynamic, 16)
    for (int j = 0; j < npix; ++j) {
      if (!buf || !Tb) continue;
      const int p = pix ? pix[j] : j;
      const int px = p % W, py = p / W;
      const double* gC = dL_dimg + 3 * (size_t)j;
      if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) continue;
      double C[3], T;
      const int cnt = compact_kept(buf, gather_pixel(n, P, S, px, py, buf));
      const int nb = composite(P, S, buf, cnt, bg, C, &T);
      pixel_backward(P, buf, nb, T, bg, gC, px, py, S, Tb, g2);
    }
    free(buf);
    free(Tb);
  }
  for (int t = 0; t < nthreads; ++t)
    for (size_t k = 0; k < (size_t)n * G_STRIDE; ++k) grad2d[k] += part[(size_t)t * n * G_STRIDE + k];
  free(part);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    const double* g2 = grad2d + (size_t)i * G_STRIDE;
    int any = 0;
    for (int k = 0; k < G_STRIDE; ++k) any |= (g2[k] != 0.0);
    if (!any) continue;
    gfwd f;
    forward_one(i, sh_deg, mode, mean4, logscale4, ql, qr, opac, rgb, sh, nt, sch, cam, S, &f);
    chain_to_params(i, sh_deg, mode, sh, nt, sch, cam, &f, g2, g_mean4, g_logscale4, g_ql, g_qr, g_opac, g_rgb,
                    g_sh, g_sch);
  }
  free(P);
  return err;
}

/* ------------------------------------------------------------------------------------------ */
/* Tile lists (the (tile, depth, id) order of the binning step)                                 */
/* ------------------------------------------------------------------------------------------ */
typedef struct { int tile; double depth; int id; int status; } tentry;

static int tentry_cmp(const void* pa, const void* pb) {
  const tentry* a = (const tentry*)pa;
  const tentry* b = (const tentry*)pb;
  if (a->tile != b->tile) return (a->tile > b->tile) - (a->tile < b->tile);
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  return (a->id > b->id) - (a->id < b->id);
}

/*
 * Tiles of one Gaussian that hold a blendable pixel centre.  By the coverage rule of the
 * compositing, the Gaussian takes part at pixel centre p = (px + 0.5, py + 0.5) only where
 * q(p) = (p - uv)^T conic (p - uv) <= q_max and alpha = o_t exp(-q/2) >= alpha_min, so a tile must
 * list it exactly when one of its pixel centres (inside the view) satisfies both.  Every pixel
 * centre of the box of the ellipse q <= q_max (half-widths sqrt(q_max Sigma2_xx), sqrt(q_max
 * Sigma2_yy), Sigma2 the inverse conic) is tested, so none is missed.  Status per tile: 1 when a
 * pixel centre passes both tests with relative slack above `margin`, 2 when no pixel does but one
 * lies within `margin` of a threshold (a float32 evaluation may take or drop the tile), no entry
 * otherwise.  Calls emit(tile index ty * tiles_x + tx, status) in row-major tile order.
 */
typedef void (*tile_sink)(void* ctx, int tile, int status);

static void gaussian_tiles(const double* r, int W, int H, int tile_w, int tile_h, const double* S, double margin,
                           int* scratch, tile_sink emit, void* ctx) {
  const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
  const double u = r[P_U], v = r[P_V], ca = r[P_CA], cb = r[P_CB], cc = r[P_CC], ot = r[P_OT];
  const double det = ca * cc - cb * cb;
  if (!(det > 0.0)) return;
  const double qm = S[S_Q_MAX] * (1.0 + 2.0 * margin);
  const double hx = sqrt(qm * cc / det) + 1.0, hy = sqrt(qm * ca / det) + 1.0;
  int px0 = (int)floor(u - hx), px1 = (int)ceil(u + hx), py0 = (int)floor(v - hy), py1 = (int)ceil(v + hy);
  if (px0 < 0) px0 = 0;
  if (py0 < 0) py0 = 0;
  if (px1 > W - 1) px1 = W - 1;
  if (py1 > H - 1) py1 = H - 1;
  if (px0 > px1 || py0 > py1) return;
  const int tx0 = px0 / tile_w, tx1 = px1 / tile_w, ty0 = py0 / tile_h, ty1 = py1 / tile_h;
  const int ntx = tx1 - tx0 + 1;
  for (int k = 0; k < ntx * (ty1 - ty0 + 1); ++k) scratch[k] = 0;
  for (int py = py0; py <= py1; ++py)
    for (int px = px0; px <= px1; ++px) {
      const double dx = px + 0.5 - u, dy = py + 0.5 - v;
      const double q = ca * dx * dx + 2.0 * cb * dx * dy + cc * dy * dy;
      const double alpha = ot * exp(-0.5 * q);
      const int blend = q <= S[S_Q_MAX] && alpha >= S[S_ALPHA_MIN];
      const int near = rel_margin(q, S[S_Q_MAX]) < margin || rel_margin(alpha, S[S_ALPHA_MIN]) < margin;
      int* st = &scratch[(py / tile_h - ty0) * ntx + (px / tile_w - tx0)];
      if (blend && !near) *st = 1;
      else if (near && *st == 0) *st = 2;
    }
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      const int st = scratch[(ty - ty0) * ntx + (tx - tx0)];
      if (st) emit(ctx, ty * tiles_x + tx, st);
    }
  (void)tiles_y;
}

typedef struct { long count; tentry* out; int id, tile_offset; double depth; } tile_ctx;

static void count_sink(void* c, int tile, int status) {
  (void)tile; (void)status;
  ((tile_ctx*)c)->count++;
}

static void store_sink(void* c, int tile, int status) {
  tile_ctx* t = (tile_ctx*)c;
  tentry* e = &t->out[t->count++];
  e->tile = t->tile_offset + tile;
  e->depth = t->depth;
  e->id = t->id;
  e->status = status;
}

/*
 * The tile lists of one view (the binning step of the 3D splatting renderer, Sec. 3.1): every
 * (tile, Gaussian) pair of the visible Gaussians whose tile holds a blendable pixel centre (see
 * gaussian_tiles), ordered by (tile, depth, id); tile = tile_offset + ty * tiles_x + tx.  Writes the
 * pair's status (1 needed, 2 near a threshold) to out_status.  Returns the pair count, -1 if it
 * exceeds capacity, -2 on allocation failure.
 */
long orc_tile_lists(int n, const double* P, const double* cam, int tile_w, int tile_h, int tile_offset,
                    const double* S, double margin, long capacity, int* out_tile, int* out_id, int* out_status) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  if (tile_w <= 0 || tile_h <= 0 || W <= 0 || H <= 0) return -3;
  const int max_tiles = ((W + tile_w - 1) / tile_w + 1) * ((H + tile_h - 1) / tile_h + 1);
  long* cnt = (long*)calloc((size_t)(n > 0 ? n : 1) + 1, sizeof(long));
  if (!cnt) return -2;
  int err = 0;
#pragma omp parallel
  {
    int* scratch = (int*)malloc(sizeof(int) * (size_t)max_tiles);
    if (!scratch) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 256)
      for (int i = 0; i < n; ++i) {
        const double* r = P + (size_t)i * P_STRIDE;
        if (r[P_VISIBLE] == 0.0) continue;
        tile_ctx c = {0, NULL, i, tile_offset, r[P_DEPTH]};
        gaussian_tiles(r, W, H, tile_w, tile_h, S, margin, scratch, count_sink, &c);
        cnt[i + 1] = c.count;
      }
      free(scratch);
    }
  }
  if (err) { free(cnt); return -2; }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  const long total = cnt[n > 0 ? n : 0];
  if (total > capacity) { free(cnt); return -1; }
  tentry* e = (tentry*)malloc(sizeof(tentry) * (size_t)(total > 0 ? total : 1));
  if (!e) { free(cnt); return -2; }
#pragma omp parallel
  {
    int* scratch = (int*)malloc(sizeof(int) * (size_t)max_tiles);
    if (!scratch) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 256)
      for (int i = 0; i < n; ++i) {
        const double* r = P + (size_t)i * P_STRIDE;
        if (r[P_VISIBLE] == 0.0 || cnt[i + 1] == cnt[i]) continue;
        tile_ctx c = {0, e + cnt[i], i, tile_offset, r[P_DEPTH]};
        gaussian_tiles(r, W, H, tile_w, tile_h, S, margin, scratch, store_sink, &c);
      }
      free(scratch);
    }
  }
  free(cnt);
  if (err) { free(e); return -2; }
  qsort(e, (size_t)total, sizeof(tentry), tentry_cmp);
  for (long j = 0; j < total; ++j) {
    out_tile[j] = e[j].tile;
    out_id[j] = e[j].id;
    out_status[j] = e[j].status;
  }
  free(e);
  return total;
}

/* ------------------------------------------------------------------------------------------ */
/* Back-projection (Eq. 5) and grid pruning (Sec. 3.2)                                         */
/* ------------------------------------------------------------------------------------------ */
/*
 * X = G o pi^{-1}(p, D, K^{-1}): pixel centre (px + 0.5, py + 0.5), z-depth D, camera-space
 * point D K^{-1} (px + 0.5, py + 0.5, 1)^T, world point W^T (X_c - tau) with (W, tau) the
 * world->camera pose of the frame.  depth: H x W; xyz out: H*W x 3 (double).
 */
void orc_backproject(const double* cam, const float* depth, double* xyz) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const double D = depth[(size_t)py * W + px];
      const double xc[3] = {D * (px + 0.5 - cam[C_CX]) / cam[C_FX], D * (py + 0.5 - cam[C_CY]) / cam[C_FY], D};
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = xc[a] - cam[C_T + a];
      double* out = xyz + 3 * ((size_t)py * W + px);
      for (int a = 0; a < 3; ++a)
        out[a] = cam[C_R + 0 * 3 + a] * d[0] + cam[C_R + 1 * 3 + a] * d[1] + cam[C_R + 2 * 3 + a] * d[2];
    }
}

/*
 * The same Eq. 5 as a fixed sequence of correctly rounded float32 operations, the reading under
 * which the back-projected cloud (and so the voxel keys of the grid pruning) is bit-reproducible
 * on any IEEE-754 machine.  The camera is first rounded to float32.  Per pixel, every line one
 * rounding, evaluated in exactly this order and never contracted into a fused multiply-add:
 *   u_x = px + 0.5                      (exact)
 *   a_x = u_x - c_x                     n_x = a_x / f_x          X_c,x = D * n_x
 *   (the same for y with c_y, f_y)      X_c,z = D
 *   d_j = X_c,j - tau_j                 (j = x, y, z)
 *   X_a = (W_xa d_x + W_ya d_y) + W_za d_z   (two products, their sum, the third product, the sum)
 * depth: H x W float32; xyz out: H*W x 3 float32.
 */
void orc_backproject_f32(const double* cam, const float* depth, float* xyz) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  float R[9], tau[3];
  for (int k = 0; k < 9; ++k) R[k] = (float)cam[C_R + k];
  for (int k = 0; k < 3; ++k) tau[k] = (float)cam[C_T + k];
  const float fx = (float)cam[C_FX], fy = (float)cam[C_FY], cx = (float)cam[C_CX], cy = (float)cam[C_CY];
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const float D = depth[(size_t)py * W + px];
      volatile float ux = (float)px + 0.5f, uy = (float)py + 0.5f;
      volatile float ax = ux - cx, ay = uy - cy;
      volatile float nx = ax / fx, ny = ay / fy;
      volatile float xc[3];
      xc[0] = D * nx;
      xc[1] = D * ny;
      xc[2] = D;
      volatile float d[3];
      for (int a = 0; a < 3; ++a) d[a] = xc[a] - tau[a];
      float* out = xyz + 3 * ((size_t)py * W + px);
      for (int a = 0; a < 3; ++a) {
        volatile float p0 = R[0 * 3 + a] * d[0];
        volatile float p1 = R[1 * 3 + a] * d[1];
        volatile float s01 = p0 + p1;
        volatile float p2 = R[2 * 3 + a] * d[2];
        volatile float s = s01 + p2;
        out[a] = s;
      }
    }
}

typedef struct { int64_t k[4]; long idx; } pkey;

static int pkey_cmp(const void* pa, const void* pb) {
  const pkey* a = (const pkey*)pa;
  const pkey* b = (const pkey*)pb;
  for (int j = 0; j < 4; ++j)
    if (a->k[j] != b->k[j]) return (a->k[j] > b->k[j]) - (a->k[j] < b->k[j]);
  return (a->idx > b->idx) - (a->idx < b->idx);
}

typedef struct { long rep; long first, count; } vgroup;

static int vgroup_cmp(const void* pa, const void* pb) {
  const vgroup* a = (const vgroup*)pa;
  const vgroup* b = (const vgroup*)pb;
  return (a->rep > b->rep) - (a->rep < b->rep);
}

/*
 * Voxel index of a float32 coordinate: floor of ONE correctly rounded float32 product x * (1/S_v)
 * (the paper's "integer division with S_v", read as floor so that negative coordinates get cells
 * of the same size).  `volatile` keeps the product a separate float32 rounding step.
 */
static int64_t voxel_coord(float x, float inv) {
  volatile float p = x * inv;
  return (int64_t)floorf(p);
}

/*
 * Grid pruning of a point cloud: key = (dynamic flag, voxel coordinates); the flag makes static
 * and dynamic points never share a voxel, each with its own voxel size.  inv_dynamic = 0 leaves
 * the dynamic points unpruned (Sec. 4.1, Full model): each is its own group, kept whatever
 * min_support.  Points are grouped by
 * key; groups with fewer than min_support points are dropped; each kept voxel reports its point
 * count, the minimum point index (the representative), the centroid and the mean colour and
 * time.  Output is ordered by representative index.  rgb, t, dyn may be NULL (zero / static).
 * Returns the kept count, or -1 if it exceeds capacity, -2 on allocation failure.
 */
long orc_prune(long npts, const float* xyz, const float* rgb, const float* t, const uint8_t* dyn, float inv_static,
               float inv_dynamic, int min_support, long capacity, uint32_t* rep, int32_t* count, double* centroid,
               double* mean_rgb, double* mean_t, uint8_t* flag) {
  pkey* keys = (pkey*)malloc(sizeof(pkey) * (size_t)(npts > 0 ? npts : 1));
  if (!keys) return -2;
  for (long i = 0; i < npts; ++i) {
    const int f = dyn ? (dyn[i] != 0) : 0;
    const float inv = f ? inv_dynamic : inv_static;
    keys[i].k[0] = f;
    if (f && inv_dynamic == 0.0f) {  /* unpruned: a key of its own (no voxel key has k[1] = INT64_MIN) */
      keys[i].k[1] = INT64_MIN;
      keys[i].k[2] = i;
      keys[i].k[3] = 0;
    } else {
      keys[i].k[1] = voxel_coord(xyz[3 * i + 0], inv);
      keys[i].k[2] = voxel_coord(xyz[3 * i + 1], inv);
      keys[i].k[3] = voxel_coord(xyz[3 * i + 2], inv);
    }
    keys[i].idx = i;
  }
  qsort(keys, npts, sizeof(pkey), pkey_cmp);
  vgroup* g = (vgroup*)malloc(sizeof(vgroup) * (size_t)(npts > 0 ? npts : 1));
  if (!g) { free(keys); return -2; }
  long ng = 0;
  for (long i = 0; i < npts;) {
    long j = i;
    while (j < npts && memcmp(keys[j].k, keys[i].k, sizeof(keys[i].k)) == 0) ++j;
    if (j - i >= min_support || (keys[i].k[0] && inv_dynamic == 0.0f)) {
      g[ng].rep = keys[i].idx; /* sorted by idx within the group: first is the minimum */
      g[ng].first = i;
      g[ng].count = j - i;
      ++ng;
    }
    i = j;
  }
  if (ng > capacity) { free(keys); free(g); return -1; }
  qsort(g, ng, sizeof(vgroup), vgroup_cmp);
  for (long v = 0; v < ng; ++v) {
    double sx = 0, sy = 0, sz = 0, sr = 0, sg = 0, sb = 0, st = 0;
    for (long j = g[v].first; j < g[v].first + g[v].count; ++j) {
      const long p = keys[j].idx;
      sx += xyz[3 * p]; sy += xyz[3 * p + 1]; sz += xyz[3 * p + 2];
      if (rgb) { sr += rgb[3 * p]; sg += rgb[3 * p + 1]; sb += rgb[3 * p + 2]; }
      if (t) st += t[p];
    }
    const double cnt = (double)g[v].count;
    rep[v] = (uint32_t)g[v].rep;
    count[v] = (int32_t)g[v].count;
    centroid[3 * v] = sx / cnt; centroid[3 * v + 1] = sy / cnt; centroid[3 * v + 2] = sz / cnt;
    mean_rgb[3 * v] = sr / cnt; mean_rgb[3 * v + 1] = sg / cnt; mean_rgb[3 * v + 2] = sb / cnt;
    mean_t[v] = st / cnt;
    flag[v] = (uint8_t)keys[g[v].first].k[0];
  }
  free(keys);
  free(g);
  return ng;
}

/* The 4D covariance Sigma = R diag(s^2) R^T of one Gaussian (for the conditioning pins). */
void orc_cov4(int mode, const double* logscale4, const double* ql, const double* qr, double* Sigma) {
  const double mean4[4] = {0, 0, 0, 0}, opac = 0.0, rgb[3] = {0, 0, 0};
  double sh[45] = {0};
  const double cam[C_COUNT] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 5, 1, 1, 0, 0, 1, 1, 0};
  const double S[S_COUNT] = {0.99, 1.0 / 255.0, 1e-4, 9.0, 1.0 / 255.0, 0.2, 0.3, 1.3};
  gfwd f;
  forward_one(0, 0, mode, mean4, logscale4, ql, qr, &opac, rgb, sh, 0, NULL, cam, S, &f);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Sigma[4 * a + b] = f.Sig[a][b];
}
