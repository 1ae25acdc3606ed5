/*
 * FP64 CPU oracle for the articulated radiance-field render path of
 * InstantAvatar (arXiv 2212.10550).  TEST INFRASTRUCTURE ONLY: the test suite,
 * the smoke check and the benchmark's CPU-baseline leg call it; the CUDA library
 * never does, and the two share no code.
 *
 * Every function follows the paper's definition step by step, in fp64, with the
 * readings the paper leaves open written out where they are used:
 *   Sec. 3.1, Eq. 1-2        canonical field f: x -> (sigma, c), hash grid + MLP
 *   Sec. 3.1, Eq. 5-7        skinning-weight voxel grid, linear blend skinning
 *   Sec. 3.1 (Fast-SNARF)    correspondence x* by root finding of Eq. 7
 *   Sec. 3.2, Eq. 8          ray samples and front-to-back compositing
 *   Sec. 3.3                 per-pose occupancy grid (threshold + dilation),
 *                            empty-space skipping, normalised space
 *
 * Sample and ray indexing (pixel -> ray, ray -> slot positions, slot -> cell)
 * is computed in fp32 with a fixed operation order and no contraction, the same
 * definition the library documents, so the set of evaluated samples is a
 * bit-exact contract; everything downstream of a sample position is fp64.
 */
#ifndef IA_ORACLE_H
#define IA_ORACLE_H

#include <stdint.h>

#define OR_MAX_BONES 32
#define OR_MAX_LEVELS 32
#define OR_MAX_STARTS (OR_MAX_BONES + 4)

#ifdef __cplusplus
extern "C" {
#endif

/* Everything the path reads.  Arrays are caller-owned, fp64 copies of the fp32
 * inputs the library receives (exact), except the skeleton rest pose (fp64). */
typedef struct or_model {
  int nb;                    /* number of bones n_b (Eq. 5) */
  const int32_t *parent;     /* [nb]; -1 for the root; parents precede children */
  const double *rest;        /* [nb][3] rest-pose joint positions (canonical) */
  int rw;                    /* skinning grid vertices per axis */
  const double *skin;        /* [rw][rw][rw][nb], index ((z*rw+y)*rw+x)*nb+i */
  double cmin[3], cmax[3];   /* canonical box: skinning grid corners, hash-grid unit cube */
  float nmin[3], nmax[3];    /* normalised-space box: occupancy grid and ray clipping */
  int occ_res;               /* occupancy cells per axis */
  int L, F;                  /* hash levels, features per level */
  const int32_t *res;        /* [L] grid resolution per level */
  int log2_T;                /* hash table size per level, log2 */
  const double *table;       /* [entries][F], levels concatenated */
  int n_in, width;           /* MLP input (L*F) and hidden width */
  const double *W1, *b1, *W2, *b2, *W3, *b3; /* row-major [out][in] */
  int max_iter;              /* Broyden iterations per start */
  double tol;                /* Broyden convergence: |r|_2 < tol */
  int n_slots;               /* samples per ray N */
  double early_T;            /* stop a ray once T < early_T; <= 0 disables */
  double tau;                /* occupancy density threshold */
  int dilate;                /* occupancy dilation radius (cells, Chebyshev) */
  int quantize_fp32;         /* round bone transforms to fp32 (library storage) */
  int h0_analytic;           /* Broyden's initial inverse Jacobian: 0 = LBS with the weights
                                frozen at x0, (sum_i w_i(x0) R_i)^-1; 1 = the full analytic
                                J(x0)^-1 (weight gradients included) */
} or_model;

typedef struct or_pose {
  double B[OR_MAX_BONES][12];    /* world bone transforms [R | t], row-major 3x4 */
  double N[OR_MAX_BONES][12];    /* normalised-space transforms B_0^-1 B_k */
  double Ninv[OR_MAX_BONES][12]; /* inverses of N */
  float B0inv[12];               /* world -> normalised space, fp32 */
} or_pose;

typedef struct or_camera {
  float fx, fy, cx, cy;
  int width, height;
  float c2w[12];                 /* camera-to-world [R | c], row-major 3x4 */
} or_camera;

/* Per-sample diagnostics of the posed field f'(x') = f(x*). */
enum {
  OR_FLAG_CONV = 1,   /* a start's last residual check is within 2x of tol */
  OR_FLAG_BOX = 2,    /* a converged root lies within 1e-4 of the canonical box */
  OR_FLAG_DUP = 4,    /* two roots at a distance near the 1e-4 merge radius */
  OR_FLAG_TIE = 8,    /* best and runner-up density within 1e-3 relative */
  OR_FLAG_SING = 16,  /* a start's Jacobian determinant near the 1e-6 cutoff */
  OR_FLAG_TERM = 32,  /* transmittance within 1e-3 relative of the stopping threshold */
  OR_FLAG_PROP = 64,  /* the last proposed and the next logit within 0.05 */
};

typedef struct or_sample {
  double sigma;        /* density of the selected root (0 if none) */
  double rgb[3];
  double xstar[3];     /* selected canonical root */
  int start;           /* bone whose start produced it, -1 if none */
  int n_conv;          /* starts that converged inside the box */
  int n_unique;        /* distinct roots after merging */
  int flags;
  int iters;           /* Broyden updates summed over starts */
} or_sample;

/* cos a and sin a by their power series in fixed-order fp64 steps (reproducible
 * on any IEEE machine; used by the pose chain's Rodrigues rotations). */
void or_cos_sin(double a, double *c, double *s);
/* Sec. 3.1 / Sec. 3.3: bone transforms from axis-angle pose and root translation. */
void or_pose_chain(const or_model *m, const double *theta, const double *trans, or_pose *out);
/* Eq. 5-6: trilinear skinning weights at canonical x (and d w / d x, [nb][3]). */
void or_skin(const or_model *m, const double x[3], double *w, double *dw);
/* Eq. 7 in normalised space: y = sum_i w_i(x) N_i [x;1], and its Jacobian. */
void or_lbs(const or_model *m, const or_pose *p, const double x[3], double y[3], double *J);
/* Broyden root search of LBS(x) = xn from x0; returns 1 if it converged. */
int or_broyden(const or_model *m, const or_pose *p, const double xn[3], const double x0[3],
               double x[3], int *iters, double *res_norm, int *flags);
/* Newton polish to |r| < 1e-12 (fp64); returns the final residual norm. */
double or_polish(const or_model *m, const or_pose *p, const double xn[3], double x[3]);
/* Multi-start roots: distinct valid roots (polished), their starts; returns count. */
int or_roots(const or_model *m, const or_pose *p, const double xn[3], double *roots,
             int *starts, int *flags);
/* Roots from an explicit list of starts (x0s [ns][3], labels [ns]). */
int or_roots_from_starts(const or_model *m, const or_pose *p, const double xn[3], int ns,
                         const double *x0s, const int *labels, double *roots, int *starts, int *flags,
                         int *iters_sum, int *n_conv);
/* Max-density selection over a root set (fills s). */
void or_select_root(const or_model *m, int n, const double *roots, const int *starts, int flags,
                    int iters, int n_conv, or_sample *s);
/* Eq. 1-2: hash-grid encoding, MLP, density and colour at canonical x. */
void or_encode(const or_model *m, const double x[3], double *feat);
void or_mlp(const or_model *m, const double *feat, double out[4]);
void or_field(const or_model *m, const double x[3], double *sigma, double rgb[3]);
/* f'(x') at a normalised-space point: multi-start roots, max-density selection. */
void or_posed_field(const or_model *m, const or_pose *p, const double xn[3], or_sample *s);

/* fp32 indexing: normalised ray for pixel (u, v) and its clip interval. */
int or_ray(const or_model *m, const or_pose *p, const or_camera *c, int u, int v, float o[3],
           float d[3], float *t_near, float *t_far);
int or_cell(const or_model *m, const float x[3]);
void or_cell_center(const or_model *m, int cell, float x[3]);

/* Sec. 3.2: full image; rgb [H*W][3], alpha [H*W]; ray_flags and ray_nsamp
 * (occupied slots evaluated) may be NULL.  occ: packed bits of the grid. */
void or_render(const or_model *m, const or_pose *p, const or_camera *c, const uint32_t *occ,
               double *rgb, double *alpha, int *ray_flags, int *ray_nsamp, int64_t *ray_iters,
               int nthreads);
/* Same, for an explicit list of pixel indices (v*W+u). */
void or_render_pixels(const or_model *m, const or_pose *p, const or_camera *c,
                      const uint32_t *occ, int n, const int32_t *pix, double *rgb,
                      double *alpha, int *ray_flags, int *ray_nsamp, int nthreads);
/* Per pixel, a bitmask of the slots that fall in occupied cells:
 * bit i of mask[pixel * ceil(N/32) + i/32]. */
void or_march_mask(const or_model *m, const or_pose *p, const or_camera *c, const uint32_t *occ,
                   uint32_t *mask);
/* Sec. 3.3: density at every cell centre, then threshold + dilation + packing. */
void or_occupancy(const or_model *m, const or_pose *p, double *sigma, uint32_t *bits,
                  int nthreads);
/* Density at the centres of n given cells (a bounded part of the grid). */
/* Training-mode occupancy update (Sec. 3.3): d <- max(decay d, sigma(x_c)) with
 * x_c = norm_min + (c + jitter[c]) * cell size (jitter NULL = centres); bits of d. */
void or_occupancy_ema(const or_model *m, const or_pose *p, const float *jitter, double decay, double *d,
                      uint32_t *bits, int nthreads);
void or_occupancy_cells(const or_model *m, const or_pose *p, int n, const int32_t *cells,
                        double *sigma, int nthreads);
void or_occ_bits(int R, int dilate, double tau, const double *sigma, uint32_t *bits);
void or_occ_bits_f32(int R, int dilate, float tau, const float *sigma, uint32_t *bits);
/* Training step (oracle_grad.c): L2 loss over world rays of several poses and
 * its fp64 reverse-mode gradient, including the implicit-function gradient
 * through the root to the skinning grid and the bone transforms N. */
/* Loss set of Sec. 3.4 per ray, averaged over the rays:
 *   w_rgb * (huber ? rho_delta(|C - C_gt|_2) : sum_channels (C - C_gt)^2)     (Eq. 9)
 * + w_alpha * |alpha - alpha_gt|                                              (Eq. 10)
 * + w_hard * (-log(exp(-|alpha|) + exp(-|alpha - 1|)) + log(1 + exp(-1)))    (Eq. 11)
 * with alpha = 1 - final transmittance and rho_delta the Huber function
 * (r^2 / 2 below delta, delta (r - delta / 2) above). */
typedef struct or_loss {
  int huber;
  double delta;
  double w_rgb, w_alpha, w_hard;
  const double *alpha_target; /* [n], read when w_alpha != 0 */
} or_loss;

double or_train(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                const float *o, const float *d, const int32_t *pose_id, const double *target,
                double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                double *g_bones, int nthreads);
/* Learned correspondence proposal (oracle_prop.c; not part of the paper). */
typedef struct or_prop {
  int L, log2_T;              /* hash grid over the normalised box */
  const int32_t *res;         /* [L] */
  const double *table;        /* [entries][2] */
  int n_in, width, n_out;     /* n_in = 2L + 3 nb, n_out = nb + 3 */
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4; /* row-major [out][in] */
  int top_k;
  double offset_weight;
} or_prop;
void or_prop_encode(const or_model *m, const or_prop *q, const double xn[3], double *feat, long *entry,
                    double *weight);
void or_prop_forward(const or_model *m, const or_prop *q, const double xn[3], const double *theta,
                     double *out);
int or_prop_label(const or_model *m, const or_pose *p, const double xs[3], const double xn[3],
                  double offset[3]);
long or_prop_mlp_count(const or_prop *q);
double or_prop_loss_grad(const or_model *m, const or_prop *q, int n, const float *x, const int32_t *pose_id,
                         const double *theta_all, const int32_t *label, const double *target,
                         double *g_table, double *g_mlp);
void or_posed_field_prop(const or_model *m, const or_pose *p, const or_prop *q, const double *theta,
                         const double xn[3], or_sample *s, int *fallback);
/* or_render_pixels with the proposal choosing every sample's starts (Sec. 3.2
 * compositing, each sample's field from or_posed_field_prop; theta [nb][3] the
 * pose's axis-angles); ray_fallbacks [n] (may be NULL) counts each ray's
 * samples whose proposed starts found no valid root, so that the search over
 * every bone ran. */
void or_render_pixels_prop(const or_model *m, const or_pose *p, const or_prop *q, const double *theta,
                           const or_camera *c, const uint32_t *occ, int n, const int32_t *pix, double *rgb,
                           double *alpha, int *ray_flags, int *ray_nsamp, int *ray_fallbacks, int nthreads);
/* or_train with the proposal choosing each sample's starts; theta_all
 * [n_poses][nb][3] axis-angles of the poses (the proposal's pose input);
 * ray_fallbacks [n] (may be NULL) counts each ray's samples that fell back to
 * the search over every bone. */
double or_train_prop(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                     const float *o, const float *d, const int32_t *pose_id, const double *target,
                     double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                     double *g_bones, int nthreads, const or_prop *q, const double *theta_all,
                     int *ray_fallbacks);

/* or_train with the loss set lc (NULL = or_train's L2). */
double or_train_loss(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                     const float *o, const float *d, const int32_t *pose_id, const double *target,
                     double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                     double *g_bones, int nthreads, const or_loss *lc);

/* The same backward for dL/dC [n][3] and dL/dalpha [n] (NULL: zero) given by
 * the caller (a loss built elsewhere on the rendered colour and opacity);
 * rgb_out [n][3], alpha_out [n] (alpha = 1 - final transmittance), ray_flags
 * and the gradients (overwritten) as or_train; any output may be NULL. */
void or_train_upstream(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                       const float *o, const float *d, const int32_t *pose_id, const double *up_rgb,
                       const double *up_alpha, double *rgb_out, double *alpha_out, int *ray_flags, double *g_table,
                       double *g_mlp, double *g_skin, double *g_bones, int nthreads);

/* Occupancy-based density regulariser (Eq. 12) at n normalised-space points x
 * [n][3] fp32 of poses pose_id [n]: L = weight / n * sum of sigma(x) over the
 * points whose cell (or_cell) is empty in occ.  Its gradient is ADDED to the
 * four buffers (dL/dsigma = weight / n, dL/dc = 0 through the same backward as
 * the photometric loss).  point_flags [n] may be NULL. */
double or_density_reg(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                      const float *x, const int32_t *pose_id, double weight, int *point_flags, double *g_table,
                      double *g_mlp, double *g_skin, double *g_bones);
/* Brute-force root set: Newton from every point of an n^3 canonical lattice. */
int or_bruteforce_roots(const or_model *m, const or_pose *p, const double xn[3], int n,
                        double seed_thresh, double *roots, int max_roots);

#ifdef __cplusplus
}
#endif
#endif
