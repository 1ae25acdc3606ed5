/*
 * ia.h — C ABI of the B300 (sm_103a) articulated radiance-field render path.
 *
 * The library computes InstantAvatar's per-sample render path (arXiv
 * 2212.10550): a canonical radiance field f: x -> (sigma, c) held in a
 * multiresolution hash grid decoded by a small MLP (Sec. 3.1, Eq. 1-2), a
 * skinning-weight voxel grid with linear blend skinning x' = sum_i w_i(x) B_i x
 * (Sec. 3.1, Eq. 5-7), the canonical correspondence x* of a posed point found by
 * bone-wise Broyden root finding (Sec. 3.1, Fast-SNARF), volume rendering
 * C = sum_i alpha_i prod_{j<i}(1 - alpha_j) c_i with alpha_i = 1 - exp(-sigma_i
 * delta_i) (Sec. 3.2, Eq. 8; the sign of the exponent is printed without its
 * minus in the paper), and a per-pose occupancy grid that skips empty space in a
 * normalised space with the root's rigid motion removed (Sec. 3.3).
 *
 * Conventions shared by every call:
 *  - Every call returns an ia_status and never aborts; on failure
 *    ia_last_error(ctx) holds a message.  Arguments are checked on the host
 *    before any launch; invalid ones return IA_ERR_ARG and launch nothing.
 *  - Pointers marked "host or device" may point to either (the library copies
 *    through unified addressing).  Pointers marked "device" must be device
 *    memory of the context's GPU.  Output pointers of ia_render may be host
 *    memory: the call then renders into library scratch, copies back and
 *    synchronises the stream before returning.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it; calls returning device results do not
 *    synchronise unless stated.
 *  - The caller keeps ownership of everything it passes; the library copies what
 *    it keeps.  Parameters (hash table, MLP) and per-pose state are owned by the
 *    context and freed by ia_destroy.
 *  - Device loops are bounded by construction (starts <= n_bones, Broyden
 *    iterations <= broyden_max_iter, slots <= max_samples); non-convergence of a
 *    start is a normal outcome, counted in ia_render_stats, not an error.
 *  - Layouts are row-major.  A 3x4 transform [R | t] is 12 floats, row by row.
 */
#ifndef IA_H
#define IA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IA_MAX_BONES 32
#define IA_MAX_LEVELS 16

typedef struct ia_ctx ia_ctx;

typedef enum ia_status {
  IA_OK = 0,
  IA_ERR_ARG = 1,   /* invalid argument (checked on the host) */
  IA_ERR_STATE = 2, /* call out of order (e.g. render before set_pose) */
  IA_ERR_CUDA = 3,  /* a CUDA runtime error; message in ia_last_error */
  IA_ERR_OOM = 4,   /* device allocation failed */
  IA_ERR_LIMIT = 5  /* a documented size limit was exceeded */
} ia_status;

typedef enum ia_precision { IA_FP32 = 0, IA_FP16 = 1, IA_BF16 = 2 } ia_precision;

typedef enum ia_occ_mode {
  IA_OCC_POSE = 0,  /* rebuild the render grid for one pose (Sec. 3.3, inference) */
  IA_OCC_UNION = 1  /* OR one pose's grid into the training grid (union over frames) */
} ia_occ_mode;

/* Sizes of the path.  level_res[l] = floor(N_min * b^l) is computed by the
 * caller once (the paper defers the schedule to Instant-NGP) so that every
 * consumer agrees on the integers. */
typedef struct ia_config {
  int n_levels;                  /* L, 1..16 */
  int n_features;                /* F per level; must be 2 */
  int log2_table;                /* T = 2^log2_table entries per hashed level, 10..24 */
  int level_res[IA_MAX_LEVELS];  /* grid resolution N_l per level, >= 2 */
  int mlp_width;                 /* hidden width; must be 64 (two hidden layers, ReLU) */
  int max_samples;               /* ray slots N, 1..1024 */
  int broyden_max_iter;          /* Broyden updates per start, 1..64 */
  float broyden_tol;             /* converged when |LBS(x) - x'|_2 < tol */
  int occ_res;                   /* occupancy cells per axis R, multiple of 4, 4..256 */
  float occ_tau;                 /* occupied when density > tau */
  int occ_dilate;                /* dilation radius in cells (Chebyshev), 0..4 */
  float early_stop_T;            /* stop a ray once transmittance < this; <= 0 disables */
  int precision;                 /* ia_precision of the MLP and hash features */
} ia_config;

typedef struct ia_camera {
  float fx, fy, cx, cy;          /* pinhole intrinsics (pixels) */
  int width, height;             /* image size; pixel (u, v) has ray id v * width + u */
  float c2w[12];                 /* camera-to-world [R | centre], OpenCV axes */
} ia_camera;

/* Counters of one ia_render / ia_update_occupancy call (summed over the grid).
 * With the wavefront render path every slot of a hit ray is marched and every
 * kept sample searched, behind the early-termination point too (compositing
 * still stops there); the fused path stops marching a ray once it stops. */
typedef struct ia_render_stats {
  int64_t rays;              /* rays launched */
  int64_t hit_rays;          /* rays whose clipped interval is non-empty */
  int64_t marched_slots;     /* slots tested against the occupancy grid */
  int64_t occupied_samples;  /* slots in occupied cells reached (evaluated or culled) */
  int64_t starts;            /* Broyden starts run */
  int64_t broyden_iters;     /* Broyden updates run (summed over starts) */
  int64_t converged;         /* starts that converged inside the canonical box */
  int64_t roots;             /* distinct roots kept (one field evaluation each) */
  int64_t early_stopped;     /* rays stopped by the transmittance threshold */
  int64_t proposed;          /* samples whose first starts came from the proposal network */
  int64_t fallbacks;         /* of those, samples that fell back to every bone-wise start */
  int64_t culled;            /* render: occupied samples, occupancy: cells, whose point can
                                have no root (density 0 without a search; see
                                ia_update_occupancy) */
  int64_t grid_gathers;      /* search evaluations of M(x) that read their cell's 8 corner
                                records from the blended grid: every start and update on
                                the fused schedule; on the wavefront, those whose cell
                                differs from the previous evaluation's (the others reuse
                                the records a lane holds) */
  int64_t rooted_samples;    /* searched samples with a selected root (wavefront schedule;
                                0 on the fused one) */
  int64_t point_culled;      /* proposal search, wavefront render: samples whose proposed
                                starts found no root and whose point lies in no grown
                                image box of a canonical skinning cell (the culling bound
                                point by point): density 0 without the fallback search */
} ia_render_stats;

/* Create a context on the current CUDA device.  cfg is copied. */
ia_status ia_create(const ia_config *cfg, ia_ctx **out);
/* Free everything the context owns (NULL is allowed).  Waits for its work. */
void ia_destroy(ia_ctx *ctx);
/* Message of the last failed call on this context (or of the last failed
 * ia_create when ctx is NULL).  Library-owned, valid until the next call. */
const char *ia_last_error(const ia_ctx *ctx);
/* Library version string. */
const char *ia_version(void);

/* Skeleton and skinning-weight grid (Sec. 3.1, Eq. 5-7).
 *  parent      [n_bones] int32, host; -1 for bone 0 (the root), parent[k] < k.
 *  rest_joints [n_bones][3] fp64, host; canonical rest-pose joint positions.
 *  skin_grid   [skin_res]^3 x [n_bones] fp32, host or device, index
 *              ((z * skin_res + y) * skin_res + x) * n_bones + i; vertex (x,y,z)
 *              sits at canon_min + (x,y,z) / (skin_res - 1) * (canon_max - canon_min).
 *  canon_min/max  canonical box: skinning grid corners, hash-grid unit cube, and
 *              the region where a root counts as valid.
 *  norm_min/max   normalised-space box: the occupancy grid's extent; rays are
 *              clipped to it.
 * n_bones 1..32, skin_res 2..256.  Invalidates per-pose state. */
ia_status ia_set_skeleton(ia_ctx *ctx, int n_bones, const int32_t *parent,
                          const double *rest_joints, const float *skin_grid, int skin_res,
                          const float canon_min[3], const float canon_max[3],
                          const float norm_min[3], const float norm_max[3]);

/* Number of fp32 values of the hash table ([entries][F], levels concatenated;
 * level l holds min((N_l+1)^3, T) entries, dense vertex (i,j,k) at
 * i + (N_l+1)(j + (N_l+1) k), hashed vertex at (i ^ 2654435761 j ^ 805459861 k)
 * mod T) and of the packed MLP (W1 [64][L*F], b1 [64], W2 [64][64], b2 [64],
 * W3 [4][64], b3 [4], each row-major [out][in]). */
ia_status ia_param_sizes(const ia_ctx *ctx, int64_t *table_floats, int64_t *mlp_floats);
/* Load / read the canonical field's parameters (Eq. 1-2); host or device. */
ia_status ia_set_params(ia_ctx *ctx, const float *table, const float *mlp, void *stream);
ia_status ia_get_params(ia_ctx *ctx, float *table, float *mlp, void *stream);

/* Bone transforms for n_poses poses (Sec. 3.1 B, Sec. 3.3 normalised space),
 * composed down the kinematic tree in fp64 on the GPU:
 *   R_k = Rodrigues(axis_angle[p][k]);  G_0 = [R_0 | j_0];
 *   G_k = G_parent(k) [R_k | j_k - j_parent(k)];  B_k = G_k [I | -j_k] + t_root;
 *   N_k = B_0^-1 B_k  (normalised space), stored fp32 with N_k^-1 and B_0^-1.
 * Also builds, per pose, the blended transform grid M(v) = sum_i W(v, i) N_i
 * (fp32, 12 floats per skinning-grid vertex), exact under trilinear
 * interpolation because LBS is linear in the weights.
 *  axis_angle [n_poses][n_bones][3] fp64, root_trans [n_poses][3] fp64, host.
 * n_poses 1..4096.  Replaces previously set poses. */
ia_status ia_set_pose(ia_ctx *ctx, int n_poses, const double *axis_angle,
                      const double *root_trans, void *stream);
/* Read back pose p's transforms: N and Ninv [n_bones][12], B0inv [12] (any may
 * be NULL); host or device.  Synchronises the stream. */
ia_status ia_get_transforms(ia_ctx *ctx, int pose, float *N, float *Ninv, float *B0inv,
                            void *stream);

/* Occupancy grid of pose p (Sec. 3.3): density of the posed field at every cell
 * centre norm_min + (c + 1/2) * (norm_max - norm_min) / R (fp32, fixed order),
 * then occupied = density > occ_tau, dilated by occ_dilate cells, packed so that
 * cell b = x + R (y + R z) is bit b % 32 of word b / 32.  IA_OCC_POSE replaces
 * the render grid; IA_OCC_UNION ORs the result into the training grid.  The
 * cells take the context's search (ia_set_search).  Culling (on by default,
 * ia_set_occupancy_culling) searches only the cells whose query point can have
 * a root: a root lies in the canonical box, and the LBS image of each
 * skinning-grid cell lies in the bounding box of its corner images grown by the
 * variation of the blended rotation over the cell (times the cell's edges), the
 * Broyden tolerance and a rounding margin.  The boxes are recorded per 4x4x4
 * sub-cells of each occupancy cell; a point whose sub-cell meets no box gets
 * density 0 without a search, which is what the search would return.  The
 * masks also serve ia_render of the same pose (until ia_set_pose or a skinning
 * update changes its blended grid), whose samples in such sub-cells are not
 * searched.  Densities are the same with culling on or off (each cell's starts
 * are merged in start order either way).  The search and field run on the
 * render's per-sample kernels; the first call allocates their arrays for R^3
 * query points (0.1 GB at 64^3 and 24 bones, 0.2 GB with the proposal search).
 * With the proposal search (IA_OCC_POSE, culling on) the call also records each
 * skinning cell's grown box ((skin_res - 1)^3 x 32 B, allocated by
 * ia_set_skeleton) and, per occupied cell of the new grid, up to 64 of the boxes
 * meeting it (R^3 x 65 ints, 68 MB at 64^3, allocated by ia_create): ia_render
 * of the same pose then skips the fallback search of a sample whose proposed
 * starts found no root and whose point lies in none of its cell's boxes (no
 * root is possible there), counted in ia_render_stats.point_culled.  The lists
 * follow the grid: ia_set_occupancy and ia_occupancy_from_density rebuild them
 * for the new bits; ia_set_pose, a skinning-grid update and
 * ia_update_occupancy_static drop them.
 *  sigma_out [R^3] fp32 device or NULL; bits_out [R^3 / 32] uint32 device or NULL. */
ia_status ia_update_occupancy(ia_ctx *ctx, int pose, int mode, float *sigma_out,
                              uint32_t *bits_out, ia_render_stats *stats, void *stream);
/* Training-mode occupancy (Sec. 3.3, training stage): one grid for the whole
 * sequence, kept in the normalised space.  Each call queries the posed field of
 * frame `pose` at one point per cell, x = norm_min + (c + u) * (norm_max -
 * norm_min) / R (fp32, fixed order; u = jitter[c] in [0, 1)^3 from the caller's
 * random draw, or the cell centre when jitter is NULL), folds it into the
 * context's running density d <- max(decay * d, sigma) (the paper's averaging
 * of old and new values read as a decaying maximum; d starts at 0 when the context is
 * created, and decay 0 restarts it), and replaces the training grid (the one
 * ia_train_step uses with IA_OCC_UNION) by d thresholded at occ_tau and dilated.
 *  jitter [R^3][3] fp32 device or NULL; decay in [0, 1]; density_out [R^3] fp32
 *  device (the updated d) or NULL; bits_out [R^3 / 32] uint32 device or NULL. */
ia_status ia_update_occupancy_ema(ia_ctx *ctx, int pose, const float *jitter, float decay, float *density_out,
                                  uint32_t *bits_out, ia_render_stats *stats, void *stream);

/* Threshold + dilation + packing alone, from a caller density array.
 *  sigma [R^3] fp32 device; bits_out [R^3 / 32] uint32 device.  Also installs
 *  the result as the render grid. */
ia_status ia_occupancy_from_density(ia_ctx *ctx, const float *sigma, uint32_t *bits_out,
                                    void *stream);
/* Install caller bits as the render grid ([R^3 / 32] uint32, host or device). */
ia_status ia_set_occupancy(ia_ctx *ctx, const uint32_t *bits, void *stream);

/* Posed field f'(x') = f(x*) at n normalised-space points of pose p (Sec. 3.1):
 * bone-wise Broyden starts x0 = N_k^-1 x', validity = converged and inside the
 * canonical box, one Newton polish of each distinct root, the root with the
 * highest density selected.  x [n][3] fp32 device; sigma [n], rgb [n][3],
 * x_canon [n][3], start [n] int32 (bone of the selected root, -1 if none) device,
 * any output may be NULL. */
ia_status ia_query_posed(ia_ctx *ctx, int pose, int n, const float *x, float *sigma,
                         float *rgb, float *x_canon, int32_t *start, void *stream);
/* Canonical field f(x) (Eq. 1-2) at n canonical points; x [n][3], sigma [n],
 * rgb [n][3] fp32 device. */
ia_status ia_query_canonical(ia_ctx *ctx, int n, const float *x, float *sigma, float *rgb,
                             void *stream);

/* Render pose p through camera cam (Sec. 3.2-3.3): for pixel (u, v) the ray
 * d = normalize(R_c [(u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1]) from the camera
 * centre, mapped to normalised space, clipped to the normalised box [t_n, t_f],
 * N midpoint slots t_i = t_n + (i + 1/2) delta, delta = (t_f - t_n) / N (all
 * fp32, fixed order, no contraction); slots in empty cells are skipped; the
 * others are composited front to back with alpha_i = 1 - exp(-sigma_i delta);
 * a ray stops once its transmittance falls below early_stop_T.
 *  rgb [H*W][3], alpha [H*W] fp32 (alpha = 1 - final transmittance), device or
 *  host (see conventions).  stats may be NULL (host struct).
 *  With the default render path (ia_set_render_path) the call waits on its
 *  stream once, after the march, for the frame's sample count; the kernels
 *  after it are queued without waiting (device outputs).  The first frames,
 *  and any frame with more samples than the context's arrays hold, allocate. */
ia_status ia_render(ia_ctx *ctx, int pose, const ia_camera *cam, float *rgb, float *alpha,
                    ia_render_stats *stats, void *stream);

/* How ia_render schedules the frame; results are the same up to the merge
 * order of the fused path's shared queues (within rounding).
 *  IA_RENDER_WAVEFRONT (default): a sequence of kernels over arrays -- march
 *    (each ray's kept samples, contiguous), the proposal (proposal search),
 *    the search with one thread per (sample, start) item, the fallback starts
 *    of the proposal search as a second wave, the field per sample, then
 *    compositing per ray.  The samples' count is read back after the march
 *    (so ia_render waits on its stream there), and the context keeps arrays
 *    for the frame's samples (~0.5 KB per sample with 24 bones).  Samples
 *    behind the point where early termination stops a ray are evaluated too.
 *  IA_RENDER_FUSED: one persistent kernel per frame, each warp marching,
 *    searching, evaluating and compositing its own pool of 32 rays; rays stop
 *    at early termination; no read-back. */
typedef enum ia_render_path { IA_RENDER_FUSED = 0, IA_RENDER_WAVEFRONT = 1 } ia_render_path;
ia_status ia_set_render_path(ia_ctx *ctx, int path);

/* A batch of training rays (all device pointers), and optionally the points of
 * the occupancy-based density regulariser (Eq. 12). */
typedef struct ia_batch {
  int n_rays;                /* 1..2^24 */
  const float *origin;       /* [n][3] world-space ray origins */
  const float *direction;    /* [n][3] world-space unit directions */
  const int32_t *pose;       /* [n] index of a pose set by ia_set_pose */
  const float *target;       /* [n][3] target colours */
  int n_reg;                 /* 0..2^24 regulariser points (0: no regulariser) */
  const float *reg_x;        /* [n_reg][3] points in the normalised space of their pose */
  const int32_t *reg_pose;   /* [n_reg] pose of each point */
  float reg_weight;          /* weight of the regulariser term */
  const float *alpha_target; /* [n] mask values (Eq. 10); read when the loss has w_alpha != 0 */
} ia_batch;

/* The per-ray loss of ia_train_step (Sec. 3.4), averaged over the rays:
 *   w_rgb * (rgb_loss == IA_LOSS_HUBER ? rho(|C - C_gt|_2) : sum_channels (C - C_gt)^2)   (Eq. 9)
 * + w_alpha * |alpha - alpha_gt|                                                       (Eq. 10)
 * + w_hard * (-log(exp(-|alpha|) + exp(-|alpha - 1|)) + log(1 + exp(-1)))              (Eq. 11)
 * with alpha = 1 - the ray's final transmittance and rho the Huber function with
 * threshold huber_delta (r^2 / 2 below, huber_delta (r - huber_delta / 2)
 * above).  The paper prints no weights or threshold; a new context uses
 * {IA_LOSS_L2, 0, 1, 0, 0}. */
typedef enum ia_rgb_loss { IA_LOSS_L2 = 0, IA_LOSS_HUBER = 1 } ia_rgb_loss;
typedef struct ia_loss {
  int rgb_loss;       /* ia_rgb_loss */
  float huber_delta;  /* > 0 for IA_LOSS_HUBER */
  float w_rgb, w_alpha, w_hard;
} ia_loss;
ia_status ia_set_loss(ia_ctx *ctx, const ia_loss *loss);

/* Floats of the skinning-grid and bone-transform gradients of ia_train_step
 * for the current skeleton and poses: skin_res^3 * n_bones and
 * n_poses * n_bones * 12 (either pointer may be NULL). */
ia_status ia_grad_sizes(const ia_ctx *ctx, int64_t *skin_floats, int64_t *bone_floats);

/* Gradient buffers (device, caller-owned, overwritten by each step).  table must
 * be 8-byte aligned (IA_ERR_ARG otherwise); a 16-byte aligned skin with n_bones
 * a multiple of 4 takes the skinning-grid gradient four bones per atomic. */
typedef struct ia_grads {
  float *table;   /* [entries][F], same layout as the hash table */
  float *mlp;     /* packed like the MLP of ia_set_params */
  float *skin;    /* [skin_res^3][n_bones], same layout as the skinning grid */
  float *bones;   /* [n_poses][n_bones][12]: d loss / d N_k of each pose (row-major [R | t]) */
} ia_grads;

/* One differentiable training step (Sec. 3.2, Sec. 3.4 with an L2 photometric
 * loss): every ray is mapped into the normalised space of its pose, its slots
 * in occupied cells (occ_grid: IA_OCC_POSE = the render grid, IA_OCC_UNION = the
 * training grid) are evaluated with the posed field and composited front to
 * back (no early termination), and the loss set by ia_set_loss (by default
 *   loss = (1 / n) sum_rays sum_channels (C - target)^2)
 * is added to *loss (device scalar; the caller zeroes it).  The backward is
 * exact reverse mode: compositing, activations, MLP, hash-table scatter-add, and
 * the implicit-function gradient through the root x* of LBS(x*) = x' (Eq. 7):
 * with lambda = J(x*)^-T dL/dx* (J the analytic Jacobian),
 *   dL/dN_k = -lambda w_k(x*) [x*;1]^T,  dL/dW(v, k) = -c_v(x*) lambda . N_k [x*;1].
 * The selected root is treated as constant.  rgb_out [n][3] (device) may be
 * NULL.  Workspace for n_rays * max_samples samples (about 1.2 KB each in fp32,
 * 0.8 KB in fp16 / bf16, plus the search's item results: 16 B per start, i.e.
 * 384 B per sample with every bone as a start, 32 B with the proposal's two
 * and 384 B more for its fallback) is allocated by the context on first use
 * and grown when a larger batch comes.  With the proposal search and culling on,
 * the first step after the poses change also records every pose's grown boxes
 * and, per cell of the grid, up to 64 of the boxes meeting it (per pose 8 MB of
 * boxes and 68 MB of lists at 64^3; skipped when the lists of all poses would
 * pass 4 GiB): a sample whose proposed starts found no root and whose point
 * lies in none of at most 16 listed boxes of its cell skips its fallback search.
 *
 * Precision (Sec. 3.4 trains in half precision): with IA_FP16 / IA_BF16 the
 * forward uses the reduced-precision field (fp16 hash features, tensor-core MLP),
 * the MLP backward runs on fp16 / bf16 operands with fp32 accumulation, the
 * weight gradients are one tensor-core GEMM over the samples, and every
 * gradient is delivered in fp32 against the fp32 master parameters.  fp16 uses
 * a dynamic loss scale S (initially 2^14): the output gradient is multiplied by
 * S before the MLP backward and divided out of every result.  If a scaled
 * gradient leaves the fp16 range, the step is skipped: all four gradient
 * buffers are zeroed and S halves; after 1000 clean steps S doubles (at most
 * 2^24).  bf16 keeps S = 1.  ia_loss_scale reports S and whether the last step
 * was skipped.
 *
 * Regulariser (Eq. 12): with n_reg > 0 the loss gains
 *   reg_weight / n_reg * sum of sigma(x) over the points x whose cell is empty
 * in the occupancy grid the step uses (density is non-negative, so |sigma| =
 * sigma); those points are evaluated with the posed field like the ray samples
 * and their gradient (dL/dsigma = reg_weight / n_reg) goes through the same
 * backward.  Points with an invalid pose or in occupied cells contribute nothing.
 *
 * Search: with ia_set_search(ctx, IA_SEARCH_PROPOSAL) (fp16 / bf16 only) each
 * sample's correspondence search starts from the proposal's top_k bones of the
 * sample's own pose and falls back to every bone-wise start when they find no
 * valid root, as in ia_render; the backward is unchanged (the selected root is
 * a constant of the gradient). */
ia_status ia_train_step(ia_ctx *ctx, const ia_batch *batch, int occ_grid, float *loss, float *rgb_out,
                        const ia_grads *grads, void *stream);

/* The training step split in two, for a loss computed by the caller (Sec. 3.2:
 * the rendering is differentiable, so any loss on the rendered colour and
 * opacity can be trained; Sec. 3.4 uses Eq. 9-12).
 *
 * ia_train_forward renders the batch's rays as ia_train_step does (normalised
 * space of each ray's pose, occupied slots of occ_grid, posed field, front-to-
 * back compositing of every sample, no early termination) and writes
 *  rgb_out [n][3] (device) and alpha_out [n] (device or NULL; alpha = 1 - the
 *  ray's final transmittance).
 * table / mlp (device, fp32, laid out as in ia_set_params; NULL = the
 * context's own) are the canonical field's parameters for this forward and its
 * backward; they are read in place and must stay unchanged until the
 * backward has run (a reduced-precision context converts a caller table into
 * a context-owned fp16 copy).  The batch's target, alpha_target and
 * regulariser are not used (n_reg must be 0).  The per-sample state (sample
 * positions, selected roots, density and colour) stays in the context's
 * training workspace; per-sample activations are not kept.
 *
 * ia_train_backward differentiates that forward: given the caller's
 *  grad_rgb [n][3] = dL/dC and grad_alpha [n] = dL/dalpha (device; grad_alpha
 *  may be NULL for zero)
 * it runs the reverse compositing sweep and the same hand-written backward as
 * ia_train_step (activations recomputed from the roots, MLP, hash-table
 * scatter-add, implicit-function gradient through the root to the skinning
 * grid and the bone transforms N_k; fp16 / bf16 with the dynamic loss scale),
 * overwriting the four buffers of g (layouts as ia_grads).  It may be called
 * more than once for one forward.  IA_ERR_STATE when there is no forward to
 * differentiate: none ran, or ia_train_step, ia_set_pose, ia_set_skeleton, a
 * skinning-grid ia_adam_step, or (when the forward read the context's own
 * parameters) ia_set_params / ia_adam_step ran since.  One forward is kept per
 * context: forwards for two batches need two contexts. */
ia_status ia_train_forward(ia_ctx *ctx, const ia_batch *batch, int occ_grid, const float *table, const float *mlp,
                           float *rgb_out, float *alpha_out, void *stream);
ia_status ia_train_backward(ia_ctx *ctx, const float *grad_rgb, const float *grad_alpha, const ia_grads *grads,
                            void *stream);

/* Counters of the last ia_train_step (host struct; waits on `stream`): rays,
 * rays that cross the normalised box (hit_rays), their slots (marched_slots),
 * occupied samples, Broyden starts / iterations / converged chains / distinct
 * roots, and with the proposal search the proposed samples and fallbacks.
 * early_stopped is 0 (training composites every sample). */
ia_status ia_train_stats(ia_ctx *ctx, ia_render_stats *stats, void *stream);

/* One Adam step (beta1, beta2, eps; bias-corrected) on the context's canonical
 * field, hash table and MLP (the fp32 masters; the fp16 shadow table is
 * refreshed), from gradients laid out as ia_grads' table and mlp (device).
 * With g_skin (ia_grads' skin layout, device; NULL keeps the grid fixed) the
 * skinning-weight grid is a learnable parameter too (unconstrained: its rows
 * are not renormalised), and every pose's blended transform grid is rebuilt
 * from it.  The moments live in the context and restart with ia_set_params /
 * ia_set_skeleton.  In an fp16 context a step that ia_train_step skipped on
 * overflow changes nothing.  The bone transforms (poses) are inputs. */
ia_status ia_adam_step(ia_ctx *ctx, const float *g_table, const float *g_mlp, const float *g_skin, float lr,
                       float beta1, float beta2, float eps, void *stream);

/* The loss scale S after the last ia_train_step (host float) and whether that
 * step was skipped (host int32, 1 = skipped: a scaled gradient or activation
 * overflowed, or the tensor-core weight-gradient reduction gave up; every
 * gradient buffer of a skipped step is zeroed and ia_adam_step leaves the
 * parameters alone); either may be NULL, not both.  Waits on `stream`.  fp32
 * contexts report S = 1, never skipped.  Returns IA_ERR_CUDA (after filling
 * both outputs) if the last step's weight-gradient reduction gave up waiting
 * on its copy / MMA pipeline (see ia_set_wait_limit); ia_train_stats reports
 * the same. */
ia_status ia_loss_scale(ia_ctx *ctx, float *scale, int32_t *skipped, void *stream);

/* Bound, in nanoseconds, on every wait of the reduced-precision training step's
 * tensor-core pipeline (TMA loads and MMAs on shared-memory barriers; a wait
 * past it makes the kernel stop issuing, wait with a 1 s bound for the copies
 * and MMAs it already started, free its tensor memory and skip the step,
 * reported by ia_loss_scale / ia_train_stats as IA_ERR_CUDA).  0 restores the
 * default (200 ms, far above the reduction's normal time); 1..1e10 otherwise.
 * Not a method parameter: a diagnostics setting, also used to exercise the
 * failure path. */
ia_status ia_set_wait_limit(ia_ctx *ctx, int64_t limit_ns);

/* Failure injection for tests of the bounded-wait path (no fault, no hang):
 * with IA_INJECT_WITHHOLD_COPY the weight-gradient pipeline of the following
 * reduced-precision training steps never issues the TMA copy of each CTA's last
 * operand chunk, so the MMA thread's wait for it runs out after the wait limit
 * (ia_set_wait_limit) and the step is skipped and reported as IA_ERR_CUDA.
 * 0 turns injection off.  Not a method parameter. */
#define IA_INJECT_WITHHOLD_COPY 1
ia_status ia_set_fault_injection(ia_ctx *ctx, int flags);

/* Same result as ia_update_occupancy(ctx, pose, IA_OCC_POSE, NULL, bits_out,
 * NULL, stream), for callers that cannot allocate device memory while they run:
 * code whose device memory is owned by another allocator (a framework's caching
 * pool, a fixed arena sized at start-up) or a frame loop in which a cudaMalloc,
 * with its implicit device-wide synchronisation, would stall other streams.
 * This call allocates nothing: the per-cell density scratch is a fixed array of
 * 64^3 floats (1 MiB) compiled into the library, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart of this
 * call; it is an interface convenience.
 *  - occ_res above 64 returns IA_ERR_LIMIT (use ia_update_occupancy).
 *  - The context's device must be current.  The first call on a device looks up
 *    the array's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's densities:
 *    every call rewrites the cells it reads before reading them, but calls that
 *    overlap on the GPU (different streams, or different contexts on the same
 *    device) race on it and must be serialised by the caller.
 *  bits_out [R^3 / 32] uint32 device or NULL; the render grid is replaced. */
ia_status ia_update_occupancy_static(ia_ctx *ctx, int pose, uint32_t *bits_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned correspondence proposal.  The paper starts the search from every bone
 * (Sec. 3.1); this optional network (not in the paper) proposes the first starts
 * instead: input [hash features of x' over the normalised box (n_levels x 2) |
 * the pose's axis-angles (n_bones x 3)], MLP 64-64-64 (ReLU), output n_bones
 * logits and a 3-D start offset.  In IA_SEARCH_PROPOSAL mode every posed-field
 * evaluation (render, occupancy, queries) starts from the top_k bones by logit
 * (the first shifted by the offset) and falls back to every bone-wise start when
 * those find no valid root.  Inference runs on tensor cores, so the mode needs
 * precision IA_FP16 or IA_BF16.  Training pairs come from the plain search; the
 * label is the bone with the largest skinning weight at the selected root x*,
 * the offset target x* - N_label^-1 x'; loss per pair = cross-entropy +
 * offset_weight |offset - target|^2, averaged over the batch; Adam (0.9, 0.999).
 * ------------------------------------------------------------------------- */
typedef struct ia_proposal_config {
  int n_levels;                  /* 1..8 */
  int log2_table;                /* 10..24 */
  int level_res[IA_MAX_LEVELS];  /* grid resolution per level, >= 2 */
  int top_k;                     /* proposed starts before the fallback: 1 or 2 */
  float offset_weight;           /* weight of the offset term, >= 0 */
} ia_proposal_config;

typedef enum ia_search { IA_SEARCH_ALL_BONES = 0, IA_SEARCH_PROPOSAL = 1 } ia_search;

/* Allocate the network (parameters zero until ia_proposal_set_params). */
ia_status ia_proposal_init(ia_ctx *ctx, const ia_proposal_config *cfg);
/* fp32 values of the table ([entries][2], same layout rules as the canonical
 * grid over the normalised box) and of the packed MLP (W1 [64][2L + 3 n_b], b1,
 * W2 [64][64], b2, W3 [64][64], b3, W4 [n_b + 3][64], b4). */
ia_status ia_proposal_param_sizes(const ia_ctx *ctx, int64_t *table_floats, int64_t *mlp_floats);
/* Load (host or device; resets the optimiser state) / read the parameters. */
ia_status ia_proposal_set_params(ia_ctx *ctx, const float *table, const float *mlp, void *stream);
ia_status ia_proposal_get_params(ia_ctx *ctx, float *table, float *mlp, void *stream);
/* Training pairs for n normalised-space points x [n][3] of pose p from the
 * plain search: label [n] int32 (-1 where no valid root), offset [n][3] (device). */
ia_status ia_proposal_pairs(ia_ctx *ctx, int pose, int n, const float *x, int32_t *label, float *offset,
                            void *stream);
/* Loss and gradients over n pairs (device: x [n][3], pose [n], label [n] in
 * [0, n_b), target [n][3]); *loss is overwritten; g_table and g_mlp are laid out
 * like the parameters. */
ia_status ia_proposal_grad(ia_ctx *ctx, int n, const float *x, const int32_t *pose, const int32_t *label,
                           const float *target, float *loss, float *g_table, float *g_mlp, void *stream);
/* `steps` Adam steps of `batch` pairs each, taking pairs in order and wrapping
 * around (shuffle them beforehand); loss_out [steps] (device, may be NULL)
 * receives each step's batch loss.  Workspace for `batch` pairs (~2.3 KB each)
 * is allocated on first use. */
ia_status ia_proposal_train(ia_ctx *ctx, int n, const float *x, const int32_t *pose, const int32_t *label,
                            const float *target, int steps, int batch, float lr, float *loss_out,
                            void *stream);
/* IA_SEARCH_ALL_BONES (the paper's search) or IA_SEARCH_PROPOSAL. */
ia_status ia_set_search(ia_ctx *ctx, int mode);
/* Root culling (see ia_update_occupancy): 1 (default) skips the search of
 * occupancy cells, render samples (pose of the last occupancy update) and
 * training samples and regulariser points (masks of every pose, built on the
 * first training step after the blended grids change; skipped when they would
 * exceed 4 GiB) whose point can have no root; 0 searches them all.  Results
 * are the same either way. */
ia_status ia_set_occupancy_culling(ia_ctx *ctx, int on);

/* The sample set of ia_render without evaluating it (the indexing contract):
 * bit i of slot_mask[(v * W + u) * ceil(N / 32) + i / 32] is set iff slot i of
 * pixel (u, v) lies in an occupied cell of the render grid.  Without early
 * termination these are exactly the samples ia_render evaluates.
 *  slot_mask [H*W][ceil(N/32)] uint32 device. */
ia_status ia_march_mask(ia_ctx *ctx, int pose, const ia_camera *cam, uint32_t *slot_mask, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IA_H */
