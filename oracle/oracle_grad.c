/*
 * FP64 CPU oracle, training step: L2 photometric loss over a batch of rays and
 * its exact reverse-mode gradient.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Forward per ray: the same steps as rendering (Sec. 3.2-3.3), with world rays
 * mapped into the normalised space of the ray's pose.  Loss
 *   L = (1 / n) sum_rays sum_channels (C - C_target)^2.
 * Backward, in the reverse order of the forward:
 *   compositing (Eq. 8):  dL/dc_i = T_i alpha_i g,
 *                         dL/dsigma_i = delta (T_{i+1} c_i.g - g.(C - C_{<=i}))
 *   activations, MLP (Eq. 1-2), hash-table entries (trilinear weights) and the
 *   canonical position x*;
 *   the root x* of g(x*, theta) = LBS(x*) - x' = 0 (Eq. 7) by the implicit
 *   function theorem: d(x*) / d(theta) = -J^-1 d(g) / d(theta), J the analytic
 *   Jacobian at x*, so with lambda = J^-T dL/dx*:
 *     dL/dN_k[a][b]  = -lambda_a w_k(x*) [x*;1]_b
 *     dL/dW(v, i)    = -c_v(x*) lambda . (N_i [x*;1])   (c_v trilinear coefficient)
 * The selected root and its validity are treated as constants (they are
 * discrete choices).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct fsamp {
  double xs[3], sigma, rgb[3];
  int has, pose;
} fsamp;

/* world ray -> normalised space of one pose, fp32 fixed order (as or_ray) */
static int norm_ray(const or_model *m, const or_pose *p, const float ow[3], const float dw[3],
                    float o[3], float d[3], float *tn, float *tf) {
  const float *M = p->B0inv;
  for (int i = 0; i < 3; ++i) {
    o[i] = (((M[i * 4 + 0] * ow[0]) + (M[i * 4 + 1] * ow[1])) + (M[i * 4 + 2] * ow[2])) + M[i * 4 + 3];
    d[i] = ((M[i * 4 + 0] * dw[0]) + (M[i * 4 + 1] * dw[1])) + (M[i * 4 + 2] * dw[2]);
  }
  float tmin = 0.0f, tmax = INFINITY;
  for (int a = 0; a < 3; ++a) {
    float inv = 1.0f / d[a];
    float t0 = (m->nmin[a] - o[a]) * inv;
    float t1 = (m->nmax[a] - o[a]) * inv;
    tmin = fmaxf(tmin, fminf(t0, t1));
    tmax = fminf(tmax, fmaxf(t0, t1));
  }
  *tn = tmin;
  *tf = tmax;
  return tmax > tmin;
}

/* forward of one ray: samples in march order, colour, final transmittance */
static int forward_ray(const or_model *m, const or_pose *poses, int pose, const uint32_t *occ,
                       const float ow[3], const float dw[3], fsamp *S, double C[3], double *T_out,
                       double *dt_out, int *flags, const or_prop *q, const double *theta_all, int *n_fallback) {
  const or_pose *p = &poses[pose];
  float o[3], d[3], tn, tf;
  int n = 0, fl = 0;
  double T = 1.0;
  C[0] = C[1] = C[2] = 0.0;
  *dt_out = 0.0;
  if (norm_ray(m, p, ow, dw, o, d, &tn, &tf)) {
    float dt = (tf - tn) / (float)m->n_slots;
    *dt_out = (double)dt;
    for (int i = 0; i < m->n_slots; ++i) {
      float t = tn + (((float)i + 0.5f) * dt);
      float x[3];
      for (int a = 0; a < 3; ++a) x[a] = o[a] + (t * d[a]);
      int cell = or_cell(m, x);
      if (!((occ[cell >> 5] >> (cell & 31)) & 1u)) continue;
      or_sample s;
      double xn[3] = {(double)x[0], (double)x[1], (double)x[2]};
      if (q) {
        int fb = 0;
        or_posed_field_prop(m, p, q, theta_all + (long)pose * 3 * m->nb, xn, &s, &fb);
        if (n_fallback) *n_fallback += fb;
      } else {
        or_posed_field(m, p, xn, &s);
      }
      fl |= s.flags;
      fsamp *q = &S[n++];
      q->has = s.start >= 0;
      q->pose = pose;
      q->sigma = s.sigma;
      for (int k = 0; k < 3; ++k) { q->rgb[k] = s.rgb[k]; q->xs[k] = s.xstar[k]; }
      if (q->has) {
        double a = 1.0 - exp(-s.sigma * (double)dt);
        for (int k = 0; k < 3; ++k) C[k] += T * a * s.rgb[k];
        T *= 1.0 - a;
      }
      if (m->early_T > 0.0 && fabs(T / m->early_T - 1.0) < 1e-3) fl |= OR_FLAG_TERM;
      if (m->early_T > 0.0 && T < m->early_T) break;
    }
  }
  *T_out = T;
  if (flags) *flags = fl;
  return n;
}

static long mlp_count(const or_model *m) {
  int W = m->width;
  return (long)W * m->n_in + W + (long)W * W + W + 4L * W + 4;
}

/* backward of one evaluated sample given dL/dsigma and dL/dc */
static void backward_sample(const or_model *m, const or_pose *poses, const fsamp *q, double dsig,
                            const double dc[3], double *g_table, double *g_mlp, double *g_skin,
                            double *g_bones) {
  const int W = m->width, nin = m->n_in, L = m->L, F = m->F;
  /* ---- recompute the forward activations at x* */
  double feat[OR_MAX_LEVELS * 8], h1p[256], h1[256], h2p[256], h2[256], o[4];
  or_encode(m, q->xs, feat);
  for (int j = 0; j < W; ++j) {
    double s = m->b1[j];
    for (int i = 0; i < nin; ++i) s += m->W1[j * nin + i] * feat[i];
    h1p[j] = s;
    h1[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < W; ++j) {
    double s = m->b2[j];
    for (int i = 0; i < W; ++i) s += m->W2[j * W + i] * h1[i];
    h2p[j] = s;
    h2[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < 4; ++j) {
    double s = m->b3[j];
    for (int i = 0; i < W; ++i) s += m->W3[j * W + i] * h2[i];
    o[j] = s;
  }
  /* ---- activations: sigma = exp(clamp(o0)), c = sigmoid(o1..3) */
  double dO[4];
  double sig = exp(o[0] < -15.0 ? -15.0 : (o[0] > 15.0 ? 15.0 : o[0]));
  dO[0] = (o[0] > -15.0 && o[0] < 15.0) ? dsig * sig : 0.0;
  for (int c = 0; c < 3; ++c) {
    double s = 1.0 / (1.0 + exp(-o[1 + c]));
    dO[1 + c] = dc[c] * s * (1.0 - s);
  }
  /* ---- MLP backward (gradient layout: W1, b1, W2, b2, W3, b3) */
  double *gW1 = g_mlp, *gb1 = gW1 + (long)W * nin, *gW2 = gb1 + W, *gb2 = gW2 + (long)W * W;
  double *gW3 = gb2 + W, *gb3 = gW3 + 4L * W;
  double dh2[256], dh1[256], dfeat[OR_MAX_LEVELS * 8];
  for (int j = 0; j < 4; ++j) {
    gb3[j] += dO[j];
    for (int i = 0; i < W; ++i) gW3[j * W + i] += dO[j] * h2[i];
  }
  for (int i = 0; i < W; ++i) {
    double s = 0.0;
    for (int j = 0; j < 4; ++j) s += m->W3[j * W + i] * dO[j];
    dh2[i] = h2p[i] > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < W; ++j) {
    gb2[j] += dh2[j];
    for (int i = 0; i < W; ++i) gW2[j * W + i] += dh2[j] * h1[i];
  }
  for (int i = 0; i < W; ++i) {
    double s = 0.0;
    for (int j = 0; j < W; ++j) s += m->W2[j * W + i] * dh2[j];
    dh1[i] = h1p[i] > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < W; ++j) {
    gb1[j] += dh1[j];
    for (int i = 0; i < nin; ++i) gW1[j * nin + i] += dh1[j] * feat[i];
  }
  for (int i = 0; i < nin; ++i) {
    double s = 0.0;
    for (int j = 0; j < W; ++j) s += m->W1[j * nin + i] * dh1[j];
    dfeat[i] = s;
  }
  /* ---- hash encoding backward: table entries and the canonical position */
  double gx[3] = {0.0, 0.0, 0.0};
  {
    long T = 1L << m->log2_T, off = 0;
    double u[3], ext[3];
    for (int a = 0; a < 3; ++a) {
      ext[a] = m->cmax[a] - m->cmin[a];
      u[a] = (q->xs[a] - m->cmin[a]) / ext[a];
    }
    for (int l = 0; l < L; ++l) {
      long r1 = (long)m->res[l] + 1, size = r1 * r1 * r1 <= T ? r1 * r1 * r1 : T;
      int res = m->res[l], p0[3];
      double f[3];
      for (int a = 0; a < 3; ++a) {
        double pos = u[a] * (double)res;
        int c = (int)floor(pos);
        if (c > res - 1) c = res - 1;
        if (c < 0) c = 0;
        p0[a] = c;
        f[a] = pos - (double)c;
      }
      for (int corner = 0; corner < 8; ++corner) {
        int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
        double wx = cx ? f[0] : 1.0 - f[0], wy = cy ? f[1] : 1.0 - f[1], wz = cz ? f[2] : 1.0 - f[2];
        int i = p0[0] + cx, j = p0[1] + cy, k = p0[2] + cz;
        long e;
        if (r1 * r1 * r1 <= size) {
          e = (long)i + r1 * ((long)j + r1 * (long)k);
        } else {
          uint32_t h = (uint32_t)i * 1u ^ (uint32_t)j * 2654435761u ^ (uint32_t)k * 805459861u;
          e = (long)(h % (uint32_t)size);
        }
        e += off;
        double proj = 0.0;
        for (int q2 = 0; q2 < F; ++q2) {
          g_table[e * F + q2] += wx * wy * wz * dfeat[l * F + q2];
          proj += m->table[e * F + q2] * dfeat[l * F + q2];
        }
        double sx = (cx ? 1.0 : -1.0) * wy * wz, sy = (cy ? 1.0 : -1.0) * wx * wz,
               sz = (cz ? 1.0 : -1.0) * wx * wy;
        gx[0] += proj * sx * (double)res / ext[0];
        gx[1] += proj * sy * (double)res / ext[1];
        gx[2] += proj * sz * (double)res / ext[2];
      }
      off += size;
    }
  }
  /* ---- implicit function theorem through the root of LBS(x*) = x' */
  const or_pose *p = &poses[q->pose];
  double y[3], J[9];
  or_lbs(m, p, q->xs, y, J);
  double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
  double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (fabs(det) < 1e-300) return;
  double Hi[9];
  Hi[0] = c00 / det;
  Hi[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Hi[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Hi[3] = c01 / det;
  Hi[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Hi[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Hi[6] = c02 / det;
  Hi[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Hi[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  /* lambda = J^-T gx */
  double lam[3];
  for (int a = 0; a < 3; ++a) lam[a] = Hi[0 * 3 + a] * gx[0] + Hi[1 * 3 + a] * gx[1] + Hi[2 * 3 + a] * gx[2];
  const double xb[4] = {q->xs[0], q->xs[1], q->xs[2], 1.0};
  const int nb = m->nb, R = m->rw;
  double w[OR_MAX_BONES];
  or_skin(m, q->xs, w, NULL);
  double *gB = g_bones + (long)q->pose * nb * 12;
  for (int k = 0; k < nb; ++k)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 4; ++b) gB[k * 12 + a * 4 + b] -= lam[a] * w[k] * xb[b];
  /* skinning grid: trilinear coefficient of each corner vertex */
  int i0[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    double ext = m->cmax[a] - m->cmin[a];
    double u = (q->xs[a] - m->cmin[a]) / ext * (double)(R - 1);
    if (u < 0.0) u = 0.0;
    if (u > (double)(R - 1)) u = (double)(R - 1);
    int c = (int)floor(u);
    if (c > R - 2) c = R - 2;
    i0[a] = c;
    f[a] = u - (double)c;
  }
  double lNx[OR_MAX_BONES];
  for (int i = 0; i < nb; ++i) {
    double Nx[3];
    for (int a = 0; a < 3; ++a)
      Nx[a] = p->N[i][a * 4 + 0] * xb[0] + p->N[i][a * 4 + 1] * xb[1] + p->N[i][a * 4 + 2] * xb[2] +
              p->N[i][a * 4 + 3];
    lNx[i] = lam[0] * Nx[0] + lam[1] * Nx[1] + lam[2] * Nx[2];
  }
  for (int corner = 0; corner < 8; ++corner) {
    int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
    double cw = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
    long v = ((long)(i0[2] + cz) * R + (i0[1] + cy)) * R + (i0[0] + cx);
    for (int i = 0; i < nb; ++i) g_skin[v * nb + i] -= cw * lNx[i];
  }
}

/* Loss and gradients for a batch.  poses [n_poses]; rays: o, d [n][3] world
 * (fp32), pose_id [n], target [n][3].  Gradients are overwritten:
 * g_table [entries][F], g_mlp (packed), g_skin [rw^3][nb], g_bones [n_poses][nb][12]
 * (all NULL: loss only).  rgb_out [n][3], ray_flags [n] may be NULL. */
/* Loss of ray r (Sec. 3.4) divided by the batch size n, and its gradients
   g = dL/dC, *ga = dL/dalpha (alpha = 1 - the ray's final transmittance). */
static double ray_loss(const or_loss *lc, int n, const double C[3], const double target[3], double alpha, int r,
                       double g[3], double *ga) {
  double e[3], ee = 0.0;
  for (int k = 0; k < 3; ++k) {
    e[k] = C[k] - target[k];
    ee += e[k] * e[k];
  }
  /* colour term (Eq. 9): L2 over channels, or Huber of the colour error's norm */
  double lr;
  if (!lc->huber) {
    lr = ee;
    for (int k = 0; k < 3; ++k) g[k] = 2.0 * e[k];
  } else {
    const double rn = sqrt(ee);
    if (rn <= lc->delta) {
      lr = 0.5 * ee;
      for (int k = 0; k < 3; ++k) g[k] = e[k];
    } else {
      lr = lc->delta * (rn - 0.5 * lc->delta);
      for (int k = 0; k < 3; ++k) g[k] = lc->delta * e[k] / rn;
    }
  }
  for (int k = 0; k < 3; ++k) g[k] *= lc->w_rgb / (double)n;
  /* opacity terms: L1 to the mask (Eq. 10), hard surface (Eq. 11) */
  double la = 0.0, gal = 0.0;
  if (lc->w_alpha != 0.0) {
    const double da = alpha - lc->alpha_target[r];
    la += lc->w_alpha * fabs(da);
    gal += lc->w_alpha * (da > 0.0 ? 1.0 : (da < 0.0 ? -1.0 : 0.0));
  }
  if (lc->w_hard != 0.0) {
    const double e0 = exp(-fabs(alpha)), e1 = exp(-fabs(alpha - 1.0));
    la += lc->w_hard * (-log(e0 + e1) + log(1.0 + exp(-1.0)));
    const double s0 = alpha > 0.0 ? 1.0 : (alpha < 0.0 ? -1.0 : 0.0);
    const double s1 = alpha > 1.0 ? 1.0 : (alpha < 1.0 ? -1.0 : 0.0);
    gal += lc->w_hard * (s0 * e0 + s1 * e1) / (e0 + e1);
  }
  *ga = gal / (double)n;
  return (lc->w_rgb * lr + la) / (double)n;
}

/* up_rgb [n][3] / up_alpha [n] (optional): dL/dC and dL/dalpha given by the
   caller instead of a loss (the loss returned is then 0); alpha_out [n] may be NULL. */
static double train_impl(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                         const float *o, const float *d, const int32_t *pose_id, const double *target,
                         double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                         double *g_bones, int nthreads, const or_prop *q, const double *theta_all,
                         int *ray_fallbacks, const or_loss *lc, const double *up_rgb, const double *up_alpha,
                         double *alpha_out) {
  static const or_loss l2 = {0, 0.0, 1.0, 0.0, 0.0, NULL};
  if (!lc) lc = &l2;
  long entries = 0;
  {
    long T = 1L << m->log2_T;
    for (int l = 0; l < m->L; ++l) {
      long r1 = (long)m->res[l] + 1;
      entries += r1 * r1 * r1 <= T ? r1 * r1 * r1 : T;
    }
  }
  if (g_table) memset(g_table, 0, (size_t)entries * m->F * sizeof(double));
  if (g_mlp) memset(g_mlp, 0, (size_t)mlp_count(m) * sizeof(double));
  if (g_skin) memset(g_skin, 0, (size_t)m->rw * m->rw * m->rw * m->nb * sizeof(double));
  if (g_bones) memset(g_bones, 0, (size_t)n_poses * m->nb * 12 * sizeof(double));
  fsamp *S = (fsamp *)malloc((size_t)(n > 0 ? n : 1) * m->n_slots * sizeof(fsamp));
  int *cnt = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  double *Cs = (double *)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(double));
  double *dts = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
  for (int r = 0; r < n; ++r) {
    int fl = 0, nfb = 0;
    cnt[r] = forward_ray(m, poses, pose_id[r], occ, o + 3 * r, d + 3 * r, S + (long)r * m->n_slots,
                         Cs + 4 * r, Cs + 4 * r + 3, dts + r, &fl, q, theta_all, &nfb);
    if (ray_fallbacks) ray_fallbacks[r] = nfb;
    if (ray_flags) ray_flags[r] = fl;
  }
  double loss = 0.0;
  for (int r = 0; r < n; ++r) {
    const double *C = Cs + 4 * r;
    for (int k = 0; k < 3; ++k)
      if (rgb_out) rgb_out[3 * r + k] = C[k];
    if (alpha_out) alpha_out[r] = 1.0 - Cs[4 * r + 3];
    double g[3], ga;
    if (up_rgb) {
      /* the caller's dL/dC and dL/dalpha: no loss of ours */
      for (int k = 0; k < 3; ++k) g[k] = up_rgb[3 * r + k];
      ga = up_alpha ? up_alpha[r] : 0.0;
    } else if (target) {
      loss += ray_loss(lc, n, C, target + 3 * r, 1.0 - Cs[4 * r + 3], r, g, &ga);
    } else {
      continue; /* forward only */
    }
    const double TN = Cs[4 * r + 3];
    if (!g_table || !g_mlp || !g_skin || !g_bones) continue;
    /* compositing backward, front to back */
    double T = 1.0, Cle[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < cnt[r]; ++i) {
      const fsamp *q = S + (long)r * m->n_slots + i;
      if (!q->has) continue;
      double a = 1.0 - exp(-q->sigma * dts[r]);
      double Tn = T * (1.0 - a);
      double dc[3], cg = 0.0, rest = 0.0;
      for (int k = 0; k < 3; ++k) {
        Cle[k] += T * a * q->rgb[k];
        dc[k] = T * a * g[k];
        cg += q->rgb[k] * g[k];
        rest += g[k] * (C[k] - Cle[k]);
      }
      /* d alpha / d sigma_i = delta T_N */
      double dsig = dts[r] * (Tn * cg - rest) + ga * dts[r] * TN;
      backward_sample(m, poses, q, dsig, dc, g_table, g_mlp, g_skin, g_bones);
      T = Tn;
    }
  }
  free(S);
  free(cnt);
  free(Cs);
  free(dts);
  return loss;
}

double or_train(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                const float *o, const float *d, const int32_t *pose_id, const double *target,
                double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                double *g_bones, int nthreads) {
  return train_impl(m, poses, n_poses, occ, n, o, d, pose_id, target, rgb_out, ray_flags, g_table, g_mlp, g_skin,
                    g_bones, nthreads, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* The same step with the correspondence proposal choosing each sample's starts
 * (or_posed_field_prop; theta_all [n_poses][nb][3] the poses' axis-angles).
 * ray_fallbacks [n] (may be NULL): samples of each ray whose proposed starts
 * found no valid root, so that the search over every bone ran. */
double or_train_prop(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                     const float *o, const float *d, const int32_t *pose_id, const double *target,
                     double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                     double *g_bones, int nthreads, const or_prop *q, const double *theta_all,
                     int *ray_fallbacks) {
  return train_impl(m, poses, n_poses, occ, n, o, d, pose_id, target, rgb_out, ray_flags, g_table, g_mlp, g_skin,
                    g_bones, nthreads, q, theta_all, ray_fallbacks, NULL, NULL, NULL, NULL);
}

/* or_train with the paper's loss set (config lc; alpha of a ray = 1 - its final
 * transmittance). */
double or_train_loss(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                     const float *o, const float *d, const int32_t *pose_id, const double *target,
                     double *rgb_out, int *ray_flags, double *g_table, double *g_mlp, double *g_skin,
                     double *g_bones, int nthreads, const or_loss *lc) {
  return train_impl(m, poses, n_poses, occ, n, o, d, pose_id, target, rgb_out, ray_flags, g_table, g_mlp, g_skin,
                    g_bones, nthreads, NULL, NULL, NULL, lc, NULL, NULL, NULL);
}

/* The backward of the same forward for a loss computed elsewhere: the caller
   gives dL/dC [n][3] and dL/dalpha [n] (NULL: zero) of every ray; the reverse
   sweep and everything after it are those of or_train.  rgb_out, alpha_out
   receive the forward's colour and alpha = 1 - final transmittance. */
void or_train_upstream(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                       const float *o, const float *d, const int32_t *pose_id, const double *up_rgb,
                       const double *up_alpha, double *rgb_out, double *alpha_out, int *ray_flags, double *g_table,
                       double *g_mlp, double *g_skin, double *g_bones, int nthreads) {
  train_impl(m, poses, n_poses, occ, n, o, d, pose_id, NULL, rgb_out, ray_flags, g_table, g_mlp, g_skin, g_bones,
             nthreads, NULL, NULL, NULL, NULL, up_rgb, up_alpha, alpha_out);
}

double or_density_reg(const or_model *m, const or_pose *poses, int n_poses, const uint32_t *occ, int n,
                      const float *x, const int32_t *pose_id, double weight, int *point_flags, double *g_table,
                      double *g_mlp, double *g_skin, double *g_bones) {
  double loss = 0.0;
  const double w = n > 0 ? weight / (double)n : 0.0;
  const double dc[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    if (point_flags) point_flags[i] = 0;
    const int pose = pose_id[i];
    if (pose < 0 || pose >= n_poses) continue;
    const int cell = or_cell(m, x + 3 * i);
    if ((occ[cell >> 5] >> (cell & 31)) & 1u) continue; /* occupied: no penalty */
    const double xn[3] = {(double)x[3 * i], (double)x[3 * i + 1], (double)x[3 * i + 2]};
    or_sample s;
    or_posed_field(m, &poses[pose], xn, &s);
    if (point_flags) point_flags[i] = s.flags;
    if (s.start < 0) continue; /* no root: density 0, nothing to differentiate */
    loss += w * s.sigma;
    if (g_table && g_mlp && g_skin && g_bones) {
      fsamp q;
      q.has = 1;
      q.pose = pose;
      q.sigma = s.sigma;
      for (int k = 0; k < 3; ++k) {
        q.xs[k] = s.xstar[k];
        q.rgb[k] = s.rgb[k];
      }
      backward_sample(m, poses, &q, w, dc, g_table, g_mlp, g_skin, g_bones);
    }
  }
  return loss;
}
