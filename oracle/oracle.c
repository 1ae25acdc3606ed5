/*
 * FP64 CPU oracle, forward path.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain loops, one sample at a time, in the order the paper states the method.
 * Compiled with -ffp-contract=off so that the fp32 indexing functions perform
 * exactly the documented sequence of rounded operations.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* small 3x3 / 3x4 helpers (row-major)                                        */
/* ------------------------------------------------------------------------- */

static void mat34_mul(const double a[12], const double b[12], double c[12]) {
  /* [Ra|ta] [Rb|tb] = [Ra Rb | Ra tb + ta] */
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j) {
      double s = a[i * 4 + 0] * b[0 * 4 + j] + a[i * 4 + 1] * b[1 * 4 + j] +
                 a[i * 4 + 2] * b[2 * 4 + j];
      if (j == 3) s += a[i * 4 + 3];
      c[i * 4 + j] = s;
    }
  }
}

static void mat34_rigid_inv(const double a[12], double c[12]) {
  /* [R|t]^-1 = [R^T | -R^T t]  (all transforms here are rigid) */
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) c[i * 4 + j] = a[j * 4 + i];
    c[i * 4 + 3] = -(a[0 * 4 + i] * a[3] + a[1 * 4 + i] * a[7] + a[2 * 4 + i] * a[11]);
  }
}

static void mat34_apply(const double a[12], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i)
    y[i] = a[i * 4 + 0] * x[0] + a[i * 4 + 1] * x[1] + a[i * 4 + 2] * x[2] + a[i * 4 + 3];
}

/* inverse via the adjugate; returns 0 if |det| < 1e-6 (treated as singular) */
static int inv3(const double J[9], double H[9], double *det_out) {
  double c00 = J[4] * J[8] - J[5] * J[7];
  double c01 = J[5] * J[6] - J[3] * J[8];
  double c02 = J[3] * J[7] - J[4] * J[6];
  double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (det_out) *det_out = det;
  if (!(fabs(det) >= 1e-6)) return 0;
  double id = 1.0 / det;
  H[0] = c00 * id;
  H[1] = (J[2] * J[7] - J[1] * J[8]) * id;
  H[2] = (J[1] * J[5] - J[2] * J[4]) * id;
  H[3] = c01 * id;
  H[4] = (J[0] * J[8] - J[2] * J[6]) * id;
  H[5] = (J[2] * J[3] - J[0] * J[5]) * id;
  H[6] = c02 * id;
  H[7] = (J[1] * J[6] - J[0] * J[7]) * id;
  H[8] = (J[0] * J[4] - J[1] * J[3]) * id;
  return 1;
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* ------------------------------------------------------------------------- */
/* Pose chain (Sec. 3.1 bone transforms B; Sec. 3.3 normalised space)         */
/* ------------------------------------------------------------------------- */

/* cos a and sin a from their Maclaurin series
     sin x = sum_k (-1)^k x^(2k+1) / (2k+1)!,   cos x = sum_k (-1)^k x^(2k) / (2k)!,
   after one reduction of a by the nearest multiple of 2 pi (fp64 constant),
   each term from the previous one, t_{k+1} = t_k (-x^2) r_k with the
   correctly rounded reciprocal r_k = 1 / ((2k+2)(2k+3)) for sin and
   1 / ((2k+1)(2k+2)) for cos, added in order; 22 terms (the first omitted one
   is below pi^46 / 46! < 1e-32).  Every step is one correctly rounded fp64
   operation in a fixed order, so the values are the same on any IEEE machine
   (the library's pose chain takes the same steps, which keeps the fp32 bone
   transforms bit-identical); they agree with the C library's cos / sin to a
   few 1e-16. */
void or_cos_sin(double a, double *c, double *s) {
  const double two_pi = 6.283185307179586;
  const double x = a - rint(a / two_pi) * two_pi;
  const double mx2 = -(x * x);
  double ts = x, tc = 1.0, sn = x, cs = 1.0;
  for (int k = 0; k < 22; ++k) {
    const double rs = 1.0 / (double)((2 * k + 2) * (2 * k + 3));
    const double rc = 1.0 / (double)((2 * k + 1) * (2 * k + 2));
    ts = ts * mx2 * rs;
    tc = tc * mx2 * rc;
    sn = sn + ts;
    cs = cs + tc;
  }
  *c = cs;
  *s = sn;
}

/* Rodrigues: rotation by |th| about th/|th|. */
static void rodrigues(const double th[3], double R[9]) {
  double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
  if (a == 0.0) {
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    return;
  }
  double k0 = th[0] / a, k1 = th[1] / a, k2 = th[2] / a;
  double c, s;
  or_cos_sin(a, &c, &s);
  double C = 1.0 - c;
  R[0] = c + C * k0 * k0;
  R[1] = C * k0 * k1 - s * k2;
  R[2] = C * k0 * k2 + s * k1;
  R[3] = C * k1 * k0 + s * k2;
  R[4] = c + C * k1 * k1;
  R[5] = C * k1 * k2 - s * k0;
  R[6] = C * k2 * k0 - s * k1;
  R[7] = C * k2 * k1 + s * k0;
  R[8] = c + C * k2 * k2;
}

static double round32(double v, int q) { return q ? (double)(float)v : v; }

void or_pose_chain(const or_model *m, const double *theta, const double *trans, or_pose *out) {
  double G[OR_MAX_BONES][12];
  memset(out, 0, sizeof(*out));
  for (int k = 0; k < m->nb; ++k) {
    double R[9], L[12];
    rodrigues(theta + 3 * k, R);
    int p = m->parent[k];
    /* local joint frame: rotate about joint k, offset from the parent joint */
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) L[i * 4 + j] = R[i * 3 + j];
      L[i * 4 + 3] = (p < 0) ? m->rest[3 * k + i] : m->rest[3 * k + i] - m->rest[3 * p + i];
    }
    if (p < 0)
      memcpy(G[k], L, sizeof(L));
    else
      mat34_mul(G[p], L, G[k]);
    /* rest-relative bone transform B_k = G_k [I | -j_k], plus global translation */
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) out->B[k][i * 4 + j] = G[k][i * 4 + j];
      double Rj = G[k][i * 4 + 0] * m->rest[3 * k + 0] + G[k][i * 4 + 1] * m->rest[3 * k + 1] +
                  G[k][i * 4 + 2] * m->rest[3 * k + 2];
      out->B[k][i * 4 + 3] = G[k][i * 4 + 3] - Rj + trans[i];
    }
  }
  /* normalised space: remove the root's rigid motion, N_k = B_0^-1 B_k */
  double B0i[12];
  mat34_rigid_inv(out->B[0], B0i);
  for (int k = 0; k < m->nb; ++k) {
    mat34_mul(B0i, out->B[k], out->N[k]);
    for (int i = 0; i < 12; ++i) out->N[k][i] = round32(out->N[k][i], m->quantize_fp32);
    double Ni[12];
    double Nexact[12];
    mat34_mul(B0i, out->B[k], Nexact);
    mat34_rigid_inv(Nexact, Ni);
    for (int i = 0; i < 12; ++i) out->Ninv[k][i] = round32(Ni[i], m->quantize_fp32);
  }
  for (int i = 0; i < 12; ++i) out->B0inv[i] = (float)B0i[i];
}

/* ------------------------------------------------------------------------- */
/* Skinning-weight grid (Sec. 3.1): trilinear, corners aligned to the box     */
/* ------------------------------------------------------------------------- */

void or_skin(const or_model *m, const double x[3], double *w, double *dw) {
  int nb = m->nb, R = m->rw;
  int i0[3];
  double f[3], scale[3], live[3];
  for (int a = 0; a < 3; ++a) {
    double ext = m->cmax[a] - m->cmin[a];
    double u = (x[a] - m->cmin[a]) / ext * (double)(R - 1);
    live[a] = 1.0;
    if (u < 0.0) { u = 0.0; live[a] = 0.0; }          /* clamp to the border */
    if (u > (double)(R - 1)) { u = (double)(R - 1); live[a] = 0.0; }
    int c = (int)floor(u);
    if (c > R - 2) c = R - 2;
    i0[a] = c;
    f[a] = u - (double)c;
    scale[a] = (double)(R - 1) / ext;
  }
  for (int i = 0; i < nb; ++i) {
    w[i] = 0.0;
    if (dw) dw[3 * i] = dw[3 * i + 1] = dw[3 * i + 2] = 0.0;
  }
  for (int corner = 0; corner < 8; ++corner) {
    int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
    double wx = cx ? f[0] : 1.0 - f[0];
    double wy = cy ? f[1] : 1.0 - f[1];
    double wz = cz ? f[2] : 1.0 - f[2];
    double gx = (cx ? 1.0 : -1.0) * wy * wz * scale[0] * live[0];
    double gy = (cy ? 1.0 : -1.0) * wx * wz * scale[1] * live[1];
    double gz = (cz ? 1.0 : -1.0) * wx * wy * scale[2] * live[2];
    long v = ((long)(i0[2] + cz) * R + (i0[1] + cy)) * R + (i0[0] + cx);
    const double *W = m->skin + v * nb;
    double tw = wx * wy * wz;
    for (int i = 0; i < nb; ++i) {
      w[i] += tw * W[i];
      if (dw) {
        dw[3 * i + 0] += gx * W[i];
        dw[3 * i + 1] += gy * W[i];
        dw[3 * i + 2] += gz * W[i];
      }
    }
  }
}

/* Eq. 7 with the normalised-space transforms; J = sum w_i R_i + sum (N_i x) dw_i^T */
void or_lbs(const or_model *m, const or_pose *p, const double x[3], double y[3], double *J) {
  double w[OR_MAX_BONES], dw[OR_MAX_BONES * 3];
  or_skin(m, x, w, J ? dw : NULL);
  y[0] = y[1] = y[2] = 0.0;
  if (J) memset(J, 0, 9 * sizeof(double));
  for (int i = 0; i < m->nb; ++i) {
    double xi[3];
    mat34_apply(p->N[i], x, xi);
    for (int a = 0; a < 3; ++a) y[a] += w[i] * xi[a];
    if (J) {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          J[a * 3 + b] += w[i] * p->N[i][a * 4 + b] + xi[a] * dw[3 * i + b];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Correspondence search (Fast-SNARF style Broyden, Sec. 3.1)                 */
/* ------------------------------------------------------------------------- */

/* Broyden's method on g(x) = LBS(x) - x' from x0.  The initial inverse Jacobian
   is that of LBS with the skinning weights held at their value at x0, i.e.
   (sum_i w_i(x0) R_i)^-1 (with m->h0_analytic: the full analytic J(x0)^-1);
   the good-Broyden rank-one updates then correct it. */
int or_broyden(const or_model *m, const or_pose *p, const double xn[3], const double x0[3],
               double x[3], int *iters, double *res_norm, int *flags) {
  double y[3], J[9], H[9], r[3], det, w[OR_MAX_BONES];
  int fl = 0;
  for (int a = 0; a < 3; ++a) x[a] = x0[a];
  if (m->h0_analytic) {
    or_lbs(m, p, x, y, J);
  } else {
    or_lbs(m, p, x, y, NULL);
    or_skin(m, x, w, NULL);
    for (int i = 0; i < 9; ++i) J[i] = 0.0;
    for (int i = 0; i < m->nb; ++i)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) J[a * 3 + b] += w[i] * p->N[i][a * 4 + b];
  }
  for (int a = 0; a < 3; ++a) r[a] = y[a] - xn[a];
  int ok = inv3(J, H, &det);
  if (fabs(det) > 0.5e-6 && fabs(det) < 2e-6) fl |= OR_FLAG_SING;
  if (!ok) {
    if (iters) *iters = 0;
    if (res_norm) *res_norm = norm3(r);
    if (flags) *flags |= fl;
    return 0;
  }
  double tol2 = m->tol * m->tol;
  int n = 0;
  for (; n < m->max_iter; ++n) {
    double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (rr < tol2) break;
    double dx[3], rn[3], dr[3], u[3];
    for (int a = 0; a < 3; ++a) dx[a] = -(H[a * 3 + 0] * r[0] + H[a * 3 + 1] * r[1] + H[a * 3 + 2] * r[2]);
    for (int a = 0; a < 3; ++a) x[a] += dx[a];
    or_lbs(m, p, x, y, NULL);
    for (int a = 0; a < 3; ++a) {
      rn[a] = y[a] - xn[a];
      dr[a] = rn[a] - r[a];
      r[a] = rn[a];
    }
    /* good Broyden update of the inverse Jacobian:
       H += (dx - H dr) (dx^T H) / (dx^T H dr) */
    for (int a = 0; a < 3; ++a) u[a] = H[a * 3 + 0] * dr[0] + H[a * 3 + 1] * dr[1] + H[a * 3 + 2] * dr[2];
    double den = dx[0] * u[0] + dx[1] * u[1] + dx[2] * u[2];
    if (fabs(den) > 1e-12) {
      double aa[3], bt[3];
      for (int a = 0; a < 3; ++a) aa[a] = dx[a] - u[a];
      for (int b = 0; b < 3; ++b) bt[b] = dx[0] * H[0 * 3 + b] + dx[1] * H[1 * 3 + b] + dx[2] * H[2 * 3 + b];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) H[a * 3 + b] += aa[a] * bt[b] / den;
    }
  }
  double rnorm = norm3(r);
  int conv = rnorm < m->tol;
  /* the convergence decision at the iteration cap is the one an fp32 trajectory
     can take differently; flag residuals within a factor 2 of the tolerance */
  if (n == m->max_iter && rnorm > 0.5 * m->tol && rnorm < 2.0 * m->tol) fl |= OR_FLAG_CONV;
  if (iters) *iters = n;
  if (res_norm) *res_norm = rnorm;
  if (flags) *flags |= fl;
  return conv;
}

double or_polish(const or_model *m, const or_pose *p, const double xn[3], double x[3]) {
  double y[3], J[9], H[9], r[3];
  double rn = 0.0;
  for (int it = 0; it < 30; ++it) {
    or_lbs(m, p, x, y, J);
    for (int a = 0; a < 3; ++a) r[a] = y[a] - xn[a];
    rn = norm3(r);
    if (rn < 1e-12) break;
    if (!inv3(J, H, NULL)) break;
    for (int a = 0; a < 3; ++a) x[a] -= H[a * 3 + 0] * r[0] + H[a * 3 + 1] * r[1] + H[a * 3 + 2] * r[2];
  }
  return rn;
}

static int in_box(const or_model *m, const double x[3]) {
  for (int a = 0; a < 3; ++a)
    if (!(x[a] >= m->cmin[a] && x[a] <= m->cmax[a])) return 0;
  return 1;
}

static double box_margin(const or_model *m, const double x[3]) {
  double d = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double e = fmin(fabs(x[a] - m->cmin[a]), fabs(x[a] - m->cmax[a]));
    if (e < d) d = e;
  }
  return d;
}

/* Roots reached from a list of starts x0s[j] (labelled labels[j]); valid =
   converged and inside the canonical box; roots are polished and merged when
   closer than 1e-4 (the earliest start kept).  A start whose convergence
   decision at the iteration cap is marginal (see or_broyden) only raises
   OR_FLAG_CONV when its nearby root would be a root no other start found, i.e.
   when an fp32 trajectory could change the root set. */
int or_roots_from_starts(const or_model *m, const or_pose *p, const double xn[3], int ns,
                         const double *x0s, const int *labels, double *roots, int *starts, int *flags,
                         int *iters_sum, int *n_conv) {
  int n = 0, fl = 0, its = 0, nc = 0;
  double xs[OR_MAX_STARTS][3];
  int conv[OR_MAX_STARTS], marg[OR_MAX_STARTS];
  for (int k = 0; k < ns; ++k) {
    double rn;
    int it = 0, f = 0;
    conv[k] = or_broyden(m, p, xn, x0s + 3 * k, xs[k], &it, &rn, &f);
    marg[k] = (f & OR_FLAG_CONV) != 0;
    fl |= f & ~OR_FLAG_CONV;
    its += it;
    if (conv[k] || marg[k]) or_polish(m, p, xn, xs[k]);
  }
  for (int k = 0; k < ns; ++k) {
    if (!conv[k]) continue;
    double *x = xs[k];
    if (box_margin(m, x) < 1e-4) fl |= OR_FLAG_BOX;
    if (!in_box(m, x)) continue;
    nc++;
    int dup = 0;
    for (int j = 0; j < n; ++j) {
      double d[3] = {x[0] - roots[3 * j], x[1] - roots[3 * j + 1], x[2] - roots[3 * j + 2]};
      double dist = norm3(d);
      if (dist > 0.5e-4 && dist < 2e-4) fl |= OR_FLAG_DUP;
      if (dist < 1e-4) { dup = 1; break; }
    }
    if (dup) continue;
    roots[3 * n] = x[0];
    roots[3 * n + 1] = x[1];
    roots[3 * n + 2] = x[2];
    starts[n] = labels[k];
    n++;
  }
  for (int k = 0; k < ns; ++k) {
    if (!marg[k] || !in_box(m, xs[k])) continue;
    int shared = 0;
    for (int q = 0; q < ns; ++q) {
      if (q == k || !conv[q] || marg[q]) continue;
      double d[3] = {xs[k][0] - xs[q][0], xs[k][1] - xs[q][1], xs[k][2] - xs[q][2]};
      if (norm3(d) < 1e-4) { shared = 1; break; }
    }
    if (!shared) fl |= OR_FLAG_CONV;
  }
  if (flags) *flags |= fl;
  if (iters_sum) *iters_sum = its;
  if (n_conv) *n_conv = nc;
  return n;
}

/* All bone-wise starts x0 = N_k^-1 x', labelled by their bone. */
static int roots_impl(const or_model *m, const or_pose *p, const double xn[3], double *roots,
                      int *starts, int *flags, int *iters_sum, int *n_conv) {
  double x0s[OR_MAX_BONES * 3];
  int labels[OR_MAX_BONES];
  for (int k = 0; k < m->nb; ++k) {
    mat34_apply(p->Ninv[k], xn, x0s + 3 * k);
    labels[k] = k;
  }
  return or_roots_from_starts(m, p, xn, m->nb, x0s, labels, roots, starts, flags, iters_sum, n_conv);
}

int or_roots(const or_model *m, const or_pose *p, const double xn[3], double *roots, int *starts,
             int *flags) {
  return roots_impl(m, p, xn, roots, starts, flags, NULL, NULL);
}

/* ------------------------------------------------------------------------- */
/* Canonical field (Eq. 1-2): multiresolution hash encoding + MLP              */
/* ------------------------------------------------------------------------- */

static void level_layout(const or_model *m, long *offset, long *size) {
  long T = 1L << m->log2_T, off = 0;
  for (int l = 0; l < m->L; ++l) {
    long r1 = (long)m->res[l] + 1;
    long dense = r1 * r1 * r1;
    size[l] = dense <= T ? dense : T;
    offset[l] = off;
    off += size[l];
  }
}

/* grid vertex (i,j,k) of level l -> entry within the level: dense row-major
   index when the level fits the table, else the XOR spatial hash with the
   primes 1, 2654435761, 805459861 taken modulo the table size */
static long vertex_index(const or_model *m, int l, long size, int i, int j, int k) {
  long r1 = (long)m->res[l] + 1;
  if (r1 * r1 * r1 <= size) return (long)i + r1 * ((long)j + r1 * (long)k);
  uint32_t h = (uint32_t)i * 1u ^ (uint32_t)j * 2654435761u ^ (uint32_t)k * 805459861u;
  return (long)(h % (uint32_t)size);
}

void or_encode(const or_model *m, const double x[3], double *feat) {
  long offset[OR_MAX_LEVELS], size[OR_MAX_LEVELS];
  level_layout(m, offset, size);
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (x[a] - m->cmin[a]) / (m->cmax[a] - m->cmin[a]);
  for (int l = 0; l < m->L; ++l) {
    int res = m->res[l];
    int p0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double pos = u[a] * (double)res;
      int c = (int)floor(pos);
      if (c > res - 1) c = res - 1;
      if (c < 0) c = 0;
      p0[a] = c;
      f[a] = pos - (double)c;
    }
    for (int q = 0; q < m->F; ++q) feat[l * m->F + q] = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
      int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
      double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
      long e = offset[l] + vertex_index(m, l, size[l], p0[0] + cx, p0[1] + cy, p0[2] + cz);
      for (int q = 0; q < m->F; ++q) feat[l * m->F + q] += w * m->table[e * m->F + q];
    }
  }
}

void or_mlp(const or_model *m, const double *feat, double out[4]) {
  double h1[256], h2[256];
  int W = m->width;
  for (int j = 0; j < W; ++j) {
    double s = m->b1[j];
    for (int i = 0; i < m->n_in; ++i) s += m->W1[j * m->n_in + i] * feat[i];
    h1[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < W; ++j) {
    double s = m->b2[j];
    for (int i = 0; i < W; ++i) s += m->W2[j * W + i] * h1[i];
    h2[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < 4; ++j) {
    double s = m->b3[j];
    for (int i = 0; i < W; ++i) s += m->W3[j * W + i] * h2[i];
    out[j] = s;
  }
}

/* density = exp(clamp(o0, -15, 15)), colour = sigmoid(o1..3) */
void or_field(const or_model *m, const double x[3], double *sigma, double rgb[3]) {
  double feat[OR_MAX_LEVELS * 8], o[4];
  or_encode(m, x, feat);
  or_mlp(m, feat, o);
  double s = o[0] < -15.0 ? -15.0 : (o[0] > 15.0 ? 15.0 : o[0]);
  *sigma = exp(s);
  for (int c = 0; c < 3; ++c) rgb[c] = 1.0 / (1.0 + exp(-o[1 + c]));
}

/* f'(x') = f(x*): the root with the highest density among the distinct valid
   roots (ties -> earliest start); no valid root -> density 0 */
/* f'(x') = f(x*) over a root set: the root with the highest density (ties ->
   the earlier root); no root -> density 0 */
void or_select_root(const or_model *m, int n, const double *roots, const int *starts, int flags,
                    int iters, int n_conv, or_sample *s) {
  memset(s, 0, sizeof(*s));
  s->start = -1;
  double best = -1.0, second = -1.0;
  for (int j = 0; j < n; ++j) {
    double sig, rgb[3];
    or_field(m, roots + 3 * j, &sig, rgb);
    if (sig > best) {
      second = best;
      best = sig;
      s->sigma = sig;
      for (int c = 0; c < 3; ++c) { s->rgb[c] = rgb[c]; s->xstar[c] = roots[3 * j + c]; }
      s->start = starts[j];
    } else if (sig > second) {
      second = sig;
    }
  }
  if (n >= 2 && best - second <= 1e-3 * best) flags |= OR_FLAG_TIE;
  s->n_conv = n_conv;
  s->n_unique = n;
  s->flags = flags;
  s->iters = iters;
}

/* f'(x') = f(x*): the root with the highest density among the distinct valid
   roots of all bone-wise starts */
void or_posed_field(const or_model *m, const or_pose *p, const double xn[3], or_sample *s) {
  double roots[OR_MAX_BONES * 3];
  int starts[OR_MAX_BONES];
  int fl = 0, its = 0, nc = 0;
  int n = roots_impl(m, p, xn, roots, starts, &fl, &its, &nc);
  or_select_root(m, n, roots, starts, fl, its, nc, s);
}

/* ------------------------------------------------------------------------- */
/* fp32 indexing (Sec. 3.2 ray samples, Sec. 3.3 occupancy cells)             */
/* ------------------------------------------------------------------------- */

int or_ray(const or_model *m, const or_pose *p, const or_camera *c, int u, int v, float o[3],
           float d[3], float *t_near, float *t_far) {
  float dc[3], dw[3], ow[3];
  dc[0] = (((float)u + 0.5f) - c->cx) / c->fx;
  dc[1] = (((float)v + 0.5f) - c->cy) / c->fy;
  dc[2] = 1.0f;
  for (int i = 0; i < 3; ++i) {
    dw[i] = ((c->c2w[i * 4 + 0] * dc[0]) + (c->c2w[i * 4 + 1] * dc[1])) + (c->c2w[i * 4 + 2] * dc[2]);
    ow[i] = c->c2w[i * 4 + 3];
  }
  float nrm = sqrtf(((dw[0] * dw[0]) + (dw[1] * dw[1])) + (dw[2] * dw[2]));
  for (int i = 0; i < 3; ++i) dw[i] = dw[i] / nrm;
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
  *t_near = tmin;
  *t_far = tmax;
  return tmax > tmin;
}

int or_cell(const or_model *m, const float x[3]) {
  int R = m->occ_res, c[3];
  for (int a = 0; a < 3; ++a) {
    float s = (float)R / (m->nmax[a] - m->nmin[a]);
    int q = (int)floorf((x[a] - m->nmin[a]) * s);
    if (q < 0) q = 0;
    if (q > R - 1) q = R - 1;
    c[a] = q;
  }
  return c[0] + R * (c[1] + R * c[2]);
}

void or_cell_center(const or_model *m, int cell, float x[3]) {
  int R = m->occ_res;
  int c[3] = {cell % R, (cell / R) % R, cell / (R * R)};
  for (int a = 0; a < 3; ++a) {
    float cs = (m->nmax[a] - m->nmin[a]) / (float)R;
    x[a] = m->nmin[a] + (((float)c[a] + 0.5f) * cs);
  }
}

static void slot_position(const float o[3], const float d[3], float tn, float dt, int i, float x[3]) {
  float t = tn + (((float)i + 0.5f) * dt);
  for (int a = 0; a < 3; ++a) x[a] = o[a] + (t * d[a]);
}

/* ------------------------------------------------------------------------- */
/* Volume rendering (Eq. 8, with alpha = 1 - exp(-sigma delta))               */
/* ------------------------------------------------------------------------- */

/* One pixel's ray.  With q (a correspondence proposal and the pose's
   axis-angles theta) every sample's search starts from the proposal's bones
   and falls back to every bone-wise start when they find no valid root
   (or_posed_field_prop); *nfb counts those fallbacks (may be NULL). */
static void render_ray(const or_model *m, const or_pose *p, const or_camera *c, const uint32_t *occ,
                       int u, int v, double rgb[3], double *alpha, int *flags, int *nsamp,
                       int64_t *iters, const or_prop *q, const double *theta, int *nfb) {
  float o[3], d[3], tn, tf;
  double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
  int fl = 0, ns = 0;
  int64_t its = 0;
  if (or_ray(m, p, c, u, v, o, d, &tn, &tf)) {
    float dt = (tf - tn) / (float)m->n_slots;
    for (int i = 0; i < m->n_slots; ++i) {
      float x[3];
      slot_position(o, d, tn, dt, i, x);
      int cell = or_cell(m, x);
      if (!((occ[cell >> 5] >> (cell & 31)) & 1u)) continue; /* empty-space skipping */
      ns++;
      or_sample s;
      double xn[3] = {(double)x[0], (double)x[1], (double)x[2]};
      if (q) {
        int fb = 0;
        or_posed_field_prop(m, p, q, theta, xn, &s, &fb);
        if (nfb) *nfb += fb;
      } else {
        or_posed_field(m, p, xn, &s);
      }
      fl |= s.flags;
      its += s.iters;
      if (s.start >= 0) {
        double a = 1.0 - exp(-s.sigma * (double)dt);
        for (int k = 0; k < 3; ++k) C[k] += T * a * s.rgb[k];
        T *= 1.0 - a;
      }
      if (m->early_T > 0.0 && fabs(T / m->early_T - 1.0) < 1e-3) fl |= OR_FLAG_TERM;
      if (m->early_T > 0.0 && T < m->early_T) break;
    }
  }
  for (int k = 0; k < 3; ++k) rgb[k] = C[k];
  *alpha = 1.0 - T;
  if (flags) *flags = fl;
  if (nsamp) *nsamp = ns;
  if (iters) *iters = its;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

void or_render(const or_model *m, const or_pose *p, const or_camera *c, const uint32_t *occ,
               double *rgb, double *alpha, int *ray_flags, int *ray_nsamp, int64_t *ray_iters,
               int nthreads) {
  set_threads(nthreads);
  int W = c->width, H = c->height;
#pragma omp parallel for schedule(dynamic, 16)
  for (int r = 0; r < W * H; ++r) {
    int fl, ns;
    int64_t it;
    render_ray(m, p, c, occ, r % W, r / W, rgb + 3 * r, alpha + r, &fl, &ns, &it, NULL, NULL, NULL);
    if (ray_flags) ray_flags[r] = fl;
    if (ray_nsamp) ray_nsamp[r] = ns;
    if (ray_iters) ray_iters[r] = it;
  }
}

void or_render_pixels(const or_model *m, const or_pose *p, const or_camera *c,
                      const uint32_t *occ, int n, const int32_t *pix, double *rgb,
                      double *alpha, int *ray_flags, int *ray_nsamp, int nthreads) {
  set_threads(nthreads);
  int W = c->width;
#pragma omp parallel for schedule(dynamic, 4)
  for (int r = 0; r < n; ++r) {
    int fl, ns;
    int64_t it;
    render_ray(m, p, c, occ, pix[r] % W, pix[r] / W, rgb + 3 * r, alpha + r, &fl, &ns, &it, NULL, NULL, NULL);
    if (ray_flags) ray_flags[r] = fl;
    if (ray_nsamp) ray_nsamp[r] = ns;
  }
}

void or_render_pixels_prop(const or_model *m, const or_pose *p, const or_prop *q, const double *theta,
                           const or_camera *c, const uint32_t *occ, int n, const int32_t *pix, double *rgb,
                           double *alpha, int *ray_flags, int *ray_nsamp, int *ray_fallbacks, int nthreads) {
  set_threads(nthreads);
  int W = c->width;
#pragma omp parallel for schedule(dynamic, 4)
  for (int r = 0; r < n; ++r) {
    int fl, ns, fb = 0;
    int64_t it;
    render_ray(m, p, c, occ, pix[r] % W, pix[r] / W, rgb + 3 * r, alpha + r, &fl, &ns, &it, q, theta, &fb);
    if (ray_flags) ray_flags[r] = fl;
    if (ray_nsamp) ray_nsamp[r] = ns;
    if (ray_fallbacks) ray_fallbacks[r] = fb;
  }
}

void or_march_mask(const or_model *m, const or_pose *p, const or_camera *c, const uint32_t *occ,
                   uint32_t *mask) {
  int W = c->width, H = c->height, words = (m->n_slots + 31) / 32;
  for (int r = 0; r < W * H; ++r) {
    uint32_t *mk = mask + (long)r * words;
    for (int w = 0; w < words; ++w) mk[w] = 0u;
    float o[3], d[3], tn, tf;
    if (!or_ray(m, p, c, r % W, r / W, o, d, &tn, &tf)) continue;
    float dt = (tf - tn) / (float)m->n_slots;
    for (int i = 0; i < m->n_slots; ++i) {
      float x[3];
      slot_position(o, d, tn, dt, i, x);
      int cell = or_cell(m, x);
      if ((occ[cell >> 5] >> (cell & 31)) & 1u) mk[i >> 5] |= 1u << (i & 31);
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Occupancy grid, inference mode (Sec. 3.3)                                  */
/* ------------------------------------------------------------------------- */

/* threshold (sigma > tau), dilation by a (2r+1)^3 cube clipped to the grid,
   packing: bit b = x + R (y + R z) lives in word b / 32 at position b % 32 */
void or_occ_bits(int R, int dilate, double tau, const double *sigma, uint32_t *bits) {
  long n = (long)R * R * R;
  memset(bits, 0, (size_t)((n + 31) / 32) * sizeof(uint32_t));
  for (long b = 0; b < n; ++b) {
    int x = (int)(b % R), y = (int)((b / R) % R), z = (int)(b / ((long)R * R));
    int on = 0;
    for (int dz = -dilate; dz <= dilate && !on; ++dz)
      for (int dy = -dilate; dy <= dilate && !on; ++dy)
        for (int dx = -dilate; dx <= dilate && !on; ++dx) {
          int xx = x + dx, yy = y + dy, zz = z + dz;
          if (xx < 0 || yy < 0 || zz < 0 || xx >= R || yy >= R || zz >= R) continue;
          if (sigma[xx + (long)R * (yy + (long)R * zz)] > tau) on = 1;
        }
    if (on) bits[b >> 5] |= 1u << (b & 31);
  }
}

void or_occ_bits_f32(int R, int dilate, float tau, const float *sigma, uint32_t *bits) {
  long n = (long)R * R * R;
  double *s = (double *)malloc((size_t)n * sizeof(double));
  for (long i = 0; i < n; ++i) s[i] = (double)sigma[i];
  or_occ_bits(R, dilate, (double)tau, s, bits);
  free(s);
}

void or_occupancy(const or_model *m, const or_pose *p, double *sigma, uint32_t *bits,
                  int nthreads) {
  set_threads(nthreads);
  int R = m->occ_res;
  long n = (long)R * R * R;
#pragma omp parallel for schedule(dynamic, 64)
  for (long cell = 0; cell < n; ++cell) {
    float x[3];
    or_cell_center(m, (int)cell, x);
    double xn[3] = {(double)x[0], (double)x[1], (double)x[2]};
    or_sample s;
    or_posed_field(m, p, xn, &s);
    sigma[cell] = s.start >= 0 ? s.sigma : 0.0;
  }
  if (bits) or_occ_bits(R, m->dilate, m->tau, sigma, bits);
}

/* Training-mode occupancy (Sec. 3.3, training stage): one grid for the whole
 * sequence.  Each update queries the posed field of one frame at one point per
 * cell, x = norm_min + (c + u) * (norm_max - norm_min) / R (fp32, fixed order;
 * u = jitter[cell][3] in [0, 1), NULL = the cell centre), and folds it into the
 * running density d <- max(decay * d, sigma); the bits are d thresholded and
 * dilated as in or_occ_bits. */
void or_occupancy_ema(const or_model *m, const or_pose *p, const float *jitter, double decay, double *d,
                      uint32_t *bits, int nthreads) {
  set_threads(nthreads);
  int R = m->occ_res;
  long n = (long)R * R * R;
#pragma omp parallel for schedule(dynamic, 64)
  for (long cell = 0; cell < n; ++cell) {
    int c[3] = {(int)(cell % R), (int)((cell / R) % R), (int)(cell / ((long)R * R))};
    float x[3];
    for (int a = 0; a < 3; ++a) {
      float cs = (m->nmax[a] - m->nmin[a]) / (float)R;
      float u = jitter ? jitter[3 * cell + a] : 0.5f;
      x[a] = m->nmin[a] + (((float)c[a] + u) * cs);
    }
    double xn[3] = {(double)x[0], (double)x[1], (double)x[2]};
    or_sample s;
    or_posed_field(m, p, xn, &s);
    double sig = s.start >= 0 ? s.sigma : 0.0;
    double old = decay * d[cell];
    d[cell] = sig > old ? sig : old;
  }
  if (bits) or_occ_bits(R, m->dilate, m->tau, d, bits);
}

void or_occupancy_cells(const or_model *m, const or_pose *p, int n, const int32_t *cells,
                        double *sigma, int nthreads) {
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) {
    float x[3];
    or_cell_center(m, cells[i], x);
    double xn[3] = {(double)x[0], (double)x[1], (double)x[2]};
    or_sample s;
    or_posed_field(m, p, xn, &s);
    sigma[i] = s.start >= 0 ? s.sigma : 0.0;
  }
}

/* ------------------------------------------------------------------------- */
/* Brute-force root set (pin for the multi-start search)                      */
/* ------------------------------------------------------------------------- */

int or_bruteforce_roots(const or_model *m, const or_pose *p, const double xn[3], int n,
                        double seed_thresh, double *roots, int max_roots) {
  int count = 0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double x[3], y[3];
        int idx[3] = {i, j, k};
        for (int a = 0; a < 3; ++a)
          x[a] = m->cmin[a] + (m->cmax[a] - m->cmin[a]) * ((double)idx[a] + 0.5) / (double)n;
        or_lbs(m, p, x, y, NULL);
        double r[3] = {y[0] - xn[0], y[1] - xn[1], y[2] - xn[2]};
        if (norm3(r) > seed_thresh) continue;
        double rn = or_polish(m, p, xn, x);
        if (!(rn < 1e-10) || !in_box(m, x)) continue;
        int dup = 0;
        for (int q = 0; q < count; ++q) {
          double d[3] = {x[0] - roots[3 * q], x[1] - roots[3 * q + 1], x[2] - roots[3 * q + 2]};
          if (norm3(d) < 1e-4) { dup = 1; break; }
        }
        if (dup || count >= max_roots) continue;
        for (int a = 0; a < 3; ++a) roots[3 * count + a] = x[a];
        count++;
      }
  return count;
}
