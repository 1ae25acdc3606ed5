/*
 * FP64 CPU oracle, learned correspondence proposal.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper searches for x* from every bone-wise start (Sec. 3.1, Fast-SNARF)
 * and has no learned component for it.  The proposal network maps a posed point
 * and the pose to a guess of the bone whose region holds x* and to an offset of
 * the start, so the search can begin from one or two starts; the plain search
 * over all bones remains the fallback whenever the proposed starts find no valid
 * root.
 *
 *   input   [hash features of x' in the normalised box (L levels x 2) | pose
 *           axis-angles (n_b x 3)]
 *   MLP     -> 64 -> ReLU -> 64 -> ReLU -> 64 -> ReLU -> (n_b logits, 3 offset)
 *   label   the bone with the largest skinning weight at the selected root x*
 *   target  offset = x* - N_label^-1 x'
 *   loss    mean over pairs of  CE(logits, label) + w |offset - target|^2
 *   search  starts N_k1^-1 x' + offset and N_k2^-1 x' for the two largest logits
 *           (ties to the lower bone); no valid root -> all bone-wise starts.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static void prop_layout(const or_prop *q, long *offset, long *size) {
  long T = 1L << q->log2_T, off = 0;
  for (int l = 0; l < q->L; ++l) {
    long r1 = (long)q->res[l] + 1;
    size[l] = r1 * r1 * r1 <= T ? r1 * r1 * r1 : T;
    offset[l] = off;
    off += size[l];
  }
}

/* trilinear hash encoding of x' over the normalised box (same rules as the
   canonical grid: dense row-major levels, else the XOR spatial hash) */
void or_prop_encode(const or_model *m, const or_prop *q, const double xn[3], double *feat, long *entry,
                    double *weight) {
  long offset[OR_MAX_LEVELS], size[OR_MAX_LEVELS];
  prop_layout(q, offset, size);
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (xn[a] - (double)m->nmin[a]) / ((double)m->nmax[a] - (double)m->nmin[a]);
  for (int l = 0; l < q->L; ++l) {
    int res = q->res[l], p0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double pos = u[a] * (double)res;
      int c = (int)floor(pos);
      if (c > res - 1) c = res - 1;
      if (c < 0) c = 0;
      p0[a] = c;
      f[a] = pos - (double)c;
    }
    feat[2 * l] = feat[2 * l + 1] = 0.0;
    long r1 = (long)res + 1;
    for (int corner = 0; corner < 8; ++corner) {
      int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
      double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
      int i = p0[0] + cx, j = p0[1] + cy, k = p0[2] + cz;
      long e;
      if (r1 * r1 * r1 <= size[l]) {
        e = (long)i + r1 * ((long)j + r1 * (long)k);
      } else {
        uint32_t h = (uint32_t)i * 1u ^ (uint32_t)j * 2654435761u ^ (uint32_t)k * 805459861u;
        e = (long)(h % (uint32_t)size[l]);
      }
      e += offset[l];
      if (entry) { entry[8 * l + corner] = e; weight[8 * l + corner] = w; }
      feat[2 * l] += w * q->table[2 * e];
      feat[2 * l + 1] += w * q->table[2 * e + 1];
    }
  }
}

typedef struct prop_acts {
  double in[OR_MAX_LEVELS * 2 + OR_MAX_BONES * 3];
  double h1p[64], h1[64], h2p[64], h2[64], h3p[64], h3[64];
  double out[OR_MAX_BONES + 3];
  long entry[OR_MAX_LEVELS * 8];
  double weight[OR_MAX_LEVELS * 8];
} prop_acts;

static void dense_relu(const double *W, const double *b, const double *x, int nin, int nout, double *pre,
                       double *post) {
  for (int j = 0; j < nout; ++j) {
    double s = b[j];
    for (int i = 0; i < nin; ++i) s += W[j * nin + i] * x[i];
    pre[j] = s;
    if (post) post[j] = s > 0.0 ? s : 0.0;
  }
}

static void prop_forward_acts(const or_model *m, const or_prop *q, const double xn[3], const double *theta,
                              prop_acts *A) {
  const int W = q->width, nb = m->nb;
  or_prop_encode(m, q, xn, A->in, A->entry, A->weight);
  for (int i = 0; i < 3 * nb; ++i) A->in[2 * q->L + i] = theta[i];
  dense_relu(q->W1, q->b1, A->in, q->n_in, W, A->h1p, A->h1);
  dense_relu(q->W2, q->b2, A->h1, W, W, A->h2p, A->h2);
  dense_relu(q->W3, q->b3, A->h2, W, W, A->h3p, A->h3);
  dense_relu(q->W4, q->b4, A->h3, W, q->n_out, A->out, NULL);
}

void or_prop_forward(const or_model *m, const or_prop *q, const double xn[3], const double *theta,
                     double *out) {
  prop_acts A;
  prop_forward_acts(m, q, xn, theta, &A);
  memcpy(out, A.out, sizeof(double) * q->n_out);
}

/* label = bone of the largest skinning weight at x* (ties -> lower bone),
   offset target = x* - N_label^-1 x' */
int or_prop_label(const or_model *m, const or_pose *p, const double xs[3], const double xn[3],
                  double offset[3]) {
  double w[OR_MAX_BONES];
  or_skin(m, xs, w, NULL);
  int best = 0;
  for (int i = 1; i < m->nb; ++i)
    if (w[i] > w[best]) best = i;
  for (int a = 0; a < 3; ++a) {
    double s = p->Ninv[best][a * 4 + 3];
    for (int b = 0; b < 3; ++b) s += p->Ninv[best][a * 4 + b] * xn[b];
    offset[a] = xs[a] - s;
  }
  return best;
}

long or_prop_mlp_count(const or_prop *q) {
  int W = q->width;
  return (long)W * q->n_in + W + 2L * (W * W + W) + (long)q->n_out * W + q->n_out;
}

/* Mean loss over n pairs and its gradient (table [entries][2], packed MLP). */
double or_prop_loss_grad(const or_model *m, const or_prop *q, int n, const float *x, const int32_t *pose_id,
                         const double *theta_all, const int32_t *label, const double *target, double *g_table,
                         double *g_mlp) {
  const int W = q->width, nb = m->nb, nin = q->n_in, no = q->n_out;
  long offset[OR_MAX_LEVELS], size[OR_MAX_LEVELS], entries = 0;
  prop_layout(q, offset, size);
  for (int l = 0; l < q->L; ++l) entries += size[l];
  if (g_table) memset(g_table, 0, sizeof(double) * 2 * entries);
  if (g_mlp) memset(g_mlp, 0, sizeof(double) * or_prop_mlp_count(q));
  double *gW1 = g_mlp, *gb1 = gW1 + (long)W * nin, *gW2 = gb1 + W, *gb2 = gW2 + (long)W * W;
  double *gW3 = gb2 + W, *gb3 = gW3 + (long)W * W, *gW4 = gb3 + W, *gb4 = gW4 + (long)no * W;
  double loss = 0.0;
  prop_acts A;
  for (int s = 0; s < n; ++s) {
    double xn[3] = {(double)x[3 * s], (double)x[3 * s + 1], (double)x[3 * s + 2]};
    prop_forward_acts(m, q, xn, theta_all + (long)pose_id[s] * nb * 3, &A);
    double mx = A.out[0];
    for (int i = 1; i < nb; ++i) mx = fmax(mx, A.out[i]);
    double z = 0.0;
    for (int i = 0; i < nb; ++i) z += exp(A.out[i] - mx);
    const double lse = mx + log(z);
    double l = lse - A.out[label[s]];
    double dout[OR_MAX_BONES + 3];
    for (int i = 0; i < nb; ++i) dout[i] = (exp(A.out[i] - lse) - (i == label[s] ? 1.0 : 0.0)) / n;
    for (int a = 0; a < 3; ++a) {
      double e = A.out[nb + a] - target[3 * s + a];
      l += q->offset_weight * e * e;
      dout[nb + a] = 2.0 * q->offset_weight * e / n;
    }
    loss += l / n;
    if (!g_mlp) continue;
    double d3[64], d2[64], d1[64], din[OR_MAX_LEVELS * 2 + OR_MAX_BONES * 3];
    for (int j = 0; j < no; ++j) {
      gb4[j] += dout[j];
      for (int i = 0; i < W; ++i) gW4[j * W + i] += dout[j] * A.h3[i];
    }
    for (int i = 0; i < W; ++i) {
      double t = 0.0;
      for (int j = 0; j < no; ++j) t += q->W4[j * W + i] * dout[j];
      d3[i] = A.h3p[i] > 0.0 ? t : 0.0;
    }
    for (int j = 0; j < W; ++j) {
      gb3[j] += d3[j];
      for (int i = 0; i < W; ++i) gW3[j * W + i] += d3[j] * A.h2[i];
    }
    for (int i = 0; i < W; ++i) {
      double t = 0.0;
      for (int j = 0; j < W; ++j) t += q->W3[j * W + i] * d3[j];
      d2[i] = A.h2p[i] > 0.0 ? t : 0.0;
    }
    for (int j = 0; j < W; ++j) {
      gb2[j] += d2[j];
      for (int i = 0; i < W; ++i) gW2[j * W + i] += d2[j] * A.h1[i];
    }
    for (int i = 0; i < W; ++i) {
      double t = 0.0;
      for (int j = 0; j < W; ++j) t += q->W2[j * W + i] * d2[j];
      d1[i] = A.h1p[i] > 0.0 ? t : 0.0;
    }
    for (int j = 0; j < W; ++j) {
      gb1[j] += d1[j];
      for (int i = 0; i < nin; ++i) gW1[j * nin + i] += d1[j] * A.in[i];
    }
    for (int i = 0; i < 2 * q->L; ++i) {
      double t = 0.0;
      for (int j = 0; j < W; ++j) t += q->W1[j * nin + i] * d1[j];
      din[i] = t;
    }
    for (int l2 = 0; l2 < q->L; ++l2)
      for (int c = 0; c < 8; ++c) {
        long e = A.entry[8 * l2 + c];
        double w = A.weight[8 * l2 + c];
        g_table[2 * e] += w * din[2 * l2];
        g_table[2 * e + 1] += w * din[2 * l2 + 1];
      }
  }
  return loss;
}

/* f'(x') with the proposal: starts from the top_k proposed bones (the first
   shifted by the predicted offset); the plain search over all bones when they
   find no valid root.  *fallback = 1 when the plain search ran. */
/* The proposal-mode search from an ordered list of K proposed bones (the first
   start shifted by the predicted offset), with the fallback to every bone-wise
   start when none of them yields a valid root. */
static void prop_search(const or_model *m, const or_pose *p, const int *bones, int K, const double offset[3],
                        const double xn[3], or_sample *s, int *fallback) {
  double x0s[OR_MAX_STARTS * 3], roots[OR_MAX_STARTS * 3];
  int labels[OR_MAX_STARTS], starts[OR_MAX_STARTS];
  for (int j = 0; j < K; ++j) {
    const int k = bones[j];
    for (int a = 0; a < 3; ++a) {
      double v = p->Ninv[k][a * 4 + 3];
      for (int b = 0; b < 3; ++b) v += p->Ninv[k][a * 4 + b] * xn[b];
      x0s[3 * j + a] = v + (j == 0 ? offset[a] : 0.0);
    }
    labels[j] = k;
  }
  int flags = 0, its = 0, nc = 0;
  int n = or_roots_from_starts(m, p, xn, K, x0s, labels, roots, starts, &flags, &its, &nc);
  *fallback = 0;
  if (n == 0) {
    *fallback = 1;
    or_sample t;
    or_posed_field(m, p, xn, &t);
    t.flags |= flags;
    t.iters += its;
    *s = t;
    return;
  }
  or_select_root(m, n, roots, starts, flags, its, nc, s);
}

/* the same selected sample: both without a root, or the same root */
static int same_outcome(const or_sample *a, const or_sample *b) {
  if ((a->start >= 0) != (b->start >= 0)) return 0;
  if (a->start < 0) return 1;
  const double d[3] = {a->xstar[0] - b->xstar[0], a->xstar[1] - b->xstar[1], a->xstar[2] - b->xstar[2]};
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < 1e-12;
}

/* f'(x') with the proposal choosing the starts: the top_k bones by logit (ties
   to the lower bone), the first shifted by the predicted offset; every
   bone-wise start when those find no valid root.  Two choices here are
   discrete: which bones make the top k (the k-th against the next logit) and
   which of them takes the offset (the first against the second).  Where a
   choice is within 0.05 of going the other way -- a reduced-precision network
   may take it differently -- the search is also run with the other choice,
   and OR_FLAG_PROP is raised only if that changes the selected sample (root
   or none) or whether the fallback ran. */
void or_posed_field_prop(const or_model *m, const or_pose *p, const or_prop *q, const double *theta,
                         const double xn[3], or_sample *s, int *fallback) {
  double out[OR_MAX_BONES + 3];
  or_prop_forward(m, q, xn, theta, out);
  int order[OR_MAX_BONES];
  for (int i = 0; i < m->nb; ++i) order[i] = i;
  /* stable selection of the largest logits (ties -> lower bone) */
  for (int a = 0; a < m->nb; ++a)
    for (int b = a + 1; b < m->nb; ++b)
      if (out[order[b]] > out[order[a]]) { int t = order[a]; order[a] = order[b]; order[b] = t; }
  int K = q->top_k < m->nb ? q->top_k : m->nb;
  const double *offset = out + m->nb;
  prop_search(m, p, order, K, offset, xn, s, fallback);
  int alt[2][OR_MAX_BONES], n_alt = 0;
  if (K < m->nb && out[order[K - 1]] - out[order[K]] < 0.05) {
    for (int j = 0; j < K; ++j) alt[n_alt][j] = order[j];
    alt[n_alt][K - 1] = order[K];
    n_alt++;
  }
  if (K >= 2 && out[order[0]] - out[order[1]] < 0.05) {
    for (int j = 0; j < K; ++j) alt[n_alt][j] = order[j];
    alt[n_alt][0] = order[1];
    alt[n_alt][1] = order[0];
    n_alt++;
  }
  for (int i = 0; i < n_alt; ++i) {
    or_sample t;
    int fb = 0;
    prop_search(m, p, alt[i], K, offset, xn, &t, &fb);
    if (fb != *fallback || !same_outcome(s, &t)) s->flags |= OR_FLAG_PROP;
  }
}
