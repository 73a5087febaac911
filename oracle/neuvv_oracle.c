/*
 * FP64 oracle for VOctree volume rendering (NeuVV, arxiv 2202.06088).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the bench's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two meet only through
 * the seeded input generator.
 *
 * Everything is plain double-precision C, written to be checked against the
 * paper by eye, slow on purpose:
 *   - real 4D hyperspherical harmonics (Eq. complex-HSH, Eq. real-SH, App. A),
 *     evaluated from their definition with generic recurrences;
 *   - density sigma = ReLU(a(t) . w_sigma)            (Eq. project-sigma)
 *   - hyper angle gamma = pi * sigmoid(b(t) . w_gamma) (Eq. project-gamma)
 *   - colour c = act(sum w_nlm H_nlm(theta, phi, gamma)) (Eq. HH-color-2)
 *   - voxels on the ray and their chord lengths         (Sec. 4.3 "Rendering")
 *   - front-to-back compositing, alpha                  (Eq. volume-rendering)
 *   - the analytic gradient of both with respect to the leaf coefficients
 *     (Sec. 4.3 "Optimization")
 *   - spatial/temporal edits and depth-ordered blending (Eq. st_composite_affine,
 *     Algorithm 1)
 *   - Adam on touched leaves, BF16 rounding of stored coefficients, FP8 E4M3
 *     rounding with per-leaf power-of-two scales (a storage ablation);
 *   - appearance edits (Sec. 5 "Appearance editing": the terminating voxel of
 *     a ray where its accumulated alpha reaches a threshold, and rendering
 *     with per-voxel target colour, density and time);
 *   - the time slice (Sec. 7 and the caption of the HH-colour figure: at a
 *     fixed time the hyper angle gamma(t) is a constant, and the 4D
 *     harmonics reduce to 3D spherical harmonics with coefficients
 *     s_lm = sum_n w_nlm R_nl(gamma(t))), and volume rendering of a slice.
 *
 * Readings taken where the paper is garbled or silent (kept identical in the
 * design notes):
 *   A1 normalisation  Abar_{n,l} = 2^l l! sqrt(2(n+1)(n-l)! / (pi (n+l+1)!))
 *      (the printed (n-l+1)! is not orthonormal on S^3);
 *   A2 radial factor  C^{l+1}_{n-l}(cos gamma);
 *   A3 real SH on the unit view direction, theta from +z, phi = atan2(y, x),
 *      no Condon-Shortley phase, sqrt(2) for m != 0, cos for m > 0, sin for m < 0;
 *   A4 harmonic index idx(n,l,m) = n(n+1)(2n+1)/6 + l^2 + l + m;
 *   A6 frame coordinate u = t (T-1), basis rows linearly interpolated;
 *   A7 colour activation sigmoid (identity available);
 *   A8 the ray visits the occupied leaves it crosses with positive chord, found
 *      by a finest-level grid walk (exact ties: x before y before z);
 *   A11 depth = sum(w_i t_mid,i) / alpha if alpha >= 1e-4, else +inf;
 *   A12 compose: layers sorted by depth (stable), premultiplied "over"; or
 *      Algorithm 1 applied literally to premultiplied layers.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EMPTY 0xFFFFFFFFu
#define OR_LEAF 0x80000000u

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int depth, K, T, degree;
  int64_t n_nodes, n_leaves;
  const uint32_t *child;   /* [n_nodes][8], slot = 4x + 2y + z */
  const void *w_sigma;     /* [K][n_leaves] */
  const void *w_gamma;     /* [K][n_leaves] */
  const void *w_hh;        /* [3][N_h][n_leaves] */
  int coeff_f64;           /* 1: planes are double, 0: float */
  const double *A;         /* [T][K] density basis */
  const double *B;         /* [T][K] hyper-angle basis */
  double bmin[3], bmax[3];
} or_tree;

typedef struct {
  double t_stop;    /* early termination threshold on transmittance */
  int act;          /* 0 sigmoid, 1 identity */
} or_opts;

/* ------------------------------------------------------------------------ */
/* Special functions                                                        */
/* ------------------------------------------------------------------------ */

static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

int or_n_hh(int degree) {
  int s = 0;
  for (int n = 0; n <= degree; ++n) s += (n + 1) * (n + 1);
  return s;
}

int or_hh_index(int n, int l, int m) { return n * (n + 1) * (2 * n + 1) / 6 + l * l + l + m; }

/* Gegenbauer polynomial C^lambda_k(x) by the three-term recurrence
   k C_k = 2x(k + lambda - 1) C_{k-1} - (k + 2 lambda - 2) C_{k-2}. */
double or_gegenbauer(int k, double lambda, double x) {
  if (k < 0) return 0.0;
  double c0 = 1.0;
  if (k == 0) return c0;
  double c1 = 2.0 * lambda * x;
  for (int j = 2; j <= k; ++j) {
    double c2 = (2.0 * x * (j + lambda - 1.0) * c1 - (j + 2.0 * lambda - 2.0) * c0) / j;
    c0 = c1;
    c1 = c2;
  }
  return c1;
}

/* Associated Legendre P_l^m(x), m >= 0, WITHOUT the Condon-Shortley phase:
   P_m^m = (2m-1)!! (1-x^2)^{m/2}, P_{m+1}^m = x (2m+1) P_m^m,
   (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m. */
double or_legendre(int l, int m, double x) {
  if (m < 0 || m > l) return 0.0;
  double pmm = 1.0;
  double s = sqrt(fmax(0.0, 1.0 - x * x));
  for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
  if (l == m) return pmm;
  double pm1 = x * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pm1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pm1;
    pm1 = pll;
  }
  return pll;
}

/* Real spherical harmonic Y_lm of a unit direction d (reading A3). */
double or_sh_real(int l, int m, const double d[3]) {
  int am = m < 0 ? -m : m;
  double z = d[2];
  if (z > 1.0) z = 1.0;
  if (z < -1.0) z = -1.0;
  double phi = atan2(d[1], d[0]);
  double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
  double P = or_legendre(l, am, z);
  if (m == 0) return K * P;
  if (m > 0) return sqrt(2.0) * K * P * cos(am * phi);
  return sqrt(2.0) * K * P * sin(am * phi);
}

/* Abar_{n,l}: (2l)!! sqrt(2(n+1)(n-l)! / (pi (n+l+1)!)), reading A1. */
double or_hh_norm(int n, int l) {
  double dfact = pow(2.0, l) * fact(l); /* (2l)!! */
  return dfact * sqrt(2.0 * (n + 1.0) * fact(n - l) / (M_PI * fact(n + l + 1)));
}

/* Radial factor R_nl(gamma) = Abar_{n,l} sin^l(gamma) C^{l+1}_{n-l}(cos gamma). */
double or_hh_radial(int n, int l, double gamma) {
  return or_hh_norm(n, l) * pow(sin(gamma), l) * or_gegenbauer(n - l, l + 1.0, cos(gamma));
}

/* d R_nl / d gamma, using d/dx C^lambda_k(x) = 2 lambda C^{lambda+1}_{k-1}(x). */
double or_hh_radial_dgamma(int n, int l, double gamma) {
  double s = sin(gamma), c = cos(gamma);
  double C = or_gegenbauer(n - l, l + 1.0, c);
  double dC = 2.0 * (l + 1.0) * or_gegenbauer(n - l - 1, l + 2.0, c);
  double t1 = l > 0 ? l * pow(s, l - 1) * c * C : 0.0;
  double t2 = pow(s, l + 1) * dC;
  return or_hh_norm(n, l) * (t1 - t2);
}

/* One real 4D harmonic H_nlm(theta, phi, gamma) (Eq. complex-HSH with Eq. real-SH). */
double or_hh(int n, int l, int m, double gamma, const double d[3]) {
  return or_hh_radial(n, l, gamma) * or_sh_real(l, m, d);
}

/* All harmonics with n <= degree, in idx order; optionally d/dgamma too. */
void or_hh_all(int degree, double gamma, const double d[3], double *out, double *dout) {
  for (int n = 0; n <= degree; ++n)
    for (int l = 0; l <= n; ++l) {
      double R = or_hh_radial(n, l, gamma);
      double dR = dout ? or_hh_radial_dgamma(n, l, gamma) : 0.0;
      for (int m = -l; m <= l; ++m) {
        double Y = or_sh_real(l, m, d);
        out[or_hh_index(n, l, m)] = R * Y;
        if (dout) dout[or_hh_index(n, l, m)] = dR * Y;
      }
    }
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------ */
/* Leaf quantities                                                          */
/* ------------------------------------------------------------------------ */

static double coef(const or_tree *tr, const void *plane, int64_t row, int64_t leaf) {
  int64_t i = row * tr->n_leaves + leaf;
  return tr->coeff_f64 ? ((const double *)plane)[i] : (double)((const float *)plane)[i];
}

/* Basis rows at frame coordinate u in [0, T-1], linearly interpolated (A6). */
static void basis_rows(const or_tree *tr, double u, double *a, double *b) {
  if (u < 0.0) u = 0.0;
  if (u > tr->T - 1) u = tr->T - 1;
  int f0 = (int)floor(u);
  if (f0 > tr->T - 1) f0 = tr->T - 1;
  int f1 = f0 + 1 < tr->T ? f0 + 1 : tr->T - 1;
  double fr = u - f0;
  for (int k = 0; k < tr->K; ++k) {
    a[k] = (1.0 - fr) * tr->A[f0 * tr->K + k] + fr * tr->A[f1 * tr->K + k];
    b[k] = (1.0 - fr) * tr->B[f0 * tr->K + k] + fr * tr->B[f1 * tr->K + k];
  }
}

typedef struct {
  double pre_sigma, sigma;     /* a . w_sigma and its ReLU */
  double pre_gamma, gamma;     /* b . w_gamma and pi * sigmoid of it */
  double z[3], c[3];           /* pre-activation colour and colour */
} or_leaf_eval;

static void eval_leaf(const or_tree *tr, const or_opts *op, int64_t leaf, const double *a, const double *b,
                      const double d[3], double *H, double *dH, or_leaf_eval *e) {
  e->pre_sigma = 0.0;
  e->pre_gamma = 0.0;
  for (int k = 0; k < tr->K; ++k) {
    e->pre_sigma += a[k] * coef(tr, tr->w_sigma, k, leaf);
    e->pre_gamma += b[k] * coef(tr, tr->w_gamma, k, leaf);
  }
  e->sigma = e->pre_sigma > 0.0 ? e->pre_sigma : 0.0;
  e->gamma = M_PI * sigmoid(e->pre_gamma);
  int Nh = or_n_hh(tr->degree);
  or_hh_all(tr->degree, e->gamma, d, H, dH);
  for (int ch = 0; ch < 3; ++ch) {
    double z = 0.0;
    for (int i = 0; i < Nh; ++i) z += coef(tr, tr->w_hh, (int64_t)ch * Nh + i, leaf) * H[i];
    e->z[ch] = z;
    e->c[ch] = op->act == 0 ? sigmoid(z) : z;
  }
}

/* ------------------------------------------------------------------------ */
/* Traversal: finest-level grid walk, consecutive cells of one leaf merged   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t leaf;
  double t0, t1;
} or_seg;

/* Leaf id of the tree cell containing finest cell (x, y, z), or -1 if empty. */
static int64_t lookup(const or_tree *tr, const int64_t cell[3]) {
  uint32_t node = 0;
  for (int L = 0; L < tr->depth; ++L) {
    int bit = tr->depth - 1 - L;
    int slot = (int)(((cell[0] >> bit) & 1) * 4 + ((cell[1] >> bit) & 1) * 2 + ((cell[2] >> bit) & 1));
    uint32_t e = tr->child[(int64_t)node * 8 + slot];
    if (e == OR_EMPTY) return -1;
    if (e & OR_LEAF) return (int64_t)(e & ~OR_LEAF);
    node = e;
  }
  return -1;
}

/* As lookup, and -1 for a cell outside the root box. */
static int64_t lookup_any(const or_tree *tr, const int64_t cell[3]) {
  int64_t N = (int64_t)1 << tr->depth;
  for (int a = 0; a < 3; ++a)
    if (cell[a] < 0 || cell[a] >= N) return -1;
  return lookup(tr, cell);
}

/* The occupied leaves met going from finest cell c one cell along axis a
   (direction sa) and then one along axis b (direction sb): empty cells
   dropped, repeats merged.  Returns their number (<= 3). */
static int path_leaves(const or_tree *tr, const int64_t c[3], int a, int sa, int b, int sb, int64_t out[3]) {
  int64_t c1[3] = {c[0], c[1], c[2]};
  c1[a] += sa;
  int64_t c2[3] = {c1[0], c1[1], c1[2]};
  c2[b] += sb;
  int64_t ids[3] = {lookup_any(tr, c), lookup_any(tr, c1), lookup_any(tr, c2)};
  int n = 0;
  for (int i = 0; i < 3; ++i)
    if (ids[i] >= 0 && (n == 0 || out[n - 1] != ids[i])) out[n++] = ids[i];
  return n;
}

/* Whether crossing a plane of axis a and one of axis b in the other order
   (the two crossings meet at an edge or nearly so) changes the sequence of
   occupied leaves the ray visits. */
static int order_matters(const or_tree *tr, const int64_t c[3], int a, int sa, int b, int sb) {
  int64_t p[3], q[3];
  int np = path_leaves(tr, c, a, sa, b, sb, p), nq = path_leaves(tr, c, b, sb, a, sa, q);
  if (np != nq) return 1;
  for (int i = 0; i < np; ++i)
    if (p[i] != q[i]) return 1;
  return 0;
}

/* Cell index on one axis of the point p moving with velocity v: the cell the
   ray occupies just after this instant. */
static int64_t cell_of(double p, double v, int64_t N) {
  double f = floor(p);
  int64_t c = (int64_t)f;
  if (v < 0.0 && f == p) c -= 1;
  if (c < 0) c = 0;
  if (c > N - 1) c = N - 1;
  return c;
}

/* Occupied-leaf segments of a ray (unit direction dn), in order.  Returns the
   count (<= max_seg), or -1 if max_seg was too small.

   Decision margin (reading A8), when margin != NULL: the smallest distance
   along the ray between two plane crossings on different axes whose order
   decides which occupied leaves the ray visits (order_matters), over the
   crossings at distances up to t_limit; the ray's entry into the root box
   counts as a crossing of its entry plane.  +inf when no such pair exists.
   A ray whose margin exceeds the error of a traversal's crossing distances
   visits the same leaves in that traversal. */
int or_trace_m(const or_tree *tr, const double o[3], const double dn[3], or_seg *segs, int max_seg, double t_limit,
               double *margin) {
  int64_t N = (int64_t)1 << tr->depth;
  double go[3], gd[3];
  double tn = -INFINITY, tf = INFINITY;
  int ax_in = -1;
  if (margin) *margin = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double sc = (double)N / (tr->bmax[a] - tr->bmin[a]);
    go[a] = (o[a] - tr->bmin[a]) * sc;
    gd[a] = dn[a] * sc;
    if (gd[a] == 0.0) {
      if (go[a] < 0.0 || go[a] > (double)N) return 0;
    } else {
      double t0 = (0.0 - go[a]) / gd[a], t1 = ((double)N - go[a]) / gd[a];
      if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
      if (t0 > tn) { tn = t0; ax_in = a; }
      if (t1 < tf) tf = t1;
    }
  }
  double tin = tn > 0.0 ? tn : 0.0;
  if (!(tin < tf)) return 0;
  int64_t cell[3];
  for (int a = 0; a < 3; ++a) cell[a] = cell_of(go[a] + tin * gd[a], gd[a], N);
  if (margin) {
    /* crossings next to the start: the planes of the other axes just behind
       and just ahead of the entry point (or of an origin inside the box) */
    for (int x = 0; x < 3; ++x) {
      if (gd[x] == 0.0 || (tn > 0.0 && x == ax_in)) continue;
      int sx = gd[x] > 0.0 ? 1 : -1;
      double behind = ((double)(sx > 0 ? cell[x] : cell[x] + 1) - go[x]) / gd[x];
      double ahead = ((double)(sx > 0 ? cell[x] + 1 : cell[x]) - go[x]) / gd[x];
      if (tn > 0.0) {
        int si = gd[ax_in] > 0.0 ? 1 : -1;
        int64_t c_out[3] = {cell[0], cell[1], cell[2]};
        c_out[ax_in] -= si;                       /* the cell just outside the entry face */
        if (ahead - tin < *margin && order_matters(tr, c_out, ax_in, si, x, sx)) *margin = ahead - tin;
        int64_t c_prev[3] = {c_out[0], c_out[1], c_out[2]};
        c_prev[x] -= sx;
        if (tin - behind < *margin && order_matters(tr, c_prev, x, sx, ax_in, si)) *margin = tin - behind;
      } else {
        /* origin inside: it could start in the cell behind plane x instead */
        int64_t c_b[3] = {cell[0], cell[1], cell[2]};
        c_b[x] -= sx;
        int64_t lb = lookup_any(tr, c_b), lc = lookup_any(tr, cell);
        if (tin - behind < *margin && lb >= 0 && lb != lc) *margin = tin - behind;
      }
    }
  }
  double t_cur = tin;
  int count = 0;
  int64_t cur = -1;
  double c0 = 0.0, c1 = 0.0;
  for (;;) {
    double tnext[3];
    for (int a = 0; a < 3; ++a) {
      if (gd[a] > 0.0) tnext[a] = ((double)(cell[a] + 1) - go[a]) / gd[a];
      else if (gd[a] < 0.0) tnext[a] = ((double)cell[a] - go[a]) / gd[a];
      else tnext[a] = INFINITY;
    }
    int ax = 0;
    if (tnext[1] < tnext[ax]) ax = 1;
    if (tnext[2] < tnext[ax]) ax = 2;
    if (margin && tnext[ax] <= t_limit) {
      int sa = gd[ax] > 0.0 ? 1 : -1;
      for (int x = 0; x < 3; ++x) {
        if (x == ax || gd[x] == 0.0) continue;
        double gap = tnext[x] - tnext[ax];
        if (gap < *margin && order_matters(tr, cell, ax, sa, x, gd[x] > 0.0 ? 1 : -1)) *margin = gap;
      }
    }
    double t_end = tnext[ax] < tf ? tnext[ax] : tf;
    int64_t leaf = lookup(tr, cell);
    if (leaf >= 0 && leaf == cur) {
      c1 = t_end;
    } else {
      if (cur >= 0 && c1 > c0) {
        if (count >= max_seg) return -1;
        segs[count].leaf = cur; segs[count].t0 = c0; segs[count].t1 = c1; ++count;
      }
      cur = leaf;
      c0 = t_cur;
      c1 = t_end;
    }
    if (tnext[ax] >= tf) break;
    t_cur = tnext[ax];
    cell[ax] += gd[ax] > 0.0 ? 1 : -1;
    if (cell[ax] < 0 || cell[ax] >= N) break;
  }
  if (cur >= 0 && c1 > c0) {
    if (count >= max_seg) return -1;
    segs[count].leaf = cur; segs[count].t0 = c0; segs[count].t1 = c1; ++count;
  }
  return count;
}

int or_trace(const or_tree *tr, const double o[3], const double dn[3], or_seg *segs, int max_seg) {
  return or_trace_m(tr, o, dn, segs, max_seg, INFINITY, NULL);
}

/* Edge of the tree's finest cell (the smallest over the axes), the unit of
   the reported decision margins. */
static double finest_cell(const or_tree *tr) {
  double c = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double e = (tr->bmax[a] - tr->bmin[a]) / (double)((int64_t)1 << tr->depth);
    if (e < c) c = e;
  }
  return c;
}

static int max_segments(const or_tree *tr) { return 3 * (1 << tr->depth) + 8; }

static void unit(const double v[3], double out[3]) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  out[0] = v[0] / n; out[1] = v[1] / n; out[2] = v[2] / n;
}

/* ------------------------------------------------------------------------ */
/* Single-ray rendering (Eq. volume-rendering, Sec. 4.3 "Rendering")        */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rgb[3], alpha, depth, tau;
  int nseg;              /* segments composited (early stop included) */
  double stop_margin;    /* min |tau_{i+1} - ln(1/t_stop)| over composited segments */
  double trace_margin;   /* decision margin of the traversal up to the early stop, in finest cells
                            (computed only when render_ray is asked for it) */
} or_ray_out;

/* Per-sample record kept for the gradient. */
typedef struct {
  int64_t leaf;
  double delta, T, w;
  or_leaf_eval e;
} or_sample;

/* Renders one ray at frame coordinate u.  If samples != NULL, fills it with the
   composited samples (capacity max_segments).  Scratch: segs, H (N_h). */
static void render_ray(const or_tree *tr, const or_opts *op, const double o[3], const double d[3], double u,
                       or_seg *segs, double *H, double *a, double *b, or_ray_out *out, or_sample *samples,
                       int want_margin) {
  double dn[3];
  unit(d, dn);
  basis_rows(tr, u, a, b);
  int ns = or_trace(tr, o, dn, segs, max_segments(tr));
  double tau = 0.0, acc[3] = {0, 0, 0}, alpha = 0.0, dnum = 0.0;
  double lnstop = log(1.0 / op->t_stop);
  out->stop_margin = INFINITY;
  int composited = 0;
  for (int i = 0; i < ns; ++i) {
    or_leaf_eval e;
    eval_leaf(tr, op, segs[i].leaf, a, b, dn, H, NULL, &e);
    double delta = segs[i].t1 - segs[i].t0;
    double T = exp(-tau);                        /* T_i = exp(-sum_{j<i} sigma_j delta_j) */
    double w = T * (1.0 - exp(-e.sigma * delta)); /* T_i (1 - exp(-sigma_i delta_i)) */
    for (int ch = 0; ch < 3; ++ch) acc[ch] += w * e.c[ch];
    alpha += w;
    dnum += w * 0.5 * (segs[i].t0 + segs[i].t1);
    if (samples) {
      samples[i].leaf = segs[i].leaf;
      samples[i].delta = delta;
      samples[i].T = T;
      samples[i].w = w;
      samples[i].e = e;
    }
    tau += e.sigma * delta;
    composited = i + 1;
    double m = fabs(tau - lnstop);
    if (m < out->stop_margin) out->stop_margin = m;
    if (exp(-tau) < op->t_stop) break;
  }
  for (int ch = 0; ch < 3; ++ch) out->rgb[ch] = acc[ch];
  out->alpha = alpha;
  out->tau = tau;
  out->depth = alpha >= 1e-4 ? dnum / alpha : INFINITY;
  out->nseg = composited;
  out->trace_margin = INFINITY;
  if (want_margin) {
    /* crossings after an early stop cannot change the composited segments */
    double t_limit = composited < ns ? segs[composited - 1].t1 : INFINITY, m;
    or_trace_m(tr, o, dn, segs, max_segments(tr), t_limit, &m);
    out->trace_margin = m / finest_cell(tr);
  }
}

/* ------------------------------------------------------------------------ */
/* Threading helper                                                         */
/* ------------------------------------------------------------------------ */

typedef void (*or_range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { or_range_fn fn; void *ctx; int64_t lo, hi; } or_job;

static void *or_job_main(void *p) {
  or_job *j = (or_job *)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(int64_t n, int nthreads, or_range_fn fn, void *ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < nthreads) nthreads = n > 0 ? (int)n : 1;
  pthread_t th[256];
  or_job jobs[256];
  for (int i = 0; i < nthreads; ++i) {
    jobs[i].fn = fn; jobs[i].ctx = ctx;
    jobs[i].lo = n * i / nthreads; jobs[i].hi = n * (i + 1) / nthreads;
  }
  for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, or_job_main, &jobs[i]);
  or_job_main(&jobs[0]);
  for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* Public: render a batch of rays                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  const or_tree *tr;
  const or_opts *op;
  const double *o, *d, *t; /* o, d: [3][n] planes; t: [n] */
  int64_t n;
  double *rgb, *alpha, *depth, *tau, *margin, *trace_margin;
  int32_t *nseg;
} render_ctx;

static void render_range(void *p, int64_t lo, int64_t hi) {
  render_ctx *c = (render_ctx *)p;
  const or_tree *tr = c->tr;
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * max_segments(tr));
  double *H = (double *)malloc(sizeof(double) * or_n_hh(tr->degree));
  double *a = (double *)malloc(sizeof(double) * tr->K), *b = (double *)malloc(sizeof(double) * tr->K);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]};
    double t = c->t[r];
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    or_ray_out out;
    render_ray(tr, c->op, o, d, t * (tr->T - 1), segs, H, a, b, &out, NULL, c->trace_margin != NULL);
    for (int ch = 0; ch < 3; ++ch) c->rgb[3 * r + ch] = out.rgb[ch];
    c->alpha[r] = out.alpha;
    c->depth[r] = out.depth;
    c->tau[r] = out.tau;
    c->nseg[r] = out.nseg;
    if (c->margin) c->margin[r] = out.stop_margin;
    if (c->trace_margin) c->trace_margin[r] = out.trace_margin;
  }
  free(segs); free(H); free(a); free(b);
}

void or_render(const or_tree *tr, const or_opts *op, int64_t n, const double *o, const double *d, const double *t,
               double *rgb, double *alpha, double *depth, double *tau, int32_t *nseg, double *margin,
               double *trace_margin, int nthreads) {
  render_ctx c = {tr, op, o, d, t, n, rgb, alpha, depth, tau, margin, trace_margin, nseg};
  parallel_for(n, nthreads, render_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Public: trace (occupied leaves and chords of each ray)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  const or_tree *tr;
  const double *o, *d;
  int64_t n;
  int max_out;
  int64_t *leaf;
  double *t0, *t1;
  int32_t *count;
  double *margin;     /* decision margin over the whole ray, in finest cells (may be NULL) */
} trace_ctx;

static void trace_range(void *p, int64_t lo, int64_t hi) {
  trace_ctx *c = (trace_ctx *)p;
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * max_segments(c->tr));
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    unit(d, dn);
    double m;
    int ns = or_trace_m(c->tr, o, dn, segs, max_segments(c->tr), INFINITY, c->margin ? &m : NULL);
    c->count[r] = ns;
    if (c->margin) c->margin[r] = m / finest_cell(c->tr);
    for (int i = 0; i < ns && i < c->max_out; ++i) {
      c->leaf[r * c->max_out + i] = segs[i].leaf;
      c->t0[r * c->max_out + i] = segs[i].t0;
      c->t1[r * c->max_out + i] = segs[i].t1;
    }
  }
  free(segs);
}

void or_trace_batch(const or_tree *tr, int64_t n, const double *o, const double *d, int max_out, int64_t *leaf,
                    double *t0, double *t1, int32_t *count, double *margin, int nthreads) {
  trace_ctx c = {tr, o, d, n, max_out, leaf, t0, t1, count, margin};
  parallel_for(n, nthreads, trace_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Public: analytic gradient of a loss L(C, alpha) w.r.t. leaf coefficients  */
/* ------------------------------------------------------------------------ */
/*
 * For composited samples i = 1..M of a ray with C = sum w_i c_i,
 * alpha = sum w_i, w_i = T_i (1 - exp(-sigma_i delta_i)):
 *   dC/dc_i       = w_i
 *   dC/dsigma_i   = delta_i (T_{i+1} c_i - sum_{j>i} w_j c_j)
 *   dalpha/dsigma_i = delta_i (T_{i+1} - sum_{j>i} w_j)
 * (T_{i+1} = T_i exp(-sigma_i delta_i); segments after the early stop do not
 * exist for the loss).  The chain continues through the ReLU (zero slope at
 * pre-activation <= 0), pi * sigmoid, the activation and d H / d gamma.
 */

#define OR_NLOCK 4096

typedef struct {
  const or_tree *tr;
  const or_opts *op;
  const double *o, *d, *t, *g_rgb, *g_alpha;
  int64_t n;
  double *g_sigma, *g_gamma, *g_hh; /* [K][L], [K][L], [3][N_h][L] */
  pthread_mutex_t *locks;
} grad_ctx;

static void grad_range(void *p, int64_t lo, int64_t hi) {
  grad_ctx *c = (grad_ctx *)p;
  const or_tree *tr = c->tr;
  int K = tr->K, Nh = or_n_hh(tr->degree);
  int64_t L = tr->n_leaves;
  int ms = max_segments(tr);
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * ms);
  or_sample *sm = (or_sample *)malloc(sizeof(or_sample) * ms);
  double *H = (double *)malloc(sizeof(double) * Nh), *dH = (double *)malloc(sizeof(double) * Nh);
  double *a = (double *)malloc(sizeof(double) * K), *b = (double *)malloc(sizeof(double) * K);
  double *suffix = (double *)malloc(sizeof(double) * 4 * (ms + 1));
  double *gs = (double *)malloc(sizeof(double) * K), *gg = (double *)malloc(sizeof(double) * K);
  double *gh = (double *)malloc(sizeof(double) * 3 * Nh);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    unit(d, dn);
    double t = c->t[r];
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    or_ray_out out;
    render_ray(tr, c->op, o, d, t * (tr->T - 1), segs, H, a, b, &out, sm, 0);
    int M = out.nseg;
    /* suffix sums over j > i of w_j c_j and w_j */
    for (int q = 0; q < 4; ++q) suffix[4 * M + q] = 0.0;
    for (int i = M - 1; i >= 0; --i)
      for (int q = 0; q < 4; ++q)
        suffix[4 * i + q] = suffix[4 * (i + 1) + q] + sm[i].w * (q < 3 ? sm[i].e.c[q] : 1.0);
    double g[3] = {c->g_rgb[3 * r], c->g_rgb[3 * r + 1], c->g_rgb[3 * r + 2]};
    double gA = c->g_alpha ? c->g_alpha[r] : 0.0;
    for (int i = 0; i < M; ++i) {
      const or_sample *s = &sm[i];
      double Tn = s->T * exp(-s->e.sigma * s->delta);
      double dsig = 0.0;
      for (int ch = 0; ch < 3; ++ch) dsig += g[ch] * s->delta * (Tn * s->e.c[ch] - suffix[4 * (i + 1) + ch]);
      dsig += gA * s->delta * (Tn - suffix[4 * (i + 1) + 3]);
      /* colour */
      or_hh_all(tr->degree, s->e.gamma, dn, H, dH);
      double dz[3], dgamma = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        double dc = s->w * g[ch];
        dz[ch] = c->op->act == 0 ? dc * s->e.c[ch] * (1.0 - s->e.c[ch]) : dc;
        for (int i2 = 0; i2 < Nh; ++i2) {
          gh[ch * Nh + i2] = dz[ch] * H[i2];
          dgamma += dz[ch] * coef(tr, tr->w_hh, (int64_t)ch * Nh + i2, s->leaf) * dH[i2];
        }
      }
      double sg = sigmoid(s->e.pre_gamma);
      double dpre_gamma = dgamma * M_PI * sg * (1.0 - sg);
      double dpre_sigma = s->e.pre_sigma > 0.0 ? dsig : 0.0;
      for (int k = 0; k < K; ++k) {
        gs[k] = dpre_sigma * a[k];
        gg[k] = dpre_gamma * b[k];
      }
      pthread_mutex_t *lk = &c->locks[s->leaf % OR_NLOCK];
      pthread_mutex_lock(lk);
      for (int k = 0; k < K; ++k) {
        c->g_sigma[(int64_t)k * L + s->leaf] += gs[k];
        c->g_gamma[(int64_t)k * L + s->leaf] += gg[k];
      }
      for (int q = 0; q < 3 * Nh; ++q) c->g_hh[(int64_t)q * L + s->leaf] += gh[q];
      pthread_mutex_unlock(lk);
    }
  }
  free(segs); free(sm); free(H); free(dH); free(a); free(b); free(suffix); free(gs); free(gg); free(gh);
}

void or_render_grad(const or_tree *tr, const or_opts *op, int64_t n, const double *o, const double *d,
                    const double *t, const double *g_rgb, const double *g_alpha, double *g_sigma, double *g_gamma,
                    double *g_hh, int nthreads) {
  pthread_mutex_t *locks = (pthread_mutex_t *)malloc(sizeof(pthread_mutex_t) * OR_NLOCK);
  for (int i = 0; i < OR_NLOCK; ++i) pthread_mutex_init(&locks[i], NULL);
  grad_ctx c = {tr, op, o, d, t, g_rgb, g_alpha, n, g_sigma, g_gamma, g_hh, locks};
  parallel_for(n, nthreads, grad_range, &c);
  for (int i = 0; i < OR_NLOCK; ++i) pthread_mutex_destroy(&locks[i]);
  free(locks);
}

/* ------------------------------------------------------------------------ */
/* Public: composition of edited primitives (Eq. st_composite_affine, Alg. 1) */
/* ------------------------------------------------------------------------ */
/*
 * Primitive j: tree trees[j], world-from-local affine M_j = [S | tr] (3x4,
 * row-major; S = s R, uniform scale s > 0), time offset off_j frames, tint.
 * The ray is taken into local space (o' = S^-1 (o - tr), d' = S^-1 d normalised),
 * rendered there (chords in local units, so the look of the object does not
 * change with its size), at frame u' = (u + off_j) mod (T-1) (looping re-time);
 * the layer colour is tint * C_j, its depth s * D_j in world units.
 * mode 0: layers sorted by depth (ties: lower j first), front-to-back "over"
 * on premultiplied colour; mode 1: Algorithm 1 literally, premultiplied.
 */

static void inv3(const double *M, double *Mi) { /* M: 3x4 row-major, uses the 3x3 part */
  double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9], i = M[10];
  double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
  double det = a * A + b * B + c * C;
  Mi[0] = A / det; Mi[1] = -(b * i - c * h) / det; Mi[2] = (b * f - c * e) / det;
  Mi[3] = B / det; Mi[4] = (a * i - c * g) / det; Mi[5] = -(a * f - c * d) / det;
  Mi[6] = C / det; Mi[7] = -(a * h - b * g) / det; Mi[8] = (a * e - b * d) / det;
}

typedef struct {
  const or_tree *const *trees;
  const double *xf, *toff, *tint;
  int n_prims, mode;
  const or_opts *op;
  const double *o, *d, *t;
  int64_t n;
  double *rgb, *alpha, *depth, *margin;
  double *trace_margin;  /* min over the layers of their decision margins, in finest cells (may be NULL) */
  double *depth_margin;  /* min |D_i - D_j| over pairs of layers with finite depths (may be NULL) */
} compose_ctx;

static void compose_range(void *p, int64_t lo, int64_t hi) {
  compose_ctx *c = (compose_ctx *)p;
  int P = c->n_prims;
  int maxK = 1, maxNh = 1, maxseg = 1;
  for (int j = 0; j < P; ++j) {
    if (c->trees[j]->K > maxK) maxK = c->trees[j]->K;
    if (or_n_hh(c->trees[j]->degree) > maxNh) maxNh = or_n_hh(c->trees[j]->degree);
    if (max_segments(c->trees[j]) > maxseg) maxseg = max_segments(c->trees[j]);
  }
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * maxseg);
  double *H = (double *)malloc(sizeof(double) * maxNh);
  double *a = (double *)malloc(sizeof(double) * maxK), *b = (double *)malloc(sizeof(double) * maxK);
  double *LC = (double *)malloc(sizeof(double) * 3 * P), *LA = (double *)malloc(sizeof(double) * P);
  double *LD = (double *)malloc(sizeof(double) * P);
  int *ord = (int *)malloc(sizeof(int) * P);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    unit(d, dn);
    double t = c->t[r];
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double margin = INFINITY, tmargin = INFINITY, dmargin = INFINITY;
    for (int j = 0; j < P; ++j) {
      const or_tree *tr = c->trees[j];
      const double *M = c->xf + 12 * j;
      double Mi[9];
      inv3(M, Mi);
      double q[3] = {o[0] - M[3], o[1] - M[7], o[2] - M[11]}, ol[3], dl[3];
      for (int k = 0; k < 3; ++k) {
        ol[k] = Mi[3 * k] * q[0] + Mi[3 * k + 1] * q[1] + Mi[3 * k + 2] * q[2];
        dl[k] = Mi[3 * k] * dn[0] + Mi[3 * k + 1] * dn[1] + Mi[3 * k + 2] * dn[2];
      }
      double inv_s = sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]); /* = 1/s */
      double period = tr->T - 1;
      double u = fmod(t * period + c->toff[j], period);
      if (u < 0.0) u += period;
      or_ray_out out;
      render_ray(tr, c->op, ol, dl, u, segs, H, a, b, &out, NULL, c->trace_margin != NULL);
      if (out.stop_margin < margin) margin = out.stop_margin;
      if (out.trace_margin < tmargin) tmargin = out.trace_margin;
      for (int ch = 0; ch < 3; ++ch) LC[3 * j + ch] = c->tint[3 * j + ch] * out.rgb[ch];
      LA[j] = out.alpha;
      LD[j] = isinf(out.depth) ? INFINITY : out.depth / inv_s;
    }
    for (int i = 0; i < P; ++i)
      for (int j = i + 1; j < P; ++j)
        if (!isinf(LD[i]) && !isinf(LD[j]) && fabs(LD[i] - LD[j]) < dmargin) dmargin = fabs(LD[i] - LD[j]);
    double I[3], A, D;
    if (c->mode == 0) {
      for (int j = 0; j < P; ++j) ord[j] = j;
      for (int i = 1; i < P; ++i) { /* stable insertion sort by depth */
        int x = ord[i], k = i - 1;
        while (k >= 0 && LD[ord[k]] > LD[x]) { ord[k + 1] = ord[k]; --k; }
        ord[k + 1] = x;
      }
      I[0] = I[1] = I[2] = 0.0; A = 0.0; D = INFINITY;
      for (int i = 0; i < P; ++i) {
        int j = ord[i];
        for (int ch = 0; ch < 3; ++ch) I[ch] += (1.0 - A) * LC[3 * j + ch];
        A += (1.0 - A) * LA[j];
        if (LD[j] < D) D = LD[j];
      }
    } else {
      for (int ch = 0; ch < 3; ++ch) I[ch] = LC[ch];
      A = LA[0];
      D = LD[0];
      for (int i = 1; i < P; ++i) {
        if (LD[i] <= D) {
          for (int ch = 0; ch < 3; ++ch) I[ch] = LC[3 * i + ch] + (1.0 - LA[i]) * I[ch];
          D = LD[i];
        } else {
          for (int ch = 0; ch < 3; ++ch) I[ch] = I[ch] + (1.0 - A) * LC[3 * i + ch];
        }
        A = A + LA[i] * (1.0 - A);
      }
    }
    for (int ch = 0; ch < 3; ++ch) c->rgb[3 * r + ch] = I[ch];
    c->alpha[r] = A;
    c->depth[r] = D;
    if (c->margin) c->margin[r] = margin;
    if (c->trace_margin) c->trace_margin[r] = tmargin;
    if (c->depth_margin) c->depth_margin[r] = dmargin;
  }
  free(segs); free(H); free(a); free(b); free(LC); free(LA); free(LD); free(ord);
}

void or_compose(const or_tree *const *trees, const double *xf, const double *toff, const double *tint, int n_prims,
                int mode, const or_opts *op, int64_t n, const double *o, const double *d, const double *t,
                double *rgb, double *alpha, double *depth, double *margin, double *trace_margin,
                double *depth_margin, int nthreads) {
  compose_ctx c = {trees, xf, toff, tint, n_prims, mode, op, o, d, t, n, rgb, alpha, depth, margin, trace_margin,
                   depth_margin};
  parallel_for(n, nthreads, compose_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Public: Adam on touched leaves (Sec. 4.3 "Optimization": SGD or Adam)     */
/* ------------------------------------------------------------------------ */
/* Rows of `rec` values per leaf.  Leaves with touched[leaf] == 0 are left as
   they are (moments included): the update is sparse.  Bias-corrected Adam:
   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
   w -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
void or_adam(int64_t n_leaves, int rec, double *w, double *m, double *v, const double *g, const uint8_t *touched,
             double lr, double b1, double b2, double eps, int step) {
  double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
  for (int64_t l = 0; l < n_leaves; ++l) {
    if (!touched[l]) continue;
    for (int k = 0; k < rec; ++k) {
      int64_t i = l * rec + k;
      m[i] = b1 * m[i] + (1.0 - b1) * g[i];
      v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
      w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Public: storage quantisation                                             */
/* ------------------------------------------------------------------------ */

/* float -> bfloat16 -> float, round to nearest, ties to even. */
void or_round_bf16(const float *in, float *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u;
    memcpy(&u, &in[i], 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
      u |= 0x00400000u; /* keep NaN quiet */
    } else {
      uint32_t lsb = (u >> 16) & 1u;
      u += 0x7FFFu + lsb;
    }
    u &= 0xFFFF0000u;
    memcpy(&out[i], &u, 4);
  }
}

/* ------------------------------------------------------------------------ */
/* Public: FP8 E4M3 storage with per-leaf scales (storage ablation)         */
/* ------------------------------------------------------------------------ */

/* The E4M3 value nearest to x: 1 sign bit, 4 exponent bits with bias 7, 3
 * fraction bits, subnormals down to 2^-9, largest finite magnitude 448, no
 * infinities.  Ties go to the even code; magnitudes from 448 up saturate. */
static double e4m3_nearest(double x) {
  double a = fabs(x);
  if (a >= 448.0) return copysign(448.0, x);
  if (a == 0.0) return x;
  int e;
  frexp(a, &e);                 /* a in [2^(e-1), 2^e) */
  int binade = e - 1;
  if (binade < -6) binade = -6; /* subnormals are spaced like binade -6 */
  double spacing = ldexp(1.0, binade - 3);
  /* nearbyint rounds half to even in the default mode; an even multiple of
   * the spacing is an even code (the code's last bit is the multiple's) */
  return copysign(nearbyint(a / spacing) * spacing, x);
}

/* The smallest power of two s with max |w| <= 448 s over a group (1 for an
 * all-zero group), so that w / s fits E4M3 without saturating. */
static double fp8_group_scale(const float *w, int len) {
  double mx = 0.0;
  for (int i = 0; i < len; ++i)
    if (fabs((double)w[i]) > mx) mx = fabs((double)w[i]);
  if (mx == 0.0) return 1.0;
  int e;
  frexp(mx, &e);                /* mx >= 2^(e-1) > 448 * 2^(e-10) */
  int p = e - 10;
  while (ldexp(448.0, p) < mx) ++p;
  return ldexp(1.0, p);
}

/* Quantises n_groups groups of len float32 values each ([group][len]): every
 * group gets its own power-of-two scale s, each value becomes
 * s * e4m3_nearest(w / s).  Writes the dequantised values and the scales. */
void or_quantize_fp8(const float *in, int64_t n_groups, int len, double *out, double *scale) {
  for (int64_t g = 0; g < n_groups; ++g) {
    const float *w = in + g * len;
    double s = fp8_group_scale(w, len);
    scale[g] = s;
    for (int i = 0; i < len; ++i) out[g * len + i] = e4m3_nearest((double)w[i] / s) * s;
  }
}

/* The plain E4M3 rounding of each value (no scale), for the pins. */
void or_round_e4m3(const double *in, double *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = e4m3_nearest(in[i]);
}

/* ------------------------------------------------------------------------ */
/* Time slice: density and spherical-harmonic colour coefficients of every   */
/* leaf at one time (Sec. 7; the HH-colour figure's caption)                */
/* ------------------------------------------------------------------------ */

/* sigma: [n_leaves]; sh: [n_leaves][3][(degree+1)^2], index l^2 + l + m.  u is
   the frame coordinate t (T - 1).  For each leaf gamma = pi sigmoid(b(u) .
   w_gamma) is fixed, so sum_{n,l,m} w_nlm R_nl(gamma) Y_lm(d) regroups as
   sum_{l,m} (sum_{n >= l} w_nlm R_nl(gamma)) Y_lm(d). */
void or_slice(const or_tree *tr, double u, double *sigma, double *sh) {
  double *a = (double *)malloc(sizeof(double) * tr->K), *b = (double *)malloc(sizeof(double) * tr->K);
  basis_rows(tr, u, a, b);
  const int Nh = or_n_hh(tr->degree), NY = (tr->degree + 1) * (tr->degree + 1);
  for (int64_t leaf = 0; leaf < tr->n_leaves; ++leaf) {
    double ps = 0.0, pg = 0.0;
    for (int k = 0; k < tr->K; ++k) {
      ps += a[k] * coef(tr, tr->w_sigma, k, leaf);
      pg += b[k] * coef(tr, tr->w_gamma, k, leaf);
    }
    sigma[leaf] = ps > 0.0 ? ps : 0.0;
    const double gamma = M_PI * sigmoid(pg);
    for (int ch = 0; ch < 3; ++ch)
      for (int l = 0; l <= tr->degree; ++l)
        for (int m = -l; m <= l; ++m) {
          double acc = 0.0;
          for (int n = l; n <= tr->degree; ++n)
            acc += coef(tr, tr->w_hh, (int64_t)ch * Nh + or_hh_index(n, l, m), leaf) * or_hh_radial(n, l, gamma);
          sh[(leaf * 3 + ch) * NY + l * l + l + m] = acc;
        }
  }
  free(a);
  free(b);
}

/* Volume rendering of a slice (Eq. volume-rendering): the same voxels and
   chords as the tree's walk, density sigma[leaf], colour act(sum_lm s_lm Y_lm(d)). */
typedef struct {
  const or_tree *tr;
  const or_opts *op;
  const double *sigma, *sh;
  const double *o, *d;
  int64_t n;
  double *rgb, *alpha, *depth, *tau;
  int32_t *nseg;
} slice_ctx;

static void slice_range(void *p, int64_t lo, int64_t hi) {
  slice_ctx *c = (slice_ctx *)p;
  const or_tree *tr = c->tr;
  const int NY = (tr->degree + 1) * (tr->degree + 1);
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * max_segments(tr));
  double *Y = (double *)malloc(sizeof(double) * NY);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    unit(d, dn);
    for (int l = 0; l <= tr->degree; ++l)
      for (int m = -l; m <= l; ++m) Y[l * l + l + m] = or_sh_real(l, m, dn);
    int ns = or_trace(tr, o, dn, segs, max_segments(tr));
    double tau = 0.0, acc[3] = {0, 0, 0}, alpha = 0.0, dnum = 0.0;
    int composited = 0;
    for (int i = 0; i < ns; ++i) {
      const int64_t leaf = segs[i].leaf;
      const double sg = c->sigma[leaf];
      double col[3];
      for (int ch = 0; ch < 3; ++ch) {
        double z = 0.0;
        for (int k = 0; k < NY; ++k) z += c->sh[(leaf * 3 + ch) * NY + k] * Y[k];
        col[ch] = c->op->act == 0 ? sigmoid(z) : z;
      }
      double delta = segs[i].t1 - segs[i].t0;
      const double Ti = exp(-tau);                 /* transmittance in front of segment i */
      double w = Ti * (1.0 - exp(-sg * delta));
      for (int ch = 0; ch < 3; ++ch) acc[ch] += w * col[ch];
      alpha += w;
      dnum += 0.5 * w * (segs[i].t0 + segs[i].t1);
      tau += sg * delta;
      composited = i + 1;
      if (exp(-tau) < c->op->t_stop) break;
    }
    for (int ch = 0; ch < 3; ++ch) c->rgb[3 * r + ch] = acc[ch];
    c->alpha[r] = alpha;
    c->tau[r] = tau;
    c->depth[r] = alpha >= 1e-4 ? dnum / alpha : INFINITY;
    c->nseg[r] = composited;
  }
  free(segs);
  free(Y);
}

void or_render_slice(const or_tree *tr, const or_opts *op, const double *sigma, const double *sh, int64_t n,
                     const double *o, const double *d, double *rgb, double *alpha, double *depth, double *tau,
                     int32_t *nseg, int nthreads) {
  slice_ctx c = {tr, op, sigma, sh, o, d, n, rgb, alpha, depth, tau, nseg};
  parallel_for(n, nthreads, slice_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Appearance edits (Sec. 5 "Appearance editing")                           */
/* ------------------------------------------------------------------------ */

/* Terminating voxel of each ray: the leaf of the segment at which the
   accumulated alpha 1 - exp(-sum sigma delta) of the unedited render first
   reaches `threshold`; -1 when it never does. */
typedef struct {
  const or_tree *tr;
  const or_opts *op;
  const double *o, *d, *t;
  int64_t n;
  double threshold;
  int64_t *leaf;
} pick_ctx;

static void pick_range(void *p, int64_t lo, int64_t hi) {
  pick_ctx *c = (pick_ctx *)p;
  const or_tree *tr = c->tr;
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * max_segments(tr));
  double *H = (double *)malloc(sizeof(double) * or_n_hh(tr->degree));
  double *a = (double *)malloc(sizeof(double) * tr->K), *b = (double *)malloc(sizeof(double) * tr->K);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    double t = c->t[r] < 0.0 ? 0.0 : (c->t[r] > 1.0 ? 1.0 : c->t[r]);
    unit(d, dn);
    basis_rows(tr, t * (tr->T - 1), a, b);
    int ns = or_trace(tr, o, dn, segs, max_segments(tr));
    double optical = 0.0;
    c->leaf[r] = -1;
    for (int i = 0; i < ns; ++i) {
      or_leaf_eval e;
      eval_leaf(tr, c->op, segs[i].leaf, a, b, dn, H, NULL, &e);
      optical += e.sigma * (segs[i].t1 - segs[i].t0);
      if (1.0 - exp(-optical) >= c->threshold) {
        c->leaf[r] = segs[i].leaf;
        break;
      }
    }
  }
  free(segs); free(H); free(a); free(b);
}

void or_pick(const or_tree *tr, const or_opts *op, int64_t n, const double *o, const double *d, const double *t,
             double threshold, int64_t *leaf, int nthreads) {
  pick_ctx c = {tr, op, o, d, t, n, threshold, leaf};
  parallel_for(n, nthreads, pick_range, &c);
}

/* Rendering with edits.  edit [n_leaves][5] = target colour c_d (3), target
   density sigma_d, time t_d.  An edit is active at time t when t >= t_d; then
   sigma becomes sigma_d when sigma_d >= 0, and the colour becomes
   (1 - beta) c + beta c_d.  Otherwise Eq. volume-rendering as or_render. */
typedef struct {
  const or_tree *tr;
  const or_opts *op;
  const double *edit;
  double beta;
  const double *o, *d, *t;
  int64_t n;
  double *rgb, *alpha, *depth, *tau;
  int32_t *nseg;
} edit_ctx;

static void edit_range(void *p, int64_t lo, int64_t hi) {
  edit_ctx *c = (edit_ctx *)p;
  const or_tree *tr = c->tr;
  or_seg *segs = (or_seg *)malloc(sizeof(or_seg) * max_segments(tr));
  double *H = (double *)malloc(sizeof(double) * or_n_hh(tr->degree));
  double *a = (double *)malloc(sizeof(double) * tr->K), *b = (double *)malloc(sizeof(double) * tr->K);
  for (int64_t r = lo; r < hi; ++r) {
    double o[3] = {c->o[r], c->o[c->n + r], c->o[2 * c->n + r]};
    double d[3] = {c->d[r], c->d[c->n + r], c->d[2 * c->n + r]}, dn[3];
    double t = c->t[r] < 0.0 ? 0.0 : (c->t[r] > 1.0 ? 1.0 : c->t[r]);
    unit(d, dn);
    basis_rows(tr, t * (tr->T - 1), a, b);
    int ns = or_trace(tr, o, dn, segs, max_segments(tr));
    double optical = 0.0, col[3] = {0, 0, 0}, alpha = 0.0, dnum = 0.0;
    int composited = 0;
    for (int i = 0; i < ns; ++i) {
      or_leaf_eval e;
      eval_leaf(tr, c->op, segs[i].leaf, a, b, dn, H, NULL, &e);
      const double *E = c->edit + 5 * segs[i].leaf;
      if (t >= E[4]) {
        if (E[3] >= 0.0) e.sigma = E[3];
        for (int ch = 0; ch < 3; ++ch) e.c[ch] = (1.0 - c->beta) * e.c[ch] + c->beta * E[ch];
      }
      const double len = segs[i].t1 - segs[i].t0;
      const double Tin = exp(-optical);
      const double wi = Tin * (1.0 - exp(-e.sigma * len));
      for (int ch = 0; ch < 3; ++ch) col[ch] += wi * e.c[ch];
      alpha += wi;
      dnum += wi * (segs[i].t0 + 0.5 * len);
      optical += e.sigma * len;
      composited = i + 1;
      if (exp(-optical) < c->op->t_stop) break;
    }
    for (int ch = 0; ch < 3; ++ch) c->rgb[3 * r + ch] = col[ch];
    c->alpha[r] = alpha;
    c->tau[r] = optical;
    c->depth[r] = alpha >= 1e-4 ? dnum / alpha : INFINITY;
    c->nseg[r] = composited;
  }
  free(segs); free(H); free(a); free(b);
}

void or_render_edit(const or_tree *tr, const or_opts *op, const double *edit, double beta, int64_t n, const double *o,
                    const double *d, const double *t, double *rgb, double *alpha, double *depth, double *tau,
                    int32_t *nseg, int nthreads) {
  edit_ctx c = {tr, op, edit, beta, o, d, t, n, rgb, alpha, depth, tau, nseg};
  parallel_for(n, nthreads, edit_range, &c);
}
