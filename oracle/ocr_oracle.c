/* FP64 CPU oracle for the forest-of-octrees raycaster.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.  Parity of every function here is pinned by the
 * CPU test suite against closed forms, invariants and brute force (see
 * tests/test_oracle_pins.py); no function is "parity unpinned".
 *
 * Equation numbers follow the paper's sections (Sec. 2.x, Eq. 2.y).
 */
#include "ocr_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Segment algebra, Sec. 2.4-2.5.  A segment is (A, B_r, B_g, B_b).           */
/* ------------------------------------------------------------------------ */

/* Eq. 2.14: (A2, B2) (+) (A1, B1) = (A2 A1, B2 + A2 B1), 2 = nearer. */
void orc_combine(const double *n, const double *f, double *out) {
  double r[4];
  r[0] = n[0] * f[0];
  for (int c = 1; c < 4; ++c) r[c] = n[c] + n[0] * f[c];
  memcpy(out, r, sizeof r);
}

/* Eq. 2.15: inverse (1/A, -B/A). */
void orc_inverse(const double *s, double *out) {
  double r[4];
  r[0] = 1.0 / s[0];
  for (int c = 1; c < 4; ++c) r[c] = -s[c] / s[0];
  memcpy(out, r, sizeof r);
}

/* Eq. 2.20: the piece of relative length frac: A_i = A^frac,
 * B_i = B (1 - A_i) / (1 - A); for A = 1, B_i = B frac.  1 - A^f is formed
 * as -expm1(f ln A) so that A -> 1 loses no digits. */
void orc_cut(const double *s, double frac, double *out) {
  double r[4];
  double la = log(s[0]);
  r[0] = exp(frac * la);
  double ratio = (la == 0.0) ? frac : expm1(frac * la) / expm1(la);
  for (int c = 1; c < 4; ++c) r[c] = s[c] * ratio;
  memcpy(out, r, sizeof r);
}

/* Eq. 2.21: geometric mean of A, arithmetic mean of B. */
void orc_average(const double *s1, const double *s2, double *out) {
  double r[4];
  r[0] = sqrt(s1[0] * s2[0]);
  for (int c = 1; c < 4; ++c) r[c] = 0.5 * (s1[c] + s2[c]);
  memcpy(out, r, sizeof r);
}

/* ------------------------------------------------------------------------ */
/* Field and transfer function                                               */
/* ------------------------------------------------------------------------ */

/* Piecewise-linear interpolation between 8 knots spaced uniformly over
 * [s_min, s_max], constant outside. */
void orc_tf_eval(const orc_forest *F, double s, double *kq) {
  double z = (s - F->s_min) / (F->s_max - F->s_min) * 7.0;
  if (z < 0.0) z = 0.0;
  if (z > 7.0) z = 7.0;
  int k = (int)floor(z);
  if (k > 6) k = 6;
  double w = z - k;
  for (int c = 0; c < 4; ++c)
    kq[c] = (1.0 - w) * (double)F->tf[4 * k + c] + w * (double)F->tf[4 * (k + 1) + c];
}

/* Trilinear Lagrange interpolation of the 8 corner values. */
double orc_trilinear(const float *nd, double u, double v, double w) {
  double s = 0.0;
  for (int c = 0; c < 8; ++c) {
    double wx = (c & 1) ? u : 1.0 - u;
    double wy = (c & 2) ? v : 1.0 - v;
    double wz = (c & 4) ? w : 1.0 - w;
    s += (double)nd[c] * wx * wy * wz;
  }
  return s;
}

/* The leaf's box in the reference coordinates of its tree (for the cube, the
 * identity map, in space). */
static void leaf_box(const orc_forest *F, int leaf, double *lo, double *h) {
  double scale = ldexp(1.0, -F->max_level);
  *h = ldexp(1.0, -(int)F->level[leaf]);
  for (int a = 0; a < 3; ++a) lo[a] = F->anchor[3 * leaf + a] * scale;
}

static int nodal_stride(const orc_forest *F) { return F->geometry == 1 ? 27 : 8; }

/* Degree-2 Lagrange basis on {0, 1/2, 1} at t. */
static void quad_basis(double t, double *l) {
  l[0] = 2.0 * (t - 0.5) * (t - 1.0);
  l[1] = -4.0 * t * (t - 1.0);
  l[2] = 2.0 * t * (t - 0.5);
}

double orc_triquadratic(const float *nd, double u, double v, double w) {
  double lu[3], lv[3], lw[3], s = 0.0;
  quad_basis(u, lu);
  quad_basis(v, lv);
  quad_basis(w, lw);
  for (int c = 0; c < 27; ++c) s += (double)nd[c] * lu[c % 3] * lv[(c / 3) % 3] * lw[c / 9];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Cubed-sphere shell: the equiangular map (the paper's tree-to-space map of  */
/* Sec. 2.1 taken as the six-tree cubed sphere)                               */
/* ------------------------------------------------------------------------ */

static const double ORC_PI = 3.14159265358979323846;

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* tan(pi/4 (2 xi - 1)): the tangent-plane coordinate of reference xi */
static double eq_tan(double xi) { return tan(0.25 * ORC_PI * (2.0 * xi - 1.0)); }

static double shell_radius(const orc_forest *F, double zeta) {
  return F->r0 + (F->r1 - F->r0) * zeta;
}

/* unit direction of reference (xi, eta) in tree k */
static void shell_dir(const orc_forest *F, int k, double xi, double eta, double *d) {
  double a = eq_tan(xi), b = eq_tan(eta);
  for (int c = 0; c < 3; ++c) d[c] = F->frames[k][0][c] + a * F->frames[k][1][c] + b * F->frames[k][2][c];
  double nn = sqrt(dot3(d, d));
  for (int c = 0; c < 3; ++c) d[c] /= nn;
}

void orc_shell_map(const orc_forest *F, int tree, const double *ref, double *x) {
  double d[3], r = shell_radius(F, ref[2]);
  shell_dir(F, tree, ref[0], ref[1], d);
  for (int c = 0; c < 3; ++c) x[c] = r * d[c];
}

/* xi = atan(x.e1 / x.n) 2/pi + 1/2, eta likewise with e2, zeta from |x| */
void orc_shell_inverse(const orc_forest *F, int tree, const double *x, double *ref) {
  double pn = dot3(x, F->frames[tree][0]);
  ref[0] = atan2(dot3(x, F->frames[tree][1]), pn) * 2.0 / ORC_PI + 0.5;
  ref[1] = atan2(dot3(x, F->frames[tree][2]), pn) * 2.0 / ORC_PI + 0.5;
  ref[2] = (sqrt(dot3(x, x)) - F->r0) / (F->r1 - F->r0);
}

/* The 8 mapped corners of a leaf and a distance delta such that every point
 * of the leaf lies within delta of their convex hull.  Cube: delta = 0.
 * Shell: a point r d of the leaf has d = p / |p| with p a convex combination
 * of the 4 unit corner directions d_i, and r p lies in the hull of the 8
 * corners; |r d - r p| = r (1 - |p|) <= r_out (1 - min_i d_i . c) for any
 * unit c, here c = normalize(sum_i d_i). */
static void leaf_corners(const orc_forest *F, int leaf, double x[8][3], double *delta) {
  double lo[3], h;
  leaf_box(F, leaf, lo, &h);
  *delta = 0.0;
  if (F->geometry != 1) {
    for (int c = 0; c < 8; ++c) {
      x[c][0] = lo[0] + ((c & 1) ? h : 0.0);
      x[c][1] = lo[1] + ((c & 2) ? h : 0.0);
      x[c][2] = lo[2] + ((c & 4) ? h : 0.0);
    }
    return;
  }
  int k = F->tree[leaf];
  double d[4][3], csum[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 4; ++c) {
    shell_dir(F, k, lo[0] + ((c & 1) ? h : 0.0), lo[1] + ((c & 2) ? h : 0.0), d[c]);
    for (int a = 0; a < 3; ++a) csum[a] += d[c][a];
  }
  double cn = sqrt(dot3(csum, csum)), cmin = 1.0;
  for (int c = 0; c < 4; ++c) {
    double cc = dot3(d[c], csum) / cn;
    if (cc < cmin) cmin = cc;
  }
  double rin = shell_radius(F, lo[2]), rout = shell_radius(F, lo[2] + h);
  for (int c = 0; c < 8; ++c) {
    double r = (c & 4) ? rout : rin;
    for (int a = 0; a < 3; ++a) x[c][a] = r * d[c & 3][a];
  }
  *delta = rout * (1.0 - cmin);
}

/* ------------------------------------------------------------------------ */
/* Camera, Sec. 2.2                                                          */
/* ------------------------------------------------------------------------ */

/* Eq. 2.5: r = v + ell ((i - (w-1)/2) t + (j - (h-1)/2) u), rays o + alpha r,
 * alpha in [1, f/n] (the near plane is the projection plane).  The
 * orthographic variant moves the origin by the same offset and uses the
 * direction v/n, alpha >= 0. */
void orc_pixel_ray(const orc_camera *C, int i, int j, double *org, double *dir, double *amin,
                   double *amax) {
  double di = i - 0.5 * (C->w - 1), dj = j - 0.5 * (C->h - 1);
  if (C->ortho) {
    for (int a = 0; a < 3; ++a) {
      org[a] = C->o[a] + C->ell * (di * C->t[a] + dj * C->u[a]);
      dir[a] = C->v[a] / C->near_;
    }
    *amin = 0.0;
    *amax = C->far_;
  } else {
    for (int a = 0; a < 3; ++a) {
      org[a] = C->o[a];
      dir[a] = C->v[a] + C->ell * (di * C->t[a] + dj * C->u[a]);
    }
    *amin = 1.0;
    *amax = C->far_ / C->near_;
  }
}

/* Eq. 2.6: X = (t, u, v/n)^T (x - o). */
static void camera_transform(const orc_camera *C, const double *x, double *X) {
  double d[3] = {x[0] - C->o[0], x[1] - C->o[1], x[2] - C->o[2]};
  X[0] = C->t[0] * d[0] + C->t[1] * d[1] + C->t[2] * d[2];
  X[1] = C->u[0] * d[0] + C->u[1] * d[1] + C->u[2] * d[2];
  X[2] = (C->v[0] * d[0] + C->v[1] * d[1] + C->v[2] * d[2]) / C->near_;
}

static int axis_visible(double pmin, double pmax, int lim) {
  double lo = ceil(pmin), hi = floor(pmax);
  if (lo < 0.0) lo = 0.0;
  if (hi > lim) hi = lim;
  return lo <= hi;
}

/* Sec. 2.2 / App. A.2: the camera-space AABB is the min/max of the 8
 * transformed corners; it is clipped to the visible depth range and the
 * corners of the clipped brick are projected into the image plane; the
 * rectangle holds the pixel centres inside that projection.  pext receives
 * the projected extents {i_min, i_max, j_min, j_max} in pixel units (may be
 * NULL).  *vis_unc is set when moving any threshold by band_px pixels (or the
 * depth clip by band_px relative) would change the rectangle or the
 * visibility decision. */
int orc_leaf_rect(const orc_forest *F, const orc_camera *C, int leaf, int32_t *rect,
                  double *pext, double band_px, int *vis_unc) {
  double xc[8][3], delta;
  leaf_corners(F, leaf, xc, &delta);
  double bmin[3] = {INFINITY, INFINITY, INFINITY}, bmax[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int c = 0; c < 8; ++c) {
    double X[3];
    camera_transform(C, xc[c], X);
    for (int a = 0; a < 3; ++a) {
      if (X[a] < bmin[a]) bmin[a] = X[a];
      if (X[a] > bmax[a]) bmax[a] = X[a];
    }
  }
  if (delta > 0.0) { /* widen by delta along each camera axis (t, u, v / n) */
    double ext[3] = {delta * sqrt(dot3(C->t, C->t)), delta * sqrt(dot3(C->u, C->u)),
                     delta * sqrt(dot3(C->v, C->v)) / C->near_};
    for (int a = 0; a < 3; ++a) {
      bmin[a] -= ext[a];
      bmax[a] += ext[a];
    }
  }
  double zlo_lim = C->ortho ? 0.0 : C->near_;
  double zlo = bmin[2] > zlo_lim ? bmin[2] : zlo_lim;
  double zhi = bmax[2] < C->far_ ? bmax[2] : C->far_;
  int unc = 0;
  rect[0] = 0; rect[1] = -1; rect[2] = 0; rect[3] = -1;
  if (pext) { pext[0] = pext[2] = INFINITY; pext[1] = pext[3] = -INFINITY; }
  if (fabs(zhi - zlo) <= band_px * 1e-3 * (fabs(zhi) + fabs(zlo))) unc = 1;
  if (!(zlo <= zhi)) {
    if (vis_unc) *vis_unc = unc;
    return 0;
  }
  /* project the 8 corners of the depth-clipped brick to pixel coordinates */
  double pmin[2] = {INFINITY, INFINITY}, pmax[2] = {-INFINITY, -INFINITY};
  for (int c = 0; c < 8; ++c) {
    double X[3] = {(c & 1) ? bmax[0] : bmin[0], (c & 2) ? bmax[1] : bmin[1], (c & 4) ? zhi : zlo};
    for (int a = 0; a < 2; ++a) {
      double plane = C->ortho ? X[a] : X[a] * C->near_ / X[2];
      double p = plane / C->ell + 0.5 * ((a == 0 ? C->w : C->h) - 1);
      if (p < pmin[a]) pmin[a] = p;
      if (p > pmax[a]) pmax[a] = p;
    }
  }
  int lim[2] = {C->w - 1, C->h - 1};
  int vis = 1, vis_in = 1, vis_out = 1;
  for (int a = 0; a < 2; ++a) {
    vis = vis && axis_visible(pmin[a], pmax[a], lim[a]);
    vis_in = vis_in && axis_visible(pmin[a] + band_px, pmax[a] - band_px, lim[a]);
    vis_out = vis_out && axis_visible(pmin[a] - band_px, pmax[a] + band_px, lim[a]);
  }
  if (vis_in != vis_out) unc = 1;
  for (int a = 0; a < 2; ++a) { /* an edge of the rectangle itself is a near tie */
    if (pmin[a] > -1.0 && pmin[a] < lim[a] + 1.0 && fabs(pmin[a] - nearbyint(pmin[a])) < band_px)
      unc = 1;
    if (pmax[a] > -1.0 && pmax[a] < lim[a] + 1.0 && fabs(pmax[a] - nearbyint(pmax[a])) < band_px)
      unc = 1;
  }
  if (vis_unc) *vis_unc = unc;
  if (pext) { pext[0] = pmin[0]; pext[1] = pmax[0]; pext[2] = pmin[1]; pext[3] = pmax[1]; }
  if (!vis) return 0;
  for (int a = 0; a < 2; ++a) {
    double lo_f = ceil(pmin[a]), hi_f = floor(pmax[a]);
    if (lo_f < 0.0) lo_f = 0.0;
    if (hi_f > lim[a]) hi_f = lim[a];
    rect[2 * a] = (int32_t)lo_f;
    rect[2 * a + 1] = (int32_t)hi_f;
  }
  return 1;
}

/* Slab test: the ray's parameter interval inside the axis-aligned leaf box. */
static int ray_cube_leaf(const orc_forest *F, int leaf, const double *org, const double *dir,
                         double amin, double amax, double *a_in, double *a_out, double band_rel,
                         int *tie) {
  double lo[3], h;
  leaf_box(F, leaf, lo, &h);
  double t0 = amin, t1 = amax;
  for (int a = 0; a < 3; ++a) {
    double b0 = lo[a], b1 = lo[a] + h;
    if (dir[a] == 0.0) {
      /* parallel to the slab: a tie when the ray runs within the band of a face */
      double sc = fabs(org[a]) > 1.0 ? fabs(org[a]) : 1.0;
      if (tie && (fabs(org[a] - b0) <= band_rel * sc || fabs(org[a] - b1) <= band_rel * sc))
        *tie = 1;
      if (org[a] < b0 || org[a] > b1) { /* parallel to the slab and outside it */
        a_in[0] = INFINITY;
        a_out[0] = -INFINITY;
        return 0;
      }
      continue;
    }
    double s0 = (b0 - org[a]) / dir[a], s1 = (b1 - org[a]) / dir[a];
    if (s0 > s1) { double tmp = s0; s0 = s1; s1 = tmp; }
    if (s0 > t0) t0 = s0;
    if (s1 < t1) t1 = s1;
  }
  a_in[0] = t0;
  a_out[0] = t1;
  if (tie && isfinite(t0) && isfinite(t1)) {
    double scale = fabs(t1) > fabs(t0) ? fabs(t1) : fabs(t0);
    if (fabs(t1 - t0) <= band_rel * scale) *tie = 1;
  }
  return t1 > t0;
}

/* Shell leaf: its angular extent is the cone of the four half-spaces
 * x . (e1 - tan0 n) >= 0, x . (tan1 n - e1) >= 0 (and the same with e2), whose
 * boundary planes pass through the origin; its radial extent is the shell
 * R_in <= |x| <= R_out.  The ray meets the cone in one interval, the outer
 * ball in one interval, and leaves out the inner ball's interval: at most two
 * pieces.  The sphere crossings are alpha = -b +- sqrt((R^2 - |p|^2) / |r|^2)
 * with b = (o . r) / |r|^2 and p = o - b r the ray's point nearest the centre. */
static int ray_shell_leaf(const orc_forest *F, int leaf, const double *org, const double *dir,
                          double amin, double amax, double *a_in, double *a_out, double band_rel,
                          int *tie) {
  double lo[3], h;
  leaf_box(F, leaf, lo, &h);
  const double(*fr)[3] = F->frames[F->tree[leaf]];
  double t0 = amin, t1 = amax;
  for (int s = 0; s < 4; ++s) {
    const double *e = fr[1 + s / 2];
    double tn = eq_tan(lo[s / 2] + ((s & 1) ? h : 0.0)), sg = (s & 1) ? -1.0 : 1.0, m[3];
    for (int c = 0; c < 3; ++c) m[c] = sg * (e[c] - tn * fr[0][c]);
    double g0 = dot3(org, m), g1 = dot3(dir, m);
    if (g1 == 0.0) { /* parallel to the plane: a tie when it runs within the band of it */
      if (tie && fabs(g0) <= band_rel * sqrt(dot3(org, org) * dot3(m, m))) *tie = 1;
      if (g0 < 0.0) return 0;
      continue;
    }
    double a = -g0 / g1;
    if (g1 > 0.0) {
      if (a > t0) t0 = a;
    } else if (a < t1) {
      t1 = a;
    }
  }
  double rr = dot3(dir, dir), b = dot3(org, dir) / rr, p[3];
  for (int c = 0; c < 3; ++c) p[c] = org[c] - b * dir[c];
  double pp = dot3(p, p);
  double rin = shell_radius(F, lo[2]), rout = shell_radius(F, lo[2] + h);
  double hout = rout * rout - pp, hin = rin * rin - pp;
  if (tie && (fabs(hout) <= band_rel * rout * rout || fabs(hin) <= band_rel * rin * rin)) *tie = 1;
  if (!(hout > 0.0)) return 0;
  double so = sqrt(hout / rr);
  if (-b - so > t0) t0 = -b - so;
  if (-b + so < t1) t1 = -b + so;
  double lo_p[2] = {t0, t0}, hi_p[2] = {t1, t1};
  int npieces = 1;
  if (hin > 0.0) {
    double si = sqrt(hin / rr);
    if (-b - si < hi_p[0]) hi_p[0] = -b - si;
    if (-b + si > lo_p[1]) lo_p[1] = -b + si;
    npieces = 2;
  }
  int n = 0;
  for (int k = 0; k < npieces; ++k) {
    if (tie && isfinite(lo_p[k]) && isfinite(hi_p[k])) {
      double scale = fabs(hi_p[k]) > fabs(lo_p[k]) ? fabs(hi_p[k]) : fabs(lo_p[k]);
      if (fabs(hi_p[k] - lo_p[k]) <= band_rel * scale) *tie = 1;
    }
    if (hi_p[k] > lo_p[k]) {
      a_in[n] = lo_p[k];
      a_out[n] = hi_p[k];
      ++n;
    }
  }
  return n;
}

int orc_ray_leaf_tie(const orc_forest *F, int leaf, const double *org, const double *dir,
                     double amin, double amax, double *a_in, double *a_out, double band_rel,
                     int *tie) {
  if (F->geometry == 1) return ray_shell_leaf(F, leaf, org, dir, amin, amax, a_in, a_out, band_rel, tie);
  return ray_cube_leaf(F, leaf, org, dir, amin, amax, a_in, a_out, band_rel, tie);
}

int orc_ray_leaf(const orc_forest *F, int leaf, const double *org, const double *dir, double amin,
                 double amax, double *a_in, double *a_out) {
  return orc_ray_leaf_tie(F, leaf, org, dir, amin, amax, a_in, a_out, 0.0, NULL);
}

/* ------------------------------------------------------------------------ */
/* Index decisions in FP32                                                   */
/* ------------------------------------------------------------------------ */
/* Which leaves a camera sees, which (leaf, ray) pairs give segments and where
 * a segment ends are thresholds decided by floating point.  The oracle takes
 * these decisions in FP32, the precision of the GPU path, by one canonical
 * evaluation of the formulas above: the camera constants of Eq. 2.5 rounded
 * once from FP64 to FP32 (step a1 of the path), then every operation rounded
 * to nearest once, in the order written here, a fused multiply-add only where
 * fma32 is written, subnormal operands and results flushed to signed zero
 * (the GPU runs with flush-to-zero).  The mathematics is that of
 * orc_pixel_ray, orc_leaf_rect and orc_ray_leaf; only the precision and the
 * fixed order differ.  The segment values are still integrated in FP64, over
 * the FP32 ray and end points. */

static float fz(float x) { return fabsf(x) < FLT_MIN ? copysignf(0.0f, x) : x; }
static float add32(float a, float b) { return fz(fz(a) + fz(b)); }
static float sub32(float a, float b) { return fz(fz(a) - fz(b)); }
static float mul32(float a, float b) { return fz(fz(a) * fz(b)); }
static float div32(float a, float b) { return fz(fz(a) / fz(b)); }
static float fma32(float a, float b, float c) { return fz(fmaf(fz(a), fz(b), fz(c))); }
static float sqrt32(float a) { return fz(sqrtf(fz(a))); }
static float min32(float a, float b) { return fminf(fz(a), fz(b)); }
static float max32(float a, float b) { return fmaxf(fz(a), fz(b)); }

void orc_camera32(const orc_camera *C, orc_cam32 *K) {
  for (int a = 0; a < 3; ++a) {
    K->o[a] = (float)C->o[a];
    K->v[a] = (float)(C->ortho ? C->v[a] / C->near_ : C->v[a]);
    K->lt[a] = (float)(C->ell * C->t[a]);
    K->lu[a] = (float)(C->ell * C->u[a]);
    K->t[a] = (float)C->t[a];
    K->u[a] = (float)C->u[a];
    K->vn[a] = (float)(C->v[a] / C->near_);
  }
  K->n = (float)C->near_;
  K->f = (float)C->far_;
  K->ell = (float)C->ell;
  K->cw = 0.5f * (float)(C->w - 1);
  K->ch = 0.5f * (float)(C->h - 1);
  K->amin = C->ortho ? 0.0f : 1.0f;
  K->amax = (float)(C->ortho ? C->far_ : C->far_ / C->near_);
  K->w = C->w;
  K->h = C->h;
  K->ortho = C->ortho;
}

/* Eq. 2.5 in FP32: offset ell ((i - cw) t + (j - ch) u) with ell t, ell u
 * rounded once; perspective: origin o, direction v + offset; orthographic:
 * origin o + offset, direction v/n. */
void orc_pixel_ray32(const orc_cam32 *K, int i, int j, float *org, float *dir) {
  float di = sub32((float)i, K->cw), dj = sub32((float)j, K->ch);
  for (int a = 0; a < 3; ++a) {
    float off = fma32(dj, K->lu[a], mul32(di, K->lt[a]));
    if (K->ortho) {
      org[a] = add32(K->o[a], off);
      dir[a] = K->v[a];
    } else {
      org[a] = K->o[a];
      dir[a] = add32(K->v[a], off);
    }
  }
}

/* Sec. 2.2: project the camera-space box [blo, bhi] clipped to the visible
 * depth range; the rectangle of the pixel centres inside (closed), clipped to
 * the image.  Returns 1 if it is not empty. */
static int project_box32(const orc_cam32 *K, const float *blo, const float *bhi, int32_t *rect) {
  rect[0] = 0; rect[1] = -1; rect[2] = 0; rect[3] = -1;
  float zlo = max32(blo[2], K->ortho ? 0.0f : K->n), zhi = min32(bhi[2], K->f);
  if (!(zlo <= zhi)) return 0;
  float pmin[2], pmax[2];
  for (int a = 0; a < 2; ++a) {
    float x0 = blo[a], x1 = bhi[a], lo_p, hi_p;
    if (K->ortho) {
      lo_p = div32(x0, K->ell);
      hi_p = div32(x1, K->ell);
    } else {
      /* the projection x n / (z ell) at the box's nearest and farthest depth */
      float sl = div32(K->n, mul32(zlo, K->ell)), sh = div32(K->n, mul32(zhi, K->ell));
      float p00 = mul32(x0, sl), p01 = mul32(x0, sh), p10 = mul32(x1, sl), p11 = mul32(x1, sh);
      lo_p = min32(min32(p00, p01), min32(p10, p11));
      hi_p = max32(max32(p00, p01), max32(p10, p11));
    }
    float cen = a == 0 ? K->cw : K->ch;
    pmin[a] = add32(lo_p, cen);
    pmax[a] = add32(hi_p, cen);
  }
  float i0 = fmaxf(ceilf(pmin[0]), 0.0f), i1 = fminf(floorf(pmax[0]), (float)(K->w - 1));
  float j0 = fmaxf(ceilf(pmin[1]), 0.0f), j1 = fminf(floorf(pmax[1]), (float)(K->h - 1));
  if (!(i0 <= i1 && j0 <= j1)) return 0;
  rect[0] = (int32_t)i0; rect[1] = (int32_t)i1; rect[2] = (int32_t)j0; rect[3] = (int32_t)j1;
  return 1;
}

/* The shell's plane and radius tables in FP32: tan(pi/4 (2 k 2^-L - 1)) (odd
 * about the tree centre, exactly -+1 at its edges) and r0 + (r1 - r0) k 2^-L,
 * k = 0 .. 2^L, each rounded once from FP64.  tan and rad hold 2^L + 1 floats. */
void orc_shell_tables32(const orc_forest *F, float *tan_t, float *rad_t) {
  int L = F->max_level, n = (1 << L) + 1;
  for (int k = 0; k < n; ++k) {
    double x = ldexp(2.0 * k, -L) - 1.0, ax = fabs(x);
    double v = ax == 1.0 ? 1.0 : tan(0.25 * ORC_PI * ax);
    tan_t[k] = (float)(x < 0.0 ? -v : v);
    rad_t[k] = (float)(F->r0 + (F->r1 - F->r0) * ldexp((double)k, -L));
  }
}

/* One shell leaf in FP32: its frame, the tangents of its four planes (xi low,
 * xi high, eta low, eta high) and its radii. */
typedef struct {
  float n[3], e1[3], e2[3], T[4], rin, rout;
} leaf32;

static void shell_leaf32(const orc_forest *F, const float *tan_t, const float *rad_t, int leaf,
                         leaf32 *q) {
  int L = F->max_level, sz = 1 << (L - F->level[leaf]);
  const int32_t *a = F->anchor + 3 * (size_t)leaf;
  const double(*fr)[3] = F->frames[F->tree[leaf]];
  for (int c = 0; c < 3; ++c) {
    q->n[c] = (float)fr[0][c];
    q->e1[c] = (float)fr[1][c];
    q->e2[c] = (float)fr[2][c];
  }
  q->T[0] = tan_t[a[0]];
  q->T[1] = tan_t[a[0] + sz];
  q->T[2] = tan_t[a[1]];
  q->T[3] = tan_t[a[1] + sz];
  q->rin = rad_t[a[2]];
  q->rout = rad_t[a[2] + sz];
}

/* Sec. 2.2 in FP32, cube: the box [lo, lo + h]^3 mapped by Eq. 2.6 (an affine
 * map: centre +- half-extent |R| h/2 per camera axis); shell: the 8 mapped
 * corners' box widened by delta = r_out (1 - min_i d_i . c) (the bound of
 * leaf_corners) times |t|, |u|, |v|/n.  Then project_box32. */
int orc_leaf_rect32(const orc_forest *F, const orc_cam32 *K, const float *tan_t,
                    const float *rad_t, int leaf, int32_t *rect) {
  const float *rows[3] = {K->t, K->u, K->vn};
  float blo[3], bhi[3];
  if (F->geometry != 1) {
    float scale = ldexpf(1.0f, -F->max_level), h = ldexpf(1.0f, -(int)F->level[leaf]);
    float hh = mul32(0.5f, h), cc[3];
    for (int a = 0; a < 3; ++a)
      cc[a] = sub32(add32((float)F->anchor[3 * (size_t)leaf + a] * scale, hh), K->o[a]);
    for (int r = 0; r < 3; ++r) {
      const float *R = rows[r];
      float X = fma32(R[0], cc[0], fma32(R[1], cc[1], mul32(R[2], cc[2])));
      float E = mul32(hh, add32(add32(fabsf(R[0]), fabsf(R[1])), fabsf(R[2])));
      blo[r] = sub32(X, E);
      bhi[r] = add32(X, E);
    }
    return project_box32(K, blo, bhi, rect);
  }
  leaf32 q;
  shell_leaf32(F, tan_t, rad_t, leaf, &q);
  float len[3];
  for (int r = 0; r < 3; ++r) {
    const float *R = rows[r];
    len[r] = sqrt32(fma32(R[2], R[2], fma32(R[1], R[1], mul32(R[0], R[0]))));
  }
  float d[4][3], cs[3] = {0.0f, 0.0f, 0.0f};
  for (int c = 0; c < 4; ++c) {
    float ta = (c & 1) ? q.T[1] : q.T[0], tb = (c & 2) ? q.T[3] : q.T[2];
    for (int a = 0; a < 3; ++a) d[c][a] = fma32(tb, q.e2[a], fma32(ta, q.e1[a], q.n[a]));
    float nn = fma32(d[c][2], d[c][2], fma32(d[c][1], d[c][1], mul32(d[c][0], d[c][0])));
    float inv = div32(1.0f, sqrt32(nn));
    for (int a = 0; a < 3; ++a) {
      d[c][a] = mul32(d[c][a], inv);
      cs[a] = add32(cs[a], d[c][a]);
    }
  }
  float csn = div32(1.0f, sqrt32(fma32(cs[2], cs[2], fma32(cs[1], cs[1], mul32(cs[0], cs[0])))));
  float cmin = 1.0f;
  for (int c = 0; c < 4; ++c)
    cmin = min32(cmin, mul32(fma32(d[c][2], cs[2], fma32(d[c][1], cs[1], mul32(d[c][0], cs[0]))),
                             csn));
  float delta = mul32(q.rout, sub32(1.0f, cmin));
  for (int r = 0; r < 3; ++r) {
    blo[r] = INFINITY;
    bhi[r] = -INFINITY;
  }
  for (int c = 0; c < 8; ++c) {
    float rad = (c & 4) ? q.rout : q.rin, x[3];
    for (int a = 0; a < 3; ++a) x[a] = fma32(rad, d[c & 3][a], -K->o[a]);
    for (int r = 0; r < 3; ++r) {
      const float *R = rows[r];
      float X = fma32(R[0], x[0], fma32(R[1], x[1], mul32(R[2], x[2])));
      blo[r] = min32(blo[r], X);
      bhi[r] = max32(bhi[r], X);
    }
  }
  for (int r = 0; r < 3; ++r) {
    float ext = mul32(delta, len[r]);
    blo[r] = sub32(blo[r], ext);
    bhi[r] = add32(bhi[r], ext);
  }
  return project_box32(K, blo, bhi, rect);
}

/* Ray / leaf intersection in FP32, clipped to [amin, amax]: the slab test for
 * the cube (1/d rounded once, 0 for d = 0); for the shell the four half-spaces
 * of ray_shell_leaf, each crossing -(o . m) / (r . m) with m = e - T n, and the
 * spheres at -b -+ sqrt((R^2 - |p|^2) / |r|^2), b = (o . r) / |r|^2,
 * p = o - b r.  Returns the number of intervals (0..2), nearest first. */
int orc_ray_leaf32(const orc_forest *F, const float *tan_t, const float *rad_t, int leaf,
                   const float *org, const float *dir, float amin, float amax, float *a_in,
                   float *a_out) {
  float t0 = amin, t1 = amax;
  if (F->geometry != 1) {
    float scale = ldexpf(1.0f, -F->max_level), h = ldexpf(1.0f, -(int)F->level[leaf]);
    for (int a = 0; a < 3; ++a) {
      float b0 = (float)F->anchor[3 * (size_t)leaf + a] * scale, b1 = add32(b0, h);
      if (dir[a] == 0.0f) {
        if (org[a] < b0 || org[a] > b1) return 0;
        continue;
      }
      float iv = div32(1.0f, dir[a]);
      float s0 = mul32(sub32(b0, org[a]), iv), s1 = mul32(sub32(b1, org[a]), iv);
      t0 = max32(t0, min32(s0, s1));
      t1 = min32(t1, max32(s0, s1));
    }
    if (!(t1 > t0)) return 0;
    a_in[0] = t0;
    a_out[0] = t1;
    return 1;
  }
  leaf32 q;
  shell_leaf32(F, tan_t, rad_t, leaf, &q);
  for (int s = 0; s < 4; ++s) {
    const float *e = s < 2 ? q.e1 : q.e2;
    float m[3];
    for (int c = 0; c < 3; ++c) m[c] = fma32(-q.T[s], q.n[c], e[c]);
    float g0 = fma32(m[0], org[0], fma32(m[1], org[1], mul32(m[2], org[2])));
    float g1 = fma32(m[0], dir[0], fma32(m[1], dir[1], mul32(m[2], dir[2])));
    int upper = s & 1; /* the cone is x . m >= 0 for the lower planes, <= 0 for the upper */
    if (g1 == 0.0f) {
      if ((upper ? -g0 : g0) < 0.0f) return 0;
      continue;
    }
    float a = div32(-g0, g1);
    if ((upper ? -g1 : g1) > 0.0f)
      t0 = max32(t0, a);
    else
      t1 = min32(t1, a);
  }
  float rr = fma32(dir[0], dir[0], fma32(dir[1], dir[1], mul32(dir[2], dir[2])));
  float b = div32(fma32(org[0], dir[0], fma32(org[1], dir[1], mul32(org[2], dir[2]))), rr);
  float p[3];
  for (int c = 0; c < 3; ++c) p[c] = fma32(-b, dir[c], org[c]);
  float pp = fma32(p[0], p[0], fma32(p[1], p[1], mul32(p[2], p[2])));
  float hout = fma32(q.rout, q.rout, -pp);
  if (!(hout > 0.0f)) return 0;
  float so = sqrt32(div32(hout, rr));
  t0 = max32(t0, sub32(-b, so));
  t1 = min32(t1, add32(-b, so));
  float hin = fma32(q.rin, q.rin, -pp);
  int n = 0;
  if (hin > 0.0f) { /* the inner ball's chord is cut out */
    float si = sqrt32(div32(hin, rr));
    float c0 = min32(t1, sub32(-b, si)), c1 = max32(t0, add32(-b, si));
    if (c0 > t0) { a_in[n] = t0; a_out[n] = c0; ++n; }
    if (t1 > c1) { a_in[n] = c1; a_out[n] = t1; ++n; }
  } else if (t1 > t0) {
    a_in[0] = t0;
    a_out[0] = t1;
    n = 1;
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Segment values, Sec. 2.3 and 2.7                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_forest *F;
  const float *nodal;
  int tree;
  double lo[3], h;
  double org[3], dir[3];
  double a_out, rlen; /* x runs from the far end: alpha(x) = a_out - x / |r| */
} seg_ctx;

/* Local coordinates in [0, 1]^3 of the leaf at distance x from the far end of
 * the segment (the shell goes through the inverse map). */
static void local_coords(const seg_ctx *S, double x, double *u) {
  double alpha = S->a_out - x / S->rlen, p[3];
  for (int a = 0; a < 3; ++a) p[a] = S->org[a] + alpha * S->dir[a];
  if (S->F->geometry == 1) {
    double ref[3];
    orc_shell_inverse(S->F, S->tree, p, ref);
    memcpy(p, ref, sizeof ref);
  }
  for (int a = 0; a < 3; ++a) u[a] = (p[a] - S->lo[a]) / S->h;
}

static double field_at(const seg_ctx *S, const double *u) {
  if (S->F->geometry == 1) return orc_triquadratic(S->nodal, u[0], u[1], u[2]);
  return orc_trilinear(S->nodal, u[0], u[1], u[2]);
}

/* kappa and q at distance x from the far end of the segment. */
static void medium_at(const seg_ctx *S, double x, double *kq) {
  double u[3];
  local_coords(S, x, u);
  orc_tf_eval(S->F, field_at(S, u), kq);
}

static void seg_init(seg_ctx *S, const orc_forest *F, int leaf, const double *org,
                     const double *dir, double a_out) {
  S->F = F;
  S->nodal = F->nodal + (size_t)nodal_stride(F) * (size_t)leaf;
  S->tree = F->geometry == 1 ? F->tree[leaf] : 0;
  leaf_box(F, leaf, S->lo, &S->h);
  memcpy(S->org, org, sizeof S->org);
  memcpy(S->dir, dir, sizeof S->dir);
  S->a_out = a_out;
  S->rlen = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
}

/* f(x, Y) = (-kappa A, q - kappa B) of Eq. 2.29 */
#define RHS(kq, Y, K) do { (K)[0] = -(kq)[0] * (Y)[0]; \
      for (int c = 1; c < 4; ++c) (K)[c] = (kq)[c] - (kq)[0] * (Y)[c]; } while (0)

/* Classical RK4 on A' = -kappa A, B' = q - kappa B (Eq. 2.29), x from the far
 * end: one step of length hs from x0, from the state y0 (NULL: from (1, 0)). */
static void rk4_segment_from(const seg_ctx *S, double x0, double hs, const double *y0,
                             double *out) {
  double y[4] = {1.0, 0.0, 0.0, 0.0};
  if (y0) memcpy(y, y0, sizeof y);
  double kq0[4], kq1[4], kq2[4], k1[4], k2[4], k3[4], k4[4], yt[4];
  medium_at(S, x0, kq0);
  medium_at(S, x0 + 0.5 * hs, kq1);
  medium_at(S, x0 + hs, kq2);
  RHS(kq0, y, k1);
  for (int c = 0; c < 4; ++c) yt[c] = y[c] + 0.5 * hs * k1[c];
  RHS(kq1, yt, k2);
  for (int c = 0; c < 4; ++c) yt[c] = y[c] + 0.5 * hs * k2[c];
  RHS(kq1, yt, k3);
  for (int c = 0; c < 4; ++c) yt[c] = y[c] + hs * k3[c];
  RHS(kq2, yt, k4);
  for (int c = 0; c < 4; ++c) out[c] = y[c] + hs / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
}

/* Dormand-Prince 5(4) tableau (Dormand & Prince, J. Comput. Appl. Math. 6,
 * 1980): nodes c, coefficients a, fifth-order weights b and fourth-order
 * weights bs.  The seventh stage sits at the end point (c = 1). */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_BS[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

/* One Dormand-Prince step over [x1, x2] from (1, 0), Eq. 2.31.  Returns the
 * fifth-order values, the largest dx kappa(xi_j) and the embedded error. */
static void dopri_step(const seg_ctx *S, double x1, double x2, double *y5, double *kmax,
                       double *err) {
  double dx = x2 - x1;
  double K[7][4];
  *kmax = 0.0;
  for (int i = 0; i < 7; ++i) {
    double Y[4] = {1.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < i; ++j)
      for (int c = 0; c < 4; ++c) Y[c] += dx * DP_A[i][j] * K[j][c];
    double kq[4];
    medium_at(S, x1 + DP_C[i] * dx, kq);
    if (dx * kq[0] > *kmax) *kmax = dx * kq[0];
    RHS(kq, Y, K[i]);
  }
  double e = 0.0;
  for (int c = 0; c < 4; ++c) {
    double s5 = (c == 0) ? 1.0 : 0.0, s4 = s5;
    for (int i = 0; i < 7; ++i) {
      s5 += dx * DP_B[i] * K[i][c];
      s4 += dx * DP_BS[i] * K[i][c];
    }
    y5[c] = s5;
    if (fabs(s5 - s4) > e) e = fabs(s5 - s4);
  }
  *err = e;
}

/* Eqs. 2.32-2.33: the implicit two-stage Gauss method solved in closed form.
 * With x measured from the far end x1, the formula is the Gauss-Legendre
 * method when xi_0 = x1 + (1/2 - sqrt(3)/6) dx and xi_1 = x1 + (1/2 + sqrt(3)/6) dx. */
static void gauss2_step(const seg_ctx *S, double x1, double x2, double *y, double *kmax) {
  double dx = x2 - x1, r3 = sqrt(3.0);
  double k0[4], k1[4];
  medium_at(S, x1 + (0.5 - r3 / 6.0) * dx, k0);
  medium_at(S, x1 + (0.5 + r3 / 6.0) * dx, k1);
  double a1 = dx * (k0[0] + k1[0]) / 4.0;
  double a2 = dx * dx * k0[0] * k1[0] / 12.0;
  double den = 1.0 + a1 + a2;
  y[0] = (1.0 - a1 + a2) / den;
  for (int c = 1; c < 4; ++c) {
    double b1 = dx * (k0[c] + k1[c]) / 2.0;
    double b2 = dx * dx * (k0[0] * k1[c] - k1[0] * k0[c]) * r3 / 12.0;
    y[c] = (b1 + b2) / den;
  }
  *kmax = dx * (k0[0] > k1[0] ? k0[0] : k1[0]);
}

/* Eq. 2.34: Simpson's rule on the closed form Eq. 2.12, nodes at the far end,
 * the midpoint and the near end. */
static void simpson_step(const seg_ctx *S, double x1, double x2, double *y, double *kmax) {
  double dx = x2 - x1;
  double k0[4], kh[4], k2[4];
  medium_at(S, x1, k0);
  medium_at(S, 0.5 * (x1 + x2), kh);
  medium_at(S, x2, k2);
  y[0] = exp(-dx * (k0[0] + 4.0 * kh[0] + k2[0]) / 6.0);
  double sa = sqrt(y[0]);
  for (int c = 1; c < 4; ++c) y[c] = dx * (y[0] * k0[c] + 4.0 * sa * kh[c] + k2[c]) / 6.0;
  double m = k0[0] > kh[0] ? k0[0] : kh[0];
  *kmax = dx * (m > k2[0] ? m : k2[0]);
}

/* Eq. 2.18 as an interface (Sec. 2.5): the application supplies the
 * absorption kappa and the intensity I it wants to see; A follows from the
 * absorption (Simpson's rule on the optical depth, nodes far end, midpoint,
 * near end) and B = I (1 - A), 1 - A formed as -expm1.  For constant
 * coefficients this is exactly Eq. 2.13 with q = kappa I. */
static void equilibrium_step(const seg_ctx *S, double x1, double x2, double *y, double *kmax) {
  double dx = x2 - x1;
  double k0[4], kh[4], k2[4];
  medium_at(S, x1, k0);
  medium_at(S, 0.5 * (x1 + x2), kh);
  medium_at(S, x2, k2);
  double e = -dx * (k0[0] + 4.0 * kh[0] + k2[0]) / 6.0;
  double om = -expm1(e);
  y[0] = exp(e);
  for (int c = 1; c < 4; ++c) y[c] = kh[c] * om;
  double m = k0[0] > kh[0] ? k0[0] : kh[0];
  *kmax = dx * (m > k2[0] ? m : k2[0]);
}

/* Algorithm 1: if a stage sees dx kappa > c_RK (or, for DOPRI5, the embedded
 * error exceeds tol), split at the midpoint and return
 * segeval(mid, x2) (+) segeval(x1, mid). */
static void segeval(const seg_ctx *S, const orc_integrator *I, double x1, double x2, int depth,
                    double *out, int64_t *nsteps) {
  double y5[4], kmax, err = 0.0;
  if (I->method == ORC_GAUSS2)
    gauss2_step(S, x1, x2, y5, &kmax);
  else if (I->method == ORC_SIMPSON)
    simpson_step(S, x1, x2, y5, &kmax);
  else if (I->method == ORC_EQUILIBRIUM)
    equilibrium_step(S, x1, x2, y5, &kmax);
  else
    dopri_step(S, x1, x2, y5, &kmax, &err);
  ++*nsteps;
  if (depth < I->max_depth && (kmax > I->c_rk || err > I->tol)) {
    double xm = 0.5 * (x1 + x2), near_s[4], far_s[4];
    segeval(S, I, x1, xm, depth + 1, far_s, nsteps);
    segeval(S, I, xm, x2, depth + 1, near_s, nsteps);
    orc_combine(near_s, far_s, out);
    return;
  }
  memcpy(out, y5, sizeof y5);
}

/* The volume between distances x1 < x2 from the far end: RK4 with nsteps
 * equal steps over the piece, or Algorithm 1 on it. */
static void volume_piece(const seg_ctx *S, const orc_integrator *I, double x1, double x2,
                         double *seg4, int64_t *nsteps) {
  if (I->method == ORC_RK4) {
    double y[4] = {1.0, 0.0, 0.0, 0.0}, hs = (x2 - x1) / I->nsteps;
    for (int n = 0; n < I->nsteps; ++n) rk4_segment_from(S, x1 + n * hs, hs, y, y);
    memcpy(seg4, y, sizeof y);
    *nsteps += I->nsteps;
  } else {
    segeval(S, I, x1, x2, 0, seg4, nsteps);
  }
}

/* Gradient of the field in space at distance x from the far end: the
 * derivatives of the interpolant in the leaf's local coordinates times the
 * derivatives of those coordinates in space (cube: 1/h; shell: through the
 * inverse map, xi = atan2(x.e1, x.n) 2/pi + 1/2 (eta with e2) and
 * zeta = (|x| - r0) / (r1 - r0), divided by h). */
static void field_grad(const seg_ctx *S, double x, double *g) {
  double u[3], d[3] = {0.0, 0.0, 0.0};
  local_coords(S, x, u);
  if (S->F->geometry == 1) {
    double l[3][3], dl[3][3];
    for (int a = 0; a < 3; ++a) {
      quad_basis(u[a], l[a]);
      dl[a][0] = 4.0 * u[a] - 3.0; /* derivatives of the degree-2 Lagrange basis */
      dl[a][1] = 4.0 - 8.0 * u[a];
      dl[a][2] = 4.0 * u[a] - 1.0;
    }
    for (int c = 0; c < 27; ++c) {
      int i = c % 3, j = (c / 3) % 3, k = c / 9;
      double v = (double)S->nodal[c];
      d[0] += v * dl[0][i] * l[1][j] * l[2][k];
      d[1] += v * l[0][i] * dl[1][j] * l[2][k];
      d[2] += v * l[0][i] * l[1][j] * dl[2][k];
    }
    double alpha = S->a_out - x / S->rlen, p[3];
    for (int a = 0; a < 3; ++a) p[a] = S->org[a] + alpha * S->dir[a];
    const double(*fr)[3] = S->F->frames[S->tree];
    double z = dot3(p, fr[0]), y1 = dot3(p, fr[1]), y2 = dot3(p, fr[2]), r = sqrt(dot3(p, p));
    double k_ang = 2.0 / ORC_PI / S->h, k_rad = 1.0 / ((S->F->r1 - S->F->r0) * S->h);
    for (int a = 0; a < 3; ++a) {
      double dxi = (z * fr[1][a] - y1 * fr[0][a]) / (y1 * y1 + z * z);
      double deta = (z * fr[2][a] - y2 * fr[0][a]) / (y2 * y2 + z * z);
      g[a] = d[0] * k_ang * dxi + d[1] * k_ang * deta + d[2] * k_rad * p[a] / r;
    }
    return;
  }
  for (int c = 0; c < 8; ++c) {
    double w[3], dw[3];
    for (int a = 0; a < 3; ++a) {
      int b = (c >> a) & 1;
      w[a] = b ? u[a] : 1.0 - u[a];
      dw[a] = b ? 1.0 : -1.0;
    }
    d[0] += (double)S->nodal[c] * dw[0] * w[1] * w[2];
    d[1] += (double)S->nodal[c] * w[0] * dw[1] * w[2];
    d[2] += (double)S->nodal[c] * w[0] * w[1] * dw[2];
  }
  for (int a = 0; a < 3; ++a) g[a] = d[a] / S->h;
}

/* Crossings of the isosurface inside a segment of length dx: sign changes of
 * s - s_iso between the samples x_k = k dx / 8, each located by bisection.
 * Returns their number (far to near) in xs; *tie is raised when a sample lies
 * within band of s_iso. */
static int iso_crossings(const seg_ctx *S, const orc_integrator *I, double dx, double *xs,
                         double band, int *tie) {
  double g[9];
  for (int k = 0; k <= 8; ++k) {
    double u[3];
    local_coords(S, dx * k / 8.0, u);
    g[k] = field_at(S, u) - I->s_iso;
    if (tie && fabs(g[k]) <= band) *tie = 1;
  }
  int n = 0;
  for (int k = 0; k < 8; ++k) {
    if (!((g[k] < 0.0 && g[k + 1] > 0.0) || (g[k] > 0.0 && g[k + 1] < 0.0))) continue;
    double lo = dx * k / 8.0, hi = dx * (k + 1) / 8.0, glo = g[k];
    for (int it = 0; it < 60; ++it) {
      double mid = 0.5 * (lo + hi), u[3];
      local_coords(S, mid, u);
      double gm = field_at(S, u) - I->s_iso;
      if ((gm < 0.0) == (glo < 0.0)) {
        lo = mid;
        glo = gm;
      } else {
        hi = mid;
      }
    }
    xs[n++] = 0.5 * (lo + hi);
  }
  return n;
}

/* Eqs. 2.18 and 2.35: the surface segment at distance x from the far end. */
static void iso_segment(const seg_ctx *S, const orc_integrator *I, double x, double *seg4) {
  double g[3];
  field_grad(S, x, g);
  double gn = sqrt(dot3(g, g));
  double cphi = gn > 0.0 ? fabs(dot3(g, S->dir)) / (gn * S->rlen) : 1.0;
  double A = I->a_s >= 1.0 ? 1.0 : (cphi <= 0.0 ? 0.0 : pow(I->a_s, 1.0 / cphi));
  seg4[0] = A;
  for (int c = 0; c < 3; ++c) seg4[1 + c] = I->i_s[c] * (1.0 - A);
}

void orc_field_probe(const orc_forest *F, int leaf, const double *org, const double *dir,
                     double a_out, double x, double *s, double *grad) {
  seg_ctx S;
  seg_init(&S, F, leaf, org, dir, a_out);
  double u[3];
  local_coords(&S, x, u);
  *s = field_at(&S, u);
  field_grad(&S, x, grad);
}

static void segment_value(const orc_forest *F, const orc_integrator *I, int leaf,
                          const double *org, const double *dir, double a_in, double a_out,
                          double *seg4, int64_t *nsteps, int *ncross, double band, int *tie) {
  seg_ctx S;
  seg_init(&S, F, leaf, org, dir, a_out);
  double dx = S.rlen * (a_out - a_in);
  int64_t dummy = 0;
  if (!nsteps) nsteps = &dummy;
  if (!I->surface) {
    volume_piece(&S, I, 0.0, dx, seg4, nsteps);
    return;
  }
  double xs[8], acc[4] = {1.0, 0.0, 0.0, 0.0}, piece[4], x1 = 0.0;
  int m = iso_crossings(&S, I, dx, xs, band, tie);
  if (ncross) *ncross += m;
  for (int k = 0; k <= m; ++k) {  /* far to near: volume, surface, volume, ... */
    double x2 = k < m ? xs[k] : dx;
    volume_piece(&S, I, x1, x2, piece, nsteps);
    orc_combine(piece, acc, acc);
    if (k < m) {
      iso_segment(&S, I, x2, piece);
      orc_combine(piece, acc, acc);
    }
    x1 = x2;
  }
  memcpy(seg4, acc, sizeof acc);
}

void orc_segment_ab(const orc_forest *F, const orc_integrator *I, int leaf, const double *org,
                    const double *dir, double a_in, double a_out, double *seg4, int64_t *nsteps) {
  segment_value(F, I, leaf, org, dir, a_in, a_out, seg4, nsteps, NULL, 0.0, NULL);
}

/* ------------------------------------------------------------------------ */
/* Culling and rendering                                                     */
/* ------------------------------------------------------------------------ */

/* The shell's FP32 tables for the decisions (NULL for the cube); freed by
 * the caller. */
static int tables32(const orc_forest *F, float **tan_t, float **rad_t) {
  *tan_t = *rad_t = NULL;
  if (F->geometry != 1) return 0;
  size_t n = ((size_t)1 << F->max_level) + 1;
  *tan_t = (float *)malloc(sizeof(float) * n);
  *rad_t = (float *)malloc(sizeof(float) * n);
  if (!*tan_t || !*rad_t) {
    free(*tan_t);
    free(*rad_t);
    return -1;
  }
  orc_shell_tables32(F, *tan_t, *rad_t);
  return 0;
}

void orc_cull(const orc_forest *F, const orc_camera *C, int32_t *rect, uint8_t *visible,
              uint8_t *uncertain, double band_px, int decide32) {
  orc_cam32 K;
  float *tan_t = NULL, *rad_t = NULL;
  if (decide32) {
    orc_camera32(C, &K);
    if (tables32(F, &tan_t, &rad_t)) return;
  }
#pragma omp parallel for schedule(static)
  for (int l = 0; l < F->nleaves; ++l) {
    int32_t r[4];
    int unc = 0;
    int vis = decide32 ? orc_leaf_rect32(F, &K, tan_t, rad_t, l, r)
                       : orc_leaf_rect(F, C, l, r, NULL, band_px, &unc);
    if (rect) memcpy(rect + 4 * (size_t)l, r, sizeof r);
    visible[l] = (uint8_t)vis;
    if (uncertain) uncertain[l] = (uint8_t)unc;
  }
  free(tan_t);
  free(rad_t);
}

typedef struct {
  double a_in, a_out, s[4];
} orc_seg;

static int cmp_seg(const void *pa, const void *pb) {
  const orc_seg *a = (const orc_seg *)pa, *b = (const orc_seg *)pb;
  if (a->a_in != b->a_in) return a->a_in < b->a_in ? -1 : 1;
  return (a->a_out < b->a_out) ? -1 : (a->a_out > b->a_out);
}

static int cmp_dbl(const void *pa, const void *pb) {
  double a = *(const double *)pa, b = *(const double *)pb;
  return (a > b) - (a < b);
}

/* Back-to-front compositing of one pixel's segments (Eq. 2.11 applied from the
 * farthest segment to the nearest, starting from the background).  Where
 * segments overlap, the ray is cut at every segment end into elementary
 * intervals; each segment covering an interval is cut to it (Eq. 2.20) and the
 * covering pieces are averaged (Eq. 2.21, geometric mean of A, arithmetic mean
 * of B, over all covering pieces). */
static void composite(orc_seg *sg, int n, const double *bg, double *rgba) {
  double I[3] = {bg[0], bg[1], bg[2]}, T = 1.0;
  qsort(sg, (size_t)n, sizeof *sg, cmp_seg);
  int overlap = 0;
  for (int k = 0; k + 1 < n; ++k)
    if (sg[k + 1].a_in < sg[k].a_out) overlap = 1;
  if (!overlap) {
    for (int k = n - 1; k >= 0; --k) {
      for (int c = 0; c < 3; ++c) I[c] = sg[k].s[0] * I[c] + sg[k].s[1 + c];
      T *= sg[k].s[0];
    }
  } else {
    double *pts = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    for (int k = 0; k < n; ++k) { pts[2 * k] = sg[k].a_in; pts[2 * k + 1] = sg[k].a_out; }
    qsort(pts, 2 * (size_t)n, sizeof(double), cmp_dbl);
    for (int p = 2 * n - 2; p >= 0; --p) { /* elementary intervals, far to near */
      double lo = pts[p], hi = pts[p + 1];
      if (!(hi > lo)) continue;
      double logA = 0.0, Bs[3] = {0, 0, 0};
      int cover = 0;
      for (int k = 0; k < n; ++k) {
        if (sg[k].a_in <= lo && sg[k].a_out >= hi) {
          double piece[4];
          orc_cut(sg[k].s, (hi - lo) / (sg[k].a_out - sg[k].a_in), piece);
          logA += log(piece[0]);
          for (int c = 0; c < 3; ++c) Bs[c] += piece[1 + c];
          ++cover;
        }
      }
      if (!cover) continue;
      double A = exp(logA / cover);
      for (int c = 0; c < 3; ++c) I[c] = A * I[c] + Bs[c] / cover;
      T *= A;
    }
    free(pts);
  }
  rgba[0] = I[0]; rgba[1] = I[1]; rgba[2] = I[2]; rgba[3] = 1.0 - T;
}

int64_t orc_render(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                   const int *rows, int nrows, double *rgba, int32_t *counts,
                   uint8_t *uncertain, double band_px, double band_rel, int nthreads,
                   int64_t *nsteps_total) {
  return orc_render_ex(F, C, I, rows, nrows, rgba, counts, NULL, uncertain, band_px, band_rel,
                       nthreads, nsteps_total, 1);
}

int64_t orc_render_ex(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                      const int *rows, int nrows, double *rgba, int32_t *counts,
                      int32_t *crossings, uint8_t *uncertain, double band_px, double band_rel,
                      int nthreads, int64_t *nsteps_total, int decide32) {
  const int W = C->w, H = C->h;
  /* isosurface ties: a sample within this of s_iso (FP32 field values carry
   * relative errors of a few 1e-7 of the data's magnitude) */
  const double smag = fabs(F->s_max) > fabs(F->s_min) ? fabs(F->s_max) : fabs(F->s_min);
  const double sband = 10.0 * band_rel * (smag > 0.0 ? smag : 1.0);
  if (!rows) nrows = H;
  /* FP32 decisions: the candidate pairs are exactly those of the FP32
   * rectangles.  FP64 decisions: every leaf's pixel rectangle widened by one
   * pixel, so that a ray hitting the leaf is never missed through rounding,
   * and the decisions' margins reported as ties. */
  const int widen = decide32 ? 0 : 1;
  orc_cam32 K;
  float *tan_t = NULL, *rad_t = NULL;
  if (decide32) {
    orc_camera32(C, &K);
    if (tables32(F, &tan_t, &rad_t)) return -1;
  }
  int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)F->nleaves);
  uint8_t *vis = (uint8_t *)malloc((size_t)F->nleaves);
  double *pext = (double *)malloc(sizeof(double) * 4 * (size_t)F->nleaves);
  int *rowpos = (int *)malloc(sizeof(int) * (size_t)H);
  if (!rect || !vis || !pext || !rowpos) {
    free(rect); free(vis); free(pext); free(rowpos); free(tan_t); free(rad_t);
    return -1;
  }
  for (int j = 0; j < H; ++j) rowpos[j] = -1;
  for (int r = 0; r < nrows; ++r) rowpos[rows ? rows[r] : r] = r;
#pragma omp parallel for schedule(static)
  for (int l = 0; l < F->nleaves; ++l) {
    int unc = 0;
    vis[l] = (uint8_t)(decide32 ? orc_leaf_rect32(F, &K, tan_t, rad_t, l, rect + 4 * (size_t)l)
                                : orc_leaf_rect(F, C, l, rect + 4 * (size_t)l,
                                                pext + 4 * (size_t)l, band_px, &unc));
  }
  /* rows -> candidate leaves (CSR) */
  int64_t *rstart = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
  for (int l = 0; l < F->nleaves; ++l) {
    if (!vis[l]) continue;
    int j0 = rect[4 * l + 2] - widen, j1 = rect[4 * l + 3] + widen;
    if (j0 < 0) j0 = 0;
    if (j1 > H - 1) j1 = H - 1;
    for (int j = j0; j <= j1; ++j)
      if (rowpos[j] >= 0) rstart[rowpos[j] + 1]++;
  }
  for (int r = 0; r < nrows; ++r) rstart[r + 1] += rstart[r];
  int32_t *rleaf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rstart[nrows] > 0 ? rstart[nrows] : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrows + 1));
  memcpy(fill, rstart, sizeof(int64_t) * (size_t)(nrows + 1));
  for (int l = 0; l < F->nleaves; ++l) {
    if (!vis[l]) continue;
    int j0 = rect[4 * l + 2] - widen, j1 = rect[4 * l + 3] + widen;
    if (j0 < 0) j0 = 0;
    if (j1 > H - 1) j1 = H - 1;
    for (int j = j0; j <= j1; ++j)
      if (rowpos[j] >= 0) rleaf[fill[rowpos[j]]++] = l;
  }
  int64_t total = 0, steps = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : total, steps)
  {
    int cap_pairs = 1024, cap_seg = 256;
    int32_t *pl = (int32_t *)malloc(sizeof(int32_t) * cap_pairs); /* leaf per pair */
    int32_t *pi = (int32_t *)malloc(sizeof(int32_t) * cap_pairs); /* column per pair */
    int32_t *cstart = (int32_t *)malloc(sizeof(int32_t) * (size_t)(W + 1));
    int32_t *pord = (int32_t *)malloc(sizeof(int32_t) * cap_pairs);
    orc_seg *sg = (orc_seg *)malloc(sizeof(orc_seg) * cap_seg);
#pragma omp for schedule(dynamic, 1)
    for (int r = 0; r < nrows; ++r) {
      int j = rows ? rows[r] : r;
      int np = 0;
      for (int64_t q = rstart[r]; q < rstart[r + 1]; ++q) {
        int l = rleaf[q];
        int i0 = rect[4 * l] - widen, i1 = rect[4 * l + 1] + widen;
        if (i0 < 0) i0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        for (int i = i0; i <= i1; ++i) {
          if (np == cap_pairs) {
            cap_pairs *= 2;
            pl = (int32_t *)realloc(pl, sizeof(int32_t) * cap_pairs);
            pi = (int32_t *)realloc(pi, sizeof(int32_t) * cap_pairs);
            pord = (int32_t *)realloc(pord, sizeof(int32_t) * cap_pairs);
          }
          pl[np] = l;
          pi[np] = i;
          ++np;
        }
      }
      /* bucket the candidate pairs by column */
      memset(cstart, 0, sizeof(int32_t) * (size_t)(W + 1));
      for (int p = 0; p < np; ++p) cstart[pi[p] + 1]++;
      for (int i = 0; i < W; ++i) cstart[i + 1] += cstart[i];
      for (int p = 0; p < np; ++p) pord[cstart[pi[p]]++] = p;
      for (int i = W; i > 0; --i) cstart[i] = cstart[i - 1];
      cstart[0] = 0;
      for (int i = 0; i < W; ++i) {
        double org[3], dir[3], amin, amax;
        float org32[3], dir32[3];
        if (decide32) { /* the FP32 ray; its values integrated in FP64 */
          orc_pixel_ray32(&K, i, j, org32, dir32);
          for (int a = 0; a < 3; ++a) { org[a] = org32[a]; dir[a] = dir32[a]; }
          amin = K.amin;
          amax = K.amax;
        } else {
          orc_pixel_ray(C, i, j, org, dir, &amin, &amax);
        }
        int ns = 0, nties = 0, ncross = 0;
        for (int q = cstart[i]; q < cstart[i + 1]; ++q) {
          int l = pl[pord[q]];
          double a_in[2], a_out[2];
          int tie = 0, nhit;
          if (decide32) {
            float f_in[2], f_out[2];
            nhit = orc_ray_leaf32(F, tan_t, rad_t, l, org32, dir32, K.amin, K.amax, f_in, f_out);
            for (int k = 0; k < nhit; ++k) { a_in[k] = f_in[k]; a_out[k] = f_out[k]; }
          } else {
            nhit = orc_ray_leaf_tie(F, l, org, dir, amin, amax, a_in, a_out, band_rel, &tie);
            /* a hit outside the leaf's own rectangle, or within band_px of its edge */
            if (nhit) {
              const double *pe = pext + 4 * (size_t)l;
              if (i < pe[0] + band_px || i > pe[1] - band_px || j < pe[2] + band_px ||
                  j > pe[3] - band_px)
                tie = 1;
            }
          }
          nties += tie;
          if (!nhit) continue;
          for (int k = 0; k < nhit; ++k) {
            if (ns == cap_seg) {
              cap_seg *= 2;
              sg = (orc_seg *)realloc(sg, sizeof(orc_seg) * cap_seg);
            }
            sg[ns].a_in = a_in[k];
            sg[ns].a_out = a_out[k];
            int64_t st = 0;
            int stie = 0;
            segment_value(F, I, l, org, dir, a_in[k], a_out[k], sg[ns].s, &st, &ncross, sband,
                          &stie);
            nties += stie;
            steps += st;
            ++ns;
          }
        }
        size_t pix = (size_t)r * W + i;
        composite(sg, ns, I->bg, rgba + 4 * pix);
        if (counts) counts[pix] = ns;
        if (crossings) crossings[pix] = ncross;
        if (uncertain) uncertain[pix] = (uint8_t)(nties < 255 ? nties : 255);
        total += ns;
      }
    }
    free(pl); free(pi); free(cstart); free(pord); free(sg);
  }
  free(rect); free(vis); free(pext); free(rowpos); free(rstart); free(rleaf); free(fill);
  free(tan_t); free(rad_t);
  if (nsteps_total) *nsteps_total = steps;
  return total;
}

/* ------------------------------------------------------------------------ */
/* Gradient (reverse mode, FP64)                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  double *g_nodal; /* [N*8] */
  double *g_tf;    /* [32] */
  uint8_t *tree_tie; /* [N] or NULL: a split test of Algorithm 1 near its threshold */
  double tree_band;
  double *a_nodal, *a_tf; /* or NULL: the sums of the terms' magnitudes (the sums'
                             condition: the scale of their rounding in another
                             precision) */
} grad_acc;

/* Adjoint of the medium at distance x from the far end: vbar = dL/d(kappa,
 * q_r, q_g, q_b) there; accumulates into the knot values and, through the
 * transfer function's slope and the trilinear weights, into the leaf's 8
 * nodal values. */
static void medium_bwd(const seg_ctx *S, int leaf, double x, const double *vbar, grad_acc *G) {
  const orc_forest *F = S->F;
  double u[3];
  local_coords(S, x, u);
  double s = field_at(S, u);
  double zr = (s - F->s_min) / (F->s_max - F->s_min) * 7.0;
  int inside = zr > 0.0 && zr < 7.0;
  double z = zr < 0.0 ? 0.0 : (zr > 7.0 ? 7.0 : zr);
  int k = (int)floor(z);
  if (k > 6) k = 6;
  double w = z - k, sbar = 0.0, sabs = 0.0;
  for (int c = 0; c < 4; ++c) {
#pragma omp atomic
    G->g_tf[4 * k + c] += (1.0 - w) * vbar[c];
#pragma omp atomic
    G->g_tf[4 * (k + 1) + c] += w * vbar[c];
    if (G->a_tf) {
#pragma omp atomic
      G->a_tf[4 * k + c] += fabs((1.0 - w) * vbar[c]);
#pragma omp atomic
      G->a_tf[4 * (k + 1) + c] += fabs(w * vbar[c]);
    }
    if (inside) {
      double t = vbar[c] * ((double)F->tf[4 * (k + 1) + c] - (double)F->tf[4 * k + c]) * 7.0 /
                 (F->s_max - F->s_min);
      sbar += t;
      sabs += fabs(t);
    }
  }
  if (F->geometry == 1) {
    double lu[3], lv[3], lw[3];
    quad_basis(u[0], lu);
    quad_basis(u[1], lv);
    quad_basis(u[2], lw);
    for (int c = 0; c < 27; ++c) {
      double wt = lu[c % 3] * lv[(c / 3) % 3] * lw[c / 9];
#pragma omp atomic
      G->g_nodal[27 * (size_t)leaf + c] += sbar * wt;
      if (G->a_nodal) {
#pragma omp atomic
        G->a_nodal[27 * (size_t)leaf + c] += sabs * fabs(wt);
      }
    }
    return;
  }
  for (int c = 0; c < 8; ++c) {
    double wx = (c & 1) ? u[0] : 1.0 - u[0];
    double wy = (c & 2) ? u[1] : 1.0 - u[1];
    double wz = (c & 4) ? u[2] : 1.0 - u[2];
#pragma omp atomic
    G->g_nodal[8 * (size_t)leaf + c] += sbar * wx * wy * wz;
    if (G->a_nodal) {
#pragma omp atomic
      G->a_nodal[8 * (size_t)leaf + c] += sabs * fabs(wx * wy * wz);
    }
  }
}

/* Adjoint of one explicit RK step from (1, 0) over [x1, x1 + dx] with nodes
 * c[i], coefficients a[i][j] and weights b[i] (Eq. 2.31): given ybar =
 * dL/d(output), accumulates dL/d(kappa, q) at every node. */
static void rk_step_bwd(const seg_ctx *S, int leaf, double x1, double dx, int ns, const double *c,
                        const double *a, int lda, const double *b, const double *ybar,
                        grad_acc *G) {
  double kq[7][4], Y[7][4], K[7][4], Kb[7][4];
  for (int i = 0; i < ns; ++i) {
    for (int q = 0; q < 4; ++q) Y[i][q] = (q == 0) ? 1.0 : 0.0;
    for (int j = 0; j < i; ++j)
      for (int q = 0; q < 4; ++q) Y[i][q] += dx * a[i * lda + j] * K[j][q];
    medium_at(S, x1 + c[i] * dx, kq[i]);
    RHS(kq[i], Y[i], K[i]);
  }
  for (int i = 0; i < ns; ++i)
    for (int q = 0; q < 4; ++q) Kb[i][q] = dx * b[i] * ybar[q];
  for (int i = ns - 1; i >= 0; --i) {
    double vbar[4];
    /* K_i = (-kappa Y_A, q_c - kappa Y_c) */
    vbar[0] = 0.0;
    for (int q = 0; q < 4; ++q) vbar[0] -= Kb[i][q] * Y[i][q];
    for (int q = 1; q < 4; ++q) vbar[q] = Kb[i][q];
    medium_bwd(S, leaf, x1 + c[i] * dx, vbar, G);
    double Yb[4];
    for (int q = 0; q < 4; ++q) Yb[q] = -kq[i][0] * Kb[i][q];
    for (int j = 0; j < i; ++j)
      for (int q = 0; q < 4; ++q) Kb[j][q] += dx * a[i * lda + j] * Yb[q];
  }
}

static const double RK4_C[4] = {0.0, 0.5, 0.5, 1.0};
static const double RK4_A[4][4] = {{0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}};
static const double RK4_B[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};

/* Adjoint of a near (+) far combination: result (A, B) = (An Af, Bn + An Bf). */
static void combine_bwd(const double *nr, const double *fr, const double *ybar, double *nbar,
                        double *fbar) {
  nbar[0] = ybar[0] * fr[0];
  for (int c = 1; c < 4; ++c) {
    nbar[0] += ybar[c] * fr[c];
    nbar[c] = ybar[c];
    fbar[c] = nr[0] * ybar[c];
  }
  fbar[0] = ybar[0] * nr[0];
}

/* Adjoint of the Gauss-2 closed form (Eqs. 2.32-2.33) over [x1, x2]: A and B
 * are rational in (kappa, q) at the two Gauss nodes; ybar = dL/d(A, B). */
static void gauss2_step_bwd(const seg_ctx *S, int leaf, double x1, double x2, const double *ybar,
                            grad_acc *G) {
  const double r3 = sqrt(3.0), dx = x2 - x1;
  const double xa = x1 + (0.5 - r3 / 6.0) * dx, xb = x1 + (0.5 + r3 / 6.0) * dx;
  double k0[4], k1[4];
  medium_at(S, xa, k0);
  medium_at(S, xb, k1);
  const double a1 = dx * (k0[0] + k1[0]) / 4.0, a2 = dx * dx * k0[0] * k1[0] / 12.0;
  const double den = 1.0 + a1 + a2, s = dx * dx * r3 / 12.0;
  /* d(den)/d(kappa_0), d(den)/d(kappa_1); d(numerator of A) = d(den) - dx/2 */
  const double d0 = dx / 4.0 + dx * dx * k1[0] / 12.0, d1 = dx / 4.0 + dx * dx * k0[0] / 12.0;
  double v0[4], v1[4];
  v0[0] = ybar[0] * (2.0 * a1 * d0 - 0.5 * dx * den) / (den * den);
  v1[0] = ybar[0] * (2.0 * a1 * d1 - 0.5 * dx * den) / (den * den);
  for (int c = 1; c < 4; ++c) {
    const double Bc = (dx * (k0[c] + k1[c]) / 2.0 + s * (k0[0] * k1[c] - k1[0] * k0[c])) / den;
    v0[0] += ybar[c] * (s * k1[c] - Bc * d0) / den;
    v1[0] += ybar[c] * (-s * k0[c] - Bc * d1) / den;
    v0[c] = ybar[c] * (0.5 * dx - s * k1[0]) / den;
    v1[c] = ybar[c] * (0.5 * dx + s * k0[0]) / den;
  }
  medium_bwd(S, leaf, xa, v0, G);
  medium_bwd(S, leaf, xb, v1, G);
}

/* Adjoint of Simpson's rule on the closed form (Eq. 2.34), nodes far end,
 * midpoint, near end: A = exp(e), e = -dx (k_0 + 4 k_h + k_2) / 6,
 * B_c = dx (A q_0 + 4 sqrt(A) q_h + q_2) / 6. */
static void simpson_step_bwd(const seg_ctx *S, int leaf, double x1, double x2, const double *ybar,
                             grad_acc *G) {
  const double dx = x2 - x1, xm = 0.5 * (x1 + x2);
  double k0[4], kh[4], k2[4];
  medium_at(S, x1, k0);
  medium_at(S, xm, kh);
  medium_at(S, x2, k2);
  const double A = exp(-dx * (k0[0] + 4.0 * kh[0] + k2[0]) / 6.0), sa = sqrt(A);
  double s0 = 0.0, sh = 0.0;
  for (int c = 1; c < 4; ++c) {
    s0 += ybar[c] * k0[c];
    sh += ybar[c] * kh[c];
  }
  /* dL/de: through A directly and through A and sqrt(A) in B */
  const double Fe = ybar[0] * A + dx / 6.0 * (s0 * A + 2.0 * sh * sa);
  double v0[4], vh[4], v2[4];
  v0[0] = -dx / 6.0 * Fe;
  vh[0] = -4.0 * dx / 6.0 * Fe;
  v2[0] = -dx / 6.0 * Fe;
  for (int c = 1; c < 4; ++c) {
    v0[c] = ybar[c] * dx * A / 6.0;
    vh[c] = ybar[c] * 4.0 * dx * sa / 6.0;
    v2[c] = ybar[c] * dx / 6.0;
  }
  medium_bwd(S, leaf, x1, v0, G);
  medium_bwd(S, leaf, xm, vh, G);
  medium_bwd(S, leaf, x2, v2, G);
}

/* Adjoint of the Eq. 2.18 interface: A = exp(e) (Simpson's rule on the optical
 * depth), B_c = I_c (1 - A) with I_c read at the midpoint. */
static void equilibrium_step_bwd(const seg_ctx *S, int leaf, double x1, double x2,
                                 const double *ybar, grad_acc *G) {
  const double dx = x2 - x1, xm = 0.5 * (x1 + x2);
  double k0[4], kh[4], k2[4];
  medium_at(S, x1, k0);
  medium_at(S, xm, kh);
  medium_at(S, x2, k2);
  const double e = -dx * (k0[0] + 4.0 * kh[0] + k2[0]) / 6.0, A = exp(e), om = -expm1(e);
  double sI = 0.0;
  for (int c = 1; c < 4; ++c) sI += ybar[c] * kh[c];
  const double Fe = A * (ybar[0] - sI); /* dL/de */
  double v0[4] = {-dx / 6.0 * Fe, 0.0, 0.0, 0.0}, v2[4] = {-dx / 6.0 * Fe, 0.0, 0.0, 0.0};
  double vh[4] = {-4.0 * dx / 6.0 * Fe, 0.0, 0.0, 0.0};
  for (int c = 1; c < 4; ++c) vh[c] = ybar[c] * om;
  medium_bwd(S, leaf, x1, v0, G);
  medium_bwd(S, leaf, xm, vh, G);
  medium_bwd(S, leaf, x2, v2, G);
}

/* Adjoint of Algorithm 1 (the step tree is re-derived with the same tests). */
static void segeval_bwd(const seg_ctx *S, const orc_integrator *I, int leaf, double x1, double x2,
                        int depth, const double *ybar, grad_acc *G) {
  double y5[4], kmax, err = 0.0;
  if (I->method == ORC_GAUSS2)
    gauss2_step(S, x1, x2, y5, &kmax);
  else if (I->method == ORC_SIMPSON)
    simpson_step(S, x1, x2, y5, &kmax);
  else if (I->method == ORC_EQUILIBRIUM)
    equilibrium_step(S, x1, x2, y5, &kmax);
  else
    dopri_step(S, x1, x2, y5, &kmax, &err);
  /* a test within the band of its threshold can go either way in another
   * precision: the gradient of that leaf then belongs to another step tree */
  if (G->tree_tie && depth < I->max_depth &&
      (fabs(err - I->tol) <= G->tree_band * I->tol ||
       fabs(kmax - I->c_rk) <= G->tree_band * I->c_rk)) {
#pragma omp atomic write
    G->tree_tie[leaf] = 1;
  }
  if (depth < I->max_depth && (kmax > I->c_rk || err > I->tol)) {
    double xm = 0.5 * (x1 + x2), nr[4], fr[4], nb[4], fb[4];
    int64_t dummy = 0;
    segeval(S, I, x1, xm, depth + 1, fr, &dummy);
    segeval(S, I, xm, x2, depth + 1, nr, &dummy);
    combine_bwd(nr, fr, ybar, nb, fb);
    segeval_bwd(S, I, leaf, x1, xm, depth + 1, fb, G);
    segeval_bwd(S, I, leaf, xm, x2, depth + 1, nb, G);
    return;
  }
  if (I->method == ORC_GAUSS2)
    gauss2_step_bwd(S, leaf, x1, x2, ybar, G);
  else if (I->method == ORC_SIMPSON)
    simpson_step_bwd(S, leaf, x1, x2, ybar, G);
  else if (I->method == ORC_EQUILIBRIUM)
    equilibrium_step_bwd(S, leaf, x1, x2, ybar, G);
  else
    rk_step_bwd(S, leaf, x1, x2 - x1, 6, DP_C, &DP_A[0][0], 6, DP_B, ybar, G);
}

/* Adjoint of orc_segment_ab (RK4 and DOPRI5). */
static void segment_bwd(const orc_forest *F, const orc_integrator *I, int leaf, const double *org,
                        const double *dir, double a_in, double a_out, const double *ybar,
                        grad_acc *G) {
  seg_ctx S;
  seg_init(&S, F, leaf, org, dir, a_out);
  double dx = S.rlen * (a_out - a_in);
  if (I->method == ORC_RK4) {
    /* y_{n+1} = step_n(y_n) = R_n y_n + G_n: keep every y_n, then sweep back */
    int n = I->nsteps;
    double hs = dx / n;
    double *ys = (double *)malloc(sizeof(double) * 4 * (size_t)(n + 1));
    ys[0] = 1.0; ys[1] = ys[2] = ys[3] = 0.0;
    for (int m = 0; m < n; ++m) { /* step from the state y_m: the same as rk4_segment */
      double st[4];
      rk4_segment_from(&S, m * hs, hs, ys + 4 * m, st);
      memcpy(ys + 4 * (m + 1), st, sizeof st);
    }
    double yb[4];
    memcpy(yb, ybar, sizeof yb);
    for (int m = n - 1; m >= 0; --m) {
      /* step m maps y_m to y_{m+1} = S_m (+) y_m with S_m the step from (1, 0):
       * adjoint of the step's own value, then of the carried state */
      double sm[4], sb[4], yprev_b[4];
      rk4_segment_from(&S, m * hs, hs, NULL, sm);
      combine_bwd(sm, ys + 4 * m, yb, sb, yprev_b);
      rk_step_bwd(&S, leaf, m * hs, hs, 4, RK4_C, &RK4_A[0][0], 4, RK4_B, sb, G);
      memcpy(yb, yprev_b, sizeof yb);
    }
    free(ys);
  } else {
    segeval_bwd(&S, I, leaf, 0.0, dx, 0, ybar, G);
  }
}

int orc_render_grad(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                    const double *dL_drgba, double *g_nodal, double *g_tf, int nthreads,
                    int decide32, uint8_t *tree_tie, double tree_band, double *a_nodal,
                    double *a_tf) {
  if (I->surface) return -2;
  const int W = C->w, H = C->h, widen = decide32 ? 0 : 1;
  orc_cam32 K;
  float *tan_t = NULL, *rad_t = NULL;
  if (decide32) {
    orc_camera32(C, &K);
    if (tables32(F, &tan_t, &rad_t)) return -1;
  }
  int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)F->nleaves);
  if (!rect) {
    free(tan_t);
    free(rad_t);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int l = 0; l < F->nleaves; ++l) {
    int unc = 0;
    if (decide32)
      orc_leaf_rect32(F, &K, tan_t, rad_t, l, rect + 4 * (size_t)l);
    else
      orc_leaf_rect(F, C, l, rect + 4 * (size_t)l, NULL, 0.0, &unc);
  }
  /* the leaves whose (widened) rectangle meets each row with a non-zero
   * image adjoint (CSR) */
  int64_t *rs = (int64_t *)calloc((size_t)H + 1, sizeof(int64_t));
  uint8_t *live = (uint8_t *)calloc((size_t)H, 1);
  if (!rs || !live) {
    free(rs); free(live); free(rect); free(tan_t); free(rad_t);
    return -1;
  }
  for (int p = 0; p < W * H; ++p) {
    const double *gb = dL_drgba + 4 * (size_t)p;
    if (gb[0] != 0.0 || gb[1] != 0.0 || gb[2] != 0.0 || gb[3] != 0.0) live[p / W] = 1;
  }
  for (int l = 0; l < F->nleaves; ++l) {
    const int32_t *rc = rect + 4 * (size_t)l;
    if (rc[0] > rc[1]) continue;
    for (int j = rc[2] - widen; j <= rc[3] + widen; ++j)
      if (j >= 0 && j < H && live[j]) rs[j + 1]++;
  }
  for (int j = 0; j < H; ++j) rs[j + 1] += rs[j];
  int32_t *rl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rs[H] > 0 ? rs[H] : 1));
  int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(H + 1));
  if (!rl || !fillp) {
    free(rs); free(live); free(rect); free(rl); free(fillp); free(tan_t); free(rad_t);
    return -1;
  }
  memcpy(fillp, rs, sizeof(int64_t) * (size_t)(H + 1));
  for (int l = 0; l < F->nleaves; ++l) {
    const int32_t *rc = rect + 4 * (size_t)l;
    if (rc[0] > rc[1]) continue;
    for (int j = rc[2] - widen; j <= rc[3] + widen; ++j)
      if (j >= 0 && j < H && live[j]) rl[fillp[j]++] = l;
  }
  memset(g_nodal, 0, sizeof(double) * (size_t)nodal_stride(F) * (size_t)F->nleaves);
  memset(g_tf, 0, sizeof(double) * 32);
  grad_acc G = {g_nodal, g_tf, tree_tie, tree_band, a_nodal, a_tf};
  if (tree_tie) memset(tree_tie, 0, (size_t)F->nleaves);
  if (a_nodal) memset(a_nodal, 0, sizeof(double) * (size_t)nodal_stride(F) * (size_t)F->nleaves);
  if (a_tf) memset(a_tf, 0, sizeof(double) * 32);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    int cap = 256;
    orc_seg *sg = (orc_seg *)malloc(sizeof(orc_seg) * cap);
    int *sl = (int *)malloc(sizeof(int) * cap);
#pragma omp for schedule(dynamic, 16)
    for (int p = 0; p < W * H; ++p) {
      int i = p % W, j = p / W;
      const double *gb = dL_drgba + 4 * (size_t)p;
      if (gb[0] == 0.0 && gb[1] == 0.0 && gb[2] == 0.0 && gb[3] == 0.0) continue;
      double org[3], dir[3], amin, amax;
      float org32[3], dir32[3];
      if (decide32) {
        orc_pixel_ray32(&K, i, j, org32, dir32);
        for (int a = 0; a < 3; ++a) { org[a] = org32[a]; dir[a] = dir32[a]; }
        amin = K.amin;
        amax = K.amax;
      } else {
        orc_pixel_ray(C, i, j, org, dir, &amin, &amax);
      }
      int ns = 0;
      for (int64_t qq = rs[j]; qq < rs[j + 1]; ++qq) {
        const int l = rl[qq];
        const int32_t *rc = rect + 4 * (size_t)l;
        if (i < rc[0] - widen || i > rc[1] + widen) continue;
        double a0[2], a1[2];
        int nhit;
        if (decide32) {
          float f0[2], f1[2];
          nhit = orc_ray_leaf32(F, tan_t, rad_t, l, org32, dir32, K.amin, K.amax, f0, f1);
          for (int k = 0; k < nhit; ++k) { a0[k] = f0[k]; a1[k] = f1[k]; }
        } else {
          nhit = orc_ray_leaf(F, l, org, dir, amin, amax, a0, a1);
        }
        for (int k = 0; k < nhit; ++k) {
          if (ns == cap) {
            cap *= 2;
            sg = (orc_seg *)realloc(sg, sizeof(orc_seg) * cap);
            sl = (int *)realloc(sl, sizeof(int) * cap);
          }
          sg[ns].a_in = a0[k];
          sg[ns].a_out = a1[k];
          orc_segment_ab(F, I, l, org, dir, a0[k], a1[k], sg[ns].s, NULL);
          sl[ns] = l;
          ++ns;
        }
      }
      /* order near to far by alpha (an index sort carrying the leaf ids) */
      for (int a = 1; a < ns; ++a) {
        orc_seg v = sg[a];
        int vl = sl[a], b = a - 1;
        while (b >= 0 && sg[b].a_in > v.a_in) {
          sg[b + 1] = sg[b];
          sl[b + 1] = sl[b];
          --b;
        }
        sg[b + 1] = v;
        sl[b + 1] = vl;
      }
      /* near transmittance T_k and far aggregate G_k of every segment */
      double far[4] = {1.0, 0.0, 0.0, 0.0};
      double *Gk = (double *)malloc(sizeof(double) * 4 * (size_t)(ns > 0 ? ns : 1));
      for (int k = ns - 1; k >= 0; --k) {
        memcpy(Gk + 4 * k, far, sizeof far);
        orc_combine(sg[k].s, far, far);
      }
      double T = 1.0;
      for (int k = 0; k < ns; ++k) {
        const double *g = Gk + 4 * k;
        double ybar[4];
        /* I_c = near.B + T (B_k + A_k (g.B_c + g.A bg_c)), alpha = 1 - T A_k g.A */
        ybar[0] = 0.0;
        for (int c = 0; c < 3; ++c) ybar[0] += T * gb[c] * (g[1 + c] + g[0] * I->bg[c]);
        ybar[0] -= T * gb[3] * g[0];
        for (int c = 0; c < 3; ++c) ybar[1 + c] = T * gb[c];
        segment_bwd(F, I, sl[k], org, dir, sg[k].a_in, sg[k].a_out, ybar, &G);
        T *= sg[k].s[0];
      }
      free(Gk);
    }
    free(sg);
    free(sl);
  }
  free(rect); free(rs); free(live); free(rl); free(fillp); free(tan_t); free(rad_t);
  return 0;
}
