/* FP64 CPU oracle for the forest-of-octrees raycaster (Burstedde 2018,
 * "Distributed-Memory Forest-of-Octrees Raycasting").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_1809_01334_gb300/csrc, and neither includes the other.
 *
 * Everything is plain, slow, obviously-correct double-precision C:
 *   - segment algebra: combine (Eq. 2.14), inverse (Eq. 2.15), cut (Eq. 2.20),
 *     average (Eq. 2.21);
 *   - camera rays (Eq. 2.5), camera transform (Eq. 2.6), axis-aligned bounding
 *     boxes projected to pixel rectangles (Sec. 2.2, App. A.2);
 *   - per-segment (A, B) by explicit Runge-Kutta on the decoupled ODEs
 *     (Eqs. 2.29 and 2.31) with the adaptive bisection of Algorithm 1;
 *   - per-pixel compositing by the classical back-to-front recursion
 *     I <- A I + B (Eq. 2.11), with overlaps resolved by cut + average (Sec. 2.5).
 */
#ifndef OCR_ORACLE_H
#define OCR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A forest: one unit-cube tree with the identity map (geometry 0), or the six
 * trees of a cubed-sphere shell (geometry 1).  Shell tree k maps reference
 * (xi, eta, zeta) to r(zeta) normalize(n + tan(pi/4 (2 xi - 1)) e1 +
 * tan(pi/4 (2 eta - 1)) e2), r(zeta) = r0 + (r1 - r0) zeta, with (n, e1, e2)
 * = frames[k]. */
typedef struct {
  int nleaves;
  int max_level;            /* anchors are integers in units of 2^-max_level */
  const int32_t *anchor;    /* [nleaves*3] */
  const uint8_t *level;     /* [nleaves] */
  const float *nodal;       /* [nleaves*stride]: cube, 8 corners c = bx + 2 by + 4 bz;
                               shell, 27 nodes a + 3 b + 9 c at (a, b, c)/2 */
  const float *tf;          /* [8*4]: kappa, q_r, q_g, q_b at the 8 knots */
  double s_min, s_max;      /* knot k sits at s_min + k (s_max - s_min) / 7 */
  int geometry;             /* 0 cube, 1 shell */
  const int32_t *tree;      /* [nleaves] (shell) */
  double frames[6][3][3];
  double r0, r1;
} orc_forest;

typedef struct {
  double o[3], v[3], t[3], u[3];
  double ell, near_, far_;
  int w, h, ortho;
} orc_camera;

enum { ORC_RK4 = 0, ORC_DOPRI5 = 1, ORC_GAUSS2 = 2, ORC_SIMPSON = 3, ORC_EQUILIBRIUM = 4 };
typedef struct {
  int method;      /* ORC_RK4: nsteps equal classical RK4 steps; the others inside Algorithm 1:
                      ORC_DOPRI5 Dormand-Prince 5(4), ORC_GAUSS2 the implicit 2-stage Gauss
                      closed form (Eqs. 2.32-2.33), ORC_SIMPSON quadrature (Eq. 2.34),
                      ORC_EQUILIBRIUM the intensity interface of Eq. 2.18: the transfer
                      function's colour channels are the desired intensity I, a step's A is
                      exp(-Simpson integral of kappa) and its B = I(1 - A), I taken at the
                      step's midpoint */
  int nsteps;
  double tol;      /* DOPRI5 only: split when the embedded error estimate exceeds tol */
  double c_rk;     /* split when dx * kappa(xi_j) > c_rk at any stage point */
  int max_depth;   /* bisection depth cap */
  double bg[3];    /* background intensity I_b per channel */
  /* Sec. 2.8 on the isosurface s = s_iso of the field (cube forests): where a
   * segment's field crosses s_iso, the segment is cut there and a surface
   * segment A_phi = a_s^(1 / cos phi), B_phi = i_s (1 - A_phi) (Eqs. 2.18,
   * 2.35) inserted, phi the angle between the ray and the field gradient.
   * Crossings are the sign changes of s - s_iso between 9 equally spaced
   * samples of the segment (far end to near end), located by bisection.
   * Both geometries (the shell's gradient through its inverse map). */
  int surface;
  double s_iso, a_s, i_s[3];
} orc_integrator;

/* FP32 camera constants of step a1 (Eq. 2.5), each rounded once from FP64:
 * o, v (v/n when orthographic), ell t, ell u, t, u, v/n, n, f, ell, the image
 * centre (w-1)/2, (h-1)/2, and the alpha range [1, f/n] ([0, f]). */
typedef struct {
  float o[3], v[3], lt[3], lu[3], t[3], u[3], vn[3];
  float n, f, ell, cw, ch, amin, amax;
  int w, h, ortho;
} orc_cam32;

/* Segment algebra on (A, B_r, B_g, B_b). */
void orc_combine(const double *near_seg, const double *far_seg, double *out);
void orc_inverse(const double *s, double *out);
void orc_cut(const double *s, double frac, double *out);
void orc_average(const double *s1, const double *s2, double *out);

/* Transfer function and trilinear field evaluation. */
void orc_tf_eval(const orc_forest *F, double s, double *kq /* [4] */);
double orc_trilinear(const float *nodal8, double u, double v, double w);

/* Ray of pixel (i, j): origin, direction and admissible alpha range. */
void orc_pixel_ray(const orc_camera *C, int i, int j, double *org, double *dir,
                   double *amin, double *amax);

/* Pixel rectangle of a leaf's camera-space bounding box.  Returns 1 if the
 * leaf is visible.  rect = {i0, i1, j0, j1} (inclusive; {0,-1,0,-1} when not
 * visible).  pext (may be NULL) receives the continuous projected extents;
 * *vis_unc is set when a threshold within band_px of a decision would change
 * the rectangle or the visibility. */
int orc_leaf_rect(const orc_forest *F, const orc_camera *C, int leaf, int32_t *rect,
                  double *pext, double band_px, int *vis_unc);

/* Intersection of a ray with a leaf, clipped to [amin, amax]: a slab test
 * for the cube; for a shell leaf the four half-spaces through the origin
 * bounding its angular extent and the spherical shell between its two radii
 * (at most two intervals).  Returns the number of non-empty intervals and
 * fills a_in[k], a_out[k] (arrays of 2), nearest first. */
int orc_ray_leaf(const orc_forest *F, int leaf, const double *org, const double *dir,
                 double amin, double amax, double *a_in, double *a_out);

/* The same, also raising *tie (when tie is not NULL) for a decision within
 * band_rel of flipping: an interval of relative length <= band_rel, or a ray
 * whose squared distance from the shell's centre is within band_rel of a
 * leaf's squared radius.  For the cube, a_in[0], a_out[0] receive the slab
 * interval even when it is empty. */
int orc_ray_leaf_tie(const orc_forest *F, int leaf, const double *org, const double *dir,
                     double amin, double amax, double *a_in, double *a_out, double band_rel,
                     int *tie);

/* Index decisions in FP32 (the GPU path's precision), by one canonical
 * evaluation: every operation rounded once, in a fixed order, subnormals
 * flushed.  orc_camera32 rounds the camera; orc_pixel_ray32 is Eq. 2.5;
 * orc_shell_tables32 fills the shell's plane tangents and radii
 * (2^max_level + 1 floats each; unused for the cube, may be NULL there);
 * orc_leaf_rect32 is orc_leaf_rect's rectangle and orc_ray_leaf32
 * orc_ray_leaf's intervals. */
void orc_camera32(const orc_camera *C, orc_cam32 *K);
void orc_pixel_ray32(const orc_cam32 *K, int i, int j, float *org, float *dir);
void orc_shell_tables32(const orc_forest *F, float *tan_t, float *rad_t);
int orc_leaf_rect32(const orc_forest *F, const orc_cam32 *K, const float *tan_t,
                    const float *rad_t, int leaf, int32_t *rect);
int orc_ray_leaf32(const orc_forest *F, const float *tan_t, const float *rad_t, int leaf,
                   const float *org, const float *dir, float amin, float amax, float *a_in,
                   float *a_out);

/* The equiangular map of tree reference coordinates to space and its inverse
 * (shell forests). */
void orc_shell_map(const orc_forest *F, int tree, const double *ref, double *x);
void orc_shell_inverse(const orc_forest *F, int tree, const double *x, double *ref);

/* Degree-2 Lagrange interpolation on the nodes {0, 1/2, 1}^3. */
double orc_triquadratic(const float *nodal27, double u, double v, double w);

/* The field s and its gradient in space at the point of the ray o + alpha r
 * inside the leaf with alpha = a_out - x / |r| (the surfaces' normal,
 * Sec. 2.8). */
void orc_field_probe(const orc_forest *F, int leaf, const double *org, const double *dir,
                     double a_out, double x, double *s, double *grad);

/* (A, B) of the segment [a_in, a_out] of the ray inside the leaf. */
void orc_segment_ab(const orc_forest *F, const orc_integrator *I, int leaf,
                    const double *org, const double *dir, double a_in, double a_out,
                    double *seg4, int64_t *nsteps);

/* Visibility of every leaf.  rect may be NULL.  decide32 != 0: the
 * rectangles of orc_leaf_rect32 (uncertain all 0); else orc_leaf_rect's with
 * its tie flags. */
void orc_cull(const orc_forest *F, const orc_camera *C, int32_t *rect, uint8_t *visible,
              uint8_t *uncertain, double band_px, int decide32);

/* Render the listed image rows (rows == NULL: all rows).  rgba[nrows*w*4],
 * counts[nrows*w] (segments per ray), uncertain[nrows*w] (the number of this
 * ray's leaves, saturating at 255, with a decision within the tie band; each
 * such leaf can change the ray's segment count by at most two).  Returns the total number of segments, or a
 * negative number on allocation failure. */
int64_t orc_render(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                   const int *rows, int nrows, double *rgba, int32_t *counts,
                   uint8_t *uncertain, double band_px, double band_rel, int nthreads,
                   int64_t *nsteps_total);

/* The same, also writing crossings[nrows*w] (isosurface crossings per ray;
 * may be NULL); a ray with a sample within the tie band of s_iso counts as a
 * tie in uncertain.  decide32 != 0 (orc_render's choice): rectangles, rays
 * and intervals from the FP32 decisions (orc_leaf_rect32, orc_pixel_ray32,
 * orc_ray_leaf32; no geometric ties are flagged), the segment values in FP64
 * over the FP32 ray and end points; decide32 == 0: all in FP64, geometric
 * ties flagged. */
int64_t orc_render_ex(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                      const int *rows, int nrows, double *rgba, int32_t *counts,
                      int32_t *crossings, uint8_t *uncertain, double band_px, double band_rel,
                      int nthreads, int64_t *nsteps_total, int decide32);

/* Gradient of L with respect to the nodal values and the transfer-function
 * knots, given dL/d(rgba) per pixel [h*w*4] (row-major).  FP64 reverse mode:
 * per pixel the segments are ordered by alpha, each one's adjoint follows
 * from the transmittance of the nearer ones and the aggregate of the farther
 * ones (with the background), and is carried back through the integrator
 * (RK4, or Algorithm 1 with DOPRI5, the Gauss-2 closed form, Simpson's rule
 * or the Eq. 2.18 interface; the step tree is re-derived with the same
 * tests), the transfer function and the trilinear (cube) or triquadratic
 * (shell) interpolation.  g_nodal [nleaves*8 or *27], g_tf [32] are
 * overwritten.  decide32 as in orc_render_ex.  tree_tie [nleaves] (may be
 * NULL) flags the leaves with a DOPRI5 split test of Algorithm 1 within
 * tree_band (relative) of its threshold (the embedded error against tol, or
 * dx kappa against c_RK): a computation in another precision may take
 * another step tree there, and with it the derivative of another
 * discretisation.  a_nodal, a_tf (may be NULL) receive, per coordinate, the
 * sum of the magnitudes of the terms summed into it (at the transfer function
 * and the interpolation weights): the scale of the rounding error of that
 * sum.  Returns 0, -1 when out of memory, or -2 with a surface. */
int orc_render_grad(const orc_forest *F, const orc_camera *C, const orc_integrator *I,
                    const double *dL_drgba, double *g_nodal, double *g_tf, int nthreads,
                    int decide32, uint8_t *tree_tie, double tree_band, double *a_nodal,
                    double *a_tf);

#ifdef __cplusplus
}
#endif
#endif
