// Device helpers of the cubed-sphere shell shared by the render
// (ocr_shell.cu) and the adjoint (ocr_backward.cu): a leaf's geometry from the
// shared tables, the ray / leaf intersection, the field along a segment, and
// the values of a ray's sorted segments.
#pragma once
#include "ocr_common.h"
#include "ocr_device.cuh"

namespace ocr {
namespace {

// One leaf's geometry, float32: its tree frame, the tangents of its four
// planes and its two radii (read from the shared tables).
struct LeafShell {
  float n[3], e1[3], e2[3];
  float ta0, ta1, tb0, tb1;
  float rin, rout;
  int level;
};

__device__ __forceinline__ LeafShell leaf_shell(const Shell &S, int4 g) {
  LeafShell q;
  q.level = g.w & 255;
  const int tree = g.w >> 8, sz = 1 << (S.L - q.level);
  const float *fr = S.frames + 9 * tree;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    q.n[c] = __ldg(fr + c);
    q.e1[c] = __ldg(fr + 3 + c);
    q.e2[c] = __ldg(fr + 6 + c);
  }
  q.ta0 = __ldg(S.tan_tab + g.x);
  q.ta1 = __ldg(S.tan_tab + g.x + sz);
  q.tb0 = __ldg(S.tan_tab + g.y);
  q.tb1 = __ldg(S.tan_tab + g.y + sz);
  q.rin = __ldg(S.rad_tab + g.z);
  q.rout = __ldg(S.rad_tab + g.z + sz);
  return q;
}

__device__ __forceinline__ float dot3(const float *a, float3 b) {
  return fmaf(a[0], b.x, fmaf(a[1], b.y, a[2] * b.z));
}

// The normal m = e - T n of one of the leaf's four planes (s: xi low, xi
// high, eta low, eta high); the plane table holds exactly these values.
__device__ __forceinline__ float3 plane_normal(const LeafShell &q, int s) {
  const float *e = s < 2 ? q.e1 : q.e2;
  const float T = s == 0 ? q.ta0 : s == 1 ? q.ta1 : s == 2 ? q.tb0 : q.tb1;
  return make_float3(fmaf(-T, q.n[0], e[0]), fmaf(-T, q.n[1], e[1]), fmaf(-T, q.n[2], e[2]));
}

// Intervals of the ray o + alpha r inside the leaf, clipped to [amin, amax],
// nearest first; returns their number (0..2).  m: the normals of the leaf's
// four planes (xi low, xi high, eta low, eta high), r_in, r_out its radii.
// The cone: x . m >= 0 for the lower planes and <= 0 for the upper ones; each
// crossing is -(o . m) / (r . m) from m alone, so neighbours (whose shared
// plane has the same T, e, n, or at a tree boundary an exactly negated m)
// agree bit for bit.  The spheres: alpha = -b -+ sqrt((R^2 - |p|^2) / |r|^2),
// b = o.r / |r|^2, p = o - b r.
__device__ __forceinline__ int shell_ray_leaf_m(const float3 *m, float rin, float rout,
                                                float3 org, float3 dir, float amin, float amax,
                                                float *a_in, float *a_out) {
  // the canonical FP32 evaluation of the index decisions (ocr_device.cuh)
  float t0 = amin, t1 = amax;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const float g0 = fmaf(m[s].x, org.x, fmaf(m[s].y, org.y, __fmul_rn(m[s].z, org.z)));
    const float g1 = fmaf(m[s].x, dir.x, fmaf(m[s].y, dir.y, __fmul_rn(m[s].z, dir.z)));
    const bool upper = (s & 1) != 0;
    if (g1 == 0.f) {
      if ((upper ? -g0 : g0) < 0.f) return 0;  // parallel to the plane and outside
      continue;
    }
    const float a = __fdiv_rn(-g0, g1);
    if ((upper ? -g1 : g1) > 0.f)
      t0 = fmaxf(t0, a);
    else
      t1 = fminf(t1, a);
  }
  const float rr = fmaf(dir.x, dir.x, fmaf(dir.y, dir.y, __fmul_rn(dir.z, dir.z)));
  const float b = __fdiv_rn(fmaf(org.x, dir.x, fmaf(org.y, dir.y, __fmul_rn(org.z, dir.z))), rr);
  const float px = fmaf(-b, dir.x, org.x), py = fmaf(-b, dir.y, org.y), pz = fmaf(-b, dir.z, org.z);
  const float pp = fmaf(px, px, fmaf(py, py, __fmul_rn(pz, pz)));
  const float hout = fmaf(rout, rout, -pp);
  if (!(hout > 0.f)) return 0;
  const float so = __fsqrt_rn(__fdiv_rn(hout, rr));
  t0 = fmaxf(t0, __fsub_rn(-b, so));
  t1 = fminf(t1, __fadd_rn(-b, so));
  const float hin = fmaf(rin, rin, -pp);
  int n = 0;
  if (hin > 0.f) {
    const float si = __fsqrt_rn(__fdiv_rn(hin, rr));
    const float c0 = fminf(t1, __fsub_rn(-b, si)), c1 = fmaxf(t0, __fadd_rn(-b, si));
    if (c0 > t0) {
      a_in[n] = t0;
      a_out[n] = c0;
      ++n;
    }
    if (t1 > c1) {
      a_in[n] = c1;
      a_out[n] = t1;
      ++n;
    }
  } else if (t1 > t0) {
    a_in[0] = t0;
    a_out[0] = t1;
    n = 1;
  }
  return n;
}

// The same with the normals formed from the leaf's frame and tangents (the
// per-segment kernels, whose leaves change from lane to lane) ...
__device__ __forceinline__ int shell_ray_leaf(const LeafShell &q, float3 org, float3 dir,
                                              float amin, float amax, float *a_in, float *a_out) {
  float3 m[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) m[s] = plane_normal(q, s);
  return shell_ray_leaf_m(m, q.rin, q.rout, org, dir, amin, amax, a_in, a_out);
}

// ... or read from the per-leaf plane table, which holds the same values (the
// pair passes, where consecutive threads share a leaf).
__device__ __forceinline__ int shell_ray_leaf(const float4 *__restrict__ pl, float3 org,
                                              float3 dir, float amin, float amax, float *a_in,
                                              float *a_out) {
  float3 m[4];
  float w[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const float4 v = __ldg(pl + s);
    m[s] = make_float3(v.x, v.y, v.z);
    w[s] = v.w;
  }
  return shell_ray_leaf_m(m, w[0], w[1], org, dir, amin, amax, a_in, a_out);
}

// -------------------------------------------------------------- the field --
// The field along one segment, tau in [0, 1] from the far end to the near end:
// the point's coordinates in the tree frame (x.n, x.e1, x.e2) are affine in
// tau; the local coordinates follow from the inverse map,
//   u = (2/pi) (atan(x.e1 / x.n) - atan(ta)) / h
//     = (2/pi) atan2(x.e1 - ta x.n, x.n + ta x.e1) / h
// (for fine leaves the arctangent of the small ratio by its series),
//   w = (|x| - r_in) / (r_out - r_in),
// then the leaf's degree-2 tensor-product polynomial at (u, v, w).  The
// kernels hold that polynomial in monomial form (shell_monomials converts the
// 27 Lagrange nodal values once per render): cf[9 k + 3 j + i] multiplies
// u^i v^j w^k, evaluated by nested Horner steps.
struct ShellSeg {
  float pf[3], dp[3];
  float ta, tb, ka, rin, kr;
  int series;  // leaf level >= kSeriesLevel: the angles by atan_small
  float cf[27];
};

// Leaves of level >= kSeriesLevel span at most (pi/2) 2^-3 = pi/16 in each
// angle, so the tangent of a point's angle from the leaf's lower plane stays
// below tan(pi/16) = 0.199 (a little more for rounding at the faces).
constexpr int kSeriesLevel = 3;

// arctan(z) for |z| <= 0.2 by its Maclaurin series z - z^3/3 + z^5/5 - ... up
// to z^11: the first omitted term, z^13/13, is below 3e-10 of z there.
__device__ __forceinline__ float atan_small(float z) {
  const float t = z * z;
  float p = fmaf(t, -1.f / 11.f, 1.f / 9.f);
  p = fmaf(p, t, -1.f / 7.f);
  p = fmaf(p, t, 1.f / 5.f);
  p = fmaf(p, t, -1.f / 3.f);
  p = fmaf(p, t, 1.f);
  return z * p;
}

// Lagrange basis of degree 2 on the nodes 0, 1/2, 1 (the adjoint's weights).
__device__ __forceinline__ void quad_basis(float t, float *l) {
  l[0] = 2.f * (t - 0.5f) * (t - 1.f);
  l[1] = -4.f * t * (t - 1.f);
  l[2] = 2.f * t * (t - 0.5f);
}

// The field value at tau and the local coordinates (u, v, w) there.
__device__ __forceinline__ float shell_field(const ShellSeg &g, float tau, float &u, float &v,
                                             float &w) {
  const float pn = fmaf(tau, g.dp[0], g.pf[0]), p1 = fmaf(tau, g.dp[1], g.pf[1]),
              p2 = fmaf(tau, g.dp[2], g.pf[2]);
  const float ya = fmaf(-g.ta, pn, p1), xa = fmaf(g.ta, p1, pn);
  const float yb = fmaf(-g.tb, pn, p2), xb = fmaf(g.tb, p2, pn);
  if (g.series) {
    u = atan_small(ya / xa) * g.ka;
    v = atan_small(yb / xb) * g.ka;
  } else {
    u = atan2f(ya, xa) * g.ka;
    v = atan2f(yb, xb) * g.ka;
  }
  w = (sqrtf(fmaf(pn, pn, fmaf(p1, p1, p2 * p2))) - g.rin) * g.kr;
  float q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float r[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float *c = g.cf + 9 * k + 3 * j;
      r[j] = fmaf(fmaf(c[2], u, c[1]), u, c[0]);
    }
    q[k] = fmaf(fmaf(r[2], v, r[1]), v, r[0]);
  }
  return fmaf(fmaf(q[2], w, q[1]), w, q[0]);
}

__device__ __forceinline__ float4 medium(const ShellSeg &g, const TF &tf, float tau) {
  float u, v, w;
  return tf_lookup(tf, shell_field(g, tau, u, v, w));
}

// ------------------------------------------------------------ surfaces --
// The piece [ta, ta + L] of a segment's parameter, rescaled to [0, 1].
struct ShellSub {
  const ShellSeg *g;
  float ta, L;
};

__device__ __forceinline__ float4 medium(const ShellSub &s, const TF &tf, float tau) {
  return medium(*s.g, tf, fmaf(tau, s.L, s.ta));
}

// cos phi between the segment and the field's gradient at tau (Sec. 2.8, the
// surface normal of Eq. 2.35).  In the tree frame (components along n, e1,
// e2, where p = (pn, p1, p2)): the local coordinates change with p as
//   du/dp = ka (-p1, pn, 0) / (pn^2 + p1^2),  dv/dp = ka (-p2, 0, pn) / (pn^2 + p2^2),
//   dw/dp = kr p / |p|,
// and the polynomial's derivatives in (u, v, w) come from its monomial form.
// The frame is orthonormal, so the angle is the one in space.
__device__ __forceinline__ float shell_cos_phi(const ShellSeg &g, float tau) {
  float u, v, w;
  shell_field(g, tau, u, v, w);
  float Q[3], Qu[3], Qv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float R[3], Ru[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float *c = g.cf + 9 * k + 3 * j;
      R[j] = fmaf(fmaf(c[2], u, c[1]), u, c[0]);
      Ru[j] = fmaf(2.f * c[2], u, c[1]);
    }
    Q[k] = fmaf(fmaf(R[2], v, R[1]), v, R[0]);
    Qu[k] = fmaf(fmaf(Ru[2], v, Ru[1]), v, Ru[0]);
    Qv[k] = fmaf(2.f * R[2], v, R[1]);
  }
  const float Pu = fmaf(fmaf(Qu[2], w, Qu[1]), w, Qu[0]);
  const float Pv = fmaf(fmaf(Qv[2], w, Qv[1]), w, Qv[0]);
  const float Pw = fmaf(2.f * Q[2], w, Q[1]);
  const float pn = fmaf(tau, g.dp[0], g.pf[0]), p1 = fmaf(tau, g.dp[1], g.pf[1]),
              p2 = fmaf(tau, g.dp[2], g.pf[2]);
  const float a = Pu * g.ka / fmaf(pn, pn, p1 * p1), b = Pv * g.ka / fmaf(pn, pn, p2 * p2);
  const float c = Pw * g.kr / sqrtf(fmaf(pn, pn, fmaf(p1, p1, p2 * p2)));
  const float gx = fmaf(-a, p1, fmaf(-b, p2, c * pn)), gy = fmaf(a, pn, c * p1),
              gz = fmaf(b, pn, c * p2);
  const float gn2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
  const float dn2 = fmaf(g.dp[0], g.dp[0], fmaf(g.dp[1], g.dp[1], g.dp[2] * g.dp[2]));
  const float dot = fmaf(gx, g.dp[0], fmaf(gy, g.dp[1], gz * g.dp[2]));
  return gn2 > 0.f && dn2 > 0.f ? fabsf(dot) / sqrtf(gn2 * dn2) : 1.f;
}

// Sec. 2.8 on the isosurface s = s_iso of a shell segment, as for the cube:
// sign changes of s - s_iso between 9 equally spaced samples (far end to near
// end), each located by 24 bisection steps; the segment is cut there and the
// surface segment A = a_s^(1 / cos phi), B = i_s (1 - A) (Eqs. 2.18, 2.35)
// goes between the pieces.
__device__ float4 shell_iso_split(const ShellSeg &g, const TF &tf, float dx, const Integ &I,
                                  int &steps) {
  float4 acc = seg_identity();
  float t1 = 0.f, u, v, w;
  float gp = shell_field(g, 0.f, u, v, w) - I.s_iso;
  for (int k = 0; k < 8; ++k) {
    const float tk1 = (float)(k + 1) * 0.125f;
    const float gn = shell_field(g, tk1, u, v, w) - I.s_iso;
    if ((gp < 0.f && gn > 0.f) || (gp > 0.f && gn < 0.f)) {
      float lo = (float)k * 0.125f, hi = tk1, glo = gp;
      for (int it = 0; it < 24; ++it) {
        const float mid = 0.5f * (lo + hi), gm = shell_field(g, mid, u, v, w) - I.s_iso;
        if ((gm < 0.f) == (glo < 0.f)) {
          lo = mid;
          glo = gm;
        } else {
          hi = mid;
        }
      }
      const float tc = 0.5f * (lo + hi);
      acc = seg_combine(integrate_segment(ShellSub{&g, t1, tc - t1}, tf, dx * (tc - t1), I, steps),
                        acc);
      const float cphi = shell_cos_phi(g, tc);
      const float A = I.a_s >= 1.f ? 1.f
                      : (I.a_s <= 0.f || cphi <= 0.f) ? 0.f
                                                      : exp2f(log2f(I.a_s) / cphi);
      const float om = 1.f - A;
      acc = seg_combine(make_float4(A, I.i_s[0] * om, I.i_s[1] * om, I.i_s[2] * om), acc);
      t1 = tc;
    }
    gp = gn;
  }
  return seg_combine(integrate_segment(ShellSub{&g, t1, 1.f - t1}, tf, dx * (1.f - t1), I, steps),
                     acc);
}

// The segment of the ray inside one leaf (the piece-th of its intervals):
// its field (coef: the monomial coefficients of every leaf), its world length,
// and the interval itself.  Returns false if the
// ray does not have that piece.
__device__ __forceinline__ bool shell_segment(const Shell &S, const float *__restrict__ coef,
                                              const Cam &c, int4 geo, int leaf, int piece,
                                              float3 org, float3 dir, float rl, ShellSeg &g,
                                              float &dx, float2 &iv) {
  const LeafShell q = leaf_shell(S, geo);
  float ai[2], ao[2];
  if (shell_ray_leaf(q, org, dir, c.amin, c.amax, ai, ao) <= piece) return false;
  const float a_in = ai[piece], a_out = ao[piece];
  const float3 pf = make_float3(fmaf(a_out, dir.x, org.x), fmaf(a_out, dir.y, org.y),
                                fmaf(a_out, dir.z, org.z));
  const float da = a_in - a_out;
  const float3 dv = make_float3(da * dir.x, da * dir.y, da * dir.z);
  g.pf[0] = dot3(q.n, pf);
  g.pf[1] = dot3(q.e1, pf);
  g.pf[2] = dot3(q.e2, pf);
  g.dp[0] = dot3(q.n, dv);
  g.dp[1] = dot3(q.e1, dv);
  g.dp[2] = dot3(q.e2, dv);
  g.ta = q.ta0;
  g.tb = q.tb0;
  g.ka = ldexpf(0.63661977236758134f, q.level);  // (2 / pi) / h
  g.series = q.level >= kSeriesLevel;
  g.rin = q.rin;
  g.kr = 1.f / (q.rout - q.rin);
  const float *cf = coef + 27 * (size_t)leaf;
#pragma unroll
  for (int a = 0; a < 27; ++a) g.cf[a] = __ldg(cf + a);
  dx = (a_out - a_in) * rl;
  iv = make_float2(a_in, a_out);
  return true;
}

// The values of the n segments of one ray, one warp: key[0..n) the ray's
// sorted list, val[k] the k-th segment (A, B) and, when iv is given, its
// interval (iv may alias key: entry k is read before it is written).  With
// Dormand-Prince inside Algorithm 1 every lane advances its segment one step at
// a time and takes the ray's next segment as soon as it is done, so the lanes
// stay busy while some of them bisect.  Returns this lane's count of entries
// that are not a segment of the ray (unwritten entries, missing pieces).
// SURF: the isosurface of Sec. 2.8 is rendered inside the segments.
template <bool SURF = false>
__device__ __forceinline__ int shell_ray_values(const int4 *__restrict__ geo, int N,
                                                const Shell &S, const float *__restrict__ nodal,
                                                const Cam &c, const Integ &I, const TF &tf,
                                                const unsigned long long *key, int n,
                                                float3 org, float3 dir, float rl, float4 *val,
                                                float2 *iv, int lane, int &steps) {
  int errs = 0;
  if (I.method == 1 && !SURF) {
    int next = 0, k = 0, depth = 0;
    unsigned idx = 0;
    bool busy = false;
    ShellSeg g;
    float dx = 0.f;
    float2 ivk = make_float2(0.f, 0.f);
    float4 kq0 = seg_identity(), sacc = seg_identity();
    for (;;) {
      const unsigned idle = __ballot_sync(0xffffffffu, !busy);
      const int kk = next + __popc(idle & ((1u << lane) - 1u));
      next += __popc(idle);
      if (!busy && kk < n) {
        k = kk;
        const unsigned lp = (unsigned)(key[k] & 0xffffffffu);
        const int leaf = (int)(lp >> 1), piece = (int)(lp & 1u);
        if (leaf >= N || !shell_segment(S, nodal, c, __ldg(geo + leaf), leaf, piece, org, dir,
                                        rl, g, dx, ivk)) {
          ++errs;
          val[k] = seg_identity();
          if (iv) iv[k] = make_float2(0.f, 0.f);
        } else {
          busy = true;
          depth = 0;
          idx = 0;
          sacc = seg_identity();
          kq0 = medium(g, tf, 0.f);
        }
      }
      if (!__any_sync(0xffffffffu, busy)) {
        if (next >= n) break;
        continue;
      }
      if (busy && dopri_advance(g, tf, dx, I, depth, idx, kq0, sacc, steps)) {
        val[k] = sacc;
        if (iv) iv[k] = ivk;
        busy = false;
      }
    }
  } else {
    for (int k = lane; k < n; k += 32) {
      const unsigned lp = (unsigned)(key[k] & 0xffffffffu);
      const int leaf = (int)(lp >> 1), piece = (int)(lp & 1u);
      ShellSeg g;
      float dx;
      float2 ivk;
      if (leaf >= N ||
          !shell_segment(S, nodal, c, __ldg(geo + leaf), leaf, piece, org, dir, rl, g, dx, ivk)) {
        ++errs;
        val[k] = seg_identity();
        if (iv) iv[k] = make_float2(0.f, 0.f);
        continue;
      }
      val[k] = SURF ? shell_iso_split(g, tf, dx, I, steps) : integrate_segment(g, tf, dx, I, steps);
      if (iv) iv[k] = ivk;
    }
  }
  return errs;
}

}  // namespace
}  // namespace ocr
