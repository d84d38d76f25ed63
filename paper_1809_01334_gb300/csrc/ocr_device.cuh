// Device helpers shared by the render kernels (ocr_kernels.cu) and the
// adjoint (ocr_backward.cu): camera rays, slab test, the field along a
// segment, the transfer function, the integrators and the pixel rectangle.
#pragma once
#include "ocr_common.h"

namespace ocr {
namespace {

constexpr float kOne = 1.0f;

// Ascending bitonic sort of P = 32 E keys (E <= 16) held by one warp in
// registers, blocked: lane l holds the keys of indices l E + j (j < E).
// Stages whose partner index differs in a bit below E compare two of a lane's
// own registers; the others swap with lane l ^ (st / E) by shuffles.  With
// PAY the int payload p moves along.  The stage loops stay loops (small
// code); only the loops over a lane's E registers are unrolled.
template <int E, int JS, bool PAY>
__device__ __forceinline__ void bitonic_in_lane(unsigned long long (&k)[E], int (&p)[E], int sz,
                                                int lane) {
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int jp = j ^ JS;
    if (jp > j && jp < E) {
      const bool up = ((lane * E + j) & sz) == 0;
      if ((k[j] > k[jp]) == up) {
        const unsigned long long t = k[j];
        k[j] = k[jp];
        k[jp] = t;
        if (PAY) {
          const int u = p[j];
          p[j] = p[jp];
          p[jp] = u;
        }
      }
    }
  }
}

template <int E, bool PAY>
__device__ __forceinline__ void warp_bitonic_regs(unsigned long long (&k)[E], int (&p)[E],
                                                  int lane) {
  static_assert(E == 1 || E == 2 || E == 4 || E == 8 || E == 16, "E: 1 to 16 keys per lane");
#pragma unroll 1
  for (int sz = 2; sz <= 32 * E; sz <<= 1) {
#pragma unroll 1
    for (int st = sz >> 1; st > 0; st >>= 1) {
      if (st < E) {
        if (st == 8) bitonic_in_lane<E, 8, PAY>(k, p, sz, lane);
        else if (st == 4) bitonic_in_lane<E, 4, PAY>(k, p, sz, lane);
        else if (st == 2) bitonic_in_lane<E, 2, PAY>(k, p, sz, lane);
        else bitonic_in_lane<E, 1, PAY>(k, p, sz, lane);
      } else {
        // sz >= 2 E here, so the direction is the same for all of a lane's
        // registers; keys are distinct (padding aside, which may swap with
        // itself), so "take the partner's key" is (o < k) == keep_min
        const int ls = st / E;
        const bool keep_min = ((lane & ls) == 0) == (((lane * E) & sz) == 0);
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, k[j], ls);
          const int op = PAY ? __shfl_xor_sync(0xffffffffu, p[j], ls) : 0;
          if ((o < k[j]) == keep_min) {
            k[j] = o;
            if (PAY) p[j] = op;
          }
        }
      }
    }
  }
}

// Loads the n <= 32 E keys src[0..n) (padded with ~0), sorts them in
// registers and stores the first nst of them in order to dst (shared or
// global memory); with PAY also the payloads (psrc, padded with -1) to pdst.
template <int E, bool PAY>
__device__ __forceinline__ void warp_sort_list(const unsigned long long *__restrict__ src,
                                               const unsigned *__restrict__ psrc, int n,
                                               unsigned long long *dst, int *pdst, int nst,
                                               int lane) {
  unsigned long long k[E];
  int p[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    k[j] = i < n ? src[i] : ~0ull;
    p[j] = (PAY && i < n) ? (int)psrc[i] : -1;
  }
  warp_bitonic_regs<E, PAY>(k, p, lane);
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    if (i < nst) {
      dst[i] = k[j];
      if (PAY) pdst[i] = p[j];
    }
  }
  __syncwarp();
}

// 2^e for an integer e in [-126, 127]: the biased exponent written directly
// (exact, like ldexpf(1, e), without its range handling).
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ float4 seg_identity() { return make_float4(1.f, 0.f, 0.f, 0.f); }

// Eq. 2.14: (A2, B2) (+) (A1, B1) = (A2 A1, B2 + A2 B1), n = nearer, f = farther.
__device__ __forceinline__ float4 seg_combine(float4 n, float4 f) {
  return make_float4(n.x * f.x, fmaf(n.x, f.y, n.y), fmaf(n.x, f.z, n.z), fmaf(n.x, f.w, n.w));
}

// ------------------------------------------------- index decisions (FP32) --
// Which leaves a camera sees, which (leaf, ray) pairs give segments and where
// those segments end are decided by the floating-point code below (pixel_ray,
// slab, box_rect / project_box, and the shell's intersection and culling in
// ocr_shell.cuh / ocr_shell.cu).  It is written in one canonical FP32
// evaluation: every operation rounded to nearest once (the _rn intrinsics,
// which the compiler neither fuses nor approximates under fast math), in the
// order written, a fused multiply-add exactly where fmaf is written.  The
// oracle takes these decisions with the same evaluation, so index results
// (visible leaves, rectangles, per-ray segment counts) agree bit for bit.

__device__ __forceinline__ void pixel_ray(const Cam &c, int i, int j, float3 &org, float3 &dir) {
  const float di = __fsub_rn((float)i, c.cw), dj = __fsub_rn((float)j, c.ch);
  const float ox = fmaf(dj, c.lu[0], __fmul_rn(di, c.lt[0]));
  const float oy = fmaf(dj, c.lu[1], __fmul_rn(di, c.lt[1]));
  const float oz = fmaf(dj, c.lu[2], __fmul_rn(di, c.lt[2]));
  if (c.ortho) {
    org = make_float3(__fadd_rn(c.o[0], ox), __fadd_rn(c.o[1], oy), __fadd_rn(c.o[2], oz));
    dir = make_float3(c.v[0], c.v[1], c.v[2]);
  } else {
    org = make_float3(c.o[0], c.o[1], c.o[2]);
    dir = make_float3(__fadd_rn(c.v[0], ox), __fadd_rn(c.v[1], oy), __fadd_rn(c.v[2], oz));
  }
}

// 1/d rounded to nearest (IEEE), 0 for d == 0
__device__ __forceinline__ float recip_or_zero(float d) { return d != 0.f ? __frcp_rn(d) : 0.f; }

// Slab test of the ray against the axis-aligned box [lo, lo + h]^3, clipped to
// [amin, amax].  A zero direction component keeps the ray inside the slab or
// misses it entirely.
__device__ __forceinline__ bool slab(float3 org, float3 dir, float3 inv, float3 lo, float h,
                                     float amin, float amax, float &a_in, float &a_out) {
  float t0 = amin, t1 = amax;
  const float o[3] = {org.x, org.y, org.z}, d[3] = {dir.x, dir.y, dir.z};
  const float iv[3] = {inv.x, inv.y, inv.z}, l[3] = {lo.x, lo.y, lo.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float b0 = l[a], b1 = __fadd_rn(l[a], h);
    if (d[a] == 0.f) {
      if (o[a] < b0 || o[a] > b1) return false;
    } else {
      const float s0 = __fmul_rn(__fsub_rn(b0, o[a]), iv[a]);
      const float s1 = __fmul_rn(__fsub_rn(b1, o[a]), iv[a]);
      t0 = fmaxf(t0, fminf(s0, s1));
      t1 = fminf(t1, fmaxf(s0, s1));
    }
  }
  a_in = t0;
  a_out = t1;
  return t1 > t0;
}

__device__ __forceinline__ float3 node_lo(int4 g, float scale) {
  return make_float3((float)g.x * scale, (float)g.y * scale, (float)g.z * scale);
}

// ------------------------------------------------------------------ medium --
// The trilinear field along a straight segment is a cubic in the segment
// parameter tau (tau = 0 at the far end, 1 at the near end): its four
// coefficients are formed once per segment and each evaluation is three FMAs.
struct Cubic {
  float p0, p1, p2, p3;
};

__device__ __forceinline__ Cubic field_cubic(const float *__restrict__ nd, float3 a, float3 d) {
  const float4 lo = __ldg(reinterpret_cast<const float4 *>(nd));
  const float4 hi = __ldg(reinterpret_cast<const float4 *>(nd) + 1);
  const float n0 = lo.x, n1 = lo.y, n2 = lo.z, n3 = lo.w, n4 = hi.x, n5 = hi.y, n6 = hi.z,
              n7 = hi.w;
  // monomial form of the trilinear interpolant in (U, V, W)
  const float c0 = n0, cu = n1 - n0, cv = n2 - n0, cw = n4 - n0;
  const float cuv = (n3 - n2) - (n1 - n0), cuw = (n5 - n4) - (n1 - n0),
              cvw = (n6 - n4) - (n2 - n0);
  const float cuvw = ((n7 - n6) - (n5 - n4)) - ((n3 - n2) - (n1 - n0));
  // substitute U = a.x + tau d.x, V = a.y + tau d.y, W = a.z + tau d.z
  Cubic c;
  const float ab = a.x * a.y, ac = a.x * a.z, bc = a.y * a.z;
  c.p0 = c0 + cu * a.x + cv * a.y + cw * a.z + cuv * ab + cuw * ac + cvw * bc + cuvw * ab * a.z;
  c.p1 = cu * d.x + cv * d.y + cw * d.z + cuv * (a.x * d.y + a.y * d.x) +
         cuw * (a.x * d.z + a.z * d.x) + cvw * (a.y * d.z + a.z * d.y) +
         cuvw * (ab * d.z + ac * d.y + bc * d.x);
  c.p2 = cuv * d.x * d.y + cuw * d.x * d.z + cvw * d.y * d.z +
         cuvw * (a.x * d.y * d.z + a.y * d.x * d.z + a.z * d.x * d.y);
  c.p3 = cuvw * d.x * d.y * d.z;
  return c;
}

struct TF {
  const float4 *v, *s;  // knot values and slopes (shared memory)
  float s_min, inv;
};

// (kappa, q_r, q_g, q_b) of the field value s: piecewise-linear transfer
// function, constant outside the knot range.
__device__ __forceinline__ float4 tf_lookup(const TF &tf, float s) {
  float z = (s - tf.s_min) * tf.inv;
  z = fminf(fmaxf(z, 0.f), 7.f);
  const int k = min((int)z, 6);
  const float w = z - (float)k;
  const float4 a = tf.v[k], d = tf.s[k];
  return make_float4(fmaf(w, d.x, a.x), fmaf(w, d.y, a.y), fmaf(w, d.z, a.z), fmaf(w, d.w, a.w));
}

__device__ __forceinline__ float cubic_at(const Cubic &c, float tau) {
  return fmaf(fmaf(fmaf(c.p3, tau, c.p2), tau, c.p1), tau, c.p0);
}

// The medium at parameter tau of a segment through a cube leaf.
__device__ __forceinline__ float4 medium(const Cubic &c, const TF &tf, float tau) {
  return tf_lookup(tf, fmaf(fmaf(fmaf(c.p3, tau, c.p2), tau, c.p1), tau, c.p0));
}

// Right-hand side of Eq. 2.29 for the state Y = (A, B_r, B_g, B_b).
__device__ __forceinline__ float4 rhs(float4 kq, float4 Y) {
  return make_float4(-kq.x * Y.x, fmaf(-kq.x, Y.y, kq.y), fmaf(-kq.x, Y.z, kq.z),
                     fmaf(-kq.x, Y.w, kq.w));
}

__device__ __forceinline__ float4 axpy(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Classical RK4 from (1, 0) over one step of length H with the medium at the
// step's far end (k0), midpoint (kh) and near end (k1).
__device__ __forceinline__ float4 rk4_step(float H, float4 k0, float4 kh, float4 k1) {
  const float4 one = seg_identity();
  const float4 K1 = rhs(k0, one);
  const float4 K2 = rhs(kh, axpy(0.5f * H, K1, one));
  const float4 K3 = rhs(kh, axpy(0.5f * H, K2, one));
  const float4 K4 = rhs(k1, axpy(H, K3, one));
  float4 s = axpy(2.f, K2, K1);
  s = axpy(2.f, K3, s);
  s.x += K4.x; s.y += K4.y; s.z += K4.z; s.w += K4.w;
  return axpy(H * (1.f / 6.f), s, one);
}

// Dormand & Prince (1980) 5(4) tableau.
namespace dp {
constexpr float c2 = 1.f / 5, c3 = 3.f / 10, c4 = 4.f / 5, c5 = 8.f / 9;
constexpr float a21 = 1.f / 5;
constexpr float a31 = 3.f / 40, a32 = 9.f / 40;
constexpr float a41 = 44.f / 45, a42 = -56.f / 15, a43 = 32.f / 9;
constexpr float a51 = 19372.f / 6561, a52 = -25360.f / 2187, a53 = 64448.f / 6561,
                a54 = -212.f / 729;
constexpr float a61 = 9017.f / 3168, a62 = -355.f / 33, a63 = 46732.f / 5247, a64 = 49.f / 176,
                a65 = -5103.f / 18656;
constexpr float b1 = 35.f / 384, b3 = 500.f / 1113, b4 = 125.f / 192, b5 = -2187.f / 6784,
                b6 = 11.f / 84;
// e = b - b* (fifth- minus fourth-order weights), seventh stage at the end point
constexpr float e1 = 71.f / 57600, e3 = -71.f / 16695, e4 = 71.f / 1920, e5 = -17253.f / 339200,
                e6 = 22.f / 525, e7 = -1.f / 40;
}  // namespace dp

__device__ __forceinline__ float4 lin4(float a, float4 x, float b, float4 y) {
  return make_float4(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z),
                     fmaf(a, x.w, b * y.w));
}

// One Dormand-Prince 5(4) step from (1, 0) over the dyadic interval
// [idx, idx + 1] 2^-depth of tau (kq0: the medium at its far end): the
// fifth-order value Y5, the medium at the near end kq6, the embedded error and
// the largest H kappa at the nodes (the split tests of Algorithm 1).
template <class Fld>
__device__ __forceinline__ void dopri_eval(const Fld &cu, const TF &tf, float dx, int depth,
                                           unsigned idx, float4 kq0, float4 &Y5, float4 &kq6,
                                           float &err, float &hkmax) {
  const float4 one = seg_identity();
  const float dtau = exp2i(-depth);
  const float t0 = (float)idx * dtau;
  const float H = dx * dtau;
  const float4 kq2 = medium(cu, tf, fmaf(dp::c2, dtau, t0));
  const float4 kq3 = medium(cu, tf, fmaf(dp::c3, dtau, t0));
  const float4 kq4 = medium(cu, tf, fmaf(dp::c4, dtau, t0));
  const float4 kq5 = medium(cu, tf, fmaf(dp::c5, dtau, t0));
  kq6 = medium(cu, tf, t0 + dtau);
  const float4 K1 = rhs(kq0, one);
  const float4 K2 = rhs(kq2, axpy(H * dp::a21, K1, one));
  const float4 K3 = rhs(kq3, axpy(H, lin4(dp::a31, K1, dp::a32, K2), one));
  float4 t = lin4(dp::a41, K1, dp::a42, K2);
  t = axpy(dp::a43, K3, t);
  const float4 K4 = rhs(kq4, axpy(H, t, one));
  t = lin4(dp::a51, K1, dp::a52, K2);
  t = axpy(dp::a53, K3, t);
  t = axpy(dp::a54, K4, t);
  const float4 K5 = rhs(kq5, axpy(H, t, one));
  t = lin4(dp::a61, K1, dp::a62, K2);
  t = axpy(dp::a63, K3, t);
  t = axpy(dp::a64, K4, t);
  t = axpy(dp::a65, K5, t);
  const float4 K6 = rhs(kq6, axpy(H, t, one));
  t = lin4(dp::b1, K1, dp::b3, K3);
  t = axpy(dp::b4, K4, t);
  t = axpy(dp::b5, K5, t);
  t = axpy(dp::b6, K6, t);
  Y5 = axpy(H, t, one);
  const float4 K7 = rhs(kq6, Y5);
  float4 e = lin4(dp::e1, K1, dp::e3, K3);
  e = axpy(dp::e4, K4, e);
  e = axpy(dp::e5, K5, e);
  e = axpy(dp::e6, K6, e);
  e = axpy(dp::e7, K7, e);
  err = H * fmaxf(fmaxf(fabsf(e.x), fabsf(e.y)), fmaxf(fabsf(e.z), fabsf(e.w)));
  hkmax = H * fmaxf(fmaxf(fmaxf(kq0.x, kq2.x), fmaxf(kq3.x, kq4.x)), fmaxf(kq5.x, kq6.x));
}

// Algorithm 1's bisection with Dormand-Prince steps, one step per call, walked
// far half first: the step at (depth, idx) is taken; if the split test fails
// it is replaced by its halves (depth + 1), else its value is combined behind
// acc (Eq. 2.14) and the walk moves on.  Returns true when the segment is done.
template <class Fld>
__device__ __forceinline__ bool dopri_advance(const Fld &cu, const TF &tf, float dx,
                                              const Integ &I, int &depth, unsigned &idx,
                                              float4 &kq0, float4 &acc, int &steps) {
  float4 Y5, kq6;
  float err, hkmax;
  dopri_eval(cu, tf, dx, depth, idx, kq0, Y5, kq6, err, hkmax);
  ++steps;
  if (depth < I.max_depth && (hkmax > I.c_rk || err > I.tol)) {
    ++depth;  // far half first; it starts where this step started
    idx <<= 1;
    return false;
  }
  acc = seg_combine(Y5, acc);
  kq0 = kq6;
  ++idx;
  while (depth > 0 && !(idx & 1u)) {
    idx >>= 1;
    --depth;
  }
  return depth == 0;
}

// (A, B) of one segment of world length dx: RK4 x nsteps, or DOPRI5 inside
// the midpoint bisection of Algorithm 1, walked far half first so that each
// accepted piece is nearer than everything accumulated so far.
template <class Fld>
__device__ float4 integrate_segment(const Fld &cu, const TF &tf, float dx, const Integ &I,
                                    int &steps) {
  float4 acc = seg_identity();
  if (I.method == 0) {
    const int n = I.nsteps;
    const float H = dx / (float)n, dt = 1.f / (float)n;
    float4 k0 = medium(cu, tf, 0.f);
    for (int s = 0; s < n; ++s) {
      const float t0 = (float)s * dt;
      const float4 kh = medium(cu, tf, t0 + 0.5f * dt);
      const float4 k1 = medium(cu, tf, (s + 1 == n) ? 1.f : t0 + dt);
      acc = seg_combine(rk4_step(H, k0, kh, k1), acc);
      k0 = k1;
    }
    steps += n;
    return acc;
  }
  int depth = 0;
  unsigned idx = 0;
  float4 kq0 = medium(cu, tf, 0.f);
  const float4 one = seg_identity();
  if (I.method != 1) {  // Gauss-2 (Eqs. 2.32-2.33), Simpson (Eq. 2.34) or Eq. 2.18, Algorithm 1
    for (;;) {
      const float dtau = exp2i(-depth);
      const float t0 = (float)idx * dtau;
      const float H = dx * dtau;
      float4 S, kq1 = kq0;
      float kmax;
      if (I.method == 2) {
        // Gauss points c = 1/2 -+ sqrt(3)/6, measured from the step's far end
        const float4 g0 = medium(cu, tf, fmaf(0.21132486540518713f, dtau, t0));
        const float4 g1 = medium(cu, tf, fmaf(0.78867513459481287f, dtau, t0));
        const float a1 = 0.25f * H * (g0.x + g1.x), a2 = (H * H / 12.f) * g0.x * g1.x;
        const float inv = 1.f / (1.f + a1 + a2);
        const float h2 = H * H * 0.14433756729740644f;  // H^2 sqrt(3) / 12
        S.x = (1.f - a1 + a2) * inv;
        S.y = (0.5f * H * (g0.y + g1.y) + h2 * (g0.x * g1.y - g1.x * g0.y)) * inv;
        S.z = (0.5f * H * (g0.z + g1.z) + h2 * (g0.x * g1.z - g1.x * g0.z)) * inv;
        S.w = (0.5f * H * (g0.w + g1.w) + h2 * (g0.x * g1.w - g1.x * g0.w)) * inv;
        kmax = H * fmaxf(g0.x, g1.x);
      } else if (I.method == 4) {
        // Eq. 2.18 as an interface: the colour channels are the intensity I;
        // A from Simpson's rule on the optical depth, B = I_mid (1 - A)
        const float4 kh = medium(cu, tf, t0 + 0.5f * dtau);
        kq1 = medium(cu, tf, t0 + dtau);
        const float e = -(H / 6.f) * (kq0.x + 4.f * kh.x + kq1.x);
        const float om = -expm1f(e);
        S = make_float4(1.f - om, kh.y * om, kh.z * om, kh.w * om);
        kmax = H * fmaxf(fmaxf(kq0.x, kh.x), kq1.x);
      } else {
        // Simpson nodes: far end, midpoint, near end
        const float4 kh = medium(cu, tf, t0 + 0.5f * dtau);
        kq1 = medium(cu, tf, t0 + dtau);
        const float e = -(H / 6.f) * (kq0.x + 4.f * kh.x + kq1.x);
        const float sa = __expf(0.5f * e), A = sa * sa;
        const float w0 = (H / 6.f) * A, wh = (H / 6.f) * 4.f * sa, w1 = H / 6.f;
        S = make_float4(A, fmaf(w0, kq0.y, fmaf(wh, kh.y, w1 * kq1.y)),
                        fmaf(w0, kq0.z, fmaf(wh, kh.z, w1 * kq1.z)),
                        fmaf(w0, kq0.w, fmaf(wh, kh.w, w1 * kq1.w)));
        kmax = H * fmaxf(fmaxf(kq0.x, kh.x), kq1.x);
      }
      ++steps;
      if (depth < I.max_depth && kmax > I.c_rk) {
        ++depth;  // far half first
        idx <<= 1;
        continue;
      }
      acc = seg_combine(S, acc);
      kq0 = kq1;  // Simpson: the next step starts where this one ended (unused by Gauss)
      ++idx;
      while (depth > 0 && !(idx & 1u)) {
        idx >>= 1;
        --depth;
      }
      if (depth == 0) break;
    }
    return acc;
  }
  for (;;) {
    float4 Y5, kq6;
    float err, hkmax;
    dopri_eval(cu, tf, dx, depth, idx, kq0, Y5, kq6, err, hkmax);
    ++steps;
    if (depth < I.max_depth && (hkmax > I.c_rk || err > I.tol)) {
      ++depth;  // far half first; it starts where this step started
      idx <<= 1;
      continue;
    }
    acc = seg_combine(Y5, acc);
    kq0 = kq6;
    ++idx;
    while (depth > 0 && !(idx & 1u)) {
      idx >>= 1;
      --depth;
    }
    if (depth == 0) break;
  }
  return acc;
}

// ----------------------------------------------------------------- culling --
__device__ __forceinline__ int4 empty_rect() { return make_int4(0, -1, 0, -1); }

// The order of a rectangle's (node, ray) slots: the rectangle is cut into
// bands of 4 rows and a band's slots go column by column, 4 to a column (the
// last band's height to a column), so that 32 consecutive slots cover an 8 x 4
// block of pixels, whose rays are closer to one another than a row's.
// slot_pixel: the pixel of the local-th slot; slot_of_pixel: the inverse.
__device__ __forceinline__ void slot_pixel(int4 r, unsigned local, int &i, int &j) {
  const unsigned w = (unsigned)(r.y - r.x + 1), h = (unsigned)(r.w - r.z + 1);
  const unsigned band = local / (4u * w);  // 4 w h < 2^32 for rectangles of the image
  const unsigned rem = local - band * 4u * w;
  const unsigned hb = min(4u, h - 4u * band);
  const unsigned col = hb == 4u ? rem >> 2 : rem / hb;
  i = r.x + (int)col;
  j = r.z + (int)(4u * band + rem - col * hb);
}

__device__ __forceinline__ long long slot_of_pixel(int4 r, int i, int j) {
  const unsigned w = (unsigned)(r.y - r.x + 1), h = (unsigned)(r.w - r.z + 1);
  const unsigned dj = (unsigned)(j - r.z), band = dj >> 2;
  const unsigned hb = min(4u, h - 4u * band);
  return (long long)(4u * w) * band + (long long)(i - r.x) * hb + (dj & 3u);
}

// Pixel rectangle of the camera-space bounding box of the cube [lo, lo+h]^3:
// the box is mapped by X = (t, u, v/n)^T (x - o) (an affine map, so its AABB is
// centre +- half-extent), clipped to the visible depth range, and projected.
// Pixel rectangle of the camera-space box [blo, bhi]: clipped to the visible
// depth range, its corners projected, the pixel centres inside kept.
__device__ int4 project_box(const Cam &c, const float *blo, const float *bhi) {
  const float zlo = fmaxf(blo[2], c.ortho ? 0.f : c.n);
  const float zhi = fminf(bhi[2], c.f);
  if (!(zlo <= zhi)) return empty_rect();
  float pmin[2], pmax[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float x0 = blo[a], x1 = bhi[a];
    float lo_p, hi_p;
    if (c.ortho) {
      lo_p = __fdiv_rn(x0, c.ell);
      hi_p = __fdiv_rn(x1, c.ell);
    } else {
      const float sl = __fdiv_rn(c.n, __fmul_rn(zlo, c.ell));
      const float sh = __fdiv_rn(c.n, __fmul_rn(zhi, c.ell));
      const float p00 = __fmul_rn(x0, sl), p01 = __fmul_rn(x0, sh);
      const float p10 = __fmul_rn(x1, sl), p11 = __fmul_rn(x1, sh);
      lo_p = fminf(fminf(p00, p01), fminf(p10, p11));
      hi_p = fmaxf(fmaxf(p00, p01), fmaxf(p10, p11));
    }
    const float cen = a == 0 ? c.cw : c.ch;
    pmin[a] = __fadd_rn(lo_p, cen);
    pmax[a] = __fadd_rn(hi_p, cen);
  }
  const float wl = (float)(c.w - 1), hl = (float)(c.h - 1);
  const float i0 = fmaxf(ceilf(pmin[0]), 0.f), i1 = fminf(floorf(pmax[0]), wl);
  const float j0 = fmaxf(ceilf(pmin[1]), 0.f), j1 = fminf(floorf(pmax[1]), hl);
  if (!(i0 <= i1 && j0 <= j1)) return empty_rect();
  return make_int4((int)i0, (int)i1, (int)j0, (int)j1);
}

__device__ int4 box_rect(const Cam &c, float3 lo, float h) {
  const float hh = __fmul_rn(0.5f, h);
  const float cx = __fsub_rn(__fadd_rn(lo.x, hh), c.o[0]);
  const float cy = __fsub_rn(__fadd_rn(lo.y, hh), c.o[1]);
  const float cz = __fsub_rn(__fadd_rn(lo.z, hh), c.o[2]);
  float blo[3], bhi[3];
  const float *rows[3] = {c.t, c.u, c.vn};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float *R = rows[r];
    const float X = fmaf(R[0], cx, fmaf(R[1], cy, __fmul_rn(R[2], cz)));
    const float E = __fmul_rn(hh, __fadd_rn(__fadd_rn(fabsf(R[0]), fabsf(R[1])), fabsf(R[2])));
    blo[r] = __fsub_rn(X, E);
    bhi[r] = __fadd_rn(X, E);
  }
  return project_box(c, blo, bhi);
}


// ----------------------------------------------------------- surfaces --
// The cubic on [ta, tb], reparametrised to [0, 1].
__device__ __forceinline__ Cubic sub_cubic(const Cubic &c, float ta, float tb) {
  const float L = tb - ta;
  Cubic r;
  r.p0 = fmaf(fmaf(fmaf(c.p3, ta, c.p2), ta, c.p1), ta, c.p0);
  r.p1 = L * fmaf(fmaf(3.f * c.p3, ta, 2.f * c.p2), ta, c.p1);
  r.p2 = L * L * fmaf(3.f * c.p3, ta, c.p2);
  r.p3 = L * L * L * c.p3;
  return r;
}

// Sec. 2.8 on the isosurface s = s_iso: the sign changes of s - s_iso between
// 9 equally spaced samples (far end to near end) are located by bisection;
// the segment is cut there and, at each crossing, the surface segment of
// Eqs. 2.18 and 2.35 (A = a_s^(1 / cos phi), B = i_s (1 - A), phi between the
// ray and the field gradient) goes between the two pieces.
__device__ float4 iso_split_segment(const Cubic &cu, const float *__restrict__ nd,
                                                 float3 uf, float3 du, float3 dir, const TF &tf,
                                                 float dx, const Integ &I, int &steps) {
  float4 acc = seg_identity();
  float t1 = 0.f;
  float gp = cubic_at(cu, 0.f) - I.s_iso;
  for (int k = 0; k < 8; ++k) {
    const float tk1 = (float)(k + 1) * 0.125f;
    const float gn = cubic_at(cu, tk1) - I.s_iso;
    if ((gp < 0.f && gn > 0.f) || (gp > 0.f && gn < 0.f)) {
      float lo = (float)k * 0.125f, hi = tk1, glo = gp;
      for (int it = 0; it < 24; ++it) {
        const float mid = 0.5f * (lo + hi), gm = cubic_at(cu, mid) - I.s_iso;
        if ((gm < 0.f) == (glo < 0.f)) {
          lo = mid;
          glo = gm;
        } else {
          hi = mid;
        }
      }
      const float tc = 0.5f * (lo + hi);
      acc = seg_combine(integrate_segment(sub_cubic(cu, t1, tc), tf, dx * (tc - t1), I, steps),
                        acc);
      // gradient of the trilinear interpolant (its direction is all that counts)
      const float u = fmaf(tc, du.x, uf.x), v = fmaf(tc, du.y, uf.y), w = fmaf(tc, du.z, uf.z);
      float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float n = __ldg(nd + c);
        const float wx = (c & 1) ? u : 1.f - u, wy = (c & 2) ? v : 1.f - v,
                    wz = (c & 4) ? w : 1.f - w;
        const float sx = (c & 1) ? 1.f : -1.f, sy = (c & 2) ? 1.f : -1.f,
                    sz = (c & 4) ? 1.f : -1.f;
        g[0] = fmaf(n * sx, wy * wz, g[0]);
        g[1] = fmaf(n * sy, wx * wz, g[1]);
        g[2] = fmaf(n * sz, wx * wy, g[2]);
      }
      const float gn2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      const float rl = sqrtf(dir.x * dir.x + dir.y * dir.y + dir.z * dir.z);
      const float cphi = gn2 > 0.f ? fabsf(g[0] * dir.x + g[1] * dir.y + g[2] * dir.z) /
                                         (sqrtf(gn2) * rl)
                                   : 1.f;
      const float A = I.a_s >= 1.f ? 1.f
                      : (I.a_s <= 0.f || cphi <= 0.f) ? 0.f
                                                      : exp2f(log2f(I.a_s) / cphi);
      const float om = 1.f - A;
      acc = seg_combine(make_float4(A, I.i_s[0] * om, I.i_s[1] * om, I.i_s[2] * om), acc);
      t1 = tc;
    }
    gp = gn;
  }
  return seg_combine(integrate_segment(sub_cubic(cu, t1, 1.f), tf, dx * (1.f - t1), I, steps),
                     acc);
}

// The set-up of one leaf's segment along one ray: slab interval, reference
// coordinates of its far end (ufar) and their change to the near end (du),
// world length dx, the field's cubic along the segment.
__device__ __forceinline__ Cubic leaf_setup(const Topo &T, const Field &Fd, const Cam &c,
                                            int leaf, float3 org, float3 dir, float3 inv,
                                            float scale, float3 &ufar, float3 &du, float &dx) {
  const int4 g = __ldg(T.geo + leaf);
  const float ih = exp2i(g.w);  // 1 / edge length
  const float3 lo = node_lo(g, scale);
  float a_in, a_out;
  slab(org, dir, inv, lo, exp2i(-g.w), c.amin, c.amax, a_in, a_out);
  ufar = make_float3((fmaf(a_out, dir.x, org.x) - lo.x) * ih,
                     (fmaf(a_out, dir.y, org.y) - lo.y) * ih,
                     (fmaf(a_out, dir.z, org.z) - lo.z) * ih);
  const float da = a_in - a_out;
  du = make_float3(da * dir.x * ih, da * dir.y * ih, da * dir.z * ih);
  dx = fmaxf(a_out - a_in, 0.f) * sqrtf(dir.x * dir.x + dir.y * dir.y + dir.z * dir.z);
  return field_cubic(Fd.nodal + 8 * (size_t)leaf, ufar, du);
}

// The segment of one leaf along one ray: its set-up, then the integration.
template <bool SURF = false>
__device__ __forceinline__ float4 leaf_segment(const Topo &T, const Field &Fd, const Cam &c,
                                               const Integ &I, const TF &tf, int leaf, float3 org,
                                               float3 dir, float3 inv, float scale, int &steps) {
  float3 ufar, du;
  float dx;
  const Cubic cu = leaf_setup(T, Fd, c, leaf, org, dir, inv, scale, ufar, du, dx);
  if (SURF)
    return iso_split_segment(cu, Fd.nodal + 8 * (size_t)leaf, ufar, du, dir, tf, dx, I, steps);
  return integrate_segment(cu, tf, dx, I, steps);
}

}  // namespace
}  // namespace ocr
