// CUDA kernels of the forest-of-octrees raycaster (sm_103a).
//
//   cull_leaves   - pixel rectangle of each leaf's camera-space bounding box
//                   (Sec. 2.2, Sec. 3.1): the pruning step
//   union_level   - rectangle of each internal octree node = bounding box of
//                   its children's rectangles (one launch per level)
//   area_scan     - exclusive prefix of the internal nodes' rectangle areas:
//                   the slot (node, ray) layout of the per-level aggregates,
//                   in Morton order (the load balance of Sec. 3.1 / 3.2)
//   coarsen       - one octree level of Sec. 3.3: for every (node, ray) slot
//                   of the level, the node's leaf children are intersected
//                   with the ray and integrated in shared memory (Sec. 3.2,
//                   Eqs. 2.29 and 2.31, Algorithm 1); the children's segments are
//                   then combined nearest-first with Eq. 2.14 in the ray's
//                   octant order, and the node's aggregate is stored.  The
//                   last pass (the super-root) writes I_v = A I_b + B.
#include "ocr_common.h"

#include <cstdio>

namespace ocr {
namespace {

constexpr float kOne = 1.0f;

__device__ __forceinline__ float4 seg_identity() { return make_float4(1.f, 0.f, 0.f, 0.f); }

// Eq. 2.14: (A2, B2) (+) (A1, B1) = (A2 A1, B2 + A2 B1), n = nearer, f = farther.
__device__ __forceinline__ float4 seg_combine(float4 n, float4 f) {
  return make_float4(n.x * f.x, fmaf(n.x, f.y, n.y), fmaf(n.x, f.z, n.z), fmaf(n.x, f.w, n.w));
}

__device__ __forceinline__ void pixel_ray(const Cam &c, int i, int j, float3 &org, float3 &dir) {
  float di = (float)i - c.cw, dj = (float)j - c.ch;
  float ox = fmaf(dj, c.lu[0], fmaf(di, c.lt[0], 0.f));
  float oy = fmaf(dj, c.lu[1], fmaf(di, c.lt[1], 0.f));
  float oz = fmaf(dj, c.lu[2], fmaf(di, c.lt[2], 0.f));
  if (c.ortho) {
    org = make_float3(c.o[0] + ox, c.o[1] + oy, c.o[2] + oz);
    dir = make_float3(c.v[0], c.v[1], c.v[2]);
  } else {
    org = make_float3(c.o[0], c.o[1], c.o[2]);
    dir = make_float3(c.v[0] + ox, c.v[1] + oy, c.v[2] + oz);
  }
}

__device__ __forceinline__ float recip_or_zero(float d) { return d != 0.f ? 1.f / d : 0.f; }

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
    float b0 = l[a], b1 = l[a] + h;
    if (d[a] == 0.f) {
      if (o[a] < b0 || o[a] > b1) return false;
    } else {
      float s0 = (b0 - o[a]) * iv[a], s1 = (b1 - o[a]) * iv[a];
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

// (kappa, q_r, q_g, q_b) at parameter tau: piecewise-linear transfer function
// of the field value, constant outside the knot range.
__device__ __forceinline__ float4 medium(const Cubic &c, const TF &tf, float tau) {
  const float s = fmaf(fmaf(fmaf(c.p3, tau, c.p2), tau, c.p1), tau, c.p0);
  float z = (s - tf.s_min) * tf.inv;
  z = fminf(fmaxf(z, 0.f), 7.f);
  const int k = min((int)z, 6);
  const float w = z - (float)k;
  const float4 a = tf.v[k], d = tf.s[k];
  return make_float4(fmaf(w, d.x, a.x), fmaf(w, d.y, a.y), fmaf(w, d.z, a.z), fmaf(w, d.w, a.w));
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

// (A, B) of one segment of world length dx: RK4 x nsteps, or DOPRI5 inside
// the midpoint bisection of Algorithm 1, walked far half first so that each
// accepted piece is nearer than everything accumulated so far.
__device__ float4 integrate_segment(const Cubic &cu, const TF &tf, float dx, const Integ &I,
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
  if (I.method != 1) {  // Gauss-2 (Eqs. 2.32-2.33) or Simpson (Eq. 2.34) inside Algorithm 1
    for (;;) {
      const float dtau = ldexpf(1.f, -depth);
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
    const float dtau = ldexpf(1.f, -depth);
    const float t0 = (float)idx * dtau;
    const float H = dx * dtau;
    const float4 kq2 = medium(cu, tf, fmaf(dp::c2, dtau, t0));
    const float4 kq3 = medium(cu, tf, fmaf(dp::c3, dtau, t0));
    const float4 kq4 = medium(cu, tf, fmaf(dp::c4, dtau, t0));
    const float4 kq5 = medium(cu, tf, fmaf(dp::c5, dtau, t0));
    const float4 kq6 = medium(cu, tf, t0 + dtau);
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
    const float4 Y5 = axpy(H, t, one);
    const float4 K7 = rhs(kq6, Y5);
    float4 e = lin4(dp::e1, K1, dp::e3, K3);
    e = axpy(dp::e4, K4, e);
    e = axpy(dp::e5, K5, e);
    e = axpy(dp::e6, K6, e);
    e = axpy(dp::e7, K7, e);
    const float err = H * fmaxf(fmaxf(fabsf(e.x), fabsf(e.y)), fmaxf(fabsf(e.z), fabsf(e.w)));
    const float kmax =
        fmaxf(fmaxf(fmaxf(kq0.x, kq2.x), fmaxf(kq3.x, kq4.x)), fmaxf(kq5.x, kq6.x));
    ++steps;
    if (depth < I.max_depth && (H * kmax > I.c_rk || err > I.tol)) {
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

// Pixel rectangle of the camera-space bounding box of the cube [lo, lo+h]^3:
// the box is mapped by X = (t, u, v/n)^T (x - o) (an affine map, so its AABB is
// centre +- half-extent), clipped to the visible depth range, and projected.
__device__ int4 box_rect(const Cam &c, float3 lo, float h) {
  const float hh = 0.5f * h;
  const float cx = lo.x + hh - c.o[0], cy = lo.y + hh - c.o[1], cz = lo.z + hh - c.o[2];
  float X[3], E[3];
  const float *rows[3] = {c.t, c.u, c.vn};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float *R = rows[r];
    X[r] = fmaf(R[0], cx, fmaf(R[1], cy, R[2] * cz));
    E[r] = hh * (fabsf(R[0]) + fabsf(R[1]) + fabsf(R[2]));
  }
  const float zlo = fmaxf(X[2] - E[2], c.ortho ? 0.f : c.n);
  const float zhi = fminf(X[2] + E[2], c.f);
  if (!(zlo <= zhi)) return empty_rect();
  float pmin[2], pmax[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float x0 = X[a] - E[a], x1 = X[a] + E[a];
    float lo_p, hi_p;
    if (c.ortho) {
      lo_p = x0 / c.ell;
      hi_p = x1 / c.ell;
    } else {
      const float sl = c.n / (zlo * c.ell), sh = c.n / (zhi * c.ell);
      lo_p = fminf(fminf(x0 * sl, x0 * sh), fminf(x1 * sl, x1 * sh));
      hi_p = fmaxf(fmaxf(x0 * sl, x0 * sh), fmaxf(x1 * sl, x1 * sh));
    }
    const float cen = a == 0 ? c.cw : c.ch;
    pmin[a] = lo_p + cen;
    pmax[a] = hi_p + cen;
  }
  const float wl = (float)(c.w - 1), hl = (float)(c.h - 1);
  const float i0 = fmaxf(ceilf(pmin[0]), 0.f), i1 = fminf(floorf(pmax[0]), wl);
  const float j0 = fmaxf(ceilf(pmin[1]), 0.f), j1 = fminf(floorf(pmax[1]), hl);
  if (!(i0 <= i1 && j0 <= j1)) return empty_rect();
  return make_int4((int)i0, (int)i1, (int)j0, (int)j1);
}

__global__ void cull_leaves_kernel(Topo T, Cam c, Scratch S) {
  const float scale = ldexpf(1.f, -T.L);
  unsigned nvis = 0;
  // the loop bound is warp-uniform so that the ballot below sees full warps
  const int stride = gridDim.x * blockDim.x;
  for (int k0 = blockIdx.x * blockDim.x; k0 < T.N; k0 += stride) {
    const int k = k0 + threadIdx.x;
    bool vis = false;
    if (k < T.N) {
      const int4 g = T.geo[k];
      const int4 r = box_rect(c, node_lo(g, scale), ldexpf(1.f, -g.w));
      S.rect[k] = r;
      vis = r.x <= r.y;
      if (S.visible) S.visible[k] = (unsigned char)vis;
    }
    nvis += __popc(__ballot_sync(0xffffffffu, vis));
  }
  if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(S.stats + kStatVisible, (unsigned long long)nvis);
}

__global__ void union_level_kernel(Topo T, int nb, int ne, Scratch S) {
  for (int k = nb + blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
    int4 u = make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int id = T.child[8 * k + c];
      if (id < 0) continue;
      const int4 r = S.rect[id];
      if (r.x > r.y) continue;
      u.x = min(u.x, r.x); u.y = max(u.y, r.y); u.z = min(u.z, r.z); u.w = max(u.w, r.w);
    }
    S.rect[T.N + k] = (u.x <= u.y) ? u : empty_rect();
  }
}

// ------------------------------------------------------------------- scan --
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long rect_area(int4 r) {
  return r.x > r.y ? 0ll : (long long)(r.y - r.x + 1) * (long long)(r.w - r.z + 1);
}

// slots of internal node k: its rectangle's area, or none below the tile level
__device__ __forceinline__ long long node_slots(const Topo &T, const Scratch &S, int k) {
  return T.geo[T.N + k].w > T.lt ? 0ll : rect_area(S.rect[T.N + k]);
}

__device__ long long block_exclusive_scan(long long v, long long *warp_tot, long long &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ll;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;  // inclusive prefix of warp totals
  }
  __syncthreads();
  total = warp_tot[(blockDim.x >> 5) - 1];
  const long long before = wid ? warp_tot[wid - 1] : 0ll;
  const long long r = before + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) area_reduce_kernel(Topo T, Scratch S,
                                                                   long long *block_sums) {
  __shared__ long long wt[32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  long long s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q)
    if (base + q < T.M) s += node_slots(T, S, base + q);
  long long tot;
  block_exclusive_scan(s, wt, tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) block_sums_scan_kernel(long long *block_sums, int n) {
  __shared__ long long wt[32];
  long long carry = 0;
  for (int b = 0; b < n; b += blockDim.x) {
    const int k = b + threadIdx.x;
    const long long v = k < n ? block_sums[k] : 0ll;
    long long tot;
    const long long ex = block_exclusive_scan(v, wt, tot);
    if (k < n) block_sums[k] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[n] = carry;
}

__global__ void __launch_bounds__(kScanThreads) area_downsweep_kernel(Topo T, Scratch S,
                                                                      const long long *block_sums,
                                                                      int nblk) {
  __shared__ long long wt[32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  long long a[kScanItems], s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    a[q] = (base + q < T.M) ? node_slots(T, S, base + q) : 0ll;
    s += a[q];
  }
  long long tot;
  long long run = block_sums[blockIdx.x] + block_exclusive_scan(s, wt, tot);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < T.M) S.off[base + q] = run;
    run += a[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) S.off[T.M] = block_sums[nblk];
}

// chunk_node[c] = the internal node whose slot range holds slot c * kChunk
__global__ void chunk_map_kernel(Topo T, Scratch S) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < T.M; n += gridDim.x * blockDim.x) {
    const long long a = S.off[n], b = S.off[n + 1];
    if (b <= a) continue;
    for (long long c = (a + kChunk - 1) / kChunk; c * kChunk < b; ++c) S.chunk_node[c] = n;
  }
}

__global__ void gather_level_slots_kernel(const long long *off, const int *level_nodes, int n,
                                          long long *out) {
  const int k = threadIdx.x;
  if (k < n) out[k] = off[level_nodes[k]];
}

// ---------------------------------------------------------------- coarsen --
constexpr int kCoarsenThreads = kChunk;

// Node and pixel of a slot of the non-final passes.  The CTA's chunk of slots
// lies in the nodes [chunk_node[chunk], chunk_node[chunk + 1]].
__device__ __forceinline__ void slot_lookup(const Topo &T, const Scratch &S, int nb, int ne,
                                            long long chunk, long long slot, int &node, int &i,
                                            int &j) {
  const long long nch = (S.off[T.M] + kChunk - 1) / kChunk;
  int lo = max(S.chunk_node[chunk], nb);
  int hi = (chunk + 1 < nch) ? min(S.chunk_node[chunk + 1], ne - 1) + 1 : ne;
  while (lo < hi) {  // first node whose offset exceeds the slot
    const int mid = (lo + hi) >> 1;
    if (S.off[mid] <= slot) lo = mid + 1; else hi = mid;
  }
  node = lo - 1;
  const int4 r = S.rect[T.N + node];
  const long long local = slot - S.off[node];
  const int rw = r.y - r.x + 1;
  i = r.x + (int)(local % rw);
  j = r.z + (int)(local / rw);
}

__device__ __forceinline__ unsigned spread3_9(unsigned v) {  // 3 bits -> positions 0, 3, 6
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

// The segment of one leaf along one ray: slab interval, reference coordinates
// of its far end and their change to the near end, field cubic, integration.
__device__ __forceinline__ float4 leaf_segment(const Topo &T, const Field &Fd, const Cam &c,
                                               const Integ &I, const TF &tf, int leaf, float3 org,
                                               float3 dir, float3 inv, float scale, int &steps) {
  const int4 g = __ldg(T.geo + leaf);
  const float ih = ldexpf(1.f, g.w);  // 1 / edge length
  const float3 lo = node_lo(g, scale);
  float a_in, a_out;
  slab(org, dir, inv, lo, ldexpf(1.f, -g.w), c.amin, c.amax, a_in, a_out);
  const float3 ufar = make_float3((fmaf(a_out, dir.x, org.x) - lo.x) * ih,
                                  (fmaf(a_out, dir.y, org.y) - lo.y) * ih,
                                  (fmaf(a_out, dir.z, org.z) - lo.z) * ih);
  const float da = a_in - a_out;
  const float3 du = make_float3(da * dir.x * ih, da * dir.y * ih, da * dir.z * ih);
  const float dx =
      fmaxf(a_out - a_in, 0.f) * sqrtf(dir.x * dir.x + dir.y * dir.y + dir.z * dir.z);
  const Cubic cu = field_cubic(Fd.nodal + 8 * (size_t)leaf, ufar, du);
  return integrate_segment(cu, tf, dx, I, steps);
}

// Subtree pass (Sec. 3.2 + Sec. 3.3 for the deepest levels).  A CTA owns a
// chunk of kChunk consecutive (tile-level node, ray) slots, one thread each.
//  A. per node of the chunk, the leaves of its subtree whose pixel rectangle
//     meets the chunk's rows are gathered in shared memory (Morton order);
//     every ray scans that list, slab-tests the leaves whose rectangle holds
//     its pixel and appends the hits to its own list;
//  B. each ray sorts its hits by their Morton key inside the tile node with
//     every axis mirrored where the ray runs towards negative coordinates:
//     the ray's front-to-back order for disjoint cells;
//  C. each warp integrates the hits of its 32 rays, one hit per lane, in
//     batches, and
//  D. every lane folds its own ray's results nearest-first with Eq. 2.14.
constexpr int kCand = 128;     // candidate leaves per round of phase A
constexpr int kWarpBatch = 64; // hits per warp batch of phase C

__global__ void __launch_bounds__(kChunk, 6)
    subtree_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, int nb, int ne, long long s0,
                   long long s1) {
  constexpr int NT = kChunk, NW = NT / 32;
  __shared__ float4 s_tfv[8], s_tfs[8];
  __shared__ float4 s_ro[NT], s_rd[NT], s_ri[NT];        // ray origin, direction, 1/direction
  __shared__ int s_node[NT];                             // node of each slot, -1 inactive
  __shared__ int s_tnode[NT];                            // distinct nodes of the chunk
  __shared__ int4 s_cbox[kCand];                         // candidate leaf: rectangle ∩ chunk band
  __shared__ int s_cl[kCand], s_cpre[kCand];             // candidate leaf index, pair prefix
  __shared__ int s_cnt[NT];                              // hits of each ray
  __shared__ unsigned char s_live[NT];
  __shared__ unsigned s_flip[NT];
  __shared__ unsigned s_list[kMaxSubtreeHits][NT];       // (mirrored key << 22) | leaf - base
  __shared__ float4 s_res[NW][kWarpBatch];
  __shared__ int s_wcnt[NW], s_nn, s_leaf_base;
  __shared__ unsigned long long s_acc[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  if (tid < 4) s_acc[tid] = 0ull;

  // slot -> node, pixel, ray; rays that miss the node's box skip all leaves
  const long long chunk = s0 / NT + blockIdx.x, cs = chunk * NT;
  const long long slot = cs + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = -1, i = 0, j = 0;
  if (active) slot_lookup(T, S, nb, ne, chunk, slot, node, i, j);
  float3 org, dir;
  pixel_ray(c, i, j, org, dir);
  const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
  const float scale = ldexpf(1.f, -T.L);
  bool live = false;
  if (active) {
    const int4 gn = __ldg(T.geo + T.N + node);
    float a0, a1;
    live = slab(org, dir, inv, node_lo(gn, scale), ldexpf(1.f, -gn.w), c.amin, c.amax, a0, a1);
  }
  const unsigned flip =
      (dir.x < 0.f ? 0x49u : 0u) | (dir.y < 0.f ? 0x92u : 0u) | (dir.z < 0.f ? 0x124u : 0u);
  s_ro[tid] = make_float4(org.x, org.y, org.z, 0.f);
  s_rd[tid] = make_float4(dir.x, dir.y, dir.z, 0.f);
  s_ri[tid] = make_float4(inv.x, inv.y, inv.z, 0.f);
  s_node[tid] = active ? node : -1;
  s_live[tid] = live;
  s_flip[tid] = flip;
  __syncthreads();

  // distinct nodes of the chunk (a node's slots are contiguous)
  {
    const bool head = active && (tid == 0 || s_node[tid - 1] != node);
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (lane == 0) s_wcnt[wid] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += s_wcnt[w];
    if (head) s_tnode[base + __popc(bal & ((1u << lane) - 1u))] = node;
    if (tid == NT - 1) {
      int tot = 0;
      for (int w = 0; w < NW; ++w) tot += s_wcnt[w];
      s_nn = tot;
    }
    __syncthreads();
    if (tid == 0) s_leaf_base = s_nn ? __ldg(T.leaves + s_tnode[0]).x : 0;
  }
  __syncthreads();

  // A. candidates and hits: (candidate leaf, pixel) pairs, spread evenly
  // over the CTA by a prefix sum of their counts
  unsigned ntest = 0;
  const int nn = s_nn, leaf_base = s_leaf_base;
  s_cnt[tid] = 0;
  for (int q = 0; q < nn; ++q) {
    const int nd = s_tnode[q];
    const int2 lr = __ldg(T.leaves + nd);
    const int4 rn = __ldg(S.rect + T.N + nd);
    const long long off = __ldg(S.off + nd);
    const int rw = rn.y - rn.x + 1;
    const long long la = max(cs, off) - off;  // node-local slots inside the chunk
    const long long lb = min(min(cs + NT, s1), __ldg(S.off + nd + 1)) - off;
    const int jr0 = rn.z + (int)(la / rw), jr1 = rn.z + (int)((lb - 1) / rw);
    const unsigned dm = (1u << (T.L - __ldg(T.geo + T.N + nd).w)) - 1u;
    for (int l0 = lr.x; l0 < lr.y; l0 += kCand) {
      const int l = l0 + tid;
      int cnt = 0;
      int4 box = empty_rect();  // overlap of the leaf's rectangle with the chunk band
      if (tid < kCand && l < lr.y) {
        const int4 r = __ldg(S.rect + l);
        box = make_int4(max(r.x, rn.x), min(r.y, rn.y), max(r.z, jr0), min(r.w, jr1));
        if (box.x <= box.y && box.z <= box.w) cnt = (box.y - box.x + 1) * (box.w - box.z + 1);
      }
      // exclusive prefix of the pair counts over the CTA
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      __syncthreads();  // previous round's pair table fully consumed
      if (lane == 31) s_wcnt[wid] = x;
      __syncthreads();
      int base = 0, tot = 0;
      for (int w = 0; w < NW; ++w) {
        if (w < wid) base += s_wcnt[w];
        tot += s_wcnt[w];
      }
      s_cpre[tid] = base + x - cnt;
      s_cbox[tid] = box;
      s_cl[tid] = l;
      __syncthreads();
      for (int pq = tid; pq < tot; pq += NT) {
        int lo = 0, hi = kCand;  // candidate: last k with s_cpre[k] <= pq
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_cpre[mid] <= pq) lo = mid; else hi = mid;
        }
        const int4 b = s_cbox[lo];
        const int loc = pq - s_cpre[lo], bw = b.y - b.x + 1;
        const int jj = b.z + loc / bw, ii = b.x + loc % bw;
        const long long ls = (long long)(jj - rn.z) * rw + (ii - rn.x);
        if (ls < la || ls >= lb) continue;
        const int t = (int)(off + ls - cs);
        if (!s_live[t]) continue;
        ++ntest;
        const int lf = s_cl[lo];
        const int4 g = __ldg(T.geo + lf);
        const float4 ro = s_ro[t], rd = s_rd[t], ri = s_ri[t];
        float b0, b1;
        if (!slab(make_float3(ro.x, ro.y, ro.z), make_float3(rd.x, rd.y, rd.z),
                  make_float3(ri.x, ri.y, ri.z), node_lo(g, scale), ldexpf(1.f, -g.w), c.amin,
                  c.amax, b0, b1))
          continue;
        const unsigned key = spread3_9((unsigned)g.x & dm) | (spread3_9((unsigned)g.y & dm) << 1) |
                             (spread3_9((unsigned)g.z & dm) << 2);
        const int k = atomicAdd(&s_cnt[t], 1);
        if (k < kMaxSubtreeHits)
          s_list[k][t] = ((key ^ s_flip[t]) << 22) | (unsigned)(lf - leaf_base);
      }
    }
  }
  __syncthreads();
  const unsigned nhit = (unsigned)s_cnt[tid];

  // B. sort the ray's hits into its front-to-back order
  const int n = min((int)nhit, kMaxSubtreeHits);
  for (int a = 1; a < n; ++a) {
    const unsigned v = s_list[a][tid];
    int b = a - 1;
    while (b >= 0 && s_list[b][tid] > v) {
      s_list[b + 1][tid] = s_list[b][tid];
      --b;
    }
    s_list[b + 1][tid] = v;
  }

  // C + D. per warp: integrate the warp's hits, one per lane; fold per ray
  int pre = n;  // inclusive prefix of the hit counts over the warp's lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += y;
  }
  const int Hw = __shfl_sync(0xffffffffu, pre, 31);
  const int my0 = pre - n;
  float4 acc = seg_identity();
  int steps = 0;
  TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  for (int b0 = 0; b0 < Hw; b0 += kWarpBatch) {
    const int b1 = min(Hw, b0 + kWarpBatch);
    for (int hb = b0; hb < b1; hb += 32) {
      const int h = hb + lane;
      // owner lane: the first lane whose inclusive prefix exceeds h
      int lo = 0;
#pragma unroll
      for (int st = 16; st > 0; st >>= 1) {
        const int p = __shfl_sync(0xffffffffu, pre, lo + st - 1);
        if (p <= h) lo += st;
      }
      const int ow = lo;
      const int owpre = __shfl_sync(0xffffffffu, my0, ow & 31);
      if (h < b1) {
        const int t = wid * 32 + ow;
        const int leaf = leaf_base + (int)(s_list[h - owpre][t] & 0x3fffffu);
        const float4 ro = s_ro[t], rd = s_rd[t], ri = s_ri[t];
        s_res[wid][h - b0] = leaf_segment(T, Fd, c, I, tf, leaf, make_float3(ro.x, ro.y, ro.z),
                                          make_float3(rd.x, rd.y, rd.z),
                                          make_float3(ri.x, ri.y, ri.z), scale, steps);
      }
    }
    __syncwarp();
    for (int h = max(my0, b0); h < min(my0 + n, b1); ++h) acc = seg_combine(acc, s_res[wid][h - b0]);
    __syncwarp();
  }
  if (active) {
    S.entries[slot] = acc;
    if (nhit > (unsigned)kMaxSubtreeHits) atomicAdd(S.stats + kStatErrors, 1ull);
    if (nhit && S.counts) atomicAdd(S.counts + (size_t)j * c.w + i, (int)nhit);
  }
  unsigned long long v[4] = {nhit, (unsigned long long)steps, ntest, active ? 1ull : 0ull};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0 && x) atomicAdd(&s_acc[q], x);
  }
  __syncthreads();
  if (tid < 4 && s_acc[tid]) atomicAdd(S.stats + tid, s_acc[tid]);
}

template <bool FINAL>
__global__ void __launch_bounds__(kCoarsenThreads, 8)
    coarsen_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, int nb, int ne, long long s0,
                   long long s1, float4 *rgba) {
  constexpr int NT = kCoarsenThreads;
  __shared__ float4 s_tfv[8], s_tfs[8];
  __shared__ float4 s_seg[8][NT];           // child segment of each slot (identity if none)
  __shared__ unsigned short s_hit[8 * NT];  // (slot << 3) | child octant of each hit
  __shared__ int2 s_pix[NT];
  __shared__ int s_node[NT];
  __shared__ int s_nhit;
  __shared__ unsigned long long s_cnt[4];

  const int tid = threadIdx.x;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  if (tid < 4) s_cnt[tid] = 0ull;
  if (tid == 0) s_nhit = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s_seg[q][tid] = seg_identity();

  // non-final passes work on whole chunks of the global slot space, so that
  // chunk_node gives the first node of the CTA without a search
  const long long chunk = FINAL ? 0 : s0 / NT + blockIdx.x;
  const long long slot = FINAL ? s0 + (long long)blockIdx.x * NT + tid : chunk * NT + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = T.M;  // super-root in the final pass
  int i = 0, j = 0;
  if (active) {
    if (FINAL) {
      i = (int)(slot % c.w);
      j = (int)(slot / c.w);
    } else {
      slot_lookup(T, S, nb, ne, chunk, slot, node, i, j);
    }
  }
  s_pix[tid] = make_int2(i, j);
  s_node[tid] = node;
  int ch[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ch[q] = active ? __ldg(T.child + 8 * node + q) : -1;

  float3 org, dir;
  pixel_ray(c, i, j, org, dir);
  const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
  const float scale = ldexpf(1.f, -T.L);

  // a ray that misses the node's box misses every child: its aggregate is the
  // identity and all child work is skipped
  bool live = active;
  if (!FINAL && active) {
    const int4 g = __ldg(T.geo + T.N + node);
    float a0, a1;
    live = slab(org, dir, inv, node_lo(g, scale), ldexpf(1.f, -g.w), c.amin, c.amax, a0, a1);
  }
  __syncthreads();

  // phase 1: slab tests against the leaf children whose rectangle holds the ray
  unsigned local_tests = 0, local_hits = 0;
  if (live) {
    int4 rc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      rc[q] = (ch[q] >= 0 && ch[q] < T.N) ? __ldg(S.rect + ch[q]) : empty_rect();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int4 r = rc[q];
      if (i < r.x || i > r.y || j < r.z || j > r.w) continue;
      ++local_tests;
      const int4 g = __ldg(T.geo + ch[q]);
      float a0, a1;
      if (slab(org, dir, inv, node_lo(g, scale), ldexpf(1.f, -g.w), c.amin, c.amax, a0, a1)) {
        s_hit[atomicAdd(&s_nhit, 1)] = (unsigned short)((tid << 3) | q);
        ++local_hits;
      }
    }
    if (local_hits && S.counts) atomicAdd(S.counts + (size_t)j * c.w + i, (int)local_hits);
  }
  __syncthreads();

  // phase 2: integrate the hits, one per thread, into s_seg[child][slot]; the
  // slab interval is recomputed (same inputs, same arithmetic as phase 1)
  const int nh = s_nhit;
  TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  int steps = 0;
  for (int h = tid; h < nh; h += NT) {
    const int key = s_hit[h];
    const int st = key >> 3, q = key & 7;
    const int2 p = s_pix[st];
    const int leaf = __ldg(T.child + 8 * s_node[st] + q);
    float3 o2, d2;
    pixel_ray(c, p.x, p.y, o2, d2);
    const float3 iv2 = make_float3(recip_or_zero(d2.x), recip_or_zero(d2.y), recip_or_zero(d2.z));
    s_seg[q][st] = leaf_segment(T, Fd, c, I, tf, leaf, o2, d2, iv2, scale, steps);
  }
  __syncthreads();

  // phase 3: combine the children nearest-first.  Along a ray with direction
  // signs (sx, sy, sz) the octants come in increasing order of q ^ mask; the
  // same sequence is formed by combining along x, then y, then z, each pair
  // nearer-first (Eq. 2.14 is associative), with every index static.
  if (active) {
    float4 cs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (!live) {
        cs[q] = seg_identity();
        continue;
      }
      const int id = ch[q];
      float4 s = seg_identity();
      if (id >= 0 && id < T.N) {
        s = s_seg[q][tid];
      } else if (id >= T.N) {
        const int4 r = S.rect[id];
        if (i >= r.x && i <= r.y && j >= r.z && j <= r.w) {
          const long long e =
              S.off[id - T.N] + (long long)(j - r.z) * (r.y - r.x + 1) + (i - r.x);
          s = S.entries[e];
        }
      }
      cs[q] = s;
    }
    const bool fx = dir.x < 0.f, fy = dir.y < 0.f, fz = dir.z < 0.f;
    float4 px[4], py[2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      px[q] = fx ? seg_combine(cs[2 * q + 1], cs[2 * q]) : seg_combine(cs[2 * q], cs[2 * q + 1]);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      py[q] = fy ? seg_combine(px[2 * q + 1], px[2 * q]) : seg_combine(px[2 * q], px[2 * q + 1]);
    const float4 acc = fz ? seg_combine(py[1], py[0]) : seg_combine(py[0], py[1]);
    if (FINAL) {
      rgba[slot] = make_float4(fmaf(acc.x, I.bg[0], acc.y), fmaf(acc.x, I.bg[1], acc.z),
                               fmaf(acc.x, I.bg[2], acc.w), kOne - acc.x);
    } else {
      S.entries[slot] = acc;
    }
  }

  // counters: segments, RK steps, leaf tests, slots
  unsigned long long v[4] = {local_hits, (unsigned long long)steps, local_tests,
                             active ? 1ull : 0ull};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0 && x) atomicAdd(&s_cnt[q], x);
  }
  __syncthreads();
  if (tid < 4 && s_cnt[tid]) atomicAdd(S.stats + kStatCoarse + tid, s_cnt[tid]);
}

}  // namespace

// ------------------------------------------------------------- launchers --
static int grid_for(long long n, int threads, int cap = 152 * 16) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g > cap ? cap : g);
}

cudaError_t launch_cull_leaves(const Topo &T, const Cam &C, Scratch S, cudaStream_t stream) {
  cull_leaves_kernel<<<grid_for(T.N, 256), 256, 0, stream>>>(T, C, S);
  return cudaGetLastError();
}

cudaError_t launch_union_level(const Topo &T, int nb, int ne, const Cam &C, Scratch S,
                               cudaStream_t stream) {
  (void)C;
  if (ne <= nb) return cudaSuccess;
  union_level_kernel<<<grid_for(ne - nb, 256), 256, 0, stream>>>(T, nb, ne, S);
  return cudaGetLastError();
}

int area_scan_blocks(int M) { return (M + kScanTile - 1) / kScanTile; }

cudaError_t launch_area_scan(const Topo &T, Scratch S, long long *block_sums, int nblk_cap,
                             long long *level_slots, const int *level_nodes, int nlevels,
                             cudaStream_t stream) {
  const int nblk = area_scan_blocks(T.M);
  if (nblk + 1 > nblk_cap) return cudaErrorInvalidValue;
  if (nblk > 0) {
    area_reduce_kernel<<<nblk, kScanThreads, 0, stream>>>(T, S, block_sums);
    block_sums_scan_kernel<<<1, 1024, 0, stream>>>(block_sums, nblk);
    area_downsweep_kernel<<<nblk, kScanThreads, 0, stream>>>(T, S, block_sums, nblk);
  } else {
    cudaMemsetAsync(S.off, 0, sizeof(long long), stream);
  }
  if (nlevels > 1024) return cudaErrorInvalidValue;
  gather_level_slots_kernel<<<1, 1024, 0, stream>>>(S.off, level_nodes, nlevels, level_slots);
  return cudaGetLastError();
}

cudaError_t launch_chunk_map(const Topo &T, Scratch S, cudaStream_t stream) {
  if (T.M < 1) return cudaSuccess;
  chunk_map_kernel<<<grid_for(T.M, 256), 256, 0, stream>>>(T, S);
  return cudaGetLastError();
}

cudaError_t launch_subtree(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                           Scratch S, int nb, int ne, long long s0, long long s1,
                           cudaStream_t stream) {
  if (s1 <= s0) return cudaSuccess;
  const long long nblk = (s1 - 1) / kChunk - s0 / kChunk + 1;
  if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  subtree_kernel<<<(unsigned)nblk, kChunk, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1);
  return cudaGetLastError();
}

cudaError_t launch_coarsen(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                           Scratch S, int nb, int ne, long long s0, long long s1, float4 *rgba,
                           cudaStream_t stream) {
  if (s1 <= s0) return cudaSuccess;
  const long long nblk = rgba ? (s1 - s0 + kCoarsenThreads - 1) / kCoarsenThreads
                              : (s1 - 1) / kCoarsenThreads - s0 / kCoarsenThreads + 1;
  if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  if (rgba)
    coarsen_kernel<true><<<(unsigned)nblk, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne,
                                                                          s0, s1, rgba);
  else
    coarsen_kernel<false><<<(unsigned)nblk, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne,
                                                                           s0, s1, nullptr);
  return cudaGetLastError();
}

}  // namespace ocr

// ==========================================================================
// Pruning without device allocation (ocr_prune_noalloc).
//
// Some callers cannot allocate device memory when they need a result: an
// application that hands out all device memory from a pool it reserved up
// front, a real-time loop that must not take the device-wide synchronisation
// cudaMalloc implies, or a plug-in that runs inside another program's memory
// budget.  For them this entry point computes the pruning step -- every
// leaf's pixel rectangle, exactly as cull_leaves_kernel does, plus the list of
// visible leaves in Morton order -- using only caller-provided inputs and
// outputs and one fixed scratch array that lives in the library's image on
// each device.  The scratch holds the tile ticket, an error word and one
// status word per tile of the single-pass (decoupled look-back) compaction.
// ==========================================================================
#include "../../include/ocraycast.h"

#include <mutex>

namespace ocr {
namespace {

constexpr int kNoAllocThreads = 256, kNoAllocItems = 4;
constexpr int kNoAllocTile = kNoAllocThreads * kNoAllocItems;
constexpr long long kNoAllocMaxTiles = (long long)OCR_NOALLOC_MAX_LEAVES / kNoAllocTile;
constexpr unsigned long long kTileAggregate = 1ull << 62, kTilePrefix = 2ull << 62;
constexpr unsigned long long kTileValue = (1ull << 62) - 1;
constexpr int kLookbackSpins = 1 << 20;
constexpr int kNoAllocMaxDevices = 64;

// [0] tile ticket, [1] error word, [2 + t] status of tile t (flag << 62 | count).
// 2 + 65536 words = 512 KiB on every device that loads the library.
static __device__ __align__(256) unsigned long long g_prune_scratch[2 + kNoAllocMaxTiles];

__global__ void __launch_bounds__(kNoAllocThreads)
    prune_compact_kernel(const int4 *__restrict__ geo, int n, int L, Cam c, int4 *rects,
                         int *vis_idx, unsigned long long *scratch) {
  __shared__ int s_tile, s_wsum[kNoAllocThreads / 32];
  __shared__ long long s_excl;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // tiles are numbered in the order CTAs start, so every predecessor a CTA
  // waits for is already running
  if (tid == 0) s_tile = (int)atomicAdd(scratch, 1ull);
  __syncthreads();
  const int tile = s_tile;
  const int base = tile * kNoAllocTile + tid * kNoAllocItems;
  const float scale = ldexpf(1.f, -L);
  bool vis[kNoAllocItems];
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < kNoAllocItems; ++q) {
    const int k = base + q;
    vis[q] = false;
    if (k < n) {
      const int4 g = geo[k];
      const int4 r = box_rect(c, node_lo(g, scale), ldexpf(1.f, -g.w));
      if (rects) rects[k] = r;
      vis[q] = r.x <= r.y;
      cnt += vis[q];
    }
  }
  int x = cnt;  // inclusive prefix within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[wid] = x;
  __syncthreads();
  int before = 0, total = 0;
  for (int w = 0; w < kNoAllocThreads / 32; ++w) {
    if (w < wid) before += s_wsum[w];
    total += s_wsum[w];
  }
  if (tid == 0) {
    unsigned long long *st = scratch + 2;
    long long excl = 0;
    if (tile == 0) {
      atomicExch(st, kTilePrefix | (unsigned long long)total);
    } else {
      atomicExch(st + tile, kTileAggregate | (unsigned long long)total);
      for (int p = tile - 1; p >= 0; --p) {
        unsigned long long w = 0;
        int spins = 0;
        while (((w = atomicAdd(st + p, 0ull)) >> 62) == 0ull) {
          if (++spins > kLookbackSpins) {  // never expected: give up, flag, return
            atomicExch(scratch + 1, 1ull);
            break;
          }
          __nanosleep(64);
        }
        excl += (long long)(w & kTileValue);
        if ((w >> 62) != 1ull) break;  // an inclusive prefix (or a timeout) ends the walk
      }
      atomicExch(st + tile, kTilePrefix | (unsigned long long)(excl + total));
    }
    s_excl = excl;
  }
  __syncthreads();
  long long pos = s_excl + before + x - cnt;
#pragma unroll
  for (int q = 0; q < kNoAllocItems; ++q)
    if (vis[q]) vis_idx[pos++] = base + q;
}

}  // namespace
}  // namespace ocr

extern "C" int ocr_prune_noalloc(const int32_t *d_leaf_geo, int64_t nleaves, int max_level,
                                 const ocr_camera *cam, int32_t *d_rects, int32_t *d_visible_idx,
                                 int64_t *h_nvisible, void *stream) {
  using namespace ocr;
  if (!d_leaf_geo || !cam || !d_visible_idx || !h_nvisible) return OCR_ERR_INVALID;
  if (nleaves < 1 || nleaves > OCR_NOALLOC_MAX_LEAVES) return OCR_ERR_INVALID;
  if (max_level < 0 || max_level > 20) return OCR_ERR_INVALID;
  if (((uintptr_t)d_leaf_geo & 15) || ((uintptr_t)d_rects & 15)) return OCR_ERR_INVALID;
  const ocr_camera &cc = *cam;
  if (cc.w < 1 || cc.h < 1 || (int64_t)cc.w * cc.h > (1ll << 31) - 1 || !(cc.near_ > 0.0) ||
      !(cc.far_ > cc.near_) || !(cc.ell > 0.0))
    return OCR_ERR_INVALID;
  // the same float32 camera constants as ocr_set_camera
  Cam k{};
  for (int a = 0; a < 3; ++a) {
    k.o[a] = (float)cc.o[a];
    k.v[a] = (float)(cc.ortho ? cc.v[a] / cc.near_ : cc.v[a]);
    k.lt[a] = (float)(cc.ell * cc.t[a]);
    k.lu[a] = (float)(cc.ell * cc.u[a]);
    k.t[a] = (float)cc.t[a];
    k.u[a] = (float)cc.u[a];
    k.vn[a] = (float)(cc.v[a] / cc.near_);
  }
  k.n = (float)cc.near_;
  k.f = (float)cc.far_;
  k.ell = (float)cc.ell;
  k.cw = 0.5f * (float)(cc.w - 1);
  k.ch = 0.5f * (float)(cc.h - 1);
  k.w = cc.w;
  k.h = cc.h;
  k.ortho = cc.ortho ? 1 : 0;
  k.amin = cc.ortho ? 0.f : 1.f;
  k.amax = (float)(cc.ortho ? cc.far_ : cc.far_ / cc.near_);

  // device address of the scratch array: looked up once per device, with that
  // device current (the array's name is only a stand-in in host code)
  static std::mutex mu;
  static void *addr[kNoAllocMaxDevices] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return OCR_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return OCR_ERR_UNSUPPORTED;
  unsigned long long *scratch;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_prune_scratch) != cudaSuccess || !p) return OCR_ERR_CUDA;
      addr[dev] = p;
    }
    scratch = static_cast<unsigned long long *>(addr[dev]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ntiles = (int)((nleaves + kNoAllocTile - 1) / kNoAllocTile);
  // the ticket, the error word and the tiles' status words must start at zero
  if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (2 + (size_t)ntiles), st) !=
      cudaSuccess)
    return OCR_ERR_CUDA;
  prune_compact_kernel<<<ntiles, kNoAllocThreads, 0, st>>>(
      reinterpret_cast<const int4 *>(d_leaf_geo), (int)nleaves, max_level, k,
      reinterpret_cast<int4 *>(d_rects), d_visible_idx, scratch);
  if (cudaGetLastError() != cudaSuccess) return OCR_ERR_CUDA;
  unsigned long long h_err = 0, h_last = 0;
  if (cudaMemcpyAsync(&h_err, scratch + 1, sizeof h_err, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&h_last, scratch + 2 + (ntiles - 1), sizeof h_last,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return OCR_ERR_CUDA;
  if (h_err) return OCR_ERR_DEVICE;
  *h_nvisible = (int64_t)(h_last & kTileValue);
  return OCR_OK;
}
