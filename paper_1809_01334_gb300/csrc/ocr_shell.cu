// Cubed-sphere shell forests (six trees, the equiangular map, degree-2 data)
// on sm_103a.
//
// A shell leaf is bounded by four planes through the centre (constant xi or
// eta of its tree) and two spheres (constant zeta), so a ray meets it in at
// most two intervals and the Morton order of the leaves is no longer the
// order along a ray.  The render therefore builds per-ray segment lists:
//   shell_cull    - per leaf: the camera-space AABB of its 8 mapped corners,
//                   widened by r_out (1 - cos phi) (every point of the leaf
//                   lies that close to the corners' hull), projected to its
//                   pixel rectangle (Sec. 3.1, Sec. 2.2);
//   shell_pairs   - over the (leaf, pixel) pairs of the rectangles (the prefix
//                   sum of rectangle areas cuts them into equal CTA chunks):
//                   ray / leaf intersection, segments counted per ray, then,
//                   after a scan, written to the ray's list with the entry
//                   depth alpha_in as the sort key (ties by (tree, Morton
//                   key) through the leaf index);
//   shell_rays    - one warp per ray: sort the list (bitonic, in shared
//                   memory), integrate every segment (RK4 or Algorithm 1 with
//                   DOPRI5 / Gauss-2 / Simpson, the field through the inverse
//                   map and the degree-2 interpolation), resolve overlaps by
//                   cut (Eq. 2.20) and average (Eq. 2.21), and merge nearest
//                   first with Eq. 2.14 into the pixel I = A I_b + B.
#include "ocr_common.h"
#include "ocr_device.cuh"
#include "ocr_shell.cuh"

namespace ocr {
namespace {

// ------------------------------------------------------ monomial form --
// Per leaf: the 27 nodal values (Lagrange form on the nodes 0, 1/2, 1 per
// axis, index 9 c + 3 b + a) to the coefficients of u^i v^j w^k at the same
// index 9 k + 3 j + i.  Along one axis the values f0, f1, f2 at 0, 1/2, 1 give
// p(t) = f0 + (-3 f0 + 4 f1 - f2) t + (2 f0 - 4 f1 + 2 f2) t^2.
__device__ __forceinline__ void lagrange_to_monomial(float &f0, float &f1, float &f2) {
  const float c1 = fmaf(-3.f, f0, fmaf(4.f, f1, -f2));
  const float c2 = 2.f * (f0 + f2) - 4.f * f1;
  f1 = c1;
  f2 = c2;
}

constexpr int kMonoLeaves = 256;  // leaves per CTA (one thread each)

// The CTA's 256 leaves (27 x 256 consecutive floats) are staged through shared
// memory with coalesced loads and stores; each thread converts one leaf
// (row stride 27, odd: the threads' rows fall in distinct banks).
__global__ void __launch_bounds__(kMonoLeaves)
    shell_monomial_kernel(const float *__restrict__ nodal, float *__restrict__ coef, int N) {
  __shared__ float s_f[27 * kMonoLeaves];
  for (long long l0 = (long long)blockIdx.x * kMonoLeaves; l0 < N;
       l0 += (long long)gridDim.x * kMonoLeaves) {
    const int nl = (int)(N - l0 < kMonoLeaves ? N - l0 : kMonoLeaves);
    const float *src = nodal + 27 * l0;
    for (int q = threadIdx.x; q < 27 * nl; q += kMonoLeaves) s_f[q] = __ldg(src + q);
    __syncthreads();
    if ((int)threadIdx.x < nl) {
      float *f = s_f + 27 * threadIdx.x;
      float g[27];
#pragma unroll
      for (int q = 0; q < 27; ++q) g[q] = f[q];
#pragma unroll
      for (int r = 0; r < 9; ++r) lagrange_to_monomial(g[3 * r], g[3 * r + 1], g[3 * r + 2]);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          lagrange_to_monomial(g[9 * c + a], g[9 * c + 3 + a], g[9 * c + 6 + a]);
#pragma unroll
      for (int r = 0; r < 9; ++r) lagrange_to_monomial(g[r], g[9 + r], g[18 + r]);
#pragma unroll
      for (int q = 0; q < 27; ++q) f[q] = g[q];
    }
    __syncthreads();
    float *dst = coef + 27 * l0;
    for (int q = threadIdx.x; q < 27 * nl; q += kMonoLeaves) dst[q] = s_f[q];
    __syncthreads();
  }
}

// ------------------------------------------------------------ plane table --
__global__ void __launch_bounds__(256)
    shell_planes_kernel(const int4 *__restrict__ geo, int N, Shell S, float4 *planes) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const LeafShell q = leaf_shell(S, __ldg(geo + k));
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float3 m = plane_normal(q, s);
      planes[4 * (size_t)k + s] = make_float4(m.x, m.y, m.z, s == 0 ? q.rin : s == 1 ? q.rout : 0.f);
    }
  }
}

// ----------------------------------------------------------------- culling --
__global__ void __launch_bounds__(256)
    shell_cull_kernel(const int4 *__restrict__ geo, int N, Shell S, Cam c, int4 *rect,
                      unsigned char *visible, unsigned long long *stats) {
  // the canonical FP32 evaluation of the index decisions (ocr_device.cuh)
  int nvis = 0;
  const float tn = __fsqrt_rn(fmaf(c.t[2], c.t[2], fmaf(c.t[1], c.t[1], __fmul_rn(c.t[0], c.t[0]))));
  const float un = __fsqrt_rn(fmaf(c.u[2], c.u[2], fmaf(c.u[1], c.u[1], __fmul_rn(c.u[0], c.u[0]))));
  const float vn =
      __fsqrt_rn(fmaf(c.vn[2], c.vn[2], fmaf(c.vn[1], c.vn[1], __fmul_rn(c.vn[0], c.vn[0]))));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const LeafShell q = leaf_shell(S, __ldg(geo + k));
    float d[4][3], cs[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float ta = (cc & 1) ? q.ta1 : q.ta0, tb = (cc & 2) ? q.tb1 : q.tb0;
#pragma unroll
      for (int a = 0; a < 3; ++a) d[cc][a] = fmaf(tb, q.e2[a], fmaf(ta, q.e1[a], q.n[a]));
      const float nn = fmaf(d[cc][2], d[cc][2], fmaf(d[cc][1], d[cc][1], __fmul_rn(d[cc][0], d[cc][0])));
      const float inv = __fdiv_rn(1.f, __fsqrt_rn(nn));
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        d[cc][a] = __fmul_rn(d[cc][a], inv);
        cs[a] = __fadd_rn(cs[a], d[cc][a]);
      }
    }
    const float csn =
        __fdiv_rn(1.f, __fsqrt_rn(fmaf(cs[2], cs[2], fmaf(cs[1], cs[1], __fmul_rn(cs[0], cs[0])))));
    float cmin = 1.f;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      cmin = fminf(cmin, __fmul_rn(fmaf(d[cc][2], cs[2], fmaf(d[cc][1], cs[1],
                                                             __fmul_rn(d[cc][0], cs[0]))),
                                   csn));
    const float delta = __fmul_rn(q.rout, __fsub_rn(1.f, cmin));
    float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const float *rows[3] = {c.t, c.u, c.vn};
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const float r = (cc & 4) ? q.rout : q.rin;
      const float x = fmaf(r, d[cc & 3][0], -c.o[0]), y = fmaf(r, d[cc & 3][1], -c.o[1]),
                  z = fmaf(r, d[cc & 3][2], -c.o[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float X = fmaf(rows[a][0], x, fmaf(rows[a][1], y, __fmul_rn(rows[a][2], z)));
        blo[a] = fminf(blo[a], X);
        bhi[a] = fmaxf(bhi[a], X);
      }
    }
    const float ext[3] = {__fmul_rn(delta, tn), __fmul_rn(delta, un), __fmul_rn(delta, vn)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      blo[a] = __fsub_rn(blo[a], ext[a]);
      bhi[a] = __fadd_rn(bhi[a], ext[a]);
    }
    const int4 r = project_box(c, blo, bhi);
    rect[k] = r;
    const bool vis = r.x <= r.y;
    if (vis && visible) visible[k] = 1;
    nvis += vis;
  }
  // one counter update per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nvis += __shfl_down_sync(0xffffffffu, nvis, o);
  if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(stats + kStatVisible, (unsigned long long)nvis);
}

// ------------------------------------------------------- segment lists --
// MODE 0 counts segments per ray (and records which pairs hit, one ballot
// word per warp, when hitmask is given); MODE 1 writes each segment's key into
// its ray's list at ray_off (the camera's plan) plus its place among the
// ray's segments; MODE 2 also appends every segment to a list grouped by leaf
// (one global append per CTA, whose pairs are consecutive in leaf order):
// lm[pos] = (pixel, 2 leaf + piece), and kpos[at] = pos beside the key, for
// the adjoint.  Every mode intersects every pair of the CTA's chunk.
template <int MODE>
__global__ void __launch_bounds__(kPairChunk)
    shell_pairs_kernel(const int4 *__restrict__ geo, int N, Shell S, Cam c,
                       const int4 *__restrict__ rect, const long long *__restrict__ leaf_off,
                       const int *__restrict__ chunk_leaf, long long npairs, int *counts,
                       const long long *__restrict__ ray_off, int *cursor,
                       unsigned long long *keys, long long key_cap, unsigned long long *stats,
                       unsigned *hitmask, unsigned *kpos, int2 *lm,
                       unsigned long long *lm_count) {
  constexpr int NW = kPairChunk / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long p = (long long)blockIdx.x * kPairChunk + threadIdx.x;  // this thread's pair
  int n = 0, leaf = 0;
  long long pix = 0;
  float ai[2], ao[2];
  if (p < npairs) {
    const long long nch = (npairs + kPairChunk - 1) / kPairChunk;
    int lo = chunk_leaf[blockIdx.x];
    int hi = (blockIdx.x + 1 < nch) ? chunk_leaf[blockIdx.x + 1] + 1 : N;
    while (lo + 1 < hi) {  // the last leaf whose offset is <= p
      const int mid = (lo + hi) >> 1;
      if (leaf_off[mid] <= p) lo = mid; else hi = mid;
    }
    leaf = lo;
    const int4 r = rect[leaf];
    // the pair's place in the rectangle: below w h < 2^31, 32-bit division
    const unsigned local = (unsigned)(p - leaf_off[leaf]);
    const unsigned rw = (unsigned)(r.y - r.x + 1), row = local / rw;
    const int i = r.x + (int)(local - row * rw), j = r.z + (int)row;
    pix = (long long)j * c.w + i;
    float3 org, dir;
    pixel_ray(c, i, j, org, dir);
    n = shell_ray_leaf(S.planes + 4 * (size_t)leaf, org, dir, c.amin, c.amax, ai, ao);
  }
  if (MODE == 0) {
    const unsigned bal = __ballot_sync(0xffffffffu, n > 0);
    if (hitmask && lane == 0) hitmask[(size_t)blockIdx.x * NW + wid] = bal;
    if (n) atomicAdd(counts + pix, n);
    return;
  }
  unsigned pos = 0;
  if (MODE == 2) {  // this pair's place in the CTA's block of the leaf-grouped list
    __shared__ unsigned s_w[NW], s_base;
    unsigned x = (unsigned)n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned tot = 0;
      for (int w = 0; w < NW; ++w) {
        const unsigned u = s_w[w];
        s_w[w] = tot;
        tot += u;
      }
      s_base = tot ? (unsigned)atomicAdd(lm_count, (unsigned long long)tot) : 0u;
    }
    __syncthreads();
    pos = s_base + s_w[wid] + x - (unsigned)n;
  }
  if (!n) return;
  const long long at = ray_off[pix] + atomicAdd(cursor + pix, n);
  const bool bad = at + n > key_cap || at + n > ray_off[pix + 1] ||
                   (MODE == 2 && (long long)pos + n > key_cap);
  if (bad) {  // more than counted and planned
    atomicAdd(stats + kStatErrors, 1ull);
    if (MODE == 2)
      for (int q = 0; q < n; ++q)
        if ((long long)pos + q < key_cap) lm[pos + q] = make_int2(-1, -1);
    return;
  }
  for (int q = 0; q < n; ++q) {  // alpha_in >= 0: its bits sort like the value
    keys[at + q] = (unsigned long long)__float_as_uint(ai[q]) << 32 | (unsigned)(2 * leaf + q);
    if (MODE == 2) {
      kpos[at + q] = pos + (unsigned)q;
      lm[pos + q] = make_int2((int)pix, 2 * leaf + q);
    }
  }
}

__global__ void __launch_bounds__(256) max_count_kernel(const int *counts, long long n,
                                                        unsigned long long *stats) {
  int m = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    m = max(m, counts[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(stats + kStatMaxHits, (unsigned long long)m);
}

// ---------------------------------------------------------- one ray, one warp --
// Eq. 2.20 (1 - A^f formed as -expm1(f ln A)) and Eq. 2.21.
__device__ __forceinline__ float4 seg_cut(float4 s, float f) {
  const float la = logf(s.x);
  const float ratio = la == 0.f ? f : expm1f(f * la) / expm1f(la);
  return make_float4(expf(f * la), s.y * ratio, s.z * ratio, s.w * ratio);
}

__device__ __forceinline__ float4 seg_average(float4 a, float4 b) {
  return make_float4(sqrtf(a.x * b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.5f * (a.w + b.w));
}

// near segment N on [a0, a1] and far segment F on [b0, b1] with b0 < a1: the
// pieces before, inside and after the overlap, the overlapped ones averaged
__device__ float4 resolve_overlap(float4 N, float2 in, float4 F, float2 iF) {
  const float e = fminf(in.y, iF.y), LN = in.y - in.x, LF = iF.y - iF.x;
  float4 r = seg_identity();
  if (iF.x > in.x) r = seg_cut(N, (iF.x - in.x) / LN);
  r = seg_combine(r, seg_average(seg_cut(N, (e - iF.x) / LN), seg_cut(F, (e - iF.x) / LF)));
  if (in.y > e)
    r = seg_combine(r, seg_cut(N, (in.y - e) / LN));
  else if (iF.y > e)
    r = seg_combine(r, seg_cut(F, (iF.y - e) / LF));
  return r;
}

// The merge of one ray's n segments (values val, intervals iv, in order of
// entry depth) by the warp: nearest first with Eq. 2.14; where consecutive
// segments overlap (rounding slivers), the pieces before, inside and after
// each overlap are cut (Eq. 2.20) and the overlapped ones averaged (Eq.
// 2.21).  The result in lane 0.
__device__ float4 fold_ray_segments(const float4 *val, const float2 *iv, int n, int lane) {
  bool ov = false;
  for (int k = lane; k + 1 < n; k += 32) ov |= iv[k + 1].x < iv[k].y;
  float4 acc = seg_identity();
  if (!__any_sync(0xffffffffu, ov)) {
    // lane l folds a contiguous run, then the runs are combined in order
    const int q = (n + 31) >> 5, k0 = lane * q, k1 = min(k0 + q, n);
    for (int k = k0; k < k1; ++k) acc = seg_combine(acc, val[k]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      float4 y;
      y.x = __shfl_down_sync(0xffffffffu, acc.x, o);
      y.y = __shfl_down_sync(0xffffffffu, acc.y, o);
      y.z = __shfl_down_sync(0xffffffffu, acc.z, o);
      y.w = __shfl_down_sync(0xffffffffu, acc.w, o);
      if ((lane & (2 * o - 1)) == 0) acc = seg_combine(acc, y);
    }
  } else if (lane == 0) {
    float4 cur = val[0];
    float2 ci = iv[0];
    for (int k = 1; k < n; ++k) {
      const float4 nv = val[k];
      const float2 ni = iv[k];
      if (ni.x < ci.y) {
        cur = resolve_overlap(cur, ci, nv, ni);
        ci = make_float2(ci.x, fmaxf(ci.y, ni.y));
      } else {
        acc = seg_combine(acc, cur);
        cur = nv;
        ci = ni;
      }
    }
    acc = seg_combine(acc, cur);
  }
  return acc;
}

// One caller-given list through fold_ray_segments (one warp).
__global__ void fold_segments_kernel(const float4 *val, const float2 *iv, int n, float4 *out) {
  const float4 acc = fold_ray_segments(val, iv, n, threadIdx.x);
  if (threadIdx.x == 0) *out = acc;
}

// The per-ray kernels' warps draw runs of kRayRun consecutive rays from a
// counter (zeroed before the launch): a warp that is done takes the next run
// at once, whatever the other warps' lists.  Returns false when none is left.
constexpr int kRayRun = 8;
__device__ __forceinline__ bool next_rays(unsigned *ticket, long long npix, int lane,
                                          long long &pix, long long &pend) {
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(ticket, 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  pix = (long long)t * kRayRun;
  pend = pix + kRayRun < npix ? pix + kRayRun : npix;
  return pix < npix;
}

// Sorts every ray's list in place by its key (entry depth, then tree and
// Morton key through the leaf index): one warp per ray, in registers for lists
// of up to 512 keys, else bitonic in shared memory (cap keys per warp).
__global__ void __launch_bounds__(256)
    shell_sort_lists_kernel(const long long *__restrict__ ray_off, long long npix,
                            unsigned long long *keys, long long key_cap, int cap,
                            unsigned *ticket) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long *key = reinterpret_cast<unsigned long long *>(s_raw) + (size_t)wid * cap;
  for (long long pix = 0, pend = 0;; ++pix) {
    if (pix == pend) {  // the warp's next run of rays
      if (!next_rays(ticket, npix, lane, pix, pend)) break;
    }
    const long long h0 = ray_off[pix];
    const int n = (int)(ray_off[pix + 1] - h0);
    if (n < 2 || n > cap || h0 + n > key_cap) continue;  // the render counts the bad ones
    unsigned long long *lst = keys + h0;
    if (n <= 32) warp_sort_list<1, false>(lst, nullptr, n, lst, nullptr, n, lane);
    else if (n <= 64) warp_sort_list<2, false>(lst, nullptr, n, lst, nullptr, n, lane);
    else if (n <= 128) warp_sort_list<4, false>(lst, nullptr, n, lst, nullptr, n, lane);
    else if (n <= 256) warp_sort_list<8, false>(lst, nullptr, n, lst, nullptr, n, lane);
    else if (n <= 512) warp_sort_list<16, false>(lst, nullptr, n, lst, nullptr, n, lane);
    else {
      int P = 1024;
      while (P < n) P <<= 1;
      for (int k = lane; k < P; k += 32) key[k] = k < n ? lst[k] : ~0ull;
      __syncwarp();
      for (int sz = 2; sz <= P; sz <<= 1)
        for (int st = sz >> 1; st > 0; st >>= 1) {
          for (int k = lane; k < P; k += 32) {
            const int m = k ^ st;
            if (m > k) {
              const bool up = (k & sz) == 0;
              const unsigned long long a = key[k], b = key[m];
              if ((a > b) == up) {
                key[k] = b;
                key[m] = a;
              }
            }
          }
          __syncwarp();
        }
      for (int k = lane; k < n; k += 32) lst[k] = key[k];
      __syncwarp();
    }
  }
}

template <bool SURF>
__global__ void __launch_bounds__(256, 2)
    shell_rays_kernel(const int4 *__restrict__ geo, int N, Shell S, Field Fd, Cam c, Integ I,
                                  const long long *__restrict__ ray_off, long long npix,
                                  const unsigned long long *__restrict__ keys, long long key_cap,
                                  int cap, float4 *rgba, int *counts,
                                  unsigned long long *stats, unsigned *ticket) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  __shared__ float4 s_tfv[8], s_tfs[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  float4 *val = reinterpret_cast<float4 *>(s_raw) + (size_t)wid * cap;
  unsigned long long *key =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<float4 *>(s_raw) + (size_t)nw * cap) +
      (size_t)wid * cap;
  float2 *iv = reinterpret_cast<float2 *>(key);  // the intervals replace the keys once sorted
  const float bg[3] = {I.bg[0], I.bg[1], I.bg[2]};
  int steps = 0, segs = 0, errs = 0;
  for (long long pix = 0, pend = 0;; ++pix) {
    if (pix == pend) {  // the warp's next run of rays
      if (!next_rays(ticket, npix, lane, pix, pend)) break;
    }
    const long long h0 = ray_off[pix];
    const int n = (int)(ray_off[pix + 1] - h0);
    if (counts && lane == 0) counts[pix] = n;
    if (n == 0) {
      if (lane == 0) rgba[pix] = make_float4(bg[0], bg[1], bg[2], 0.f);
      continue;
    }
    if (n > cap || h0 + n > key_cap) {  // larger than planned: not rendered
      if (lane == 0) {
        ++errs;
        rgba[pix] = make_float4(bg[0], bg[1], bg[2], 0.f);
      }
      continue;
    }
    for (int k = lane; k < n; k += 32) key[k] = keys[h0 + k];  // sorted by shell_sort_lists
    __syncwarp();
    const int i = (int)(pix % c.w), j = (int)(pix / c.w);
    float3 org, dir;
    pixel_ray(c, i, j, org, dir);
    const float rl = sqrtf(fmaf(dir.x, dir.x, fmaf(dir.y, dir.y, dir.z * dir.z)));
    errs += shell_ray_values<SURF>(geo, N, S, Fd.nodal, c, I, tf, key, n, org, dir, rl, val, iv,
                             lane, steps);
    segs += n;
    __syncwarp();
    // overlaps of consecutive segments are rounding slivers, if any
    const float4 acc = fold_ray_segments(val, iv, n, lane);
    if (lane == 0)
      rgba[pix] = make_float4(fmaf(acc.x, bg[0], acc.y), fmaf(acc.x, bg[1], acc.z),
                              fmaf(acc.x, bg[2], acc.w), 1.f - acc.x);
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xffffffffu, steps, o);
  if (lane == 0) {
    atomicAdd(stats + kStatSegments, (unsigned long long)segs);
    atomicAdd(stats + kStatSteps, (unsigned long long)steps);
    if (errs) atomicAdd(stats + kStatErrors, (unsigned long long)errs);
  }
}

}  // namespace

// ------------------------------------------------------------- launchers --
cudaError_t shell_planes(const int4 *geo, int N, const Shell &S, float4 *planes,
                         cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int grid = (N + 255) / 256 > 8192 ? 8192 : (N + 255) / 256;
  shell_planes_kernel<<<grid, 256, 0, st>>>(geo, N, S, planes);
  return cudaGetLastError();
}

cudaError_t shell_monomials(const float *nodal, float *coef, int N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int need = (N + kMonoLeaves - 1) / kMonoLeaves;
  shell_monomial_kernel<<<need > 8192 ? 8192 : need, kMonoLeaves, 0, st>>>(nodal, coef, N);
  return cudaGetLastError();
}

cudaError_t shell_cull(const int4 *geo, int N, const Shell &S, const Cam &C, int4 *rect,
                       unsigned char *visible, unsigned long long *stats, cudaStream_t st) {
  const int grid = (N + 255) / 256 > 8192 ? 8192 : (N + 255) / 256;
  shell_cull_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(geo, N, S, C, rect, visible, stats);
  return cudaGetLastError();
}

cudaError_t shell_fold_segments(const float4 *val, const float2 *iv, int n, float4 *out,
                                cudaStream_t st) {
  if (n < 1 || !val || !iv || !out) return cudaErrorInvalidValue;
  fold_segments_kernel<<<1, 32, 0, st>>>(val, iv, n, out);
  return cudaGetLastError();
}

cudaError_t shell_pairs(int mode, const int4 *geo, int N, const Shell &S, const Cam &C,
                        const int4 *rect, const long long *leaf_off, const int *chunk_leaf,
                        long long npairs, int *counts, const long long *ray_off, int *cursor,
                        unsigned long long *keys, long long key_cap, unsigned long long *stats,
                        unsigned *hitmask, cudaStream_t st, unsigned *kpos, int2 *lm,
                        unsigned long long *lm_count) {
  if (mode < 0 || mode > 2 || (mode == 2 && (!kpos || !lm || !lm_count)))
    return cudaErrorInvalidValue;
  if (npairs > 0) {
    const long long nblk = (npairs + kPairChunk - 1) / kPairChunk;
    if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
    if (mode == 0)
      shell_pairs_kernel<0><<<(unsigned)nblk, kPairChunk, 0, st>>>(
          geo, N, S, C, rect, leaf_off, chunk_leaf, npairs, counts, ray_off, cursor, keys,
          key_cap, stats, hitmask, kpos, lm, lm_count);
    else if (mode == 1)
      shell_pairs_kernel<1><<<(unsigned)nblk, kPairChunk, 0, st>>>(
          geo, N, S, C, rect, leaf_off, chunk_leaf, npairs, counts, ray_off, cursor, keys,
          key_cap, stats, hitmask, kpos, lm, lm_count);
    else
      shell_pairs_kernel<2><<<(unsigned)nblk, kPairChunk, 0, st>>>(
          geo, N, S, C, rect, leaf_off, chunk_leaf, npairs, counts, ray_off, cursor, keys,
          key_cap, stats, hitmask, kpos, lm, lm_count);
  }
  if (mode == 0 && stats) {  // the longest list, for planning
    const long long npix = (long long)C.w * C.h;
    const long long g = (npix + 255) / 256;
    max_count_kernel<<<(unsigned)(g > 4096 ? 4096 : (g > 0 ? g : 1)), 256, 0, st>>>(counts, npix,
                                                                                 stats);
  }
  return cudaGetLastError();
}

// Warps per CTA of shell_rays: `want` if given (0: as many as fit), within
// 96 KB of shared memory (one warp at least).
int shell_ray_warps(int cap, int want) {
  const size_t per = (size_t)cap * (sizeof(float4) + sizeof(unsigned long long));
  int w = (int)((96u << 10) / per);
  w = w < 1 ? 1 : (w > 8 ? 8 : w);
  return (want > 0 && want < w) ? want : w;
}

size_t shell_ray_smem(int cap, int want) {
  return (size_t)shell_ray_warps(cap, want) * cap * (sizeof(float4) + sizeof(unsigned long long));
}

// warps per CTA of the sort kernel and its shared memory (only lists of more
// than 512 keys use it): within 96 KB
static int sort_warps(int cap) {
  if (cap <= 512) return 8;
  const int w = (int)((96u << 10) / ((size_t)cap * sizeof(unsigned long long)));
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

static size_t sort_smem(int cap) {
  return cap <= 512 ? 0 : (size_t)sort_warps(cap) * cap * sizeof(unsigned long long);
}

cudaError_t shell_rays_prepare() {
  size_t most = 0, most_sort = 0;  // the largest launch any list capacity asks for
  for (int cap = 32; cap <= kShellMaxCap; cap <<= 1) {
    most = most > shell_ray_smem(cap, 0) ? most : shell_ray_smem(cap, 0);
    most_sort = most_sort > sort_smem(cap) ? most_sort : sort_smem(cap);
  }
  cudaError_t e = cudaFuncSetAttribute(shell_rays_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(shell_rays_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)most);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(shell_sort_lists_kernel,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most_sort);
}

// CTAs of a kernel resident on the whole GPU at once (at least one).
template <class K>
static long long resident_ctas(K kernel, int threads, size_t smem, int nsm) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  return (long long)per * nsm;
}

cudaError_t shell_sort_lists(const long long *ray_off, long long npix, unsigned long long *keys,
                             long long key_cap, int cap, int nsm, unsigned *ticket,
                             cudaStream_t st) {
  if (cap < 32 || cap > kShellMaxCap || (cap & (cap - 1)) || !ticket)
    return cudaErrorInvalidValue;
  const int warps = sort_warps(cap);
  const long long need = (npix + (long long)warps * kRayRun - 1) / ((long long)warps * kRayRun);
  const long long res = resident_ctas(shell_sort_lists_kernel, warps * 32, sort_smem(cap), nsm);
  const long long grid = need < res ? need : res;
  shell_sort_lists_kernel<<<(unsigned)(grid > 0 ? grid : 1), warps * 32, sort_smem(cap), st>>>(
      ray_off, npix, keys, key_cap, cap, ticket);
  return cudaGetLastError();
}

cudaError_t shell_rays(const int4 *geo, int N, const Shell &S, const Field &Fd, const Cam &C,
                       const Integ &I, const long long *ray_off, long long npix,
                       const unsigned long long *keys, long long key_cap, int cap, float4 *rgba,
                       int *counts, unsigned long long *stats, int nsm, int want_warps,
                       unsigned *ticket, cudaStream_t st) {
  if (cap < 32 || cap > kShellMaxCap || (cap & (cap - 1)) || !ticket)
    return cudaErrorInvalidValue;
  const size_t smem = shell_ray_smem(cap, want_warps);
  const int warps = shell_ray_warps(cap, want_warps);
  const long long need = (npix + (long long)warps * kRayRun - 1) / ((long long)warps * kRayRun);
  const long long res = I.surface ? resident_ctas(shell_rays_kernel<true>, warps * 32, smem, nsm)
                                  : resident_ctas(shell_rays_kernel<false>, warps * 32, smem, nsm);
  const long long grid = need < res ? need : res;
  const unsigned g = (unsigned)(grid > 0 ? grid : 1);
  if (I.surface)  // the isosurface of Sec. 2.8: a separate instantiation
    shell_rays_kernel<true><<<g, warps * 32, smem, st>>>(geo, N, S, Fd, C, I, ray_off, npix, keys,
                                                         key_cap, cap, rgba, counts, stats,
                                                         ticket);
  else
    shell_rays_kernel<false><<<g, warps * 32, smem, st>>>(geo, N, S, Fd, C, I, ray_off, npix,
                                                          keys, key_cap, cap, rgba, counts, stats,
                                                          ticket);
  return cudaGetLastError();
}

}  // namespace ocr
