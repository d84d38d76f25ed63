// Adjoint of the render (ocr_render_backward), sm_103a.
//
// The gradient of a loss L(rgba) with respect to the nodal values and the
// transfer-function knots, given dL/d(rgba).  Segments are recomputed, not
// stored by the forward pass.  Cube forests:
//   pair_hits<0>     - over the (visible leaf, pixel) pairs of the leaves'
//                      rectangles in Morton order (a prefix sum of rectangle
//                      areas splits them into equal CTA chunks): slab tests,
//                      hits counted per ray (rays without an image adjoint
//                      are skipped);
//   (scan)           - per-ray offsets of the hit lists;
//   pair_hits<2>     - the same traversal, writing each hit's mirrored Morton
//                      key (the ray's front-to-back order) to its ray's list,
//                      and appending (pixel, leaf) to a list grouped by leaf
//                      whose index goes beside the key;
//   seg_values       - one thread per entry of the leaf-grouped list: the
//                      segment's value (A, B);
//   ray_scans        - one warp per ray: sort the keys, form the transmittance
//                      of the nearer segments (prefix product) and the
//                      aggregate of the farther ones with the background
//                      (suffix fold with Eq. 2.14) by warp scans -- no group
//                      inverse -- and store them per list entry;
//   seg_adjoint      - one thread per entry: the segment's adjoint through the
//                      integrator (RK4, or the Dormand-Prince steps of
//                      Algorithm 1 with the same step tree), the transfer
//                      function and the interpolation weights; the nodal
//                      adjoints are summed over a warp's lanes of the same
//                      leaf before the atomics.
// Shell forests use the render's lists, built with the leaf-grouped list, and
// the same three passes with the shell's geometry and field.
#include "ocr_common.h"
#include "ocr_device.cuh"
#include "ocr_shell.cuh"

namespace ocr {
namespace {

constexpr int kPairThreads = kPairChunk;

__device__ __forceinline__ long long area_of(int4 r) {
  return r.x > r.y ? 0ll : (long long)(r.y - r.x + 1) * (long long)(r.w - r.z + 1);
}

// ------------------------------------------------------------------ scans --
constexpr int kBScanThreads = 256, kBScanItems = 4, kBScanTile = kBScanThreads * kBScanItems;

struct LeafArea {
  const int4 *rect;
  __device__ long long operator()(long long k) const { return area_of(rect[k]); }
};
struct RayCount {
  const int *cnt;
  __device__ long long operator()(long long k) const { return (long long)cnt[k]; }
};
struct ListedLeafArea {  // the rectangle areas of the leaves listed in ids
  const int4 *rect;
  const int *ids;
  __device__ long long operator()(long long k) const { return area_of(rect[ids[k]]); }
};

__device__ long long block_excl_scan(long long v, long long *wt, long long &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < (int)(blockDim.x >> 5) ? wt[lane] : 0ll;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wt[lane] = w;
  }
  __syncthreads();
  total = wt[(blockDim.x >> 5) - 1];
  const long long r = (wid ? wt[wid - 1] : 0ll) + x - v;
  __syncthreads();
  return r;
}

template <class G>
__global__ void __launch_bounds__(kBScanThreads) bscan_reduce_kernel(G get, long long n,
                                                                      long long *bs) {
  __shared__ long long wt[32];
  const long long base = (long long)blockIdx.x * kBScanTile + threadIdx.x * kBScanItems;
  long long s = 0;
#pragma unroll
  for (int q = 0; q < kBScanItems; ++q)
    if (base + q < n) s += get(base + q);
  long long tot;
  block_excl_scan(s, wt, tot);
  if (threadIdx.x == 0) bs[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) bscan_sums_kernel(long long *bs, int nblk) {
  __shared__ long long wt[32];
  long long carry = 0;
  for (int b = 0; b < nblk; b += blockDim.x) {
    const int k = b + threadIdx.x;
    const long long v = k < nblk ? bs[k] : 0ll;
    long long tot;
    const long long ex = block_excl_scan(v, wt, tot);
    if (k < nblk) bs[k] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bs[nblk] = carry;
}

template <class G>
__global__ void __launch_bounds__(kBScanThreads) bscan_down_kernel(G get, long long n,
                                                                    const long long *bs, int nblk,
                                                                    long long *out) {
  __shared__ long long wt[32];
  const long long base = (long long)blockIdx.x * kBScanTile + threadIdx.x * kBScanItems;
  long long a[kBScanItems], s = 0;
#pragma unroll
  for (int q = 0; q < kBScanItems; ++q) {
    a[q] = base + q < n ? get(base + q) : 0ll;
    s += a[q];
  }
  long long tot;
  long long run = bs[blockIdx.x] + block_excl_scan(s, wt, tot);
#pragma unroll
  for (int q = 0; q < kBScanItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += a[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bs[nblk];
}

template <class G>
cudaError_t exclusive_scan(G get, long long n, long long *bs, long long bs_cap, long long *out,
                           cudaStream_t st) {
  const long long nblk = (n + kBScanTile - 1) / kBScanTile;
  if (nblk + 1 > bs_cap || nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  if (nblk == 0) return cudaMemsetAsync(out, 0, sizeof(long long), st);
  bscan_reduce_kernel<<<(unsigned)nblk, kBScanThreads, 0, st>>>(get, n, bs);
  bscan_sums_kernel<<<1, 1024, 0, st>>>(bs, (int)nblk);
  bscan_down_kernel<<<(unsigned)nblk, kBScanThreads, 0, st>>>(get, n, bs, (int)nblk, out);
  return cudaGetLastError();
}

// chunk_leaf[c] = the leaf whose pairs hold pair c * kPairThreads
__global__ void pair_chunk_map_kernel(const long long *off, int N, int *chunk_leaf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const long long a = off[k], b = off[k + 1];
    if (b <= a) continue;
    for (long long c = (a + kPairThreads - 1) / kPairThreads; c * kPairThreads < b; ++c)
      chunk_leaf[c] = k;
  }
}

// ----------------------------------------------------------- hit lists --
// MODE 0 counts hits per ray; MODE 2 writes keys[at] and appends the hit to
// the leaf-grouped list (one global append per CTA): lm[pos] = (pixel, leaf),
// kpos[at] = pos.
template <int MODE>
__global__ void __launch_bounds__(kPairThreads)
    pair_hits_kernel(Topo T, Cam c, const int4 *rect, const long long *leaf_off,
                     const int *chunk_leaf, long long npairs, const float4 *dL, int *counts,
                     const long long *ray_off, int *cursor, const unsigned long long *mkey,
                     unsigned long long fx, unsigned long long *keys, unsigned *kpos, int2 *lm,
                     unsigned long long *lm_count, long long key_cap, unsigned long long *err) {
  const long long p = (long long)blockIdx.x * kPairThreads + threadIdx.x;
  if (MODE == 0 && p >= npairs) return;
  bool hit = false;
  int leaf = 0;
  long long pix = 0;
  float3 dir = make_float3(0.f, 0.f, 0.f);
  if (p < npairs) {
    const long long nch = (npairs + kPairThreads - 1) / kPairThreads;
    int lo = chunk_leaf[blockIdx.x];
    int hi = (blockIdx.x + 1 < nch) ? chunk_leaf[blockIdx.x + 1] + 1 : T.N;
    while (lo + 1 < hi) {  // last leaf whose offset is <= p
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
    const float4 g = dL ? dL[pix] : make_float4(1.f, 0.f, 0.f, 0.f);  // no dL: every ray
    if (g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f) {  // else no gradient on this ray
      float3 org;
      pixel_ray(c, i, j, org, dir);
      const float3 inv =
          make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
      const int4 gl = T.geo[leaf];
      float a0, a1;
      hit = slab(org, dir, inv, node_lo(gl, exp2i(-T.L)), exp2i(-gl.w), c.amin,
                 c.amax, a0, a1);
    }
  }
  if (MODE == 0) {
    if (hit) atomicAdd(counts + pix, 1);
    return;
  }
  // this hit's place in the CTA's block of the leaf-grouped list
  __shared__ unsigned s_w[kPairThreads / 32], s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, hit);
  if (lane == 0) s_w[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kPairThreads / 32; ++w) {
      const unsigned t = s_w[w];
      s_w[w] = tot;
      tot += t;
    }
    s_base = tot ? (unsigned)atomicAdd(lm_count, (unsigned long long)tot) : 0u;
  }
  __syncthreads();
  if (!hit) return;
  const unsigned pos = s_base + s_w[wid] + __popc(bal & ((1u << lane) - 1u));
  const long long at = ray_off[pix] + atomicAdd(cursor + pix, 1);
  if (at >= key_cap || at >= ray_off[pix + 1] || (long long)pos >= key_cap) {
    atomicAdd(err, 1ull);  // more hits than counted
    if ((long long)pos < key_cap) lm[pos] = make_int2(-1, -1);
    return;
  }
  const unsigned long long flip =
      (dir.x < 0.f ? fx : 0ull) | (dir.y < 0.f ? fx << 1 : 0ull) | (dir.z < 0.f ? fx << 2 : 0ull);
  keys[at] = mkey[leaf] ^ flip;
  kpos[at] = pos;
  lm[pos] = make_int2((int)pix, leaf);
}

// -------------------------------------------------------- segment adjoint --
// Accumulates the adjoint of the transfer-function knots of consecutive
// evaluations that fall in the same knot interval in registers; on a change of
// interval they are added to this thread's own column of a shared [32][NT]
// array (no atomics), which the CTA sums at its end (knot_grad_flush).
struct TfGrad {
  int k = -1;
  float4 a0, a1;  // knot k, knot k + 1
  float *col;     // this thread's column: value v at col[v * stride]
  int stride;
  __device__ void flush() {
    if (k < 0) return;
    float *g = col + 4 * k * stride;
    g[0] += a0.x;
    g[stride] += a0.y;
    g[2 * stride] += a0.z;
    g[3 * stride] += a0.w;
    g[4 * stride] += a1.x;
    g[5 * stride] += a1.y;
    g[6 * stride] += a1.z;
    g[7 * stride] += a1.w;
    k = -1;
  }
  __device__ void add(int kk, float w, float4 v) {
    if (kk != k) {
      flush();
      k = kk;
      a0 = a1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float w0 = 1.f - w;
    a0.x = fmaf(w0, v.x, a0.x); a0.y = fmaf(w0, v.y, a0.y);
    a0.z = fmaf(w0, v.z, a0.z); a0.w = fmaf(w0, v.w, a0.w);
    a1.x = fmaf(w, v.x, a1.x); a1.y = fmaf(w, v.y, a1.y);
    a1.z = fmaf(w, v.z, a1.z); a1.w = fmaf(w, v.w, a1.w);
  }
};

// The CTA's knot adjoints: s_gt [32][NT] summed over the threads (each of the
// first 32 threads one value, the columns visited in a rotated order so that
// they hit distinct banks), one atomic per value.
template <int NT>
__device__ __forceinline__ void knot_grad_flush(const float *s_gt, float *g_tf) {
  __syncthreads();
  const int v = threadIdx.x;
  if (v < 32) {
    float sum = 0.f;
    for (int t = 0; t < NT; ++t) sum += s_gt[v * NT + ((t + v) & (NT - 1))];
    if (sum != 0.f) atomicAdd(g_tf + v, sum);
  }
}

// dL/ds at a field value s from vbar = dL/d(kappa, q) (the transfer
// function's slope; zero where it is clamped), after crediting the knots
__device__ __forceinline__ float tf_bwd(const TF &tf, float s, float4 vbar, TfGrad &tg) {
  const float zr = (s - tf.s_min) * tf.inv;
  const bool inside = zr > 0.f && zr < 7.f;
  const float z = fminf(fmaxf(zr, 0.f), 7.f);
  const int k = min((int)z, 6);
  const float w = z - (float)k;
  tg.add(k, w, vbar);
  if (!inside) return 0.f;
  const float4 d = tf.s[k];
  return (vbar.x * d.x + vbar.y * d.y + vbar.z * d.z + vbar.w * d.w) * tf.inv;
}

// Segment through a cube leaf: the field is the cubic in tau; the adjoint of
// the 8 corner values goes through the trilinear weights.
struct SegAdj {
  static constexpr int kUnroll = 6;
  Cubic cu;
  float3 uf, du;    // reference coordinates at the far end, change to the near end
  float g8[8];      // adjoint of the 8 nodal values
  __device__ __forceinline__ float4 kq(const TF &tf, float tau) const {
    return medium(cu, tf, tau);
  }
  // adjoint of the medium at tau: vbar = dL/d(kappa, q) there
  __device__ __forceinline__ void bwd(const TF &tf, float tau, float4 vbar, TfGrad &tg) {
    const float s = fmaf(fmaf(fmaf(cu.p3, tau, cu.p2), tau, cu.p1), tau, cu.p0);
    const float sb = tf_bwd(tf, s, vbar, tg);
    if (sb == 0.f) return;
    const float u = fmaf(tau, du.x, uf.x), v = fmaf(tau, du.y, uf.y), ww = fmaf(tau, du.z, uf.z);
    const float u0 = 1.f - u, v0 = 1.f - v, w0 = 1.f - ww;
    g8[0] = fmaf(sb, u0 * v0 * w0, g8[0]);
    g8[1] = fmaf(sb, u * v0 * w0, g8[1]);
    g8[2] = fmaf(sb, u0 * v * w0, g8[2]);
    g8[3] = fmaf(sb, u * v * w0, g8[3]);
    g8[4] = fmaf(sb, u0 * v0 * ww, g8[4]);
    g8[5] = fmaf(sb, u * v0 * ww, g8[5]);
    g8[6] = fmaf(sb, u0 * v * ww, g8[6]);
    g8[7] = fmaf(sb, u * v * ww, g8[7]);
  }
};

// Segment through a shell leaf: the field through the inverse map and the
// degree-2 polynomial (monomial coefficients); the adjoint of the 27 nodal
// values goes through the Lagrange weights and is kept in this thread's column
// of a shared-memory array (g27[q * stride]).
struct ShellAdj {
  static constexpr int kUnroll = 1;
  ShellSeg g;
  float *g27;
  int stride;
  __device__ __forceinline__ float4 kq(const TF &tf, float tau) const {
    return medium(g, tf, tau);
  }
  __device__ __forceinline__ void bwd(const TF &tf, float tau, float4 vbar, TfGrad &tg) {
    float u, v, w;
    const float s = shell_field(g, tau, u, v, w);
    const float sb = tf_bwd(tf, s, vbar, tg);
    if (sb == 0.f) return;
    float lu[3], lv[3], lw[3];  // d s / d(nodal value) = lu[a] lv[b] lw[c]
    quad_basis(u, lu);
    quad_basis(v, lv);
    quad_basis(w, lw);
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int by = 0; by < 3; ++by) {
        const float f = sb * lw[cz] * lv[by];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) g27[(9 * cz + 3 * by + ax) * stride] += f * lu[ax];
      }
  }
};

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// dL/d(kappa, q) at a node from the stage derivative adjoint Kb and stage value Y
__device__ __forceinline__ float4 node_vbar(float4 Kb, float4 Y) {
  return make_float4(-dot4(Kb, Y), Kb.y, Kb.z, Kb.w);
}

__device__ __forceinline__ float4 scale4(float a, float4 x) {
  return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}

// adjoint of one RK4 step from (1, 0) with nodes at t0, t0 + dt/2, t0 + dt,
// where the medium is k0, kh, k1 (as the forward step evaluated it)
template <class SA>
__device__ void rk4_step_bwd(SA &S, const TF &tf, float t0, float dt, float H, float4 ybar,
                             TfGrad &tg, float4 k0, float4 kh, float4 k1) {
  const float4 one = seg_identity();
  const float4 Y1 = one, K1 = rhs(k0, Y1);
  const float4 Y2 = axpy(0.5f * H, K1, one), K2 = rhs(kh, Y2);
  const float4 Y3 = axpy(0.5f * H, K2, one), K3 = rhs(kh, Y3);
  const float4 Y4 = axpy(H, K3, one);
  float4 K4b = scale4(H / 6.f, ybar), K3b = scale4(H / 3.f, ybar), K2b = scale4(H / 3.f, ybar),
         K1b = scale4(H / 6.f, ybar);
  S.bwd(tf, t0 + dt, node_vbar(K4b, Y4), tg);
  K3b = axpy(H, scale4(-k1.x, K4b), K3b);
  float4 vh = node_vbar(K3b, Y3);
  K2b = axpy(0.5f * H, scale4(-kh.x, K3b), K2b);
  const float4 v2 = node_vbar(K2b, Y2);
  vh = make_float4(vh.x + v2.x, vh.y + v2.y, vh.z + v2.z, vh.w + v2.w);
  S.bwd(tf, t0 + 0.5f * dt, vh, tg);
  K1b = axpy(0.5f * H, scale4(-kh.x, K2b), K1b);
  S.bwd(tf, t0, node_vbar(K1b, Y1), tg);
}

// adjoint of one Dormand-Prince step from (1, 0) (stages 1..6; the seventh
// stage only feeds the error estimate)
// (kq: the medium at the six nodes, as the forward step evaluated it)
template <class SA>
__device__ void dopri_step_bwd(SA &S, const TF &tf, float t0, float dtau, float H,
                               float4 ybar, TfGrad &tg, const float4 *kq) {
  const float4 one = seg_identity();
  const float tt[6] = {t0, fmaf(dp::c2, dtau, t0), fmaf(dp::c3, dtau, t0),
                       fmaf(dp::c4, dtau, t0), fmaf(dp::c5, dtau, t0), t0 + dtau};
  float4 Y[6], K[6];
  Y[0] = one;
  K[0] = rhs(kq[0], Y[0]);
  Y[1] = axpy(H * dp::a21, K[0], one);
  K[1] = rhs(kq[1], Y[1]);
  Y[2] = axpy(H, lin4(dp::a31, K[0], dp::a32, K[1]), one);
  K[2] = rhs(kq[2], Y[2]);
  float4 t = lin4(dp::a41, K[0], dp::a42, K[1]);
  t = axpy(dp::a43, K[2], t);
  Y[3] = axpy(H, t, one);
  K[3] = rhs(kq[3], Y[3]);
  t = lin4(dp::a51, K[0], dp::a52, K[1]);
  t = axpy(dp::a53, K[2], t);
  t = axpy(dp::a54, K[3], t);
  Y[4] = axpy(H, t, one);
  K[4] = rhs(kq[4], Y[4]);
  t = lin4(dp::a61, K[0], dp::a62, K[1]);
  t = axpy(dp::a63, K[2], t);
  t = axpy(dp::a64, K[3], t);
  t = axpy(dp::a65, K[4], t);
  Y[5] = axpy(H, t, one);
  const float b[6] = {dp::b1, 0.f, dp::b3, dp::b4, dp::b5, dp::b6};
  const float a[6][5] = {{0, 0, 0, 0, 0},
                         {dp::a21, 0, 0, 0, 0},
                         {dp::a31, dp::a32, 0, 0, 0},
                         {dp::a41, dp::a42, dp::a43, 0, 0},
                         {dp::a51, dp::a52, dp::a53, dp::a54, 0},
                         {dp::a61, dp::a62, dp::a63, dp::a64, dp::a65}};
  float4 Kb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) Kb[i] = scale4(H * b[i], ybar);
  // a shell node adjoint inlines the field and its 27 weights: one copy of it
  // in the code, the stages walked by a loop (SA::kUnroll = 1)
#pragma unroll SA::kUnroll
  for (int i = 5; i >= 0; --i) {
    S.bwd(tf, tt[i], node_vbar(Kb[i], Y[i]), tg);
    const float4 Yb = scale4(-kq[i].x, Kb[i]);
#pragma unroll
    for (int j = 0; j < i; ++j) Kb[j] = axpy(H * a[i][j], Yb, Kb[j]);
  }
}

// adjoints of the closed-form steps of Algorithm 1 over [t0, t0 + dtau] of
// tau (world length H), from ybar = dL/d(A, B) of the step.  The medium at
// the nodes is passed as the forward step evaluated it.
// Gauss-2 (Eqs. 2.32-2.33): A, B rational in (kappa, q) at the two nodes.
template <class SA>
__device__ void gauss2_step_bwd(SA &S, const TF &tf, float ta, float tb, float H, float4 g0,
                                float4 g1, float4 Sv, float4 ybar, TfGrad &tg) {
  const float a1 = 0.25f * H * (g0.x + g1.x), a2 = (H * H / 12.f) * g0.x * g1.x;
  const float den = 1.f + a1 + a2, inv = 1.f / den;
  const float h2 = H * H * 0.14433756729740644f;  // H^2 sqrt(3) / 12
  const float d0 = fmaf(H * H / 12.f, g1.x, 0.25f * H), d1 = fmaf(H * H / 12.f, g0.x, 0.25f * H);
  float4 v0, v1;
  v0.x = ybar.x * (2.f * a1 * d0 - 0.5f * H * den) * inv * inv;
  v1.x = ybar.x * (2.f * a1 * d1 - 0.5f * H * den) * inv * inv;
  const float q0[3] = {g0.y, g0.z, g0.w}, q1[3] = {g1.y, g1.z, g1.w};
  const float yb[3] = {ybar.y, ybar.z, ybar.w}, B[3] = {Sv.y, Sv.z, Sv.w};
  float w0[3], w1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v0.x += yb[c] * (h2 * q1[c] - B[c] * d0) * inv;
    v1.x += yb[c] * (-h2 * q0[c] - B[c] * d1) * inv;
    w0[c] = yb[c] * (0.5f * H - h2 * g1.x) * inv;
    w1[c] = yb[c] * (0.5f * H + h2 * g0.x) * inv;
  }
  v0.y = w0[0]; v0.z = w0[1]; v0.w = w0[2];
  v1.y = w1[0]; v1.z = w1[1]; v1.w = w1[2];
  S.bwd(tf, ta, v0, tg);
  S.bwd(tf, tb, v1, tg);
}

// Simpson's rule on the closed form (Eq. 2.34) and the Eq. 2.18 interface:
// nodes at the far end, midpoint and near end, A = exp(e) with
// e = -H (k_0 + 4 k_h + k_1) / 6; Simpson: B = H (A q_0 + 4 sqrt(A) q_h + q_1) / 6;
// Eq. 2.18: B = I_h (1 - A).
template <class SA>
__device__ void simpson_step_bwd(SA &S, const TF &tf, bool equilibrium, float t0, float dtau,
                                 float H, float4 k0, float4 kh, float4 k1, float A, float sa,
                                 float4 ybar, TfGrad &tg) {
  const float h6 = H / 6.f;
  float4 v0, vh, v1;
  if (equilibrium) {
    const float om = 1.f - A;
    const float Fe = A * (ybar.x - (ybar.y * kh.y + ybar.z * kh.z + ybar.w * kh.w));
    v0 = make_float4(-h6 * Fe, 0.f, 0.f, 0.f);
    v1 = v0;
    vh = make_float4(-4.f * h6 * Fe, ybar.y * om, ybar.z * om, ybar.w * om);
  } else {
    const float s0 = ybar.y * k0.y + ybar.z * k0.z + ybar.w * k0.w;
    const float sh = ybar.y * kh.y + ybar.z * kh.z + ybar.w * kh.w;
    const float Fe = fmaf(ybar.x, A, h6 * fmaf(s0, A, 2.f * sh * sa));
    const float w0 = h6 * A, wh = 4.f * h6 * sa;
    v0 = make_float4(-h6 * Fe, ybar.y * w0, ybar.z * w0, ybar.w * w0);
    vh = make_float4(-4.f * h6 * Fe, ybar.y * wh, ybar.z * wh, ybar.w * wh);
    v1 = make_float4(-h6 * Fe, ybar.y * h6, ybar.z * h6, ybar.w * h6);
  }
  S.bwd(tf, t0, v0, tg);
  S.bwd(tf, t0 + 0.5f * dtau, vh, tg);
  S.bwd(tf, t0 + dtau, v1, tg);
}

// adjoint of one step with value Sm, near transmittance Tm and far aggregate
// Gm (background folded in through bg): dL/d(A, B) of the step
__device__ __forceinline__ float4 step_adjoint(float Tm, float4 Gm, float4 Ib, float ab,
                                               const float *bg) {
  const float F0 = fmaf(Gm.x, bg[0], Gm.y), F1 = fmaf(Gm.x, bg[1], Gm.z),
              F2 = fmaf(Gm.x, bg[2], Gm.w);
  return make_float4(Tm * (Ib.x * F0 + Ib.y * F1 + Ib.z * F2 - ab * Gm.x), Tm * Ib.x, Tm * Ib.y,
                     Tm * Ib.z);
}

// The steps of one segment, revisited far to near with the forward's step
// tree: near transmittance Tn, far aggregate G (with the background folded in
// through bg), the segment's own transmittance Aseg.
// METHOD: the integrator (Integ::method: 0 RK4, 1 Dormand-Prince, 2 Gauss-2,
// 3 Simpson, 4 the Eq. 2.18 interface), a template parameter so that each
// kernel holds the registers of its own step adjoint only.
template <int METHOD, class SA>
__device__ void segment_steps_bwd(SA &S, const TF &tf, float dx, const Integ &I, float Tn,
                                  float4 G, float Aseg, float4 Ib, float ab, TfGrad &tg) {
  float4 acc = seg_identity();  // steps farther than the current one
  if constexpr (METHOD == 0) {
    const int n = I.nsteps;
    const float H = dx / (float)n, dt = 1.f / (float)n;
    for (int s = 0; s < n; ++s) {
      const float t0 = (float)s * dt, dts = (s + 1 == n) ? 1.f - t0 : dt;
      const float4 k0 = S.kq(tf, t0), kh = S.kq(tf, t0 + 0.5f * dts), k1 = S.kq(tf, t0 + dts);
      const float4 Sm = rk4_step(H, k0, kh, k1);
      const float4 accn = seg_combine(Sm, acc);
      const float Tm = Tn * (Aseg / accn.x);
      const float4 Gm = seg_combine(acc, G);
      rk4_step_bwd(S, tf, t0, dts, H, step_adjoint(Tm, Gm, Ib, ab, I.bg), tg, k0, kh, k1);
      acc = accn;
    }
    return;
  }
  int depth = 0;
  unsigned idx = 0;
  float4 kq0 = S.kq(tf, 0.f);
  const float4 one = seg_identity();
  if constexpr (METHOD != 1) {  // the closed forms inside Algorithm 1 (c_RK test alone)
    for (;;) {
      const float dtau = exp2i(-depth);
      const float t0 = (float)idx * dtau;
      const float H = dx * dtau;
      // the forward step (value, split test) exactly as integrate_segment
      float4 Sv, kq1 = kq0, g0, g1, kh;
      float kmax, A = 0.f, sa = 0.f;
      const float ta = fmaf(0.21132486540518713f, dtau, t0);
      const float tb = fmaf(0.78867513459481287f, dtau, t0);
      if constexpr (METHOD == 2) {
        g0 = S.kq(tf, ta);
        g1 = S.kq(tf, tb);
        const float a1 = 0.25f * H * (g0.x + g1.x), a2 = (H * H / 12.f) * g0.x * g1.x;
        const float inv = 1.f / (1.f + a1 + a2);
        const float h2 = H * H * 0.14433756729740644f;
        Sv.x = (1.f - a1 + a2) * inv;
        Sv.y = (0.5f * H * (g0.y + g1.y) + h2 * (g0.x * g1.y - g1.x * g0.y)) * inv;
        Sv.z = (0.5f * H * (g0.z + g1.z) + h2 * (g0.x * g1.z - g1.x * g0.z)) * inv;
        Sv.w = (0.5f * H * (g0.w + g1.w) + h2 * (g0.x * g1.w - g1.x * g0.w)) * inv;
        kmax = H * fmaxf(g0.x, g1.x);
      } else {
        kh = S.kq(tf, t0 + 0.5f * dtau);
        kq1 = S.kq(tf, t0 + dtau);
        const float e = -(H / 6.f) * (kq0.x + 4.f * kh.x + kq1.x);
        if constexpr (METHOD == 4) {
          const float om = -expm1f(e);
          A = 1.f - om;
          Sv = make_float4(A, kh.y * om, kh.z * om, kh.w * om);
        } else {
          sa = __expf(0.5f * e);
          A = sa * sa;
          const float w0 = (H / 6.f) * A, wh = (H / 6.f) * 4.f * sa, w1 = H / 6.f;
          Sv = make_float4(A, fmaf(w0, kq0.y, fmaf(wh, kh.y, w1 * kq1.y)),
                           fmaf(w0, kq0.z, fmaf(wh, kh.z, w1 * kq1.z)),
                           fmaf(w0, kq0.w, fmaf(wh, kh.w, w1 * kq1.w)));
        }
        kmax = H * fmaxf(fmaxf(kq0.x, kh.x), kq1.x);
      }
      if (depth < I.max_depth && kmax > I.c_rk) {
        ++depth;
        idx <<= 1;
        continue;
      }
      const float4 accn = seg_combine(Sv, acc);
      const float Tm = Tn * (Aseg / accn.x);
      const float4 Gm = seg_combine(acc, G);
      const float4 yb = step_adjoint(Tm, Gm, Ib, ab, I.bg);
      if constexpr (METHOD == 2)
        gauss2_step_bwd(S, tf, ta, tb, H, g0, g1, Sv, yb, tg);
      else
        simpson_step_bwd(S, tf, METHOD == 4, t0, dtau, H, kq0, kh, kq1, A, sa, yb, tg);
      acc = accn;
      kq0 = kq1;
      ++idx;
      while (depth > 0 && !(idx & 1u)) {
        idx >>= 1;
        --depth;
      }
      if (depth == 0) break;
    }
    return;
  }
  for (;;) {
    const float dtau = exp2i(-depth);
    const float t0 = (float)idx * dtau;
    const float H = dx * dtau;
    // the forward step (value, split test) exactly as integrate_segment
    const float4 kq2 = S.kq(tf, fmaf(dp::c2, dtau, t0));
    const float4 kq3 = S.kq(tf, fmaf(dp::c3, dtau, t0));
    const float4 kq4 = S.kq(tf, fmaf(dp::c4, dtau, t0));
    const float4 kq5 = S.kq(tf, fmaf(dp::c5, dtau, t0));
    const float4 kq6 = S.kq(tf, t0 + dtau);
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
    if (depth < I.max_depth && (H * kmax > I.c_rk || err > I.tol)) {
      ++depth;
      idx <<= 1;
      continue;
    }
    const float4 accn = seg_combine(Y5, acc);
    const float Tm = Tn * (Aseg / accn.x);
    const float4 Gm = seg_combine(acc, G);
    const float4 kq[6] = {kq0, kq2, kq3, kq4, kq5, kq6};
    dopri_step_bwd(S, tf, t0, dtau, H, step_adjoint(Tm, Gm, Ib, ab, I.bg), tg, kq);
    acc = accn;
    kq0 = kq6;
    ++idx;
    while (depth > 0 && !(idx & 1u)) {
      idx >>= 1;
      --depth;
    }
    if (depth == 0) break;
  }
}

// Adjoint of one segment of a cube leaf: near transmittance T, far aggregate
// G, its value A_seg; the adjoints of the leaf's 8 nodal values into g8.
template <int METHOD>
__device__ void segment_bwd(const Topo &T, const Field &Fd, const Cam &c, const Integ &I,
                            const TF &tf, int leaf, float3 org, float3 dir, float3 inv,
                            float scale, float Tn, float4 G, float Aseg, float4 Ib, float ab,
                            float *g8, TfGrad &tg) {
  const int4 g = __ldg(T.geo + leaf);
  const float ih = exp2i(g.w);
  const float3 lo = node_lo(g, scale);
  float a_in, a_out;
  slab(org, dir, inv, lo, exp2i(-g.w), c.amin, c.amax, a_in, a_out);
  SegAdj S;
  S.uf = make_float3((fmaf(a_out, dir.x, org.x) - lo.x) * ih,
                     (fmaf(a_out, dir.y, org.y) - lo.y) * ih,
                     (fmaf(a_out, dir.z, org.z) - lo.z) * ih);
  const float da = a_in - a_out;
  S.du = make_float3(da * dir.x * ih, da * dir.y * ih, da * dir.z * ih);
  const float dx =
      fmaxf(a_out - a_in, 0.f) * sqrtf(dir.x * dir.x + dir.y * dir.y + dir.z * dir.z);
  S.cu = field_cubic(Fd.nodal + 8 * (size_t)leaf, S.uf, S.du);
#pragma unroll
  for (int q = 0; q < 8; ++q) S.g8[q] = 0.f;
  segment_steps_bwd<METHOD>(S, tf, dx, I, Tn, G, Aseg, Ib, ab, tg);
#pragma unroll
  for (int q = 0; q < 8; ++q) g8[q] = S.g8[q];
}

// ------------------------------------------------------------ ray adjoint --
// Over a ray's n segment values val[0..n) (nearest first), one warp: the
// transmittance of the nearer segments Tk (exclusive product of A), the
// segment's own Ak, and, in place of val, the aggregate of the farther ones
// (suffix fold with Eq. 2.14) -- no group inverse.
__device__ void near_far_scans(int n, int lane, float4 *val, float *Tk, float *Ak) {
  float carry = 1.f;
  const int nb = (n + 31) / 32;
  for (int b = 0; b < nb; ++b) {
    const int k = b * 32 + lane;
    const float a = k < n ? val[k].x : 1.f;
    float x = a;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x *= y;
    }
    float ex = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) ex = 1.f;
    if (k < n) {
      Tk[k] = carry * ex;
      Ak[k] = a;
    }
    carry *= __shfl_sync(0xffffffffu, x, 31);
  }
  __syncwarp();
  float4 fc = seg_identity();
  for (int b = nb - 1; b >= 0; --b) {
    const int k = b * 32 + lane;
    float4 x = k < n ? val[k] : seg_identity();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      float4 y;
      y.x = __shfl_down_sync(0xffffffffu, x.x, o);
      y.y = __shfl_down_sync(0xffffffffu, x.y, o);
      y.z = __shfl_down_sync(0xffffffffu, x.z, o);
      y.w = __shfl_down_sync(0xffffffffu, x.w, o);
      if (lane + o < 32) x = seg_combine(x, y);
    }
    float4 nx;
    nx.x = __shfl_down_sync(0xffffffffu, x.x, 1);
    nx.y = __shfl_down_sync(0xffffffffu, x.y, 1);
    nx.z = __shfl_down_sync(0xffffffffu, x.z, 1);
    nx.w = __shfl_down_sync(0xffffffffu, x.w, 1);
    if (lane == 31) nx = seg_identity();
    const float4 Gk = seg_combine(nx, fc);
    float4 x0;
    x0.x = __shfl_sync(0xffffffffu, x.x, 0);
    x0.y = __shfl_sync(0xffffffffu, x.y, 0);
    x0.z = __shfl_sync(0xffffffffu, x.z, 0);
    x0.w = __shfl_sync(0xffffffffu, x.w, 0);
    __syncwarp();
    if (k < n) val[k] = Gk;
    fc = seg_combine(x0, fc);
  }
  __syncwarp();
}

// bitonic sort of keys[0..P) (P a power of two >= 32) by one warp, ascending,
// carrying an int payload when lf is not null
__device__ void warp_sort(unsigned long long *key, int *lf, int P, int lane) {
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
            if (lf) {
              const int t = lf[k];
              lf[k] = lf[m];
              lf[m] = t;
            }
          }
        }
      }
      __syncwarp();
    }
}

// The transfer-function table of a CTA in shared memory.
__device__ __forceinline__ void load_tf(const Field &Fd, float4 *s_tfv, float4 *s_tfs) {
  const int tid = threadIdx.x;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
}

__device__ __forceinline__ bool nonzero4(float4 g) {
  return g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f;
}

constexpr int kSegThreads = 128;
constexpr int kSegStride = kSegThreads + 1;  // row stride: lanes summing rows hit distinct banks
static_assert((kSegThreads & (kSegThreads - 1)) == 0, "rotated column order needs a power of two");

// The CTA's contiguous range [b, end) of the nseg list entries, whole
// multiples of kSegThreads: consecutive entries of a thread then belong to
// nearby leaves (coherent knot intervals and nodal data).
__device__ __forceinline__ void seg_range(long long nseg, long long &b, long long &end) {
  const long long per =
      ((nseg + gridDim.x - 1) / gridDim.x + kSegThreads - 1) / kSegThreads * kSegThreads;
  b = (long long)blockIdx.x * per;
  end = b + per < nseg ? b + per : nseg;
}

// Pass 1, one thread per entry e of the leaf-grouped list (pixel, leaf): the
// segment's value (A, B) into val[e].  Cube leaves.
__global__ void __launch_bounds__(kSegThreads)
    cube_seg_values_kernel(Topo T, Field Fd, Cam c, Integ I, const int2 *lm, long long nseg,
                           const unsigned long long *ncount, float4 *val) {
  if (ncount) nseg = min(nseg, (long long)*ncount);  // the entries written, within the capacity
  __shared__ float4 s_tfv[8], s_tfs[8];
  load_tf(Fd, s_tfv, s_tfs);
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  const float scale = exp2i(-T.L);
  const long long npix = (long long)c.w * c.h;
  int steps = 0;
  for (long long e = (long long)blockIdx.x * kSegThreads + threadIdx.x; e < nseg;
       e += (long long)gridDim.x * kSegThreads) {
    const int2 m = lm[e];
    if (m.x < 0 || (long long)m.x >= npix || m.y < 0 || m.y >= T.N) continue;
    float3 org, dir;
    pixel_ray(c, m.x % c.w, m.x / c.w, org, dir);
    const float3 inv =
        make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
    val[e] = leaf_segment(T, Fd, c, I, tf, m.y, org, dir, inv, scale, steps);
  }
}

// The same for shell leaves: entries (pixel, 2 leaf + piece); rays without an
// image adjoint are skipped.  A piece the ray does not have is counted in err.
__global__ void __launch_bounds__(kSegThreads)
    shell_seg_values_kernel(const int4 *__restrict__ geo, int N, Shell S, Field Fd, Cam c,
                            Integ I, const float4 *dL, const int2 *lm, long long nseg,
                            float4 *val, unsigned long long *err) {
  __shared__ float4 s_tfv[8], s_tfs[8];
  load_tf(Fd, s_tfv, s_tfs);
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  const long long npix = (long long)c.w * c.h;
  int steps = 0, bad = 0;
  for (long long e = (long long)blockIdx.x * kSegThreads + threadIdx.x; e < nseg;
       e += (long long)gridDim.x * kSegThreads) {
    const int2 m = lm[e];
    const int lf = m.y >> 1, piece = m.y & 1;
    if (m.x < 0 || (long long)m.x >= npix || m.y < 0 || lf >= N) continue;
    if (!nonzero4(dL[m.x])) continue;
    float3 org, dir;
    pixel_ray(c, m.x % c.w, m.x / c.w, org, dir);
    const float rl = sqrtf(fmaf(dir.x, dir.x, fmaf(dir.y, dir.y, dir.z * dir.z)));
    ShellSeg g;
    float dx;
    float2 iv;
    if (!shell_segment(S, Fd.nodal, c, __ldg(geo + lf), lf, piece, org, dir, rl, g, dx, iv)) {
      ++bad;
      val[e] = seg_identity();
      continue;
    }
    val[e] = integrate_segment(g, tf, dx, I, steps);
  }
  if (bad) atomicAdd(err, (unsigned long long)bad);
}

// Pass 2, one warp per ray: sort the ray's keys (nearest first), carrying each
// segment's index in the leaf-grouped list; gather the segment values there
// (from rec_g), and store there the transmittance of the nearer segments and
// the segment's own (rec_ta) and the aggregate of the farther ones (rec_g).
// Rays without an image adjoint are skipped.  Geometry-free.
__global__ void __launch_bounds__(256)
    ray_scans_kernel(Cam c, const float4 *dL, const long long *ray_off, const int *count,
                     const unsigned long long *keys, const unsigned *kpos, long long key_cap,
                     int cap, float2 *rec_ta, float4 *rec_g, unsigned long long *err) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float4 *val = reinterpret_cast<float4 *>(s_raw) + (size_t)wid * cap;
  unsigned long long *key =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<float4 *>(s_raw) + (size_t)nw * cap) +
      (size_t)wid * cap;
  int *pos = reinterpret_cast<int *>(reinterpret_cast<unsigned long long *>(
                 reinterpret_cast<float4 *>(s_raw) + (size_t)nw * cap) + (size_t)nw * cap) +
             (size_t)wid * cap;
  float *Tk = reinterpret_cast<float *>(key);  // reuses the key array after sorting
  float *Ak = reinterpret_cast<float *>(key) + cap;
  const long long npix = (long long)c.w * c.h;
  const long long nwarp = (long long)gridDim.x * nw;
  int bad = 0;
  for (long long pix = (long long)blockIdx.x * nw + wid; pix < npix; pix += nwarp) {
    const long long h0 = ray_off[pix];
    const int n = count ? count[pix] : (int)(ray_off[pix + 1] - h0);
    if (n == 0) continue;
    if (n > cap || h0 + n > key_cap) {
      if (lane == 0) ++bad;
      continue;
    }
    if (!nonzero4(dL[pix])) continue;
    if (n <= 32) {  // one entry per lane: sort and scans in registers
      unsigned long long kk = lane < n ? keys[h0 + lane] : ~0ull;
      int q = lane < n ? (int)kpos[h0 + lane] : -1;
      for (int sz = 2; sz <= 32; sz <<= 1)  // bitonic, ascending; keys are distinct
        for (int st = sz >> 1; st > 0; st >>= 1) {
          const unsigned long long ok = __shfl_xor_sync(0xffffffffu, kk, st);
          const int oq = __shfl_xor_sync(0xffffffffu, q, st);
          const bool low = (lane & st) == 0, up = (lane & sz) == 0;
          if (low == up ? ok < kk : ok > kk) {
            kk = ok;
            q = oq;
          }
        }
      const bool live = lane < n && (long long)(unsigned)q < key_cap;
      const float4 v = live ? rec_g[(unsigned)q] : seg_identity();
      float x = v.x;  // transmittance of this and the nearer segments
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x *= y;
      }
      float tn = __shfl_up_sync(0xffffffffu, x, 1);
      if (lane == 0) tn = 1.f;
      float4 f = v;  // this and the farther segments, Eq. 2.14
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        float4 y;
        y.x = __shfl_down_sync(0xffffffffu, f.x, o);
        y.y = __shfl_down_sync(0xffffffffu, f.y, o);
        y.z = __shfl_down_sync(0xffffffffu, f.z, o);
        y.w = __shfl_down_sync(0xffffffffu, f.w, o);
        if (lane + o < 32) f = seg_combine(f, y);
      }
      float4 g;
      g.x = __shfl_down_sync(0xffffffffu, f.x, 1);
      g.y = __shfl_down_sync(0xffffffffu, f.y, 1);
      g.z = __shfl_down_sync(0xffffffffu, f.z, 1);
      g.w = __shfl_down_sync(0xffffffffu, f.w, 1);
      if (lane == 31) g = seg_identity();
      if (live) {
        rec_ta[(unsigned)q] = make_float2(tn, v.x);
        rec_g[(unsigned)q] = g;
      }
      continue;
    }
    int P = 64;
    while (P < n) P <<= 1;
    if (P <= 256) {  // sorted in registers
      if (P == 64) warp_sort_list<2, true>(keys + h0, kpos + h0, n, key, pos, P, lane);
      else if (P == 128) warp_sort_list<4, true>(keys + h0, kpos + h0, n, key, pos, P, lane);
      else warp_sort_list<8, true>(keys + h0, kpos + h0, n, key, pos, P, lane);
    } else {
      for (int k = lane; k < P; k += 32) {
        key[k] = k < n ? keys[h0 + k] : ~0ull;
        pos[k] = k < n ? (int)kpos[h0 + k] : -1;
      }
      __syncwarp();
      warp_sort(key, pos, P, lane);
    }
    for (int k = lane; k < n; k += 32) {
      const unsigned q = (unsigned)pos[k];
      val[k] = (long long)q < key_cap ? rec_g[q] : seg_identity();
    }
    __syncwarp();
    near_far_scans(n, lane, val, Tk, Ak);
    for (int k = lane; k < n; k += 32) {
      const unsigned q = (unsigned)pos[k];
      if ((long long)q < key_cap) {
        rec_ta[q] = make_float2(Tk[k], Ak[k]);
        rec_g[q] = val[k];
      }
    }
    __syncwarp();
  }
  if (bad) atomicAdd(err, (unsigned long long)bad);
}

// Sums the NV nodal adjoints in the shared columns (row stride kSegStride) of
// the warp's lanes over the lanes that hold the same leaf (leaf < 0: nothing),
// one atomic per value and leaf.
template <int NV>
__device__ __forceinline__ void leaf_group_flush(const float *s_rows, int leaf, int lane, int wid,
                                                 float *g_nodal) {
  unsigned todo = __ballot_sync(0xffffffffu, leaf >= 0);
  while (todo) {
    const int lf = __shfl_sync(0xffffffffu, leaf, __ffs(todo) - 1);
    const unsigned grp = __ballot_sync(0xffffffffu, leaf == lf);
    todo &= ~grp;
    if (lane < NV) {
      const float *row = s_rows + lane * kSegStride + (wid << 5);
      float sum = 0.f;
      for (unsigned mm = grp; mm; mm &= mm - 1) sum += row[__ffs(mm) - 1];
      if (sum != 0.f) atomicAdd(g_nodal + NV * (size_t)lf + lane, sum);
    }
  }
}

// Pass 3, one thread per entry of the leaf-grouped list: the segment's step
// adjoints with the near transmittance and far aggregate of pass 2, through
// the trilinear weights; the 8 nodal adjoints summed over the warp's lanes of
// the same leaf (the list keeps a leaf's segments together).  Cube leaves.
template <int METHOD>
__global__ void __launch_bounds__(kSegThreads, 4)
    cube_seg_adjoint_kernel(Topo T, Field Fd, Cam c, Integ I, const float4 *dL, const int2 *lm,
                            const float2 *rec_ta, const float4 *rec_g, long long nseg,
                            const unsigned long long *ncount, float *g_nodal, float *g_tf) {
  if (ncount) nseg = min(nseg, (long long)*ncount);  // the entries written, within the capacity
  __shared__ float s_g8[8 * kSegStride];
  __shared__ float s_gt[32 * kSegThreads];
  __shared__ float4 s_tfv[8], s_tfs[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  load_tf(Fd, s_tfv, s_tfs);
#pragma unroll
  for (int v = 0; v < 32; ++v) s_gt[v * kSegThreads + tid] = 0.f;
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  TfGrad tg;
  tg.col = s_gt + tid;
  tg.stride = kSegThreads;
  const float scale = exp2i(-T.L);
  const long long npix = (long long)c.w * c.h;
  long long b, end;
  seg_range(nseg, b, end);
  for (; b < end; b += kSegThreads) {
    const long long e = b + tid;
    int leaf = -1;
    if (e < end) {
      const int2 m = lm[e];
      if (m.x >= 0 && (long long)m.x < npix && m.y >= 0 && m.y < T.N) {
        const float4 gp = dL[m.x];
        float3 org, dir;
        pixel_ray(c, m.x % c.w, m.x / c.w, org, dir);
        const float3 inv =
            make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
        const float2 ta = rec_ta[e];
        float g8[8];
        segment_bwd<METHOD>(T, Fd, c, I, tf, m.y, org, dir, inv, scale, ta.x, rec_g[e], ta.y,
                    make_float4(gp.x, gp.y, gp.z, 0.f), gp.w, g8, tg);
#pragma unroll
        for (int q = 0; q < 8; ++q) s_g8[q * kSegStride + tid] = g8[q];
        leaf = m.y;
      }
    }
    __syncwarp();
    leaf_group_flush<8>(s_g8, leaf, lane, wid, g_nodal);
    __syncwarp();
  }
  tg.flush();
  knot_grad_flush<kSegThreads>(s_gt, g_tf);
}

// The same for shell leaves: the field through the inverse map and the
// degree-2 weights; the 27 nodal adjoints go to this thread's column of the
// shared array directly.  Rays without an image adjoint are skipped.
template <int METHOD>
__global__ void __launch_bounds__(kSegThreads, 4)
    shell_seg_adjoint_kernel(const int4 *__restrict__ geo, int N, Shell S, Field Fd, Cam c,
                             Integ I, const float4 *dL, const int2 *lm, const float2 *rec_ta,
                             const float4 *rec_g, long long nseg, float *g_nodal, float *g_tf) {
  __shared__ float s_g27[27 * kSegStride];
  __shared__ float s_gt[32 * kSegThreads];
  __shared__ float4 s_tfv[8], s_tfs[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  load_tf(Fd, s_tfv, s_tfs);
#pragma unroll
  for (int v = 0; v < 32; ++v) s_gt[v * kSegThreads + tid] = 0.f;
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  TfGrad tg;
  tg.col = s_gt + tid;
  tg.stride = kSegThreads;
  const long long npix = (long long)c.w * c.h;
  float *g27 = s_g27 + tid;
  long long b, end;
  seg_range(nseg, b, end);
  for (; b < end; b += kSegThreads) {
    const long long e = b + tid;
#pragma unroll
    for (int q = 0; q < 27; ++q) g27[q * kSegStride] = 0.f;
    int leaf = -1;
    if (e < end) {
      const int2 m = lm[e];
      const int lf = m.y >> 1, piece = m.y & 1;
      if (m.x >= 0 && (long long)m.x < npix && m.y >= 0 && lf < N) {
        const float4 gp = dL[m.x];
        if (nonzero4(gp)) {
          float3 org, dir;
          pixel_ray(c, m.x % c.w, m.x / c.w, org, dir);
          const float rl = sqrtf(fmaf(dir.x, dir.x, fmaf(dir.y, dir.y, dir.z * dir.z)));
          ShellAdj A;
          float dx;
          float2 iv;
          if (shell_segment(S, Fd.nodal, c, __ldg(geo + lf), lf, piece, org, dir, rl, A.g, dx,
                            iv)) {
            A.g27 = g27;
            A.stride = kSegStride;
            const float2 ta = rec_ta[e];
            segment_steps_bwd<METHOD>(A, tf, dx, I, ta.x, rec_g[e], ta.y,
                              make_float4(gp.x, gp.y, gp.z, 0.f), gp.w, tg);
            leaf = lf;
          }
        }
      }
    }
    __syncwarp();
    leaf_group_flush<27>(s_g27, leaf, lane, wid, g_nodal);
    __syncwarp();
  }
  tg.flush();
  knot_grad_flush<kSegThreads>(s_gt, g_tf);
}

}  // namespace

// ------------------------------------------------------------- launchers --
cudaError_t bwd_leaf_scan(const Topo &T, const int4 *rect, long long *bs, long long bs_cap,
                          long long *leaf_off, cudaStream_t st) {
  return exclusive_scan(LeafArea{rect}, (long long)T.N, bs, bs_cap, leaf_off, st);
}

cudaError_t listed_leaf_scan(const int4 *rect, const int *ids, long long n, long long *bs,
                             long long bs_cap, long long *off, cudaStream_t st) {
  return exclusive_scan(ListedLeafArea{rect, ids}, n, bs, bs_cap, off, st);
}

cudaError_t bwd_count_scan(const int *counts, long long n, long long *bs, long long bs_cap,
                           long long *ray_off, cudaStream_t st) {
  return exclusive_scan(RayCount{counts}, n, bs, bs_cap, ray_off, st);
}

long long bwd_scan_blocks(long long n) { return (n + kBScanTile - 1) / kBScanTile; }

cudaError_t bwd_chunk_map(const long long *leaf_off, int N, int *chunk_leaf, cudaStream_t st) {
  const int grid = (int)((N + 255) / 256 > 4096 ? 4096 : (N + 255) / 256);
  pair_chunk_map_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(leaf_off, N, chunk_leaf);
  return cudaGetLastError();
}

cudaError_t bwd_pair_hits(int mode, const Topo &T, const Cam &C, const int4 *rect,
                          const long long *leaf_off, const int *chunk_leaf, long long npairs,
                          const float4 *dL, int *counts, const long long *ray_off, int *cursor,
                          const unsigned long long *mkey, unsigned long long fx,
                          unsigned long long *keys, unsigned *kpos, int2 *lm,
                          unsigned long long *lm_count, long long key_cap,
                          unsigned long long *err, cudaStream_t st) {
  if (mode != 0 && mode != 2) return cudaErrorInvalidValue;
  if (npairs <= 0) return cudaSuccess;
  const long long nblk = (npairs + kPairThreads - 1) / kPairThreads;
  if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  if (mode == 0)
    pair_hits_kernel<0><<<(unsigned)nblk, kPairThreads, 0, st>>>(
        T, C, rect, leaf_off, chunk_leaf, npairs, dL, counts, ray_off, cursor, mkey, fx, keys,
        kpos, lm, lm_count, key_cap, err);
  else
    pair_hits_kernel<2><<<(unsigned)nblk, kPairThreads, 0, st>>>(
        T, C, rect, leaf_off, chunk_leaf, npairs, dL, counts, ray_off, cursor, mkey, fx, keys,
        kpos, lm, lm_count, key_cap, err);
  return cudaGetLastError();
}

// err += the device error counter of the render passes (one thread)
__global__ void fold_errors_kernel(unsigned long long *err, const unsigned long long *stat_err) {
  if (*stat_err) *err += *stat_err;
}

cudaError_t bwd_fold_errors(unsigned long long *err, const unsigned long long *stat_err,
                            cudaStream_t st) {
  fold_errors_kernel<<<1, 1, 0, st>>>(err, stat_err);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) hits_max_kernel(const int *counts, long long n,
                                                       unsigned long long *out) {
  int m = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    m = max(m, counts[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, (unsigned long long)m);
}

cudaError_t bwd_max_hits(const int *counts, long long n, unsigned long long *out,
                         cudaStream_t st) {
  const long long g = (n + 255) / 256;
  hits_max_kernel<<<(unsigned)(g > 4096 ? 4096 : (g > 0 ? g : 1)), 256, 0, st>>>(counts, n, out);
  return cudaGetLastError();
}

// grid of the per-entry passes: one thread per entry, at most `per_sm` CTAs
// per SM (grid-stride beyond)
static unsigned seg_grid(long long nseg, int nsm, int per_sm) {
  const long long need = (nseg + kSegThreads - 1) / kSegThreads;
  const long long most = (long long)nsm * per_sm;
  return (unsigned)(need < most ? need : most);
}

cudaError_t bwd_cube_values(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                            const int2 *lm, long long nseg, const unsigned long long *ncount,
                            float4 *val, int nsm, cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  cube_seg_values_kernel<<<seg_grid(nseg, nsm, 16), kSegThreads, 0, st>>>(T, Fd, C, I, lm, nseg,
                                                                          ncount, val);
  return cudaGetLastError();
}

cudaError_t bwd_shell_values(const int4 *geo, int N, const Shell &S, const Field &Fd,
                             const Cam &C, const Integ &I, const float4 *dL, const int2 *lm,
                             long long nseg, float4 *val, unsigned long long *err, int nsm,
                             cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  shell_seg_values_kernel<<<seg_grid(nseg, nsm, 16), kSegThreads, 0, st>>>(
      geo, N, S, Fd, C, I, dL, lm, nseg, val, err);
  return cudaGetLastError();
}

// warps per CTA of the per-ray scans: up to 8, within 200 KB of shared memory
static int scans_warps(int cap) {
  const size_t per = (size_t)cap * (sizeof(float4) + sizeof(unsigned long long) + sizeof(int));
  const int w = (int)((200u << 10) / per);
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

size_t bwd_scans_smem(int cap) {
  return (size_t)scans_warps(cap) * cap *
         (sizeof(float4) + sizeof(unsigned long long) + sizeof(int));
}

cudaError_t bwd_scans_prepare() {
  size_t most = 0;
  for (int cap = 32; cap <= kShellMaxCap; cap <<= 1)
    most = most > bwd_scans_smem(cap) ? most : bwd_scans_smem(cap);
  return cudaFuncSetAttribute(ray_scans_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)most);
}

cudaError_t bwd_ray_scans(const Cam &C, const float4 *dL, const long long *ray_off,
                          const int *count, const unsigned long long *keys, const unsigned *kpos,
                          long long key_cap, int cap, float2 *rec_ta, float4 *rec_g,
                          unsigned long long *err, int nsm, cudaStream_t st) {
  if (cap < 32 || cap > kShellMaxCap || (cap & (cap - 1))) return cudaErrorInvalidValue;
  const int warps = scans_warps(cap);
  const long long npix = (long long)C.w * C.h;
  const long long need = (npix + warps - 1) / warps;
  const long long grid = need < (long long)nsm * 8 ? need : (long long)nsm * 8;
  ray_scans_kernel<<<(unsigned)(grid > 0 ? grid : 1), warps * 32, bwd_scans_smem(cap), st>>>(
      C, dL, ray_off, count, keys, kpos, key_cap, cap, rec_ta, rec_g, err);
  return cudaGetLastError();
}

cudaError_t bwd_cube_adjoint(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                             const float4 *dL, const int2 *lm, const float2 *rec_ta,
                             const float4 *rec_g, long long nseg,
                             const unsigned long long *ncount, float *g_nodal, float *g_tf,
                             int nsm, cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  const unsigned g = seg_grid(nseg, nsm, 16);
  switch (I.method) {  // one kernel per integrator
    case 0: cube_seg_adjoint_kernel<0><<<g, kSegThreads, 0, st>>>(
                T, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, ncount, g_nodal, g_tf); break;
    case 1: cube_seg_adjoint_kernel<1><<<g, kSegThreads, 0, st>>>(
                T, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, ncount, g_nodal, g_tf); break;
    case 2: cube_seg_adjoint_kernel<2><<<g, kSegThreads, 0, st>>>(
                T, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, ncount, g_nodal, g_tf); break;
    case 3: cube_seg_adjoint_kernel<3><<<g, kSegThreads, 0, st>>>(
                T, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, ncount, g_nodal, g_tf); break;
    case 4: cube_seg_adjoint_kernel<4><<<g, kSegThreads, 0, st>>>(
                T, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, ncount, g_nodal, g_tf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t bwd_shell_adjoint(const int4 *geo, int N, const Shell &S, const Field &Fd,
                              const Cam &C, const Integ &I, const float4 *dL, const int2 *lm,
                              const float2 *rec_ta, const float4 *rec_g, long long nseg,
                              float *g_nodal, float *g_tf, int nsm, cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  const unsigned g = seg_grid(nseg, nsm, 16);
  switch (I.method) {  // one kernel per integrator
    case 0: shell_seg_adjoint_kernel<0><<<g, kSegThreads, 0, st>>>(
                geo, N, S, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, g_nodal, g_tf); break;
    case 1: shell_seg_adjoint_kernel<1><<<g, kSegThreads, 0, st>>>(
                geo, N, S, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, g_nodal, g_tf); break;
    case 2: shell_seg_adjoint_kernel<2><<<g, kSegThreads, 0, st>>>(
                geo, N, S, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, g_nodal, g_tf); break;
    case 3: shell_seg_adjoint_kernel<3><<<g, kSegThreads, 0, st>>>(
                geo, N, S, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, g_nodal, g_tf); break;
    case 4: shell_seg_adjoint_kernel<4><<<g, kSegThreads, 0, st>>>(
                geo, N, S, Fd, C, I, dL, lm, rec_ta, rec_g, nseg, g_nodal, g_tf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ocr
