// The chunk passes of the cube render as device functions: the subtree pass
// (Sec. 3.2 and Sec. 3.3 below the tile level), a coarsening level (Sec. 3.3)
// and the pixel pass.  One call does one CTA's chunk; the standalone kernels
// (ocr_kernels.cu) call them once per CTA, the persistent batch kernel
// (ocr_batch.cu) once per work item it draws.
#pragma once
#include "ocr_common.h"
#include "ocr_device.cuh"

namespace ocr {
namespace {

// ---------------------------------------------------------------- coarsen --
constexpr int kCoarsenThreads = kChunk;

// Loads of the per-render scratch.  The rectangles, slot offsets and chunk
// map (ldp) are complete before any chunk of a pass reads them: the read-only
// path serves the single-camera kernels (written by earlier launches); in the
// persistent batch kernel (COH) they were written earlier in the same launch,
// but every item that reads them waits for the stages that write them and no
// line of them is read (and cached in L1) before, so plain loads serve there.
// The aggregates of the previous level (ldw) are different: in the persistent
// kernel a cache line of them can hold slots of the level being written, so
// they are read through L2 (ld.global.cg), never from a possibly stale L1
// line.
template <bool COH, class V>
__device__ __forceinline__ V ldp(const V *p) {
  if constexpr (COH) return *p;
  else return __ldg(p);
}
template <bool COH, class V>
__device__ __forceinline__ V ldw(const V *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// The internal node whose slot range holds the slot (a binary search of the
// slot offsets; COH: offsets written earlier in the same launch, read
// through L2).
template <bool COH>
__device__ __forceinline__ int node_of_slot(const long long *off, int M, long long slot) {
  int lo = 0, hi = M;
  while (lo < hi) {  // first node whose offset exceeds the slot
    const int mid = (lo + hi) >> 1;
    if (ldw<COH>(off + mid) <= slot) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Node, its box and the pixel of a slot of the non-final passes.  The group
// of kGroup slots holding the slot lies in the nodes [chunk_node[grp],
// chunk_node[grp + 1]]; the first of them holds most of the group, so its
// offsets, rectangle and box are loaded at once and the search runs only for
// the slots past its end.
__device__ __forceinline__ void slot_lookup(const Topo &T, const Scratch &S, int nb, int ne,
                                            long long slot, int &node, int &i, int &j,
                                            int4 &geo) {
  const long long grp = slot / kGroup;
  node = max(S.chunk_node[grp], nb);
  long long o0 = S.off[node];
  const long long o1 = S.off[node + 1];
  int4 r = S.rect[T.N + node];
  geo = __ldg(T.geo + T.N + node);
  if (slot >= o1) {
    const long long ngr = (S.off[T.M] + kGroup - 1) / kGroup;
    int lo = node + 1;
    int hi = (grp + 1 < ngr) ? min(S.chunk_node[grp + 1], ne - 1) + 1 : ne;
    while (lo < hi) {  // first node whose offset exceeds the slot
      const int mid = (lo + hi) >> 1;
      if (S.off[mid] <= slot) lo = mid + 1; else hi = mid;
    }
    node = lo - 1;
    o0 = S.off[node];
    r = S.rect[T.N + node];
    geo = __ldg(T.geo + T.N + node);
  }
  slot_pixel(r, (unsigned)(slot - o0), i, j);  // < w * h < 2^31
}

// Subtree pass (Sec. 3.2 + Sec. 3.3 for the deepest levels).  A warp owns 32
// consecutive (tile-level node, ray) slots, one lane each, and works alone
// (no CTA barrier): the standalone kernel runs resident one-warp CTAs that
// draw their groups of 32 slots from a counter, so that a warp that is done
// takes the next group at once.
//  A. every ray descends its tile node's subtree front to back: at each
//     internal node its box is cut by the three mid-planes, and the ray's
//     crossings of the node's planes give the slab interval of all 8 children
//     at once (the same rounded operands as a slab test of each child, so the
//     same decisions); the children it meets are taken in the order of their
//     octant index mirrored by the direction's sign bits, which is the ray's
//     front-to-back order for the disjoint cells of an octree.  A leaf met
//     is appended to the ray's list, an internal node is descended into.  A
//     child box nests in its parent, and monotone rounding keeps its FP32
//     slab interval inside the parent's, so a subtree the ray misses holds no
//     leaf the ray meets;
//  B. each warp integrates the hits of its 32 rays, one hit per lane, in
//     batches; a hit whose leaf's pixel rectangle does not hold the pixel (a
//     rounding edge case: the pair is no candidate) gives no segment, and
//  C. every lane folds its own ray's results nearest-first with Eq. 2.14.
constexpr int kWarpBatch = 32;  // hits per warp batch of phase B

// Shared memory of one subtree warp.
struct SubtreeSmem {
  float4 tfv[8], tfs[8];
  float ray[6][32];                  // ray: varying part, reciprocal direction
  float4 res[kWarpBatch];            // phase B: segment values of a batch
  int2 pix[32];                      // pixel of each ray
  int drop[32];                      // hits outside the leaf's rectangle
  int first[32];                     // first leaf of each ray's tile node
  int2 stk[kSubtreeDepth - 1][32];   // the descent's ancestors: node, children left
  unsigned short list[kMaxSubtreeHits][32];  // hits of each ray in order: leaf - first
};
// a tile node's subtree holds at most 8^kSubtreeDepth leaves
static_assert(kSubtreeDepth <= 5, "list entries are 16-bit leaf offsets");

// Child id of octant q from the node's 8 children held in two int4.
__device__ __forceinline__ int pick_child(int4 c0, int4 c1, int q) {
  const int4 c = (q & 4) ? c1 : c0;
  return (q & 2) ? ((q & 1) ? c.w : c.z) : ((q & 1) ? c.y : c.x);
}

// The children of the node with low corner lo whose boxes (side hc) the ray
// meets, as a mask over the mirrored octants (bit q ^ flip for octant
// q = bx + 2 by + 4 bz, flip the direction's sign bits).  Anchors are integers
// below 2^20 in units of 2^-L (L <= 20), so every face is exact in FP32: per
// axis the faces lo, lo + hc, lo + 2 hc are the very values a slab test of
// each child forms (its low corner, and low corner + side rounded once), and
// their crossings (face - o) x (1/d) are formed once.  Rounding is monotone, so
// the crossings are ordered like the faces along the ray: the half the ray
// enters first spans (first face, mid face), the other (mid face, last face),
// which are the min / max a slab test takes, and taking the halves in that
// order gives the mirrored bits directly.  Each child's interval is the same
// max / min chain over the axes x, y, z as its own slab test (the chains share
// their common prefixes).
__device__ __forceinline__ unsigned child_hits(float3 o, float3 d, float3 iv, float3 lo,
                                               float hc, float amin, float amax) {
  const float oa[3] = {o.x, o.y, o.z}, da[3] = {d.x, d.y, d.z}, va[3] = {iv.x, iv.y, iv.z};
  const float la[3] = {lo.x, lo.y, lo.z};
  constexpr unsigned kHalf[3][2] = {{0x55u, 0xaau}, {0x33u, 0xccu}, {0x0fu, 0xf0u}};
  float mn[3][2], mx[3][2];
  unsigned ok = 0xffu;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p0 = la[a], p1 = __fadd_rn(p0, hc), p2 = __fadd_rn(p1, hc);
    if (da[a] == 0.f) {  // parallel (no mirroring): inside a half's slab or not, no bound on alpha
      if (oa[a] < p0 || oa[a] > p1) ok &= ~kHalf[a][0];
      if (oa[a] < p1 || oa[a] > p2) ok &= ~kHalf[a][1];
      mn[a][0] = mn[a][1] = -INFINITY;
      mx[a][0] = mx[a][1] = INFINITY;
    } else {
      const bool neg = da[a] < 0.f;
      const float s0 = __fmul_rn(__fsub_rn(neg ? p2 : p0, oa[a]), va[a]);
      const float s1 = __fmul_rn(__fsub_rn(p1, oa[a]), va[a]);
      const float s2 = __fmul_rn(__fsub_rn(neg ? p0 : p2, oa[a]), va[a]);
      mn[a][0] = s0;
      mx[a][0] = s1;
      mn[a][1] = s1;
      mx[a][1] = s2;
    }
  }
  float e0[4], e1[4];  // the chains after x and y, per (bx, by)
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const float f0 = fmaxf(amin, mn[0][x]), f1 = fminf(amax, mx[0][x]);
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      e0[x + 2 * y] = fmaxf(f0, mn[1][y]);
      e1[x + 2 * y] = fminf(f1, mx[1][y]);
    }
  }
  unsigned m = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    m |= (fminf(e1[q & 3], mx[2][q >> 2]) > fmaxf(e0[q & 3], mn[2][q >> 2]) ? 1u : 0u) << q;
  return m & ok;
}

// A child mask in octant order from one in mirrored order, or back: bit
// q ^ flip <-> bit q.
__device__ __forceinline__ unsigned mirror_bits(unsigned m, unsigned flip) {
  if (flip & 1u) m = ((m & 0x55u) << 1) | ((m >> 1) & 0x55u);
  if (flip & 2u) m = ((m & 0x33u) << 2) | ((m >> 2) & 0x33u);
  if (flip & 4u) m = ((m & 0x0fu) << 4) | ((m >> 4) & 0x0fu);
  return m;
}

// Phase A of the subtree pass for one ray: the descent of its tile node's
// subtree (node, box gn) front to back, the leaves met appended to list (16-bit
// offsets from the tile node's first leaf, entry k at list[k * stride], at
// most kMaxSubtreeHits kept; nhit counts them all).  The path's ancestors
// (node, children still to visit) are kept at stk[d * stride], the current
// anchor is cleared to an ancestor's on the way up and the current node's
// children are loaded once per visit; the leaves up to the next internal child
// are taken in one run.  deep: an internal node below the subtree depth was
// met.
__device__ __forceinline__ void subtree_walk(const Topo &T, const Cam &c, bool active, int node,
                                             int4 gn, float3 org, float3 dir, float3 inv,
                                             float scale, int first, unsigned short *list,
                                             int2 *stk, int stride, unsigned &nhit,
                                             unsigned &nvisit, bool &deep) {
  const unsigned flip = (dir.x < 0.f ? 1u : 0u) | (dir.y < 0.f ? 2u : 0u) | (dir.z < 0.f ? 4u : 0u);
  // (a ray that misses the tile node meets none of its children)
  int cur = node, lev = gn.w, gx = gn.x, gy = gn.y, gz = gn.z, d = 0;
  unsigned msk = active ? child_hits(org, dir, inv, node_lo(gn, scale), exp2i(-(lev + 1)),
                                     c.amin, c.amax)
                        : 0u;
  const int4 *child4 = reinterpret_cast<const int4 *>(T.child);
  int4 c0 = make_int4(-1, -1, -1, -1), c1 = c0;
  if (msk) {
    c0 = __ldg(child4 + 2 * cur);
    c1 = __ldg(child4 + 2 * cur + 1);
  }
  nhit = 0;
  nvisit = active ? 1u : 0u;
  deep = false;
  // each round of the outer loop visits one internal node per lane: the inner
  // loop takes the leaves up to the lane's next internal child, going back up
  // through the nodes it finishes, so that the lanes' visits line up
  while (true) {
    int q = 0, id = -1;
    bool done = false;
    while (true) {
      while (msk) {
        q = (__ffs(msk) - 1) ^ (int)flip;
        msk &= msk - 1u;
        id = pick_child(c0, c1, q);
        if (id >= T.N) break;
        if (id >= 0) {
          if (nhit < (unsigned)kMaxSubtreeHits) list[nhit * stride] = (unsigned short)(id - first);
          ++nhit;
        }
      }
      if (id >= T.N) break;  // the next internal child to visit
      if (d == 0) {          // the walk is over
        done = true;
        break;
      }
      // this node is done: back to its parent
      --d;
      --lev;
      const int keep = ~((1 << (T.L - lev)) - 1);
      gx &= keep;
      gy &= keep;
      gz &= keep;
      const int2 e = stk[d * stride];
      cur = e.x;
      msk = (unsigned)e.y;
      id = -1;
      if (msk) {
        c0 = __ldg(child4 + 2 * cur);
        c1 = __ldg(child4 + 2 * cur + 1);
      }
    }
    if (done) break;
    if (d >= kSubtreeDepth - 1) {  // below the subtree depth: not a tile node's subtree
      deep = true;
      continue;
    }
    stk[d * stride] = make_int2(cur, (int)msk);
    const int hs = 1 << (T.L - lev - 1);
    gx += (q & 1) * hs;
    gy += ((q >> 1) & 1) * hs;
    gz += (q >> 2) * hs;
    ++d;
    ++lev;
    cur = id - T.N;
    msk = child_hits(org, dir, inv, node_lo(make_int4(gx, gy, gz, 0), scale),
                     exp2i(-(lev + 1)), c.amin, c.amax);
    ++nvisit;
    if (msk) {
      c0 = __ldg(child4 + 2 * cur);
      c1 = __ldg(child4 + 2 * cur + 1);
    }
  }
}

// The 32 slots [ws, ws + 32) of the pass over the slots [s0, s1) of the
// nodes [nb, ne), ws a multiple of 32; one warp, its own shared memory.
template <bool SURF, bool COH>
__device__ __forceinline__ void subtree_warp(const Topo &T, const Field &Fd, const Cam &c,
                                             const Integ &I, const Scratch &S, int nb, int ne,
                                             long long s0, long long s1, long long ws,
                                             SubtreeSmem &sm) {
  float4(&s_tfv)[8] = sm.tfv;
  float4(&s_tfs)[8] = sm.tfs;
  float(&s_ray)[6][32] = sm.ray;
  unsigned short(&s_list)[kMaxSubtreeHits][32] = sm.list;
  int(&s_first)[32] = sm.first;
  float4(&s_res)[kWarpBatch] = sm.res;
  int2(&s_pix)[32] = sm.pix;
  int(&s_drop)[32] = sm.drop;
  const int tid = threadIdx.x & 31, lane = tid;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }

  // slot -> node, pixel, ray; rays that miss the node's box skip all leaves
  const long long slot = ws + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = -1, i = 0, j = 0;
  int4 gn = make_int4(0, 0, 0, 0);
  if (active) slot_lookup(T, S, nb, ne, slot, node, i, j, gn);
  float3 org, dir;
  pixel_ray(c, i, j, org, dir);
  const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
  const float scale = exp2i(-T.L);
  // the part of the ray that varies over the pixels (the origin of an
  // orthographic camera, the direction of a perspective one) and the
  // reciprocal direction, taken once per ray
  s_ray[0][tid] = c.ortho ? org.x : dir.x;
  s_ray[1][tid] = c.ortho ? org.y : dir.y;
  s_ray[2][tid] = c.ortho ? org.z : dir.z;
  s_ray[3][tid] = inv.x;
  s_ray[4][tid] = inv.y;
  s_ray[5][tid] = inv.z;
  s_pix[tid] = make_int2(i, j);
  s_drop[tid] = 0;
  const int first = active ? __ldg(T.leaves + node).x : 0;  // the tile node's first leaf
  s_first[tid] = first;

  __syncwarp();  // the transfer function table

  // A. the ray's front-to-back descent of its tile node's subtree
  unsigned nhit, nvisit;
  bool deep;
  subtree_walk(T, c, active, node, gn, org, dir, inv, scale, first, &s_list[0][tid],
               &sm.stk[0][tid], 32, nhit, nvisit, deep);
  __syncwarp();  // the warp's rays and lists


  // B + C. per warp: integrate the warp's hits, one per lane; fold per ray
  const int n = min((int)nhit, kMaxSubtreeHits);
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
      const int ow = lo & 31;
      const int owpre = __shfl_sync(0xffffffffu, my0, ow);
      if (h < b1) {
        const int t = ow;
        const int leaf = s_first[t] + (int)s_list[h - owpre][t];
        const float3 rv = make_float3(s_ray[0][t], s_ray[1][t], s_ray[2][t]);
        const float3 ro = c.ortho ? rv : make_float3(c.o[0], c.o[1], c.o[2]);
        const float3 rd = c.ortho ? make_float3(c.v[0], c.v[1], c.v[2]) : rv;
        const int4 r = ldp<COH>(S.rect + leaf);
        const int2 p = s_pix[t];
        const bool inside = p.x >= r.x && p.x <= r.y && p.y >= r.z && p.y <= r.w;
        int st = 0;
        const float4 sg = leaf_segment<SURF>(T, Fd, c, I, tf, leaf, ro, rd,
                                             make_float3(s_ray[3][t], s_ray[4][t], s_ray[5][t]),
                                             scale, st);
        if (inside) {
          s_res[h - b0] = sg;
          steps += st;
        } else {
          s_res[h - b0] = seg_identity();
          atomicAdd(&s_drop[t], 1);
        }
      }
    }
    __syncwarp();
    for (int h = max(my0, b0); h < min(my0 + n, b1); ++h) acc = seg_combine(acc, s_res[h - b0]);
    __syncwarp();
  }
  __syncwarp();
  if (nhit > (unsigned)kMaxSubtreeHits || deep) atomicAdd(S.stats + kStatErrors, 1ull);
  nhit -= (unsigned)s_drop[tid];
  if (active) {
    S.entries[slot] = acc;
    if (nhit && S.counts) atomicAdd(S.counts + (size_t)j * c.w + i, (int)nhit);
  }
  // counters, when asked for: one atomic per warp and counter
  if (S.counters) {
    const unsigned v[4] = {nhit, (unsigned)steps, nvisit, active ? 1u : 0u};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned x = __reduce_add_sync(0xffffffffu, v[q]);
      if (lane == 0 && x) atomicAdd(S.counters + q, (unsigned long long)x);
    }
  }
}

// Shared memory of one coarsening chunk.
struct CoarsenSmem {
  float4 tfv[8], tfs[8];
  float4 seg[8][kCoarsenThreads];           // child segment of each slot (identity if none)
  unsigned short hit[8 * kCoarsenThreads];  // (slot << 3) | child octant of each hit
  int2 pix[kCoarsenThreads];
  int node[kCoarsenThreads];
  int nhit;
  unsigned long long cnt[4];
};

// One chunk (CTA bid) of a coarsening pass over the slots [s0, s1) of the
// nodes [nb, ne), or, FINAL, of the pixel pass over the pixels [s0, s1).
template <bool FINAL, bool SURF, bool COH>
__device__ __forceinline__ void coarsen_chunk(const Topo &T, const Field &Fd, const Cam &c,
                                              const Integ &I, const Scratch &S, int nb, int ne,
                                              long long s0, long long s1, long long bid,
                                              float4 *rgba, CoarsenSmem &sm) {
  constexpr int NT = kCoarsenThreads;
  float4(&s_tfv)[8] = sm.tfv;
  float4(&s_tfs)[8] = sm.tfs;
  float4(&s_seg)[8][NT] = sm.seg;
  unsigned short(&s_hit)[8 * NT] = sm.hit;
  int2(&s_pix)[NT] = sm.pix;
  int(&s_node)[NT] = sm.node;
  int &s_nhit = sm.nhit;
  unsigned long long(&s_cnt)[4] = sm.cnt;

  const int tid = threadIdx.x;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  if (tid < 4) s_cnt[tid] = 0ull;
  if (tid == 0) s_nhit = 0;

  // non-final passes work on whole chunks of the global slot space, so that
  // chunk_node gives the first node of the CTA without a search
  const long long chunk = FINAL ? 0 : s0 / NT + bid;
  const long long slot = FINAL ? s0 + bid * NT + tid : chunk * NT + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = T.M;  // super-root in the final pass
  int i = 0, j = 0;
  int4 g = make_int4(0, 0, 0, 0);
  if (active) {
    if (FINAL) {
      i = (int)(slot % c.w);
      j = (int)(slot / c.w);
    } else {
      slot_lookup(T, S, nb, ne, slot, node, i, j, g);
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
  const float scale = exp2i(-T.L);

  // the children the ray meets (by octant), from the node's shared face
  // crossings: a ray that misses the node meets none of them, and a child it
  // misses contributes the identity.  The final pass's node is the
  // super-root, whose one child is the tree root.
  unsigned msk = 0u;
  if (active) {
    if (FINAL) {
      if (ch[0] >= 0) {
        const int4 gr = __ldg(T.geo + ch[0]);
        float a0, a1;
        if (slab(org, dir, inv, node_lo(gr, scale), exp2i(-gr.w), c.amin, c.amax, a0, a1))
          msk = 1u;
      }
    } else {
      const unsigned flip =
          (dir.x < 0.f ? 1u : 0u) | (dir.y < 0.f ? 2u : 0u) | (dir.z < 0.f ? 4u : 0u);
      msk = mirror_bits(child_hits(org, dir, inv, node_lo(g, scale), exp2i(-(g.w + 1)), c.amin,
                                   c.amax),
                        flip);
    }
  }
  __syncthreads();

  // phase 1: the leaf children the ray meets whose rectangle holds the pixel
  unsigned local_tests = 0, local_hits = 0, lhit = 0u;
  if (msk) {
    int4 rc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      rc[q] = ((msk >> q) & 1u) && ch[q] >= 0 && ch[q] < T.N ? ldp<COH>(S.rect + ch[q])
                                                               : empty_rect();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      local_tests += (ch[q] >= 0 && ch[q] < T.N) ? 1u : 0u;
      const int4 r = rc[q];
      if (i < r.x || i > r.y || j < r.z || j > r.w) continue;
      s_hit[atomicAdd(&s_nhit, 1)] = (unsigned short)((tid << 3) | q);
      lhit |= 1u << q;
      ++local_hits;
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
    s_seg[q][st] = leaf_segment<SURF>(T, Fd, c, I, tf, leaf, o2, d2, iv2, scale, steps);
  }
  __syncthreads();

  // phase 3: combine the children nearest-first.  Along a ray with direction
  // signs (sx, sy, sz) the octants come in increasing order of q ^ mask; the
  // same sequence is formed by combining along x, then y, then z, each pair
  // nearer-first (Eq. 2.14 is associative), with every index static.
  if (active) {
    // the internal children's slots of this pixel: rectangles and offsets in
    // one round of independent loads, then the aggregates in another
    long long e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int id = ch[q];
      e[q] = -1;
      if (((msk >> q) & 1u) && id >= T.N) {
        const int4 r = ldp<COH>(S.rect + id);
        const long long o = ldp<COH>(S.off + id - T.N);
        if (i >= r.x && i <= r.y && j >= r.z && j <= r.w)
          e[q] = o + slot_of_pixel(r, i, j);
      }
    }
    float4 cs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float4 s = seg_identity();
      if ((lhit >> q) & 1u) s = s_seg[q][tid];
      else if (e[q] >= 0) s = ldw<COH>(S.entries + e[q]);
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

  // counters, when asked for: segments, RK steps, leaf tests, slots
  if (S.counters) {
    const unsigned v[4] = {local_hits, (unsigned)steps, local_tests, active ? 1u : 0u};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned x = __reduce_add_sync(0xffffffffu, v[q]);
      if ((tid & 31) == 0 && x) atomicAdd(&s_cnt[q], (unsigned long long)x);
    }
    __syncthreads();
    if (tid < 4 && s_cnt[tid]) atomicAdd(S.counters + kStatCoarse + tid, s_cnt[tid]);
  }
}

}  // namespace
}  // namespace ocr
