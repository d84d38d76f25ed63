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

// Node and pixel of a slot of the non-final passes.  The CTA's chunk of slots
// lies in the nodes [chunk_node[chunk], chunk_node[chunk + 1]].
template <bool COH>
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
  const unsigned local = (unsigned)(slot - S.off[node]);  // < w * h < 2^31
  const unsigned rw = (unsigned)(r.y - r.x + 1);
  const unsigned row = local / rw;
  i = r.x + (int)(local - row * rw);
  j = r.z + (int)row;
}

__device__ __forceinline__ unsigned spread3_9(unsigned v) {  // 3 bits -> positions 0, 3, 6
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

// Subtree pass (Sec. 3.2 + Sec. 3.3 for the deepest levels).  A CTA owns a
// chunk of kChunk consecutive (tile-level node, ray) slots, one thread each.
//  A. per node of the chunk, the leaves of its subtree whose pixel rectangle
//     meets the node's rows in the chunk are compacted into a shared table
//     (Morton order): each with its box (rectangle within those rows), its
//     anchor relative to the node and its level.  The table's (candidate,
//     pixel) pairs are spread evenly over the CTA by a prefix sum of the box
//     areas; every pair whose pixel is a live ray of the candidate's node is
//     slab-tested and a hit appended to that ray's list;
//  B. each ray sorts its hits by their Morton key inside the tile node with
//     every axis mirrored where the ray runs towards negative coordinates:
//     the ray's front-to-back order for disjoint cells;
//  C. each warp integrates the hits of its 32 rays, one hit per lane, in
//     batches, and
//  D. every lane folds its own ray's results nearest-first with Eq. 2.14.
constexpr int kSubtreeThreads = kChunk;  // one chunk per CTA
constexpr int kCand = kSubtreeThreads;  // candidate table of phase A
constexpr int kPairWin = 1024;          // (candidate, pixel) pairs resolved per window
static_assert(kCand <= 256, "candidate indices are stored in one byte");
static_assert(sizeof(int4) * kCand == sizeof(float4) * kChunk,
              "phase A's candidate boxes and phase C's values share their storage");
constexpr int kWarpBatch = 32; // hits per warp batch of phase C

// Shared memory of one subtree chunk.
struct SubtreeSmem {
  float4 tfv[8], tfs[8];
  float ray[6][kSubtreeThreads];                   // ray: varying part, reciprocal direction
  signed char liveq[kSubtreeThreads];              // live ray: index of its node, else -1
  int4 qinfo[kSubtreeThreads];                     // node: {rect x0, rect y0, width, off - cs}
  int2 qlr[kSubtreeThreads];                       // node: its leaves [first, end)
  int2 qrows[kSubtreeThreads];                     // node: its rows in the chunk
  unsigned long long qgeo[kSubtreeThreads];        // node: anchor x | y << 21 | z << 42
  union {
    int4 cbox[kCand];                              // phase A: candidate rectangle within the rows
    float4 res[kSubtreeThreads / 32][kWarpBatch];  // phase C: the warps' segment values
  };
  int cpre[kCand + 1];                             // candidate: pair count, then prefix
  unsigned crel[kCand];                            // candidate: anchor in the node, level
  int cl[kCand];                                   // candidate: (node index << 22) | leaf - base
  unsigned char pc[kPairWin];                      // candidate of each pair in the window
  int cnt[kSubtreeThreads];                        // hits of each ray
  unsigned list[kMaxSubtreeHits][kSubtreeThreads]; // (mirrored key << 22) | leaf - base
  int wcnt[kSubtreeThreads / 32], nn, leaf_base, ncand, ltot;
};

// One chunk (CTA bid of the pass over the slots [s0, s1) of the nodes
// [nb, ne)); a CTA of kSubtreeThreads threads.
template <bool SURF, bool COH>
__device__ __forceinline__ void subtree_chunk(const Topo &T, const Field &Fd, const Cam &c,
                                              const Integ &I, const Scratch &S, int nb, int ne,
                                              long long s0, long long s1, long long bid,
                                              SubtreeSmem &sm) {
  constexpr int NT = kSubtreeThreads, NW = NT / 32;
  static_assert(kCand == NT, "one table entry per thread in the prefix sum");
  float4(&s_tfv)[8] = sm.tfv;
  float4(&s_tfs)[8] = sm.tfs;
  float(&s_ray)[6][NT] = sm.ray;
  signed char(&s_liveq)[NT] = sm.liveq;
  int4(&s_qinfo)[NT] = sm.qinfo;
  int2(&s_qlr)[NT] = sm.qlr;
  int2(&s_qrows)[NT] = sm.qrows;
  unsigned long long(&s_qgeo)[NT] = sm.qgeo;
  int4(&s_cbox)[kCand] = sm.cbox;
  int(&s_cpre)[kCand + 1] = sm.cpre;
  unsigned(&s_crel)[kCand] = sm.crel;
  int(&s_cl)[kCand] = sm.cl;
  unsigned char(&s_pc)[kPairWin] = sm.pc;
  int(&s_cnt)[NT] = sm.cnt;
  unsigned(&s_list)[kMaxSubtreeHits][NT] = sm.list;
  float4(&s_res)[NW][kWarpBatch] = sm.res;
  int(&s_wcnt)[NW] = sm.wcnt;
  int &s_nn = sm.nn, &s_leaf_base = sm.leaf_base, &s_ncand = sm.ncand, &s_ltot = sm.ltot;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }

  // slot -> node, pixel, ray; rays that miss the node's box skip all leaves
  const long long cs = (s0 / kChunk) * kChunk + bid * NT;
  const long long slot = cs + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = -1, i = 0, j = 0;
  if (active) slot_lookup<COH>(T, S, nb, ne, slot / kChunk, slot, node, i, j);
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
  // the part of the ray that varies over the pixels (the origin of an
  // orthographic camera, the direction of a perspective one) and the
  // reciprocal direction, taken once per ray
  s_ray[0][tid] = c.ortho ? org.x : dir.x;
  s_ray[1][tid] = c.ortho ? org.y : dir.y;
  s_ray[2][tid] = c.ortho ? org.z : dir.z;
  s_ray[3][tid] = inv.x;
  s_ray[4][tid] = inv.y;
  s_ray[5][tid] = inv.z;
  int *s_node = s_cnt;  // node of each slot (-1 inactive) until phase A
  s_node[tid] = active ? node : -1;
  __syncthreads();

  // distinct nodes of the chunk (a node's slots are contiguous), this slot's
  // node index among them, and each node's layout in the chunk
  {
    const bool head = active && (tid == 0 || s_node[tid - 1] != node);
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (lane == 0) s_wcnt[wid] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += s_wcnt[w];
    const int myq = base + __popc(bal & (0xffffffffu >> (31 - lane))) - 1;
    if (head) {
      const int4 rn = ldp<COH>(S.rect + T.N + node);
      const long long off = ldp<COH>(S.off + node), off1 = ldp<COH>(S.off + node + 1);
      const int4 gq = __ldg(T.geo + T.N + node);
      const int2 lr = __ldg(T.leaves + node);
      const int w = rn.y - rn.x + 1, ow = (int)(off - cs);
      s_qinfo[myq] = make_int4(rn.x, rn.z, w, ow);
      s_qgeo[myq] = (unsigned long long)gq.x | (unsigned long long)gq.y << 21 |
                    (unsigned long long)gq.z << 42;
      s_qlr[myq] = lr;
      // the node's slots [la, lb) in the chunk, and their rows
      const int la = max(0, -ow), lb = (int)(min(min(cs + NT, s1), off1) - off);
      s_qrows[myq] = make_int2(rn.z + la / w, rn.z + (lb - 1) / w);
    }
    s_liveq[tid] = (signed char)(live ? myq : -1);
    if (tid == NT - 1) {
      int tot = 0;
      for (int w = 0; w < NW; ++w) tot += s_wcnt[w];
      s_nn = tot;
      s_ncand = 0;
    }
    __syncthreads();
    if (tid == 0) {
      int lt = 0;
      for (int q = 0; q < s_nn; ++q) lt += s_qlr[q].y - s_qlr[q].x;
      s_ltot = lt;
      s_leaf_base = s_nn ? s_qlr[0].x : 0;
    }
  }
  __syncthreads();

  // A. candidates and hits
  unsigned ntest = 0;
  const int nn = s_nn, leaf_base = s_leaf_base;
  s_cnt[tid] = 0;
  // the table's pairs: prefix of the pair counts, then one pair per thread at a time
  auto flush = [&]() {
    __syncthreads();
    const int nc = s_ncand;
    const int n0 = tid < nc ? s_cpre[tid] : 0;
    int x = n0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wcnt[wid] = x;
    __syncthreads();
    int base = 0, tot = 0;
    for (int w = 0; w < NW; ++w) {
      if (w < wid) base += s_wcnt[w];
      tot += s_wcnt[w];
    }
    if (tid < nc) s_cpre[tid] = base + x - n0;
    if (tid == 0) s_cpre[nc] = tot;
    __syncthreads();
    // pairs in windows of kPairWin: each candidate marks its pairs in the
    // window with its index, then every pair finds its candidate in one load
    const int my_pre = tid < nc ? s_cpre[tid] : 0, my_end = my_pre + n0;
    for (int w0 = 0; w0 < tot; w0 += kPairWin) {
      const int w1 = min(tot, w0 + kPairWin);
      for (int p = max(my_pre, w0); p < min(my_end, w1); ++p) s_pc[p - w0] = (unsigned char)tid;
      __syncthreads();
    for (int pq = w0 + tid; pq < w1; pq += NT) {
      const int lo = s_pc[pq - w0];
      const int4 b = s_cbox[lo];
      const int loc = pq - s_cpre[lo];
      // row = floor(loc / width) from the rounded reciprocal: exact, as the
      // quotient of (loc + 1/2) stays 1/(2 width) away from an integer
      const int bw = b.y - b.x + 1;
      const int row = (int)(((float)loc + 0.5f) * (1.f / (float)bw));
      const int ii = b.x + loc - row * bw, jj = b.z + row;
      const int tl = s_cl[lo];
      const int q = tl >> 22;
      const int4 qi = s_qinfo[q];
      const int t = qi.w + (jj - qi.y) * qi.z + (ii - qi.x);
      if (t < 0 || t >= NT || s_liveq[t] != q) continue;
      ++ntest;
      const unsigned rel = s_crel[lo];
      const unsigned rx = rel & 255u, ry = (rel >> 8) & 255u, rz = (rel >> 16) & 255u;
      const unsigned long long gq = s_qgeo[q];
      const int4 g = make_int4((int)(gq & 0x1fffffu) + (int)rx, (int)((gq >> 21) & 0x1fffffu) + (int)ry,
                               (int)(gq >> 42) + (int)rz, (int)(rel >> 24));
      const float3 rv = make_float3(s_ray[0][t], s_ray[1][t], s_ray[2][t]);
      const float3 ro = c.ortho ? rv : make_float3(c.o[0], c.o[1], c.o[2]);
      const float3 rd = c.ortho ? make_float3(c.v[0], c.v[1], c.v[2]) : rv;
      const float3 ri = make_float3(s_ray[3][t], s_ray[4][t], s_ray[5][t]);
      float b0, b1;
      if (!slab(ro, rd, ri, node_lo(g, scale), ldexpf(1.f, -g.w), c.amin, c.amax, b0, b1))
        continue;
      const unsigned key = spread3_9(rx) | (spread3_9(ry) << 1) | (spread3_9(rz) << 2);
      const unsigned flip =
          (rd.x < 0.f ? 0x49u : 0u) | (rd.y < 0.f ? 0x92u : 0u) | (rd.z < 0.f ? 0x124u : 0u);
      const int k = atomicAdd(&s_cnt[t], 1);
      if (k < kMaxSubtreeHits) s_list[k][t] = ((key ^ flip) << 22) | (unsigned)(tl & 0x3fffff);
    }
      __syncthreads();
    }
    if (tid == 0) s_ncand = 0;
  };
  // the candidate leaf l of node q: kept if its rectangle meets the node's
  // columns and its rows in the chunk
  auto candidate = [&](int q, int l, bool in_range, int &cnt) -> int4 {
    int4 box = empty_rect();
    cnt = 0;
    if (in_range) {
      const int4 qi = s_qinfo[q];
      const int2 rows = s_qrows[q];
      const int4 r = ldp<COH>(S.rect + l);
      box = make_int4(max(r.x, qi.x), min(r.y, qi.x + qi.z - 1), max(r.z, rows.x), min(r.w, rows.y));
      if (box.x <= box.y && box.z <= box.w) cnt = (box.y - box.x + 1) * (box.w - box.z + 1);
    }
    return box;
  };
  auto store = [&](int at, int q, int l, int4 box, int cnt) {
    const unsigned long long gq = s_qgeo[q];
    const int4 g = __ldg(T.geo + l);
    s_cbox[at] = box;
    s_cpre[at] = cnt;
    s_crel[at] = (unsigned)(g.x - (int)(gq & 0x1fffffu)) |
                 (unsigned)(g.y - (int)((gq >> 21) & 0x1fffffu)) << 8 |
                 (unsigned)(g.z - (int)(gq >> 42)) << 16 | (unsigned)g.w << 24;
    s_cl[at] = (q << 22) | (l - leaf_base);
  };
  if (s_ltot <= kCand) {
    // all the chunk's leaves fit the table: the warps take 32-leaf blocks in
    // turn and append their candidates without CTA barriers
    int q = 0, b = wid;  // this warp's block: the b-th 32-leaf block of node q
    while (q < nn) {
      const int2 lr = s_qlr[q];
      const int nb32 = (lr.y - lr.x + 31) >> 5;
      if (b >= nb32) {
        b -= nb32;
        ++q;
        continue;
      }
      const int l = lr.x + 32 * b + lane;
      int cnt;
      const int4 box = candidate(q, l, l < lr.y, cnt);
      const unsigned bal = __ballot_sync(0xffffffffu, cnt > 0);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&s_ncand, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (cnt > 0) store(base + __popc(bal & ((1u << lane) - 1u)), q, l, box, cnt);
      b += NW;
    }
  } else {
    for (int q = 0; q < nn; ++q) {
      const int2 lr = s_qlr[q];
      for (int l0 = lr.x; l0 < lr.y; l0 += NT) {
        __syncthreads();
        if (s_ncand + NT > kCand) flush();
        const int l = l0 + tid;
        int cnt;
        const int4 box = candidate(q, l, l < lr.y, cnt);
        const unsigned bal = __ballot_sync(0xffffffffu, cnt > 0);
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        int base = s_ncand;
        for (int w = 0; w < wid; ++w) base += s_wcnt[w];
        if (cnt > 0) store(base + __popc(bal & ((1u << lane) - 1u)), q, l, box, cnt);
        __syncthreads();
        if (tid == NT - 1) s_ncand = base + __popc(bal);
      }
    }
  }
  flush();
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
      const int ow = lo & 31;
      const int owpre = __shfl_sync(0xffffffffu, my0, ow);
      if (h < b1) {
        const int t = wid * 32 + ow;
        const int leaf = leaf_base + (int)(s_list[h - owpre][t] & 0x3fffffu);
        const float3 rv = make_float3(s_ray[0][t], s_ray[1][t], s_ray[2][t]);
        const float3 ro = c.ortho ? rv : make_float3(c.o[0], c.o[1], c.o[2]);
        const float3 rd = c.ortho ? make_float3(c.v[0], c.v[1], c.v[2]) : rv;
        s_res[wid][h - b0] = leaf_segment<SURF>(T, Fd, c, I, tf, leaf, ro, rd,
                                                make_float3(s_ray[3][t], s_ray[4][t], s_ray[5][t]),
                                                scale, steps);
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
  // counters: one atomic per warp and counter, no CTA-wide barrier at the end
  unsigned long long v[4] = {nhit, (unsigned long long)steps, ntest, active ? 1ull : 0ull};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0 && x) atomicAdd(S.stats + q, x);
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
#pragma unroll
  for (int q = 0; q < 8; ++q) s_seg[q][tid] = seg_identity();

  // non-final passes work on whole chunks of the global slot space, so that
  // chunk_node gives the first node of the CTA without a search
  const long long chunk = FINAL ? 0 : s0 / NT + bid;
  const long long slot = FINAL ? s0 + bid * NT + tid : chunk * NT + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = T.M;  // super-root in the final pass
  int i = 0, j = 0;
  if (active) {
    if (FINAL) {
      i = (int)(slot % c.w);
      j = (int)(slot / c.w);
    } else {
      slot_lookup<COH>(T, S, nb, ne, chunk, slot, node, i, j);
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
      rc[q] = (ch[q] >= 0 && ch[q] < T.N) ? ldp<COH>(S.rect + ch[q]) : empty_rect();
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
      if (live && id >= T.N) {
        const int4 r = ldp<COH>(S.rect + id);
        const long long o = ldp<COH>(S.off + id - T.N);
        if (i >= r.x && i <= r.y && j >= r.z && j <= r.w)
          e[q] = o + (long long)(j - r.z) * (r.y - r.x + 1) + (i - r.x);
      }
    }
    float4 cs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int id = ch[q];
      float4 s = seg_identity();
      if (live && id >= 0 && id < T.N) s = s_seg[q][tid];
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
}  // namespace ocr
