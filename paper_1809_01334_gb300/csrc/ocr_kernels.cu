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
#include "ocr_device.cuh"

#include <cstdio>

namespace ocr {
namespace {

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
      if (S.visible && vis) S.visible[k] = 1;  // zeroed by the host; OR over cameras
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
constexpr int kWarpBatch = 32; // hits per warp batch of phase C

template <bool SURF>
__global__ void __launch_bounds__(kSubtreeThreads, 1024 / kSubtreeThreads)
    subtree_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, int nb, int ne, long long s0,
                   long long s1) {
  constexpr int NT = kSubtreeThreads, NW = NT / 32;
  static_assert(kCand == NT, "one table entry per thread in the prefix sum");
  __shared__ float4 s_tfv[8], s_tfs[8];
  __shared__ float s_ray[6][NT];                         // ray origin and direction, by component
  __shared__ signed char s_liveq[NT];                    // live ray: index of its node, else -1
  __shared__ int4 s_qinfo[NT];                           // node: {rect x0, rect y0, width, off - cs}
  __shared__ int2 s_qlr[NT];                             // node: its leaves [first, end)
  __shared__ int2 s_qrows[NT];                           // node: its rows in the chunk
  __shared__ unsigned long long s_qgeo[NT];              // node: anchor x | y << 21 | z << 42
  __shared__ int4 s_cbox[kCand];                         // candidate: rectangle within the rows
  __shared__ int s_cpre[kCand + 1];                      // candidate: pair count, then prefix
  __shared__ unsigned s_crel[kCand];                     // candidate: anchor in the node, level
  __shared__ int s_cl[kCand];                            // candidate: (node index << 22) | leaf - base
  __shared__ unsigned char s_pc[kPairWin];               // candidate of each pair in the window
  __shared__ int s_cnt[NT];                              // hits of each ray
  __shared__ unsigned s_list[kMaxSubtreeHits][NT];       // (mirrored key << 22) | leaf - base
  __shared__ float4 s_res[NW][kWarpBatch];
  __shared__ int s_wcnt[NW], s_nn, s_leaf_base, s_ncand, s_ltot;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }

  // slot -> node, pixel, ray; rays that miss the node's box skip all leaves
  const long long cs = (s0 / kChunk) * kChunk + (long long)blockIdx.x * NT;
  const long long slot = cs + tid;
  const bool active = slot >= s0 && slot < s1;
  int node = -1, i = 0, j = 0;
  if (active) slot_lookup(T, S, nb, ne, slot / kChunk, slot, node, i, j);
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
  s_ray[0][tid] = org.x;
  s_ray[1][tid] = org.y;
  s_ray[2][tid] = org.z;
  s_ray[3][tid] = dir.x;
  s_ray[4][tid] = dir.y;
  s_ray[5][tid] = dir.z;
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
      const int4 rn = __ldg(S.rect + T.N + node);
      const long long off = __ldg(S.off + node), off1 = __ldg(S.off + node + 1);
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
      const float3 ro = make_float3(s_ray[0][t], s_ray[1][t], s_ray[2][t]);
      const float3 rd = make_float3(s_ray[3][t], s_ray[4][t], s_ray[5][t]);
      const float3 ri = make_float3(recip_or_zero(rd.x), recip_or_zero(rd.y), recip_or_zero(rd.z));
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
      const int4 r = __ldg(S.rect + l);
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
        const float3 ro = make_float3(s_ray[0][t], s_ray[1][t], s_ray[2][t]);
        const float3 rd = make_float3(s_ray[3][t], s_ray[4][t], s_ray[5][t]);
        s_res[wid][h - b0] = leaf_segment<SURF>(T, Fd, c, I, tf, leaf, ro, rd,
                                          make_float3(recip_or_zero(rd.x), recip_or_zero(rd.y),
                                                      recip_or_zero(rd.z)),
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

template <bool FINAL, bool SURF>
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
        const int4 r = __ldg(S.rect + id);
        const long long o = __ldg(S.off + id - T.N);
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
      else if (e[q] >= 0) s = S.entries[e[q]];
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

// Top-down merge of the levels above the tile level, one thread per pixel:
// the octree is walked from the super-root in the ray's front-to-back order
// of octants (q ^ mask, mask the direction's sign bits), descending into
// internal nodes whose rectangle holds the pixel; a tile-level node
// contributes its (node, ray) aggregate, a leaf above the tile level its
// segment; the contributions are combined nearest first (Eq. 2.14).  The same
// result as the per-level passes up to rounding order (Eq. 2.14 is
// associative), in one launch and without intermediate aggregates in HBM.
constexpr int kTopDownThreads = 128;
constexpr int kMaxTopDownDepth = 24;

template <bool SURF>
__global__ void __launch_bounds__(kTopDownThreads)
    topdown_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, long long npix, float4 *rgba) {
  __shared__ float4 s_tfv[8], s_tfs[8];
  __shared__ unsigned long long s_cnt[3];
  const int tid = threadIdx.x;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  if (tid < 3) s_cnt[tid] = 0ull;
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  const float scale = ldexpf(1.f, -T.L);
  unsigned hits = 0, tests = 0;
  int steps = 0;
  for (long long pix = (long long)blockIdx.x * kTopDownThreads + tid; pix < npix;
       pix += (long long)gridDim.x * kTopDownThreads) {
    const int i = (int)(pix % c.w), j = (int)(pix / c.w);
    float3 org, dir;
    pixel_ray(c, i, j, org, dir);
    const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
    const int mask = (dir.x < 0.f ? 1 : 0) | (dir.y < 0.f ? 2 : 0) | (dir.z < 0.f ? 4 : 0);
    float4 acc = seg_identity();
    int nhit = 0;
    int stk[kMaxTopDownDepth];  // internal index of the node and the next octant to visit
    unsigned char sq[kMaxTopDownDepth];
    int sp = 0;
    stk[0] = T.M;  // the super-root
    sq[0] = 0;
    sp = 1;
    while (sp > 0) {
      const int nd = stk[sp - 1];
      const int q = sq[sp - 1];
      if (q == 8) {
        --sp;
        continue;
      }
      sq[sp - 1] = (unsigned char)(q + 1);
      const int ch = __ldg(T.child + 8 * nd + (q ^ mask));
      if (ch < 0) continue;
      const int4 r = __ldg(S.rect + ch);
      if (i < r.x || i > r.y || j < r.z || j > r.w) continue;
      if (ch < T.N) {  // a leaf above the tile level
        ++tests;
        const int4 g = __ldg(T.geo + ch);
        float a0, a1;
        if (slab(org, dir, inv, node_lo(g, scale), ldexpf(1.f, -g.w), c.amin, c.amax, a0, a1)) {
          acc = seg_combine(acc, leaf_segment<SURF>(T, Fd, c, I, tf, ch, org, dir, inv, scale,
                                                    steps));
          ++nhit;
        }
      } else if (__ldg(T.geo + ch).w == T.lt) {  // a tile-level node: its aggregate
        const long long e = __ldg(S.off + ch - T.N) + (long long)(j - r.z) * (r.y - r.x + 1) +
                            (i - r.x);
        acc = seg_combine(acc, S.entries[e]);
      } else if (sp < kMaxTopDownDepth) {
        stk[sp] = ch - T.N;
        sq[sp] = 0;
        ++sp;
      }
    }
    rgba[pix] = make_float4(fmaf(acc.x, I.bg[0], acc.y), fmaf(acc.x, I.bg[1], acc.z),
                            fmaf(acc.x, I.bg[2], acc.w), kOne - acc.x);
    if (nhit && S.counts) S.counts[pix] += nhit;  // after the subtree pass, in stream order
    hits += nhit;
  }
  // counters: segments, RK steps and leaf tests of the levels above the tile level
  unsigned long long v[3] = {hits, (unsigned long long)steps, tests};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0 && x) atomicAdd(&s_cnt[q], x);
  }
  __syncthreads();
  if (tid < 3 && s_cnt[tid]) atomicAdd(S.stats + kStatCoarse + tid, s_cnt[tid]);
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
  const long long per = kSubtreeThreads / kChunk;  // chunks per CTA
  const long long nblk = ((s1 - 1) / kChunk - s0 / kChunk + per) / per;
  if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  if (I.surface)  // isosurface segments (Sec. 2.8): a separate instantiation
    subtree_kernel<true><<<(unsigned)nblk, kSubtreeThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne,
                                                                         s0, s1);
  else
    subtree_kernel<false><<<(unsigned)nblk, kSubtreeThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne,
                                                                          s0, s1);
  return cudaGetLastError();
}

cudaError_t launch_coarsen(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                           Scratch S, int nb, int ne, long long s0, long long s1, float4 *rgba,
                           cudaStream_t stream) {
  if (s1 <= s0) return cudaSuccess;
  const long long nblk = rgba ? (s1 - s0 + kCoarsenThreads - 1) / kCoarsenThreads
                              : (s1 - 1) / kCoarsenThreads - s0 / kCoarsenThreads + 1;
  if (nblk > 0x7fffffffll) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)nblk;
  if (rgba && I.surface)
    coarsen_kernel<true, true><<<g, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1,
                                                                   rgba);
  else if (rgba)
    coarsen_kernel<true, false><<<g, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1,
                                                                    rgba);
  else if (I.surface)
    coarsen_kernel<false, true><<<g, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1,
                                                                    nullptr);
  else
    coarsen_kernel<false, false><<<g, kCoarsenThreads, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0,
                                                                     s1, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_topdown(const Topo &T, const Field &Fd, const Cam &C, const Integ &I, Scratch S,
                           long long npix, float4 *rgba, int nsm, cudaStream_t stream) {
  if (npix <= 0) return cudaSuccess;
  const long long need = (npix + kTopDownThreads - 1) / kTopDownThreads;
  const long long cap = (long long)(nsm > 0 ? nsm : 1) * 16;
  const unsigned g = (unsigned)(need < cap ? need : cap);
  if (I.surface)
    topdown_kernel<true><<<g, kTopDownThreads, 0, stream>>>(T, Fd, C, I, S, npix, rgba);
  else
    topdown_kernel<false><<<g, kTopDownThreads, 0, stream>>>(T, Fd, C, I, S, npix, rgba);
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
      if (g.w < 0 || g.w > L) {
        // not a cube leaf record of this depth (e.g. a shell record, whose
        // fourth word carries the tree above bit 8): flagged, never culled
        atomicOr(scratch + 1, 2ull);
        if (rects) rects[k] = empty_rect();
        continue;
      }
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
            atomicOr(scratch + 1, 1ull);
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
  // the same float32 camera constants as ocr_set_camera (one routine for both)
  Cam k{};
  to_cam(cc, k);

  // device address of the scratch array: looked up once per device, with that
  // device current (the array's name is only a stand-in in host code).  The
  // address is kept for the life of the process, so the call must not be used
  // on a device after cudaDeviceReset (which unloads the module holding it).
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
  if (h_err & 2ull) return OCR_ERR_INVALID;  // a record that is not a cube leaf of this depth
  if (h_err) return OCR_ERR_DEVICE;          // a look-back wait that gave up
  *h_nvisible = (int64_t)(h_last & kTileValue);
  return OCR_OK;
}
