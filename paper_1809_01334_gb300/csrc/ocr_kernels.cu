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
#include "ocr_passes.cuh"

#include <algorithm>
#include <cstdio>

namespace ocr {
namespace {

__global__ void cull_leaves_kernel(Topo T, Cam c, Scratch S) {
  const float scale = exp2i(-T.L);
  unsigned nvis = 0;
  // the loop bound is warp-uniform so that the ballot below sees full warps
  const int stride = gridDim.x * blockDim.x;
  for (int k0 = blockIdx.x * blockDim.x; k0 < T.N; k0 += stride) {
    const int k = k0 + threadIdx.x;
    bool vis = false;
    if (k < T.N) {
      const int4 g = T.geo[k];
      const int4 r = box_rect(c, node_lo(g, scale), exp2i(-g.w));
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

// chunk_node[g] = the internal node whose slot range holds slot g * kGroup:
// one thread per group
__global__ void chunk_map_kernel(Topo T, Scratch S, long long ngroups) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ngroups;
       g += (long long)gridDim.x * blockDim.x)
    S.chunk_node[g] = node_of_slot<false>(S.off, T.M, g * kGroup);
}

__global__ void gather_level_slots_kernel(const long long *off, const int *level_nodes, int n,
                                          long long *out) {
  const int k = threadIdx.x;
  if (k < n) out[k] = off[level_nodes[k]];
}

// ------------------------------------------------- subtree and coarsen --
// The bodies are in ocr_passes.cuh.  The subtree pass: resident one-warp
// CTAs, 32 per SM, that draw the groups of 32 slots in turn from a counter
// (a warp that is done takes the next group at once, with no block launch per
// group).
template <bool SURF>
__global__ void __launch_bounds__(32, 32)
    subtree_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, int nb, int ne,
                          long long s0, long long s1, unsigned ngroups) {
  __shared__ SubtreeSmem sm;
  while (true) {
    unsigned t = 0;
    if (threadIdx.x == 0) t = atomicAdd(S.ticket, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ngroups) break;
    subtree_warp<SURF, false>(T, Fd, c, I, S, nb, ne, s0, s1, (s0 / 32 + t) * 32, sm);
    __syncwarp();
  }
}

template <bool FINAL, bool SURF>
__global__ void __launch_bounds__(kCoarsenThreads, 8)
    coarsen_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, int nb, int ne, long long s0,
                   long long s1, float4 *rgba) {
  __shared__ CoarsenSmem sm;
  coarsen_chunk<FINAL, SURF, false>(T, Fd, c, I, S, nb, ne, s0, s1, blockIdx.x, rgba, sm);
}

// The segments of the leaves at or above the tile level, one thread per
// (leaf, ray) slot of the listed leaves' rectangles: the slot's leaf (the
// group's slot-map entry, a search past that leaf's end), pixel and ray; a
// ray that meets the leaf (slab test) gets the leaf's segment, integrated as
// in the other passes, else the identity.
template <bool SURF>
__global__ void __launch_bounds__(128)
    coarse_leaves_kernel(Topo T, Field Fd, Cam c, Integ I, Scratch S, CoarseLeaves CL) {
  __shared__ float4 s_tfv[8], s_tfs[8];
  const int tid = threadIdx.x;
  if (tid < 8) {
    const float4 v = Fd.tf[tid];
    const float4 w = Fd.tf[tid < 7 ? tid + 1 : 7];
    s_tfv[tid] = v;
    s_tfs[tid] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
  }
  __syncthreads();
  const TF tf{s_tfv, s_tfs, Fd.s_min, Fd.inv_ds7};
  const float scale = exp2i(-T.L);
  const long long slot = (long long)blockIdx.x * 128 + tid;
  unsigned hit = 0;
  int steps = 0;
  if (slot < CL.total) {
    int k = CL.group[slot / kGroup];
    if (slot >= CL.off[k + 1]) {  // past the group's first leaf: the last k with off[k] <= slot
      int lo = k + 1, hi = CL.n;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (CL.off[mid] <= slot) lo = mid + 1; else hi = mid;
      }
      k = lo - 1;
    }
    const int leaf = CL.ids[k];
    const int4 r = S.rect[leaf];
    int i, j;
    slot_pixel(r, (unsigned)(slot - CL.off[k]), i, j);  // < w * h < 2^31
    float3 org, dir;
    pixel_ray(c, i, j, org, dir);
    const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
    const int4 g = __ldg(T.geo + leaf);
    float a0, a1;
    float4 v = seg_identity();
    if (slab(org, dir, inv, node_lo(g, scale), exp2i(-g.w), c.amin, c.amax, a0, a1)) {
      v = leaf_segment<SURF>(T, Fd, c, I, tf, leaf, org, dir, inv, scale, steps);
      hit = 1;
      if (S.counts) atomicAdd(S.counts + (size_t)j * c.w + i, 1);
    }
    CL.val[slot] = v;
  }
  if (S.counters) {  // segments, RK steps, slab tests above the tile level
    const unsigned v[3] = {hit, (unsigned)steps, slot < CL.total ? 1u : 0u};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const unsigned x = __reduce_add_sync(0xffffffffu, v[q]);
      if ((tid & 31) == 0 && x) atomicAdd(S.counters + kStatCoarse + q, (unsigned long long)x);
    }
  }
}

// group[g] = the listed leaf whose slots hold slot g * kGroup
__global__ void coarse_leaf_map_kernel(CoarseLeaves CL, long long ngroups) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ngroups;
       g += (long long)gridDim.x * blockDim.x) {
    const long long slot = g * kGroup;
    int lo = 0, hi = CL.n;
    while (lo < hi) {  // first leaf whose offset exceeds the slot
      const int mid = (lo + hi) >> 1;
      if (CL.off[mid] <= slot) lo = mid + 1; else hi = mid;
    }
    CL.group[g] = lo - 1;
  }
}

// Top-down merge of the levels above the tile level, one thread per pixel:
// the octree is walked from the tree root in the ray's front-to-back order of
// octants (bit q ^ flip, flip the direction's sign bits).  At each internal
// node above the tile level the children the ray meets come from one
// child_hits (the children's exact slab tests); a tile-level node whose pixel
// rectangle holds the pixel contributes its (node, ray) aggregate of the
// subtree pass, a leaf (at or above the tile level) whose rectangle holds it
// its segment from the listed leaves' pass, and an internal node is descended
// into.  The contributions are combined nearest first (Eq. 2.14): the result
// of the per-level passes up to rounding order (Eq. 2.14 is associative), in
// one launch and without intermediate aggregates in HBM.  A node the ray
// misses holds nothing the ray meets (nested boxes, monotone rounding), and a
// node whose rectangle misses the pixel holds no leaf whose rectangle holds
// it, so only the contributors' rectangles are checked.
constexpr int kTopDownThreads = 128;

__global__ void __launch_bounds__(kTopDownThreads)
    topdown_kernel(Topo T, Cam c, Integ I, Scratch S, CoarseLeaves CL, long long npix,
                   float4 *rgba) {
  extern __shared__ int2 s_stk[];  // [(lt + 1) * kTopDownThreads] ancestors: node, children left
  const int tid = threadIdx.x;
  const float scale = exp2i(-T.L);
  // a CTA takes a 16 x 8 tile of pixels (rays closer together than a row's)
  const int tiles_x = (c.w + 15) / 16;
  const int i = (int)(blockIdx.x % tiles_x) * 16 + (tid & 15);
  const int j = (int)(blockIdx.x / tiles_x) * 8 + (tid >> 4);
  if (i >= c.w || j >= c.h) return;
  const long long pix = (long long)j * c.w + i;
  (void)npix;
  float3 org, dir;
  pixel_ray(c, i, j, org, dir);
  const float3 inv = make_float3(recip_or_zero(dir.x), recip_or_zero(dir.y), recip_or_zero(dir.z));
  const unsigned flip = (dir.x < 0.f ? 1u : 0u) | (dir.y < 0.f ? 2u : 0u) | (dir.z < 0.f ? 4u : 0u);
  const int4 *child4 = reinterpret_cast<const int4 *>(T.child);
  float4 acc = seg_identity();
  // the super-root (internal index M, level -1): its one child is the tree root
  int cur = T.M, lev = -1, gx = 0, gy = 0, gz = 0, d = 0;
  int4 c0 = __ldg(child4 + 2 * T.M), c1 = __ldg(child4 + 2 * T.M + 1);
  unsigned msk = 0u;
  if (c0.x >= 0) {
    const int4 g = __ldg(T.geo + c0.x);
    float a0, a1;
    if (slab(org, dir, inv, node_lo(g, scale), exp2i(-g.w), c.amin, c.amax, a0, a1))
      msk = 1u << flip;  // octant 0, mirrored
  }
  while (true) {
    if (msk == 0u) {  // this node is done: back to its parent
      if (d == 0) break;
      --d;
      --lev;
      const int keep = ~((1 << (T.L - lev)) - 1);
      gx &= keep;
      gy &= keep;
      gz &= keep;
      const int2 e = s_stk[d * kTopDownThreads + tid];
      cur = e.x;
      msk = (unsigned)e.y;
      c0 = __ldg(child4 + 2 * cur);
      c1 = __ldg(child4 + 2 * cur + 1);
      continue;
    }
    const int q = (__ffs(msk) - 1) ^ (int)flip;
    msk &= msk - 1u;
    const int id = pick_child(c0, c1, q);
    if (id < 0) continue;
    if (id < T.N || lev + 1 == T.lt) {
      const bool leaf = id < T.N;
      const int4 r = __ldg(S.rect + id);
      const long long o = leaf ? __ldg(CL.off + __ldg(CL.index + id)) : __ldg(S.off + id - T.N);
      if (i < r.x || i > r.y || j < r.z || j > r.w) continue;
      const long long e = o + slot_of_pixel(r, i, j);
      acc = seg_combine(acc, leaf ? CL.val[e] : S.entries[e]);
      continue;
    }
    // an internal node above the tile level
    s_stk[d * kTopDownThreads + tid] = make_int2(cur, (int)msk);
    ++d;
    const int hs = 1 << (T.L - lev - 1);
    gx += (q & 1) * hs;
    gy += ((q >> 1) & 1) * hs;
    gz += (q >> 2) * hs;
    ++lev;
    cur = id - T.N;
    msk = child_hits(org, dir, inv, node_lo(make_int4(gx, gy, gz, 0), scale),
                     exp2i(-(lev + 1)), c.amin, c.amax);
    if (msk) {
      c0 = __ldg(child4 + 2 * cur);
      c1 = __ldg(child4 + 2 * cur + 1);
    }
  }
  rgba[pix] = make_float4(fmaf(acc.x, I.bg[0], acc.y), fmaf(acc.x, I.bg[1], acc.z),
                          fmaf(acc.x, I.bg[2], acc.w), kOne - acc.x);
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

cudaError_t launch_chunk_map(const Topo &T, Scratch S, long long total, cudaStream_t stream) {
  const long long ngroups = (total + kGroup - 1) / kGroup;
  if (T.M < 1 || ngroups < 1) return cudaSuccess;
  chunk_map_kernel<<<grid_for(ngroups, 256), 256, 0, stream>>>(T, S, ngroups);
  return cudaGetLastError();
}

cudaError_t launch_subtree(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                           Scratch S, int nb, int ne, long long s0, long long s1,
                           cudaStream_t stream) {
  if (s1 <= s0) return cudaSuccess;
  const long long nblk = (s1 - 1) / 32 - s0 / 32 + 1;  // one warp per 32 slots
  if (nblk > 0x7fffffffll || !S.ticket) return cudaErrorInvalidValue;
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const unsigned g = (unsigned)std::min<long long>(nblk, 32ll * nsm);
  if (I.surface)  // isosurface segments (Sec. 2.8): a separate instantiation
    subtree_kernel<true><<<g, 32, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1, (unsigned)nblk);
  else
    subtree_kernel<false><<<g, 32, 0, stream>>>(T, Fd, C, I, S, nb, ne, s0, s1, (unsigned)nblk);
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

cudaError_t launch_coarse_leaf_map(const CoarseLeaves &CL, cudaStream_t stream) {
  const long long ngroups = (CL.total + kGroup - 1) / kGroup;
  if (CL.n < 1 || ngroups < 1) return cudaSuccess;
  coarse_leaf_map_kernel<<<grid_for(ngroups, 256), 256, 0, stream>>>(CL, ngroups);
  return cudaGetLastError();
}

cudaError_t launch_coarse_leaves(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                                 Scratch S, const CoarseLeaves &CL, cudaStream_t stream) {
  if (CL.n < 1 || CL.total < 1) return cudaSuccess;
  const long long need = (CL.total + 127) / 128;
  if (need > 0x7fffffffll) return cudaErrorInvalidValue;
  if (I.surface)  // isosurface segments (Sec. 2.8): a separate instantiation
    coarse_leaves_kernel<true><<<(unsigned)need, 128, 0, stream>>>(T, Fd, C, I, S, CL);
  else
    coarse_leaves_kernel<false><<<(unsigned)need, 128, 0, stream>>>(T, Fd, C, I, S, CL);
  return cudaGetLastError();
}

cudaError_t launch_topdown(const Topo &T, const Cam &C, const Integ &I, Scratch S,
                           const CoarseLeaves &CL, long long npix, float4 *rgba,
                           cudaStream_t stream) {
  if (npix <= 0) return cudaSuccess;
  static_assert(kTopDownThreads == 128, "16 x 8 pixel tiles");
  const long long need = (long long)((C.w + 15) / 16) * ((C.h + 7) / 8);
  if (need > 0x7fffffffll || (long long)C.w * C.h != npix) return cudaErrorInvalidValue;
  const size_t stk = sizeof(int2) * kTopDownThreads * (size_t)(T.lt + 1);  // the walk's ancestors
  topdown_kernel<<<(unsigned)need, kTopDownThreads, stk, stream>>>(T, C, I, S, CL, npix, rgba);
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
  const float scale = exp2i(-L);
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
      const int4 r = box_rect(c, node_lo(g, scale), exp2i(-g.w));
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
