// Persistent multi-camera render of a cube forest (the paper's multiple image
// instances, Sec. 3; the pipeline of Algorithm 2 for every camera).
//
// One kernel renders every camera of the batch.  Its CTAs (a few per SM, for
// the whole launch) draw tickets from a device-wide counter; the tickets
// enumerate a static work queue built when the cameras are planned: for each
// stage of the pipeline -- pruning (Sec. 3.1), the rectangle unions of the
// internal nodes level by level, the two halves of the slot prefix sum and the
// chunk map (the load balance, Sec. 3.1 / 3.2), the subtree pass (Sec. 3.2
// and Sec. 3.3 below the tile level), one coarsening level at a time
// (Sec. 3.3), the pixel pass (Sec. 2.4) -- the items of every camera, stage
// after stage.  An item first waits until its camera's previous stage is
// complete (a per-(camera, stage) counter of finished tickets), then runs the
// same chunk code as the single-camera kernels, reading data that other CTAs
// wrote during this launch through L2.
//
// Every item waits only for tickets drawn before its own, and a drawn ticket
// belongs to a running CTA that finishes it without waiting for later
// tickets, so the queue always drains.  A wait is nevertheless bounded: after
// about two seconds it raises the abort word and the error counter, and every
// CTA leaves at its next ticket; the host then reports a device error.
#include "ocr_common.h"
#include "ocr_device.cuh"
#include "ocr_passes.cuh"

#include <climits>

namespace ocr {
namespace {

constexpr int kBT = kChunk;                 // threads per CTA
constexpr int kBItems = 8;                  // units per thread of the set-up items
constexpr int kBTile = kBT * kBItems;       // leaves / nodes per set-up item
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

struct ScanSmem {
  long long wsum[kBT / 32];
  long long total, before;
};

union BatchSmem {
  SubtreeSmem st[kBT / 32];
  CoarsenSmem co;
  ScanSmem sc;
};

__device__ __forceinline__ long long rect_area_b(int4 r) {
  return r.x > r.y ? 0ll : (long long)(r.y - r.x + 1) * (long long)(r.w - r.z + 1);
}

// slots of internal node k: its rectangle's area at or above the tile level
__device__ __forceinline__ long long node_slots_b(const Topo &T, const int4 *rect, int k) {
  return __ldg(T.geo + T.N + k).w > T.lt ? 0ll : rect_area_b(__ldcg(rect + T.N + k));
}

// Sum of v over the CTA (every thread gets it).
__device__ __forceinline__ long long cta_sum(long long v, ScanSmem &sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sm.wsum[wid] = v;
  __syncthreads();
  long long t = 0;
#pragma unroll
  for (int w = 0; w < kBT / 32; ++w) t += sm.wsum[w];
  __syncthreads();
  return t;
}

// Exclusive prefix of v over the CTA in thread order; *total the sum.
__device__ __forceinline__ long long cta_exclusive(long long v, ScanSmem &sm, long long &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm.wsum[wid] = x;
  __syncthreads();
  long long before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kBT / 32; ++w) {
    if (w < wid) before += sm.wsum[w];
    tot += sm.wsum[w];
  }
  __syncthreads();
  total = tot;
  return before + x - v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// MINB: the CTAs per SM the kernel is compiled for (8: at most 64 registers,
// with some spills; 7: 72; 6: up to 80, none).
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB)
    batch_kernel(Topo T, Field Fd, Integ I, const BatchSeg *__restrict__ seg, int nseg,
                 const BatchCam *__restrict__ cams, unsigned *ctl, long long ntickets,
                 float4 *rgba, int *counts, unsigned char *visible,
                 unsigned long long *stats, unsigned long long *counters) {
  __shared__ BatchSmem sm;
  // the current item's camera and scratch, its segment and ticket, and the
  // queue state of thread 0 (kept in shared memory, not in registers)
  __shared__ Cam s_cam;
  __shared__ Scratch s_S;
  __shared__ float4 *s_rgba;
  __shared__ BatchSeg s_seg;
  __shared__ long long s_ticket, s_next;
  __shared__ int s_go, s_cs, s_ready, s_cur_cam;
  const int tid = threadIdx.x;
  unsigned *abort_word = ctl + 1, *done = ctl + 2;
  unsigned long long *ticket_ctr = reinterpret_cast<unsigned long long *>(ctl + 2 + kBatchMaxSegs);
  if (tid == 0) {
    s_next = (long long)atomicAdd(ticket_ctr, 1ull);
    s_cs = 0;
    s_ready = -1;  // a segment whose previous stage was seen complete
    s_cur_cam = -1;
  }
  for (;;) {
    if (tid == 0) {
      const long long t = s_next;
      if (t < ntickets && !ld_acquire(abort_word)) {
        s_next = (long long)atomicAdd(ticket_ctr, 1ull);  // used at the next trip
        // the segment holding ticket t (tickets rise with the segment index)
        int cs = s_cs;
        if (!(t >= seg[cs].first && (cs + 1 == nseg || t < seg[cs + 1].first))) {
          int lo = 0, hi = nseg - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg[mid].first <= t) lo = mid; else hi = mid - 1;
          }
          cs = lo;
          s_cs = cs;
        }
        s_seg = seg[cs];
        s_ticket = t - seg[cs].first;
        s_go = 1;
        // wait for the camera's previous stage (once per segment and CTA)
        const int dep = seg[cs].dep;
        if (dep >= 0 && s_ready != cs) {
          const unsigned need = (unsigned)seg[dep].ntickets;
          const long long t0 = clock64();
          while (ld_acquire(done + dep) < need) {
            if (ld_acquire(abort_word)) {
              s_go = 0;
              break;
            }
            if (clock64() - t0 > kWaitCycles) {
              atomicExch(abort_word, 1u);
              atomicAdd(stats + kStatErrors, 1ull);
              s_go = 0;
              break;
            }
            __nanosleep(256);
          }
          s_ready = cs;
        }
        const int cam = seg[cs].cam;
        if (cam != s_cur_cam) {  // this camera's scratch
          const BatchCam &bc = cams[cam];
          s_S = Scratch{bc.rect, bc.off, bc.entries, stats,
                        counts ? counts + bc.pix_off : nullptr, visible, bc.chunk, counters};
          s_rgba = rgba + bc.pix_off;
        }
      } else {
        s_go = 0;
      }
    }
    __syncthreads();
    if (!s_go) break;
    const BatchSeg &g = s_seg;
    const long long tk = s_ticket;
    if (g.cam != s_cur_cam) {  // this camera's constants into shared memory
      const int *src = reinterpret_cast<const int *>(&cams[g.cam].cam);
      int *dst = reinterpret_cast<int *>(&s_cam);
      for (int q = tid; q < (int)(sizeof(Cam) / sizeof(int)); q += kBT) dst[q] = __ldg(src + q);
      __syncthreads();
      if (tid == 0) s_cur_cam = g.cam;
    }
    const Scratch &S = s_S;
    const float scale = exp2i(-T.L);
    for (long long it = tk * g.per; it < min((tk + 1) * g.per, g.nitems); ++it) {
      if (g.kind == kBatchCull) {
        unsigned nvis = 0;
#pragma unroll 1
        for (int q = 0; q < kBItems; ++q) {
          const long long k = it * kBTile + q * kBT + tid;
          bool vis = false;
          if (k < T.N) {
            const int4 gg = __ldg(T.geo + k);
            const int4 r = box_rect(s_cam, node_lo(gg, scale), exp2i(-gg.w));
            S.rect[k] = r;
            vis = r.x <= r.y;
            if (visible && vis) visible[k] = 1;
          }
          nvis += __popc(__ballot_sync(0xffffffffu, vis));
        }
        if ((tid & 31) == 0 && nvis) atomicAdd(stats + kStatVisible, (unsigned long long)nvis);
      } else if (g.kind == kBatchUnion) {
#pragma unroll 1
        for (int q = 0; q < kBItems; ++q) {
          const long long k = g.a + it * kBTile + q * kBT + tid;
          if (k >= g.b) continue;
          int4 u = make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int id = __ldg(T.child + 8 * k + c);
            if (id < 0) continue;
            const int4 r = __ldcg(S.rect + id);
            if (r.x > r.y) continue;
            u.x = min(u.x, r.x); u.y = max(u.y, r.y); u.z = min(u.z, r.z); u.w = max(u.w, r.w);
          }
          S.rect[T.N + k] = (u.x <= u.y) ? u : empty_rect();
        }
      } else if (g.kind == kBatchReduce) {
        long long v = 0;
#pragma unroll 1
        for (int q = 0; q < kBItems; ++q) {
          const long long k = it * kBTile + q * kBT + tid;
          if (k < T.M) v += node_slots_b(T, S.rect, (int)k);
        }
        const long long tot = cta_sum(v, sm.sc);
        if (tid == 0) cams[g.cam].bsums[it] = tot;
      } else if (g.kind == kBatchDown) {
        // the prefix of the earlier blocks, then this block's 1024 nodes in order
        long long v = 0;
        const long long *bsums = cams[g.cam].bsums;
        for (long long b = tid; b < it; b += kBT) v += __ldcg(bsums + b);
        long long run = cta_sum(v, sm.sc);
        const long long base = it * kBTile + (long long)tid * kBItems;
        long long a[kBItems], s = 0;
#pragma unroll
        for (int q = 0; q < kBItems; ++q) {
          a[q] = base + q < T.M ? node_slots_b(T, S.rect, (int)(base + q)) : 0ll;
          s += a[q];
        }
        long long tot;
        run += cta_exclusive(s, sm.sc, tot);
#pragma unroll
        for (int q = 0; q < kBItems; ++q) {
          if (base + q < T.M) S.off[base + q] = run;
          run += a[q];
        }
        if (it == g.nitems - 1 && tid == kBT - 1) S.off[T.M] = run;
      } else if (g.kind == kBatchChunkMap) {
#pragma unroll 1
        for (int q = 0; q < kBItems; ++q) {
          const long long gi = it * kBTile + q * kBT + tid;  // a group of kGroup slots
          if (gi < g.b) S.chunk_node[gi] = node_of_slot<true>(S.off, T.M, gi * kGroup);
        }
      } else if (g.kind == kBatchSubtree) {
        subtree_warp<false, true>(T, Fd, s_cam, I, S, g.nb, g.ne, g.a, g.b,
                                  (g.a / kChunk + it) * kChunk + (tid & ~31), sm.st[tid >> 5]);
      } else if (g.kind == kBatchCoarse) {
        coarsen_chunk<false, false, true>(T, Fd, s_cam, I, S, g.nb, g.ne, g.a, g.b, it, nullptr,
                                          sm.co);
      } else {  // kBatchPixel
        coarsen_chunk<true, false, true>(T, Fd, s_cam, I, S, T.M, T.M, 0, g.b, it, s_rgba,
                                         sm.co);
      }
      __syncthreads();  // shared memory free for the next item
    }
    // publish the ticket: every thread's writes, then the counter of the
    // segment thread 0 found for it
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done + s_cs, 1u);
  }
}

}  // namespace

cudaError_t launch_batch(const Topo &T, const Field &Fd, const Integ &I, const BatchSeg *d_seg,
                         int nseg, const BatchCam *d_cams, unsigned *d_ctl, long long ntickets,
                         float4 *rgba, int *counts, unsigned char *visible,
                         unsigned long long *stats, bool count, int nsm, int ctas_per_sm,
                         cudaStream_t stream) {
  unsigned long long *counters = count ? stats : nullptr;
  if (nseg < 1 || nseg > kBatchMaxSegs || ntickets < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(d_ctl, 0, sizeof(unsigned) * kBatchCtlWords, stream);
  if (e != cudaSuccess) return e;
  // the variant compiled for the CTAs per SM asked for (1..6: the one for 6,
  // 7: for 7, 0 or 8: for 8 -- fewer CTAs per SM leave more registers)
  const int v = ctas_per_sm == 0 ? 8 : ctas_per_sm <= 6 ? 6 : ctas_per_sm;
  static int fit[9] = {};  // resident CTAs per SM of each variant
  if (!fit[v]) {
    e = v == 6   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit[v], batch_kernel<6>, kBT, 0)
        : v == 7 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit[v], batch_kernel<7>, kBT, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit[v], batch_kernel<8>, kBT, 0);
    if (e != cudaSuccess) return e;
  }
  int per_sm = fit[v];
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)(nsm > 0 ? nsm : 1) * per_sm;
  if (grid > ntickets) grid = ntickets;
  const unsigned g = (unsigned)grid;
  if (v == 6)
    batch_kernel<6><<<g, kBT, 0, stream>>>(T, Fd, I, d_seg, nseg, d_cams, d_ctl, ntickets, rgba,
                                           counts, visible, stats, counters);
  else if (v == 7)
    batch_kernel<7><<<g, kBT, 0, stream>>>(T, Fd, I, d_seg, nseg, d_cams, d_ctl, ntickets, rgba,
                                           counts, visible, stats, counters);
  else
    batch_kernel<8><<<g, kBT, 0, stream>>>(T, Fd, I, d_seg, nseg, d_cams, d_ctl, ntickets, rgba,
                                           counts, visible, stats, counters);
  return cudaGetLastError();
}

}  // namespace ocr
