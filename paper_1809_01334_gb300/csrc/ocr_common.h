// Internal declarations shared by the host API (ocr_capi.cu) and the kernels
// (ocr_kernels.cu).  Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ocraycast.h"

namespace ocr {

// Camera constants in float32, derived once per ocr_set_camera.
//  perspective: ray (i, j) = o + alpha r, r = v + (i - cw) lt + (j - ch) lu
//  orthographic: origin o + (i - cw) lt + (j - ch) lu, direction v (= v/n)
// (t, u, vn) are the rows of the camera transform X = (t, u, v/n)^T (x - o).
struct Cam {
  float o[3], v[3], lt[3], lu[3];
  float t[3], u[3], vn[3];
  float n, f, ell, cw, ch;
  float amin, amax;
  int w, h, ortho;
};

// The float32 constants of a host camera: one routine for every entry point
// that reads a camera (ocr_set_camera, ocr_prune_noalloc).
void to_cam(const ocr_camera &c, Cam &k);

struct Integ {
  int method;  // 0 RK4 x nsteps; inside Algorithm 1: 1 DOPRI5, 2 Gauss-2, 3 Simpson, 4 Eq. 2.18
  int nsteps;
  float tol, c_rk;
  int max_depth;
  float bg[3];
  int surface;           // isosurface s = s_iso rendered with (a_s, i_s) (Sec. 2.8)
  float s_iso, a_s, i_s[3];
};

// Unified node numbering: [0, N) leaves in Morton order, [N, N + M) internal
// octree nodes grouped by level from the deepest to the root, N + M the
// super-root whose only child is the tree root.  geo = {x, y, z, level} with
// anchors in units of 2^-L (level -1 for the super-root).
// Internal nodes deeper than the tile level lt keep no per-ray aggregates: the
// subtree pass handles each tile-level node's whole subtree (depth L - lt <= 3)
// in one thread per ray.
struct Topo {
  const int4 *geo;     // [N + M + 1]
  const int *child;    // [(M + 1) * 8]  unified ids, -1 = none; slot = octant bx + 2 by + 4 bz
  const int2 *leaves;  // [M] Morton range [first, last + 1) of each internal node's leaves
  int N, M, L, lt;
};

// Subtree pass: a ray crosses at most 3 * 2^D - 2 = 46 cells of a depth-4
// subtree; the per-ray list holds 48 to leave room for rays running exactly
// along cell faces (closed slab tests accept both sides).  Overflow is counted
// as a device error.
constexpr int kSubtreeDepth = 4;
constexpr int kMaxSubtreeHits = 48;
constexpr int kDefaultTileDepth = 4;  // the tile depth of a new forest (1..kSubtreeDepth)

struct Field {
  const float *nodal;  // [N * 8]
  const float4 *tf;    // [8] (kappa, q_r, q_g, q_b) at the knots
  float s_min, inv_ds7;  // knot position z = (s - s_min) * inv_ds7, inv_ds7 = 7 / (s_max - s_min)
};

struct Scratch {
  int4 *rect;                // [N + M + 1] {i0, i1, j0, j1}; empty = {0, -1, 0, -1}
  long long *off;            // [M + 1] exclusive prefix of internal-node rectangle areas
  float4 *entries;           // [total slots] per (internal node, ray) aggregate (A, B_r, B_g, B_b)
  unsigned long long *stats; // [kStats] counters, see below
  int *counts;               // optional [w * h]
  unsigned char *visible;    // optional [N]
  int *chunk_node;           // [ceil(total / kGroup) + 1] internal node holding slot g * kGroup
  unsigned long long *counters;  // optional [kStats]: the passes' work counters, when asked for
  unsigned *ticket;          // optional, zeroed: the subtree pass's warps draw their groups here
};

// Device counters: [0, 4) subtree pass, [kStatCoarse, kStatCoarse + 4) coarse
// passes, each {segments, RK steps, slab tests (subtree: node visits), slots},
// counted only when Scratch::counters is set; then device errors and visible
// leaves, always counted.
constexpr int kStats = 16;
constexpr int kStatSegments = 0, kStatSteps = 1, kStatTests = 2, kStatSlots = 3;
constexpr int kStatCoarse = 8, kStatErrors = 4, kStatVisible = 5;

// Slots are processed in chunks of kChunk consecutive slots, one chunk per CTA;
// the slot map (Scratch::chunk_node) has one entry per group of kGroup slots
// (one warp's slots).
constexpr int kChunk = 128;
constexpr int kGroup = 32;

// (leaf, pixel) pair spaces (the adjoint, the shell) are cut into chunks of
// kPairChunk pairs, one CTA each.
constexpr int kPairChunk = 256;

// Cubed-sphere shell (geometry 1).  Leaf geo = {x, y, z, level | tree << 8},
// anchors in units of 2^-L of the tree's reference cube.  The tangents of the
// equiangular planes and the radii of the spherical faces come from tables
// rounded once on the host, so that two leaves sharing a face compute
// bit-identical crossings of a ray with it.
struct Shell {
  const float *frames;   // [6 * 9] per tree: n, e1, e2
  const float *tan_tab;  // [2^L + 1] tan(pi/4 (2 k 2^-L - 1))
  const float *rad_tab;  // [2^L + 1] r0 + (r1 - r0) k 2^-L
  const float4 *planes;  // [N * 4] per leaf the normals m = e - T n of its four planes
                         // (xi low, xi high, eta low, eta high); w: r_in, r_out, 0, 0
  int L;
};
constexpr int kStatMaxHits = 6;  // shell: the most segments on one ray (atomicMax)

// Launch wrappers (ocr_kernels.cu).  All enqueue on `stream` and return the
// launch error.
cudaError_t launch_cull_leaves(const Topo &T, const Cam &C, Scratch S, cudaStream_t stream);
cudaError_t launch_union_level(const Topo &T, int node_begin, int node_end, const Cam &C,
                               Scratch S, cudaStream_t stream);
cudaError_t launch_area_scan(const Topo &T, Scratch S, long long *d_block_sums, int nblk_cap,
                             long long *d_level_slots, const int *d_level_nodes, int nlevels,
                             cudaStream_t stream);
int area_scan_blocks(int M);
cudaError_t launch_chunk_map(const Topo &T, Scratch S, long long total, cudaStream_t stream);
// S.ticket is required and must be zero (stream-ordered) before the launch.
cudaError_t launch_subtree(const Topo &T, const Field &Fd, const Cam &C, const Integ &I, Scratch S,
                           int node_begin, int node_end, long long slot_begin, long long slot_end,
                           cudaStream_t stream);
cudaError_t launch_coarsen(const Topo &T, const Field &Fd, const Cam &C, const Integ &I, Scratch S,
                           int node_begin, int node_end, long long slot_begin, long long slot_end,
                           float4 *rgba, cudaStream_t stream);
// The leaves at or above the tile level (level <= lt) of a cube forest, for
// the top-down merge: their (leaf, ray) segments are formed by one pass of
// their own, one slot per pixel of each listed leaf's rectangle.
struct CoarseLeaves {
  const int *ids;        // [n] the listed leaves, in Morton order
  const int *index;      // [N] a leaf's place in ids, -1 for the others
  long long *off;        // [n + 1] exclusive prefix of their rectangle areas (per render)
  int *group;            // [ceil(total / kGroup) + 1] listed leaf holding slot g * kGroup
  float4 *val;           // [total] (A, B) of each (leaf, ray) slot, the identity where the
                         // ray misses the leaf
  int n;
  long long total;       // slots (the plan's; every render has the same)
};
// the slot map of the listed leaves (after their offsets)
cudaError_t launch_coarse_leaf_map(const CoarseLeaves &CL, cudaStream_t stream);
// the listed leaves' segments, one thread per slot; the segment counts of
// S.counts and the coarse counters of S.counters
cudaError_t launch_coarse_leaves(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                                 Scratch S, const CoarseLeaves &CL, cudaStream_t stream);
// the levels above the tile level and the pixels in one pass: one thread per
// pixel walks the octree top-down, combining the tile-level aggregates and
// the listed leaves' segments (instead of the per-level coarsen passes)
cudaError_t launch_topdown(const Topo &T, const Cam &C, const Integ &I, Scratch S,
                           const CoarseLeaves &CL, long long npix, float4 *rgba,
                           cudaStream_t stream);

// Persistent multi-camera render of a cube forest (ocr_batch.cu).  The work
// queue is a list of segments, one per (pipeline stage, camera), in queue
// order (stage after stage, each stage for every camera); a segment's items
// are grouped `per` to a ticket.
constexpr int kBatchCull = 0, kBatchUnion = 1, kBatchReduce = 2, kBatchDown = 3,
              kBatchChunkMap = 4, kBatchSubtree = 5, kBatchCoarse = 6, kBatchPixel = 7;
constexpr int kBatchMaxSegs = 8192;
// control words: [1] abort, [2, 2 + kBatchMaxSegs) finished tickets per
// segment, then the 64-bit ticket counter; zeroed before every launch
constexpr int kBatchCtlWords = 2 + kBatchMaxSegs + 2;
struct BatchSeg {
  long long first;     // first ticket of the segment
  long long nitems;    // items of the stage for this camera
  long long ntickets;  // ceil(nitems / per)
  long long a, b;      // union: internal nodes [a, b); subtree / coarse: slots [a, b);
                       // pixel: b = the camera's pixels
  int cam, kind;
  int dep;             // the segment of the camera's previous stage, -1 for pruning
  int per;             // items per ticket
  int nb, ne;          // subtree / coarse: internal nodes [nb, ne) of the level
};
struct BatchCam {
  Cam cam;
  int4 *rect;
  long long *off, *bsums;
  int *chunk;
  float4 *entries;
  long long pix_off;
};
cudaError_t launch_batch(const Topo &T, const Field &Fd, const Integ &I, const BatchSeg *d_seg,
                         int nseg, const BatchCam *d_cams, unsigned *d_ctl, long long ntickets,
                         float4 *rgba, int *counts, unsigned char *visible,
                         unsigned long long *stats, bool count, int nsm, int ctas_per_sm,
                         cudaStream_t stream);

// Adjoint (ocr_backward.cu)
cudaError_t bwd_leaf_scan(const Topo &T, const int4 *rect, long long *bs, long long bs_cap,
                          long long *leaf_off, cudaStream_t st);
cudaError_t bwd_count_scan(const int *counts, long long n, long long *bs, long long bs_cap,
                           long long *ray_off, cudaStream_t st);
long long bwd_scan_blocks(long long n);
cudaError_t bwd_chunk_map(const long long *leaf_off, int N, int *chunk_leaf, cudaStream_t st);
// exclusive prefix of the rectangle areas of the leaves ids[0..n) into off
// [n + 1] (bs: block sums, [bwd_scan_blocks(n) + 1] at least)
cudaError_t listed_leaf_scan(const int4 *rect, const int *ids, long long n, long long *bs,
                             long long bs_cap, long long *off, cudaStream_t st);
// mode 0: hits per ray into counts (rays with a zero image adjoint skipped;
// dL null: every ray);
// mode 2: each hit's mirrored Morton key into its ray's list, and the hit
// appended to the leaf-grouped list lm (pixel, leaf) through *lm_count (zeroed
// by the caller), its index in kpos beside the key; more than key_cap hits
// are counted in err
cudaError_t bwd_pair_hits(int mode, const Topo &T, const Cam &C, const int4 *rect,
                          const long long *leaf_off, const int *chunk_leaf, long long npairs,
                          const float4 *dL, int *counts, const long long *ray_off, int *cursor,
                          const unsigned long long *mkey, unsigned long long fx,
                          unsigned long long *keys, unsigned *kpos, int2 *lm,
                          unsigned long long *lm_count, long long key_cap,
                          unsigned long long *err, cudaStream_t st);
// the most hits on one ray (atomicMax into *out, which the caller zeroes)
cudaError_t bwd_max_hits(const int *counts, long long n, unsigned long long *out,
                         cudaStream_t st);
// *err += *stat_err (the render passes' device error counter), on the stream
cudaError_t bwd_fold_errors(unsigned long long *err, const unsigned long long *stat_err,
                            cudaStream_t st);
// The three passes over a leaf-grouped list of nseg entries (cube: at most
// nseg, the count read from *ncount on the device when it is given).  Values:
// one thread per entry, the segment's (A, B) into val (shell: entries of rays
// with a zero image adjoint are skipped; missing pieces counted in err).
cudaError_t bwd_cube_values(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                            const int2 *lm, long long nseg, const unsigned long long *ncount,
                            float4 *val, int nsm, cudaStream_t st);
cudaError_t bwd_shell_values(const int4 *geo, int N, const Shell &S, const Field &Fd,
                             const Cam &C, const Integ &I, const float4 *dL, const int2 *lm,
                             long long nseg, float4 *val, unsigned long long *err, int nsm,
                             cudaStream_t st);
// Scans: one warp per ray, lists of up to cap entries (a power of two,
// 32..kShellMaxCap; longer lists are counted in err) starting at ray_off[pix],
// count[pix] entries long (count null: up to ray_off[pix + 1]): the values
// gathered from rec_g by the list indices in kpos, then per entry the near
// transmittance and own transmittance into rec_ta and the far aggregate into
// rec_g.
// bwd_scans_prepare raises the kernel's shared-memory limit for every cap.
size_t bwd_scans_smem(int cap);
cudaError_t bwd_scans_prepare();
cudaError_t bwd_ray_scans(const Cam &C, const float4 *dL, const long long *ray_off,
                          const int *count, const unsigned long long *keys, const unsigned *kpos,
                          long long key_cap, int cap, float2 *rec_ta, float4 *rec_g,
                          unsigned long long *err, int nsm, cudaStream_t st);
// Adjoint: one thread per entry; nodal adjoints summed over a warp's lanes of
// the same leaf, then accumulated into g_nodal, the knot adjoints into g_tf.
cudaError_t bwd_cube_adjoint(const Topo &T, const Field &Fd, const Cam &C, const Integ &I,
                             const float4 *dL, const int2 *lm, const float2 *rec_ta,
                             const float4 *rec_g, long long nseg,
                             const unsigned long long *ncount, float *g_nodal, float *g_tf,
                             int nsm, cudaStream_t st);

// Cubed-sphere shell (ocr_shell.cu)
// the per-leaf plane table (Shell::planes) from the frames and tables, once
// per forest
cudaError_t shell_planes(const int4 *geo, int N, const Shell &S, float4 *planes,
                         cudaStream_t st);
// the leaves' degree-2 data (27 Lagrange nodal values each) in monomial form
// (27 coefficients each, the polynomial the shell kernels evaluate)
cudaError_t shell_monomials(const float *nodal, float *coef, int N, cudaStream_t st);
cudaError_t shell_cull(const int4 *geo, int N, const Shell &S, const Cam &C, int4 *rect,
                       unsigned char *visible, unsigned long long *stats, cudaStream_t st);
// mode 0, the count pass: segments per ray into counts, which pairs hit into
// hitmask when it is given (one bit per pair, [ceil(npairs / kPairChunk) *
// kPairChunk / 32] words), and, when stats is given, the longest list into
// stats[kStatMaxHits]; mode 1, the fill pass: every pair intersected, each
// segment's key written at ray_off[pixel] + its place among the ray's
// segments (through cursor), at most key_cap of them and within the ray's
// list (more is a device error); mode 2: the fill pass that also appends
// every segment to the leaf-grouped list lm (pixel, 2 leaf + piece) through
// the counter *lm_count (zeroed by the caller) and stores its index there in
// kpos beside the key
cudaError_t shell_pairs(int mode, const int4 *geo, int N, const Shell &S, const Cam &C,
                        const int4 *rect, const long long *leaf_off, const int *chunk_leaf,
                        long long npairs, int *counts, const long long *ray_off, int *cursor,
                        unsigned long long *keys, long long key_cap, unsigned long long *stats,
                        unsigned *hitmask, cudaStream_t st, unsigned *kpos = nullptr,
                        int2 *lm = nullptr, unsigned long long *lm_count = nullptr);
// per-CTA warps and dynamic shared memory of shell_rays for rays of up to cap
// segments (cap a power of two, 32..kShellMaxCap); shell_rays_prepare raises the
// kernel's shared-memory limit to the largest of these and must run before the
// first launch
constexpr int kShellMaxCap = 4096;
int shell_ray_warps(int cap, int want);
size_t shell_ray_smem(int cap, int want);
cudaError_t shell_rays_prepare();
// the shell's per-ray merge (Eq. 2.14, cut and average of overlaps) of one
// list of n segments (values, intervals in order of entry) into *out
cudaError_t shell_fold_segments(const float4 *val, const float2 *iv, int n, float4 *out,
                                cudaStream_t st);
// every ray's list sorted in place by its key (before shell_rays); ticket: a
// counter zeroed before the launch (the warps draw their rays there)
cudaError_t shell_sort_lists(const long long *ray_off, long long npix, unsigned long long *keys,
                             long long key_cap, int cap, int nsm, unsigned *ticket,
                             cudaStream_t st);
cudaError_t shell_rays(const int4 *geo, int N, const Shell &S, const Field &Fd, const Cam &C,
                       const Integ &I, const long long *ray_off, long long npix,
                       const unsigned long long *keys, long long key_cap, int cap, float4 *rgba,
                       int *counts, unsigned long long *stats, int nsm, int want_warps,
                       unsigned *ticket, cudaStream_t st);

// Shell adjoint, the cube's three passes with the shell's geometry and field
// (values by bwd_shell_values, scans by bwd_ray_scans) over lists built by
// shell_pairs in mode 2.
cudaError_t bwd_shell_adjoint(const int4 *geo, int N, const Shell &S, const Field &Fd,
                              const Cam &C, const Integ &I, const float4 *dL, const int2 *lm,
                              const float2 *rec_ta, const float4 *rec_g, long long nseg,
                              float *g_nodal, float *g_tf, int nsm, cudaStream_t st);

}  // namespace ocr
