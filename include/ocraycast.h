/* ocraycast: forest-of-octrees raycasting on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the CUDA library built from paper_1809_01334_gb300/csrc.  The
 * operations follow C. Burstedde, "Distributed-Memory Forest-of-Octrees
 * Raycasting" (2018):
 *
 *   prune   - drop the leaves whose camera-space bounding box covers no pixel
 *             centre (Sec. 3.1, Sec. 2.2);
 *   segment - intersect each remaining leaf with every ray of its pixel
 *             rectangle and integrate A' = -kappa A, B' = q - kappa B along
 *             the piece (Sec. 2.3, Eqs. 2.29 and 2.31, Algorithm 1);
 *   merge   - aggregate the segments of each ray up the octree with the
 *             segment group action (Eq. 2.14, Sec. 3.3) into its pixel,
 *             I_v = A I_b + B (Sec. 2.4), without a global depth sort;
 *   adjoint - the gradient of a loss on the image with respect to the nodal
 *             data and the transfer function (ocr_render_backward).
 *
 * Conventions
 *  - Every entry point returns OCR_OK (0) or a negative OCR_ERR_* code and
 *    never aborts.  ocr_strerror() names the code.
 *  - "d_" pointers are device pointers owned by the caller; "h_" pointers
 *    are host pointers read during the call only.  The library owns only its
 *    internal copies of the forest topology and a scratch arena, both freed
 *    by ocr_destroy().
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; ocr_render returns without waiting
 *    for the device unless counters or phase times are requested.
 *  - Two geometries: one unit-cube tree with the identity map
 *    (OCR_GEOM_CUBE) and the six-tree cubed-sphere shell with the equiangular
 *    map (OCR_GEOM_SHELL, the paper's forest of octrees with a curved tree
 *    map, Sec. 2.1).
 */
#ifndef OCRAYCAST_H
#define OCRAYCAST_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCR_OK 0
#define OCR_ERR_INVALID (-1)     /* bad argument, forest not complete or not Morton-sorted */
#define OCR_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define OCR_ERR_OOM (-3)         /* device or host allocation failed */
#define OCR_ERR_UNSUPPORTED (-4) /* geometry or option not implemented */
#define OCR_ERR_DEVICE (-5)      /* a kernel's own bounds check fired */
#define OCR_ERR_STATE (-6)       /* call order violated (no data / no camera set) */

#define OCR_GEOM_CUBE 0
#define OCR_GEOM_SHELL 1

#define OCR_RK4 0     /* nsteps equal classical RK4 steps per segment */
#define OCR_DOPRI5 1  /* Dormand-Prince 5(4) inside the bisection of Algorithm 1 */
#define OCR_GAUSS2 2  /* implicit 2-stage Gauss closed form (Eqs. 2.32-2.33), Algorithm 1 */
#define OCR_SIMPSON 3 /* Simpson quadrature of the closed form (Eq. 2.34), Algorithm 1 */
#define OCR_EQUILIBRIUM 4 /* intensity interface of Eq. 2.18, Algorithm 1 (see ocr_integrator) */

typedef struct ocr_forest ocr_forest;

/* Linear forest of octrees (Sec. 2.1, Sec. 3).  anchor[3*k + a] is leaf k's
 * lower corner along axis a of its tree's reference cube in integer units of
 * 2^-max_level; level[k] its level (edge length 2^-level).  max_level <= 20.
 *
 * OCR_GEOM_CUBE: one tree, the identity map onto the unit cube; leaves in
 * Morton order of their anchors, tiling the cube.  h_tree, frames, r0, r1 are
 * ignored.
 *
 * OCR_GEOM_SHELL: six trees; leaves sorted by (h_tree[k], Morton key), each
 * tree's leaves tiling its reference cube.  Tree t maps reference
 * (xi, eta, zeta) to r(zeta) normalize(n + tan(pi/4 (2 xi - 1)) e1 +
 * tan(pi/4 (2 eta - 1)) e2) with (n, e1, e2) = frames[t] (orthonormal rows),
 * r(zeta) = r0 + (r1 - r0) zeta, 0 < r0 < r1: the equiangular cubed sphere,
 * whose six normals n must be the +-x, +-y, +-z axes, one per tree. */
typedef struct {
  int geometry;          /* OCR_GEOM_CUBE or OCR_GEOM_SHELL */
  int max_level;
  int64_t nleaves;
  const int32_t *h_anchor; /* [nleaves * 3] */
  const uint8_t *h_level;  /* [nleaves] */
  const int32_t *h_tree;   /* [nleaves] tree 0..5 (shell) */
  double frames[6][3][3];  /* shell: rows n, e1, e2 of each tree */
  double r0, r1;           /* shell radii */
} ocr_forest_desc;

/* Pinhole camera of Sec. 2.2, Eq. 2.5: ray (i, j) is o + alpha r with
 * r = v + ell ((i - (w-1)/2) t + (j - (h-1)/2) u), alpha in [1, far/near]
 * (near = |v|, the projection plane).  ortho != 0: the origin moves to
 * o + ell ((i - (w-1)/2) t + (j - (h-1)/2) u), the direction is v/near and
 * alpha in [0, far].  Values are read as float32. */
typedef struct {
  double o[3], v[3], t[3], u[3];
  double ell, near_, far_;
  int w, h, ortho;
} ocr_camera;

/* Per-segment integrator.  RK4: nsteps equal steps from the far end, each
 * combined by Eq. 2.14.  DOPRI5, GAUSS2, SIMPSON: a step over [x1, x2] is
 * replaced by its two halves, combined near (+) far, while
 * dx * kappa(xi) > c_rk at a node of the step (or, for DOPRI5, the embedded
 * error estimate exceeds tol), up to max_depth halvings (Algorithm 1).  The
 * Gauss nodes are x1 + (1/2 -+ sqrt(3)/6) dx, x1 the far end.  EQUILIBRIUM
 * (the interface of Eq. 2.18, Sec. 2.5): the transfer function's colour
 * channels are read as the intensity I the application wants to see, not as
 * an emission density; a step's A = exp(-dx (kappa_far + 4 kappa_mid +
 * kappa_near) / 6) and B = I_mid (1 - A), split by the c_rk test of
 * Algorithm 1.  bg is the background intensity I_b per channel.
 *
 * surface != 0 (Sec. 2.8, both geometries): the isosurface s = s_iso of the
 * field is rendered as a surface of transparency a_s (in [0, 1]) and
 * intensity i_s.  Where the field along a segment changes sign against s_iso
 * between two of 9 equally spaced samples (far end to near end), the crossing
 * is located by bisection, the segment is cut there and the surface segment
 * A = a_s^(1 / cos phi), B = i_s (1 - A) (Eqs. 2.18 and 2.35; phi the angle
 * between the ray and the field gradient; on the shell the gradient goes
 * through the inverse map) goes between the two pieces.  The adjoint does not
 * support it (OCR_ERR_UNSUPPORTED). */
typedef struct {
  int method;
  int nsteps;
  float tol, c_rk;
  int max_depth;
  float bg[3];
  int surface;
  float s_iso, a_s, i_s[3];
} ocr_integrator;

/* Optional extras of ocr_render.  Device buffers are written when non-NULL:
 *   d_counts  [w*h]      int32   segments on each ray (row-major, j*w + i)
 *   d_visible [nleaves]  uint8   1 if the leaf survived pruning
 *   d_rects   [nleaves*4] int32  pixel rectangle {i0, i1, j0, j1} (inclusive;
 *                                {0,-1,0,-1} when pruned)
 * The counters are filled when fill_counters != 0, and the phase times
 * (device time between CUDA events recorded on `stream`) when time_phases != 0;
 * either blocks the host once more, at the end of the call. */
typedef struct {
  int32_t *d_counts;
  uint8_t *d_visible;
  int32_t *d_rects;
  int fill_counters;
  int time_phases;
  int64_t visible_leaves; /* (camera, leaf) pairs that survived pruning */
  int64_t segments;       /* ray segments integrated (sum of d_counts) */
  int64_t rk_steps;       /* Runge-Kutta steps taken over all segments */
  int64_t leaf_tests;     /* (cell, ray) slab tests performed: 8 per subtree node visit
                             plus the coarsening passes' (leaf, ray) tests */
  int64_t slots;          /* (node, ray) aggregates formed while merging */
  int64_t subtree_segments; /* segments integrated by the subtree pass */
  int64_t subtree_rk_steps; /* RK steps taken by the subtree pass */
  int64_t subtree_node_visits; /* (internal node, ray) visits of the subtree pass, each
                                  testing the node's 8 children */
  int64_t launches;       /* kernels launched by this call */
  float ms_prune;         /* cube: pruning, rectangle unions, slot layout, host readback;
                             shell: the monomial form, pruning, the per-ray lists */
  float ms_merge;         /* cube: subtree pass + coarsening passes + pixel pass;
                             shell: sorting the lists + the per-ray kernel */
  float ms_subtree;       /* cube: the subtree pass alone; shell: the per-ray kernel alone */
} ocr_stats;

/* Copy the forest topology to the device and derive its internal octree
 * nodes (the coarsening hierarchy of Sec. 3.3).  Returns OCR_ERR_INVALID if
 * the leaves are not Morton-sorted or do not tile the cube. */
int ocr_build_forest(const ocr_forest_desc *desc, void *stream, ocr_forest **out);

/* Attach the field and the transfer function (not copied, not owned):
 * d_nodal float32, cube: [nleaves*8], corner c = bx + 2 by + 4 bz of each
 * leaf (trilinear data); shell: [nleaves*27], node c = a + 3 b + 9 c' at local
 * coordinates (a, b, c')/2 (degree-2 Lagrange data); d_tf [8*4] float32, (kappa, q_r, q_g, q_b) at 8 knots
 * spaced uniformly over [s_min, s_max], piecewise linear, constant outside. */
int ocr_forest_set_data(ocr_forest *F, const float *d_nodal, const float *d_tf, float s_min,
                        float s_max, void *stream);

int ocr_set_integrator(ocr_forest *F, const ocr_integrator *integ);

/* Set the cameras (host structs, copied), 1 <= ncams <= 4096.  Plans every
 * camera once: its pruning and slot layout run on the device, on a stream the
 * forest owns (nothing is ordered on the legacy default stream; the host
 * blocks until the sizes are read back), to size its scratch, which is
 * allocated here.  Must not overlap a render of the same forest.  Rendering
 * then never waits for the host, so ocr_render without counters can be
 * captured in a CUDA graph.  Several cameras are rendered by one ocr_render
 * call (batching: the paper's multiple image instances, Sec. 3).  Shell
 * forests also size each camera's segment lists here; a ray with more than
 * 4096 segments returns OCR_ERR_UNSUPPORTED. */
int ocr_set_camera(ocr_forest *F, const ocr_camera *cams, int ncams);

/* Render the images of all cameras: d_rgba float32, the cameras' images
 * concatenated in order, each [h*w*4] row-major, (I_r, I_g, I_b, 1 - A) per
 * pixel.  With several cameras the work is spread over internal streams that
 * fork from and join back into `stream`.  stats may be NULL; its d_counts is
 * indexed like the concatenated image, d_visible is the union over cameras,
 * d_rects belongs to the first camera, time_phases applies to single-camera
 * renders only.
 * Shell forests: a ray meets a leaf in up to two intervals and the Morton
 * order is not the order along a ray, so each ray's segments are listed over
 * the leaves' pixel rectangles, ordered by entry depth (ties by tree and
 * Morton key), integrated, and merged nearest first with Eq. 2.14; overlapping
 * neighbours are cut (Eq. 2.20) and averaged (Eq. 2.21).  A ray with more
 * segments than ocr_set_camera found on any ray is left at the background
 * and counted as a device error (OCR_ERR_DEVICE when counters are filled). */
int ocr_render(ocr_forest *F, float *d_rgba, void *stream, ocr_stats *stats);

/* Render one camera of the last ocr_set_camera alone: camera `view`
 * (0 <= view < ncams) into d_rgba [h*w*4] (its own image only), on `stream`,
 * with the same pipeline as a single-camera ocr_render; stats as in
 * ocr_render, for this camera.  Lets a caller render the views of a planned
 * batch one at a time (the paper's image instances, Sec. 3, taken singly)
 * without planning again.  OCR_ERR_INVALID for a view out of range. */
int ocr_render_view(ocr_forest *F, int view, float *d_rgba, void *stream, ocr_stats *stats);

/* Pruning for callers that cannot allocate device memory at the time they
 * need it: an application that serves all device memory from a pool it
 * reserved up front, a real-time loop that must not take the device-wide
 * synchronisation an allocation implies, a plug-in living inside another
 * program's memory budget.  The paper has no counterpart.
 *
 * Cube forests only (OCR_GEOM_CUBE leaf records).  Inputs (device,
 * caller-owned): d_leaf_geo [nleaves * 4] int32, per leaf {x, y, z, level}
 * with anchors in units of 2^-max_level, Morton order; 16-byte aligned.  A
 * record whose level is negative or above max_level (a shell record, whose
 * fourth word carries the tree in its upper bits, is one) returns
 * OCR_ERR_INVALID after the kernel has run; the outputs are then undefined.  cam: host struct, read as float32 exactly like
 * ocr_set_camera.  Outputs (device, caller-owned): d_rects [nleaves * 4]
 * int32, the same rectangles ocr_render reports in ocr_stats.d_rects (may be
 * NULL; 16-byte aligned); d_visible_idx [nleaves] int32, the indices of the
 * visible leaves in increasing order (entries past the count are left
 * untouched).  *h_nvisible (host) receives the number of visible leaves.
 *
 * It calls no allocation routine.  Its only scratch is a fixed array of
 * OCR_NOALLOC_MAX_LEAVES / 1024 + 2 eight-byte words (512 KiB) compiled into
 * the library, which every device that loads the library keeps until the
 * process exits.  nleaves above OCR_NOALLOC_MAX_LEAVES returns
 * OCR_ERR_INVALID.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current), so make the first
 * call before any stream capture; the address is kept for the life of the
 * process, so do not call this on a device after cudaDeviceReset.  All calls share the one array and reset
 * it at their start: calls that overlap on the GPU (different streams,
 * different host threads on one device) race and must be serialised by the
 * caller.  Blocks the host until the result is ready. */
#define OCR_NOALLOC_MAX_LEAVES (1 << 26)
int ocr_prune_noalloc(const int32_t *d_leaf_geo, int64_t nleaves, int max_level,
                      const ocr_camera *cam, int32_t *d_rects, int32_t *d_visible_idx,
                      int64_t *h_nvisible, void *stream);

/* Render from host memory: the pipeline of ocr_render (pruning, Sec. 3.1;
 * segments, Sec. 2.1-2.3; merging with Eq. 2.14, Sec. 2.4 and 3.3) with the
 * inputs and the image in host memory.  Copy the field h_nodal (layout as in
 * ocr_forest_set_data) and the knots h_tf [8*4] to device memory that the
 * library owns, render every camera of the last ocr_set_camera into its own
 * device image, copy that image to h_rgba (float32, sum of w*h*4, layout as
 * in ocr_render) and return once it is there.  All work is ordered on `stream` after the caller's
 * earlier work; the copy in overlaps the data-independent pruning and layout
 * (cube forests).  Pinned host memory gives full copy speed; pageable memory
 * works.  Afterwards the forest's data is the library's copy (a later
 * ocr_forest_set_data replaces it).  s_min, s_max, stats and the error codes
 * as in ocr_forest_set_data and ocr_render; OCR_ERR_OOM if the device copies
 * cannot be allocated.  Blocks the host. */
int ocr_render_host(ocr_forest *F, const float *h_nodal, const float *h_tf, float s_min,
                    float s_max, float *h_rgba, void *stream, ocr_stats *stats);

/* Gradient of a loss L(rgba) with respect to the nodal values and the
 * transfer-function knots (Sec. 2.3-2.4, Eqs. 2.14 and 2.29-2.31 in reverse
 * mode), for the forest, data, integrator and the first camera last set.
 * d_dL_drgba [h*w*4] float32 (device): dL/d(I_r, I_g, I_b, alpha) per pixel;
 * rays whose four entries are zero are skipped.  d_grad_nodal [nleaves*8]
 * (cube) or [nleaves*27] (shell) and d_grad_tf [8*4] float32 (device) are
 * overwritten with dL/d(nodal) and dL/d(knots).  Segments are recomputed, not
 * taken from a previous render.  Cube: each ray's segments are put in
 * front-to-back order by their mirrored Morton key; a ray with more than 4096
 * segments is skipped and recorded as a device error.  Shell: the render's
 * per-ray lists are rebuilt in the first camera's scratch (so a backward call
 * must not overlap a render of the same forest on another stream) and ordered
 * by entry depth; overlapping rounding slivers are combined as if they did
 * not overlap.  More than 2^32 - 2 segments in all: OCR_ERR_UNSUPPORTED.  The
 * library keeps 32 B of scratch per segment for the adjoint (grown on demand,
 * OCR_ERR_OOM if that fails).  Every integrator: RK4, and inside Algorithm 1
 * DOPRI5 (stage recurrences run backwards), the Gauss-2 closed form, Simpson's
 * rule and the Eq. 2.18 interface (their closed forms differentiated, Eqs.
 * 2.32-2.34); surfaces return OCR_ERR_UNSUPPORTED.  Stream-ordered: the call
 * enqueues its work on `stream` and returns without waiting, so that it can be
 * captured in a CUDA graph -- except the first call after an ocr_set_camera
 * of a cube forest, which finds the sizes of that camera's pair space and hit
 * lists (geometry only) and blocks the host for them (and may allocate).
 * Device-side errors (a list overflow, a too long ray) are recorded in the
 * forest and returned by the next ocr_sync. */
int ocr_render_backward(ocr_forest *F, const float *d_dL_drgba, float *d_grad_nodal,
                        float *d_grad_tf, void *stream);

/* Wait for the work enqueued on `stream` and report the device-side errors
 * that the stream-ordered calls (ocr_render_backward) recorded since the last
 * ocr_sync: OCR_ERR_DEVICE if there were any (the record is then cleared),
 * else OCR_OK.  Blocks the host.  Not a step of the paper's method. */
int ocr_sync(ocr_forest *F, void *stream);

/* The per-ray merge of the shell render, on one list the caller gives: n
 * segments in order of entry along the ray, d_val [n*4] float32 (A, B_r, B_g,
 * B_b) and d_iv [n*2] float32 (alpha_in, alpha_out), combined nearest first
 * with Eq. 2.14; where consecutive segments overlap, the pieces before, inside
 * and after each overlap are cut with Eq. 2.20 and the overlapped pieces
 * averaged with Eq. 2.21 (Sec. 2.5).  The result (A, B_r, B_g, B_b) goes to
 * d_out [4] float32.  Device pointers (d_val and d_out 16-byte, d_iv 8-byte
 * aligned), 1 <= n <= 2^20, else OCR_ERR_INVALID; stream-ordered, no forest
 * needed.  It runs the device function the shell render uses, so that the
 * overlap handling (rounding slivers only, in a valid forest) can be checked
 * on lists with real overlaps. */
int ocr_fold_segments(const float *d_val, const float *d_iv, int n, float *d_out,
                      void *stream);

/* Tuning of the render's decomposition (the batching autotuner's knobs):
 *   tile_depth  cube forests: how many octree levels (1..4) the subtree pass
 *               walks per (tile node, ray) before the aggregates go to HBM.
 *               Deeper tiles mean fewer levels above and longer walks.
 *   streams     internal streams (1..8) over which the cameras of a
 *               multi-camera render are spread.
 *   shell_warps shell forests: warps per CTA of the per-ray kernel (1..8;
 *               0 = as many as fit in 96 KB of shared memory).
 *   merge       cube forests: the levels above the tile level are merged by
 *               one pass per level over (node, ray) aggregates (0), or (1) by
 *               a pass that forms the segments of the leaves at or above the
 *               tile level, one thread per (leaf, ray), and one pass in which
 *               each pixel's thread walks those levels top-down in its
 *               front-to-back octant order.  Equal up to rounding order (Eq.
 *               2.14 is associative).
 *   persistent  cube forests, several cameras, merge 0, no surface: render
 *               the whole batch in one persistent kernel (1) -- its CTAs draw
 *               work items (a camera's pruning block, union block, prefix-sum
 *               block, chunk of a subtree or coarsening pass, or pixel
 *               chunk) from a device queue ordered stage after stage, each
 *               waiting for its camera's previous stage -- or each camera's
 *               own kernel chain on the internal streams (0).
 *   chunks_per_item  persistent: 128-slot chunks of the subtree, coarsening
 *               and pixel passes handed out per ticket (1..64).
 *   ctas_per_sm persistent: resident CTAs per SM (1..8; 0 = as many as fit:
 *               8); 6 and 7 select variants compiled for that many, with more
 *               registers per thread (1..5 use the one for 6).
 *   ms          ocr_autotune: the measured device time of one ocr_render.
 * Defaults: tile_depth 4, streams 4, shell_warps 0, merge 1, persistent 1,
 * chunks_per_item 16, ctas_per_sm 0. */
typedef struct {
  int tile_depth;
  int streams;
  int shell_warps;
  int merge;
  int persistent;
  int chunks_per_item;
  int ctas_per_sm;
  float ms;
} ocr_tuning;

/* Apply a tuning.  Changing tile_depth of a cube forest re-plans the cameras
 * (blocking, like ocr_set_camera).  OCR_ERR_INVALID for values out of range. */
int ocr_set_tuning(ocr_forest *F, const ocr_tuning *t);
int ocr_get_tuning(const ocr_forest *F, ocr_tuning *t);

/* Autotuner: render the cameras, data and integrator last set under every
 * candidate tuning (cube: tile_depth 1..4 x merge {0, 1} x streams {1, 2, 4, 8},
 * and with several cameras the persistent kernel: tile_depth 1..4 x
 * chunks_per_item {8, 16, 32} x ctas_per_sm {8, 7, 6}; shell:
 * shell_warps {1, 2, 4, 8} x streams; streams only with several cameras),
 * one warm-up and `reps` timed renders each (CUDA events on an internal
 * stream, 1 <= reps <= 100), and keep the fastest, returned in *best.  The
 * candidates and their times go to tried[0 .. max_tried) (may be NULL when
 * max_tried is 0) and their number to *ntried (may be NULL).  Allocates a
 * scratch image for the duration of the call; blocks the host.  On error the
 * previous tuning is restored. */
int ocr_autotune(ocr_forest *F, int reps, ocr_tuning *best, ocr_tuning *tried, int max_tried,
                 int *ntried);

/* Device memory held by the library for this forest (topology + scratch). */
int64_t ocr_device_bytes(const ocr_forest *F);

void ocr_destroy(ocr_forest *F);
const char *ocr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
