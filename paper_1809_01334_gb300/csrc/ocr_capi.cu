// Host side of the C ABI declared in include/ocraycast.h.
//
// ocr_build_forest validates the linear octree (Morton order, complete
// tiling of the unit cube) and derives its internal nodes: the coarsening
// hierarchy along which ray segments are aggregated (Sec. 3.3).  ocr_render
// enqueues, on the caller's stream: pruning of the leaves (Sec. 3.1), the
// rectangle unions of the internal nodes, the prefix sum that lays out one
// aggregate per (node, ray), and one coarsening pass per octree level, the
// deepest first, ending with the pass that writes the pixels.
#include "../../include/ocraycast.h"
#include "ocr_common.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

using namespace ocr;

// Per-camera plan: the float32 camera, its pixel range in the concatenated
// image, the slot layout found when the camera was set (the render recomputes
// it on the device and launches with these sizes, so it never waits for the
// host), and the camera's own scratch.
struct CamPlan {
  Cam cam{};
  long long npix = 0, pix_off = 0;
  std::vector<long long> gslots;      // [L + 1] slot boundaries of the level groups
  int4 *d_rect = nullptr;             // [N + M + 1]
  long long *d_off = nullptr;         // [M + 1]
  long long *d_bsums = nullptr;       // [area_scan_blocks(M) + 1]
  long long *d_gslots = nullptr;      // [L + 1]
  int *d_chunk = nullptr;             // [total / kGroup + 2]
  float4 *d_entries = nullptr;        // [total slots]
  unsigned *d_ticket = nullptr;       // [2] work counters: the subtree pass's (cube), the
                                      // sort's and the per-ray kernel's (shell)
  // cube, top-down merge: the slots of the leaves at or above the tile level
  long long ctotal = 0;               // their slots (rectangle areas)
  long long *d_coff = nullptr;        // [nc + 1] exclusive prefix of their areas
  long long *d_cbsums = nullptr;      // [bwd_scan_blocks(nc) + 2] block sums of that scan
  int *d_cgroup = nullptr;            // [ctotal / kGroup + 2] their slot map
  float4 *d_cval = nullptr;           // [ctotal] their (leaf, ray) segments
  // shell forests: the (leaf, pixel) pair space and the per-ray segment lists
  long long npairs = 0, nhits = 0, bs_cap = 0;
  int cap = 0;                        // longest list found, rounded up to a power of two
  long long *d_leaf_off = nullptr;    // [N + 1]
  long long *d_sbsums = nullptr;      // [bs_cap]
  int *d_pchunk = nullptr;            // [npairs / kPairChunk + 2]
  int *d_rcount = nullptr, *d_rcursor = nullptr;  // [npix]
  long long *d_ray_off = nullptr;     // [npix + 1]
  unsigned long long *d_keys = nullptr;  // [nhits]
  // cube adjoint: sizes of its pair space and hit lists for this camera
  // (geometry only: found by the first backward call after ocr_set_camera)
  bool bwd_ready = false;
  long long bwd_npairs = 0, bwd_nh = 0;  // (leaf, pixel) pairs; hits of every ray
  int bwd_cap = 0;                      // longest list, rounded up to a power of two
};

constexpr int kMaxStreams = 8;      // cameras of a batch are spread over up to this many
constexpr int kMaxCameras = 4096;

struct ocr_forest {
  int geometry = OCR_GEOM_CUBE;
  Shell shell{};                      // shell: frames and tables (in d_shell_tabs)
  float *d_shell_tabs = nullptr;      // [54 + 2 (2^L + 1)]
  float *d_coef = nullptr;            // shell: [N * 27] the data in monomial form, per render
  float4 *d_planes = nullptr;         // shell: [N * 4] per leaf its plane normals and radii
  int N = 0, M = 0, L = 0;
  int root = 0;                       // unified id of the tree root
  std::vector<int> level_base;        // internal index of the first node of level l
  std::vector<int> level_count;       // number of internal nodes at level l
  std::vector<int> h_group_nodes;     // [L + 1] group boundaries, deepest level first, then M
  int4 *d_geo = nullptr;              // [N + M + 1]
  int bsums_blocks = 0;               // area_scan_blocks(M) + 1
  int *d_child = nullptr;             // [(M + 1) * 8]
  int2 *d_leaves = nullptr;           // [M] leaf range of each internal node
  int lt = 0;                         // tile level: deepest level with stored aggregates
  // cube: every leaf's level (host), and the leaves at or above the tile level
  std::vector<uint8_t> h_leaf_level;
  int nc = 0;                         // those leaves
  int *d_cids = nullptr;              // [nc] their ids, Morton order
  int *d_cindex = nullptr;            // [N] a leaf's place among them, -1 for the others
  int *d_group_nodes = nullptr;       // [L + 1]
  // data
  const float *d_nodal = nullptr;
  const float *d_tf = nullptr;
  float s_min = 0.f, s_max = 1.f;
  bool has_data = false, has_cam = false, has_integ = false;
  Integ integ{};
  std::vector<CamPlan> plans;         // one per camera of the last ocr_set_camera
  long long total_pix = 0;
  cudaStream_t sub[kMaxStreams] = {};
  cudaStream_t plan_st = nullptr;     // ocr_set_camera's planning (created on first use)
  cudaEvent_t fork = nullptr, join[kMaxStreams] = {};
  // tuning (ocr_set_tuning / ocr_autotune)
  int tile_depth = kDefaultTileDepth; // cube: octree levels the subtree pass walks
  int nstreams = 4;                   // internal streams of multi-camera renders
  int shell_warps = 0;                // shell: warps per CTA of the per-ray kernel (0: most)
  int merge = 1;                      // cube: levels above the tile level by the top-down pass
                                      // (0) or by one top-down pass per pixel (1)
  int persistent = 1;                 // cube, several cameras: one persistent kernel (1) or
                                      // per-camera kernel chains over the streams (0)
  int chunks_per_item = 16;           // persistent: chunks of the chunk passes per ticket
  int ctas_per_sm = 0;                // persistent: CTAs per SM (0: as many as fit)
  // persistent batch: the work queue (segments), per-camera device records and
  // the control words; rebuilt when the cameras or the decomposition change
  BatchSeg *d_bseg = nullptr;
  BatchCam *d_bcam = nullptr;
  unsigned *d_bctl = nullptr;
  int nbseg = 0, nbcam = 0;
  long long nbtickets = 0;
  bool batch_ready = false;
  long long *h_group_slots = nullptr; // pinned [L + 1 + kStats + 2] (shell [kStats + 3]); at
                                      // L + 1 + kStats: ocr_sync's word, then the cube
                                      // plan's listed-leaf slot total
  unsigned long long *d_stats = nullptr;  // [kStats]
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // start, layout, subtree, end
  // adjoint
  unsigned long long *d_mkey = nullptr;  // [N] Morton key of each leaf
  unsigned long long fx = 0;             // Morton bit positions of x
  long long *d_leaf_off = nullptr;       // [N + 1]
  long long *d_bsums = nullptr;          // scan block sums
  long long bsums_cap = 0;
  int *d_pchunk = nullptr;               // pair chunk -> leaf
  long long pchunk_cap = 0;
  int *d_rcount = nullptr, *d_rcursor = nullptr;  // [npix]
  long long *d_ray_off = nullptr;        // [npix + 1]
  long long ray_cap = 0;
  unsigned long long *d_hkey = nullptr;  // [hits]
  long long hit_cap = 0;
  // shell adjoint: per segment, its index in the leaf-grouped list (beside the
  // key), the list itself, and the near transmittance / own transmittance / far
  // aggregate per list entry
  unsigned *d_skpos = nullptr;
  int2 *d_slm = nullptr;
  float2 *d_srta = nullptr;
  float4 *d_srg = nullptr;
  long long seg_cap = 0;
  unsigned long long *d_lmcount = nullptr;
  unsigned long long *d_err = nullptr;
  // ocr_render_host: device copies of the caller's host data and image, the
  // copy stream and the event that marks the data as arrived
  float *d_hnodal = nullptr, *d_hrgba = nullptr;
  float *d_htf = nullptr;  // inside d_hnodal, after the field (not an allocation of its own)
  long long hnodal_cap = 0, hrgba_cap = 0;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev = nullptr;
  cudaEvent_t data_ready = nullptr;  // set during ocr_render_host: kernels that read data wait
  int nsm = 0;
  int64_t bytes = 0;
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? OCR_ERR_OOM : OCR_ERR_CUDA; }

#define OCR_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

uint64_t morton(int x, int y, int z) {
  return spread3((uint32_t)x) | spread3((uint32_t)y) << 1 | spread3((uint32_t)z) << 2;
}

template <typename T>
int dev_alloc(T **p, size_t n, int64_t &bytes) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e);
  }
  bytes += (int64_t)(n * sizeof(T));
  return OCR_OK;
}

// free one plan's device scratch (its camera and sizes stay)
void free_plan_buffers(ocr_forest *F, CamPlan &P) {
  void *bufs[] = {P.d_rect, P.d_off, P.d_bsums, P.d_gslots, P.d_chunk, P.d_entries, P.d_leaf_off,
                  P.d_sbsums, P.d_pchunk, P.d_rcount, P.d_rcursor, P.d_ray_off,
                  P.d_keys, P.d_coff, P.d_cbsums, P.d_cgroup, P.d_cval, P.d_ticket};
  for (void *b : bufs) cudaFree(b);
  P.d_ticket = nullptr;
  P.d_coff = nullptr;
  P.d_cbsums = nullptr;
  P.d_cgroup = nullptr;
  P.d_cval = nullptr;
  P.d_rect = nullptr;
  P.d_off = nullptr;
  P.d_bsums = nullptr;
  P.d_gslots = nullptr;
  P.d_chunk = nullptr;
  P.d_entries = nullptr;
  P.d_leaf_off = nullptr;
  P.d_sbsums = nullptr;
  P.d_pchunk = nullptr;
  P.d_rcount = nullptr;
  P.d_rcursor = nullptr;
  P.d_ray_off = nullptr;
  P.d_keys = nullptr;
  (void)F;
}

void free_plans(ocr_forest *F) {
  for (CamPlan &P : F->plans) free_plan_buffers(F, P);
  F->plans.clear();
}

void free_all(ocr_forest *F) {
  cudaFree(F->d_shell_tabs);
  cudaFree(F->d_coef);
  cudaFree(F->d_planes);
  cudaFree(F->d_geo);
  cudaFree(F->d_child);
  cudaFree(F->d_leaves);
  cudaFree(F->d_group_nodes);
  free_plans(F);
  for (int q = 0; q < kMaxStreams; ++q) {
    if (F->sub[q]) cudaStreamDestroy(F->sub[q]);
    if (F->join[q]) cudaEventDestroy(F->join[q]);
  }
  if (F->fork) cudaEventDestroy(F->fork);
  if (F->plan_st) cudaStreamDestroy(F->plan_st);
  cudaFree(F->d_stats);
  cudaFree(F->d_mkey);
  cudaFree(F->d_leaf_off);
  cudaFree(F->d_bsums);
  cudaFree(F->d_pchunk);
  cudaFree(F->d_rcount);
  cudaFree(F->d_rcursor);
  cudaFree(F->d_ray_off);
  cudaFree(F->d_hkey);
  cudaFree(F->d_skpos);
  cudaFree(F->d_slm);
  cudaFree(F->d_srta);
  cudaFree(F->d_srg);
  cudaFree(F->d_lmcount);
  cudaFree(F->d_hnodal);  // d_htf points into it
  cudaFree(F->d_hrgba);
  if (F->copy_st) cudaStreamDestroy(F->copy_st);
  if (F->copy_ev) cudaEventDestroy(F->copy_ev);
  cudaFree(F->d_cids);
  cudaFree(F->d_cindex);
  cudaFree(F->d_err);
  cudaFree(F->d_bseg);
  cudaFree(F->d_bcam);
  cudaFree(F->d_bctl);
  if (F->h_group_slots) cudaFreeHost(F->h_group_slots);
  for (cudaEvent_t &e : F->ev)
    if (e) cudaEventDestroy(e);
}

bool valid_camera(const ocr_camera &c) {
  return c.w >= 1 && c.h >= 1 && (int64_t)c.w * c.h <= (1ll << 31) - 1 && c.near_ > 0.0 &&
         c.far_ > c.near_ && c.ell > 0.0;
}

}  // namespace

// float32 camera constants (both the render and ocr_prune_noalloc read these
// exact roundings)
void ocr::to_cam(const ocr_camera &c, Cam &k) {
  for (int a = 0; a < 3; ++a) {
    k.o[a] = (float)c.o[a];
    k.v[a] = (float)(c.ortho ? c.v[a] / c.near_ : c.v[a]);
    k.lt[a] = (float)(c.ell * c.t[a]);
    k.lu[a] = (float)(c.ell * c.u[a]);
    k.t[a] = (float)c.t[a];
    k.u[a] = (float)c.u[a];
    k.vn[a] = (float)(c.v[a] / c.near_);
  }
  k.n = (float)c.near_;
  k.f = (float)c.far_;
  k.ell = (float)c.ell;
  k.cw = 0.5f * (float)(c.w - 1);
  k.ch = 0.5f * (float)(c.h - 1);
  k.w = c.w;
  k.h = c.h;
  k.ortho = c.ortho ? 1 : 0;
  k.amin = c.ortho ? 0.f : 1.f;
  k.amax = (float)(c.ortho ? c.far_ : c.far_ / c.near_);
}

namespace {

// A signed unit axis vector: the index of its non-zero entry, or -1.
int axis_of(const double *v) {
  int ax = -1;
  for (int a = 0; a < 3; ++a) {
    if (v[a] == 0.0) continue;
    if ((v[a] != 1.0 && v[a] != -1.0) || ax >= 0) return -1;
    ax = a;
  }
  return ax;
}

// Shell forest: validate the six trees and their leaves, upload the leaf
// records {x, y, z, level | tree << 8} and the tables of plane tangents and
// sphere radii every kernel reads.
int build_shell(const ocr_forest_desc *desc, cudaStream_t st, ocr_forest **out) {
  const int L = desc->max_level;
  const int64_t N64 = desc->nleaves;
  if (L < 0 || L > 20 || N64 < 6 || N64 > (1ll << 30) || !desc->h_anchor || !desc->h_level ||
      !desc->h_tree)
    return OCR_ERR_INVALID;
  if (!(desc->r0 > 0.0) || !(desc->r1 > desc->r0) || !std::isfinite(desc->r1))
    return OCR_ERR_INVALID;
  int seen = 0;
  for (int t = 0; t < 6; ++t) {
    int ax[3];
    for (int r = 0; r < 3; ++r)
      if ((ax[r] = axis_of(desc->frames[t][r])) < 0) return OCR_ERR_INVALID;
    if (ax[0] == ax[1] || ax[0] == ax[2] || ax[1] == ax[2]) return OCR_ERR_INVALID;
    const int id = 2 * ax[0] + (desc->frames[t][0][ax[0]] < 0.0);
    if (seen & (1 << id)) return OCR_ERR_INVALID;  // two trees around one axis direction
    seen |= 1 << id;
  }
  const int N = (int)N64;
  const uint64_t full = 1ull << (3 * L);
  uint64_t expect = 0;
  int tree = 0;
  std::vector<int4> geo((size_t)N + 1);
  for (int k = 0; k < N; ++k) {
    const int t = desc->h_tree[k], lv = desc->h_level[k];
    if (t < 0 || t > 5 || lv > L) return OCR_ERR_INVALID;
    if (t != tree) {  // the previous tree must be complete, trees in order 0..5
      if (t != tree + 1 || expect != full) return OCR_ERR_INVALID;
      tree = t;
      expect = 0;
    }
    const int32_t *a = desc->h_anchor + 3 * (size_t)k;
    const int32_t mask = (1 << (L - lv)) - 1;
    for (int d = 0; d < 3; ++d)
      if (a[d] < 0 || a[d] >= (1 << L) || (a[d] & mask)) return OCR_ERR_INVALID;
    if (morton(a[0], a[1], a[2]) != expect) return OCR_ERR_INVALID;
    expect += 1ull << (3 * (L - lv));
    geo[k] = make_int4(a[0], a[1], a[2], lv | t << 8);
  }
  if (tree != 5 || expect != full) return OCR_ERR_INVALID;
  geo[N] = make_int4(0, 0, 0, -1);

  const int nt = (1 << L) + 1;
  std::vector<float> tabs(54 + 2 * (size_t)nt);
  for (int t = 0; t < 6; ++t)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) tabs[9 * t + 3 * r + c] = (float)desc->frames[t][r][c];
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < nt; ++k) {
    // tan(pi/4 (2 k 2^-L - 1)): odd about the tree centre, exactly -+1 at its edges
    const double x = std::ldexp(2.0 * k, -L) - 1.0, ax = std::fabs(x);
    const double v = ax == 1.0 ? 1.0 : std::tan(0.25 * pi * ax);
    tabs[54 + k] = (float)(x < 0.0 ? -v : v);
    tabs[54 + nt + k] = (float)(desc->r0 + (desc->r1 - desc->r0) * std::ldexp((double)k, -L));
  }

  ocr_forest *F = new (std::nothrow) ocr_forest();
  if (!F) return OCR_ERR_OOM;
  F->geometry = OCR_GEOM_SHELL;
  F->N = N;
  F->L = L;
  F->M = 0;
  int rc;
  if ((rc = dev_alloc(&F->d_geo, geo.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_shell_tabs, tabs.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_coef, (size_t)F->N * 27, F->bytes)) ||
      (rc = dev_alloc(&F->d_planes, (size_t)F->N * 4, F->bytes)) ||
      (rc = dev_alloc(&F->d_stats, kStats, F->bytes)) ||
      (rc = dev_alloc(&F->d_err, 1, F->bytes))) {
    free_all(F);
    delete F;
    return rc;
  }
  if (cudaMallocHost((void **)&F->h_group_slots, sizeof(long long) * (kStats + 3)) !=
      cudaSuccess) {
    F->h_group_slots = nullptr;
    free_all(F);
    delete F;
    return OCR_ERR_OOM;
  }
  if (cudaMemsetAsync(F->d_err, 0, sizeof(unsigned long long), st) != cudaSuccess) {
    free_all(F);
    delete F;
    return OCR_ERR_CUDA;
  }
  F->shell.frames = F->d_shell_tabs;
  F->shell.tan_tab = F->d_shell_tabs + 54;
  F->shell.rad_tab = F->d_shell_tabs + 54 + nt;
  F->shell.planes = F->d_planes;
  F->shell.L = L;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&F->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_geo, geo.data(), geo.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_shell_tabs, tabs.data(), tabs.size() * sizeof(float),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = shell_planes(F->d_geo, F->N, F->shell, F->d_planes, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_all(F);
    delete F;
    return cuda_fail(e);
  }
  *out = F;
  return OCR_OK;
}

int plan_cameras(ocr_forest *F);
int plan_batch(ocr_forest *F);

// The leaves at or above the tile level of a cube forest (their ids in Morton
// order, and every leaf's place among them), whose segments the top-down
// merge takes from a pass of their own; rebuilt when the tile level changes.
// Blocks the host on st until the copies are done.
int build_listed_leaves(ocr_forest *F, cudaStream_t st) {
  if (F->d_cids) F->bytes -= (int64_t)sizeof(int) * ((F->nc > 0 ? F->nc : 1) + (int64_t)F->N);
  cudaFree(F->d_cids);
  cudaFree(F->d_cindex);
  F->d_cids = nullptr;
  F->d_cindex = nullptr;
  std::vector<int> ids, index((size_t)F->N, -1);
  for (int k = 0; k < F->N; ++k)
    if ((int)F->h_leaf_level[(size_t)k] <= F->lt) {
      index[(size_t)k] = (int)ids.size();
      ids.push_back(k);
    }
  F->nc = (int)ids.size();
  int rc;
  if ((rc = dev_alloc(&F->d_cids, ids.empty() ? 1 : ids.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_cindex, (size_t)F->N, F->bytes)))
    return rc;
  if (!ids.empty())
    OCR_CUDA(cudaMemcpyAsync(F->d_cids, ids.data(), sizeof(int) * ids.size(),
                             cudaMemcpyHostToDevice, st));
  OCR_CUDA(cudaMemcpyAsync(F->d_cindex, index.data(), sizeof(int) * index.size(),
                           cudaMemcpyHostToDevice, st));
  OCR_CUDA(cudaStreamSynchronize(st));  // the host vectors die on return
  return OCR_OK;
}

// Plan one camera of a shell forest: its pruning and pair space, the segment
// count of every ray, the size of the lists and the longest one.  Runs on the
// forest's planning stream and blocks the host until the sizes are read back.
int plan_shell(ocr_forest *F, CamPlan &P) {
  const long long npix = P.npix;
  cudaStream_t ps = F->plan_st;
  const Topo T{F->d_geo, nullptr, nullptr, F->N, 0, F->L, 0};
  int rc;
  P.bs_cap = std::max(bwd_scan_blocks(F->N), bwd_scan_blocks(npix)) + 2;
  if ((rc = dev_alloc(&P.d_rect, (size_t)F->N + 1, F->bytes)) ||
      (rc = dev_alloc(&P.d_leaf_off, (size_t)F->N + 1, F->bytes)) ||
      (rc = dev_alloc(&P.d_sbsums, (size_t)P.bs_cap, F->bytes)) ||
      (rc = dev_alloc(&P.d_rcount, (size_t)npix, F->bytes)) ||
      (rc = dev_alloc(&P.d_rcursor, (size_t)npix, F->bytes)) ||
      (rc = dev_alloc(&P.d_ray_off, (size_t)npix + 1, F->bytes)) ||
      (rc = dev_alloc(&P.d_ticket, 2, F->bytes)))
    return rc;
  long long *h = F->h_group_slots;
  OCR_CUDA(cudaMemsetAsync(F->d_stats, 0, kStats * sizeof(unsigned long long), ps));
  OCR_CUDA(shell_cull(F->d_geo, F->N, F->shell, P.cam, P.d_rect, nullptr, F->d_stats, ps));
  OCR_CUDA(bwd_leaf_scan(T, P.d_rect, P.d_sbsums, P.bs_cap, P.d_leaf_off, ps));
  OCR_CUDA(cudaMemcpyAsync(h, P.d_leaf_off + F->N, sizeof(long long), cudaMemcpyDeviceToHost, ps));
  OCR_CUDA(cudaStreamSynchronize(ps));
  P.npairs = h[0];
  if ((rc = dev_alloc(&P.d_pchunk, (size_t)(P.npairs / kPairChunk + 2), F->bytes))) return rc;
  OCR_CUDA(bwd_chunk_map(P.d_leaf_off, F->N, P.d_pchunk, ps));
  OCR_CUDA(cudaMemsetAsync(P.d_rcount, 0, sizeof(int) * (size_t)npix, ps));
  OCR_CUDA(shell_pairs(0, F->d_geo, F->N, F->shell, P.cam, P.d_rect, P.d_leaf_off,
                       P.d_pchunk, P.npairs, P.d_rcount, nullptr, nullptr, nullptr, 0,
                       F->d_stats, nullptr, ps));
  OCR_CUDA(bwd_count_scan(P.d_rcount, npix, P.d_sbsums, P.bs_cap, P.d_ray_off, ps));
  OCR_CUDA(cudaMemcpyAsync(h, P.d_ray_off + npix, sizeof(long long), cudaMemcpyDeviceToHost, ps));
  OCR_CUDA(cudaMemcpyAsync(h + 1, F->d_stats + kStatMaxHits, sizeof(long long),
                           cudaMemcpyDeviceToHost, ps));
  OCR_CUDA(cudaStreamSynchronize(ps));
  P.nhits = h[0];
  const long long longest = h[1];
  if (longest > kShellMaxCap) return OCR_ERR_UNSUPPORTED;
  P.cap = 32;
  while (P.cap < longest) P.cap <<= 1;
  return dev_alloc(&P.d_keys, (size_t)(P.nhits > 0 ? P.nhits : 1), F->bytes);
}

// Enqueue the segment lists of one camera of a shell forest on st: pruning,
// pair space, then one pass that intersects every pair and writes each
// segment into its ray's list, laid out by the camera's plan (every ray's
// segment count; for the adjoint also the leaf-grouped list, into F's adjoint
// buffers).  No host synchronisation.
int enqueue_shell_lists(ocr_forest *F, CamPlan &P, unsigned char *visible, cudaStream_t st,
                        bool adjoint = false) {
  const long long npix = P.npix;
  const Topo T{F->d_geo, nullptr, nullptr, F->N, 0, F->L, 0};
  OCR_CUDA(shell_cull(F->d_geo, F->N, F->shell, P.cam, P.d_rect, visible, F->d_stats, st));
  OCR_CUDA(bwd_leaf_scan(T, P.d_rect, P.d_sbsums, P.bs_cap, P.d_leaf_off, st));
  OCR_CUDA(bwd_chunk_map(P.d_leaf_off, F->N, P.d_pchunk, st));
  OCR_CUDA(cudaMemsetAsync(P.d_rcursor, 0, sizeof(int) * (size_t)npix, st));
  if (adjoint) {
    OCR_CUDA(cudaMemsetAsync(F->d_lmcount, 0, sizeof(unsigned long long), st));
    OCR_CUDA(shell_pairs(2, F->d_geo, F->N, F->shell, P.cam, P.d_rect, P.d_leaf_off,
                         P.d_pchunk, P.npairs, nullptr, P.d_ray_off, P.d_rcursor, P.d_keys,
                         P.nhits, F->d_stats, nullptr, st, F->d_skpos, F->d_slm,
                         F->d_lmcount));
  } else {
    OCR_CUDA(shell_pairs(1, F->d_geo, F->N, F->shell, P.cam, P.d_rect, P.d_leaf_off,
                         P.d_pchunk, P.npairs, nullptr, P.d_ray_off, P.d_rcursor, P.d_keys,
                         P.nhits, F->d_stats, nullptr, st));
  }
  return OCR_OK;
}

// Enqueue one camera's render of a shell forest on st: the segment lists, then
// one warp per ray.  No host synchronisation.
int enqueue_shell(ocr_forest *F, CamPlan &P, float4 *rgba, int *counts, unsigned char *visible,
                  cudaStream_t st, bool timed, int64_t &launches) {
  const long long npix = P.npix;
  const Field Fd{F->d_coef, reinterpret_cast<const float4 *>(F->d_tf), F->s_min,
                 7.f / (F->s_max - F->s_min)};
  const int rc = enqueue_shell_lists(F, P, visible, st);
  if (rc) return rc;
  if (timed) OCR_CUDA(cudaEventRecord(F->ev[1], st));
  OCR_CUDA(cudaMemsetAsync(P.d_ticket, 0, 2 * sizeof(unsigned), st));
  OCR_CUDA(shell_sort_lists(P.d_ray_off, npix, P.d_keys, P.nhits, P.cap, F->nsm, P.d_ticket, st));
  if (timed) OCR_CUDA(cudaEventRecord(F->ev[2], st));
  OCR_CUDA(shell_rays(F->d_geo, F->N, F->shell, Fd, P.cam, F->integ, P.d_ray_off, npix, P.d_keys,
                      P.nhits, P.cap, rgba, counts, F->d_stats, F->nsm, F->shell_warps,
                      P.d_ticket + 1, st));
  if (timed) OCR_CUDA(cudaEventRecord(F->ev[3], st));
  // cull, 2 scans of 3 kernels (1 when empty), chunk map, 2 pair passes, sort, rays
  launches += 1 + (bwd_scan_blocks(F->N) > 0 ? 3 : 0) + 1 + (P.npairs > 0 ? 2 : 0) +
              (bwd_scan_blocks(npix) > 0 ? 3 : 0) + 2;
  return OCR_OK;
}

}  // namespace

extern "C" {

const char *ocr_strerror(int code) {
  switch (code) {
    case OCR_OK: return "ok";
    case OCR_ERR_INVALID: return "invalid argument or forest";
    case OCR_ERR_CUDA: return "CUDA runtime error";
    case OCR_ERR_OOM: return "out of memory";
    case OCR_ERR_UNSUPPORTED: return "not supported";
    case OCR_ERR_DEVICE: return "device-side check failed";
    case OCR_ERR_STATE: return "data, integrator or camera not set";
    default: return "unknown error";
  }
}

int ocr_build_forest(const ocr_forest_desc *desc, void *stream, ocr_forest **out) {
  if (!desc || !out) return OCR_ERR_INVALID;
  *out = nullptr;
  if (desc->geometry == OCR_GEOM_SHELL) return build_shell(desc, (cudaStream_t)stream, out);
  if (desc->geometry != OCR_GEOM_CUBE) return OCR_ERR_UNSUPPORTED;
  const int L = desc->max_level;
  const int64_t N64 = desc->nleaves;
  if (L < 0 || L > 20 || N64 < 1 || N64 > (1ll << 30) || !desc->h_anchor || !desc->h_level)
    return OCR_ERR_INVALID;
  const int N = (int)N64;
  cudaStream_t st = (cudaStream_t)stream;

  // validate: aligned anchors, strictly increasing Morton keys, contiguous tiling
  std::vector<uint64_t> key(N);
  const uint64_t full = 1ull << (3 * L);
  uint64_t expect = 0;
  for (int k = 0; k < N; ++k) {
    const int lv = desc->h_level[k];
    if (lv > L) return OCR_ERR_INVALID;
    const int32_t *a = desc->h_anchor + 3 * (size_t)k;
    const int32_t mask = (1 << (L - lv)) - 1;
    for (int d = 0; d < 3; ++d)
      if (a[d] < 0 || a[d] >= (1 << L) || (a[d] & mask)) return OCR_ERR_INVALID;
    key[k] = morton(a[0], a[1], a[2]);
    if (key[k] != expect) return OCR_ERR_INVALID;  // not sorted, overlapping or gapped
    expect += 1ull << (3 * (L - lv));
  }
  if (expect != full) return OCR_ERR_INVALID;

  ocr_forest *F = new (std::nothrow) ocr_forest();
  if (!F) return OCR_ERR_OOM;
  F->N = N;
  F->L = L;

  // internal nodes, level by level from the deepest: parents of the nodes below
  std::vector<std::vector<uint64_t>> ikeys(L > 0 ? L : 1);
  std::vector<std::vector<uint64_t>> by_level_leaf(L + 1);
  std::vector<std::vector<int>> by_level_leaf_id(L + 1);
  for (int k = 0; k < N; ++k) {
    by_level_leaf[desc->h_level[k]].push_back(key[k]);
    by_level_leaf_id[desc->h_level[k]].push_back(k);
  }
  for (int l = L - 1; l >= 0; --l) {
    const uint64_t pmask = ~((1ull << (3 * (L - l))) - 1);
    std::vector<uint64_t> kids;
    kids.reserve(by_level_leaf[l + 1].size() + (l + 1 < L ? ikeys[l + 1].size() : 0));
    std::merge(by_level_leaf[l + 1].begin(), by_level_leaf[l + 1].end(),
               (l + 1 < L ? ikeys[l + 1].begin() : ikeys[l].end()),
               (l + 1 < L ? ikeys[l + 1].end() : ikeys[l].end()), std::back_inserter(kids));
    std::vector<uint64_t> &par = ikeys[l];
    for (uint64_t c : kids) {
      const uint64_t p = c & pmask;
      if (par.empty() || par.back() != p) par.push_back(p);
    }
  }
  int M = 0;
  F->level_base.assign(L > 0 ? L : 1, 0);
  F->level_count.assign(L > 0 ? L : 1, 0);
  for (int l = L - 1; l >= 0; --l) {
    F->level_base[l] = M;
    F->level_count[l] = (int)ikeys[l].size();
    M += F->level_count[l];
  }
  F->M = M;
  F->root = (L == 0 || M == 0) ? 0 : N + F->level_base[0];
  if (M == 0 && N != 1) {
    free_all(F);
    delete F;
    return OCR_ERR_INVALID;
  }

  std::vector<int4> geo((size_t)N + M + 1);
  std::vector<int> child((size_t)(M + 1) * 8, -1);
  for (int k = 0; k < N; ++k) {
    const int32_t *a = desc->h_anchor + 3 * (size_t)k;
    geo[k] = make_int4(a[0], a[1], a[2], desc->h_level[k]);
  }
  for (int l = L - 1; l >= 0; --l)
    for (int q = 0; q < F->level_count[l]; ++q) {
      const uint64_t kk = ikeys[l][q];
      geo[(size_t)N + F->level_base[l] + q] =
          make_int4((int)compact3(kk), (int)compact3(kk >> 1), (int)compact3(kk >> 2), l);
    }
  geo[(size_t)N + M] = make_int4(0, 0, 0, -1);
  // children: every node at level l + 1 is the octant-th child of its parent
  auto attach = [&](int l, uint64_t ckey, int cid) -> bool {
    const uint64_t pkey = ckey & ~((1ull << (3 * (L - l))) - 1);
    const int octant = (int)((ckey >> (3 * (L - l - 1))) & 7);
    const std::vector<uint64_t> &par = ikeys[l];
    auto it = std::lower_bound(par.begin(), par.end(), pkey);
    if (it == par.end() || *it != pkey) return false;
    const int pid = F->level_base[l] + (int)(it - par.begin());
    if (child[(size_t)pid * 8 + octant] != -1) return false;
    child[(size_t)pid * 8 + octant] = cid;
    return true;
  };
  bool ok = true;
  for (int l = L - 1; l >= 0 && ok; --l) {
    for (size_t q = 0; q < by_level_leaf[l + 1].size() && ok; ++q)
      ok = attach(l, by_level_leaf[l + 1][q], by_level_leaf_id[l + 1][q]);
    if (l + 1 < L)
      for (int q = 0; q < F->level_count[l + 1] && ok; ++q)
        ok = attach(l, ikeys[l + 1][q], N + F->level_base[l + 1] + q);
  }
  for (int p = 0; p < M && ok; ++p)
    for (int q = 0; q < 8; ++q)
      if (child[(size_t)p * 8 + q] < 0) ok = false;
  if (!ok) {
    free_all(F);
    delete F;
    return OCR_ERR_INVALID;
  }
  child[(size_t)M * 8] = F->root;  // super-root: one child, the tree root
  // leaves of each internal node: a contiguous range of the Morton-sorted leaves
  std::vector<int2> lrange((size_t)(M > 0 ? M : 1));
  for (int l = L - 1; l >= 0; --l)
    for (int q = 0; q < F->level_count[l]; ++q) {
      const uint64_t k0 = ikeys[l][q], k1 = k0 + (1ull << (3 * (L - l)));
      const int a = (int)(std::lower_bound(key.begin(), key.end(), k0) - key.begin());
      const int b = (int)(std::lower_bound(key.begin(), key.end(), k1) - key.begin());
      lrange[(size_t)F->level_base[l] + q] = make_int2(a, b);
    }
  F->lt = L > F->tile_depth ? L - F->tile_depth : 0;

  // group boundaries: internal levels from the deepest, then M
  for (int l = L - 1; l >= 0; --l) F->h_group_nodes.push_back(F->level_base[l]);
  F->h_group_nodes.push_back(M);

  int rc;
  if ((rc = dev_alloc(&F->d_geo, geo.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_child, child.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_leaves, lrange.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_group_nodes, F->h_group_nodes.size(), F->bytes)) ||
      (rc = dev_alloc(&F->d_stats, kStats, F->bytes)) ||
      (rc = dev_alloc(&F->d_mkey, (size_t)N, F->bytes)) ||
      (rc = dev_alloc(&F->d_leaf_off, (size_t)N + 1, F->bytes)) ||
      (rc = dev_alloc(&F->d_err, 1, F->bytes))) {
    free_all(F);
    delete F;
    return rc;
  }
  F->bsums_blocks = area_scan_blocks(M) + 1;
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&F->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      free_all(F);
      delete F;
      return cuda_fail(e);
    }
  }
  if (cudaMallocHost((void **)&F->h_group_slots,
                     sizeof(long long) * (F->h_group_nodes.size() + kStats + 2)) !=
      cudaSuccess) {
    F->h_group_slots = nullptr;
    free_all(F);
    delete F;
    return OCR_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(F->d_geo, geo.data(), geo.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_child, child.data(), child.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_leaves, lrange.data(), lrange.size() * sizeof(int2),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_mkey, key.data(), key.size() * sizeof(uint64_t),
                        cudaMemcpyHostToDevice, st);
  for (int l = 0; l < L; ++l) F->fx |= 1ull << (3 * l);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->d_group_nodes, F->h_group_nodes.data(),
                        F->h_group_nodes.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->d_err, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors die on return
  if (e != cudaSuccess) {
    free_all(F);
    delete F;
    return cuda_fail(e);
  }
  F->h_leaf_level.assign(desc->h_level, desc->h_level + N);
  if ((rc = build_listed_leaves(F, st))) {
    free_all(F);
    delete F;
    return rc;
  }
  *out = F;
  return OCR_OK;
}

int ocr_forest_set_data(ocr_forest *F, const float *d_nodal, const float *d_tf, float s_min,
                        float s_max, void *stream) {
  (void)stream;
  if (!F || !d_nodal || !d_tf || !(s_max > s_min) || !std::isfinite(s_min) ||
      !std::isfinite(s_max))
    return OCR_ERR_INVALID;
  if (((uintptr_t)d_nodal & 15) || ((uintptr_t)d_tf & 15)) return OCR_ERR_INVALID;
  F->d_nodal = d_nodal;
  F->d_tf = d_tf;
  F->s_min = s_min;
  F->s_max = s_max;
  F->has_data = true;
  return OCR_OK;
}

int ocr_set_integrator(ocr_forest *F, const ocr_integrator *I) {
  if (!F || !I) return OCR_ERR_INVALID;
  if (I->method == OCR_RK4) {
    if (I->nsteps < 1 || I->nsteps > 4096) return OCR_ERR_INVALID;
  } else if (I->method == OCR_DOPRI5) {
    if (!(I->tol > 0.f) || !(I->c_rk > 0.f) || I->max_depth < 0 || I->max_depth > 24)
      return OCR_ERR_INVALID;
  } else if (I->method == OCR_GAUSS2 || I->method == OCR_SIMPSON ||
             I->method == OCR_EQUILIBRIUM) {
    if (!(I->c_rk > 0.f) || I->max_depth < 0 || I->max_depth > 24) return OCR_ERR_INVALID;
  } else {
    return OCR_ERR_UNSUPPORTED;
  }
  if (I->surface) {
    if (!(I->a_s >= 0.f && I->a_s <= 1.f) || !std::isfinite(I->s_iso)) return OCR_ERR_INVALID;
  }
  F->integ.method = I->method;
  F->integ.nsteps = I->nsteps;
  F->integ.tol = I->tol;
  F->integ.c_rk = I->c_rk;
  F->integ.max_depth = I->max_depth;
  for (int c = 0; c < 3; ++c) F->integ.bg[c] = I->bg[c];
  F->integ.surface = I->surface ? 1 : 0;
  F->integ.s_iso = I->s_iso;
  F->integ.a_s = I->a_s;
  for (int c = 0; c < 3; ++c) F->integ.i_s[c] = I->i_s[c];
  F->has_integ = true;
  return OCR_OK;
}

int ocr_set_camera(ocr_forest *F, const ocr_camera *cams, int ncams) {
  if (!F || !cams || ncams < 1) return OCR_ERR_INVALID;
  if (ncams > kMaxCameras) return OCR_ERR_UNSUPPORTED;
  for (int k = 0; k < ncams; ++k)
    if (!valid_camera(cams[k])) return OCR_ERR_INVALID;
  free_plans(F);
  F->has_cam = false;
  F->plans.resize(ncams);
  long long pix = 0;
  for (int k = 0; k < ncams; ++k) {
    CamPlan &P = F->plans[k];
    to_cam(cams[k], P.cam);
    P.npix = (long long)cams[k].w * cams[k].h;
    P.pix_off = pix;
    pix += P.npix;
  }
  F->total_pix = pix;
  if (ncams > 1 && !F->fork) {
    OCR_CUDA(cudaEventCreateWithFlags(&F->fork, cudaEventDisableTiming));
    for (int q = 0; q < kMaxStreams; ++q) {
      OCR_CUDA(cudaStreamCreateWithFlags(&F->sub[q], cudaStreamNonBlocking));
      OCR_CUDA(cudaEventCreateWithFlags(&F->join[q], cudaEventDisableTiming));
    }
  }
  const int rc = plan_cameras(F);
  if (rc) return rc;
  F->has_cam = true;
  return OCR_OK;
}

}  // extern "C"

namespace {

// Plan every camera of the last ocr_set_camera: run its pruning and layout
// once on the device (on the forest's own planning stream, so nothing waits
// on the legacy default stream; the host blocks on that stream for the slot
// totals) and size its scratch.
int plan_cameras(ocr_forest *F) {
  for (CamPlan &P : F->plans) free_plan_buffers(F, P);
  if (!F->plan_st) OCR_CUDA(cudaStreamCreateWithFlags(&F->plan_st, cudaStreamNonBlocking));
  cudaStream_t ps = F->plan_st;
  OCR_CUDA(bwd_scans_prepare());
  if (F->geometry == OCR_GEOM_SHELL) {
    for (CamPlan &P : F->plans) {
      const int rc = plan_shell(F, P);
      if (rc) return rc;
    }
    OCR_CUDA(shell_rays_prepare());
    return OCR_OK;
  }
  const int G = (int)F->h_group_nodes.size();
  Topo T{F->d_geo, F->d_child, F->d_leaves, F->N, F->M, F->L, F->lt};
  for (CamPlan &P : F->plans) {
    int rc;
    if ((rc = dev_alloc(&P.d_rect, (size_t)F->N + F->M + 1, F->bytes)) ||
        (rc = dev_alloc(&P.d_off, (size_t)F->M + 1, F->bytes)) ||
        (rc = dev_alloc(&P.d_bsums, (size_t)F->bsums_blocks, F->bytes)) ||
        (rc = dev_alloc(&P.d_gslots, (size_t)G, F->bytes)))
      return rc;
    Scratch S{P.d_rect, P.d_off, nullptr, F->d_stats, nullptr, nullptr, nullptr};
    OCR_CUDA(launch_cull_leaves(T, P.cam, S, ps));
    for (int l = F->L - 1; l >= 0; --l)
      OCR_CUDA(launch_union_level(T, F->level_base[l], F->level_base[l] + F->level_count[l], P.cam,
                                  S, ps));
    OCR_CUDA(launch_area_scan(T, S, P.d_bsums, F->bsums_blocks, P.d_gslots, F->d_group_nodes, G,
                              ps));
    // the listed leaves' slots (the top-down merge's own pass)
    const long long cbs = bwd_scan_blocks(F->nc) + 2;
    if ((rc = dev_alloc(&P.d_coff, (size_t)F->nc + 1, F->bytes)) ||
        (rc = dev_alloc(&P.d_cbsums, (size_t)cbs, F->bytes)))
      return rc;
    OCR_CUDA(listed_leaf_scan(P.d_rect, F->d_cids, F->nc, P.d_cbsums, cbs, P.d_coff, ps));
    OCR_CUDA(cudaMemcpyAsync(F->h_group_slots, P.d_gslots, sizeof(long long) * G,
                             cudaMemcpyDeviceToHost, ps));
    OCR_CUDA(cudaMemcpyAsync(F->h_group_slots + G + kStats + 1, P.d_coff + F->nc,
                             sizeof(long long), cudaMemcpyDeviceToHost, ps));
    OCR_CUDA(cudaStreamSynchronize(ps));
    P.gslots.assign(F->h_group_slots, F->h_group_slots + G);
    P.ctotal = F->h_group_slots[G + kStats + 1];
    const long long total = P.gslots[G - 1];
    if ((rc = dev_alloc(&P.d_chunk, (size_t)(total / kGroup + 2), F->bytes)) ||
        (rc = dev_alloc(&P.d_entries, (size_t)(total > 0 ? total : 1), F->bytes)) ||
        (rc = dev_alloc(&P.d_ticket, 2, F->bytes)) ||
        (rc = dev_alloc(&P.d_cgroup, (size_t)(P.ctotal / kGroup + 2), F->bytes)) ||
        (rc = dev_alloc(&P.d_cval, (size_t)(P.ctotal > 0 ? P.ctotal : 1), F->bytes)))
      return rc;
  }
  return plan_batch(F);
}

// The persistent kernel's work queue for the cameras just planned (cube
// forests): per pipeline stage, for every camera, one segment of items, each
// waiting for the camera's previous non-empty stage.  Marks the batch
// unavailable (the stream path renders) when it does not apply.
int plan_batch(ocr_forest *F) {
  F->batch_ready = false;
  if (F->geometry != OCR_GEOM_CUBE || F->M < 1 || F->plans.empty()) return OCR_OK;
  const int K = (int)F->plans.size(), L = F->L;
  const long long per = F->chunks_per_item;
  std::vector<BatchSeg> segs;
  std::vector<int> last(K, -1);
  long long tickets = 0;
  auto add = [&](int k, int kind, long long nitems, long long a, long long b, int nb, int ne,
                 long long p) {
    if (nitems <= 0) return;
    BatchSeg g{};
    g.first = tickets;
    g.nitems = nitems;
    g.per = (int)p;
    g.ntickets = (nitems + p - 1) / p;
    g.a = a;
    g.b = b;
    g.cam = k;
    g.kind = kind;
    g.dep = last[k];
    g.nb = nb;
    g.ne = ne;
    last[k] = (int)segs.size();
    tickets += g.ntickets;
    segs.push_back(g);
  };
  const long long tile = 8ll * kChunk;  // leaves or nodes per set-up item
  auto up = [](long long n, long long d) { return (n + d - 1) / d; };
  for (int k = 0; k < K; ++k) add(k, kBatchCull, up(F->N, tile), 0, F->N, 0, 0, 1);
  for (int l = L - 1; l >= 0; --l)
    for (int k = 0; k < K; ++k)
      add(k, kBatchUnion, up(F->level_count[l], tile), F->level_base[l],
          F->level_base[l] + F->level_count[l], 0, 0, 1);
  for (int k = 0; k < K; ++k) add(k, kBatchReduce, up(F->M, tile), 0, F->M, 0, 0, 1);
  for (int k = 0; k < K; ++k) add(k, kBatchDown, up(F->M, tile), 0, F->M, 0, 0, 1);
  const int G = (int)F->h_group_nodes.size();
  for (int k = 0; k < K; ++k) {
    const long long ng = up(F->plans[k].gslots[G - 1], kGroup);
    if (ng > 0) add(k, kBatchChunkMap, up(ng, tile), 0, ng, 0, 0, 1);
  }
  for (int g = 0; g + 1 < G; ++g) {  // levels L - 1 .. 0: the tile level, then coarser
    const int level = L - 1 - g;
    if (level > F->lt) continue;
    for (int k = 0; k < K; ++k) {
      const long long a = F->plans[k].gslots[g], b = F->plans[k].gslots[g + 1];
      if (b <= a) continue;
      add(k, level == F->lt ? kBatchSubtree : kBatchCoarse, (b - 1) / kChunk - a / kChunk + 1, a,
          b, F->h_group_nodes[g], F->h_group_nodes[g + 1], per);
    }
  }
  for (int k = 0; k < K; ++k)
    add(k, kBatchPixel, up(F->plans[k].npix, kChunk), 0, F->plans[k].npix, 0, 0, per);
  if ((int)segs.size() > kBatchMaxSegs || tickets >= (1ll << 31)) return OCR_OK;
  std::vector<BatchCam> cams(K);
  for (int k = 0; k < K; ++k) {
    const CamPlan &P = F->plans[k];
    cams[k] = BatchCam{P.cam, P.d_rect, P.d_off, P.d_bsums, P.d_chunk, P.d_entries, P.pix_off};
  }
  cudaFree(F->d_bseg);
  F->d_bseg = nullptr;
  if (K > F->nbcam) {
    cudaFree(F->d_bcam);
    F->d_bcam = nullptr;
    F->nbcam = 0;
  }
  int rc;
  if ((rc = dev_alloc(&F->d_bseg, segs.size(), F->bytes))) return rc;
  if (!F->d_bcam) {
    if ((rc = dev_alloc(&F->d_bcam, (size_t)K, F->bytes))) return rc;
    F->nbcam = K;
  }
  if (!F->d_bctl && (rc = dev_alloc(&F->d_bctl, (size_t)kBatchCtlWords, F->bytes))) return rc;
  cudaStream_t ps = F->plan_st;
  OCR_CUDA(cudaMemcpyAsync(F->d_bseg, segs.data(), sizeof(BatchSeg) * segs.size(),
                           cudaMemcpyHostToDevice, ps));
  OCR_CUDA(cudaMemcpyAsync(F->d_bcam, cams.data(), sizeof(BatchCam) * (size_t)K,
                           cudaMemcpyHostToDevice, ps));
  OCR_CUDA(cudaStreamSynchronize(ps));  // the host vectors die on return
  F->nbseg = (int)segs.size();
  F->nbtickets = tickets;
  F->batch_ready = true;
  return OCR_OK;
}

}  // namespace

namespace {

// Enqueue one camera's render on stream st: pruning, rectangle unions, slot
// layout (recomputed; equal to the plan), subtree pass, coarsening passes and
// the pixel pass into rgba.  No host synchronisation.
int enqueue_camera(ocr_forest *F, CamPlan &P, float4 *rgba, int *counts, unsigned char *visible,
                   cudaStream_t st, bool timed, bool count, bool &subtree_ran,
                   int64_t &launches) {
  const int G = (int)F->h_group_nodes.size();
  Topo T{F->d_geo, F->d_child, F->d_leaves, F->N, F->M, F->L, F->lt};
  Field Fd{F->d_nodal, reinterpret_cast<const float4 *>(F->d_tf), F->s_min,
           7.f / (F->s_max - F->s_min)};
  Scratch S{P.d_rect, P.d_off, P.d_entries, F->d_stats, counts,
            visible, P.d_chunk, count ? F->d_stats : nullptr, P.d_ticket};
  OCR_CUDA(launch_cull_leaves(T, P.cam, S, st));
  ++launches;
  for (int l = F->L - 1; l >= 0; --l) {
    OCR_CUDA(launch_union_level(T, F->level_base[l], F->level_base[l] + F->level_count[l], P.cam,
                                S, st));
    launches += F->level_count[l] > 0;
  }
  OCR_CUDA(launch_area_scan(T, S, P.d_bsums, F->bsums_blocks, P.d_gslots, F->d_group_nodes, G,
                            st));
  launches += area_scan_blocks(F->M) > 0 ? 4 : 1;
  OCR_CUDA(launch_chunk_map(T, S, P.gslots[G - 1], st));
  launches += F->M > 0;
  const CoarseLeaves CL{F->d_cids, F->d_cindex, P.d_coff, P.d_cgroup, P.d_cval, F->nc, P.ctotal};
  if (F->merge == 1) {  // the listed leaves' slots (as planned)
    OCR_CUDA(listed_leaf_scan(P.d_rect, F->d_cids, F->nc, P.d_cbsums, bwd_scan_blocks(F->nc) + 2,
                              P.d_coff, st));
    OCR_CUDA(launch_coarse_leaf_map(CL, st));
    launches += 4;
  }
  // the passes below read the field: with host data, wait for its copy here
  // (the pruning and layout above overlap it)
  if (F->data_ready) OCR_CUDA(cudaStreamWaitEvent(st, F->data_ready, 0));
  if (timed) OCR_CUDA(cudaEventRecord(F->ev[1], st));
  // group g covers level L - 1 - g: the tile level runs the subtree pass, the
  // levels above it the coarsening passes, deepest first (or the top-down pass)
  for (int g = 0; g + 1 < G; ++g) {
    const int level = F->L - 1 - g;
    const long long a = P.gslots[g], b = P.gslots[g + 1];
    if (b <= a) continue;
    if (F->merge == 1 && level != F->lt) continue;
    if (level == F->lt) {
      if (P.d_ticket) OCR_CUDA(cudaMemsetAsync(P.d_ticket, 0, sizeof(unsigned), st));
      if (timed) OCR_CUDA(cudaEventRecord(F->ev[2], st));
      OCR_CUDA(launch_subtree(T, Fd, P.cam, F->integ, S, F->h_group_nodes[g],
                              F->h_group_nodes[g + 1], a, b, st));
      if (timed) OCR_CUDA(cudaEventRecord(F->ev[3], st));
      subtree_ran = true;
    } else {
      OCR_CUDA(launch_coarsen(T, Fd, P.cam, F->integ, S, F->h_group_nodes[g],
                              F->h_group_nodes[g + 1], a, b, nullptr, st));
    }
    ++launches;
  }
  // the super-root pass writes every pixel
  if (F->merge == 1) {
    OCR_CUDA(launch_coarse_leaves(T, Fd, P.cam, F->integ, S, CL, st));
    OCR_CUDA(launch_topdown(T, P.cam, F->integ, S, CL, P.npix, rgba, st));
    ++launches;
  } else
    OCR_CUDA(launch_coarsen(T, Fd, P.cam, F->integ, S, F->M, F->M, 0, P.npix, rgba, st));
  ++launches;
  return OCR_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Render the cameras [first, first + K) of the last ocr_set_camera into
// d_rgba (their images concatenated in order).
int render_plans(ocr_forest *F, int first, int K, float *d_rgba, void *stream,
                 ocr_stats *stats) {
  if (!F || !d_rgba) return OCR_ERR_INVALID;
  if (!F->has_data || !F->has_cam || !F->has_integ) return OCR_ERR_STATE;
  if ((uintptr_t)d_rgba & 15) return OCR_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const int G = (int)F->h_group_nodes.size();
  CamPlan *plans = F->plans.data() + first;
  long long range_pix = 0;
  for (int k = 0; k < K; ++k) range_pix += plans[k].npix;
  const long long pix0 = plans[0].pix_off;
  int *counts = stats ? stats->d_counts : nullptr;
  unsigned char *visible = stats ? stats->d_visible : nullptr;
  if (counts) OCR_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)range_pix, st));
  if (visible) OCR_CUDA(cudaMemsetAsync(visible, 0, (size_t)F->N, st));
  const bool timed = stats && stats->time_phases && K == 1;
  const bool count = stats && stats->fill_counters;  // the passes' work counters
  if (timed && !F->ev[0])
    for (cudaEvent_t &e : F->ev) OCR_CUDA(cudaEventCreate(&e));
  int64_t launches = 0;
  bool subtree_ran = false;
  OCR_CUDA(cudaMemsetAsync(F->d_stats, 0, kStats * sizeof(unsigned long long), st));
  float4 *rgba = reinterpret_cast<float4 *>(d_rgba);
  if (timed) OCR_CUDA(cudaEventRecord(F->ev[0], st));
  if (F->geometry == OCR_GEOM_SHELL) {  // this render's data in the kernels' monomial form
    if (F->data_ready) OCR_CUDA(cudaStreamWaitEvent(st, F->data_ready, 0));
    OCR_CUDA(shell_monomials(F->d_nodal, F->d_coef, F->N, st));
    ++launches;
  }
  const bool whole = first == 0 && K == (int)F->plans.size();
  if (whole && K > 1 && F->persistent && F->batch_ready && F->merge == 0 && !F->integ.surface) {
    // every camera in one persistent kernel
    Topo T{F->d_geo, F->d_child, F->d_leaves, F->N, F->M, F->L, F->lt};
    Field Fd{F->d_nodal, reinterpret_cast<const float4 *>(F->d_tf), F->s_min,
             7.f / (F->s_max - F->s_min)};
    if (F->data_ready) OCR_CUDA(cudaStreamWaitEvent(st, F->data_ready, 0));
    OCR_CUDA(launch_batch(T, Fd, F->integ, F->d_bseg, F->nbseg, F->d_bcam, F->d_bctl,
                          F->nbtickets, rgba, counts, visible, F->d_stats, count, F->nsm,
                          F->ctas_per_sm, st));
    launches += 1;
  } else if (K == 1) {
    int rc = F->geometry == OCR_GEOM_SHELL
                 ? enqueue_shell(F, plans[0], rgba, counts, visible, st, timed, launches)
                 : enqueue_camera(F, plans[0], rgba, counts, visible, st, timed, count,
                                  subtree_ran, launches);
    subtree_ran |= F->geometry == OCR_GEOM_SHELL;
    if (rc) return rc;
    if (timed) OCR_CUDA(cudaEventRecord(F->ev[4], st));
  } else {
    // fan the cameras out over the internal streams and join them back
    OCR_CUDA(cudaEventRecord(F->fork, st));
    const int ns = std::min(F->nstreams, K);
    for (int q = 0; q < ns; ++q) OCR_CUDA(cudaStreamWaitEvent(F->sub[q], F->fork, 0));
    for (int k = 0; k < K; ++k) {
      CamPlan &P = plans[k];
      const long long at = P.pix_off - pix0;
      int *cnt = counts ? counts + at : nullptr;
      int rc = F->geometry == OCR_GEOM_SHELL
                   ? enqueue_shell(F, P, rgba + at, cnt, visible, F->sub[k % ns], false,
                                   launches)
                   : enqueue_camera(F, P, rgba + at, cnt, visible, F->sub[k % ns], false,
                                    count, subtree_ran, launches);
      if (rc) return rc;
    }
    for (int q = 0; q < ns; ++q) {
      OCR_CUDA(cudaEventRecord(F->join[q], F->sub[q]));
      OCR_CUDA(cudaStreamWaitEvent(st, F->join[q], 0));
    }
  }

  if (stats) {
    stats->launches = launches;
    if (stats->d_rects)
      OCR_CUDA(cudaMemcpyAsync(stats->d_rects, plans[0].d_rect, sizeof(int4) * (size_t)F->N,
                               cudaMemcpyDeviceToDevice, st));
    if (timed) {
      OCR_CUDA(cudaEventSynchronize(F->ev[4]));
      OCR_CUDA(cudaEventElapsedTime(&stats->ms_prune, F->ev[0], F->ev[1]));
      OCR_CUDA(cudaEventElapsedTime(&stats->ms_merge, F->ev[1], F->ev[4]));
      stats->ms_subtree = 0.f;
      if (subtree_ran) OCR_CUDA(cudaEventElapsedTime(&stats->ms_subtree, F->ev[2], F->ev[3]));
    }
    if (stats->fill_counters) {
      unsigned long long h[kStats];
      OCR_CUDA(cudaMemcpyAsync(F->h_group_slots + G, F->d_stats, sizeof(h), cudaMemcpyDeviceToHost,
                               st));
      OCR_CUDA(cudaStreamSynchronize(st));
      memcpy(h, F->h_group_slots + G, sizeof(h));
      stats->segments = (int64_t)(h[kStatSegments] + h[kStatCoarse + kStatSegments]);
      stats->rk_steps = (int64_t)(h[kStatSteps] + h[kStatCoarse + kStatSteps]);
      stats->leaf_tests = (int64_t)(8 * h[kStatTests] + h[kStatCoarse + kStatTests]);
      stats->slots = (int64_t)(h[kStatSlots] + h[kStatCoarse + kStatSlots]);
      stats->subtree_segments = (int64_t)h[kStatSegments];
      stats->subtree_rk_steps = (int64_t)h[kStatSteps];
      stats->subtree_node_visits = (int64_t)h[kStatTests];
      stats->visible_leaves = (int64_t)h[kStatVisible];
      if (F->geometry == OCR_GEOM_SHELL) {  // one pass over every (leaf, pixel) pair
        int64_t pairs = 0;
        for (int k = 0; k < K; ++k) pairs += plans[k].npairs;
        stats->leaf_tests = pairs;
        stats->subtree_node_visits = 0;
        stats->slots = 0;
      }
      if (h[kStatErrors]) return OCR_ERR_DEVICE;
    }
  }
  return OCR_OK;
}

}  // namespace

extern "C" {

int ocr_render(ocr_forest *F, float *d_rgba, void *stream, ocr_stats *stats) {
  if (!F) return OCR_ERR_INVALID;
  if (!F->has_cam) return OCR_ERR_STATE;
  return render_plans(F, 0, (int)F->plans.size(), d_rgba, stream, stats);
}

int ocr_render_view(ocr_forest *F, int view, float *d_rgba, void *stream, ocr_stats *stats) {
  if (!F) return OCR_ERR_INVALID;
  if (!F->has_cam) return OCR_ERR_STATE;
  if (view < 0 || view >= (int)F->plans.size()) return OCR_ERR_INVALID;
  return render_plans(F, view, 1, d_rgba, stream, stats);
}

}  // extern "C"

namespace {
// the adjoint's per-segment buffers (list index beside each key, leaf-grouped
// list, records) for at least n segments, and the list's append counter
int grow_adjoint(ocr_forest *F, long long n) {
  if (F->seg_cap >= n && F->d_lmcount) return OCR_OK;
  cudaFree(F->d_skpos);
  cudaFree(F->d_slm);
  cudaFree(F->d_srta);
  cudaFree(F->d_srg);
  F->d_skpos = nullptr;
  F->d_slm = nullptr;
  F->d_srta = nullptr;
  F->d_srg = nullptr;
  F->bytes -= F->seg_cap *
              (int64_t)(sizeof(unsigned) + sizeof(int2) + sizeof(float2) + sizeof(float4));
  F->seg_cap = 0;
  const long long want = std::min(n + n / 8 + 64, 0xffffffffll);
  int rc;
  if ((rc = dev_alloc(&F->d_skpos, (size_t)want, F->bytes)) ||
      (rc = dev_alloc(&F->d_slm, (size_t)want, F->bytes)) ||
      (rc = dev_alloc(&F->d_srta, (size_t)want, F->bytes)) ||
      (rc = dev_alloc(&F->d_srg, (size_t)want, F->bytes)))
    return rc;
  F->seg_cap = want;
  if (!F->d_lmcount && (rc = dev_alloc(&F->d_lmcount, 1, F->bytes))) return rc;
  return OCR_OK;
}

// (re)allocate a scratch buffer to hold at least n elements
template <typename T>
int grow(ocr_forest *F, T **p, long long &cap, long long n) {
  if (n <= cap) return OCR_OK;
  cudaFree(*p);
  *p = nullptr;
  F->bytes -= cap * (int64_t)sizeof(T);
  cap = 0;
  const long long want = n + n / 8 + 64;
  int rc = dev_alloc(p, (size_t)want, F->bytes);
  if (rc) return rc;
  cap = want;
  return OCR_OK;
}
}  // namespace

extern "C" {

int ocr_render_host(ocr_forest *F, const float *h_nodal, const float *h_tf, float s_min,
                    float s_max, float *h_rgba, void *stream, ocr_stats *stats) {
  if (!F || !h_nodal || !h_tf || !h_rgba) return OCR_ERR_INVALID;
  if (!F->has_cam || !F->has_integ) return OCR_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nv = (F->geometry == OCR_GEOM_SHELL ? 27ll : 8ll) * F->N;
  int rc;
  const long long tf_at = (nv + 3) / 4 * 4;  // the 32 knot values after the data, 16 B aligned
  if ((rc = grow(F, &F->d_hnodal, F->hnodal_cap, tf_at + 32))) return rc;
  if ((rc = grow(F, &F->d_hrgba, F->hrgba_cap, 4 * F->total_pix))) return rc;
  F->d_htf = F->d_hnodal + tf_at;
  if (!F->copy_st) {
    OCR_CUDA(cudaStreamCreateWithFlags(&F->copy_st, cudaStreamNonBlocking));
    OCR_CUDA(cudaEventCreateWithFlags(&F->copy_ev, cudaEventDisableTiming));
  }
  // the copy in, ordered after the caller's earlier work on its stream
  OCR_CUDA(cudaEventRecord(F->copy_ev, st));
  OCR_CUDA(cudaStreamWaitEvent(F->copy_st, F->copy_ev, 0));
  OCR_CUDA(cudaMemcpyAsync(F->d_hnodal, h_nodal, sizeof(float) * (size_t)nv,
                           cudaMemcpyHostToDevice, F->copy_st));
  OCR_CUDA(cudaMemcpyAsync(F->d_htf, h_tf, sizeof(float) * 32, cudaMemcpyHostToDevice,
                           F->copy_st));
  OCR_CUDA(cudaEventRecord(F->copy_ev, F->copy_st));
  if ((rc = ocr_forest_set_data(F, F->d_hnodal, F->d_htf, s_min, s_max, stream))) {
    OCR_CUDA(cudaStreamWaitEvent(st, F->copy_ev, 0));
    return rc;
  }
  F->data_ready = F->copy_ev;
  rc = ocr_render(F, reinterpret_cast<float *>(F->d_hrgba), stream, stats);
  F->data_ready = nullptr;
  OCR_CUDA(cudaStreamWaitEvent(st, F->copy_ev, 0));  // the copy is done before we return
  if (rc) return rc;
  OCR_CUDA(cudaMemcpyAsync(h_rgba, F->d_hrgba, sizeof(float) * 4 * (size_t)F->total_pix,
                           cudaMemcpyDeviceToHost, st));
  OCR_CUDA(cudaStreamSynchronize(st));
  return OCR_OK;
}

int ocr_render_backward(ocr_forest *F, const float *d_dL_drgba, float *d_grad_nodal,
                        float *d_grad_tf, void *stream) {
  if (!F || !d_dL_drgba || !d_grad_nodal || !d_grad_tf) return OCR_ERR_INVALID;
  if (!F->has_data || !F->has_cam || !F->has_integ) return OCR_ERR_STATE;
  if (F->integ.surface) return OCR_ERR_UNSUPPORTED;
  if ((uintptr_t)d_dL_drgba & 15) return OCR_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (F->geometry == OCR_GEOM_SHELL) {
    // rebuild the first camera's lists with the leaf-grouped list, then the
    // values pass (one warp per ray) and the segment pass (one thread each)
    CamPlan &P = F->plans[0];
    const Field Fd{F->d_coef, reinterpret_cast<const float4 *>(F->d_tf), F->s_min,
                   7.f / (F->s_max - F->s_min)};
    if (P.nhits >= 0xffffffffll) return OCR_ERR_UNSUPPORTED;  // list indices are 32-bit
    int rc = grow_adjoint(F, P.nhits);
    if (rc) return rc;
    OCR_CUDA(cudaMemsetAsync(d_grad_nodal, 0, sizeof(float) * 27 * (size_t)F->N, st));
    OCR_CUDA(cudaMemsetAsync(d_grad_tf, 0, sizeof(float) * 32, st));
    OCR_CUDA(cudaMemsetAsync(F->d_stats, 0, kStats * sizeof(unsigned long long), st));
    OCR_CUDA(shell_monomials(F->d_nodal, F->d_coef, F->N, st));
    rc = enqueue_shell_lists(F, P, nullptr, st, true);
    if (rc) return rc;
    const float4 *dL = reinterpret_cast<const float4 *>(d_dL_drgba);
    OCR_CUDA(bwd_shell_values(F->d_geo, F->N, F->shell, Fd, P.cam, F->integ, dL, F->d_slm,
                              P.nhits, F->d_srg, F->d_err, F->nsm, st));
    OCR_CUDA(bwd_ray_scans(P.cam, dL, P.d_ray_off, nullptr, P.d_keys, F->d_skpos, P.nhits, P.cap,
                           F->d_srta, F->d_srg, F->d_err, F->nsm, st));
    OCR_CUDA(bwd_shell_adjoint(F->d_geo, F->N, F->shell, Fd, P.cam, F->integ, dL, F->d_slm,
                               F->d_srta, F->d_srg, P.nhits, d_grad_nodal, d_grad_tf, F->nsm,
                               st));
    OCR_CUDA(bwd_fold_errors(F->d_err, F->d_stats + kStatErrors, st));
    return OCR_OK;
  }
  CamPlan &P0 = F->plans[0];
  const Cam &cam = P0.cam;
  const long long npix = P0.npix;
  Topo T{F->d_geo, F->d_child, F->d_leaves, F->N, F->M, F->L, F->lt};
  Field Fd{F->d_nodal, reinterpret_cast<const float4 *>(F->d_tf), F->s_min,
           7.f / (F->s_max - F->s_min)};
  Scratch S{P0.d_rect, P0.d_off, nullptr, F->d_stats, nullptr, nullptr, nullptr};
  if (!F->nsm) {
    int dev = 0;
    OCR_CUDA(cudaGetDevice(&dev));
    OCR_CUDA(cudaDeviceGetAttribute(&F->nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  int rc;
  const long long nb = std::max(bwd_scan_blocks(F->N), bwd_scan_blocks(npix)) + 2;
  if ((rc = grow(F, &F->d_bsums, F->bsums_cap, nb))) return rc;
  {
    const long long c0 = F->ray_cap;
    if ((rc = grow(F, &F->d_rcount, F->ray_cap, npix))) return rc;
    if (F->ray_cap != c0 || !F->d_rcursor || !F->d_ray_off) {  // same capacity for all three
      cudaFree(F->d_rcursor);
      cudaFree(F->d_ray_off);
      F->d_rcursor = nullptr;
      F->d_ray_off = nullptr;
      if ((rc = dev_alloc(&F->d_rcursor, (size_t)F->ray_cap, F->bytes)) ||
          (rc = dev_alloc(&F->d_ray_off, (size_t)F->ray_cap + 1, F->bytes)))
        return rc;
    }
  }
  const float4 *dL = reinterpret_cast<const float4 *>(d_dL_drgba);
  if (!P0.bwd_ready) {
    // the sizes of the pair space and of the hit lists, and the lists' layout
    // (every ray's hits, an exclusive prefix in d_ray_off), depend on the
    // camera alone: found once, blocking the host twice
    OCR_CUDA(launch_cull_leaves(T, cam, S, st));
    OCR_CUDA(bwd_leaf_scan(T, P0.d_rect, F->d_bsums, F->bsums_cap, F->d_leaf_off, st));
    long long *h = F->h_group_slots + F->h_group_nodes.size();  // pinned scratch
    OCR_CUDA(cudaMemcpyAsync(h, F->d_leaf_off + F->N, sizeof(long long), cudaMemcpyDeviceToHost,
                             st));
    OCR_CUDA(cudaStreamSynchronize(st));
    const long long npairs = h[0];
    if ((rc = grow(F, &F->d_pchunk, F->pchunk_cap, npairs / 256 + 2))) return rc;
    OCR_CUDA(bwd_chunk_map(F->d_leaf_off, F->N, F->d_pchunk, st));
    OCR_CUDA(cudaMemsetAsync(F->d_rcount, 0, sizeof(int) * (size_t)npix, st));
    OCR_CUDA(bwd_pair_hits(0, T, cam, P0.d_rect, F->d_leaf_off, F->d_pchunk, npairs, nullptr,
                           F->d_rcount, nullptr, nullptr, F->d_mkey, F->fx, nullptr, nullptr,
                           nullptr, nullptr, 0, nullptr, st));
    OCR_CUDA(bwd_count_scan(F->d_rcount, npix, F->d_bsums, F->bsums_cap, F->d_ray_off, st));
    OCR_CUDA(cudaMemsetAsync(F->d_stats + kStatMaxHits, 0, sizeof(unsigned long long), st));
    OCR_CUDA(bwd_max_hits(F->d_rcount, npix, F->d_stats + kStatMaxHits, st));
    OCR_CUDA(cudaMemcpyAsync(h, F->d_ray_off + npix, sizeof(long long), cudaMemcpyDeviceToHost,
                             st));
    OCR_CUDA(cudaMemcpyAsync(h + 1, F->d_stats + kStatMaxHits, sizeof(long long),
                             cudaMemcpyDeviceToHost, st));
    OCR_CUDA(cudaStreamSynchronize(st));
    const long long nh = h[0];
    if (nh >= 0xffffffffll) return OCR_ERR_UNSUPPORTED;  // list indices are 32-bit
    int cap = 32;  // per-warp lists sized for the longest ray (longer ones: device error)
    while (cap < h[1] && cap < kShellMaxCap) cap <<= 1;
    if ((rc = grow(F, &F->d_hkey, F->hit_cap, nh)) || (rc = grow_adjoint(F, nh))) return rc;
    P0.bwd_npairs = npairs;
    P0.bwd_nh = nh;
    P0.bwd_cap = cap;
    P0.bwd_ready = true;
  }
  const long long npairs = P0.bwd_npairs, nh = P0.bwd_nh;
  OCR_CUDA(cudaMemsetAsync(d_grad_nodal, 0, sizeof(float) * 8 * (size_t)F->N, st));
  OCR_CUDA(cudaMemsetAsync(d_grad_tf, 0, sizeof(float) * 32, st));
  OCR_CUDA(cudaMemsetAsync(F->d_stats, 0, kStats * sizeof(unsigned long long), st));

  // leaf rectangles, then the (leaf, pixel) pair space in Morton order (as
  // planned: the same camera)
  OCR_CUDA(launch_cull_leaves(T, cam, S, st));
  OCR_CUDA(bwd_leaf_scan(T, P0.d_rect, F->d_bsums, F->bsums_cap, F->d_leaf_off, st));
  OCR_CUDA(bwd_chunk_map(F->d_leaf_off, F->N, F->d_pchunk, st));

  // the hit lists (mirrored Morton keys) of the rays with an image adjoint,
  // each in its place of the camera's list layout (every ray's hits, from the
  // plan), and the leaf-grouped list
  OCR_CUDA(cudaMemsetAsync(F->d_rcursor, 0, sizeof(int) * (size_t)npix, st));
  OCR_CUDA(cudaMemsetAsync(F->d_lmcount, 0, sizeof(unsigned long long), st));
  OCR_CUDA(bwd_pair_hits(2, T, cam, P0.d_rect, F->d_leaf_off, F->d_pchunk, npairs, dL, nullptr,
                         F->d_ray_off, F->d_rcursor, F->d_mkey, F->fx, F->d_hkey, F->d_skpos,
                         F->d_slm, F->d_lmcount, nh, F->d_err, st));

  // segment values, per-ray scans, segment adjoints over the entries written
  OCR_CUDA(bwd_cube_values(T, Fd, cam, F->integ, F->d_slm, nh, F->d_lmcount, F->d_srg, F->nsm,
                           st));
  OCR_CUDA(bwd_ray_scans(cam, dL, F->d_ray_off, F->d_rcursor, F->d_hkey, F->d_skpos, nh,
                         P0.bwd_cap, F->d_srta, F->d_srg, F->d_err, F->nsm, st));
  OCR_CUDA(bwd_cube_adjoint(T, Fd, cam, F->integ, dL, F->d_slm, F->d_srta, F->d_srg, nh,
                            F->d_lmcount, d_grad_nodal, d_grad_tf, F->nsm, st));
  OCR_CUDA(bwd_fold_errors(F->d_err, F->d_stats + kStatErrors, st));
  return OCR_OK;
}

int ocr_fold_segments(const float *d_val, const float *d_iv, int n, float *d_out,
                      void *stream) {
  if (!d_val || !d_iv || !d_out || n < 1 || n > (1 << 20)) return OCR_ERR_INVALID;
  if (((uintptr_t)d_val & 15) || ((uintptr_t)d_iv & 7) || ((uintptr_t)d_out & 15))
    return OCR_ERR_INVALID;
  OCR_CUDA(shell_fold_segments(reinterpret_cast<const float4 *>(d_val),
                               reinterpret_cast<const float2 *>(d_iv), n,
                               reinterpret_cast<float4 *>(d_out), (cudaStream_t)stream));
  return OCR_OK;
}

int ocr_sync(ocr_forest *F, void *stream) {
  if (!F) return OCR_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  // the last word of the pinned scratch is ocr_sync's own
  const size_t at = F->geometry == OCR_GEOM_SHELL ? kStats + 2 : F->h_group_nodes.size() + kStats;
  unsigned long long *h = reinterpret_cast<unsigned long long *>(F->h_group_slots) + at;
  OCR_CUDA(cudaMemcpyAsync(h, F->d_err, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  OCR_CUDA(cudaStreamSynchronize(st));
  if (!h[0]) return OCR_OK;
  OCR_CUDA(cudaMemsetAsync(F->d_err, 0, sizeof(unsigned long long), st));
  OCR_CUDA(cudaStreamSynchronize(st));
  return OCR_ERR_DEVICE;
}

int ocr_set_tuning(ocr_forest *F, const ocr_tuning *t) {
  if (!F || !t) return OCR_ERR_INVALID;
  if (t->tile_depth < 1 || t->tile_depth > kSubtreeDepth || t->streams < 1 ||
      t->streams > kMaxStreams || t->shell_warps < 0 || t->shell_warps > 8 || t->merge < 0 ||
      t->merge > 1 || t->persistent < 0 || t->persistent > 1 || t->chunks_per_item < 1 ||
      t->chunks_per_item > 64 || t->ctas_per_sm < 0 || t->ctas_per_sm > 8)
    return OCR_ERR_INVALID;
  F->nstreams = t->streams;
  F->shell_warps = t->shell_warps;
  F->merge = t->merge;
  F->persistent = t->persistent;
  F->ctas_per_sm = t->ctas_per_sm;
  const bool requeue = t->chunks_per_item != F->chunks_per_item;
  F->chunks_per_item = t->chunks_per_item;
  if (t->tile_depth != F->tile_depth) {
    F->tile_depth = t->tile_depth;
    F->lt = F->L > F->tile_depth ? F->L - F->tile_depth : 0;
    if (F->geometry == OCR_GEOM_CUBE) {
      if (!F->plan_st) OCR_CUDA(cudaStreamCreateWithFlags(&F->plan_st, cudaStreamNonBlocking));
      const int rc = build_listed_leaves(F, F->plan_st);
      if (rc) return rc;
    }
    if (F->has_cam && F->geometry == OCR_GEOM_CUBE) {
      F->has_cam = false;
      const int rc = plan_cameras(F);  // also rebuilds the batch queue
      if (rc) return rc;
      F->has_cam = true;
    }
  } else if (requeue && F->has_cam && F->geometry == OCR_GEOM_CUBE) {
    if (!F->plan_st) OCR_CUDA(cudaStreamCreateWithFlags(&F->plan_st, cudaStreamNonBlocking));
    const int rc = plan_batch(F);
    if (rc) return rc;
  }
  return OCR_OK;
}

int ocr_get_tuning(const ocr_forest *F, ocr_tuning *t) {
  if (!F || !t) return OCR_ERR_INVALID;
  t->tile_depth = F->tile_depth;
  t->streams = F->nstreams;
  t->shell_warps = F->shell_warps;
  t->merge = F->merge;
  t->persistent = F->persistent;
  t->chunks_per_item = F->chunks_per_item;
  t->ctas_per_sm = F->ctas_per_sm;
  t->ms = 0.f;
  return OCR_OK;
}

int ocr_autotune(ocr_forest *F, int reps, ocr_tuning *best, ocr_tuning *tried, int max_tried,
                 int *ntried) {
  if (!F || !best || reps < 1 || reps > 100 || max_tried < 0 || (max_tried > 0 && !tried))
    return OCR_ERR_INVALID;
  if (!F->has_data || !F->has_cam || !F->has_integ) return OCR_ERR_STATE;
  const int K = (int)F->plans.size();
  std::vector<ocr_tuning> cand;
  const int streams[] = {1, 2, 4, 8};
  const int warps[] = {1, 2, 4, 8};
  auto tuning = [&](int d, int s, int w, int m, int p, int c, int o) {
    ocr_tuning t{};
    t.tile_depth = d;
    t.streams = s;
    t.shell_warps = w;
    t.merge = m;
    t.persistent = p;
    t.chunks_per_item = c;
    t.ctas_per_sm = o;
    return t;
  };
  for (int si = 0; si < 4; ++si) {
    if (K == 1 && streams[si] != F->nstreams) continue;  // one camera: streams are unused
    if (F->geometry == OCR_GEOM_SHELL) {
      for (int w : warps)
        cand.push_back(tuning(F->tile_depth, streams[si], w, 0, 0, F->chunks_per_item, 0));
    } else {
      for (int m = 0; m <= 1; ++m)
        for (int d = 1; d <= kSubtreeDepth; ++d)
          if (d <= F->L || d == kSubtreeDepth)
            cand.push_back(tuning(d, streams[si], 0, m, 0, F->chunks_per_item, 0));
    }
  }
  if (F->geometry == OCR_GEOM_CUBE && K > 1) {
    // the persistent kernel: tile depth x chunks per ticket x CTAs per SM
    const int chunks[] = {8, 16, 32}, occ[] = {0, 7, 6};
    for (int d = 1; d <= kSubtreeDepth; ++d)
      if (d <= F->L || d == kSubtreeDepth)
        for (int c : chunks)
          for (int o : occ) cand.push_back(tuning(d, F->nstreams, 0, 0, 1, c, o));
  }
  float4 *rgba = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = OCR_OK;
  ocr_tuning keep;
  ocr_get_tuning(F, &keep);
  ocr_tuning win = keep;
  win.ms = INFINITY;
  int n = 0;
  cudaError_t ce = cudaMalloc((void **)&rgba, sizeof(float4) * (size_t)F->total_pix);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) rc = cuda_fail(ce);
  for (size_t c = 0; c < cand.size() && rc == OCR_OK; ++c) {
    if ((rc = ocr_set_tuning(F, &cand[c]))) break;
    if ((rc = ocr_render(F, reinterpret_cast<float *>(rgba), st, nullptr))) break;  // warm-up
    ce = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && ce == cudaSuccess && rc == OCR_OK; ++r)
      rc = ocr_render(F, reinterpret_cast<float *>(rgba), st, nullptr);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce != cudaSuccess) rc = cuda_fail(ce);
    if (rc) break;
    cand[c].ms = ms / (float)reps;
    if (n < max_tried) tried[n] = cand[c];
    ++n;
    if (cand[c].ms < win.ms) win = cand[c];
  }
  if (rgba) cudaFree(rgba);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (ntried) *ntried = n;
  if (rc) {
    ocr_set_tuning(F, &keep);
    return rc;
  }
  if ((rc = ocr_set_tuning(F, &win))) return rc;
  *best = win;
  return OCR_OK;
}

int64_t ocr_device_bytes(const ocr_forest *F) { return F ? F->bytes : 0; }

void ocr_destroy(ocr_forest *F) {
  if (!F) return;
  free_all(F);
  delete F;
}

}  // extern "C"
