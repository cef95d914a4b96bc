// Internal types shared by the host API and the kernels (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "sge.h"

namespace sge {

constexpr int SGE_MAX_TEX_DEV = SGE_MAX_TEXTURES;
constexpr int MAX_READ = 4;              // albedo, normal, roughness, metallic
constexpr int TILE = 16;                 // tile edge in pixels; one CTA thread per pixel
constexpr int TILE_PX = TILE * TILE;     // 256 threads
constexpr int kLightBin = 256;           // bins up to this size use the fast path
constexpr int kMaxPairsPerItem = 64;     // longest run of pairs one work item takes
constexpr int kHeavyCand = 32;           // candidate triangles kept per pixel of a heavy tile
constexpr int kCandWords = kHeavyCand / 8;  // int4 words of a pixel's candidate list
constexpr int kNotDrawn = (int)0x80000000;  // projected X of a vertex its triangles drop
constexpr int ROLE_ALBEDO = SGE_ROLE_ALBEDO, ROLE_NORMAL = SGE_ROLE_NORMAL;
constexpr int ROLE_ROUGHNESS = SGE_ROLE_ROUGHNESS, ROLE_METALLIC = SGE_ROLE_METALLIC;
constexpr int SHADE_UNLIT = SGE_SHADE_UNLIT, SHADE_LAMBERT = SGE_SHADE_LAMBERT, SHADE_GGX = SGE_SHADE_GGX;
constexpr int SHADE_TRANSPARENT = SGE_SHADE_TRANSPARENT;

struct TexDev {
  const float* ptr;
  int w, h, c;
  float eps;
  int role;
  int read;          // does the shading model read this texture (so its texels contribute)?
  long long offset;  // first parameter index of this texture in theta
  int index;         // position of this texture in the scene's list
};

#ifndef SGE_CHECKED
#define SGE_CHECKED 0
#endif

// Bounds of the checked build's range checks (SGE_CHECKED=1): the true sizes unless
// sge_check_limit lowered them.  Unused by the unchecked build.
struct CheckDev {
  uint32_t* status;    // the device status word a failing check writes
  uint32_t* where;     // [2]: the first failing check's site and (low 32 bits of) its index
  int nv, nuv;         // vertex and UV indices
  long long bins;      // bin entries
  long long sign_words;  // words of one estimate's sign planes
  long long params;    // parameter indices
};

// Device view of a scene, passed to kernels by value.
struct SceneDev {
  const float* pos;
  int nv;
  float eps_pos;
  const int* pidx;
  int nt;
  const float* uvs;
  const int* uvidx;
  int nuv;
  int ntex;
  TexDev tex[SGE_MAX_TEX_DEV];
  int nread;                 // textures the shading model reads (at most one per role)
  int read_k[MAX_READ];      // their indices in tex[]
  TexDev rtex[MAX_READ];     // copies of tex[read_k[r]], so kernels index them with constants
  int grouped;               // > 1 read textures, all of one size: one footprint serves them all
  const float* mvp;
  const float* cam_pos;
  int nviews;
  int W, H;
  float near_w;
  const float* targets;
  float bg[3];
  int shading;
  float light_dir[3], light_rgb[3], ambient;
  long long n_params;
  int tiles_x, tiles_y;
  int foot_nearest;  // credit the nearest texel instead of the bilinear 2x2 footprint (SGE_FOOT_NEAREST)
  CheckDev chk;
};

// Views of one estimate call, by value (graph capture bakes them in).
struct ViewList {
  int n;
  int id[SGE_MAX_VIEWS_PER_CALL];
};

// Scratch carved out of the caller's workspace.
struct Workspace {
  int4* tri_rect;        // [max_views][nt] tile rectangle (x0,y0,x1,y1) of each triangle's bin span
  int* tri_margin;       // [max_views][nt] perturbation margin of each triangle, fixed-point units
  float2* tri_z;         // [max_views][nt] depth interval of each triangle under any perturbation
  int4* pverts;          // [max_views][max_pairs][nv][2] projected perturbed vertices (X, Y, z, iw), sides +/-
  uint8_t* vbits;        // [max_views][max_pairs][nv] bits 0-2: s = -1 for x,y,z; 3: side + drawable; 4: side -
  uint32_t* tile_count;  // [max_views][n_tiles]
  uint32_t* tile_off;    // [max_views][n_tiles + 1] exclusive scan of counts
  uint32_t* tile_cur;    // [max_views][n_tiles] fill cursors
  uint32_t* bins;        // [bin_capacity] triangle ids grouped by (view slot, tile)
  uint32_t* items;       // [max_views * n_tiles] (view slot << 24 | tile): light bins first, heavy from the end
  uint32_t* tile_live;   // [max_views][n_tiles] triangles left at the front of each bin by k_bin_prune
  int4* cand;            // [max_views][n_tiles][kCandWords][256] candidate triangles of each pixel: live
                         // indices, 8-bit in the first word of a light tile, 16-bit in all words of a heavy one
  uint8_t* ncand;        // [max_views][n_tiles][256] their number (> 16: test every live triangle)
  uint32_t* counters;    // [0] light items, [1] their work counter, [2] total bin entries, [3] status,
                         // [4] heavy items, [5] their work counter
  unsigned long long* keys;  // [2][H*W] staged depth|ID buffers (both sides)
  float2* uvbuf;             // [2][H*W] staged UV buffers
  float* dfbuf;              // [H*W] staged loss differences
  uint32_t* tsign;       // [max_views][max_pairs][sgn_words] texel sign planes of each estimate: 4 bits
                         // per texel (bit c: channel c has s = -1) of every texture the shading reads
  long long sgn_words;   // 32-bit words of one estimate's planes
  int sgn_off[SGE_MAX_TEXTURES];  // word offset of texture k's plane in them (-1: not read)
  uint32_t* kcount;      // [n_kcount] transparent scenes: contributions per key of the running call
                         // (welded vertex v at v, texel t of read texture k at kc_off[k] + t), added
                         // to every channel's count and cleared by k_expand_counts; zero between calls
  long long n_kcount;
  long long kc_off[SGE_MAX_TEXTURES];
  long long bin_capacity;
  int max_views;
  int max_pairs;
  int light_bin;  // bins of at most this many triangles are light items (fast kernel)
};

// What a batched launch needs of one scene, kept in the scene's workspace (written on the
// stream by launch_put_desc) so that the launch's parameter holds one pointer per asset.
struct __align__(16) AssetDesc {
  SceneDev S;
  Workspace ws;
};
static_assert(sizeof(AssetDesc) % 16 == 0, "AssetDesc is copied as 16-byte words");

// One asset of a batched estimate call.
struct BatchAsset {
  const AssetDesc* desc;  // device
  float* grad;
  uint32_t* counts;
  float* loss;
  int n_views;
  int view[SGE_MAX_BATCH_VIEWS];
};

// A batched call: every estimate of several scenes (one shading model) in one persistent launch.
// Assets are taken in order; each asset's items come from its own work counters.
struct BatchArgs {
  uint64_t seed;
  uint32_t iter;
  const uint32_t* iter_dev;  // device iteration index read at run time instead of iter (or NULL)
  int pairs;           // pairs per view of the whole call
  int pairs_per_item;
  int pair_begin;
  int pair_count;
  int light_bin;       // tiles with at most this many live triangles are light items
  int n;
  BatchAsset as[SGE_MAX_BATCH];
};
// Pruning of every asset of P in one launch (after each asset's binning with defer_prune).
cudaError_t launch_prune_batch(const BatchArgs& P, int max_tiles, int max_views, cudaStream_t st);

// ---- kernels launchers (all asynchronous on `st`)
// Tile binning of every triangle for each view of `vl`, conservative for any
// perturbation of at most eps_pos per coordinate.  Fills ws bins / items.  With `prune`
// (the estimators), k_bin_prune then drops from each bin the triangles no perturbation can
// make visible in the tile, lists the items by their live counts and stores each pixel's
// candidate triangles.
// defer_prune: the caller prunes later (k_bin_prune_batch): the scan lists no items either.
cudaError_t launch_binning(const SceneDev& S, const Workspace& ws, const ViewList& vl, cudaStream_t st,
                           bool prune = false, bool defer_prune = false);
cudaError_t launch_prune(const SceneDev& S, const Workspace& ws, const ViewList& vl, cudaStream_t st);

struct EstimateArgs {
  uint64_t seed;
  uint32_t iter;
  int pairs;           // pairs per view of the whole call
  int pairs_per_item;
  int pair_begin;      // the block of pairs this launch covers: [pair_begin, pair_begin + pair_count)
  int pair_count;
  float* grad;
  uint32_t* counts;
  float* loss;
  float* delta_f;
  const uint32_t* iter_dev;  // device iteration index read at run time instead of iter (or NULL)
};
// Iteration index of an estimate call: the device word when the call reads it at run time.
__host__ __device__ inline uint32_t iter_of(const EstimateArgs& a) { return a.iter_dev ? *a.iter_dev : a.iter; }
// Both estimator kernels: the fast path over light bins, the general one over heavy bins.
// ev_fast (three events, or NULL) are recorded on st right before and after the fast kernel
// and after the heavy one.
cudaError_t launch_estimate(const SceneDev& S, const Workspace& ws, const ViewList& vl,
                            const EstimateArgs& a, int grid_fast, int grid_heavy, cudaStream_t st,
                            const cudaEvent_t* ev_fast = nullptr);
cudaError_t launch_fast(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                        int grid, cudaStream_t st);
// Perturbed, projected vertices of both sides for every (view slot, pair) of a block of pairs.
cudaError_t launch_vertex_pass(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                               cudaStream_t st);
int estimate_blocks_per_sm(int shading, int grouped, int group_channels);
// channels of every read texture together (the channel sums of a texel-group table entry)
int group_channels(const SceneDev& S);
int fast_blocks_per_sm(int shading, int grouped);

// Batched form of the two estimator kernels over BatchArgs' assets.
// Image error of background-only tiles (both sides show the background), added to loss[slot].
cudaError_t launch_background_loss(const SceneDev& S, const Workspace& ws, const ViewList& vl, float* loss,
                                   cudaStream_t st);
cudaError_t launch_put_desc(const AssetDesc& d, AssetDesc* dst, cudaStream_t st);
cudaError_t launch_fast_batch(const BatchArgs& P, int shading, int grid, cudaStream_t st);
cudaError_t launch_heavy_batch(const BatchArgs& P, int shading, int grid, cudaStream_t st);
int fast_batch_blocks_per_sm(int shading);
int heavy_batch_blocks_per_sm(int shading);

// Staged path: render one side of one estimate into keys/uv/rgb.
cudaError_t launch_render(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key,
                          int side, unsigned long long* keys, float2* uv, float* rgb, cudaStream_t st);
// Staged path: loss differences and scatter of one estimate from both sides' buffers.
cudaError_t launch_plain_pair(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key,
                              const EstimateArgs& a, float loss_scale, cudaStream_t st);

// Full-image estimator (Eq. 4): one estimate's whole-image loss difference added to *out (both
// renders staged in the workspace), and the accumulation of every parameter's sum over a call.
cudaError_t launch_image_delta(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key, float* out,
                               cudaStream_t st);
cudaError_t launch_full_image_grad(const SceneDev& S, const ViewList& vl, int pairs, uint64_t seed, uint32_t iter,
                                   const float* dF, float* grad, uint32_t* counts, cudaStream_t st);

// y (+)= A x for 3-vectors per row, A in CSR (row pointers, columns, weights; device).
cudaError_t launch_csr_vec3(const int32_t* ptr, const int32_t* col, const float* w, int n_rows, const float* x,
                            float* y, int accumulate, cudaStream_t st);

// Transparent geometry (Section 4.4), after launch_binning without pruning: every estimate of a
// block of pairs (deep lists, front-to-back composite, f+ - f-, credits of every listed fragment),
// and one render's deep ID buffer / composite / image error (added to loss[slot]).
cudaError_t launch_deep_estimate(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                                 cudaStream_t st);
cudaError_t launch_render_deep(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key, int side,
                               unsigned long long* deep, float* rgb, float* loss, cudaStream_t st);

// Throughput probe of global float reductions: n_threads threads, per_thread each, thread i on
// buf[i mod n_addr].
cudaError_t launch_red_bench(float* buf, long long n_addr, long long n_threads, int per_thread, cudaStream_t st);

// Image error of unperturbed renders (forward of the autograd form), added to loss[slot].
cudaError_t launch_render_loss(const SceneDev& S, const Workspace& ws, int slot, int view, float* loss,
                               cudaStream_t st);
// out = scale * grad / (2 eps n_total) per parameter (Eq. 9).
cudaError_t launch_gradient(const SceneDev& S, const float* grad, long long n_total, const float* scale, float* out,
                            cudaStream_t st);
// t_dev (device, or NULL for o.t): Adam's step number read at run time.
cudaError_t launch_step(const SceneDev& S, const sge_opt& o, float* grad, uint32_t* counts,
                        long long n_total, float* m, float* v, cudaStream_t st, const int32_t* t_dev = nullptr);
// state[0] += d_iter, state[1] += d_t (one thread).
cudaError_t launch_iter_advance(uint32_t* state, int d_iter, int d_t, cudaStream_t st);
cudaError_t launch_validate(const SceneDev& S, uint32_t* status, cudaStream_t st);
cudaError_t launch_expand_counts(const SceneDev& S, const Workspace& ws, uint32_t* counts, cudaStream_t st);

__host__ __device__ inline int n_tiles(const SceneDev& S) { return S.tiles_x * S.tiles_y; }

// Host checks of a scene descriptor shared by every entry point that takes one (targets are
// required unless need_targets is false); returns an SGE_ code and leaves the message for
// sge_last_error.
int check_desc(const sge_scene_desc* d, bool need_targets);
// Device view of a checked descriptor (texture offsets, read textures, texel groups, tiles).
void make_dev(const sge_scene_desc* d, SceneDev& S);

// The calling thread's message for sge_last_error (host).
void set_last_error(const char* msg);

}  // namespace sge
