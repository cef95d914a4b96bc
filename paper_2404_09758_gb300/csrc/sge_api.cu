// The C ABI of include/sge.h: argument checks, workspace layout and launches.
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "sge_device.cuh"

using namespace sge;

struct sge_scene {
  sge_scene_desc desc;
  sge_config cfg;
  SceneDev dev;
  Workspace ws;
  int grid_fast, grid_heavy;  // persistent CTAs of the two estimator kernels
  AssetDesc* desc_dev;        // the scene's AssetDesc in its workspace (batched calls)
  bool desc_dirty;            // desc_dev must be rewritten before the next batched call
  // kernel timing (sge_kernel_timing): event pairs around the fast kernel's launches
  static constexpr int kMaxTimed = 256;
  cudaEvent_t tev[4 * kMaxTimed];  // per timed call: before/after the fast kernel, after the heavy one
  int n_tev;                  // event pairs created (0 = timing off)
  // a second stream for the work of an estimate call that does not depend on the binning (the
  // vertex pass and the texel sign planes of its first block of pairs), forked from and joined
  // back to the caller's stream with events (graph capture follows the fork)
  cudaStream_t side;
  cudaEvent_t fork, join;
  CheckDev chk_true;  // the checked build's true bounds (sge_check_limit lowers dev.chk)
  int n_timed;                // pairs recorded since the last sge_kernel_time
};

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SGE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

namespace sge {
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace sge

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t tri_rect, tri_margin, tri_z, pverts, vbits, tile_count, tile_off, tile_cur, bins, items, counters, keys, uvbuf, dfbuf,
      desc, tile_live, cand, ncand, tsign, kcount, total;
  int max_views, max_pairs;
  long long bin_capacity;
  long long sgn_words;
  int sgn_off[SGE_MAX_TEXTURES];
  long long n_kcount;
  long long kc_off[SGE_MAX_TEXTURES];
};

int tiles_of(int n) { return (n + TILE - 1) / TILE; }

}  // namespace

namespace sge {

int check_desc(const sge_scene_desc* d, bool need_targets) {
  if (!d) return fail(SGE_ERR_INVALID_ARG, "desc is NULL");
  if (!d->positions || !d->pos_idx || !d->uvs || !d->uv_idx || !d->mvp)
    return fail(SGE_ERR_INVALID_ARG, "positions, pos_idx, uvs, uv_idx and mvp must be non-NULL");
  if (need_targets && !d->targets) return fail(SGE_ERR_INVALID_ARG, "targets must be non-NULL");
  if (d->n_vertices < 3 || d->n_vertices >= (1 << 28)) return fail(SGE_ERR_INVALID_ARG, "n_vertices %d out of [3, 2^28)", d->n_vertices);
  if (d->n_triangles < 1) return fail(SGE_ERR_INVALID_ARG, "n_triangles must be >= 1");
  if (d->n_uvs < 1) return fail(SGE_ERR_INVALID_ARG, "n_uvs must be >= 1");
  if (d->n_views < 1) return fail(SGE_ERR_INVALID_ARG, "n_views must be >= 1");
  if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384)
    return fail(SGE_ERR_INVALID_ARG, "render size %dx%d out of [1, 16384]", d->width, d->height);
  if (!(d->eps_pos >= 0.0f) || !std::isfinite(d->eps_pos)) return fail(SGE_ERR_INVALID_ARG, "eps_pos must be finite and >= 0");
  if (!(d->near_w > 0.0f)) return fail(SGE_ERR_INVALID_ARG, "near_w must be > 0");
  if (d->shading < SGE_SHADE_UNLIT || d->shading > SGE_SHADE_TRANSPARENT)
    return fail(SGE_ERR_INVALID_ARG, "bad shading %d", d->shading);
  if (d->shading == SGE_SHADE_GGX && !d->cam_pos) return fail(SGE_ERR_INVALID_ARG, "GGX shading needs cam_pos");
  if (d->n_textures < 0 || d->n_textures > SGE_MAX_TEXTURES) return fail(SGE_ERR_INVALID_ARG, "n_textures %d out of [0, %d]", d->n_textures, SGE_MAX_TEXTURES);
  for (int k = 0; k < d->n_textures; ++k) {
    const sge_texture& t = d->textures[k];
    if (!t.texels) return fail(SGE_ERR_INVALID_ARG, "texture %d has NULL texels", k);
    if (t.width < 1 || t.height < 1 || (long long)t.width * t.height >= (1ll << 28))
      return fail(SGE_ERR_INVALID_ARG, "texture %d size %dx%d out of range", k, t.width, t.height);
    if (t.channels < 1 || t.channels > 4) return fail(SGE_ERR_INVALID_ARG, "texture %d channels %d not in 1..4", k, t.channels);
    if (t.role < SGE_ROLE_ALBEDO || t.role > SGE_ROLE_METALLIC) return fail(SGE_ERR_INVALID_ARG, "texture %d bad role", k);
    if (!(t.eps >= 0.0f) || !std::isfinite(t.eps)) return fail(SGE_ERR_INVALID_ARG, "texture %d eps must be finite and >= 0", k);
  }
  // the shading model samples one texture of each role it reads: all must be present
  const int need = (d->shading == SGE_SHADE_UNLIT || d->shading == SGE_SHADE_TRANSPARENT)
                       ? 1
                       : (d->shading == SGE_SHADE_LAMBERT ? 2 : 4);
  static const int roles[4] = {SGE_ROLE_ALBEDO, SGE_ROLE_NORMAL, SGE_ROLE_ROUGHNESS, SGE_ROLE_METALLIC};
  static const char* names[4] = {"albedo", "normal", "roughness", "metallic"};
  for (int r = 0; r < need; ++r) {
    bool found = false;
    for (int k = 0; k < d->n_textures; ++k) found = found || d->textures[k].role == roles[r];
    if (!found) return fail(SGE_ERR_INVALID_ARG, "shading model %d needs a texture of role %s", d->shading, names[r]);
  }
  if (d->shading == SGE_SHADE_TRANSPARENT) {
    for (int k = 0; k < d->n_textures; ++k)
      if (d->textures[k].role == SGE_ROLE_ALBEDO) {  // the first albedo is the one read
        if (d->textures[k].channels != 4)
          return fail(SGE_ERR_INVALID_ARG, "transparent shading needs an RGBA (4-channel) albedo, texture %d has %d",
                      k, d->textures[k].channels);
        break;
      }
  }
  return SGE_OK;
}

}  // namespace sge

namespace {

int unsupported_transparent(const char* call) {
  return fail(SGE_ERR_UNSUPPORTED, "%s: transparent scenes run through sge_estimate_grad, sge_loss and "
              "sge_render_deep", call);
}

int make_layout(const sge_scene_desc* d, const sge_config* c, Layout& L) {
  if (c && c->footprint != SGE_FOOT_BILINEAR && c->footprint != SGE_FOOT_NEAREST)
    return fail(SGE_ERR_INVALID_ARG, "footprint %d is neither SGE_FOOT_BILINEAR nor SGE_FOOT_NEAREST", c->footprint);
  L.max_views = (c && c->max_views_per_call > 0) ? c->max_views_per_call : d->n_views;
  if (L.max_views > SGE_MAX_VIEWS_PER_CALL) L.max_views = SGE_MAX_VIEWS_PER_CALL;
  const long long ntl = (long long)tiles_of(d->width) * tiles_of(d->height);
  L.bin_capacity = (c && c->bin_capacity > 0) ? c->bin_capacity
                                               : (6ll * d->n_triangles + 8ll * ntl) * (long long)L.max_views;
  if (L.bin_capacity >= (1ll << 32)) return fail(SGE_ERR_INVALID_ARG, "bin_capacity must be < 2^32");
  const long long npx = (long long)d->width * d->height;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.tri_rect = take(sizeof(int4) * (size_t)L.max_views * d->n_triangles);
  L.tri_margin = take(sizeof(int) * (size_t)L.max_views * d->n_triangles);
  L.tri_z = take(sizeof(float2) * (size_t)L.max_views * d->n_triangles);
  L.max_pairs = (c && c->max_pairs_per_call > 0) ? c->max_pairs_per_call : 64;
  L.pverts = take(sizeof(int4) * 2 * (size_t)L.max_views * L.max_pairs * d->n_vertices);
  L.vbits = take((size_t)L.max_views * L.max_pairs * d->n_vertices);
  L.tile_count = take(sizeof(uint32_t) * (size_t)(L.max_views * ntl));
  L.tile_off = take(sizeof(uint32_t) * (size_t)(L.max_views * ntl + 1));
  L.tile_cur = take(sizeof(uint32_t) * (size_t)(L.max_views * ntl));
  L.bins = take(sizeof(uint32_t) * (size_t)L.bin_capacity);
  L.items = take(sizeof(uint32_t) * (size_t)(L.max_views * ntl));
  L.counters = take(64);
  L.keys = take(sizeof(unsigned long long) * 2 * (size_t)npx);
  L.uvbuf = take(sizeof(float2) * 2 * (size_t)npx);
  L.dfbuf = take(sizeof(float) * (size_t)npx);
  L.desc = take(sizeof(AssetDesc));
  L.tile_live = take(sizeof(uint32_t) * (size_t)(L.max_views * ntl));
  L.cand = take(sizeof(int4) * (size_t)(L.max_views * ntl) * kCandWords * TILE_PX);
  L.ncand = take((size_t)(L.max_views * ntl) * TILE_PX);
  // texel sign planes of every estimate of a block of pairs: 4 bits per texel of each texture the
  // shading model reads
  SceneDev S;
  make_dev(d, S);
  L.sgn_words = 0;
  for (int k = 0; k < SGE_MAX_TEXTURES; ++k) L.sgn_off[k] = -1;
  for (int r = 0; r < S.nread; ++r) {
    L.sgn_off[S.read_k[r]] = (int)L.sgn_words;
    L.sgn_words += ((long long)S.rtex[r].w * S.rtex[r].h + 7) / 8;
  }
  L.tsign = take(sizeof(uint32_t) * (size_t)L.max_views * L.max_pairs * (size_t)L.sgn_words);
  // transparent scenes: one contribution count per key (welded vertex, texel of a read texture)
  L.n_kcount = 0;
  for (int k = 0; k < SGE_MAX_TEXTURES; ++k) L.kc_off[k] = -1;
  if (d->shading == SGE_SHADE_TRANSPARENT) {
    L.n_kcount = d->n_vertices;
    for (int r = 0; r < S.nread; ++r) {
      L.kc_off[S.read_k[r]] = L.n_kcount;
      L.n_kcount += (long long)S.rtex[r].w * S.rtex[r].h;
    }
  }
  L.kcount = take(sizeof(uint32_t) * (size_t)L.n_kcount);
  L.total = o;
  return SGE_OK;
}

}  // namespace

namespace sge {

void make_dev(const sge_scene_desc* d, SceneDev& S) {
  memset(&S, 0, sizeof(S));
  S.pos = d->positions;
  S.nv = d->n_vertices;
  S.eps_pos = d->eps_pos;
  S.pidx = d->pos_idx;
  S.nt = d->n_triangles;
  S.uvs = d->uvs;
  S.uvidx = d->uv_idx;
  S.nuv = d->n_uvs;
  S.ntex = d->n_textures;
  long long off = 3ll * d->n_vertices;
  int first_of_role[4] = {-1, -1, -1, -1};
  for (int k = 0; k < d->n_textures; ++k) {
    const sge_texture& t = d->textures[k];
    TexDev& T = S.tex[k];
    T.ptr = t.texels;
    T.w = t.width;
    T.h = t.height;
    T.c = t.channels;
    T.eps = t.eps;
    T.role = t.role;
    T.offset = off;
    T.index = k;
    off += (long long)t.width * t.height * t.channels;
    if (first_of_role[t.role] < 0) first_of_role[t.role] = k;
  }
  S.n_params = off;
  for (int k = 0; k < d->n_textures; ++k) {
    const int role = d->textures[k].role;
    bool read = first_of_role[role] == k &&
                (d->shading == SGE_SHADE_GGX || role == SGE_ROLE_ALBEDO ||
                 (d->shading == SGE_SHADE_LAMBERT && role == SGE_ROLE_NORMAL));
    S.tex[k].read = read;
    if (read) S.read_k[S.nread++] = k;
  }
  for (int r = 0; r < S.nread; ++r) S.rtex[r] = S.tex[S.read_k[r]];
  S.grouped = S.nread > 1;
  for (int r = 1; r < S.nread; ++r)
    if (S.rtex[r].w != S.rtex[0].w || S.rtex[r].h != S.rtex[0].h) S.grouped = 0;
  S.mvp = d->mvp;
  S.cam_pos = d->cam_pos;
  S.nviews = d->n_views;
  S.W = d->width;
  S.H = d->height;
  S.near_w = d->near_w;
  S.targets = d->targets;
  for (int c = 0; c < 3; ++c) {
    S.bg[c] = d->background[c];
    S.light_dir[c] = d->light_dir[c];
    S.light_rgb[c] = d->light_rgb[c];
  }
  S.shading = d->shading;
  S.ambient = d->ambient;
  S.tiles_x = tiles_of(d->width);
  S.tiles_y = tiles_of(d->height);
  // the checked build's bounds: the true sizes (the workspace's own are set where it is carved)
  S.chk.nv = d->n_vertices;
  S.chk.nuv = d->n_uvs;
  S.chk.params = S.n_params;
}

}  // namespace sge

namespace {

// The binning arms the estimator kernels' work counters; every further block of pairs of the
// same call re-arms them.
cudaError_t rearm_work(const Workspace& ws, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws.counters + 1, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.counters + 5, 0, sizeof(uint32_t), st);
  return e;
}

int views_of(const sge_scene* s, const int32_t* view_ids, int32_t n, ViewList& vl) {
  if (!view_ids) return fail(SGE_ERR_INVALID_ARG, "view_ids is NULL");
  if (n < 1 || n > s->ws.max_views)
    return fail(SGE_ERR_INVALID_ARG, "n_views %d out of [1, %d] (max_views_per_call)", n, s->ws.max_views);
  vl.n = n;
  for (int i = 0; i < n; ++i) {
    if (view_ids[i] < 0 || view_ids[i] >= s->desc.n_views)
      return fail(SGE_ERR_INVALID_ARG, "view_ids[%d] = %d out of [0, %d)", i, view_ids[i], s->desc.n_views);
    for (int j = 0; j < i; ++j)
      if (view_ids[j] == view_ids[i]) return fail(SGE_ERR_INVALID_ARG, "view %d listed twice", view_ids[i]);
    vl.id[i] = view_ids[i];
  }
  return SGE_OK;
}

}  // namespace

extern "C" {

const char* sge_last_error(void) { return g_err; }

int sge_workspace_size(const sge_scene_desc* desc, const sge_config* cfg, size_t* bytes) {
  if (!bytes) return fail(SGE_ERR_INVALID_ARG, "bytes is NULL");
  int rc = check_desc(desc, true);
  if (rc) return rc;
  Layout L;
  rc = make_layout(desc, cfg, L);
  if (rc) return rc;
  *bytes = L.total;
  return SGE_OK;
}

int sge_create_scene(const sge_scene_desc* desc, const sge_config* cfg, void* workspace, size_t workspace_bytes,
                     sge_scene** out) {
  if (!out) return fail(SGE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = check_desc(desc, true);
  if (rc) return rc;
  Layout L;
  rc = make_layout(desc, cfg, L);
  if (rc) return rc;
  if (!workspace) return fail(SGE_ERR_WORKSPACE, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(SGE_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(SGE_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
  sge_scene* s = new (std::nothrow) sge_scene;
  if (!s) return fail(SGE_ERR_INVALID_ARG, "out of host memory");
  s->desc = *desc;
  s->cfg = cfg ? *cfg : sge_config{};
  make_dev(desc, s->dev);
  s->dev.foot_nearest = s->cfg.footprint == SGE_FOOT_NEAREST;
  char* base = static_cast<char*>(workspace);
  Workspace& w = s->ws;
  w.tri_rect = reinterpret_cast<int4*>(base + L.tri_rect);
  w.tri_margin = reinterpret_cast<int*>(base + L.tri_margin);
  w.tri_z = reinterpret_cast<float2*>(base + L.tri_z);
  w.pverts = reinterpret_cast<int4*>(base + L.pverts);
  w.vbits = reinterpret_cast<uint8_t*>(base + L.vbits);
  w.max_pairs = L.max_pairs;
  w.tile_count = reinterpret_cast<uint32_t*>(base + L.tile_count);
  w.tile_off = reinterpret_cast<uint32_t*>(base + L.tile_off);
  w.tile_cur = reinterpret_cast<uint32_t*>(base + L.tile_cur);
  w.bins = reinterpret_cast<uint32_t*>(base + L.bins);
  w.items = reinterpret_cast<uint32_t*>(base + L.items);
  w.counters = reinterpret_cast<uint32_t*>(base + L.counters);
  w.tile_live = reinterpret_cast<uint32_t*>(base + L.tile_live);
  w.cand = reinterpret_cast<int4*>(base + L.cand);
  w.ncand = reinterpret_cast<uint8_t*>(base + L.ncand);
  w.keys = reinterpret_cast<unsigned long long*>(base + L.keys);
  w.uvbuf = reinterpret_cast<float2*>(base + L.uvbuf);
  w.dfbuf = reinterpret_cast<float*>(base + L.dfbuf);
  w.tsign = L.sgn_words > 0 ? reinterpret_cast<uint32_t*>(base + L.tsign) : nullptr;
  w.sgn_words = L.sgn_words;
  w.kcount = L.n_kcount > 0 ? reinterpret_cast<uint32_t*>(base + L.kcount) : nullptr;
  w.n_kcount = L.n_kcount;
  for (int k = 0; k < SGE_MAX_TEXTURES; ++k) w.kc_off[k] = L.kc_off[k];
  for (int k = 0; k < SGE_MAX_TEXTURES; ++k) w.sgn_off[k] = L.sgn_off[k];
  w.bin_capacity = L.bin_capacity;
  w.max_views = L.max_views;
  w.light_bin = kLightBin;
  s->dev.chk.status = w.counters + 3;
  s->dev.chk.where = w.counters + 8;
  s->dev.chk.bins = w.bin_capacity;
  s->dev.chk.sign_words = w.sgn_words;
  s->chk_true = s->dev.chk;
  s->desc_dev = reinterpret_cast<AssetDesc*>(base + L.desc);
  s->desc_dirty = true;
  s->n_tev = 0;
  s->n_timed = 0;
  s->side = nullptr;
  s->fork = s->join = nullptr;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemset(w.counters, 0, 64);
  if (e == cudaSuccess && w.kcount) e = cudaMemset(w.kcount, 0, sizeof(uint32_t) * (size_t)w.n_kcount);
  if (e != cudaSuccess) {
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->join) cudaEventDestroy(s->join);
    delete s;
    return cuda_fail(e, "sge_create_scene");
  }
  int bps = (s->cfg.blocks_per_sm > 0) ? s->cfg.blocks_per_sm : fast_blocks_per_sm(desc->shading, s->dev.grouped);
  s->grid_fast = sms * bps;
  s->grid_heavy = sms * estimate_blocks_per_sm(desc->shading, s->dev.grouped, group_channels(s->dev));
  if (s->cfg.pairs_per_item <= 0) s->cfg.pairs_per_item = 8;
  if (s->cfg.pairs_per_item > kMaxPairsPerItem) s->cfg.pairs_per_item = kMaxPairsPerItem;
  *out = s;
  return SGE_OK;
}

int sge_num_params(const sge_scene* s, int64_t* d) {
  if (!s || !d) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  *d = s->dev.n_params;
  return SGE_OK;
}

int sge_set_targets(sge_scene* s, const float* targets) {
  if (!s || !targets) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  s->desc.targets = targets;
  s->dev.targets = targets;
  s->desc_dirty = true;
  return SGE_OK;
}

int sge_validate(sge_scene* s, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  cudaError_t e = launch_validate(s->dev, s->ws.counters + 3, (cudaStream_t)stream);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_validate");
}

int sge_render_idb(sge_scene* s, int32_t view, uint64_t seed, uint32_t iter, uint32_t pair, int32_t side,
                   uint64_t* depth_id, float* uv, float* rgb, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (side < -1 || side > 1) return fail(SGE_ERR_INVALID_ARG, "side %d not in {-1, 0, 1}", side);
  if (s->dev.shading == SHADE_TRANSPARENT) return unsupported_transparent("sge_render_idb");
  ViewList vl;
  int rc = views_of(s, &view, 1, vl);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_binning(s->dev, s->ws, vl, st);
  if (e == cudaSuccess)
    e = launch_render(s->dev, s->ws, 0, view, pair_key(seed, iter, (uint32_t)view, pair), side,
                      reinterpret_cast<unsigned long long*>(depth_id), reinterpret_cast<float2*>(uv), rgb, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_render_idb");
}

int sge_render_deep(sge_scene* s, int32_t view, uint64_t seed, uint32_t iter, uint32_t pair, int32_t side,
                    uint64_t* deep_ids, float* rgb, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (side < -1 || side > 1) return fail(SGE_ERR_INVALID_ARG, "side %d not in {-1, 0, 1}", side);
  if (s->dev.shading != SHADE_TRANSPARENT)
    return fail(SGE_ERR_UNSUPPORTED, "sge_render_deep: the scene is not transparent (shading %d)", s->dev.shading);
  ViewList vl;
  int rc = views_of(s, &view, 1, vl);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_binning(s->dev, s->ws, vl, st);  // no pruning: hidden fragments are listed
  if (e == cudaSuccess)
    e = launch_render_deep(s->dev, s->ws, 0, view, pair_key(seed, iter, (uint32_t)view, pair), side,
                           reinterpret_cast<unsigned long long*>(deep_ids), rgb, nullptr, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_render_deep");
}

}  // extern "C"

namespace {

// Every estimate of one call (sge_estimate_grad and its device-state form): iter_dev, when
// non-NULL, is the device word the kernels read the iteration index from.
int estimate_grad(sge_scene* s, uint64_t seed, uint32_t iter, const uint32_t* iter_dev, const int32_t* view_ids,
                  int32_t n_views, int32_t pairs_per_view, float* grad_sums, uint32_t* counts, float* loss_out,
                  float* delta_f_out, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (!grad_sums || !counts) return fail(SGE_ERR_INVALID_ARG, "grad_sums and counts must be non-NULL");
  if (pairs_per_view < 1) return fail(SGE_ERR_INVALID_ARG, "pairs_per_view must be >= 1");
  ViewList vl;
  int rc = views_of(s, view_ids, n_views, vl);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  EstimateArgs a{seed, iter, pairs_per_view, s->cfg.pairs_per_item, 0, pairs_per_view, grad_sums, counts, loss_out,
                 delta_f_out, iter_dev};
  cudaError_t e = cudaSuccess;
  if (delta_f_out)
    e = cudaMemsetAsync(delta_f_out, 0, sizeof(float) * (size_t)n_views * pairs_per_view * s->dev.W * s->dev.H, st);
  if (s->dev.shading == SHADE_TRANSPARENT) {
    // deep lists need every binned triangle (no pruning); per block of pairs the vertex pass
    // (projected vertices, sign bits, texel sign planes) and one launch over its estimates
    if (e == cudaSuccess) e = launch_binning(s->dev, s->ws, vl, st);
    for (int p0 = 0; p0 < pairs_per_view && e == cudaSuccess; p0 += s->ws.max_pairs) {
      EstimateArgs b = a;
      b.pair_begin = p0;
      b.pair_count = pairs_per_view - p0 < s->ws.max_pairs ? pairs_per_view - p0 : s->ws.max_pairs;
      e = launch_vertex_pass(s->dev, s->ws, vl, b, st);
      if (e == cudaSuccess) e = launch_deep_estimate(s->dev, s->ws, vl, b, st);
    }
    if (e == cudaSuccess) e = launch_expand_counts(s->dev, s->ws, counts, st);
    return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_estimate_grad");
  }
  // pairs run in blocks of at most max_pairs_per_call (the projected-vertex buffer holds one
  // block); the first block's vertex pass and sign planes run on the side stream while the caller's
  // stream bins and prunes
  EstimateArgs b0 = a;
  b0.pair_count = pairs_per_view < s->ws.max_pairs ? pairs_per_view : s->ws.max_pairs;
  if (e == cudaSuccess) e = cudaEventRecord(s->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->fork, 0);
  if (e == cudaSuccess) e = launch_vertex_pass(s->dev, s->ws, vl, b0, s->side);
  if (e == cudaSuccess) e = cudaEventRecord(s->join, s->side);
  if (e == cudaSuccess) e = launch_binning(s->dev, s->ws, vl, st, true);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->join, 0);
  for (int p0 = 0; p0 < pairs_per_view && e == cudaSuccess; p0 += s->ws.max_pairs) {
    EstimateArgs b = a;
    b.pair_begin = p0;
    b.pair_count = pairs_per_view - p0 < s->ws.max_pairs ? pairs_per_view - p0 : s->ws.max_pairs;
    if (p0 > 0) e = rearm_work(s->ws, st);
    if (e == cudaSuccess && p0 > 0) e = launch_vertex_pass(s->dev, s->ws, vl, b, st);
    const cudaEvent_t* ev = nullptr;
    if (s->n_tev && s->n_timed < sge_scene::kMaxTimed) ev = s->tev + 4 * s->n_timed++;
    if (e == cudaSuccess) e = launch_estimate(s->dev, s->ws, vl, b, s->grid_fast, s->grid_heavy, st, ev);
  }
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_estimate_grad");
}

// Descent step (sge_step and its device-state form; t_dev: Adam's step number read at run time).
int step(sge_scene* s, const sge_opt* o, const int32_t* t_dev, float* grad_sums, uint32_t* counts,
         int64_t n_pairs_total, float* adam_m, float* adam_v, sge_stream_t stream) {
  if (!s || !o) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  if (!grad_sums || !counts) return fail(SGE_ERR_INVALID_ARG, "grad_sums and counts must be non-NULL");
  if (o->kind < SGE_STEP_SGD || o->kind > SGE_STEP_SGD_MEAN) return fail(SGE_ERR_INVALID_ARG, "bad step kind %d", o->kind);
  if (o->kind != SGE_STEP_SGD_MEAN && n_pairs_total < 1) return fail(SGE_ERR_INVALID_ARG, "n_pairs_total must be >= 1");
  if (o->kind == SGE_STEP_ADAM) {
    if (!adam_m || !adam_v) return fail(SGE_ERR_INVALID_ARG, "Adam needs m and v");
    if (!t_dev && o->t < 1) return fail(SGE_ERR_INVALID_ARG, "Adam step t must be >= 1");
  }
  if (s->desc.eps_pos <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "eps_pos must be > 0 to form Eq. 9's estimate");
  for (int k = 0; k < s->dev.ntex; ++k)
    if (s->dev.tex[k].eps <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "texture %d eps must be > 0 to step", k);
  cudaError_t e = launch_step(s->dev, *o, grad_sums, counts, n_pairs_total > 0 ? n_pairs_total : 1, adam_m, adam_v,
                              (cudaStream_t)stream, t_dev);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_step");
}

bool aligned4(const void* p) { return ((uintptr_t)p & 3) == 0; }
static_assert(offsetof(sge_iter_state, iter) == 0 && offsetof(sge_iter_state, t) == 4,
              "k_iter_advance reads the state as two 32-bit words");

}  // namespace

extern "C" {

int sge_estimate_grad(sge_scene* s, uint64_t seed, uint32_t iter, const int32_t* view_ids, int32_t n_views,
                      int32_t pairs_per_view, float* grad_sums, uint32_t* counts, float* loss_out, float* delta_f_out,
                      sge_stream_t stream) {
  return estimate_grad(s, seed, iter, nullptr, view_ids, n_views, pairs_per_view, grad_sums, counts, loss_out,
                       delta_f_out, stream);
}

int sge_estimate_grad_state(sge_scene* s, uint64_t seed, const sge_iter_state* state, const int32_t* view_ids,
                            int32_t n_views, int32_t pairs_per_view, float* grad_sums, uint32_t* counts,
                            float* loss_out, float* delta_f_out, sge_stream_t stream) {
  if (!state || !aligned4(state)) return fail(SGE_ERR_INVALID_ARG, "state must be a 4-byte aligned device pointer");
  return estimate_grad(s, seed, 0, &state->iter, view_ids, n_views, pairs_per_view, grad_sums, counts, loss_out,
                       delta_f_out, stream);
}

int sge_step_state(sge_scene* s, const sge_opt* o, const sge_iter_state* state, float* grad_sums, uint32_t* counts,
                   int64_t n_pairs_total, float* adam_m, float* adam_v, sge_stream_t stream) {
  if (!state || !aligned4(state)) return fail(SGE_ERR_INVALID_ARG, "state must be a 4-byte aligned device pointer");
  return step(s, o, &state->t, grad_sums, counts, n_pairs_total, adam_m, adam_v, stream);
}

int sge_iter_advance(sge_iter_state* state, int32_t d_iter, int32_t d_t, sge_stream_t stream) {
  if (!state || !aligned4(state)) return fail(SGE_ERR_INVALID_ARG, "state must be a 4-byte aligned device pointer");
  cudaError_t e = launch_iter_advance(&state->iter, d_iter, d_t, (cudaStream_t)stream);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_iter_advance");
}

int sge_iterate_host(sge_scene* s, uint64_t seed, sge_iter_state* state, const int32_t* view_ids, int32_t n_views,
                     int32_t pairs_per_view, const sge_opt* opt, float* grad_sums, uint32_t* counts, float* adam_m,
                     float* adam_v, float* loss_dev, const sge_host_io* io, sge_stream_t stream) {
  if (!s || !io || !opt) return fail(SGE_ERR_INVALID_ARG, "scene, io and opt must be non-NULL");
  if (!state || !aligned4(state)) return fail(SGE_ERR_INVALID_ARG, "state must be a 4-byte aligned device pointer");
  if (pairs_per_view < 1) return fail(SGE_ERR_INVALID_ARG, "pairs_per_view must be >= 1");
  if (io->loss_out && !loss_dev) return fail(SGE_ERR_INVALID_ARG, "io->loss_out needs loss_dev");
  // the step's argument checks too, so that a call it would refuse enqueues nothing
  if (!grad_sums || !counts) return fail(SGE_ERR_INVALID_ARG, "grad_sums and counts must be non-NULL");
  if (opt->kind < SGE_STEP_SGD || opt->kind > SGE_STEP_SGD_MEAN)
    return fail(SGE_ERR_INVALID_ARG, "bad step kind %d", opt->kind);
  if (opt->kind == SGE_STEP_ADAM && (!adam_m || !adam_v)) return fail(SGE_ERR_INVALID_ARG, "Adam needs m and v");
  ViewList vl;
  int rc = views_of(s, view_ids, n_views, vl);
  if (rc) return rc;
  if (s->desc.eps_pos <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "eps_pos must be > 0 to form Eq. 9's estimate");
  for (int k = 0; k < s->dev.ntex; ++k)
    if (s->dev.tex[k].eps <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "texture %d eps must be > 0 to step", k);
  cudaStream_t st = (cudaStream_t)stream;
  // the parameter groups in gradient order: positions, then each texture
  const sge_scene_desc& d = s->desc;
  float* group[1 + SGE_MAX_TEXTURES];
  size_t count[1 + SGE_MAX_TEXTURES];
  int ng = 0;
  group[ng] = d.positions, count[ng++] = 3 * (size_t)d.n_vertices;
  for (int k = 0; k < d.n_textures; ++k)
    group[ng] = d.textures[k].texels,
    count[ng++] = (size_t)d.textures[k].width * d.textures[k].height * d.textures[k].channels;
  auto copy_theta = [&](float* dst_host, const float* src_host) {
    size_t off = 0;
    for (int k = 0; k < ng; ++k) {
      const size_t bytes = sizeof(float) * count[k];
      cudaError_t e = src_host ? cudaMemcpyAsync(group[k], src_host + off, bytes, cudaMemcpyHostToDevice, st)
                               : cudaMemcpyAsync(dst_host + off, group[k], bytes, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
      off += count[k];
    }
    return cudaSuccess;
  };
  cudaError_t e = io->theta_in ? copy_theta(nullptr, io->theta_in) : cudaSuccess;
  if (e == cudaSuccess && io->targets_in)
    e = cudaMemcpyAsync(const_cast<float*>(s->dev.targets), io->targets_in,
                        sizeof(float) * 3 * (size_t)d.n_views * d.width * d.height, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && loss_dev) e = cudaMemsetAsync(loss_dev, 0, sizeof(float) * (size_t)n_views, st);
  if (e != cudaSuccess) return cuda_fail(e, "sge_iterate_host (copies in)");
  rc = estimate_grad(s, seed, 0, &state->iter, view_ids, n_views, pairs_per_view, grad_sums, counts, loss_dev, nullptr,
                     stream);
  if (rc) return rc;
  rc = step(s, opt, &state->t, grad_sums, counts, (int64_t)n_views * pairs_per_view, adam_m, adam_v, stream);
  if (rc) return rc;
  e = launch_iter_advance(&state->iter, 1, 1, st);
  if (e == cudaSuccess && io->theta_out) e = copy_theta(io->theta_out, nullptr);
  if (e == cudaSuccess && io->loss_out)
    e = cudaMemcpyAsync(io->loss_out, loss_dev, sizeof(float) * (size_t)n_views, cudaMemcpyDeviceToHost, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_iterate_host (copies out)");
}

int sge_estimate_grad_plain(sge_scene* s, uint64_t seed, uint32_t iter, const int32_t* view_ids, int32_t n_views,
                            int32_t pairs_per_view, float* grad_sums, uint32_t* counts, float* loss_out,
                            sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (!grad_sums || !counts) return fail(SGE_ERR_INVALID_ARG, "grad_sums and counts must be non-NULL");
  if (pairs_per_view < 1) return fail(SGE_ERR_INVALID_ARG, "pairs_per_view must be >= 1");
  ViewList vl;
  int rc = views_of(s, view_ids, n_views, vl);
  if (rc) return rc;
  if (s->dev.shading == SHADE_TRANSPARENT) return unsupported_transparent("sge_estimate_grad_plain");
  cudaStream_t st = (cudaStream_t)stream;
  EstimateArgs a{seed, iter, pairs_per_view, 1, 0, pairs_per_view, grad_sums, counts, loss_out, nullptr};
  cudaError_t e = launch_binning(s->dev, s->ws, vl, st);
  for (int j = 0; j < n_views && e == cudaSuccess; ++j)
    for (int n = 0; n < pairs_per_view && e == cudaSuccess; ++n)
      e = launch_plain_pair(s->dev, s->ws, j, vl.id[j], pair_key(seed, iter, (uint32_t)vl.id[j], (uint32_t)n), a,
                            1.0f / (float)pairs_per_view, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_estimate_grad_plain");
}

int sge_estimate_grad_full_image(sge_scene* s, uint64_t seed, uint32_t iter, const int32_t* view_ids,
                                 int32_t n_views, int32_t pairs_per_view, float* grad_sums, uint32_t* counts,
                                 float* image_df, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (!grad_sums || !counts || !image_df) return fail(SGE_ERR_INVALID_ARG, "grad_sums, counts and image_df must be non-NULL");
  if (pairs_per_view < 1) return fail(SGE_ERR_INVALID_ARG, "pairs_per_view must be >= 1");
  ViewList vl;
  int rc = views_of(s, view_ids, n_views, vl);
  if (rc) return rc;
  if ((long long)n_views * pairs_per_view > 4096)
    return fail(SGE_ERR_INVALID_ARG, "n_views * pairs_per_view = %lld above 4096", (long long)n_views * pairs_per_view);
  if (s->dev.shading == SHADE_TRANSPARENT) return unsupported_transparent("sge_estimate_grad_full_image");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(image_df, 0, sizeof(float) * (size_t)n_views * pairs_per_view, st);
  if (e == cudaSuccess) e = launch_binning(s->dev, s->ws, vl, st);
  for (int j = 0; j < n_views && e == cudaSuccess; ++j)
    for (int n = 0; n < pairs_per_view && e == cudaSuccess; ++n)
      e = launch_image_delta(s->dev, s->ws, j, vl.id[j], pair_key(seed, iter, (uint32_t)vl.id[j], (uint32_t)n),
                             image_df + (size_t)j * pairs_per_view + n, st);
  if (e == cudaSuccess)
    e = launch_full_image_grad(s->dev, vl, pairs_per_view, seed, iter, image_df, grad_sums, counts, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_estimate_grad_full_image");
}

int sge_refine(const int32_t* row_ptr, const int32_t* col, const float* w, int32_t n_rows, const float* x, float* y,
               int32_t accumulate, sge_stream_t stream) {
  if (!row_ptr || !y || (n_rows > 0 && (!col || !w || !x))) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  if (n_rows < 0) return fail(SGE_ERR_INVALID_ARG, "n_rows must be >= 0");
  cudaError_t e = launch_csr_vec3(row_ptr, col, w, n_rows, x, y, accumulate ? 1 : 0, (cudaStream_t)stream);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_refine");
}

int sge_step(sge_scene* s, const sge_opt* o, float* grad_sums, uint32_t* counts, int64_t n_pairs_total, float* adam_m,
             float* adam_v, sge_stream_t stream) {
  return step(s, o, nullptr, grad_sums, counts, n_pairs_total, adam_m, adam_v, stream);
}

int sge_loss(sge_scene* s, const int32_t* view_ids, int32_t n_views, float* loss_out, sge_stream_t stream) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (!loss_out) return fail(SGE_ERR_INVALID_ARG, "loss_out must be non-NULL");
  ViewList vl;
  int rc = views_of(s, view_ids, n_views, vl);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_binning(s->dev, s->ws, vl, st);
  for (int j = 0; j < n_views && e == cudaSuccess; ++j)
    e = s->dev.shading == SHADE_TRANSPARENT
            ? launch_render_deep(s->dev, s->ws, j, vl.id[j], 0, 0, nullptr, nullptr, loss_out, st)
            : launch_render_loss(s->dev, s->ws, j, vl.id[j], loss_out, st);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_loss");
}

int sge_gradient(sge_scene* s, const float* grad_sums, int64_t n_pairs_total, const float* scale, float* out,
                 sge_stream_t stream) {
  if (!s || !grad_sums || !out) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  if (n_pairs_total < 1) return fail(SGE_ERR_INVALID_ARG, "n_pairs_total must be >= 1");
  if (s->desc.eps_pos <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "eps_pos must be > 0 to form Eq. 9's estimate");
  for (int k = 0; k < s->dev.ntex; ++k)
    if (s->dev.tex[k].eps <= 0.0f) return fail(SGE_ERR_INVALID_ARG, "texture %d eps must be > 0", k);
  cudaError_t e = launch_gradient(s->dev, grad_sums, n_pairs_total, scale, out, (cudaStream_t)stream);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_gradient");
}

}  // extern "C"

namespace {

// Every estimate of several scenes in one persistent launch per estimator kernel (the batched
// call and its device-state form; iter_dev as in estimate_grad).
int estimate_grad_batch(const sge_batch_entry* entries, int32_t n, uint64_t seed, uint32_t iter,
                        const uint32_t* iter_dev, int32_t pairs_per_view, const sge_batch_tuning* tuning,
                        sge_stream_t stream) {
  if (!entries) return fail(SGE_ERR_INVALID_ARG, "entries is NULL");
  if (n < 1 || n > SGE_MAX_BATCH) return fail(SGE_ERR_INVALID_ARG, "n_entries %d out of [1, %d]", n, SGE_MAX_BATCH);
  if (pairs_per_view < 1) return fail(SGE_ERR_INVALID_ARG, "pairs_per_view must be >= 1");
  sge_batch_tuning tu{};
  if (tuning) tu = *tuning;
  if (tu.pairs_per_item <= 0) tu.pairs_per_item = 8;
  if (tu.pairs_per_item > kMaxPairsPerItem) tu.pairs_per_item = kMaxPairsPerItem;
  if (tu.light_bin <= 0 || tu.light_bin > kLightBin) tu.light_bin = kLightBin;
  ViewList vls[SGE_MAX_BATCH];
  int max_pairs = 1 << 30;
  for (int i = 0; i < n; ++i) {
    const sge_batch_entry& E = entries[i];
    if (!E.scene) return fail(SGE_ERR_INVALID_ARG, "entries[%d].scene is NULL", i);
    if (E.scene->dev.shading == SHADE_TRANSPARENT) return unsupported_transparent("sge_estimate_grad_batch");
    if (!E.grad_sums || !E.counts) return fail(SGE_ERR_INVALID_ARG, "entries[%d]: grad_sums and counts must be non-NULL", i);
    if (E.n_views > SGE_MAX_BATCH_VIEWS)
      return fail(SGE_ERR_INVALID_ARG, "entries[%d].n_views %d above %d", i, E.n_views, SGE_MAX_BATCH_VIEWS);
    int rc = views_of(E.scene, E.view_ids, E.n_views, vls[i]);
    if (rc) return rc;
    for (int j = 0; j < i; ++j)
      if (entries[j].scene == E.scene) return fail(SGE_ERR_INVALID_ARG, "scene of entries[%d] listed twice", i);
    if (E.scene->ws.max_pairs < max_pairs) max_pairs = E.scene->ws.max_pairs;
  }
  // assets in decreasing triangle count: the long items first, the short ones balance the tail
  int order[SGE_MAX_BATCH];
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && entries[order[j]].scene->dev.nt > entries[order[j - 1]].scene->dev.nt; --j) {
      int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  int sms = 0, dev = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    sge_scene* s = entries[i].scene;
    if (s->desc_dirty) {
      AssetDesc d;
      memset(&d, 0, sizeof(d));
      d.S = s->dev;
      d.ws = s->ws;
      e = launch_put_desc(d, s->desc_dev, st);
      if (e == cudaSuccess) s->desc_dirty = false;
    }
    if (e == cudaSuccess) e = launch_binning(s->dev, s->ws, vls[i], st, true, true);
    if (e == cudaSuccess && entries[i].loss_out)
      e = launch_background_loss(s->dev, s->ws, vls[i], entries[i].loss_out, st);
  }
  // every asset's bins pruned and listed in one launch
  {
    BatchArgs Q;
    memset(&Q, 0, sizeof(Q));
    Q.light_bin = tu.light_bin;
    int max_tiles = 1, max_views = 1;
    for (int i = 0; i < n; ++i) {
      const sge_scene* s = entries[i].scene;
      BatchAsset& A = Q.as[Q.n++];
      A.desc = s->desc_dev;
      A.n_views = vls[i].n;
      for (int v = 0; v < vls[i].n; ++v) A.view[v] = vls[i].id[v];
      const int nt = s->dev.tiles_x * s->dev.tiles_y;
      if (nt > max_tiles) max_tiles = nt;
      if (vls[i].n > max_views) max_views = vls[i].n;
    }
    if (e == cudaSuccess) e = launch_prune_batch(Q, max_tiles, max_views, st);
  }
  // one persistent launch per kernel and shading model over every asset, per block of pairs
  for (int p0 = 0; p0 < pairs_per_view && e == cudaSuccess; p0 += max_pairs) {
    const int pc = pairs_per_view - p0 < max_pairs ? pairs_per_view - p0 : max_pairs;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      sge_scene* s = entries[i].scene;
      EstimateArgs b{seed, iter, pairs_per_view, tu.pairs_per_item, p0, pc, entries[i].grad_sums, entries[i].counts,
                     entries[i].loss_out, nullptr, iter_dev};
      if (p0 > 0) e = rearm_work(s->ws, st);
      if (e == cudaSuccess) e = launch_vertex_pass(s->dev, s->ws, vls[i], b, st);
    }
    for (int sh = SGE_SHADE_UNLIT; sh <= SGE_SHADE_GGX && e == cudaSuccess; ++sh) {
      BatchArgs P;
      memset(&P, 0, sizeof(P));
      P.seed = seed;
      P.iter = iter;
      P.iter_dev = iter_dev;
      P.pairs = pairs_per_view;
      P.pairs_per_item = tu.pairs_per_item;
      P.pair_begin = p0;
      P.pair_count = pc;
      P.light_bin = tu.light_bin;
      for (int k = 0; k < n; ++k) {
        const int i = order[k];
        sge_scene* s = entries[i].scene;
        if (s->dev.shading != sh) continue;
        BatchAsset& A = P.as[P.n++];
        A.desc = s->desc_dev;
        A.grad = entries[i].grad_sums;
        A.counts = entries[i].counts;
        A.loss = entries[i].loss_out;
        A.n_views = vls[i].n;
        for (int v = 0; v < vls[i].n; ++v) A.view[v] = vls[i].id[v];
      }
      if (P.n == 0) continue;
      const int bps = tu.blocks_per_sm > 0 ? tu.blocks_per_sm : fast_batch_blocks_per_sm(sh);
      e = launch_fast_batch(P, sh, sms * bps, st);
      if (e == cudaSuccess) e = launch_heavy_batch(P, sh, sms * heavy_batch_blocks_per_sm(sh), st);
    }
  }
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_estimate_grad_batch");
}

}  // namespace

extern "C" {

int sge_estimate_grad_batch(const sge_batch_entry* entries, int32_t n, uint64_t seed, uint32_t iter,
                            int32_t pairs_per_view, const sge_batch_tuning* tuning, sge_stream_t stream) {
  return estimate_grad_batch(entries, n, seed, iter, nullptr, pairs_per_view, tuning, stream);
}

int sge_estimate_grad_batch_state(const sge_batch_entry* entries, int32_t n, uint64_t seed,
                                  const sge_iter_state* state, int32_t pairs_per_view,
                                  const sge_batch_tuning* tuning, sge_stream_t stream) {
  if (!state || !aligned4(state)) return fail(SGE_ERR_INVALID_ARG, "state must be a 4-byte aligned device pointer");
  return estimate_grad_batch(entries, n, seed, 0, &state->iter, pairs_per_view, tuning, stream);
}

int sge_autotune_batch(const sge_batch_entry* entries, int32_t n, int32_t pairs_per_view, int32_t repeats,
                       sge_batch_tuning* out, float* best_ms, sge_stream_t stream) {
  if (!out) return fail(SGE_ERR_INVALID_ARG, "out is NULL");
  if (repeats < 1) repeats = 1;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "sge_autotune_batch");
  int rc = SGE_OK;
  // time one launch shape: one untimed call, then the mean of `repeats` calls
  auto time_of = [&](const sge_batch_tuning& t, float& ms) -> int {
    int r = sge_estimate_grad_batch(entries, n, 0x5eed, 0, pairs_per_view, &t, stream);
    if (r) return r;
    cudaError_t c = cudaEventRecord(ev[0], st);
    for (int k = 0; k < repeats && c == cudaSuccess; ++k) {
      r = sge_estimate_grad_batch(entries, n, 0x5eed, 1 + k, pairs_per_view, &t, stream);
      if (r) return r;
    }
    if (c == cudaSuccess) c = cudaEventRecord(ev[1], st);
    if (c == cudaSuccess) c = cudaEventSynchronize(ev[1]);
    if (c == cudaSuccess) c = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (c != cudaSuccess) return cuda_fail(c, "sge_autotune_batch");
    ms /= (float)repeats;
    return SGE_OK;
  };
  sge_batch_tuning best{8, 0, kLightBin};
  if (best.pairs_per_item > pairs_per_view) best.pairs_per_item = pairs_per_view;
  float best_t = 0.0f;
  rc = time_of(best, best_t);
  // coordinate search: pairs per item, then CTAs per SM, then the light-bin limit
  const int ppi[] = {1, 2, 4, 8, 16, 32, 64};
  for (int k = 0; k < 7 && !rc; ++k) {
    if (ppi[k] > pairs_per_view || ppi[k] == best.pairs_per_item) continue;
    sge_batch_tuning t = best;
    t.pairs_per_item = ppi[k];
    float ms = 0.0f;
    rc = time_of(t, ms);
    if (!rc && ms < best_t) best = t, best_t = ms;
  }
  for (int bps = 1; bps <= 2 && !rc; ++bps) {
    sge_batch_tuning t = best;
    t.blocks_per_sm = bps;
    float ms = 0.0f;
    rc = time_of(t, ms);
    if (!rc && ms < best_t) best = t, best_t = ms;
  }
  const int lb[] = {64, 128};
  for (int k = 0; k < 2 && !rc; ++k) {
    sge_batch_tuning t = best;
    t.light_bin = lb[k];
    float ms = 0.0f;
    rc = time_of(t, ms);
    if (!rc && ms < best_t) best = t, best_t = ms;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc) return rc;
  // the trials accumulated into the entries' buffers: leave them zeroed
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const sge_scene* s = entries[i].scene;
    e = cudaMemsetAsync(entries[i].grad_sums, 0, sizeof(float) * (size_t)s->dev.n_params, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(entries[i].counts, 0, sizeof(uint32_t) * (size_t)s->dev.n_params, st);
    if (e == cudaSuccess && entries[i].loss_out)
      e = cudaMemsetAsync(entries[i].loss_out, 0, sizeof(float) * (size_t)entries[i].n_views, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sge_autotune_batch");
  *out = best;
  if (best_ms) *best_ms = best_t;
  return SGE_OK;
}

int sge_status(sge_scene* s, sge_stream_t stream, int32_t* device_status) {
  if (!s || !device_status) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  uint32_t v = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&v, s->ws.counters + 3, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ws.counters + 3, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sge_status");
  *device_status = (int32_t)v;
  return SGE_OK;
}

int sge_kernel_timing(sge_scene* s, int32_t enable) {
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  if (enable && !s->n_tev) {
    for (int i = 0; i < 4 * sge_scene::kMaxTimed; ++i) {
      cudaError_t e = cudaEventCreate(&s->tev[i]);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(s->tev[j]);
        return cuda_fail(e, "sge_kernel_timing");
      }
    }
    s->n_tev = 4 * sge_scene::kMaxTimed;
  } else if (!enable && s->n_tev) {
    for (int i = 0; i < s->n_tev; ++i) cudaEventDestroy(s->tev[i]);
    s->n_tev = 0;
  }
  s->n_timed = 0;
  return SGE_OK;
}

int sge_kernel_time(sge_scene* s, float* total_ms, float* heavy_ms, int32_t* launches) {
  if (!s || !total_ms || !launches) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  float sum = 0.0f, hsum = 0.0f;
  for (int k = 0; k < s->n_timed; ++k) {
    float ms = 0.0f, hms = 0.0f;
    cudaError_t e = cudaEventSynchronize(s->tev[4 * k + 2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, s->tev[4 * k], s->tev[4 * k + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&hms, s->tev[4 * k + 1], s->tev[4 * k + 2]);
    if (e != cudaSuccess) return cuda_fail(e, "sge_kernel_time");
    sum += ms;
    hsum += hms;
  }
  *total_ms = sum;
  if (heavy_ms) *heavy_ms = hsum;
  *launches = s->n_timed;
  s->n_timed = 0;
  return SGE_OK;
}

int sge_bin_stats(sge_scene* s, sge_stream_t stream, int64_t* light_items, int64_t* heavy_items,
                  int64_t* bin_entries) {
  if (!s || !light_items || !heavy_items || !bin_entries) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  uint32_t c[6] = {0, 0, 0, 0, 0, 0};
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(c, s->ws.counters, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sge_bin_stats");
  *light_items = c[0];
  *heavy_items = c[4];
  *bin_entries = c[2];
  return SGE_OK;
}

int sge_draw_views(uint64_t seed, uint32_t iter, int32_t n_views, int32_t count, int32_t* out) {
  if (!out) return fail(SGE_ERR_INVALID_ARG, "out is NULL");
  if (n_views < 1 || count < 1 || count > n_views || count > SGE_MAX_VIEWS_PER_CALL)
    return fail(SGE_ERR_INVALID_ARG, "need 1 <= count <= n_views and count <= %d", SGE_MAX_VIEWS_PER_CALL);
  // the first `count` entries of a Fisher-Yates shuffle of 0..n_views-1 driven by the
  // generator outputs of the key (seed, iter, ~0, ~0), a key no estimate uses
  const uint64_t key = pair_key(seed, iter, 0xFFFFFFFFu, 0xFFFFFFFFu);
  int32_t perm[SGE_MAX_VIEWS_PER_CALL];
  const int32_t keep = count;
  // a partial shuffle only touches the first `count` slots and the slots it swaps with:
  // track those in a small map instead of materialising 0..n_views-1
  int32_t from[2 * SGE_MAX_VIEWS_PER_CALL], to[2 * SGE_MAX_VIEWS_PER_CALL];
  int m = 0;
  auto get = [&](int32_t i) {
    for (int q = 0; q < m; ++q)
      if (from[q] == i) return to[q];
    return i;
  };
  auto put = [&](int32_t i, int32_t v) {
    for (int q = 0; q < m; ++q)
      if (from[q] == i) {
        to[q] = v;
        return;
      }
    from[m] = i;
    to[m] = v;
    ++m;
  };
  for (int32_t i = 0; i < keep; ++i) {
    const uint64_t r = mix64(key + (uint64_t)(i + 1) * kGamma);
    const int32_t j = i + (int32_t)(r % (uint64_t)(n_views - i));
    const int32_t vi = get(i), vj = get(j);
    put(i, vj);
    put(j, vi);
    perm[i] = vj;
  }
  for (int32_t i = 0; i < keep; ++i) out[i] = perm[i];
  return SGE_OK;
}

int sge_atomic_bench(float* buf, int64_t n_addr, int64_t n_threads, int32_t per_thread, sge_stream_t stream) {
  if (!buf || n_addr < 1 || n_threads < 1 || per_thread < 1 || n_threads > 256ll * 0x7FFFFFFF)
    return fail(SGE_ERR_INVALID_ARG, "sge_atomic_bench: need buf, n_addr >= 1, 1 <= n_threads, per_thread >= 1");
  cudaError_t e = launch_red_bench(buf, n_addr, n_threads, per_thread, (cudaStream_t)stream);
  return e == cudaSuccess ? SGE_OK : cuda_fail(e, "sge_atomic_bench");
}

int sge_checked_build(void) { return SGE_CHECKED ? 1 : 0; }

int sge_check_report(sge_scene* s, sge_stream_t stream, int32_t* site, int64_t* index) {
  if (!SGE_CHECKED) return fail(SGE_ERR_UNSUPPORTED, "sge_check_report: not the checked build");
  if (!s || !site || !index) return fail(SGE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t w[2] = {0u, 0u};
  cudaError_t e = cudaMemcpyAsync(w, s->ws.counters + 8, sizeof(w), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ws.counters + 8, 0, sizeof(w), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sge_check_report");
  *site = (int32_t)w[0];
  *index = (int64_t)w[1];
  return SGE_OK;
}

int sge_check_limit(sge_scene* s, int32_t which, int64_t limit) {
  if (!SGE_CHECKED) return fail(SGE_ERR_UNSUPPORTED, "sge_check_limit: not the checked build");
  if (!s) return fail(SGE_ERR_INVALID_ARG, "scene is NULL");
  CheckDev& c = s->dev.chk;
  const CheckDev& t = s->chk_true;
  long long top;
  switch (which) {
    case SGE_LIMIT_VERTICES: top = t.nv; break;
    case SGE_LIMIT_UVS: top = t.nuv; break;
    case SGE_LIMIT_BIN_ENTRIES: top = t.bins; break;
    case SGE_LIMIT_SIGN_WORDS: top = t.sign_words; break;
    case SGE_LIMIT_PARAMS: top = t.params; break;
    default: return fail(SGE_ERR_INVALID_ARG, "sge_check_limit: bad range %d", which);
  }
  if (limit > top) return fail(SGE_ERR_INVALID_ARG, "sge_check_limit: %lld above the true size %lld", (long long)limit, top);
  const long long v = limit < 0 ? top : limit;
  switch (which) {
    case SGE_LIMIT_VERTICES: c.nv = (int)v; break;
    case SGE_LIMIT_UVS: c.nuv = (int)v; break;
    case SGE_LIMIT_BIN_ENTRIES: c.bins = v; break;
    case SGE_LIMIT_SIGN_WORDS: c.sign_words = v; break;
    default: c.params = v; break;
  }
  s->desc_dirty = true;  // batched launches read the scene's device copy
  return SGE_OK;
}

void sge_destroy_scene(sge_scene* s) {
  if (s) {
    sge_kernel_timing(s, 0);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->join) cudaEventDestroy(s->join);
  }
  delete s;
}

}  // extern "C"
