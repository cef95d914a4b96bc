// sge_render_idb_static: sge_render_idb for callers that cannot allocate device memory.
//
// The regular entry points take their scratch (tile bins and lists) from a
// workspace the caller allocates.  A caller embedded in a host application that
// owns the whole device-memory budget (an engine that hands out no allocations
// at run time), or one that must not let cudaMalloc/cudaFree synchronise the
// device in the middle of its frame, has no way to provide one.  This entry
// point needs no workspace and no scene object: its scratch is a fixed array in
// this library's device memory (every GPU that loads the library holds it until
// the process exits), and the caller passes only inputs and outputs.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address once; make that first call before any stream capture.
// Every call shares the one array and leaves its contents behind; each call
// clears what must start at zero.  Two calls whose work overlaps on the GPU (on
// different streams, or from different host threads) race on the array: order
// them on one stream.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "sge_device.cuh"

using namespace sge;

namespace {

constexpr long long kMaxTriangles = SGE_STATIC_MAX_TRIANGLES;
constexpr long long kMaxTiles = (long long)(SGE_STATIC_MAX_PIXELS / (TILE * TILE));
constexpr long long kBinEntries = SGE_STATIC_BIN_ENTRIES;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffRect = 0;
constexpr size_t kOffMargin = kOffRect + al(sizeof(int4) * kMaxTriangles);
constexpr size_t kOffZ = kOffMargin + al(sizeof(int) * kMaxTriangles);
constexpr size_t kOffCount = kOffZ + al(sizeof(float2) * kMaxTriangles);
constexpr size_t kOffTileOff = kOffCount + al(sizeof(uint32_t) * kMaxTiles);
constexpr size_t kOffCur = kOffTileOff + al(sizeof(uint32_t) * (kMaxTiles + 1));
constexpr size_t kOffItems = kOffCur + al(sizeof(uint32_t) * kMaxTiles);
constexpr size_t kOffBins = kOffItems + al(sizeof(uint32_t) * kMaxTiles);
constexpr size_t kOffCounters = kOffBins + al(sizeof(uint32_t) * kBinEntries);
constexpr size_t kScratchBytes = kOffCounters + 256;

// The scratch itself.  Host code must never pass this name to a kernel: on the
// host it is only a stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_addr[kMaxDevices] = {};

// Errors return their code and leave their message for sge_last_error.
int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

// Device address of the scratch on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(SGE_ERR_CUDA, "sge_render_idb_static: no usable current device");
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return fail(SGE_ERR_CUDA, "sge_render_idb_static: cudaGetSymbolAddress failed");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SGE_OK;
}

__global__ void k_copy_status(const uint32_t* counters, int32_t* out) { *out = (int32_t)counters[3]; }

}  // namespace

extern "C" int sge_render_idb_static(const sge_scene_desc* d, int32_t view, uint64_t seed, uint32_t iter,
                                     uint32_t pair, int32_t side, uint64_t* depth_id, float* uv, float* rgb,
                                     int32_t* device_status, sge_stream_t stream) {
  if (!d || !d->positions || !d->pos_idx || !d->uvs || !d->uv_idx || !d->mvp)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: NULL scene pointer");
  if (d->n_vertices < 3 || d->n_vertices >= (1 << 28) || d->n_triangles < 1 || d->n_uvs < 1 || d->n_views < 1)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad scene counts");
  if (d->n_triangles > kMaxTriangles)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: more triangles than SGE_STATIC_MAX_TRIANGLES");
  if (d->width < 1 || d->height < 1 ||
      (long long)((d->width + TILE - 1) / TILE) * ((d->height + TILE - 1) / TILE) > kMaxTiles)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: render larger than SGE_STATIC_MAX_PIXELS");
  if (view < 0 || view >= d->n_views) return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad view");
  if (side < -1 || side > 1) return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: side not in {-1, 0, 1}");
  if (d->shading == SGE_SHADE_TRANSPARENT)
    return fail(SGE_ERR_UNSUPPORTED, "sge_render_idb_static: transparent scenes render through sge_render_deep");
  if (d->shading < SGE_SHADE_UNLIT || d->shading > SGE_SHADE_GGX || (d->shading == SGE_SHADE_GGX && !d->cam_pos))
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad shading");
  if (d->n_textures < 0 || d->n_textures > SGE_MAX_TEXTURES)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad texture count");
  for (int k = 0; k < d->n_textures; ++k) {
    const sge_texture& t = d->textures[k];
    if (!t.texels || t.width < 1 || t.height < 1 || (long long)t.width * t.height >= (1ll << 28) || t.channels < 1 ||
        t.channels > 4 || t.role < SGE_ROLE_ALBEDO || t.role > SGE_ROLE_METALLIC)
      return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad texture");
  }

  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;

  // device view of the scene (the same fields the workspace-based entry points use)
  SceneDev S;
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
    S.tex[k] = TexDev{t.texels, t.width, t.height, t.channels, t.eps, t.role, 0, off, k};
    off += (long long)t.width * t.height * t.channels;
    if (first_of_role[t.role] < 0) first_of_role[t.role] = k;
  }
  S.n_params = off;
  for (int k = 0; k < d->n_textures; ++k) {
    const int role = d->textures[k].role;
    const bool read = first_of_role[role] == k &&
                      (d->shading == SGE_SHADE_GGX || role == SGE_ROLE_ALBEDO ||
                       (d->shading == SGE_SHADE_LAMBERT && role == SGE_ROLE_NORMAL));
    S.tex[k].read = read;
    if (read) S.read_k[S.nread++] = k;
  }
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
  S.tiles_x = (d->width + TILE - 1) / TILE;
  S.tiles_y = (d->height + TILE - 1) / TILE;

  char* b = static_cast<char*>(base);
  // every field the binning and render kernels use points into the scratch; the
  // estimator's buffers (projected vertices, staged keys) stay NULL and are never touched
  Workspace ws;
  memset(&ws, 0, sizeof(ws));
  ws.tri_rect = reinterpret_cast<int4*>(b + kOffRect);
  ws.tri_margin = reinterpret_cast<int*>(b + kOffMargin);
  ws.tri_z = reinterpret_cast<float2*>(b + kOffZ);
  ws.tile_count = reinterpret_cast<uint32_t*>(b + kOffCount);
  ws.tile_off = reinterpret_cast<uint32_t*>(b + kOffTileOff);
  ws.tile_cur = reinterpret_cast<uint32_t*>(b + kOffCur);
  ws.items = reinterpret_cast<uint32_t*>(b + kOffItems);
  ws.bins = reinterpret_cast<uint32_t*>(b + kOffBins);
  ws.counters = reinterpret_cast<uint32_t*>(b + kOffCounters);
  ws.bin_capacity = kBinEntries;
  ws.max_views = 1;
  ws.light_bin = kLightBin;

  cudaStream_t st = (cudaStream_t)stream;
  ViewList vl;
  vl.n = 1;
  vl.id[0] = view;
  // the status word must start at zero for this call (the binning counts are cleared by the binning itself)
  cudaError_t e = cudaMemsetAsync(ws.counters, 0, 64, st);
  if (e == cudaSuccess) e = launch_binning(S, ws, vl, st);
  if (e == cudaSuccess)
    e = launch_render(S, ws, 0, view, pair_key(seed, iter, (uint32_t)view, pair), side,
                      reinterpret_cast<unsigned long long*>(depth_id), reinterpret_cast<float2*>(uv), rgb, st);
  if (e == cudaSuccess && device_status) {
    k_copy_status<<<1, 1, 0, st>>>(ws.counters, device_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(SGE_ERR_CUDA, cudaGetErrorString(e));
  return SGE_OK;
}
