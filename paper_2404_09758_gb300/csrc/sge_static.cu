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
// The address belongs to the device's context: after cudaDeviceReset the next call
// looks it up again (in the new context), so that call too should precede a capture.
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
// Per device: the scratch address and the ID of the context it was looked up in.  A context
// that goes away (cudaDeviceReset) takes the address with it, so a changed ID means a new lookup.
struct Cached {
  void* addr;
  unsigned long long ctx_id;
  bool keyed;  // ctx_id is known; without it the address is looked up on every call
};
Cached g_cache[kMaxDevices] = {};

// Errors return their code and leave their message for sge_last_error.
int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

// ID of the calling thread's current CUDA context, through the driver's entry points that the
// runtime hands out (the library does not link the driver library itself).  Called with g_lock held.
bool current_context_id(unsigned long long* id) {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                         cudaEnableDefault, &q) != cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000, cudaEnableDefault,
                                         &q) != cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_id = nullptr;
  }
  if (!get_current || !get_id) return false;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch on the current device: looked up once per device and context.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(SGE_ERR_CUDA, "sge_render_idb_static: no usable current device");
  std::lock_guard<std::mutex> g(g_lock);
  unsigned long long id = 0;
  bool keyed = current_context_id(&id);
  Cached& c = g_cache[dev];
  if (!c.addr || !c.keyed || !keyed || c.ctx_id != id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return fail(SGE_ERR_CUDA, "sge_render_idb_static: cudaGetSymbolAddress failed");
    if (!keyed) keyed = current_context_id(&id);  // the lookup made the device's context current
    c.addr = p;
    c.ctx_id = id;
    c.keyed = keyed;
  }
  *out = c.addr;
  return SGE_OK;
}

__global__ void k_copy_status(const uint32_t* counters, int32_t* out) { *out = (int32_t)counters[3]; }

}  // namespace

extern "C" int sge_render_idb_static(const sge_scene_desc* d, int32_t view, uint64_t seed, uint32_t iter,
                                     uint32_t pair, int32_t side, uint64_t* depth_id, float* uv, float* rgb,
                                     int32_t* device_status, sge_stream_t stream) {
  // the same descriptor checks as every workspace-based entry point (targets are not read here)
  int rc = check_desc(d, false);
  if (rc) return rc;
  if (d->n_triangles > kMaxTriangles)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: more triangles than SGE_STATIC_MAX_TRIANGLES");
  if ((long long)((d->width + TILE - 1) / TILE) * ((d->height + TILE - 1) / TILE) > kMaxTiles)
    return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: render larger than SGE_STATIC_MAX_PIXELS");
  if (view < 0 || view >= d->n_views) return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: bad view");
  if (side < -1 || side > 1) return fail(SGE_ERR_INVALID_ARG, "sge_render_idb_static: side not in {-1, 0, 1}");
  if (d->shading == SGE_SHADE_TRANSPARENT)
    return fail(SGE_ERR_UNSUPPORTED, "sge_render_idb_static: transparent scenes render through sge_render_deep");

  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;

  // device view of the scene, built as the workspace-based entry points build it
  SceneDev S;
  make_dev(d, S);

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
  S.chk.status = ws.counters + 3;
  S.chk.where = ws.counters + 8;
  S.chk.bins = kBinEntries;

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
