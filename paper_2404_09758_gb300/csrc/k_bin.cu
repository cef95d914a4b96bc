// Tile binning shared by every pair and both sides of an estimate.
//
// The paper's rasterizer R (Section 4.3) renders theta + s eps and theta - s eps
// for every estimate.  All those scenes differ from theta by at most eps_pos per
// vertex coordinate, so one binning per view and call serves every render of
// that view: each triangle is binned into the tiles its screen bounding box can
// reach under any such perturbation (interval bounds of the projection plus a
// one-pixel margin).  A render then tests, per tile, only the triangles in the
// tile's bin, with the exact perturbed vertices.
#include <cuda_runtime.h>

#define SGE_FILE_ID 1  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

// Interval of one clip coordinate row of M over the box p +- eps (per coordinate).
__device__ __forceinline__ float clip_interval(const float* m, float x, float y, float z, float eps, float& lo,
                                               float& hi) {
  float c = m[0] * x + m[1] * y + m[2] * z + m[3];
  float r = eps * (fabsf(m[0]) + fabsf(m[1]) + fabsf(m[2]));
  r = r * 1.0001f + 1e-6f * (fabsf(c) + fabsf(m[3]) + 1.0f);
  lo = c - r;
  hi = c + r;
  return c;
}

__global__ void k_bin_rect_count(SceneDev S, Workspace ws, ViewList vl) {
  __shared__ float m[16];
  int slot = blockIdx.y;
  int view = vl.id[slot];
  if (threadIdx.x < 16) m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  int tri = blockIdx.x * blockDim.x + threadIdx.x;
  if (tri >= S.nt) return;
  int vi[3] = {vert_of(S, tri, 0), vert_of(S, tri, 1), vert_of(S, tri, 2)};
  int4 rect = make_int4(1, 1, 0, 0);  // empty
  bool skip = vi[0] == vi[1] || vi[1] == vi[2] || vi[0] == vi[2];  // welded duplicates: zero area always
  // a triangle with an index out of range is never binned, so no render reads through it
  for (int k = 0; k < 3; ++k) {
    const int ti = uv_of(S, tri, k);
    if (ti < 0 || ti >= S.nuv) skip = true;
  }
  float sx0 = 3.4e38f, sx1 = -3.4e38f, sy0 = 3.4e38f, sy1 = -3.4e38f;
  float disp = 0.0f;  // widest screen interval of a vertex under the perturbation, pixels
  float zlo = 3.4e38f, zhi = -3.4e38f;  // depth interval of the triangle under the perturbation
  bool full = false;
  for (int k = 0; k < 3 && !skip; ++k) {
    if (vi[k] < 0 || vi[k] >= S.nv) { skip = true; break; }
    const float* p = S.pos + 3ll * vi[k];
    float x = p[0], y = p[1], z = p[2];
    float xl, xh, yl, yh, zl, zh, wl, wh;
    const float cx = clip_interval(m + 0, x, y, z, S.eps_pos, xl, xh);
    const float cy = clip_interval(m + 4, x, y, z, S.eps_pos, yl, yh);
    clip_interval(m + 8, x, y, z, S.eps_pos, zl, zh);
    const float cw = clip_interval(m + 12, x, y, z, S.eps_pos, wl, wh);
    if (wh <= S.near_w) { skip = true; break; }  // always behind the near limit: triangle never drawn
    if (wl <= S.near_w) { full = true; continue; }  // may or may not be drawn: bin everywhere
    float nx0 = fminf(fminf(xl / wl, xl / wh), fminf(xh / wl, xh / wh));
    float nx1 = fmaxf(fmaxf(xl / wl, xl / wh), fmaxf(xh / wl, xh / wh));
    float ny0 = fminf(fminf(yl / wl, yl / wh), fminf(yh / wl, yh / wh));
    float ny1 = fmaxf(fmaxf(yl / wl, yl / wh), fmaxf(yh / wl, yh / wh));
    zlo = fminf(zlo, fminf(fminf(zl / wl, zl / wh), fminf(zh / wl, zh / wh)));
    zhi = fmaxf(zhi, fmaxf(fmaxf(zl / wl, zl / wh), fmaxf(zh / wl, zh / wh)));
    const float vx0 = (nx0 * 0.5f + 0.5f) * S.W, vx1 = (nx1 * 0.5f + 0.5f) * S.W;
    const float vy0 = (0.5f - ny1 * 0.5f) * S.H, vy1 = (0.5f - ny0 * 0.5f) * S.H;
    sx0 = fminf(sx0, vx0);
    sx1 = fmaxf(sx1, vx1);
    sy0 = fminf(sy0, vy0);
    sy1 = fmaxf(sy1, vy1);
    // farthest any perturbed screen position lies from the unperturbed one
    const float ux = (cx / cw * 0.5f + 0.5f) * S.W, uy = (0.5f - cy / cw * 0.5f) * S.H;
    disp = fmaxf(disp, fmaxf(fmaxf(vx1 - ux, ux - vx0), fmaxf(vy1 - uy, uy - vy0)));
    // near the guard band the drop rule may flip under the perturbation
    if (!(fmaxf(fabsf(vx0), fabsf(vx1)) < 30000.0f && fmaxf(fabsf(vy0), fabsf(vy1)) < 30000.0f)) full = true;
  }
  // Margin (fixed-point units) that bounds, per axis, how far any snapped perturbed
  // vertex can be from the snapped unperturbed one: the farthest interval end, one
  // unit for the two snaps and slack for float rounding; "full" = unbounded.
  int margin = 0x7FFFFFFF;
  if (!full && !skip && disp < 1.0e4f) margin = (int)ceilf(disp * 256.0f * 1.002f) + 4;
  ws.tri_margin[(long long)slot * S.nt + tri] = margin;
  // interpolated depth of a covered pixel lies between the vertex depths; slack for float rounding
  ws.tri_z[(long long)slot * S.nt + tri] =
      make_float2(zlo - (1e-6f + 1e-5f * fabsf(zlo)), zhi + (1e-6f + 1e-5f * fabsf(zhi)));
  if (!skip) {
    int px0, px1, py0, py1;
    if (full) {
      px0 = 0; py0 = 0; px1 = S.W - 1; py1 = S.H - 1;
    } else {
      // pixel centres px + 0.5 inside [sx0, sx1], one pixel of margin each way
      px0 = (int)fmaxf(floorf(sx0) - 1.0f, 0.0f);
      py0 = (int)fmaxf(floorf(sy0) - 1.0f, 0.0f);
      px1 = (int)fminf(floorf(sx1) + 1.0f, (float)(S.W - 1));
      py1 = (int)fminf(floorf(sy1) + 1.0f, (float)(S.H - 1));
    }
    if (px0 <= px1 && py0 <= py1) rect = make_int4(px0 / TILE, py0 / TILE, px1 / TILE, py1 / TILE);
  }
  ws.tri_rect[(long long)slot * S.nt + tri] = rect;
  int nt = n_tiles(S);
  for (int ty = rect.y; ty <= rect.w; ++ty)
    for (int tx = rect.x; tx <= rect.z; ++tx)
      atomicAdd(ws.tile_count + (long long)slot * nt + ty * S.tiles_x + tx, 1u);
}

// One CTA: exclusive scan of the per-(slot, tile) counts, list of non-empty tiles,
// fill cursors, and the estimate kernel's work counter.
__global__ void __launch_bounds__(1024) k_bin_scan(Workspace ws, int n, int nt, int list_items) {
  __shared__ uint32_t wsum[32], wne[32], wnh[32];
  int tid = threadIdx.x;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  int beg = min(n, tid * per), end = min(n, beg + per);
  uint32_t sum = 0, ne = 0, nh = 0;
  for (int i = beg; i < end; ++i) {
    uint32_t c = ws.tile_count[i];
    sum += c;
    ne += c > 0 && c <= (uint32_t)ws.light_bin;
    nh += c > (uint32_t)ws.light_bin;
  }
  // block exclusive scan of (sum, ne, nh)
  uint32_t xs = sum, xn = ne, xh = nh;
  int lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t a = __shfl_up_sync(0xffffffffu, xs, o), b = __shfl_up_sync(0xffffffffu, xn, o);
    uint32_t c = __shfl_up_sync(0xffffffffu, xh, o);
    if (lane >= o) { xs += a; xn += b; xh += c; }
  }
  if (lane == 31) { wsum[wid] = xs; wne[wid] = xn; wnh[wid] = xh; }
  __syncthreads();
  if (wid == 0) {
    const bool in = lane < (int)(blockDim.x >> 5);
    uint32_t a = in ? wsum[lane] : 0u, b = in ? wne[lane] : 0u, c = in ? wnh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t pa = __shfl_up_sync(0xffffffffu, a, o), pb = __shfl_up_sync(0xffffffffu, b, o);
      uint32_t pc = __shfl_up_sync(0xffffffffu, c, o);
      if (lane >= o) { a += pa; b += pb; c += pc; }
    }
    wsum[lane] = a;
    wne[lane] = b;
    wnh[lane] = c;
  }
  __syncthreads();
  uint32_t off = (wid ? wsum[wid - 1] : 0u) + xs - sum;
  uint32_t noff = (wid ? wne[wid - 1] : 0u) + xn - ne;
  uint32_t hoff = (wid ? wnh[wid - 1] : 0u) + xh - nh;
  for (int i = beg; i < end; ++i) {
    uint32_t c = ws.tile_count[i];
    ws.tile_off[i] = off;
    ws.tile_cur[i] = off;
    if (c > 0) {
      int slot = i / nt, tile = i - slot * nt;
      const uint32_t it = ((uint32_t)slot << 24) | (uint32_t)tile;
      // light items from the front of the list, heavy ones from the back
      if (list_items) {
        if (c <= (uint32_t)ws.light_bin) ws.items[noff++] = it;
        else ws.items[n - 1 - hoff++] = it;
      }
    }
    off += c;
  }
  if (tid == blockDim.x - 1) {
    ws.tile_off[n] = off;
    bool overflow = (long long)off > ws.bin_capacity;
    // (without the list, k_bin_prune lists the items after pruning the bins)
    ws.counters[0] = overflow || !list_items ? 0u : noff;
    ws.counters[1] = 0u;
    ws.counters[2] = off;
    ws.counters[4] = overflow || !list_items ? 0u : hoff;
    ws.counters[5] = 0u;
    if (overflow) atomicCAS(ws.counters + 3, 0u, (uint32_t)SGE_ERR_BIN_OVERFLOW);
  }
}

__global__ void k_bin_fill(SceneDev S, Workspace ws) {
  int slot = blockIdx.y;
  int tri = blockIdx.x * blockDim.x + threadIdx.x;
  if (tri >= S.nt) return;
  int4 rect = ws.tri_rect[(long long)slot * S.nt + tri];
  int nt = n_tiles(S);
  for (int ty = rect.y; ty <= rect.w; ++ty)
    for (int tx = rect.x; tx <= rect.z; ++tx) {
      uint32_t pos = atomicAdd(ws.tile_cur + (long long)slot * nt + ty * S.tiles_x + tx, 1u);
      if ((long long)pos < ws.bin_capacity && CHK(S, pos, S.chk.bins)) ws.bins[pos] = (uint32_t)tri;
    }
}

}  // namespace

cudaError_t launch_binning(const SceneDev& S, const Workspace& ws, const ViewList& vl, cudaStream_t st, bool prune,
                           bool defer_prune) {
  int nt = n_tiles(S);
  cudaError_t e = cudaMemsetAsync(ws.tile_count, 0, sizeof(uint32_t) * (size_t)vl.n * nt, st);
  if (e != cudaSuccess) return e;
  dim3 grid((S.nt + 255) / 256, vl.n);
  k_bin_rect_count<<<grid, 256, 0, st>>>(S, ws, vl);
  k_bin_scan<<<1, 1024, 0, st>>>(ws, vl.n * nt, nt, prune || defer_prune ? 0 : 1);
  k_bin_fill<<<grid, 256, 0, st>>>(S, ws);
  e = cudaGetLastError();
  if (e == cudaSuccess && prune && !defer_prune) e = launch_prune(S, ws, vl, st);
  return e;
}

}  // namespace sge
