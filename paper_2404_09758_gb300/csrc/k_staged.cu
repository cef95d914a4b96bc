// Staged kernels: one render of R with its ID and UV buffers (Section 4.4), and
// the plain one-estimate-at-a-time path (Section 5's loop of P, R and G, with G
// as in Algorithm 2: per-pixel loss difference and a global AtomicAdd per
// contributing parameter).
#include <cuda_runtime.h>

#define SGE_FILE_ID 5  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

constexpr int RCHUNK = 128;  // triangles staged per pass (two sides fit the 48 KB static limit)

struct RSmem {
  Tri t[RCHUNK];
  int tri[RCHUNK];
  float m[16];
};

// Visible triangle of every pixel of a tile for `nsides` sides (side0, -side0):
// binned triangles are set up in shared memory a chunk at a time.
template <int NS>
__device__ __forceinline__ void raster_tile(const SceneDev& S, const Workspace& ws, RSmem (&sm)[NS], int slot,
                                            int tile, uint64_t key, const int (&sides)[NS],
                                            unsigned long long (&best)[NS], long long rx, long long ry, int dx,
                                            int dy) {
  const int ntl = n_tiles(S);
  const uint32_t beg = ws.tile_off[slot * ntl + tile];
  int nb = (int)(ws.tile_off[slot * ntl + tile + 1] - beg);
  // after a bin overflow (reported in the status word) the tile's list was not stored
  if ((long long)beg + nb > ws.bin_capacity) nb = 0;
#pragma unroll
  for (int s = 0; s < NS; ++s) best[s] = ~0ull;
  for (int c0 = 0; c0 < nb; c0 += RCHUNK) {
    const int cnt = min(RCHUNK, nb - c0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int tri = (int)bin_at(S, ws, beg + c0 + threadIdx.x);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        setup_from_scene(S, sm[0].m, tri, key, sides[s], rx, ry, sm[s].t[threadIdx.x]);
        sm[s].tri[threadIdx.x] = sm[s].t[threadIdx.x].ok ? tri : -1;
      }
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int tri = sm[s].tri[j];
        if (tri < 0) continue;
        long long e[3];
        if (!cover(sm[s].t[j], dx, dy, e)) continue;
        float l[3];
        lambdas(e, sm[s].t[j].inv_area, l);
        unsigned long long k = ((unsigned long long)ordered_bits(interp_depth(l, sm[s].t[j].z)) << 32) | (uint32_t)tri;
        if (k < best[s]) best[s] = k;
      }
    }
  }
}

__global__ void __launch_bounds__(TILE_PX) k_render(SceneDev S, Workspace ws, int slot, int view, uint64_t key,
                                                    int side, unsigned long long* keys, float2* uv, float* rgb) {
  __shared__ RSmem sm[1];
  const int tile = blockIdx.x;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = threadIdx.x % TILE, dy = threadIdx.x / TILE;
  const int px = tx * TILE + dx, py = ty * TILE + dy;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  if (threadIdx.x < 16) sm[0].m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  unsigned long long best[1];
  const int sides[1] = {side};
  raster_tile<1>(S, ws, sm, slot, tile, key, sides, best, rx, ry, dx, dy);
  if (px >= S.W || py >= S.H) return;
  const long long p = (long long)py * S.W + px;
  if (keys) keys[p] = best[0];
  if (best[0] == ~0ull) {
    if (uv) uv[p] = make_float2(0.f, 0.f);
    if (rgb) rgb[3 * p] = S.bg[0], rgb[3 * p + 1] = S.bg[1], rgb[3 * p + 2] = S.bg[2];
    return;
  }
  const int tri = (int)(best[0] & 0xFFFFFFFFu);
  Tri t;
  setup_from_scene(S, sm[0].m, tri, key, side, rx, ry, t);
  long long e[3];
  cover(t, dx, dy, e);
  Surf sf;
  surface(S, view, tri, t, e, key, side, sf);
  if (uv) uv[p] = make_float2(sf.u, sf.v);
  if (rgb) rgb[3 * p] = sf.rgb.x, rgb[3 * p + 1] = sf.rgb.y, rgb[3 * p + 2] = sf.rgb.z;
}

// Unperturbed render of one view reduced to its image error f = sum_p || I_p(theta) - I_p ||^2
// (Table 1): the forward value of the autograd form.  Adds the view's sum to loss[slot].
__global__ void __launch_bounds__(TILE_PX) k_render_loss(SceneDev S, Workspace ws, int slot, int view, float* loss) {
  __shared__ RSmem sm[1];
  __shared__ float red[TILE_PX / 32];
  const int tile = blockIdx.x;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = threadIdx.x % TILE, dy = threadIdx.x / TILE;
  const int px = tx * TILE + dx, py = ty * TILE + dy;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  if (threadIdx.x < 16) sm[0].m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  unsigned long long best[1];
  const int sides[1] = {0};
  raster_tile<1>(S, ws, sm, slot, tile, 0, sides, best, rx, ry, dx, dy);
  float f = 0.0f;
  if (px < S.W && py < S.H) {
    float3 c = f3(S.bg[0], S.bg[1], S.bg[2]);
    if (best[0] != ~0ull) {
      const int tri = (int)(best[0] & 0xFFFFFFFFu);
      Tri t;
      setup_from_scene(S, sm[0].m, tri, 0, 0, rx, ry, t);
      long long e[3];
      cover(t, dx, dy, e);
      Surf sf;
      surface(S, view, tri, t, e, 0, 0, sf);
      c = sf.rgb;
    }
    const float* tp = S.targets + (((long long)view * S.H + py) * S.W + px) * 3;
    const float d0 = c.x - __ldg(tp), d1 = c.y - __ldg(tp + 1), d2 = c.z - __ldg(tp + 2);
    f = d0 * d0 + d1 * d1 + d2 * d2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.0f;
    for (int i = 0; i < TILE_PX / 32; ++i) sum += red[i];
    atomicAdd(loss + slot, sum);
  }
}

// Plain path, step R: both sides' depth|ID and UV buffers of one estimate.
__global__ void __launch_bounds__(TILE_PX) k_raster_pair(SceneDev S, Workspace ws, int slot, int view, uint64_t key) {
  __shared__ RSmem sm[2];
  const int tile = blockIdx.x;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = threadIdx.x % TILE, dy = threadIdx.x / TILE;
  const int px = tx * TILE + dx, py = ty * TILE + dy;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  if (threadIdx.x < 16) sm[0].m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  unsigned long long best[2];
  const int sides[2] = {1, -1};
  raster_tile<2>(S, ws, sm, slot, tile, key, sides, best, rx, ry, dx, dy);
  if (px >= S.W || py >= S.H) return;
  const long long npx = (long long)S.W * S.H, p = (long long)py * S.W + px;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    ws.keys[s * npx + p] = best[s];
    float2 uvv = make_float2(0.f, 0.f);
    if (best[s] != ~0ull) {
      const int tri = (int)(best[s] & 0xFFFFFFFFu);
      Tri t;
      setup_from_scene(S, sm[0].m, tri, key, sides[s], rx, ry, t);
      long long e[3];
      cover(t, dx, dy, e);
      float l[3];
      lambdas(e, t.inv_area, l);
      PerspW pw = persp(l, t.iw);
      int t0 = uv_of(S, tri, 0), t1 = uv_of(S, tri, 1), t2 = uv_of(S, tri, 2);
      uvv.x = persp_interp(pw, __ldg(S.uvs + 2 * t0), __ldg(S.uvs + 2 * t1), __ldg(S.uvs + 2 * t2));
      uvv.y = persp_interp(pw, __ldg(S.uvs + 2 * t0 + 1), __ldg(S.uvs + 2 * t1 + 1), __ldg(S.uvs + 2 * t2 + 1));
    }
    ws.uvbuf[s * npx + p] = uvv;
  }
}

// Plain path, step G part 1: shade both sides from the buffers, f+ - f- per pixel.
__global__ void k_shade_delta(SceneDev S, Workspace ws, int view, uint64_t key, float* loss, float loss_scale,
                              int slot) {
  const long long npx = (long long)S.W * S.H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float lv = 0.0f;
  if (p < npx) {
    const int px = (int)(p % S.W), py = (int)(p / S.W);
    const int tx = px / TILE, ty = py / TILE;
    const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
    const float* m = S.mvp + 16 * view;
    float3 col[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      col[s] = f3(S.bg[0], S.bg[1], S.bg[2]);
      unsigned long long k = ws.keys[s * npx + p];
      if (k == ~0ull) continue;
      const int tri = (int)(k & 0xFFFFFFFFu), side = s == 0 ? 1 : -1;
      Tri t;
      setup_from_scene(S, m, tri, key, side, rx, ry, t);
      long long e[3];
      cover(t, px - tx * TILE, py - ty * TILE, e);
      Surf sf;
      surface(S, view, tri, t, e, key, side, sf);
      col[s] = sf.rgb;
    }
    const float* tp = S.targets + ((long long)view * npx + p) * 3;
    float fp, fm;
    ws.dfbuf[p] = loss_diff(col[0], col[1], f3(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2)), fp, fm);
    lv = 0.5f * (fp + fm);
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
    if ((threadIdx.x & 31) == 0 && lv != 0.0f) atomicAdd(loss + slot, lv * loss_scale);
  }
}

// Plain path, step G part 2: AtomicAdd of (f+ - f-) s_i into every contributing parameter.
__global__ void k_scatter(SceneDev S, Workspace ws, uint64_t key, float* grad, uint32_t* counts) {
  const long long npx = (long long)S.W * S.H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npx) return;
  int tris[2];
  Foot foot[2][MAX_READ];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    unsigned long long k = ws.keys[s * npx + p];
    tris[s] = k == ~0ull ? -1 : (int)(k & 0xFFFFFFFFu);
    if (tris[s] < 0) continue;
    float2 uv = ws.uvbuf[s * npx + p];
#pragma unroll
    for (int r = 0; r < MAX_READ; ++r)
      if (r < S.nread) {
        const TexDev& T = S.tex[S.read_k[r]];
        foot[s][r] = footprint(uv.x, uv.y, T.w, T.h);
        if (S.foot_nearest) foot[s][r].nearest = nearest_texel(uv.x, uv.y, T.w, T.h);
      }
  }
  const float df = ws.dfbuf[p];
  for_each_contrib(S, tris, foot, [&](uint32_t ck) {
    long long base;
    int nch;
    key_params(S, ck, base, nch);
    for (int c = 0; c < nch; ++c) {
      if (!CHK(S, base + c, S.chk.params)) continue;
      atomicAdd(grad + base + c, sign_neg(key, (uint64_t)(base + c)) ? -df : df);
      atomicAdd(counts + base + c, 1u);
    }
  });
}

// Full-image estimator (Eq. 4), step G: the estimate's whole-image loss difference
// sum_p (f+_p - f-_p), from the staged per-pixel differences, added to *out.
__global__ void __launch_bounds__(256) k_reduce_image(const float* df, long long npx, float* out) {
  __shared__ float red[8];
  float v = 0.0f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x)
    v += df[p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.0f;
    for (int i = 0; i < 8; ++i) sum += red[i];
    atomicAdd(out, sum);
  }
}

__global__ void k_validate(SceneDev S, uint32_t* status) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3ll * S.nt) return;
  const int pv = S.pidx[i], uv = S.uvidx[i];
  bool bad = pv < 0 || pv >= S.nv || uv < 0 || uv >= S.nuv;
  if (bad) atomicCAS(status, 0u, (uint32_t)SGE_ERR_BAD_INDEX);
}

}  // namespace

cudaError_t launch_render(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key, int side,
                          unsigned long long* keys, float2* uv, float* rgb, cudaStream_t st) {
  k_render<<<n_tiles(S), TILE_PX, 0, st>>>(S, ws, slot, view, key, side, keys, uv, rgb);
  return cudaGetLastError();
}

cudaError_t launch_render_loss(const SceneDev& S, const Workspace& ws, int slot, int view, float* loss,
                               cudaStream_t st) {
  k_render_loss<<<n_tiles(S), TILE_PX, 0, st>>>(S, ws, slot, view, loss);
  return cudaGetLastError();
}

cudaError_t launch_plain_pair(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key,
                              const EstimateArgs& a, float loss_scale, cudaStream_t st) {
  const long long npx = (long long)S.W * S.H;
  const int blocks = (int)((npx + 255) / 256);
  k_raster_pair<<<n_tiles(S), TILE_PX, 0, st>>>(S, ws, slot, view, key);
  k_shade_delta<<<blocks, 256, 0, st>>>(S, ws, view, key, a.loss, loss_scale, slot);
  k_scatter<<<blocks, 256, 0, st>>>(S, ws, key, a.grad, a.counts);
  return cudaGetLastError();
}

cudaError_t launch_image_delta(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key, float* out,
                               cudaStream_t st) {
  const long long npx = (long long)S.W * S.H;
  const int blocks = (int)((npx + 255) / 256);
  k_raster_pair<<<n_tiles(S), TILE_PX, 0, st>>>(S, ws, slot, view, key);
  k_shade_delta<<<blocks, 256, 0, st>>>(S, ws, view, key, nullptr, 0.0f, slot);
  k_reduce_image<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(ws.dfbuf, npx, out);
  return cudaGetLastError();
}

cudaError_t launch_validate(const SceneDev& S, uint32_t* status, cudaStream_t st) {
  const long long n = 3ll * S.nt;
  k_validate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, status);
  return cudaGetLastError();
}

}  // namespace sge
