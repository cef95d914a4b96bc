// Transparent geometry (Section 4.4): the raster pass keeps a deep ID buffer (each pixel's
// SGE_MAX_LAYERS nearest fragments, ascending (depth bits, triangle id) keys), the shading
// composites the listed RGBA fragments front to back over the background, and G walks the list,
// crediting every listed fragment's vertices and albedo footprint as the opaque case credits
// its one visible triangle.
//
// One CTA per (16 x 16 tile, estimate).  The tile's binned triangles are set up for both sides
// in shared memory a chunk at a time; each pixel keeps both sides' lists in registers (with each
// entry's chunk slot, so that a bin of one chunk is not set up again to shade), then shades,
// forms f+ - f- and credits the union of its fragments' parameters.  When the bin fits one chunk
// the vertex credits are summed per staged triangle corner in shared memory and reach the global
// sums once per corner at the end of the CTA; texel credits (and every credit of a larger bin) go
// to global atomics per pixel.  Bins come from the conservative binning without pruning: a
// fragment behind another is still listed.
#include <cuda_runtime.h>

#define SGE_FILE_ID 2  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

constexpr int K = SGE_MAX_LAYERS;
constexpr int DCHUNK = 128;              // binned triangles staged per pass
constexpr int kDeepEstimates = 16384;    // estimates (grid rows) of one launch

template <int NS>
struct DeepSmem {
  Tri t[NS][DCHUNK];
  uint32_t span[NS][DCHUNK];  // box_span of each staged side-triangle: the pixels it may cover
  uint8_t small[NS][DCHUNK];  // its edge functions over the tile fit 32 bits
  int tri[DCHUNK];
  // estimator (two sides) with a bin of one chunk: each staged triangle's welded vertices, and
  // per corner the sum of f+ - f- and the count of the pixels that credit it through this triangle
  static constexpr int NV = NS == 2 ? DCHUNK : 1;
  int vid[NV][3];
  float vA[NV][3];
  uint32_t vn[NV][3];
  float m[16];
  float red[TILE_PX / 32];
};

// Every edge function of t over the tile fits 32 bits: |a|, |b| < 2^16 and |e0| < 2^29, so
// |e0 + a 256 dx + b 256 dy| < 2^30 for the pixel offsets 0..15.
__device__ __forceinline__ bool small_tri(const Tri& t) {
  bool small = true;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    small = small && abs(t.a[k]) < (1 << 16) && abs(t.b[k]) < (1 << 16) && t.e0[k] > -(1ll << 29) &&
            t.e0[k] < (1ll << 29);
  return small;
}

// cover() and lambdas() at pixel offset (dx, dy): the same integers and the same float
// conversions, in 32-bit arithmetic for a small triangle.
__device__ __forceinline__ bool cover_lambdas(const Tri& t, bool small, int dx, int dy, float l[3]) {
  if (small) {
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = (int)t.e0[k] + t.a[k] * (dx * 256) + t.b[k] * (dy * 256);
      in = in && (e + t.bias[k] >= 0);
      l[k] = __fmul_rn(__int2float_rn(e), t.inv_area);
    }
    return in;
  }
  long long e[3];
  const bool in = cover(t, dx, dy, e);
  lambdas(e, t.inv_area, l);
  return in;
}

// Insert key k (staged at shared-memory slot q) into the ascending list L (slots P); the
// largest key falls off the end.
__device__ __forceinline__ void deep_insert(unsigned long long (&L)[K], int (&P)[K], unsigned long long k, int q) {
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const bool lt = k < L[j];
    const unsigned long long lo = lt ? k : L[j];
    const int qlo = lt ? q : P[j];
    k = lt ? L[j] : k;
    q = lt ? P[j] : q;
    L[j] = lo;
    P[j] = qlo;
  }
}

// Deep lists of one pixel of the tile for NS sides (sides[s] = +1, -1 or 0), with each entry's
// slot in the staged chunk.  Returns the number of binned triangles it rasterized; when that is at
// most DCHUNK the whole bin fit one chunk, and sm.t[s][P[s][j]] (and sm.vid[P[s][j]]) still hold
// entry j's set-up when the raster is done.
// pv: the estimate's projected vertices from the vertex pass ([nv][2]: sides +, -), for the two
// sides of an estimate; NULL: each triangle is projected from the scene with key and sides[].
template <int NS>
__device__ __forceinline__ int deep_raster(const SceneDev& S, const Workspace& ws, DeepSmem<NS>& sm, int slot,
                                            int tile, uint64_t key, const int (&sides)[NS],
                                            unsigned long long (&L)[NS][K], int (&P)[NS][K], long long rx,
                                            long long ry, int dx, int dy, const int4* pv = nullptr) {
  const int ntl = n_tiles(S);
  const uint32_t beg = ws.tile_off[slot * ntl + tile];
  int nb = (int)(ws.tile_off[slot * ntl + tile + 1] - beg);
  // after a bin overflow (reported in the status word) the tile's list was not stored
  if ((long long)beg + nb > ws.bin_capacity) nb = 0;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int j = 0; j < K; ++j) L[s][j] = ~0ull, P[s][j] = 0;
  for (int c0 = 0; c0 < nb; c0 += DCHUNK) {
    const int cnt = min(DCHUNK, nb - c0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int tri = (int)bin_at(S, ws, beg + c0 + threadIdx.x);
      sm.tri[threadIdx.x] = tri;
      if constexpr (NS == 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sm.vid[threadIdx.x][k] = vert_of(S, tri, k);
          sm.vA[threadIdx.x][k] = 0.0f;
          sm.vn[threadIdx.x][k] = 0u;
        }
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        PVert v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int vi = vert_of(S, tri, k);
          if (pv) {
            const int4 q = __ldg(pv + 2 * vi + s);
            v[k].X = q.x;
            v[k].Y = q.y;
            v[k].z = __int_as_float(q.z);
            v[k].iw = __int_as_float(q.w);
            v[k].ok = q.x != kNotDrawn;
          } else {
            const float3 p = perturbed_pos(S, vi, key, sides[s]);
            v[k] = project(sm.m, p.x, p.y, p.z, S.W, S.H, S.near_w);
          }
        }
        Tri& t = sm.t[s][threadIdx.x];
        setup_tri(v[0], v[1], v[2], rx, ry, t);
        // a covered pixel centre lies in the triangle's vertex box
        sm.span[s][threadIdx.x] = t.ok ? box_span(v, rx, ry, 0) : 0u;
        sm.small[s][threadIdx.x] = t.ok && small_tri(t);
      }
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (!in_span(sm.span[s][j], dx, dy)) continue;
        const Tri& t = sm.t[s][j];
        if (!t.ok) continue;
        float l[3];
        if (!cover_lambdas(t, sm.small[s][j] != 0, dx, dy, l)) continue;
        deep_insert(L[s], P[s], ((unsigned long long)ordered_bits(interp_depth(l, t.z)) << 32) | (uint32_t)sm.tri[j],
                    j);
      }
    }
  }
  return nb;
}

// Front-to-back composite of one side's list at one pixel: T = 1; per listed fragment
// C += T a rgb, T *= 1 - a with a = clamp(alpha, 0, 1); C += T background.  on_fragment(tri,
// foot, j, q) is called for each listed fragment with its triangle, albedo footprint, layer and
// chunk slot.
// staged: the side's set-ups in shared memory (slots P) when the bin fit one chunk, else NULL
// (each fragment is set up again; the same arithmetic gives the same set-up).
// ps: the estimate's precomputed signs (vertex bits, texel planes), or NULL to hash with key.
template <typename F>
__device__ __forceinline__ float3 deep_composite(const SceneDev& S, const float* m, uint64_t key, int side,
                                                 const unsigned long long (&L)[K], const int (&P)[K],
                                                 const Tri* staged, long long rx, long long ry, int dx, int dy,
                                                 F&& on_fragment, const PairSigns* ps = nullptr,
                                                 const int4* pv = nullptr) {
  const TexDev& A = S.rtex[0];  // the RGBA albedo, the one texture this model reads
  float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
  // not unrolled: one copy of the fragment's set-up, sampling and credit code per side keeps the
  // kernel's code within the instruction cache (the lists are read from local memory instead)
#pragma unroll 1
  for (int j = 0; j < K; ++j) {
    if (L[j] == ~0ull) continue;
    const int tri = (int)(L[j] & 0xFFFFFFFFu);
    Tri own;
    if (!staged) {
      if (pv) {
        PVert v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int4 q = __ldg(pv + 2 * vert_of(S, tri, k) + (side < 0 ? 1 : 0));
          v[k].X = q.x;
          v[k].Y = q.y;
          v[k].z = __int_as_float(q.z);
          v[k].iw = __int_as_float(q.w);
          v[k].ok = q.x != kNotDrawn;
        }
        setup_tri(v[0], v[1], v[2], rx, ry, own);
      } else {
        setup_from_scene(S, m, tri, key, side, rx, ry, own);
      }
    }
    const Tri& t = staged ? staged[P[j]] : own;
    long long e[3];
    cover(t, dx, dy, e);
    float l[3];
    lambdas(e, t.inv_area, l);
    PerspW pw = persp(l, t.iw);
    const int t0 = uv_of(S, tri, 0), t1 = uv_of(S, tri, 1), t2 = uv_of(S, tri, 2);
    const float u = persp_interp(pw, __ldg(S.uvs + 2 * t0), __ldg(S.uvs + 2 * t1), __ldg(S.uvs + 2 * t2));
    const float v = persp_interp(pw, __ldg(S.uvs + 2 * t0 + 1), __ldg(S.uvs + 2 * t1 + 1), __ldg(S.uvs + 2 * t2 + 1));
    Foot f = footprint(u, v, A.w, A.h);
    if (S.foot_nearest) f.nearest = nearest_texel(u, v, A.w, A.h);
    float a[4];
    // an RGBA albedo in a 16-byte aligned array: one vector load per texel
    if (ps && A.c == 4 && ((reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0)) {
      const float w4[4] = {(1.0f - f.fx) * (1.0f - f.fy), f.fx * (1.0f - f.fy), (1.0f - f.fx) * f.fy, f.fx * f.fy};
      const int tx[4] = {f.x0, f.x1, f.x0, f.x1};
      const int ty[4] = {f.y0, f.y0, f.y1, f.y1};
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long tt = (long long)ty[q] * A.w + tx[q];
        const float4 v4 = __ldg(reinterpret_cast<const float4*>(A.ptr + tt * 4));
        uint32_t sb = texel_signs(*ps, A.index, tt);
        if (side < 0) sb = ~sb;
        a[0] += w4[q] * __fadd_rn(v4.x, (sb & 1) ? -A.eps : A.eps);
        a[1] += w4[q] * __fadd_rn(v4.y, (sb & 2) ? -A.eps : A.eps);
        a[2] += w4[q] * __fadd_rn(v4.z, (sb & 4) ? -A.eps : A.eps);
        a[3] += w4[q] * __fadd_rn(v4.w, (sb & 8) ? -A.eps : A.eps);
      }
    } else if (ps) {
      sample_tex_ps(A, f, *ps, side, a);
    } else {
      sample_tex(A, f, key, side, a);
    }
    const float al = fminf(fmaxf(a[3], 0.0f), 1.0f);
    const float w = T * al;
    c0 += w * a[0];
    c1 += w * a[1];
    c2 += w * a[2];
    T *= 1.0f - al;
    on_fragment(tri, f, j, P[j]);
  }
  return f3(c0 + T * S.bg[0], c1 + T * S.bg[1], c2 + T * S.bg[2]);
}

// Sum of v over the CTA, added to *out by thread 0.
__device__ __forceinline__ void cta_add(float v, float* red, float* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.0f;
    for (int i = 0; i < TILE_PX / 32; ++i) sum += red[i];
    if (sum != 0.0f) atomicAdd(out, sum);
  }
}

// One estimate per grid row: blockIdx.y = slot * pair_count + (pair - pair_begin).
__global__ void __launch_bounds__(TILE_PX, 3) k_estimate_deep(SceneDev S, Workspace ws, ViewList vl, EstimateArgs a,
                                                           int row0) {
  __shared__ DeepSmem<2> sm;
  const int tile = blockIdx.x;
  const int row = row0 + (int)blockIdx.y;
  const int slot = row / a.pair_count, pair = a.pair_begin + row % a.pair_count;
  const int view = vl.id[slot];
  const uint64_t key = pair_key(a.seed, iter_of(a), (uint32_t)view, (uint32_t)pair);
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = threadIdx.x % TILE, dy = threadIdx.x / TILE;
  const int px = tx * TILE + dx, py = ty * TILE + dy;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  if (threadIdx.x < 16) sm.m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  unsigned long long L[2][K];
  int P[2][K];
  const int sides[2] = {1, -1};
  // the estimate's projected vertices and signs, from the vertex pass and the texel sign planes
  const int pb = pair - a.pair_begin;
  const int4* pv = ws.pverts + 2 * (((long long)slot * ws.max_pairs + pb) * S.nv);
  const PairSigns ps = pair_signs(S, ws, slot, pb);
  const int nb = deep_raster<2>(S, ws, sm, slot, tile, key, sides, L, P, rx, ry, dx, dy, pv);
  const bool resident = nb <= DCHUNK;
  float lv = 0.0f;
  if (px < S.W && py < S.H) {
    const long long npx = (long long)S.W * S.H, p = (long long)py * S.W + px;
    // the contributor set, gathered while compositing: every listed fragment's welded vertices
    // and footprint texels, both sides, each key once
    const TexDev& A = S.rtex[0];
    // vertex keys and texel keys in separate lists (a key of one kind never equals one of the other)
    uint32_t vk[2 * K * 3], tk[2 * K * 4];
    int nvk = 0, ntk = 0;
    auto addv = [&](uint32_t k) {
      for (int q = 0; q < nvk; ++q)
        if (vk[q] == k) return;
      vk[nvk++] = k;
    };
    auto addt = [&](uint32_t k) {
      for (int q = 0; q < ntk; ++q)
        if (tk[q] == k) return;
      tk[ntk++] = k;
    };
    // side +'s fragments (layer j: triangle and footprint); a side - fragment on a triangle listed
    // there brings no new vertex, one with a footprint listed there no new texel
    int g_tri[K], g_fp[K];
#pragma unroll
    for (int j = 0; j < K; ++j) g_tri[j] = -1, g_fp[j] = -1;
    bool minus = false;
    // a bin of one chunk: the pixel's distinct triangles by chunk slot, each with the corners whose
    // vertex no earlier one of them has; their credits go to the shared per-corner sums
    int ds[2 * K];
    uint32_t dm[2 * K];
    int nds = 0;
    auto credit_keys = [&](int tri, const Foot& f, int j, int q) {
      // a footprint: its first texel and whether its rows were clamped to one (x1 follows from x0)
      const int fp = S.foot_nearest ? f.nearest : 2 * (f.y0 * A.w + f.x0) + (f.y1 != f.y0 ? 1 : 0);
      bool tri_seen = false, fp_seen = false;
      if (!minus) {
        g_tri[j] = tri;
        g_fp[j] = fp;
      } else {
#pragma unroll
        for (int i = 0; i < K; ++i) {
          tri_seen = tri_seen || g_tri[i] == tri;
          fp_seen = fp_seen || (g_tri[i] >= 0 && g_fp[i] == fp);
        }
      }
      if (!tri_seen && resident) {
        uint32_t mask = 7u;
        for (int i = 0; i < nds; ++i) {
          const int o = ds[i];
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk)
              if (sm.vid[q][k] == sm.vid[o][kk]) mask &= ~(1u << k);
        }
        ds[nds] = q;
        dm[nds++] = mask;
      } else if (!tri_seen) {
#pragma unroll
        for (int v = 0; v < 3; ++v) addv(vkey(vert_of(S, tri, v)));
      }
      if (fp_seen) return;
      if (S.foot_nearest) {
        addt(tkey(A.index, f.nearest));
        return;
      }
      addt(tkey(A.index, f.y0 * A.w + f.x0));
      addt(tkey(A.index, f.y0 * A.w + f.x1));
      addt(tkey(A.index, f.y1 * A.w + f.x0));
      addt(tkey(A.index, f.y1 * A.w + f.x1));
    };
    const float3 cp = deep_composite(S, sm.m, key, 1, L[0], P[0], resident ? sm.t[0] : nullptr, rx, ry, dx, dy,
                                     credit_keys, &ps, pv);
    minus = true;
    const float3 cm = deep_composite(S, sm.m, key, -1, L[1], P[1], resident ? sm.t[1] : nullptr, rx, ry, dx, dy,
                                     credit_keys, &ps, pv);
    const float* tp = S.targets + ((long long)view * npx + p) * 3;
    float fp, fm;
    const float df = loss_diff(cp, cm, f3(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2)), fp, fm);
    lv = 0.5f * (fp + fm);
    if (a.delta_f) a.delta_f[((long long)slot * a.pairs + pair) * npx + p] = df;
    for (int i = 0; i < nds; ++i) {
      const int q = ds[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (!((dm[i] >> k) & 1u)) continue;
        atomicAdd(&sm.vA[q][k], df);
        atomicAdd(&sm.vn[q][k], 1u);
      }
    }
    // one count per key (k_expand_counts gives it to every channel after the call), a signed
    // sum per channel (RGBA texels of an 8-byte aligned gradient: two vector reductions)
    const bool pairs4 = A.c == 4 && ((reinterpret_cast<uintptr_t>(a.grad + A.offset) & 7) == 0);
    for (int q = 0; q < nvk + ntk; ++q) {
      const uint32_t kq = q < nvk ? vk[q] : tk[q - nvk];
      const uint32_t kind = kq >> 28, idx = kq & 0x0FFFFFFFu;
      const long long kc = kind == 0 ? (long long)idx : ws.kc_off[kind - 1] + idx;
      if (CHK(S, kc, ws.n_kcount)) atomicAdd(ws.kcount + kc, 1u);
      if (kind != 0 && pairs4) {
        // an RGBA texel: two 2-channel reductions
        const long long base = A.offset + (long long)idx * 4;
        const uint32_t sb = texel_signs(ps, A.index, idx);
        if (CHK(S, base + 3, S.chk.params)) {
          atomicAdd(reinterpret_cast<float2*>(a.grad + base),
                    make_float2((sb & 1) ? -df : df, (sb & 2) ? -df : df));
          atomicAdd(reinterpret_cast<float2*>(a.grad + base + 2),
                    make_float2((sb & 4) ? -df : df, (sb & 8) ? -df : df));
        }
        continue;
      }
      for_each_signed_channel<false>(S, ps, kq, [&](long long p, int, bool neg) {
        if (!CHK(S, p, S.chk.params)) return;
        atomicAdd(a.grad + p, neg ? -df : df);
      });
    }
  }
  if (resident) {
    // every staged corner credited by some pixel: one count and one signed sum per channel
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nb) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint32_t n = sm.vn[t][k];
        if (!n) continue;
        const int v = sm.vid[t][k];
        if (CHK(S, v, ws.n_kcount)) atomicAdd(ws.kcount + v, n);
        const float A = sm.vA[t][k];
        if (A == 0.0f) continue;
        const uint32_t sb = vertex_signs(ps, v);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long q = 3ll * v + c;
          if (CHK(S, q, S.chk.params)) atomicAdd(a.grad + q, ((sb >> c) & 1) ? -A : A);
        }
      }
    }
  }
  if (a.loss) cta_add(lv / (float)a.pairs, sm.red, a.loss + slot);
}

// One render's deep lists and composite (side -1, 0 or +1); with loss, the image error of the
// render against the view's target is added to loss[slot].
__global__ void __launch_bounds__(TILE_PX) k_render_deep(SceneDev S, Workspace ws, int slot, int view, uint64_t key,
                                                         int side, unsigned long long* deep, float* rgb, float* loss) {
  __shared__ DeepSmem<1> sm;
  const int tile = blockIdx.x;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = threadIdx.x % TILE, dy = threadIdx.x / TILE;
  const int px = tx * TILE + dx, py = ty * TILE + dy;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  if (threadIdx.x < 16) sm.m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  unsigned long long L[1][K];
  int P[1][K];
  const int sides[1] = {side};
  const bool resident = deep_raster<1>(S, ws, sm, slot, tile, key, sides, L, P, rx, ry, dx, dy) <= DCHUNK;
  float f = 0.0f;
  if (px < S.W && py < S.H) {
    const long long npx = (long long)S.W * S.H, p = (long long)py * S.W + px;
    if (deep) {
#pragma unroll
      for (int j = 0; j < K; ++j) deep[j * npx + p] = L[0][j];
    }
    if (rgb || loss) {
      const float3 c = deep_composite(S, sm.m, key, side, L[0], P[0], resident ? sm.t[0] : nullptr, rx, ry, dx, dy,
                                      [](int, const Foot&, int, int) {});
      if (rgb) rgb[3 * p] = c.x, rgb[3 * p + 1] = c.y, rgb[3 * p + 2] = c.z;
      if (loss) {
        const float* tp = S.targets + ((long long)view * npx + p) * 3;
        const float d0 = c.x - __ldg(tp), d1 = c.y - __ldg(tp + 1), d2 = c.z - __ldg(tp + 2);
        f = d0 * d0 + d1 * d1 + d2 * d2;
      }
    }
  }
  if (loss) cta_add(f, sm.red, loss + slot);
}

}  // namespace

cudaError_t launch_deep_estimate(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                                 cudaStream_t st) {
  const int rows = vl.n * a.pair_count;
  for (int r0 = 0; r0 < rows; r0 += kDeepEstimates) {
    const int nr = rows - r0 < kDeepEstimates ? rows - r0 : kDeepEstimates;
    k_estimate_deep<<<dim3(n_tiles(S), nr), TILE_PX, 0, st>>>(S, ws, vl, a, r0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Every key's contributions of the call into the counts of its channels (each parameter belongs to
// one key: plain adds), and the key counts back to zero.
__global__ void k_expand_counts(SceneDev S, Workspace ws, uint32_t* counts) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ws.n_kcount) return;
  const uint32_t n = ws.kcount[j];
  if (n == 0) return;
  ws.kcount[j] = 0u;
  long long base = 3 * j;
  int nch = 3;
  if (j >= S.nv) {
    for (int k = 0; k < S.ntex; ++k)
      if (ws.kc_off[k] >= 0 && j >= ws.kc_off[k] && j < ws.kc_off[k] + (long long)S.tex[k].w * S.tex[k].h) {
        base = S.tex[k].offset + (j - ws.kc_off[k]) * S.tex[k].c;
        nch = S.tex[k].c;
      }
  }
  for (int c = 0; c < nch; ++c)
    if (CHK(S, base + c, S.chk.params)) counts[base + c] += n;
}

cudaError_t launch_expand_counts(const SceneDev& S, const Workspace& ws, uint32_t* counts, cudaStream_t st) {
  if (ws.n_kcount == 0) return cudaSuccess;
  k_expand_counts<<<(unsigned)((ws.n_kcount + 255) / 256), 256, 0, st>>>(S, ws, counts);
  return cudaGetLastError();
}

cudaError_t launch_render_deep(const SceneDev& S, const Workspace& ws, int slot, int view, uint64_t key, int side,
                               unsigned long long* deep, float* rgb, float* loss, cudaStream_t st) {
  k_render_deep<<<n_tiles(S), TILE_PX, 0, st>>>(S, ws, slot, view, key, side, deep, rgb, loss);
  return cudaGetLastError();
}

}  // namespace sge
