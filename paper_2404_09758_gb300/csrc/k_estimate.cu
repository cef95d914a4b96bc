// Fused, batched estimator for the tiles the fast kernel (k_fast.cu) cannot hold: more than
// kLightBin live triangles (dense meshes, poles, silhouettes seen edge-on).  With the fast kernel
// it runs every estimate of one iteration (views x antithetic pairs) in one persistent launch
// (Eq. 9, Algorithms 1-2, Section 4.3).
//
// Work item = (view, 16x16 tile, run of pairs).  A CTA owns one item at a time,
// one thread per pixel, and for every pair of its run:
//   P+R  sets up, in shared memory and a chunk of 256 at a time, both sides' versions of the
//        tile's live triangles from the vertex pass's projected perturbed vertices (nothing
//        perturbed is stored per pixel), and each thread tests its pixel's candidates (up to
//        kHeavyCand, listed by the pruning pass; more: every live triangle) for the visible
//        triangle on both sides (64-bit depth|id minimum);
//   G    shades both sides (UV buffer value, bilinear texels), forms
//        f+ - f- = sum_c (I+_c - I-_c)(I+_c + I-_c - 2 I_c) and credits it to the
//        union of both sides' contributing parameters.
// Credits go to a shared-memory hash table keyed by vertex / texel (one key per texel for all
// read textures when they share one size).  Within a pair all channels of a key share f+ - f-
// (only the sign s_i differs), so the table accumulates A_key = sum_p (f+ - f-) and n_key per
// pair, and once per pair folds s_i * A_key into per-channel sums.  At the end of the item each
// key issues one global atomic per channel for the sum and the count.  A table that fills up
// falls back to direct global atomics for the keys that do not fit.
#include <cuda_runtime.h>

#define SGE_FILE_ID 3  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

constexpr int BIN_CHUNK = 256;     // triangles staged per pass (one per thread)
// hash-table slots (power of two): unlit tiles credit one texture, the lit models up to four
template <int SH_LIT>
struct HeavyTable {
  static constexpr int SLOTS = SH_LIT ? 4096 : 2048;
};
constexpr int MAX_PROBE = 32;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;

struct SideSmem {
  long long e0[3][BIN_CHUNK];
  int a[3][BIN_CHUNK], b[3][BIN_CHUNK];
  int bias[BIN_CHUNK];  // bit k set: edge k is not top/left; bit 3: every edge function over the tile
                        // fits 32 bits (|a|, |b| < 2^16, |e0| < 2^29)
  float inv_area[BIN_CHUNK];
  float z[3][BIN_CHUNK], iw[3][BIN_CHUNK];
  int tri[BIN_CHUNK];  // -1 when not drawn on this side
};

template <int HT, int TSC>
struct TableSmem {
  uint32_t key[HT];
  float A[HT];
  uint32_t n[HT];
  float S[TSC][HT];  // channel sums: 4 per texture (4 x 4 for a texel group key)
  uint32_t cnt[HT];
};

template <int HT, int TSC>
struct Smem {
  SideSmem side[2];
  TableSmem<HT, TSC> tab;
  float m[16];
  float red[TILE_PX / 32];
  uint32_t item;
};

__device__ __forceinline__ void store_tri(SideSmem& s, int j, const Tri& t, int tri) {
  if (!t.ok) {
    s.tri[j] = -1;
    return;
  }
  int bias = 0;
  bool small = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.e0[k][j] = t.e0[k];
    s.a[k][j] = t.a[k];
    s.b[k][j] = t.b[k];
    s.z[k][j] = t.z[k];
    s.iw[k][j] = t.iw[k];
    bias |= (t.bias[k] ? 1 : 0) << k;
    // over the tile's pixel offsets (0..15) * 256: |a dx| + |b dy| < 2 * 2^28, so |e| < 2^30
    small = small && abs(t.a[k]) < (1 << 16) && abs(t.b[k]) < (1 << 16) && t.e0[k] > -(1ll << 29) &&
            t.e0[k] < (1ll << 29);
  }
  s.bias[j] = bias | (small ? 8 : 0);
  s.inv_area[j] = t.inv_area;
  s.tri[j] = tri;
}

__device__ __forceinline__ void load_tri(const SideSmem& s, int j, Tri& t) {
  int bias = s.bias[j];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    t.e0[k] = s.e0[k][j];
    t.a[k] = s.a[k][j];
    t.b[k] = s.b[k][j];
    t.z[k] = s.z[k][j];
    t.iw[k] = s.iw[k][j];
    t.bias[k] = (bias >> k) & 1 ? -1 : 0;
  }
  t.inv_area = s.inv_area[j];
  t.ok = 1;
}

// Coverage + depth of staged triangle j at pixel offset (dx, dy); returns the key or ~0.
__device__ __forceinline__ unsigned long long test_key(const SideSmem& s, int j, int dx, int dy) {
  int tri = s.tri[j];
  if (tri < 0) return ~0ull;
  int bias = s.bias[j];
  float l[3];
  bool in = true;
  if (bias & 8) {
    // the same integers in 32-bit arithmetic, and the same float conversions
    int e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e[k] = (int)s.e0[k][j] + s.a[k][j] * (dx * 256) + s.b[k][j] * (dy * 256);
      in = in && (e[k] - ((bias >> k) & 1) >= 0);
    }
    if (!in) return ~0ull;
#pragma unroll
    for (int k = 0; k < 3; ++k) l[k] = __fmul_rn(__int2float_rn(e[k]), s.inv_area[j]);
  } else {
    long long e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e[k] = s.e0[k][j] + (long long)s.a[k][j] * (dx * 256) + (long long)s.b[k][j] * (dy * 256);
      in = in && (e[k] - ((bias >> k) & 1) >= 0);
    }
    if (!in) return ~0ull;
    lambdas(e, s.inv_area[j], l);
  }
  float z[3] = {s.z[0][j], s.z[1][j], s.z[2][j]};
  float d = interp_depth(l, z);
  return ((unsigned long long)ordered_bits(d) << 32) | (uint32_t)tri;
}

template <int HT>
__device__ __forceinline__ uint32_t slot_hash(uint32_t k) {
  k ^= k >> 16;
  k *= 0x7feb352du;
  k ^= k >> 15;
  return k & (HT - 1);
}

// Credit df to key: shared-memory table, or global atomics when the table is full.
template <int HT, int TSC, bool GR>
__device__ __forceinline__ void credit(const SceneDev& S, TableSmem<HT, TSC>& tb, uint32_t key, float df,
                                       const PairSigns& ps, float* grad, uint32_t* counts) {
  uint32_t slot = slot_hash<HT>(key);
#pragma unroll 1
  for (int p = 0; p < MAX_PROBE; ++p) {
    uint32_t k = *(volatile uint32_t*)&tb.key[slot];
    if (k == EMPTY) k = atomicCAS(&tb.key[slot], EMPTY, key), k = (k == EMPTY) ? key : k;
    if (k == key) {
      atomicAdd(&tb.A[slot], df);
      atomicAdd(&tb.n[slot], 1u);
      return;
    }
    slot = (slot + 1) & (HT - 1);
  }
  for_each_signed_channel<GR>(S, ps, key, [&](long long p, int, bool neg) {
    if (!CHK(S, p, S.chk.params)) return;
    atomicAdd(grad + p, neg ? -df : df);
    atomicAdd(counts + p, 1u);
  });
}

// Fold the pair's per-key sums into the per-channel accumulators (signs of this pair).
template <int HT, int TSC, bool GR>
__device__ __forceinline__ void fold(const SceneDev& S, TableSmem<HT, TSC>& tb, const PairSigns& ps) {
  for (int slot = threadIdx.x; slot < HT; slot += blockDim.x) {
    uint32_t key = tb.key[slot];
    if (key == EMPTY) continue;
    uint32_t nn = tb.n[slot];
    if (nn == 0) continue;
    float A = tb.A[slot];
    for_each_signed_channel<GR>(S, ps, key, [&](long long, int c, bool neg) { tb.S[c][slot] += neg ? -A : A; });
    tb.cnt[slot] += nn;
    tb.A[slot] = 0.0f;
    tb.n[slot] = 0u;
  }
}

template <int HT, int TSC, bool GR>
__device__ __forceinline__ void flush_and_clear(const SceneDev& S, TableSmem<HT, TSC>& tb, float* grad,
                                                uint32_t* counts) {
  for (int slot = threadIdx.x; slot < HT; slot += blockDim.x) {
    uint32_t key = tb.key[slot];
    if (key != EMPTY) {
      const uint32_t cn = tb.cnt[slot];
      for_each_channel<GR>(S, key, [&](long long p, int c) {
        if (!CHK(S, p, S.chk.params)) return;
        atomicAdd(grad + p, tb.S[c][slot]);
        if (cn) atomicAdd(counts + p, cn);
      });
    }
    tb.key[slot] = EMPTY;
    tb.A[slot] = 0.0f;
    tb.n[slot] = 0u;
    tb.cnt[slot] = 0u;
#pragma unroll
    for (int c = 0; c < TSC; ++c) tb.S[c][slot] = 0.0f;
  }
}

// Triangle tri of side sd (0: theta + s eps, 1: theta - s eps) set up from the vertex pass's
// projected perturbed vertices of one (view slot, pair) (vb = its first vertex record).
__device__ __forceinline__ void setup_from_pverts(const SceneDev& S, const Workspace& ws, long long vb, int tri,
                                                  int sd, long long rx, long long ry, Tri& t) {
  PVert v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int4 q = __ldg(ws.pverts + 2 * (vb + vert_of(S, tri, k)) + sd);
    v[k].X = q.x;
    v[k].Y = q.y;
    v[k].z = __int_as_float(q.z);
    v[k].iw = __int_as_float(q.w);
    v[k].ok = q.x != kNotDrawn;
  }
  setup_tri(v[0], v[1], v[2], rx, ry, t);
}

// the batched kernels keep their asset after the kernel's own shared memory, 16-byte aligned
template <int HT, int TSC>
constexpr size_t heavy_batch_off() {
  return (sizeof(Smem<HT, TSC>) + 15) & ~(size_t)15;
}

template <int HT, int TSC>
__device__ __forceinline__ void clear_table(TableSmem<HT, TSC>& tb) {
  for (int s = threadIdx.x; s < HT; s += blockDim.x) {
    tb.key[s] = EMPTY;
    tb.A[s] = 0.0f;
    tb.n[s] = 0u;
    tb.cnt[s] = 0u;
#pragma unroll
    for (int c = 0; c < TSC; ++c) tb.S[c][s] = 0.0f;
  }
}

// Every heavy work item of one scene's call (the table starts and ends each item empty).
template <int HT, int TSC, bool GR>
__device__ __forceinline__ void heavy_items(const SceneDev& S, const Workspace& ws, const ViewList& vl,
                                            const EstimateArgs& a, Smem<HT, TSC>& sm) {
  const int tid = threadIdx.x;
  const int dx = tid % TILE, dy = tid / TILE;
  const int ntl = n_tiles(S);
  // heavy items cost many times a light one: a quarter of the run of pairs per work unit
  // spreads the few of them over more CTAs
  const int ppi = max(1, a.pairs_per_item / 4);
  const int n_chunks = (a.pair_count + ppi - 1) / ppi;
  const long long n_work = (long long)ws.counters[4] * n_chunks;
  const int n_all = vl.n * ntl;

  for (;;) {
    __syncthreads();
    if (tid == 0) sm.item = atomicAdd(ws.counters + 5, 1u);
    __syncthreads();
    const long long w = sm.item;
    if (w >= n_work) break;
    const uint32_t it = ws.items[n_all - 1 - (int)(w / n_chunks)];
    const int chunk = (int)(w % n_chunks);
    const int slot = it >> 24, tile = it & 0xFFFFFF;
    if (!CHK(S, slot, vl.n) || !CHK(S, tile, ntl)) continue;  // (checked build; uniform over the CTA)
    const int view = vl.id[slot];
    const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
    const int px = tx * TILE + dx, py = ty * TILE + dy;
    const bool valid = px < S.W && py < S.H;
    const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
    const uint32_t bin_beg = ws.tile_off[slot * ntl + tile];
    const int nb = (int)ws.tile_live[slot * ntl + tile];  // pruned and compacted by k_bin_prune
    const int p0 = a.pair_begin + chunk * ppi;
    const int p1 = min(a.pair_begin + a.pair_count, p0 + ppi);
    if (tid < 16) sm.m[tid] = S.mvp[16 * view + tid];
    float3 tgt = f3(0.f, 0.f, 0.f);
    if (valid) {
      const float* tp = S.targets + (((long long)view * S.H + py) * S.W + px) * 3;
      tgt = f3(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
    }
    float loss_acc = 0.0f;

    // this pixel's candidate triangles (16-bit indices into the live list, ascending; more than
    // kHeavyCand: test every live triangle)
    const long long ti = (long long)slot * ntl + tile;
    uint32_t cand[kHeavyCand / 2];
#pragma unroll
    for (int w = 0; w < kCandWords; ++w) {
      const int4 cw = ws.cand[(ti * kCandWords + w) * TILE_PX + tid];
      cand[4 * w] = (uint32_t)cw.x;
      cand[4 * w + 1] = (uint32_t)cw.y;
      cand[4 * w + 2] = (uint32_t)cw.z;
      cand[4 * w + 3] = (uint32_t)cw.w;
    }
    const int ncand = ws.ncand[ti * TILE_PX + tid];
    const bool all_live = ncand > kHeavyCand;

    for (int pair = p0; pair < p1; ++pair) {
      // the estimate's signs, from the vertex pass and the texel sign planes
      const PairSigns ps = pair_signs(S, ws, slot, pair - a.pair_begin);
      const long long vb = ((long long)slot * ws.max_pairs + (pair - a.pair_begin)) * S.nv;
      unsigned long long best[2] = {~0ull, ~0ull};
      int bestj[2] = {-1, -1}, bestc[2] = {-1, -1};
      int last_c = 0, q = 0;
      for (int c0 = 0; c0 < nb; c0 += BIN_CHUNK) {
        const int cnt = min(BIN_CHUNK, nb - c0);
        __syncthreads();
        if (tid < cnt) {
          const int tri = (int)bin_at(S, ws, bin_beg + c0 + tid);
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            Tri t;
            setup_from_pverts(S, ws, vb, tri, sd, rx, ry, t);
            store_tri(sm.side[sd], tid, t, tri);
          }
        }
        __syncthreads();
        auto test = [&](int j) {
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            unsigned long long k = test_key(sm.side[sd], j, dx, dy);
            if (k < best[sd]) {
              best[sd] = k;
              bestj[sd] = j;
              bestc[sd] = c0;
            }
          }
        };
        if (valid) {
          if (all_live) {
            for (int j = 0; j < cnt; ++j) test(j);
          } else {
            for (; q < ncand; ++q) {
              const int j = (int)((cand[q >> 1] >> (16 * (q & 1))) & 0xFFFFu) - c0;
              if (j >= cnt) break;
              if (!CHK(S, j, cnt)) continue;
              test(j);
            }
          }
        }
        last_c = c0;
      }

      // ---- G: shade both sides, loss difference, credits
      Surf sf[2];
      int tris[2] = {-1, -1};
      float3 col[2];
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        col[sd] = f3(S.bg[0], S.bg[1], S.bg[2]);
        if (!valid || best[sd] == ~0ull) continue;
        const int tri = (int)(best[sd] & 0xFFFFFFFFu);
        const int side = sd == 0 ? 1 : -1;
        Tri t;
        if (bestc[sd] == last_c) load_tri(sm.side[sd], bestj[sd], t);
        else setup_from_pverts(S, ws, vb, tri, sd, rx, ry, t);
        long long e[3];
        cover(t, dx, dy, e);
        surface_ps(S, view, tri, t, e, ps, side, sf[sd]);
        col[sd] = sf[sd].rgb;
        tris[sd] = tri;
      }
      float df = 0.0f;
      if (valid) {
        float fp, fm;
        df = loss_diff(col[0], col[1], tgt, fp, fm);
        loss_acc += 0.5f * (fp + fm);
        if (a.delta_f) a.delta_f[(((long long)slot * a.pairs + pair) * S.H + py) * S.W + px] = df;
        Foot foot[2][MAX_READ];
#pragma unroll
        for (int sd = 0; sd < 2; ++sd)
#pragma unroll
          for (int r = 0; r < MAX_READ; ++r) foot[sd][r] = sf[sd].foot[r];
        for_each_contrib<GR>(S, tris, foot,
                             [&](uint32_t key) { credit<HT, TSC, GR>(S, sm.tab, key, df, ps, a.grad, a.counts); });
      }
      __syncthreads();
      fold<HT, TSC, GR>(S, sm.tab, ps);
    }
    __syncthreads();
    flush_and_clear<HT, TSC, GR>(S, sm.tab, a.grad, a.counts);
    if (a.loss) {
      float v = loss_acc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) sm.red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        float sum = 0.0f;
        for (int i = 0; i < TILE_PX / 32; ++i) sum += sm.red[i];
        atomicAdd(a.loss + slot, sum / (float)a.pairs);
      }
    }
  }
}

template <int HT, int TSC, bool GR>
__global__ void __launch_bounds__(TILE_PX) k_estimate_heavy(SceneDev S, Workspace ws, ViewList vl, EstimateArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<HT, TSC>& sm = *reinterpret_cast<Smem<HT, TSC>*>(smem_raw);
  clear_table(sm.tab);
  heavy_items<HT, TSC, GR>(S, ws, vl, a, sm);
}

// Batched form: the assets of P in order, each until its heavy items run out (per-texture keys:
// the assets need not share texture sizes).
template <int HT>
__global__ void __launch_bounds__(TILE_PX) k_estimate_heavy_batch(const BatchArgs P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<HT, 4>& sm = *reinterpret_cast<Smem<HT, 4>*>(smem_raw);
  BatchSmem& b = *reinterpret_cast<BatchSmem*>(smem_raw + heavy_batch_off<HT, 4>());
  clear_table(sm.tab);
  for (int ai = 0; ai < P.n; ++ai) {
    __syncthreads();
    load_asset(P, ai, b);
    __syncthreads();
    heavy_items<HT, 4, false>(b.d.S, b.d.ws, b.vl, b.a, sm);
  }
}

__global__ void k_put_desc(const AssetDesc d, AssetDesc* dst) {
  const int4* src = reinterpret_cast<const int4*>(&d);
  int4* out = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(AssetDesc) / 16); i += blockDim.x) out[i] = src[i];
}

// Loss of pixels in tiles no triangle can reach: the background on both sides.
__global__ void k_background_loss(SceneDev S, Workspace ws, ViewList vl, float* loss) {
  const int slot = blockIdx.y, tile = blockIdx.x;
  const int ntl = n_tiles(S);
  if (ws.tile_count[slot * ntl + tile] != 0) return;
  const int view = vl.id[slot];
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int px = tx * TILE + threadIdx.x % TILE, py = ty * TILE + threadIdx.x / TILE;
  float v = 0.0f;
  if (px < S.W && py < S.H) {
    const float* tp = S.targets + (((long long)view * S.H + py) * S.W + px) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float d = S.bg[c] - tp[c];
      v += d * d;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0f) atomicAdd(loss + slot, v);
}

template <int HT, int TSC, bool GR>
int heavy_blocks_t() {
  int n = 0;
  cudaFuncSetAttribute(k_estimate_heavy<HT, TSC, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(Smem<HT, TSC>));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_estimate_heavy<HT, TSC, GR>, TILE_PX, sizeof(Smem<HT, TSC>));
  return n > 0 ? n : 1;
}

template <int HT>
int heavy_batch_blocks_t() {
  int n = 0;
  const int bytes = (int)(heavy_batch_off<HT, 4>() + sizeof(BatchSmem));
  cudaFuncSetAttribute(k_estimate_heavy_batch<HT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_estimate_heavy_batch<HT>, TILE_PX, bytes);
  return n > 0 ? n : 1;
}

// Table shapes: unlit 2,048 slots; lit 4,096 slots with per-texture keys, or texel-group keys
// when the read textures share one size: 1,024 slots of 12 channel sums when their channels add
// up to at most 12 (two CTAs fit an SM), else 2,048 slots of 16.
constexpr int kHtUnlit = HeavyTable<0>::SLOTS, kHtLit = HeavyTable<1>::SLOTS, kHtGroup = 2048, kHtGroupSmall = 1024;
constexpr int kGroupSmallChannels = 12;

}  // namespace

int group_channels(const SceneDev& S) {
  int n = 0;
  for (int r = 0; r < S.nread; ++r) n += S.rtex[r].c;
  return n;
}

namespace {

}  // namespace

int estimate_blocks_per_sm(int shading, int grouped, int group_ch) {
  if (shading == SHADE_UNLIT) return heavy_blocks_t<kHtUnlit, 4, false>();
  if (!grouped) return heavy_blocks_t<kHtLit, 4, false>();
  return group_ch <= kGroupSmallChannels ? heavy_blocks_t<kHtGroupSmall, kGroupSmallChannels, true>()
                                         : heavy_blocks_t<kHtGroup, 16, true>();
}

int heavy_batch_blocks_per_sm(int shading) {
  return shading == SHADE_UNLIT ? heavy_batch_blocks_t<kHtUnlit>() : heavy_batch_blocks_t<kHtLit>();
}

cudaError_t launch_put_desc(const AssetDesc& d, AssetDesc* dst, cudaStream_t st) {
  k_put_desc<<<1, 64, 0, st>>>(d, dst);
  return cudaGetLastError();
}

namespace {

template <int HT>
cudaError_t launch_heavy_batch_t(const BatchArgs& P, int grid, cudaStream_t st) {
  const int bytes = (int)(heavy_batch_off<HT, 4>() + sizeof(BatchSmem));
  cudaError_t e = cudaFuncSetAttribute(k_estimate_heavy_batch<HT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_estimate_heavy_batch<HT><<<grid, TILE_PX, bytes, st>>>(P);
  return cudaGetLastError();
}

template <int HT, int TSC, bool GR>
cudaError_t launch_heavy_t(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                           int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_estimate_heavy<HT, TSC, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(Smem<HT, TSC>));
  if (e != cudaSuccess) return e;
  k_estimate_heavy<HT, TSC, GR><<<grid, TILE_PX, sizeof(Smem<HT, TSC>), st>>>(S, ws, vl, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_heavy_batch(const BatchArgs& P, int shading, int grid, cudaStream_t st) {
  return shading == SHADE_UNLIT ? launch_heavy_batch_t<kHtUnlit>(P, grid, st) : launch_heavy_batch_t<kHtLit>(P, grid, st);
}

cudaError_t launch_estimate(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                            int grid_fast, int grid_heavy, cudaStream_t st, const cudaEvent_t* ev_fast) {
  cudaError_t e = ev_fast ? cudaEventRecord(ev_fast[0], st) : cudaSuccess;
  if (e == cudaSuccess) e = launch_fast(S, ws, vl, a, grid_fast, st);
  if (e == cudaSuccess && ev_fast) e = cudaEventRecord(ev_fast[1], st);
  if (e != cudaSuccess) return e;
  if (S.shading == SHADE_UNLIT) e = launch_heavy_t<kHtUnlit, 4, false>(S, ws, vl, a, grid_heavy, st);
  else if (S.grouped && group_channels(S) <= kGroupSmallChannels)
    e = launch_heavy_t<kHtGroupSmall, kGroupSmallChannels, true>(S, ws, vl, a, grid_heavy, st);
  else if (S.grouped) e = launch_heavy_t<kHtGroup, 16, true>(S, ws, vl, a, grid_heavy, st);
  else e = launch_heavy_t<kHtLit, 4, false>(S, ws, vl, a, grid_heavy, st);
  if (e == cudaSuccess && ev_fast) e = cudaEventRecord(ev_fast[2], st);
  if (e != cudaSuccess) return e;
  if (a.loss && a.pair_begin == 0) k_background_loss<<<dim3(n_tiles(S), vl.n), TILE_PX, 0, st>>>(S, ws, vl, a.loss);
  return cudaGetLastError();
}

cudaError_t launch_background_loss(const SceneDev& S, const Workspace& ws, const ViewList& vl, float* loss,
                                   cudaStream_t st) {
  k_background_loss<<<dim3(n_tiles(S), vl.n), TILE_PX, 0, st>>>(S, ws, vl, loss);
  return cudaGetLastError();
}

}  // namespace sge
