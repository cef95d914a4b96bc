// Batched estimator, fast path: tiles that keep at most kLightBin live triangles after pruning,
// and the pruning pass itself.
//
// Once per call and (view, tile), k_bin_prune: the bin's triangles are set up unperturbed; a
// triangle stays live if some pixel of the tile may see it under SOME perturbation of the call
// (each edge function pushed out by the triangle's margin: the support of the box every snapped
// perturbed vertex stays in) and it is not surely behind a triangle that surely covers the pixel
// (farther than the largest vertex move from each of its edges, so every perturbed version still
// covers it, and depth intervals apart).  Live triangles are compacted to the front of the bin;
// each pixel's candidates among them (at most CMAX; more: test them all) are stored, so that a
// pair tests a handful of triangles, not the bin.
//
// Work item = (view, 16x16 tile, run of antithetic pairs); one CTA thread per pixel.
// Per pair (Eq. 8 for one sign vector s, Algorithms 1-2):
//   F+S the previous pair's credits are folded into per-channel sums with that
//       pair's signs; the live triangles are set up on both sides (theta + s eps,
//       theta - s eps) in shared memory from the projected perturbed vertices of
//       the vertex pass (k_vertex.cu), with their 9 coordinate signs;
//   R   each pixel finds its visible triangle on both sides among its candidates
//       (smallest packed depth|id key);
//   U   it computes both sides' UV and inserts the texels of their bilinear
//       footprints into a shared-memory table (one key per texel for all read textures
//       when they share one size); the first pixel to touch a texel in the pair draws
//       the pair's signs of its channels;
//   G   it samples its perturbed texels (signs from the table), shades both sides,
//       forms f+ - f- and credits it: the visible triangle (all three vertices at
//       once, or single corners where the sides disagree) and the union of the
//       texel footprints.
// At the end of the item every credited vertex corner and texel issues one global
// atomic per channel for its sum and its count.
#include <cuda_runtime.h>

#define SGE_FILE_ID 4  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

constexpr int NB = kLightBin;
constexpr int CMAX = 16;  // candidate triangles kept per pixel
constexpr int MAX_PROBE = 16;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t NOSLOT = 0xFFFFu;

// GR: the read textures share one size, so every pixel's bilinear footprint is the same texels
// in all of them and one table entry (keyed by texel) carries all their channels.
template <int SH, bool GR = false>
struct Model {
  static constexpr int NREAD = SH == SHADE_UNLIT ? 1 : (SH == SHADE_LAMBERT ? 2 : 4);
  // footprints computed and inserted per side: one for a group, one per texture otherwise
  static constexpr int NFOOT = GR ? 1 : NREAD;
  // a tile's bilinear footprints over a run of pairs hold a few hundred texels at about one
  // texel per pixel, more where the surface is seen at a grazing angle
  static constexpr int TABLE = (SH == SHADE_UNLIT || GR) ? 1024 : 2048;
  static constexpr int TSC = GR ? 4 * NREAD : 4;  // channel sums per table entry
  // one footprint per side (unlit, texel groups): the table's first WCAP slots can hold an item's
  // texel window, indexed directly; the rest stay hashed for footprints outside it
  static constexpr bool DIRECT = NFOOT == 1;
  // one read texture: a footprint outside the window credits the global sums directly (its
  // texels are rarely shared with other pixels there, and hashing costs more than it saves), so
  // the window may take the whole table; texel groups keep a hashed quarter (a global credit
  // would cost one atomic per channel of every grouped texture)
  static constexpr bool HASH_OUTSIDE = NREAD > 1;
  static constexpr int WCAP = HASH_OUTSIDE ? TABLE * 3 / 4 : TABLE;
};

// A bin triangle's unperturbed edge functions for the pruning pass, with its margin; 64 bytes.
struct __align__(16) TriS {
  long long e0[3];  // oriented edge functions at the tile's first pixel centre
  int a[3], b[3];   // oriented edge steps per fixed-point unit in x and y
  int tri;          // triangle id; -2: not drawable unperturbed, so always a candidate
  int margin;       // perturbation margin, fixed-point units
  int small;        // the pruning tests fit 32 bits: |a|, |b| < 2^16, |e0| < 2^29, margin < 2^10
  int pad;
};

// One side of a live triangle set up for one pair of the estimator (the triangle's id is the
// item's btri[]); 80 bytes.
struct __align__(16) SideTri {
  long long e0[3];  // oriented edge functions at the tile's first pixel centre
  int a[3], b[3];   // oriented edge steps per fixed-point unit in x and y
  int flags;        // bits 0-2: edge k is not a top/left edge; bit 3: drawn on this side; bit 4: every
                    // edge function over the tile fits 32 bits (|a|, |b| < 2^16, |e0| < 2^29)
  float inv_area;
  float z[3], iw[3];
};
static_assert(sizeof(SideTri) == 80, "SideTri layout");
constexpr int kDrawn = 8, kSmall = 16;

template <int TABLE, int TSC>
struct FastSmem {
  SideTri side[2][NB];
  float uv[NB][6];
  int vid[NB][3];
  int btri[NB];          // triangle id of each live entry
  uint32_t zminb[NB];    // ordered bits of its smallest depth under any perturbation of the call
  uint32_t sgn9[2][NB];  // bit 3k+c: coordinate c of corner k has s = -1 (by pair parity)
  float A_tri[NB];
  uint32_t n_tri[NB];
  float A_cor[NB][3];
  uint32_t n_cor[NB][3];
  float S_cor[NB][3][3];
  uint32_t c_cor[NB][3];
  uint32_t tkey[TABLE];
  float tA[TABLE];       // the current pair's sum of f+ - f- over the pixels crediting the entry
  float tS[TSC][TABLE];
  uint32_t tcnt[TABLE];
  uint32_t tsb[TABLE];   // the current pair's sign bits of the entry's channels (4 r + c), stored by
                         // every pixel that samples the texel (all store the same value)
  uint16_t used[TABLE];  // slots holding a key in this item, in insertion order
  uint32_t n_used;
  int win[4];            // the item's texel window: x (before wrapping) from win[0] to win[1], rows
                         // win[2] to win[3]; slot (y - win[2]) * width + x - win[0]
  uint32_t n_win;        // its slots (the first entries of used[]), 0 without a window
  float m[16];
  float red[TILE_PX / 32];
  uint32_t item;
};

// Two unlit CTAs share an SM: 228 KB of shared memory less 1 KB reserved per CTA.
static_assert(2 * (sizeof(FastSmem<Model<SHADE_UNLIT>::TABLE, Model<SHADE_UNLIT>::TSC>) + 1024) <= 228 * 1024,
              "the unlit fast estimator must fit two CTAs per SM");

__device__ __forceinline__ void store_side_tri(SideTri& d, const Tri& t) {
  if (!t.ok) {
    d.flags = 0;
    return;
  }
  int flags = kDrawn;
  bool small = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d.e0[k] = t.e0[k];
    d.a[k] = t.a[k];
    d.b[k] = t.b[k];
    d.z[k] = t.z[k];
    d.iw[k] = t.iw[k];
    flags |= (t.bias[k] ? 1 : 0) << k;
    // over the tile's pixel offsets (0..15) * 256: |a dx| + |b dy| < 2 * 2^28, so |e| < 2^30
    small = small && abs(t.a[k]) < (1 << 16) && abs(t.b[k]) < (1 << 16) && t.e0[k] > -(1ll << 29) &&
            t.e0[k] < (1ll << 29);
  }
  d.flags = flags | (small ? kSmall : 0);
  d.inv_area = t.inv_area;
}

// Exact coverage at pixel offset (dx, dy) and the barycentric weights lambda_k = E_k / area there
// (as lambdas() forms them): 32-bit edge functions for a small triangle, 64-bit otherwise; the
// integers are the same, and so is each float conversion.
__device__ __forceinline__ bool cover_lambdas(const SideTri& t, int dx, int dy, float l[3]) {
  bool in = true;
  if (t.flags & kSmall) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = (int)t.e0[k] + t.a[k] * (dx * 256) + t.b[k] * (dy * 256);
      in = in && (e - ((t.flags >> k) & 1) >= 0);
      l[k] = __fmul_rn(__int2float_rn(e), t.inv_area);
    }
  } else {
    long long e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e[k] = t.e0[k] + (long long)t.a[k] * (dx * 256) + (long long)t.b[k] * (dy * 256);
      in = in && (e[k] - ((t.flags >> k) & 1) >= 0);
    }
    lambdas(e, t.inv_area, l);
  }
  return in;
}

__device__ __forceinline__ uint32_t hslot(uint32_t k, int table) {
  k ^= k >> 16;
  k *= 0x7feb352du;
  k ^= k >> 15;
  return k & (uint32_t)(table - 1);
}

// Find or insert a texel key in the hashed slots [hbase, hbase + hsize) (hsize a power of two;
// keys stay for the whole item; a new one is listed in used[]).
template <int TABLE, int TSC>
__device__ __forceinline__ uint32_t table_insert(FastSmem<TABLE, TSC>& sm, uint32_t key, uint32_t hbase,
                                                 uint32_t hsize) {
  uint32_t h = hslot(key, hsize);
#pragma unroll 1
  for (int p = 0; p < MAX_PROBE; ++p) {
    const uint32_t slot = hbase + h;
    uint32_t k = *(volatile uint32_t*)&sm.tkey[slot];
    if (k == EMPTY) {
      k = atomicCAS(&sm.tkey[slot], EMPTY, key);
      if (k == EMPTY) {
        sm.used[atomicAdd(&sm.n_used, 1u)] = (uint16_t)slot;
        return slot;
      }
    }
    if (k == key) return slot;
    h = (h + 1) & (hsize - 1);
  }
  return NOSLOT;
}

// Texel id of footprint corner q from the packed (x0,y0) id and its edge flags.
__device__ __forceinline__ int texel_of(uint32_t pk, int q, int w) {
  int t = (int)(pk & 0x3FFFFFFFu);
  if (q & 1) t += (pk & (1u << 30)) ? -(w - 1) : 1;
  if ((q & 2) && !(pk & (1u << 31))) t += w;
  return t;
}

// Sign bits of texel t's channels (bit c: s = -1) in one texture's sign plane of an estimate.
__device__ __forceinline__ uint32_t plane_nibble(const SceneDev& S, const uint32_t* planes, int off, int t) {
  const long long w = (long long)off + (t >> 3);
  if (!CHK(S, w, S.chk.sign_words)) return 0u;
  return (__ldg(planes + w) >> (4 * (t & 7))) & 0xFu;
}

// Every slot of the table empty (once per call of the estimator loop in a CTA).
template <int TABLE, int TSC>
__device__ __forceinline__ void clear_table(FastSmem<TABLE, TSC>& sm) {
  for (int s = threadIdx.x; s < TABLE; s += blockDim.x) {
    sm.tkey[s] = EMPTY;
    sm.tA[s] = 0.0f;
    sm.tcnt[s] = 0u;
    sm.tsb[s] = 0u;
#pragma unroll
    for (int c = 0; c < TSC; ++c) sm.tS[c][s] = 0.0f;
  }
  if (threadIdx.x == 0) sm.n_used = 0;
}

// The n_used slots an item used back to empty (after its flush).
template <int TABLE, int TSC>
__device__ __forceinline__ void clear_used(FastSmem<TABLE, TSC>& sm, uint32_t n_used) {
  for (uint32_t i = threadIdx.x; i < n_used; i += blockDim.x) {
    const uint32_t s = sm.used[i];
    sm.tkey[s] = EMPTY;
    sm.tA[s] = 0.0f;
    sm.tcnt[s] = 0u;
#pragma unroll
    for (int c = 0; c < TSC; ++c) sm.tS[c][s] = 0.0f;
  }
}

// Fold a pair's credits (table entries and triangle corners) into the per-channel sums with
// that pair's signs: texel signs in tsb (stored while sampling), vertex signs in sgn9[parity].
// A table entry's counts go straight to tcnt when it is credited; an entry whose pair sum is
// exactly zero is skipped (adding +-0 leaves every sum as it is).
template <int TABLE, int TSC, bool GR, int NREAD>
__device__ __forceinline__ void fold(const SceneDev& S, FastSmem<TABLE, TSC>& sm, int nb, int parity) {
  // the item's keys only (the used list, whose first n_win entries are the window's slots 0, 1, ...
  // in order: those are swept directly, lane i on slot i)
  const uint32_t n_used = sm.n_used, n_win = sm.n_win;
  for (uint32_t i = threadIdx.x; i < n_used; i += blockDim.x) {
    const uint32_t s = i < n_win ? i : sm.used[i];
    const float A = sm.tA[s];
    if (A == 0.0f) continue;
    const uint32_t sbits = sm.tsb[s];
    if (!GR) {
      const int cn = NREAD == 1 ? S.rtex[0].c : S.tex[(sm.tkey[s] >> 28) - 1].c;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < cn) sm.tS[c][s] += ((sbits >> c) & 1) ? -A : A;
    } else {
      // group entry: channel c of read texture r at 4 r + c
#pragma unroll
      for (int r = 0; r < NREAD; ++r) {
        const int cn = S.rtex[r].c;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < cn) sm.tS[4 * r + c][s] += ((sbits >> (4 * r + c)) & 1) ? -A : A;
      }
    }
    sm.tA[s] = 0.0f;
  }
  const int j = threadIdx.x;
  if (j < nb) {
    const uint32_t sg = sm.sgn9[parity][j];
    const float at = sm.A_tri[j];
    const uint32_t nt = sm.n_tri[j];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float a = at + sm.A_cor[j][k];
      const uint32_t n = nt + sm.n_cor[j][k];
      if (n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.S_cor[j][k][c] += ((sg >> (3 * k + c)) & 1) ? -a : a;
        sm.c_cor[j][k] += n;
      }
      sm.A_cor[j][k] = 0.0f;
      sm.n_cor[j][k] = 0u;
    }
    sm.A_tri[j] = 0.0f;
    sm.n_tri[j] = 0u;
  }
}

// Sum of v over the run of consecutive lanes (in lane order) that share key k, for the run's
// last lane; every lane of the warp calls it.  Returns whether the lane ends its run and sets n
// to the run's length.
__device__ __forceinline__ bool run_sum(int k, float& v, int& n) {
  const int lane = threadIdx.x & 31;
  const int kp = __shfl_up_sync(0xffffffffu, k, 1);
  const int kn = __shfl_down_sync(0xffffffffu, k, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || kp != k);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane - d >= start) v += o;
  }
  n = lane - start + 1;
  return lane == 31 || kn != k;
}

// ---------------------------------------------------------------- bin pruning
// Unperturbed set-up of a bin triangle with its perturbation margin and depth interval; a
// triangle not drawable unperturbed (zero area, a vertex behind the near limit) gets tri = -2:
// a perturbed version may still be drawable, so it is a candidate everywhere.  reach[k]: how far
// (edge-function units) a pixel must lie inside edge k to stay inside under every perturbation;
// each vertex moves at most margin per axis, so at most sqrt(2) margin (+ slack); -1: never sure.
__device__ __forceinline__ void stage_unperturbed(const SceneDev& S, const Workspace& ws, const float* m, int slot,
                                                  int tri, long long rx, long long ry, TriS& d, float2& zr,
                                                  long long (&reach)[3], uint32_t (&span)[2]) {
  PVert v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float3 q = perturbed_pos(S, vert_of(S, tri, k), 0, 0);
    v[k] = project(m, q.x, q.y, q.z, S.W, S.H, S.near_w);
  }
  Tri t;
  setup_tri(v[0], v[1], v[2], rx, ry, t);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d.e0[k] = t.e0[k];
    d.a[k] = t.a[k];
    d.b[k] = t.b[k];
  }
  d.tri = t.ok ? tri : -2;
  d.margin = ws.tri_margin[(long long)slot * S.nt + tri];
  zr = ws.tri_z[(long long)slot * S.nt + tri];
  const bool can = d.tri >= 0 && d.margin != 0x7FFFFFFF;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    long long r = -1;
    if (can) {
      const float fa = (float)d.a[k], fb = (float)d.b[k];
      r = (long long)ceilf(1.41422f * (float)d.margin * sqrtf(fa * fa + fb * fb) * 1.0001f + 2.0f);
    }
    reach[k] = r;
  }
  // pixels that may pass surely_covers (inside the triangle) and maybe_visible (inside its edges
  // pushed out by the margin terms); a triangle those tests always fail / pass: none / all
  if (can) {
    span[0] = box_span(v, rx, ry, 0);
    span[1] = box_span(v, rx, ry, d.margin);
  } else {
    span[0] = 0u;
    span[1] = 0xFFFFFFFFu;
  }
  // over the tile (offsets 0..15 * 256) |e| < 2^30 and the margin terms stay below 2^28
  bool small = can && d.margin < (1 << 10);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    small = small && abs(d.a[k]) < (1 << 16) && abs(d.b[k]) < (1 << 16) && d.e0[k] > -(1ll << 29) &&
            d.e0[k] < (1ll << 29);
  d.small = small;
}

// Does every perturbed version of t cover pixel (dx, dy)?  (exact integer comparisons against the
// staged reach)
__device__ __forceinline__ bool surely_covers(const TriS& t, const long long (&reach)[3], int dx, int dy) {
  if (reach[0] < 0) return false;
  bool sure = true;
  if (t.small) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = (int)t.e0[k] + t.a[k] * (dx * 256) + t.b[k] * (dy * 256);
      sure = sure && e > (int)reach[k];
    }
    return sure;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long e = t.e0[k] + (long long)t.a[k] * (dx * 256) + (long long)t.b[k] * (dy * 256);
    sure = sure && e > reach[k];
  }
  return sure;
}

// Can some perturbed version of t be the visible triangle at pixel (dx, dy)?  No if its
// margin-widened edge functions miss the pixel, or if it lies entirely behind the far end of
// a triangle that surely covers the pixel (zsure).
__device__ __forceinline__ bool maybe_visible(const TriS& t, float2 zr, float zsure, int dx, int dy) {
  if (t.tri == -2 || t.margin == 0x7FFFFFFF) return true;
  bool maybe = true;
  if (t.small) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = (int)t.e0[k] + t.a[k] * (dx * 256) + t.b[k] * (dy * 256);
      maybe = maybe && (e + t.margin * (abs(t.a[k]) + abs(t.b[k])) >= 0);
    }
    return maybe && zr.x <= zsure;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long e = t.e0[k] + (long long)t.a[k] * (dx * 256) + (long long)t.b[k] * (dy * 256);
    const long long reach = (long long)t.margin * (long long)(abs(t.a[k]) + abs(t.b[k]));
    maybe = maybe && (e + reach >= 0);
  }
  return maybe && zr.x <= zsure;
}

struct PruneSmem {
  TriS t[NB];
  float2 zr[NB];
  long long reach[NB][3];
  uint32_t id[NB];
  uint8_t live[NB];
  uint16_t remap[NB];  // compacted position of each live entry of a single-chunk bin
  uint16_t cl[kHeavyCand][TILE_PX];  // each pixel's first kHeavyCand candidates (column per pixel)
  uint32_t span[NB][2];  // tile_span of the sure-cover and the maybe-visible regions
  float m[16];
  int wsum[TILE_PX / 32];
};

// Exclusive prefix of flag over the CTA (256 threads); returns this thread's position and
// the total in *total.
__device__ __forceinline__ int block_prefix(int flag, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(b & ((1u << lane) - 1u));
  __syncthreads();
  if (lane == 0) wsum[wid] = __popc(b);
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < TILE_PX / 32; ++w) {
    before += w < wid ? wsum[w] : 0;
    all += wsum[w];
  }
  *total = all;
  return before + in_warp;
}

// Store a pixel's list (its column of cl, n entries found): 8-bit indices (light tile, the first
// CMAX, in ascending order of the triangles' smallest depth under any perturbation, zr(j) of live
// index j, ties in list order) or 16-bit ones (the first kHeavyCand, in list order), and its
// length min(n, 255).
template <typename ZR>
__device__ __forceinline__ void store_cands(const Workspace& ws, long long tile_index, int tid,
                                            const uint16_t (*cl)[TILE_PX], int n, bool wide, ZR&& zr) {
  const long long ci = tile_index * kCandWords * TILE_PX + tid;
  if (wide) {
    const int k = min(n, kHeavyCand);
#pragma unroll
    for (int w = 0; w < kCandWords; ++w) {
      uint32_t v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 8 * w + 2 * i;
        v[i] = (q < k ? (uint32_t)cl[q][tid] : 0u) | (q + 1 < k ? (uint32_t)cl[q + 1][tid] << 16 : 0u);
      }
      ws.cand[ci + w * TILE_PX] = make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]);
    }
  } else {
    // each entry goes to its rank in depth order: the estimator stops at the first candidate
    // that lies wholly behind the nearest covering triangle found so far.  The order compares
    // the depths' ordered bits (a total order, NaN included: a float compare would give two
    // entries one rank) with ties broken by list position, so the ranks are a permutation.
    const int k = min(n, CMAX);
    uint32_t b[CMAX / 4] = {};
    for (int q = 0; q < k; ++q) {
      const uint32_t j = cl[q][tid];
      const uint32_t zj = ordered_bits(zr(j));
      int rank = 0;
      for (int r = 0; r < k; ++r) {
        const uint32_t zo = ordered_bits(zr((uint32_t)cl[r][tid]));
        rank += (zo < zj || (zo == zj && r < q)) ? 1 : 0;
      }
      const uint32_t bits = j << (8 * (rank & 3));
#pragma unroll
      for (int i = 0; i < CMAX / 4; ++i) b[i] |= (rank >> 2) == i ? bits : 0u;
    }
    ws.cand[ci] = make_int4((int)b[0], (int)b[1], (int)b[2], (int)b[3]);
  }
  ws.ncand[tile_index * TILE_PX + tid] = (uint8_t)min(n, 255);
}

// Per (view slot, tile): drop from the bin every triangle that no perturbation of the call can
// make visible at any pixel of the tile (outside all margin-widened pixel tests, or behind a
// triangle that surely covers the pixel), compact the rest to the front of the bin's range,
// record their number in tile_live and list the tile as a light item (<= light_bin live
// triangles) or a heavy one, and store each pixel's candidate triangles in cand/ncand (light:
// up to CMAX 8-bit live indices; heavy: up to kHeavyCand 16-bit ones).  The pruned triangles
// never change any render of the call in this tile.
__device__ __forceinline__ void prune_tile(const SceneDev& S, const Workspace& ws, int n_views, int view, int slot,
                                           int tile, int light_bin, PruneSmem& sm) {
  const int tid = threadIdx.x;
  const int ntl = n_tiles(S), n_all = n_views * ntl;
  if ((long long)ws.tile_off[n_all] > ws.bin_capacity) return;  // overflow: the bins were not stored
  const uint32_t beg = ws.tile_off[slot * ntl + tile];
  const int nb = (int)(ws.tile_off[slot * ntl + tile + 1] - beg);
  if (nb == 0) return;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int dx = tid % TILE, dy = tid / TILE;
  const bool valid = tx * TILE + dx < S.W && ty * TILE + dy < S.H;
  const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
  const long long tix = (long long)slot * ntl + tile;
  if (tid < 16) sm.m[tid] = S.mvp[16 * view + tid];
  __syncthreads();
  auto stage = [&](int c0, int cnt, bool from_live) {
    if (tid < cnt) {
      const int tri = (int)bin_at(S, ws, beg + c0 + tid);
      sm.id[tid] = (uint32_t)tri;
      stage_unperturbed(S, ws, sm.m, slot, tri, rx, ry, sm.t[tid], sm.zr[tid], sm.reach[tid], sm.span[tid]);
      if (!from_live) sm.live[tid] = 0;
    }
  };
  // pass 1: nearest far end of the triangles that surely cover this pixel
  float zsure = 3.4e38f;
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int cnt = min(NB, nb - c0);
    __syncthreads();
    stage(c0, cnt, false);
    __syncthreads();
    for (int j = 0; j < cnt; ++j)
      if (in_span(sm.span[j][0], dx, dy) && surely_covers(sm.t[j], sm.reach[j], dx, dy))
        zsure = fminf(zsure, sm.zr[j].y);
  }
  // pass 2: mark and compact the triangles some pixel may see (a single chunk is still staged;
  // its pixels' candidate lists are found on the way, by bin position, and renumbered below)
  const bool single = nb <= NB;
  int n_cl = 0;  // candidates found for this pixel (the first kHeavyCand kept in sm.cl)
  int n_live = 0;
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int cnt = min(NB, nb - c0);
    if (!single) {
      __syncthreads();
      stage(c0, cnt, false);
    }
    __syncthreads();
    if (valid) {
      if (single) {
        for (int j = 0; j < cnt; ++j)
          if (in_span(sm.span[j][1], dx, dy) && maybe_visible(sm.t[j], sm.zr[j], zsure, dx, dy)) {
            sm.live[j] = 1;
            if (n_cl < kHeavyCand) sm.cl[n_cl][tid] = (uint16_t)j;
            ++n_cl;
          }
      } else {
        for (int j = 0; j < cnt; ++j)
          if (!sm.live[j] && in_span(sm.span[j][1], dx, dy) && maybe_visible(sm.t[j], sm.zr[j], zsure, dx, dy))
            sm.live[j] = 1;
      }
    }
    __syncthreads();
    const int f = tid < cnt ? sm.live[tid] : 0;
    int total;
    const int pos = block_prefix(f, sm.wsum, &total);
    // positions only move towards the front, past entries this CTA has already read
    if (f) {
      if (CHK(S, (long long)beg + n_live + pos, S.chk.bins)) ws.bins[beg + n_live + pos] = sm.id[tid];
      if (single) sm.remap[tid] = (uint16_t)pos;
    }
    n_live += total;
  }
  if (tid == 0) {
    ws.tile_live[tix] = (uint32_t)n_live;
    const uint32_t it = ((uint32_t)slot << 24) | (uint32_t)tile;
    if (n_live <= light_bin) ws.items[atomicAdd(ws.counters + 0, 1u)] = it;
    else ws.items[n_all - 1 - (int)atomicAdd(ws.counters + 4, 1u)] = it;
  }
  const bool wide = n_live > light_bin;  // heavy tile: 16-bit indices
  if (single) {
    __syncthreads();
    // bin positions -> live indices (each pixel renumbers its own column)
    const int k = min(n_cl, kHeavyCand);
    for (int q = 0; q < k; ++q) sm.cl[q][tid] = sm.remap[sm.cl[q][tid]];
    // live index -> bin position of the staged chunk, for the depth order
    if (tid < nb && sm.live[tid]) sm.id[sm.remap[tid]] = (uint32_t)tid;
    __syncthreads();
    store_cands(ws, tix, tid, sm.cl, n_cl, wide, [&](uint32_t j) { return sm.zr[sm.id[j]].x; });
    return;
  }
  // pass 3 (bins of more than one chunk): each pixel's candidates among the live triangles, in
  // their compacted order, a chunk of live triangles at a time (ascending)
  for (int c0 = 0; c0 < n_live; c0 += NB) {
    const int cnt = min(NB, n_live - c0);
    __syncthreads();
    stage(c0, cnt, true);
    __syncthreads();
    if (valid)
      for (int j = 0; j < cnt; ++j)
        if (in_span(sm.span[j][1], dx, dy) && maybe_visible(sm.t[j], sm.zr[j], zsure, dx, dy)) {
          if (n_cl < kHeavyCand) sm.cl[n_cl][tid] = (uint16_t)(c0 + j);
          ++n_cl;
        }
  }
  // a light tile's live triangles are one staged chunk here, indexed by live position
  store_cands(ws, tix, tid, sm.cl, n_cl, wide, [&](uint32_t j) { return sm.zr[j].x; });
}

__global__ void __launch_bounds__(TILE_PX, 4) k_bin_prune(SceneDev S, Workspace ws, ViewList vl) {
  __shared__ PruneSmem sm;
  prune_tile(S, ws, vl.n, vl.id[blockIdx.y], blockIdx.y, blockIdx.x, ws.light_bin, sm);
}

// Batched form: every (tile, view slot, asset) of a batched call in one launch; each CTA reads
// its asset's scene and workspace from the asset's launch descriptor in device memory.
__global__ void __launch_bounds__(TILE_PX, 4) k_bin_prune_batch(const BatchArgs P) {
  __shared__ PruneSmem sm;
  const BatchAsset& A = P.as[blockIdx.z];
  const int slot = blockIdx.y;
  if (slot >= A.n_views) return;
  const AssetDesc& D = *A.desc;
  if ((int)blockIdx.x >= D.S.tiles_x * D.S.tiles_y) return;
  prune_tile(D.S, D.ws, A.n_views, A.view[slot], slot, blockIdx.x, P.light_bin, sm);
}

// Every light work item of one scene's call, taken one at a time from the scene's work
// counter until none is left.
template <int SH, bool GR>
__device__ __forceinline__ void fast_items(const SceneDev& S, const Workspace& ws, const ViewList& vl,
                                           const EstimateArgs& a,
                                           FastSmem<Model<SH, GR>::TABLE, Model<SH, GR>::TSC>& sm) {
  constexpr int NREAD = Model<SH, GR>::NREAD;
  constexpr int NFOOT = Model<SH, GR>::NFOOT;
  constexpr int TABLE = Model<SH, GR>::TABLE;
  constexpr int TSC = Model<SH, GR>::TSC;
  const int tid = threadIdx.x;
  const int dx = tid % TILE, dy = tid / TILE;
  const int ntl = n_tiles(S);
  const int n_chunks = (a.pair_count + a.pairs_per_item - 1) / a.pairs_per_item;
  const long long n_work = (long long)ws.counters[0] * n_chunks;
  clear_table(sm);

  for (;;) {
    __syncthreads();
    if (tid == 0) sm.item = atomicAdd(ws.counters + 1, 1u);
    __syncthreads();
    const long long w = sm.item;
    if (w >= n_work) break;
    const uint32_t it = ws.items[w / n_chunks];
    const int chunk = (int)(w % n_chunks);
    const int slot = it >> 24, tile = it & 0xFFFFFF;
    if (!CHK(S, slot, vl.n) || !CHK(S, tile, ntl)) continue;  // (checked build; uniform over the CTA)
    const int view = vl.id[slot];
    const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
    const int px = tx * TILE + dx, py = ty * TILE + dy;
    const bool valid = px < S.W && py < S.H;
    const long long rx = 256ll * (tx * TILE) + 128, ry = 256ll * (ty * TILE) + 128;
    const uint32_t bin_beg = ws.tile_off[slot * ntl + tile];
    const int nb = (int)ws.tile_live[slot * ntl + tile];
    const int p0 = a.pair_begin + chunk * a.pairs_per_item;
    const int p1 = min(a.pair_begin + a.pair_count, p0 + a.pairs_per_item);
    if (tid < 16) sm.m[tid] = S.mvp[16 * view + tid];

    // ---- per item: the bin's live triangles (pruned and compacted by k_bin_prune), their
    //      smallest depths, and this pixel's candidates among them (in order of that depth)
    if (tid < nb) {
      const int tri = (int)bin_at(S, ws, bin_beg + tid);
      sm.btri[tid] = tri;
      sm.zminb[tid] = ordered_bits(ws.tri_z[(long long)slot * S.nt + tri].x);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sm.vid[tid][k] = vert_of(S, tri, k);
        const int ti = uv_of(S, tri, k);
        sm.uv[tid][2 * k] = __ldg(S.uvs + 2 * ti);
        sm.uv[tid][2 * k + 1] = __ldg(S.uvs + 2 * ti + 1);
        sm.A_cor[tid][k] = 0.0f;
        sm.n_cor[tid][k] = 0u;
        sm.c_cor[tid][k] = 0u;
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.S_cor[tid][k][c] = 0.0f;
      }
      sm.A_tri[tid] = 0.0f;
      sm.n_tri[tid] = 0u;
    }
    const long long ci = ((long long)slot * ntl + tile) * TILE_PX + tid;
    const int4 cw = ws.cand[((long long)slot * ntl + tile) * kCandWords * TILE_PX + tid];
    const uint32_t cand[CMAX / 4] = {(uint32_t)cw.x, (uint32_t)cw.y, (uint32_t)cw.z, (uint32_t)cw.w};
    const int ncand = ws.ncand[ci];
    const bool all_bin = ncand > CMAX;
    if (tid == 0) {
      sm.win[0] = sm.win[2] = 0x7FFFFFFF;
      sm.win[1] = sm.win[3] = -0x7FFFFFFF;
      sm.n_win = 0;
    }
    // the tile's target pixels: a tile inside the image whose rows start 16-byte aligned is read
    // as 16 rows of 12 float4 (each row's 16 RGB pixels) into the per-pair set-up array, which is
    // free until the first pair's set-up; any other tile pixel by pixel
    float3 tgt = f3(0.f, 0.f, 0.f);
    const float* trow = S.targets + (((long long)view * S.H + ty * TILE) * S.W + tx * TILE) * 3;
    const bool vec_tgt = (tx + 1) * TILE <= S.W && (ty + 1) * TILE <= S.H && (S.W & 3) == 0 &&
                         (reinterpret_cast<uintptr_t>(S.targets) & 15) == 0;
    if (vec_tgt) {
      float4* stage = reinterpret_cast<float4*>(&sm.side[0][0]);
      if (tid < TILE * 12) {
        const int r = tid / 12, q = tid % 12;
        stage[tid] = __ldg(reinterpret_cast<const float4*>(trow + (long long)r * S.W * 3) + q);
      }
      __syncthreads();
      const float* st = reinterpret_cast<const float*>(stage) + (dy * TILE + dx) * 3;
      tgt = f3(st[0], st[1], st[2]);
    } else if (valid) {
      const float* tp = S.targets + (((long long)view * S.H + py) * S.W + px) * 3;
      tgt = f3(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
    }
    float loss_acc = 0.0f;

    for (int pair = p0; pair < p1; ++pair) {
      const int par = pair & 1;
      const long long pb = pair - a.pair_begin;
      const uint32_t* planes = ws.tsign + ((long long)slot * ws.max_pairs + pb) * ws.sgn_words;
      // the previous pair is complete (and the item's set-up is done)
      __syncthreads();
      // ---- F: fold the previous pair's credits with its signs (other parity buffers)
      if (pair > p0) fold<TABLE, TSC, GR, NREAD>(S, sm, nb, par ^ 1);
      // ---- S: set up the bin's triangles on both sides from the projected perturbed vertices
      {
        const long long vb = ((long long)slot * ws.max_pairs + pb) * S.nv;
        for (int t2 = tid; t2 < 2 * nb; t2 += TILE_PX) {
          const int sd = t2 < nb ? 0 : 1, j = t2 - sd * nb;
          PVert v[3];
          uint32_t sg = 0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const long long o = vb + sm.vid[j][k];
            const int4 q = __ldg(ws.pverts + 2 * o + sd);
            v[k].X = q.x;
            v[k].Y = q.y;
            v[k].z = __int_as_float(q.z);
            v[k].iw = __int_as_float(q.w);
            v[k].ok = q.x != kNotDrawn;
            if (sd == 0) sg |= ((uint32_t)__ldg(ws.vbits + o) & 7u) << (3 * k);
          }
          if (sd == 0) sm.sgn9[par][j] = sg;
          Tri t;
          setup_tri(v[0], v[1], v[2], rx, ry, t);
          store_side_tri(sm.side[sd][j], t);
        }
      }
      __syncthreads();

      // ---- R: visible triangle on both sides among the candidates (nearest-first order: a
      //      candidate wholly behind both sides' best so far ends the search)
      int bj[2] = {-1, -1};
      if (valid && ncand > 0) {
        {
          unsigned long long best[2] = {~0ull, ~0ull};
          auto test = [&](int j) {
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
              const SideTri& t = sm.side[sd][j];
              if (!(t.flags & kDrawn)) continue;
              float l[3];
              if (!cover_lambdas(t, dx, dy, l)) continue;
              const unsigned long long k =
                  ((unsigned long long)ordered_bits(interp_depth(l, t.z)) << 32) | (uint32_t)sm.btri[j];
              if (k < best[sd]) {
                best[sd] = k;
                bj[sd] = j;
              }
            }
          };
          if (all_bin) {
            for (int j = 0; j < nb; ++j) test(j);
          } else {
            for (int q = 0; q < ncand; ++q) {
              const uint32_t word = q < 4 ? cand[0] : (q < 8 ? cand[1] : (q < 12 ? cand[2] : cand[3]));
              const int j = (int)((word >> (8 * (q & 3))) & 0xFFu);
              if (!CHK(S, j, nb)) continue;
              const uint32_t zb = sm.zminb[j];
              if (zb > (uint32_t)(best[0] >> 32) && zb > (uint32_t)(best[1] >> 32)) break;
              test(j);
            }
          }
        }
      }

      // ---- U: UV buffer values and footprints of both sides
      float bary[2][3];
      float ffx[2][NFOOT], ffy[2][NFOOT];
      uint32_t tpk[2][NFOOT];       // texel (x0,y0) id | 1<<30 if x1 wrapped | 1<<31 if y1 == y0
      uint32_t tslot[2][NFOOT][2];  // four 16-bit table slots per side and footprint
      int fix[2][NFOOT];            // footprint column before wrapping (nearest mode: the texel id)
      int fy0[2][NFOOT];            // footprint row y0
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        if (bj[sd] < 0) continue;
        const SideTri& t = sm.side[sd][bj[sd]];
        float l[3];
        cover_lambdas(t, dx, dy, l);
        const PerspW pw = persp(l, t.iw);
        const float* uvt = sm.uv[bj[sd]];
        const float u = persp_interp(pw, uvt[0], uvt[2], uvt[4]);
        const float v = persp_interp(pw, uvt[1], uvt[3], uvt[5]);
        if (SH == SHADE_GGX) {
#pragma unroll
          for (int k = 0; k < 3; ++k) bary[sd][k] = pw.q[k] / pw.qs;
        }
#pragma unroll
        for (int r = 0; r < NFOOT; ++r) {
          const TexDev& T = S.rtex[r];
          const Foot f = footprint(u, v, T.w, T.h);
          ffx[sd][r] = f.fx;
          ffy[sd][r] = f.fy;
          tpk[sd][r] = (uint32_t)(f.y0 * T.w + f.x0) | (f.x1 != f.x0 + 1 ? 1u << 30 : 0u) |
                       (f.y1 == f.y0 ? 1u << 31 : 0u);
          fix[sd][r] = S.foot_nearest ? nearest_texel(u, v, T.w, T.h) : f.ix;
          fy0[sd][r] = f.y0;
          if (Model<SH, GR>::DIRECT && pair == p0 && !S.foot_nearest && abs(f.ix) < (1 << 28)) {
            // the item's texel window: every footprint of its first pair, two texels of margin
            // (a perturbation moves a footprint by a fraction of a texel)
            atomicMin(&sm.win[0], f.ix - 2);
            atomicMax(&sm.win[1], f.ix + 3);
            atomicMin(&sm.win[2], max(f.y0 - 2, 0));
            atomicMax(&sm.win[3], min(f.y1 + 2, T.h - 1));
          }
        }
      }
      if (Model<SH, GR>::DIRECT && pair == p0) {
        __syncthreads();  // the window's bounds are reduced
        const long long ww = (long long)sm.win[1] - sm.win[0] + 1, wh = (long long)sm.win[3] - sm.win[2] + 1;
        if (!S.foot_nearest && ww > 0 && wh > 0 && ww * wh <= Model<SH, GR>::WCAP) {
          // window slots hold their texel's key from the start (and are listed as used)
          const TexDev& T = S.rtex[0];
          for (int s2 = tid; s2 < (int)(ww * wh); s2 += TILE_PX) {
            const int y = sm.win[2] + s2 / (int)ww, x = wrap_i(sm.win[0] + s2 % (int)ww, T.w);
            sm.tkey[s2] = tkey(T.index, y * T.w + x);
            sm.used[s2] = (uint16_t)s2;
          }
          if (tid == 0) sm.n_used = sm.n_win = (uint32_t)(ww * wh);
        } else if (tid == 0) {
          sm.win[0] = 1;  // no window: every key is hashed over the whole table
          sm.win[1] = 0;
        }
        __syncthreads();
      }
      // ---- the table slots of the footprints' texels: computed in the window, hashed outside it
      {
        const bool direct = Model<SH, GR>::DIRECT && sm.win[0] <= sm.win[1];
        // without a window every key is hashed over the whole table (nearest footprints, items
        // whose window would not fit)
        const uint32_t hbase = direct ? (uint32_t)Model<SH, GR>::WCAP : 0u;
        const uint32_t hsize = direct ? (uint32_t)(TABLE - Model<SH, GR>::WCAP) : (uint32_t)TABLE;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          if (bj[sd] < 0) continue;
#pragma unroll
          for (int r = 0; r < NFOOT; ++r) {
            const TexDev& T = S.rtex[r];
            if (S.foot_nearest) {
              // the one credited texel (Section 4.4): its slot, and its id in the second word
              const uint32_t nt = (uint32_t)fix[sd][r];
              tslot[sd][r][1] = nt;
              tslot[sd][r][0] = (sd == 1 && bj[0] >= 0 && tslot[0][r][1] == nt)
                                    ? tslot[0][r][0]
                                    : table_insert(sm, tkey(T.index, (int)nt), hbase, hsize);
              continue;
            }
            const int y0 = fy0[sd][r];
            const int y1 = (tpk[sd][r] >> 31) ? y0 : y0 + 1;
            const int ix = fix[sd][r];
            if (direct && ix >= sm.win[0] && ix + 1 <= sm.win[1] && y0 >= sm.win[2] && y1 <= sm.win[3]) {
              const int ww = sm.win[1] - sm.win[0] + 1;
              const uint32_t s00 = (uint32_t)((y0 - sm.win[2]) * ww + ix - sm.win[0]);
              const uint32_t s10 = (uint32_t)((y1 - sm.win[2]) * ww + ix - sm.win[0]);
              tslot[sd][r][0] = s00 | ((s00 + 1) << 16);
              tslot[sd][r][1] = s10 | ((s10 + 1) << 16);
              // (checked build) both rows' slots inside the window: else credit globally
              if (!CHK(S, (long long)s00 + 1, sm.n_win) || !CHK(S, (long long)s10 + 1, sm.n_win))
                tslot[sd][r][0] = tslot[sd][r][1] = NOSLOT | (NOSLOT << 16);
            } else if (!Model<SH, GR>::HASH_OUTSIDE) {
              tslot[sd][r][0] = tslot[sd][r][1] = NOSLOT | (NOSLOT << 16);  // global credits
            } else {
              uint32_t sl[4];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                sl[q] = table_insert(sm, tkey(T.index, texel_of(tpk[sd][r], q, T.w)), hbase, hsize);
              tslot[sd][r][0] = sl[0] | (sl[1] << 16);
              tslot[sd][r][1] = sl[2] | (sl[3] << 16);
            }
          }
        }
      }

      // ---- G: sample the perturbed texels (signs from the pair's planes), shade both sides,
      //      f+ - f-, credits
      float3 col[2];
      col[0] = col[1] = f3(S.bg[0], S.bg[1], S.bg[2]);
      {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          if (bj[sd] < 0) continue;
          float tex[NREAD][4];
          uint32_t gsb[4] = {0u, 0u, 0u, 0u};  // a texel group's sign bits per corner (4 r + c)
#pragma unroll
          for (int r = 0; r < NREAD; ++r) {
            const TexDev& T = S.rtex[r];
            const int poff = ws.sgn_off[T.index];
            const int fi = GR ? 0 : r;  // the footprint this texture uses
            const float fx = ffx[sd][fi], fy = ffy[sd][fi];
            const float wq[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
#pragma unroll
            for (int c = 0; c < 4; ++c) tex[r][c] = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int texel = texel_of(tpk[sd][fi], q, T.w);
              if (!CHK(S, texel, (long long)T.w * T.h)) continue;
              const uint32_t sb_s = plane_nibble(S, planes, poff, texel);
              if (GR) {
                gsb[q] |= sb_s << (4 * r);
              } else if (!S.foot_nearest) {
                const uint32_t sl = (tslot[sd][r][q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
                if (sl != NOSLOT && CHK(S, sl, TABLE)) sm.tsb[sl] = sb_s;
              } else if (texel == (int)tslot[sd][r][1] && (tslot[sd][r][0] & 0xFFFFu) != NOSLOT) {
                sm.tsb[tslot[sd][r][0] & 0xFFFFu] = sb_s;
              }
              const uint32_t sb = sd == 1 ? ~sb_s : sb_s;  // side -: theta - s eps
              const float* src = T.ptr + (long long)texel * T.c;
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (c < T.c) tex[r][c] += wq[q] * __fadd_rn(__ldg(src + c), ((sb >> c) & 1) ? -T.eps : T.eps);
            }
            if (T.c == 1) tex[r][1] = tex[r][2] = tex[r][0];
          }
          if (GR) {
            // the group entry of each corner carries every read texture's signs
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t sl;
              if (!S.foot_nearest) sl = (tslot[sd][0][q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
              else sl = texel_of(tpk[sd][0], q, S.rtex[0].w) == (int)tslot[sd][0][1] ? (tslot[sd][0][0] & 0xFFFFu)
                                                                                     : NOSLOT;
              if (sl != NOSLOT && CHK(S, sl, TABLE)) sm.tsb[sl] = gsb[q];
            }
          }
          if (SH == SHADE_UNLIT) {
            col[sd] = f3(tex[0][0], tex[0][1], tex[0][2]);
          } else {
            const int j = bj[sd];
            const uint32_t sg = sm.sgn9[par][j] ^ (sd == 1 ? 0x1FFu : 0u);
            float3 p[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float* src = S.pos + 3ll * sm.vid[j][k];
              float q[3];
#pragma unroll
              for (int c = 0; c < 3; ++c)
                q[c] = __fadd_rn(__ldg(src + c), ((sg >> (3 * k + c)) & 1) ? -S.eps_pos : S.eps_pos);
              p[k] = f3(q[0], q[1], q[2]);
            }
            const float2 uvv[3] = {make_float2(sm.uv[j][0], sm.uv[j][1]), make_float2(sm.uv[j][2], sm.uv[j][3]),
                                   make_float2(sm.uv[j][4], sm.uv[j][5])};
            float alb[4] = {1.f, 1.f, 1.f, 1.f}, nm[4] = {0.5f, 0.5f, 1.f, 0.f}, rough[4] = {0.5f, 0.f, 0.f, 0.f},
                  metal[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < NREAD; ++r) {
              const int role = S.rtex[r].role;
              float* dst = role == ROLE_ALBEDO ? alb : role == ROLE_NORMAL ? nm : role == ROLE_ROUGHNESS ? rough : metal;
#pragma unroll
              for (int c = 0; c < 4; ++c) dst[c] = tex[r][c];
            }
            const float bz[3] = {SH == SHADE_GGX ? bary[sd][0] : 0.f, SH == SHADE_GGX ? bary[sd][1] : 0.f,
                                 SH == SHADE_GGX ? bary[sd][2] : 0.f};
            col[sd] = shade(S, view, alb, nm, rough, metal, p, uvv, bz);
          }
        }
      }
      float df = 0.0f;
      if (valid) {
        float fp, fm;
        df = loss_diff(col[0], col[1], tgt, fp, fm);  // 0 where both sides show the background
        loss_acc += 0.5f * (fp + fm);
      }
      if (valid && a.delta_f) a.delta_f[(((long long)slot * a.pairs + pair) * S.H + py) * S.W + px] = df;
      // vertices: the visible triangle of side + (else side -), summed over each run of lanes that
      // share it, one shared atomic per run
      {
        const int kt = !valid ? -1 : (bj[0] >= 0 ? bj[0] : bj[1]);
        float v = df;
        int n;
        if (run_sum(kt, v, n) && kt >= 0) {
          atomicAdd(&sm.A_tri[kt], v);
          atomicAdd(&sm.n_tri[kt], (uint32_t)n);
        }
      }
      if (valid && bj[0] >= 0 && bj[1] >= 0 && bj[1] != bj[0]) {
        // side -'s corners that side +'s triangle does not share
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int v = sm.vid[bj[1]][k];
          if (v != sm.vid[bj[0]][0] && v != sm.vid[bj[0]][1] && v != sm.vid[bj[0]][2]) {
            atomicAdd(&sm.A_cor[bj[1]][k], df);
            atomicAdd(&sm.n_cor[bj[1]][k], 1u);
          }
        }
      }
      // texels: union of both sides' footprints of every read texture (of the group)
      if (valid) {
        // credit texel id (table slot sl, or NOSLOT: straight to the global sums)
        auto credit_texel = [&](int r, int id, uint32_t sl) {
          if (sl != NOSLOT) {
            if (!CHK(S, sl, TABLE)) return;
            atomicAdd(&sm.tA[sl], df);
            atomicAdd(&sm.tcnt[sl], 1u);
            return;
          }
#pragma unroll
          for (int g = 0; g < (GR ? NREAD : 1); ++g) {
            const TexDev& U = S.rtex[GR ? g : r];
            const uint32_t sb = plane_nibble(S, planes, ws.sgn_off[U.index], id);
            const long long base = U.offset + (long long)id * U.c;
            for (int c = 0; c < U.c; ++c) {
              if (!CHK(S, base + c, S.chk.params)) continue;
              atomicAdd(a.grad + base + c, ((sb >> c) & 1) ? -df : df);
              atomicAdd(a.counts + base + c, 1u);
            }
          }
        };
#pragma unroll
        for (int r = 0; r < NFOOT; ++r) {
          const TexDev& T = S.rtex[r];
          if (S.foot_nearest) {
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
              if (bj[sd] < 0) continue;
              const int id = (int)tslot[sd][r][1];
              if (sd == 1 && bj[0] >= 0 && (int)tslot[0][r][1] == id) continue;
              credit_texel(r, id, tslot[sd][r][0] & 0xFFFFu);
            }
            continue;
          }
          int id0[4] = {-1, -1, -1, -1};
          if (bj[0] >= 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) id0[q] = texel_of(tpk[0][r], q, T.w);
          }
          const bool same = bj[0] >= 0 && bj[1] >= 0 && tpk[0][r] == tpk[1][r];
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            if (bj[sd] < 0 || (sd == 1 && same)) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int id = sd == 0 ? id0[q] : texel_of(tpk[1][r], q, T.w);
              // the footprint's own repeats: its second row when the rows are clamped to one, its
              // second column in a one-texel-wide texture (texel_of gives every other corner a
              // different texel)
              bool dup = ((q & 2) && (tpk[sd][r] >> 31)) || ((q & 1) && T.w == 1);
              if (sd == 1) {
#pragma unroll
                for (int o = 0; o < 4; ++o) dup = dup || id0[o] == id;
              }
              if (dup) continue;
              credit_texel(r, id, (tslot[sd][r][q >> 1] >> (16 * (q & 1))) & 0xFFFFu);
            }
          }
        }
      }
    }
    __syncthreads();
    fold<TABLE, TSC, GR, NREAD>(S, sm, nb, (p1 - 1) & 1);
    __syncthreads();
    // ---- flush: one global atomic per credited vertex corner / texel and channel
    const uint32_t n_used = sm.n_used;
    for (uint32_t i = tid; i < n_used; i += blockDim.x) {
      const uint32_t s = sm.used[i];
      const uint32_t key = sm.tkey[s];
      if (sm.tcnt[s] == 0) continue;
      if (!GR) {
        const TexDev& T = S.tex[(key >> 28) - 1];
        const long long base = T.offset + (long long)(key & 0x0FFFFFFFu) * T.c;
        for (int c = 0; c < T.c; ++c) {
          if (!CHK(S, base + c, S.chk.params)) continue;
          atomicAdd(a.grad + base + c, sm.tS[c][s]);
          atomicAdd(a.counts + base + c, sm.tcnt[s]);
        }
      } else {
        // a group entry: the texel of every read texture, channel c of texture r at 4 r + c
#pragma unroll
        for (int r = 0; r < NREAD; ++r) {
          const TexDev& T = S.rtex[r];
          const long long base = T.offset + (long long)(key & 0x0FFFFFFFu) * T.c;
          for (int c = 0; c < T.c; ++c) {
            if (!CHK(S, base + c, S.chk.params)) continue;
            atomicAdd(a.grad + base + c, sm.tS[(4 * r + c) % TSC][s]);
            atomicAdd(a.counts + base + c, sm.tcnt[s]);
          }
        }
      }
    }
    if (tid < nb) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint32_t cn = sm.c_cor[tid][k];
        if (!cn) continue;
        const long long base = 3ll * sm.vid[tid][k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!CHK(S, base + c, S.chk.params)) continue;
          atomicAdd(a.grad + base + c, sm.S_cor[tid][k][c]);
          atomicAdd(a.counts + base + c, cn);
        }
      }
    }
    __syncthreads();
    clear_used(sm, n_used);  // n_used as read before the flush: thread 0 resets the shared count
    if (tid == 0) sm.n_used = 0;
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

template <int SH, bool GR>
__global__ void __launch_bounds__(TILE_PX, SH == SHADE_UNLIT ? 2 : 1)
    k_estimate_fast(SceneDev S, Workspace ws, ViewList vl, EstimateArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fast_items<SH, GR>(S, ws, vl, a,
                     *reinterpret_cast<FastSmem<Model<SH, GR>::TABLE, Model<SH, GR>::TSC>*>(smem_raw));
}

// The batched kernel keeps its asset after FastSmem, 16-byte aligned.  (Batched calls use the
// per-texture table: their assets need not share texture sizes.)
template <int SH>
__host__ __device__ constexpr size_t fast_batch_off() {
  return (sizeof(FastSmem<Model<SH>::TABLE, Model<SH>::TSC>) + 15) & ~(size_t)15;
}

// Batched form: the assets of P in order, each until its light items run out.
template <int SH>
__global__ void __launch_bounds__(TILE_PX, SH == SHADE_UNLIT ? 2 : 1) k_estimate_fast_batch(const BatchArgs P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<FastSmem<Model<SH>::TABLE, Model<SH>::TSC>*>(smem_raw);
  BatchSmem& b = *reinterpret_cast<BatchSmem*>(smem_raw + fast_batch_off<SH>());
  for (int ai = 0; ai < P.n; ++ai) {
    __syncthreads();
    load_asset(P, ai, b);
    __syncthreads();
    fast_items<SH, false>(b.d.S, b.d.ws, b.vl, b.a, sm);
  }
}

template <int SH, bool GR>
size_t fast_smem() {
  return sizeof(FastSmem<Model<SH, GR>::TABLE, Model<SH, GR>::TSC>);
}

template <int SH>
size_t fast_batch_smem() {
  return fast_batch_off<SH>() + sizeof(BatchSmem);
}

template <int SH>
cudaError_t launch_fast_batch_t(const BatchArgs& P, int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_estimate_fast_batch<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_batch_smem<SH>());
  if (e != cudaSuccess) return e;
  k_estimate_fast_batch<SH><<<grid, TILE_PX, fast_batch_smem<SH>(), st>>>(P);
  return cudaGetLastError();
}

template <int SH>
int fast_batch_blocks_per_sm_t() {
  int n = 0;
  cudaFuncSetAttribute(k_estimate_fast_batch<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fast_batch_smem<SH>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_estimate_fast_batch<SH>, TILE_PX, fast_batch_smem<SH>());
  return n > 0 ? n : 1;
}

template <int SH, bool GR>
cudaError_t launch_fast_t(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                          int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_estimate_fast<SH, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<SH, GR>());
  if (e != cudaSuccess) return e;
  k_estimate_fast<SH, GR><<<grid, TILE_PX, fast_smem<SH, GR>(), st>>>(S, ws, vl, a);
  return cudaGetLastError();
}

template <int SH, bool GR>
int fast_blocks_per_sm_t() {
  int n = 0;
  cudaFuncSetAttribute(k_estimate_fast<SH, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fast_smem<SH, GR>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_estimate_fast<SH, GR>, TILE_PX, fast_smem<SH, GR>());
  return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_fast(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a, int grid,
                        cudaStream_t st) {
  if (S.shading == SHADE_UNLIT) return launch_fast_t<SHADE_UNLIT, false>(S, ws, vl, a, grid, st);
  if (S.shading == SHADE_LAMBERT)
    return S.grouped ? launch_fast_t<SHADE_LAMBERT, true>(S, ws, vl, a, grid, st)
                     : launch_fast_t<SHADE_LAMBERT, false>(S, ws, vl, a, grid, st);
  return S.grouped ? launch_fast_t<SHADE_GGX, true>(S, ws, vl, a, grid, st)
                   : launch_fast_t<SHADE_GGX, false>(S, ws, vl, a, grid, st);
}

cudaError_t launch_prune(const SceneDev& S, const Workspace& ws, const ViewList& vl, cudaStream_t st) {
  k_bin_prune<<<dim3(n_tiles(S), vl.n), TILE_PX, 0, st>>>(S, ws, vl);
  return cudaGetLastError();
}

cudaError_t launch_prune_batch(const BatchArgs& P, int max_tiles, int max_views, cudaStream_t st) {
  k_bin_prune_batch<<<dim3(max_tiles, max_views, P.n), TILE_PX, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fast_batch(const BatchArgs& P, int shading, int grid, cudaStream_t st) {
  if (shading == SHADE_UNLIT) return launch_fast_batch_t<SHADE_UNLIT>(P, grid, st);
  if (shading == SHADE_LAMBERT) return launch_fast_batch_t<SHADE_LAMBERT>(P, grid, st);
  return launch_fast_batch_t<SHADE_GGX>(P, grid, st);
}

int fast_batch_blocks_per_sm(int shading) {
  if (shading == SHADE_UNLIT) return fast_batch_blocks_per_sm_t<SHADE_UNLIT>();
  if (shading == SHADE_LAMBERT) return fast_batch_blocks_per_sm_t<SHADE_LAMBERT>();
  return fast_batch_blocks_per_sm_t<SHADE_GGX>();
}

int fast_blocks_per_sm(int shading, int grouped) {
  if (shading == SHADE_UNLIT) return fast_blocks_per_sm_t<SHADE_UNLIT, false>();
  if (shading == SHADE_LAMBERT)
    return grouped ? fast_blocks_per_sm_t<SHADE_LAMBERT, true>() : fast_blocks_per_sm_t<SHADE_LAMBERT, false>();
  return grouped ? fast_blocks_per_sm_t<SHADE_GGX, true>() : fast_blocks_per_sm_t<SHADE_GGX, false>();
}

}  // namespace sge
