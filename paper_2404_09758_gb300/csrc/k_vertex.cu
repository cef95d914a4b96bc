// Perturbation P (Algorithm 1) and vertex transform for a block of estimates:
// for every (view slot, pair, welded vertex) draw the vertex's three signs,
// form theta + s eps and theta - s eps (rounded to float, as Algorithm 1 stores
// them) and project both sides to 24.8 fixed point.  The fused estimator then
// sets up triangles from these instead of redoing the hash and the projection
// for every tile a vertex's triangles touch.
#include <cuda_runtime.h>

#define SGE_FILE_ID 6  // range-check sites of this file (checked build)
#include "sge_device.cuh"

namespace sge {

namespace {

__global__ void k_vertex_pass(SceneDev S, Workspace ws, ViewList vl, EstimateArgs a) {
  __shared__ float m[16];
  const int slot = blockIdx.z, pb = blockIdx.y;
  const int view = vl.id[slot];
  if (threadIdx.x < 16) m[threadIdx.x] = S.mvp[16 * view + threadIdx.x];
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= S.nv) return;
  const uint64_t pkey = pair_key(a.seed, iter_of(a), (uint32_t)view, (uint32_t)(a.pair_begin + pb));
  const float* p = S.pos + 3ll * v;
  float qp[3], qm[3];
  uint32_t bits = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const bool neg = sign_neg(pkey, 3ull * (uint64_t)v + c);
    bits |= (uint32_t)neg << c;
    const float th = __ldg(p + c), d = neg ? -S.eps_pos : S.eps_pos;
    qp[c] = __fadd_rn(th, d);
    qm[c] = __fadd_rn(th, -d);
  }
  const PVert vp = project(m, qp[0], qp[1], qp[2], S.W, S.H, S.near_w);
  const PVert vm = project(m, qm[0], qm[1], qm[2], S.W, S.H, S.near_w);
  bits |= (uint32_t)vp.ok << 3 | (uint32_t)vm.ok << 4;
  const long long o = ((long long)slot * ws.max_pairs + pb) * S.nv + v;
  ws.pverts[2 * o] = make_int4(vp.ok ? vp.X : kNotDrawn, vp.Y, __float_as_int(vp.z), __float_as_int(vp.iw));
  ws.pverts[2 * o + 1] = make_int4(vm.ok ? vm.X : kNotDrawn, vm.Y, __float_as_int(vm.z), __float_as_int(vm.iw));
  ws.vbits[o] = (uint8_t)bits;
}

// Texel sign planes of a block of estimates: word w of estimate (slot, pair) holds the signs of
// eight consecutive texels of one read texture, four bits per texel (bit c: channel c has
// s = -1), the same signs sign_neg draws for those parameters.  The fused estimators read them
// when they sample and fold, instead of hashing per texel and pixel.  A word's 8 C parameters are
// consecutive, so they are bits [i0 mod 64, i0 mod 64 + 8 C) of the generator's output for block
// i0 / 64 followed by the next block's output: one funnel shift, then the 8 C bits are spread to
// one nibble per texel.
template <int C>
__device__ __forceinline__ uint32_t sign_word(uint64_t pkey, long long first_param, int n_texels) {
  const uint64_t i0 = (uint64_t)first_param, blk0 = i0 >> 6;
  const int sh = (int)(i0 & 63);
  uint64_t x = mix64(pkey + (blk0 + 1) * kGamma) >> sh;
  if (sh + 8 * C > 64) x |= mix64(pkey + (blk0 + 2) * kGamma) << (64 - sh);
  const uint32_t b = (uint32_t)x;
  uint32_t bits;
  if (C == 4) {
    bits = b;
  } else {
    bits = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) bits |= ((b >> (C * j)) & ((1u << C) - 1u)) << (4 * j);
  }
  return n_texels < 8 ? bits & ((1u << (4 * n_texels)) - 1u) : bits;
}

constexpr int kSignWordsPerThread = 4;

__global__ void k_texel_signs(SceneDev S, Workspace ws, ViewList vl, EstimateArgs a) {
  const int slot = blockIdx.z, pb = blockIdx.y;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kSignWordsPerThread;
  if (w0 >= ws.sgn_words) return;
  const uint64_t pkey = pair_key(a.seed, iter_of(a), (uint32_t)vl.id[slot], (uint32_t)(a.pair_begin + pb));
  uint32_t* out = ws.tsign + ((long long)slot * ws.max_pairs + pb) * ws.sgn_words;
#pragma unroll
  for (int q = 0; q < kSignWordsPerThread; ++q) {
    const long long w = w0 + q;
    if (w >= ws.sgn_words) break;
    // the read texture whose plane holds word w (planes in read order, each starting on a word)
    int r = 0;
#pragma unroll
    for (int k = 1; k < MAX_READ; ++k)
      if (k < S.nread && w >= ws.sgn_off[S.read_k[k]]) r = k;
    const TexDev& T = S.rtex[r];
    const long long t0 = (w - ws.sgn_off[S.read_k[r]]) * 8;
    const long long left = (long long)T.w * T.h - t0;
    const int n = left < 8 ? (int)left : 8;
    const long long first = T.offset + t0 * T.c;
    uint32_t bits;
    switch (T.c) {
      case 1: bits = sign_word<1>(pkey, first, n); break;
      case 2: bits = sign_word<2>(pkey, first, n); break;
      case 3: bits = sign_word<3>(pkey, first, n); break;
      default: bits = sign_word<4>(pkey, first, n); break;
    }
    if (CHK(S, w, S.chk.sign_words)) out[w] = bits;
  }
}

}  // namespace

cudaError_t launch_vertex_pass(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                               cudaStream_t st) {
  dim3 grid((S.nv + 255) / 256, a.pair_count, vl.n);
  k_vertex_pass<<<grid, 256, 0, st>>>(S, ws, vl, a);
  if (ws.tsign && ws.sgn_words > 0) {
    const long long threads = (ws.sgn_words + kSignWordsPerThread - 1) / kSignWordsPerThread;
    dim3 gs((unsigned)((threads + 255) / 256), a.pair_count, vl.n);
    k_texel_signs<<<gs, 256, 0, st>>>(S, ws, vl, a);
  }
  return cudaGetLastError();
}

}  // namespace sge
