// Perturbation P (Algorithm 1) and vertex transform for a block of estimates:
// for every (view slot, pair, welded vertex) draw the vertex's three signs,
// form theta + s eps and theta - s eps (rounded to float, as Algorithm 1 stores
// them) and project both sides to 24.8 fixed point.  The fused estimator then
// sets up triangles from these instead of redoing the hash and the projection
// for every tile a vertex's triangles touch.
#include <cuda_runtime.h>

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
  const uint64_t pkey = pair_key(a.seed, a.iter, (uint32_t)view, (uint32_t)(a.pair_begin + pb));
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

}  // namespace

cudaError_t launch_vertex_pass(const SceneDev& S, const Workspace& ws, const ViewList& vl, const EstimateArgs& a,
                               cudaStream_t st) {
  dim3 grid((S.nv + 255) / 256, a.pair_count, vl.n);
  k_vertex_pass<<<grid, 256, 0, st>>>(S, ws, vl, a);
  return cudaGetLastError();
}

}  // namespace sge
