// Descent step D (Section 5): gradient estimate of Eq. 9 from the accumulated
// sums, SGD or Adam (Kingma & Ba 2015) per parameter, then the sums and counts
// are zeroed for the next iteration.  One thread per parameter; memory bound.
#include <cuda_runtime.h>

#include "sge_device.cuh"

namespace sge {

namespace {

struct StepGroups {
  int n;
  long long begin[SGE_MAX_TEXTURES + 2];  // flat parameter index where each group starts (+ end)
  float* theta[SGE_MAX_TEXTURES + 1];
  float eps[SGE_MAX_TEXTURES + 1];
  float lr[SGE_MAX_TEXTURES + 1];
};

__global__ void k_step(StepGroups G, int kind, float* grad, uint32_t* counts, float inv_n, float b1, float b2,
                       int t_host, float aeps, float* m, float* v, const int32_t* t_dev) {
  const long long d = G.begin[G.n];
  // Adam's bias corrections 1 - beta^t for the step number t (from device memory in a replayed
  // graph's step), formed as -expm1(t log beta): no cancellation when beta^t is close to 1
  float c1 = 1.0f, c2 = 1.0f;
  if (kind == SGE_STEP_ADAM) {
    const float t = (float)(t_dev ? *t_dev : t_host);
    c1 = -expm1f(t * logf(b1));
    c2 = -expm1f(t * logf(b2));
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x) {
    int g = 0;
#pragma unroll 1
    while (g + 1 < G.n && i >= G.begin[g + 1]) ++g;
    const long long li = i - G.begin[g];
    const float s = grad[i];
    const uint32_t cn = counts[i];
    const float scale = kind == SGE_STEP_SGD_MEAN ? 1.0f / (float)(cn > 0 ? cn : 1u) : inv_n;
    const float gr = s * scale / (2.0f * G.eps[g]);
    float th = G.theta[g][li];
    if (kind == SGE_STEP_ADAM) {
      const float mm = b1 * m[i] + (1.0f - b1) * gr;
      const float vv = b2 * v[i] + (1.0f - b2) * gr * gr;
      m[i] = mm;
      v[i] = vv;
      th -= G.lr[g] * (mm / c1) / (sqrtf(vv / c2) + aeps);
    } else {
      th -= G.lr[g] * gr;
    }
    G.theta[g][li] = th;
    grad[i] = 0.0f;
    counts[i] = 0u;
  }
}

// Moves a captured loop's iteration state on: the iteration index and Adam's step number.
__global__ void k_iter_advance(uint32_t* state, int d_iter, int d_t) {
  state[0] += (uint32_t)d_iter;
  state[1] = (uint32_t)((int)state[1] + d_t);
}

// g_i = scale * grad_i / (2 eps_i n_total): the estimate of Eq. 9 (scale: device scalar or NULL).
__global__ void k_gradient(StepGroups G, const float* grad, float inv_n, const float* scale, float* out) {
  const long long d = G.begin[G.n];
  const float sc = scale ? *scale : 1.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x) {
    int g = 0;
#pragma unroll 1
    while (g + 1 < G.n && i >= G.begin[g + 1]) ++g;
    out[i] = sc * (grad[i] * inv_n / (2.0f * G.eps[g]));
  }
}

StepGroups groups_of(const SceneDev& S) {
  StepGroups G;
  G.n = 1 + S.ntex;
  G.begin[0] = 0;
  G.theta[0] = const_cast<float*>(S.pos);
  G.eps[0] = S.eps_pos;
  G.lr[0] = 0.0f;
  for (int k = 0; k < S.ntex; ++k) {
    G.begin[k + 1] = S.tex[k].offset;
    G.theta[k + 1] = const_cast<float*>(S.tex[k].ptr);
    G.eps[k + 1] = S.tex[k].eps;
    G.lr[k + 1] = 0.0f;
  }
  G.begin[G.n] = S.n_params;
  return G;
}

int grid_for(long long n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 255) / 256;
  if (blocks > 8ll * sms) blocks = 8ll * sms;
  return blocks < 1 ? 1 : (int)blocks;
}

// Full-image estimator (Eq. 4), accumulation: every parameter i gets sum_e dF_e s_i(e) over
// the call's estimates e (signs from each estimate's key) and one count per estimate.  The
// estimates' keys and differences are staged in shared memory once per CTA; one thread per
// parameter (grid-stride).
__global__ void k_full_image_grad(long long d, int n_est, int pairs, ViewList vl, uint64_t seed, uint32_t iter,
                                  const float* dF, float* grad, uint32_t* counts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem_raw);
  float* dfs = reinterpret_cast<float*>(keys + n_est);
  for (int e = threadIdx.x; e < n_est; e += blockDim.x) {
    keys[e] = pair_key(seed, iter, (uint32_t)vl.id[e / pairs], (uint32_t)(e % pairs));
    dfs[e] = dF[e];
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int e = 0; e < n_est; ++e) acc += sign_neg(keys[e], (uint64_t)i) ? -dfs[e] : dfs[e];
    grad[i] += acc;
    counts[i] += (uint32_t)n_est;
  }
}

// y[r] (+)= sum_j w_j x[col_j] for 3-vectors (xyz per row), rows of a CSR matrix in fixed order:
// the refine matrix of a subdivision (fine = R control) or its transpose (control gradient =
// R^T fine gradient).  One thread per row.
__global__ void k_csr_vec3(const int32_t* ptr, const int32_t* col, const float* w, int n_rows, const float* x,
                           float* y, int accumulate) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
  for (int j = ptr[r]; j < ptr[r + 1]; ++j) {
    const float wj = w[j];
    const long long c = 3ll * col[j];
    a0 += wj * x[c];
    a1 += wj * x[c + 1];
    a2 += wj * x[c + 2];
  }
  if (accumulate) {
    y[3ll * r] += a0;
    y[3ll * r + 1] += a1;
    y[3ll * r + 2] += a2;
  } else {
    y[3ll * r] = a0;
    y[3ll * r + 1] = a1;
    y[3ll * r + 2] = a2;
  }
}

}  // namespace

cudaError_t launch_gradient(const SceneDev& S, const float* grad, long long n_total, const float* scale, float* out,
                            cudaStream_t st) {
  k_gradient<<<grid_for(S.n_params), 256, 0, st>>>(groups_of(S), grad, (float)(1.0 / (double)n_total), scale, out);
  return cudaGetLastError();
}

cudaError_t launch_step(const SceneDev& S, const sge_opt& o, float* grad, uint32_t* counts, long long n_total,
                        float* m, float* v, cudaStream_t st, const int32_t* t_dev) {
  StepGroups G;
  G.n = 1 + S.ntex;
  G.begin[0] = 0;
  G.theta[0] = const_cast<float*>(S.pos);
  G.eps[0] = S.eps_pos;
  G.lr[0] = o.lr_pos;
  for (int k = 0; k < S.ntex; ++k) {
    G.begin[k + 1] = S.tex[k].offset;
    G.theta[k + 1] = const_cast<float*>(S.tex[k].ptr);
    G.eps[k + 1] = S.tex[k].eps;
    G.lr[k + 1] = o.lr_tex[k];
  }
  G.begin[G.n] = S.n_params;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (S.n_params + 255) / 256;
  if (blocks > 8ll * sms) blocks = 8ll * sms;
  if (blocks < 1) blocks = 1;
  k_step<<<(unsigned)blocks, 256, 0, st>>>(G, o.kind, grad, counts, (float)(1.0 / (double)n_total), o.beta1,
                                           o.beta2, o.t, o.adam_eps, m, v, t_dev);
  return cudaGetLastError();
}

cudaError_t launch_iter_advance(uint32_t* state, int d_iter, int d_t, cudaStream_t st) {
  k_iter_advance<<<1, 1, 0, st>>>(state, d_iter, d_t);
  return cudaGetLastError();
}

cudaError_t launch_full_image_grad(const SceneDev& S, const ViewList& vl, int pairs, uint64_t seed, uint32_t iter,
                                   const float* dF, float* grad, uint32_t* counts, cudaStream_t st) {
  const int n_est = vl.n * pairs;
  const size_t smem = (size_t)n_est * (sizeof(uint64_t) + sizeof(float));
  long long blocks = (S.n_params + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_full_image_grad<<<(unsigned)blocks, 256, smem, st>>>(S.n_params, n_est, pairs, vl, seed, iter, dF, grad, counts);
  return cudaGetLastError();
}

cudaError_t launch_csr_vec3(const int32_t* ptr, const int32_t* col, const float* w, int n_rows, const float* x,
                            float* y, int accumulate, cudaStream_t st) {
  if (n_rows > 0) k_csr_vec3<<<(n_rows + 255) / 256, 256, 0, st>>>(ptr, col, w, n_rows, x, y, accumulate);
  return cudaGetLastError();
}

}  // namespace sge
