// Device building blocks shared by the estimator, staged and binning kernels.
//
// Bit-exactness: every float operation whose result decides an integer (the
// snapped screen position, the depth that picks the visible triangle, the UV
// that picks texels) is written with an explicit round-to-nearest intrinsic
// (__fmul_rn, __fadd_rn, __fdiv_rn, ...), which the compiler never fuses into an
// FMA, so the result is the same whichever kernel evaluates it.  Coverage uses
// exact 64-bit integer edge functions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sge_internal.h"

namespace sge {

// ---------------------------------------------------------------- range checks (checked build)
// Is 0 <= i < n?  The unchecked build assumes so (the host validates what it can); the checked
// build tests it and, when it fails, records SGE_ERR_BOUNDS in the status word so that the caller
// skips the access.
// The first failing check also records its site (file id * 100000 + line) and the index.
__device__ __forceinline__ bool chk(const SceneDev& S, long long i, long long n, int site) {
#if SGE_CHECKED
  if (i >= 0 && i < n) return true;
  atomicCAS(S.chk.status, 0u, (uint32_t)SGE_ERR_BOUNDS);
  if (S.chk.where && atomicCAS(S.chk.where, 0u, (uint32_t)site) == 0u) S.chk.where[1] = (uint32_t)i;
  return false;
#else
  (void)S;
  (void)i;
  (void)n;
  (void)site;
  return true;
#endif
}
#ifndef SGE_FILE_ID
#define SGE_FILE_ID 0
#endif
#define CHK(S_, i_, n_) chk(S_, i_, n_, SGE_FILE_ID * 100000 + __LINE__)
#define CHK_H(S_, i_, n_) chk(S_, i_, n_, 900000 + __LINE__)

// Vertex / UV index k of triangle tri (a failing check reads as index 0).
__device__ __forceinline__ int vert_of(const SceneDev& S, int tri, int k) {
  const int v = __ldg(S.pidx + 3 * tri + k);
  return CHK_H(S, v, S.chk.nv) ? v : 0;
}
__device__ __forceinline__ int uv_of(const SceneDev& S, int tri, int k) {
  const int t = __ldg(S.uvidx + 3 * tri + k);
  return CHK_H(S, t, S.chk.nuv) ? t : 0;
}

// Bin entry i (a failing check reads as triangle 0).
__device__ __forceinline__ uint32_t bin_at(const SceneDev& S, const Workspace& ws, long long i) {
  return CHK_H(S, i, S.chk.bins) ? ws.bins[i] : 0u;
}


// ---------------------------------------------------------------- sign hash (Algorithm 1)
// The paper draws s_i with a hash function it does not name.  This uses
// SplitMix64 (Steele, Lea & Flood 2014): mix64 is its output function; one
// generator step adds the golden-ratio increment and mixes.  The key of an
// estimate chains four steps over (seed, iteration, view, pair); s_i is bit
// (i mod 64) of the (floor(i / 64) + 1)-th output of the generator seeded with
// that key: one output gives the signs of 64 consecutive parameters.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t pair_key(uint64_t seed, uint32_t iter, uint32_t view,
                                                      uint32_t pair) {
  uint64_t k = mix64(seed + kGamma);
  k = mix64((k ^ iter) + kGamma);
  k = mix64((k ^ view) + kGamma);
  return mix64((k ^ pair) + kGamma);
}

// true when s_i = -1
__device__ __forceinline__ bool sign_neg(uint64_t key, uint64_t i) {
  return ((mix64(key + ((i >> 6) + 1) * kGamma) >> (i & 63)) & 1) != 0;
}

// theta_i + side * s_i * eps_i, rounded to float (the perturbed parameter Algorithm 1 stores).
__device__ __forceinline__ float perturb(float theta, float eps, uint64_t key, uint64_t i, int side) {
  if (side == 0) return theta;
  bool neg = sign_neg(key, i) != (side < 0);
  return __fadd_rn(theta, neg ? -eps : eps);
}

// ---------------------------------------------------------------- projection
// clip = M (x,y,z,1); screen = ((x/w)/2 + 1/2) W, (1/2 - (y/w)/2) H; snapped to
// 1/256 pixel with round-half-even.  A vertex needs w > near_w and |screen| < 2^15 px.
constexpr float kGuard = 8388608.0f;  // 2^23 fixed-point units

struct PVert {
  int X, Y;
  float z, iw;
  bool ok;
};

__device__ __forceinline__ float dot4_rn(const float* m, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[0], x), __fmul_rn(m[1], y)), __fmul_rn(m[2], z)),
                   m[3]);
}

__device__ __forceinline__ PVert project(const float* m, float x, float y, float z, int W, int H,
                                         float near_w) {
  PVert v;
  float cx = dot4_rn(m + 0, x, y, z), cy = dot4_rn(m + 4, x, y, z);
  float cz = dot4_rn(m + 8, x, y, z), cw = dot4_rn(m + 12, x, y, z);
  v.ok = cw > near_w;
  v.iw = __fdiv_rn(1.0f, cw);
  float xn = __fmul_rn(cx, v.iw), yn = __fmul_rn(cy, v.iw);
  v.z = __fmul_rn(cz, v.iw);
  float xs = __fmul_rn(__fadd_rn(__fmul_rn(xn, 0.5f), 0.5f), (float)W);
  float ys = __fmul_rn(__fsub_rn(0.5f, __fmul_rn(yn, 0.5f)), (float)H);
  float xf = __fmul_rn(xs, 256.0f), yf = __fmul_rn(ys, 256.0f);
  if (!(fabsf(xf) < kGuard) || !(fabsf(yf) < kGuard)) v.ok = false;
  v.X = v.ok ? __float2int_rn(xf) : 0;
  v.Y = v.ok ? __float2int_rn(yf) : 0;
  return v;
}

// int64 -> float, correctly rounded; values that fit 32 bits take the cheaper
// 32-bit conversion, which rounds the same value to the same float.
__device__ __forceinline__ float ll2f_rn(long long v) {
  return (v == (long long)(int)v) ? __int2float_rn((int)v) : __ll2float_rn(v);
}

// ---------------------------------------------------------------- triangle setup
// Edge function of the edge opposite vertex k (a = k+1, b = k+2 mod 3):
//   E_k(P) = (Xb-Xa)(Py-Ya) - (Yb-Ya)(Px-Xa),   E_0+E_1+E_2 = twice the signed area.
// After orienting to positive area, E_k = E_k(origin) + A_k dx + B_k dy exactly, with
// A_k = Ya-Yb, B_k = Xb-Xa (times the orientation).  Pixel centres inside: every
// E_k > 0, or E_k == 0 on a top or left edge (y grows downwards: left = A_k > 0,
// top = A_k == 0 && B_k > 0).
struct Tri {
  long long e0[3];  // oriented edge functions at the reference pixel centre
  int a[3], b[3];   // oriented per-unit steps in x and y (fixed-point units)
  int bias[3];      // 0 on top/left edges, -1 elsewhere: inside <=> e + bias >= 0
  float inv_area;   // 1 / (float)area
  float z[3], iw[3];
  int ok;
};

__device__ __forceinline__ long long edge_at(int Xa, int Ya, int Xb, int Yb, long long px,
                                             long long py) {
  return (long long)(Xb - Xa) * (py - Ya) - (long long)(Yb - Ya) * (px - Xa);
}

// Set up a triangle from its three projected vertices; (rx, ry) is the fixed-point
// reference point (a pixel centre) the edge functions are stored at.
__device__ __forceinline__ void setup_tri(const PVert& v0, const PVert& v1, const PVert& v2,
                                          long long rx, long long ry, Tri& t) {
  t.ok = v0.ok && v1.ok && v2.ok;
  if (!t.ok) return;
  long long area = edge_at(v0.X, v0.Y, v1.X, v1.Y, v2.X, v2.Y);
  if (area == 0) {
    t.ok = 0;
    return;
  }
  int sg = area > 0 ? 1 : -1;
  const PVert* v[3] = {&v0, &v1, &v2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const PVert& A = *v[(k + 1) % 3];
    const PVert& B = *v[(k + 2) % 3];
    t.e0[k] = sg * edge_at(A.X, A.Y, B.X, B.Y, rx, ry);
    t.a[k] = sg * (A.Y - B.Y);
    t.b[k] = sg * (B.X - A.X);
    t.bias[k] = (t.a[k] > 0 || (t.a[k] == 0 && t.b[k] > 0)) ? 0 : -1;
  }
  t.inv_area = __fdiv_rn(1.0f, ll2f_rn(area > 0 ? area : -area));
  t.z[0] = v0.z; t.z[1] = v1.z; t.z[2] = v2.z;
  t.iw[0] = v0.iw; t.iw[1] = v1.iw; t.iw[2] = v2.iw;
}

__device__ __forceinline__ uint32_t ordered_bits(float z) {
  uint32_t b = __float_as_uint(z);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Barycentric weights lambda_k = E_k / area as floats.
__device__ __forceinline__ void lambdas(const long long e[3], float inv_area, float l[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) l[k] = __fmul_rn(ll2f_rn(e[k]), inv_area);
}

__device__ __forceinline__ float interp_depth(const float l[3], const float z[3]) {
  return __fadd_rn(__fadd_rn(__fmul_rn(l[0], z[0]), __fmul_rn(l[1], z[1])), __fmul_rn(l[2], z[2]));
}

// Perspective-correct interpolation: q_k = lambda_k / w_k, value = sum q_k a_k / sum q_k.
struct PerspW {
  float q[3], qs;
};
__device__ __forceinline__ PerspW persp(const float l[3], const float iw[3]) {
  PerspW p;
#pragma unroll
  for (int k = 0; k < 3; ++k) p.q[k] = __fmul_rn(l[k], iw[k]);
  p.qs = __fadd_rn(__fadd_rn(p.q[0], p.q[1]), p.q[2]);
  return p;
}
__device__ __forceinline__ float persp_interp(const PerspW& p, float a0, float a1, float a2) {
  return __fdiv_rn(
      __fadd_rn(__fadd_rn(__fmul_rn(p.q[0], a0), __fmul_rn(p.q[1], a1)), __fmul_rn(p.q[2], a2)), p.qs);
}

// ---------------------------------------------------------------- texture footprint
// Texel centres at half-integers: x = u W - 1/2, x0 = floor(x), fx = x - x0; u wraps, v clamps.
struct Foot {
  int x0, x1, y0, y1;  // wrapped / clamped texel coordinates
  float fx, fy;
  int ix;              // floor(u W - 1/2) before wrapping (x0 = ix mod W, x1 = (ix + 1) mod W)
  int nearest;         // texel id of the nearest texel (set where SceneDev::foot_nearest asks for it)
};

// i mod n in [0, n); one add or subtract for the i in [-n, 2n) a texel lookup produces
__device__ __forceinline__ int wrap_i(int i, int n) {
  int r = i < 0 ? i + n : (i >= n ? i - n : i);
  if (r < 0 || r >= n) {
    r = i % n;
    r = r < 0 ? r + n : r;
  }
  return r;
}
__device__ __forceinline__ int clamp_i(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

__device__ __forceinline__ Foot footprint(float u, float v, int W, int H) {
  Foot f;
  float x = __fsub_rn(__fmul_rn(u, (float)W), 0.5f);
  float y = __fsub_rn(__fmul_rn(v, (float)H), 0.5f);
  float xf = floorf(x), yf = floorf(y);
  f.fx = __fsub_rn(x, xf);
  f.fy = __fsub_rn(y, yf);
  int ix = (int)xf, iy = (int)yf;
  f.ix = ix;
  f.x0 = wrap_i(ix, W);
  f.x1 = wrap_i(ix + 1, W);
  f.y0 = clamp_i(iy, H);
  f.y1 = clamp_i(iy + 1, H);
  return f;
}

// The texel whose square holds the sample point, (floor(u W) wrapped, floor(v H) clamped): the one
// texel Section 4.4 credits ("nearest" footprint); its id y W + x.
__device__ __forceinline__ int nearest_texel(float u, float v, int W, int H) {
  const int x = wrap_i((int)floorf(__fmul_rn(u, (float)W)), W);
  const int y = clamp_i((int)floorf(__fmul_rn(v, (float)H)), H);
  return y * W + x;
}

// ---------------------------------------------------------------- device scene view
// Sample all channels of perturbed texture k at footprint f (bilinear), float32.
__device__ __forceinline__ void sample_tex(const TexDev& T, const Foot& f, uint64_t key, int side,
                                           float out[4]) {
  float w[4] = {(1.0f - f.fx) * (1.0f - f.fy), f.fx * (1.0f - f.fy), (1.0f - f.fx) * f.fy,
                f.fx * f.fy};
  int tx[4] = {f.x0, f.x1, f.x0, f.x1};
  int ty[4] = {f.y0, f.y0, f.y1, f.y1};
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    long long t = (long long)ty[j] * T.w + tx[j];
    const float* src = T.ptr + t * T.c;
    long long pi = T.offset + t * T.c;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < T.c) out[c] += w[j] * perturb(__ldg(src + c), T.eps, key, (uint64_t)(pi + c), side);
  }
  if (T.c == 1) out[1] = out[2] = out[0];
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 norm3(float3 a) {
  float n = sqrtf(dot3(a, a));
  return n > 0.0f ? f3(a.x / n, a.y / n, a.z / n) : a;
}

// Shading normal: tangent-space normal-map vector (2 t - 1) in the frame of the
// triangle's own perturbed geometry and UVs: N face normal, T along +u
// (Gram-Schmidt against N), B = N x T.
__device__ __forceinline__ float3 shading_normal(const float3 p[3], const float2 uv[3], const float nm[4]) {
  float3 e1 = sub3(p[1], p[0]), e2 = sub3(p[2], p[0]);
  float3 N = norm3(cross3(e1, e2));
  float du1 = uv[1].x - uv[0].x, dv1 = uv[1].y - uv[0].y;
  float du2 = uv[2].x - uv[0].x, dv2 = uv[2].y - uv[0].y;
  float det = du1 * dv2 - du2 * dv1;
  float3 T = det != 0.0f ? f3((e1.x * dv2 - e2.x * dv1) / det, (e1.y * dv2 - e2.y * dv1) / det,
                              (e1.z * dv2 - e2.z * dv1) / det)
                         : e1;
  float nt = dot3(N, T);
  T = norm3(f3(T.x - N.x * nt, T.y - N.y * nt, T.z - N.z * nt));
  float3 B = cross3(N, T);
  float mx = 2.0f * nm[0] - 1.0f, my = 2.0f * nm[1] - 1.0f, mz = 2.0f * nm[2] - 1.0f;
  float3 n = f3(T.x * mx + B.x * my + N.x * mz, T.y * mx + B.y * my + N.y * mz,
                T.z * mx + B.z * my + N.z * mz);
  if (dot3(n, n) == 0.0f) n = N;
  return norm3(n);
}

// Colour of a covered pixel.  p: perturbed world positions of the visible triangle,
// uvs: its UVs, b: perspective-correct barycentrics, tex samples by role.
__device__ __forceinline__ float3 shade(const SceneDev& S, int view, const float alb[4],
                                        const float nm[4], const float rough[4], const float metal[4],
                                        const float3 p[3], const float2 uv[3], const float b[3]) {
  if (S.shading == SHADE_UNLIT) return f3(alb[0], alb[1], alb[2]);
  float3 n = shading_normal(p, uv, nm);
  float3 L = f3(S.light_dir[0], S.light_dir[1], S.light_dir[2]);
  float ndl = fmaxf(dot3(n, L), 0.0f);
  if (S.shading == SHADE_LAMBERT) {
    return f3(alb[0] * (S.ambient + S.light_rgb[0] * ndl), alb[1] * (S.ambient + S.light_rgb[1] * ndl),
              alb[2] * (S.ambient + S.light_rgb[2] * ndl));
  }
  // Cook-Torrance: GGX distribution, Smith-Schlick geometry (k = alpha/2), Schlick Fresnel.
  const float* cp = S.cam_pos + 3 * view;
  float3 P = f3(b[0] * p[0].x + b[1] * p[1].x + b[2] * p[2].x, b[0] * p[0].y + b[1] * p[1].y + b[2] * p[2].y,
                b[0] * p[0].z + b[1] * p[1].z + b[2] * p[2].z);
  float3 V = norm3(f3(__ldg(cp) - P.x, __ldg(cp + 1) - P.y, __ldg(cp + 2) - P.z));
  float3 Hh = norm3(f3(L.x + V.x, L.y + V.y, L.z + V.z));
  float ndv = fmaxf(dot3(n, V), 1e-4f), ndh = fmaxf(dot3(n, Hh), 0.0f), vdh = fmaxf(dot3(V, Hh), 0.0f);
  float r = fminf(fmaxf(rough[0], 0.02f), 1.0f);
  float a = r * r, a2 = a * a;
  float dd = ndh * ndh * (a2 - 1.0f) + 1.0f;
  float D = a2 / (3.14159265358979f * dd * dd);
  float kk = 0.5f * a;
  float G = (ndl / (ndl * (1.0f - kk) + kk)) * (ndv / (ndv * (1.0f - kk) + kk));
  float mt = metal[0], om = 1.0f - vdh;
  float om5 = om * om * om * om * om;
  float out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float F0 = 0.04f * (1.0f - mt) + alb[c] * mt;
    float F = F0 + (1.0f - F0) * om5;
    float diff = (1.0f - F) * (1.0f - mt) * alb[c] * ndl * 0.318309886183791f;
    float spec = D * G * F / (4.0f * ndv);
    out[c] = S.light_rgb[c] * (diff + spec) + S.ambient * alb[c];
  }
  return f3(out[0], out[1], out[2]);
}

// ---------------------------------------------------------------- one visible surface sample
// Everything about a pixel seen through one triangle on one side: UV, colour,
// footprints of the textures the shading reads.
struct Surf {
  float u, v;
  float3 rgb;
  Foot foot[MAX_READ];  // footprint of each read texture, in read_k order
};

// Perturbed world position of welded vertex vi.
__device__ __forceinline__ float3 perturbed_pos(const SceneDev& S, int vi, uint64_t key, int side) {
  const float* p = S.pos + 3ll * vi;
  uint64_t i0 = 3ull * (uint64_t)vi;
  return f3(perturb(__ldg(p), S.eps_pos, key, i0, side), perturb(__ldg(p + 1), S.eps_pos, key, i0 + 1, side),
            perturb(__ldg(p + 2), S.eps_pos, key, i0 + 2, side));
}

// Shade triangle `tri` at a pixel whose oriented edge functions are e[3] (set up as t).
__device__ __forceinline__ void surface(const SceneDev& S, int view, int tri, const Tri& t,
                                        const long long e[3], uint64_t key, int side, Surf& out) {
  float l[3];
  lambdas(e, t.inv_area, l);
  PerspW pw = persp(l, t.iw);
  int t0 = uv_of(S, tri, 0), t1 = uv_of(S, tri, 1), t2 = uv_of(S, tri, 2);
  float2 uv[3] = {make_float2(__ldg(S.uvs + 2 * t0), __ldg(S.uvs + 2 * t0 + 1)),
                  make_float2(__ldg(S.uvs + 2 * t1), __ldg(S.uvs + 2 * t1 + 1)),
                  make_float2(__ldg(S.uvs + 2 * t2), __ldg(S.uvs + 2 * t2 + 1))};
  out.u = persp_interp(pw, uv[0].x, uv[1].x, uv[2].x);
  out.v = persp_interp(pw, uv[0].y, uv[1].y, uv[2].y);
  float alb[4] = {1.f, 1.f, 1.f, 1.f}, nm[4] = {0.5f, 0.5f, 1.f, 0.f}, rough[4] = {0.5f, 0.f, 0.f, 0.f},
        metal[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < MAX_READ; ++r) {
    if (r >= S.nread) break;
    const TexDev& T = S.tex[S.read_k[r]];
    out.foot[r] = footprint(out.u, out.v, T.w, T.h);
    if (S.foot_nearest) out.foot[r].nearest = nearest_texel(out.u, out.v, T.w, T.h);
    float* dst = T.role == ROLE_ALBEDO ? alb : T.role == ROLE_NORMAL ? nm : T.role == ROLE_ROUGHNESS ? rough : metal;
    sample_tex(T, out.foot[r], key, side, dst);
  }
  if (S.shading == SHADE_UNLIT) {
    out.rgb = f3(alb[0], alb[1], alb[2]);
    return;
  }
  int v0 = vert_of(S, tri, 0), v1 = vert_of(S, tri, 1), v2 = vert_of(S, tri, 2);
  float3 p[3] = {perturbed_pos(S, v0, key, side), perturbed_pos(S, v1, key, side),
                 perturbed_pos(S, v2, key, side)};
  float b[3] = {pw.q[0] / pw.qs, pw.q[1] / pw.qs, pw.q[2] / pw.qs};
  out.rgb = shade(S, view, alb, nm, rough, metal, p, uv, b);
}

// ---------------------------------------------------------------- signs of one estimate, precomputed
// The fused estimators read s_i from what the vertex pass stored (3 bits per welded vertex) and
// from the texel sign planes (4 bits per texel) instead of hashing: the same values sign_neg gives.
struct PairSigns {
  const uint32_t* planes;  // this estimate's texel sign planes
  const uint8_t* vbits;    // this estimate's vertex sign bits (bits 0-2: x, y, z have s = -1)
  const int* sgn_off;      // word offset of texture k's plane (Workspace::sgn_off)
#if SGE_CHECKED
  const SceneDev* S;       // range checks of the plane words
#endif
};

__device__ __forceinline__ PairSigns pair_signs(const SceneDev& S, const Workspace& ws, int slot, int pb) {
  const long long e = (long long)slot * ws.max_pairs + pb;
#if SGE_CHECKED
  return PairSigns{ws.tsign + e * ws.sgn_words, ws.vbits + e * S.nv, ws.sgn_off, &S};
#else
  return PairSigns{ws.tsign + e * ws.sgn_words, ws.vbits + e * S.nv, ws.sgn_off};
#endif
}

// Sign bits of texel t of texture k (bit c: channel c has s = -1).
__device__ __forceinline__ uint32_t texel_signs(const PairSigns& ps, int k, long long t) {
  const long long w = ps.sgn_off[k] + (t >> 3);
#if SGE_CHECKED
  if (ps.S && !CHK_H(*ps.S, w, ps.S->chk.sign_words)) return 0u;
#endif
  return (__ldg(ps.planes + w) >> (4 * (t & 7))) & 0xFu;
}

// Sign bits of welded vertex v (bit c: coordinate c has s = -1).
__device__ __forceinline__ uint32_t vertex_signs(const PairSigns& ps, int v) { return __ldg(ps.vbits + v) & 7u; }

// sample_tex with the signs of ps.
__device__ __forceinline__ void sample_tex_ps(const TexDev& T, const Foot& f, const PairSigns& ps, int side,
                                              float out[4]) {
  float w[4] = {(1.0f - f.fx) * (1.0f - f.fy), f.fx * (1.0f - f.fy), (1.0f - f.fx) * f.fy, f.fx * f.fy};
  int tx[4] = {f.x0, f.x1, f.x0, f.x1};
  int ty[4] = {f.y0, f.y0, f.y1, f.y1};
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    long long t = (long long)ty[j] * T.w + tx[j];
    const float* src = T.ptr + t * T.c;
    uint32_t sb = texel_signs(ps, T.index, t);
    if (side < 0) sb = ~sb;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < T.c) out[c] += w[j] * __fadd_rn(__ldg(src + c), ((sb >> c) & 1) ? -T.eps : T.eps);
  }
  if (T.c == 1) out[1] = out[2] = out[0];
}

// surface() with the signs of ps (side +1 or -1).
__device__ __forceinline__ void surface_ps(const SceneDev& S, int view, int tri, const Tri& t, const long long e[3],
                                           const PairSigns& ps, int side, Surf& out) {
  float l[3];
  lambdas(e, t.inv_area, l);
  PerspW pw = persp(l, t.iw);
  int t0 = uv_of(S, tri, 0), t1 = uv_of(S, tri, 1), t2 = uv_of(S, tri, 2);
  float2 uv[3] = {make_float2(__ldg(S.uvs + 2 * t0), __ldg(S.uvs + 2 * t0 + 1)),
                  make_float2(__ldg(S.uvs + 2 * t1), __ldg(S.uvs + 2 * t1 + 1)),
                  make_float2(__ldg(S.uvs + 2 * t2), __ldg(S.uvs + 2 * t2 + 1))};
  out.u = persp_interp(pw, uv[0].x, uv[1].x, uv[2].x);
  out.v = persp_interp(pw, uv[0].y, uv[1].y, uv[2].y);
  float alb[4] = {1.f, 1.f, 1.f, 1.f}, nm[4] = {0.5f, 0.5f, 1.f, 0.f}, rough[4] = {0.5f, 0.f, 0.f, 0.f},
        metal[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < MAX_READ; ++r) {
    if (r >= S.nread) break;
    const TexDev& T = S.rtex[r];
    out.foot[r] = footprint(out.u, out.v, T.w, T.h);
    if (S.foot_nearest) out.foot[r].nearest = nearest_texel(out.u, out.v, T.w, T.h);
    float* dst = T.role == ROLE_ALBEDO ? alb : T.role == ROLE_NORMAL ? nm : T.role == ROLE_ROUGHNESS ? rough : metal;
    sample_tex_ps(T, out.foot[r], ps, side, dst);
  }
  if (S.shading == SHADE_UNLIT) {
    out.rgb = f3(alb[0], alb[1], alb[2]);
    return;
  }
  float3 p[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int vi = vert_of(S, tri, k);
    uint32_t sb = vertex_signs(ps, vi);
    if (side < 0) sb = ~sb;
    const float* src = S.pos + 3ll * vi;
    p[k] = f3(__fadd_rn(__ldg(src), (sb & 1) ? -S.eps_pos : S.eps_pos),
              __fadd_rn(__ldg(src + 1), (sb & 2) ? -S.eps_pos : S.eps_pos),
              __fadd_rn(__ldg(src + 2), (sb & 4) ? -S.eps_pos : S.eps_pos));
  }
  float b[3] = {pw.q[0] / pw.qs, pw.q[1] / pw.qs, pw.q[2] / pw.qs};
  out.rgb = shade(S, view, alb, nm, rough, metal, p, uv, b);
}

// Project the three perturbed vertices of `tri` and set it up at reference point (rx, ry).
__device__ __forceinline__ void setup_from_scene(const SceneDev& S, const float* m, int tri, uint64_t key,
                                                 int side, long long rx, long long ry, Tri& t) {
  PVert v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int vi = vert_of(S, tri, k);
    float3 q = perturbed_pos(S, vi, key, side);
    v[k] = project(m, q.x, q.y, q.z, S.W, S.H, S.near_w);
  }
  setup_tri(v[0], v[1], v[2], rx, ry, t);
}

// The tile's columns (bits 0-15) and rows (bits 16-31) whose pixel centres lie in the bounding
// box of the projected vertices v grown by `grow` fixed-point units per axis (rx, ry: the tile's
// first pixel centre).  Every perturbed version of a triangle lies in its box grown by the margin
// (each snapped vertex moves at most that far per axis), and a pixel inside the triangle in its
// box: a pre-filter for maybe_visible and surely_covers, which decide inside it.
__device__ __forceinline__ uint32_t box_span(const PVert (&v)[3], long long rx, long long ry, long long grow) {
  const long long xl = (long long)min(v[0].X, min(v[1].X, v[2].X)) - rx - grow;
  const long long xh = (long long)max(v[0].X, max(v[1].X, v[2].X)) - rx + grow;
  const long long yl = (long long)min(v[0].Y, min(v[1].Y, v[2].Y)) - ry - grow;
  const long long yh = (long long)max(v[0].Y, max(v[1].Y, v[2].Y)) - ry + grow;
  // pixel (dx, dy) sits at (256 dx, 256 dy): columns ceil(xl / 256) .. floor(xh / 256)
  const long long x0 = -((-xl) >> 8), x1 = xh >> 8, y0 = -((-yl) >> 8), y1 = yh >> 8;
  if (x0 > 15 || x1 < 0 || y0 > 15 || y1 < 0 || x0 > x1 || y0 > y1) return 0u;
  const int xa = (int)max(x0, 0ll), xb = (int)min(x1, 15ll), ya = (int)max(y0, 0ll), yb = (int)min(y1, 15ll);
  const uint32_t xm = ((2u << xb) - 1u) & ~((1u << xa) - 1u);
  const uint32_t ym = ((2u << yb) - 1u) & ~((1u << ya) - 1u);
  return xm | (ym << 16);
}

__device__ __forceinline__ bool in_span(uint32_t span, int dx, int dy) {
  return ((span >> dx) & (span >> (16 + dy)) & 1u) != 0;
}

// Evaluate the oriented edge functions of t at offset (dx, dy) pixels from its reference point.
__device__ __forceinline__ bool cover(const Tri& t, int dx, int dy, long long e[3]) {
  bool in = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e[k] = t.e0[k] + (long long)t.a[k] * (dx * 256) + (long long)t.b[k] * (dy * 256);
    in = in && (e[k] + t.bias[k] >= 0);
  }
  return in;
}

// ---------------------------------------------------------------- contributor set (Algorithm 2)
// Keys name a parameter group member: kind << 28 | index; kind 0 = welded vertex
// (its x, y, z), kind k+1 = texel of texture k (all its channels).
__device__ __forceinline__ uint32_t vkey(int v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t tkey(int k, int texel) { return ((uint32_t)(k + 1) << 28) | (uint32_t)texel; }

// Every parameter channel of a contributor key: f(parameter index, its channel slot in a table
// entry).  Vertex keys: x, y, z; texel keys: the texture's channels, or with GR (a group key of
// for_each_contrib<true>) channel c of every read texture r, at slot (channels of the read
// textures before r) + c.
template <bool GR, typename F>
__device__ __forceinline__ void for_each_channel(const SceneDev& S, uint32_t key, F&& f) {
  const uint32_t kind = key >> 28, idx = key & 0x0FFFFFFFu;
  if (kind == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) f(3ll * idx + c, c);
    return;
  }
  if constexpr (GR) {
    int co = 0;
#pragma unroll
    for (int r = 0; r < MAX_READ; ++r) {
      if (r >= S.nread) break;
      const TexDev& T = S.rtex[r];
      const long long base = T.offset + (long long)idx * T.c;
      for (int c = 0; c < T.c; ++c) f(base + c, co + c);
      co += T.c;
    }
  } else {
    const TexDev& T = S.tex[kind - 1];
    const long long base = T.offset + (long long)idx * T.c;
    for (int c = 0; c < T.c; ++c) f(base + c, c);
  }
}

// Sign of every parameter channel of a contributor key under ps: f(parameter index, slot, s = -1).
template <bool GR, typename F>
__device__ __forceinline__ void for_each_signed_channel(const SceneDev& S, const PairSigns& ps, uint32_t key, F&& f) {
  const uint32_t kind = key >> 28, idx = key & 0x0FFFFFFFu;
  if (kind == 0) {
    const uint32_t sb = vertex_signs(ps, (int)idx);
#pragma unroll
    for (int c = 0; c < 3; ++c) f(3ll * idx + c, c, ((sb >> c) & 1) != 0);
    return;
  }
  if constexpr (GR) {
    int co = 0;
#pragma unroll
    for (int r = 0; r < MAX_READ; ++r) {
      if (r >= S.nread) break;
      const TexDev& T = S.rtex[r];
      const long long base = T.offset + (long long)idx * T.c;
      const uint32_t sb = texel_signs(ps, T.index, idx);
      for (int c = 0; c < T.c; ++c) f(base + c, co + c, ((sb >> c) & 1) != 0);
      co += T.c;
    }
  } else {
    const TexDev& T = S.tex[kind - 1];
    const long long base = T.offset + (long long)idx * T.c;
    const uint32_t sb = texel_signs(ps, T.index, idx);
    for (int c = 0; c < T.c; ++c) f(base + c, c, ((sb >> c) & 1) != 0);
  }
}

__device__ __forceinline__ void key_params(const SceneDev& S, uint32_t key, long long& base, int& nch) {
  uint32_t kind = key >> 28, idx = key & 0x0FFFFFFFu;
  if (kind == 0) {
    base = 3ll * idx;
    nch = 3;
  } else {
    const TexDev& T = S.tex[kind - 1];
    base = T.offset + (long long)idx * T.c;
    nch = T.c;
  }
}

// Call f(key) once for every key of the pixel's contributor set: the union over
// both sides (tris[0] = side +, tris[1] = side -, -1 = background) of the visible
// triangle's three welded vertices and the bilinear 2x2 footprint of each read
// texture.  foot[sd][r] is side sd's footprint of the r-th read texture.
template <bool GR = false, typename F>
__device__ __forceinline__ void for_each_contrib(const SceneDev& S, const int tris[2],
                                                 const Foot (&foot)[2][MAX_READ], F&& f) {
  int vid[2][3];
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    if (tris[sd] < 0) continue;
#pragma unroll
    for (int k = 0; k < 3; ++k) vid[sd][k] = vert_of(S, tris[sd], k);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bool dup = false;
      if (sd == 1 && tris[0] >= 0) dup = vid[1][k] == vid[0][0] || vid[1][k] == vid[0][1] || vid[1][k] == vid[0][2];
      if (!dup) f(vkey(vid[sd][k]));
    }
  }
#pragma unroll
  for (int r = 0; r < (GR ? 1 : MAX_READ); ++r) {
    if (r >= S.nread) break;
    const int k = S.read_k[r];
    const int tw = S.tex[k].w;
    if (S.foot_nearest) {
      // one texel per side: the nearest one (Section 4.4), each once
      const int n0 = tris[0] >= 0 ? foot[0][r].nearest : -1;
      if (n0 >= 0) f(tkey(k, n0));
      if (tris[1] >= 0 && foot[1][r].nearest != n0) f(tkey(k, foot[1][r].nearest));
      continue;
    }
    int ids[2][4];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      if (tris[sd] < 0) continue;
      const Foot& ft = foot[sd][r];
      ids[sd][0] = ft.y0 * tw + ft.x0;
      ids[sd][1] = ft.y0 * tw + ft.x1;
      ids[sd][2] = ft.y1 * tw + ft.x0;
      ids[sd][3] = ft.y1 * tw + ft.x1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bool dup = false;
#pragma unroll
        for (int o = 0; o < q; ++o) dup = dup || ids[sd][o] == ids[sd][q];
        if (sd == 1 && tris[0] >= 0) {
#pragma unroll
          for (int o = 0; o < 4; ++o) dup = dup || ids[0][o] == ids[1][q];
        }
        if (!dup) f(tkey(k, ids[sd][q]));
      }
    }
  }
}

// Loss difference f+ - f- of one pixel written without cancellation (Table 1, Algorithm 2):
// sum_c (I+_c - I-_c)(I+_c + I-_c - 2 I_c); also returns f+ and f-.
__device__ __forceinline__ float loss_diff(float3 ip, float3 im, float3 t, float& fp, float& fm) {
  float a[3] = {ip.x, ip.y, ip.z}, b[3] = {im.x, im.y, im.z}, c[3] = {t.x, t.y, t.z};
  float df = 0.0f;
  fp = fm = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float dp = a[k] - c[k], dm = b[k] - c[k];
    fp += dp * dp;
    fm += dm * dm;
    df += (a[k] - b[k]) * (a[k] + b[k] - 2.0f * c[k]);
  }
  return df;
}

// One asset of a batched launch as the per-scene code expects it, in shared memory.
struct BatchSmem {
  AssetDesc d;
  ViewList vl;
  EstimateArgs a;
};

// Load asset ai of P into b (all threads of the CTA; the caller synchronises around it).
__device__ __forceinline__ void load_asset(const BatchArgs& P, int ai, BatchSmem& b) {
  const BatchAsset& A = P.as[ai];
  const int4* src = reinterpret_cast<const int4*>(A.desc);
  int4* dst = reinterpret_cast<int4*>(&b.d);
  for (int i = threadIdx.x; i < (int)(sizeof(AssetDesc) / 16); i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) {
    b.vl.n = A.n_views;
    b.a = EstimateArgs{P.seed, P.iter, P.pairs, P.pairs_per_item, P.pair_begin, P.pair_count,
                       A.grad, A.counts, A.loss, nullptr, P.iter_dev};
  }
  if (threadIdx.x < SGE_MAX_BATCH_VIEWS) b.vl.id[threadIdx.x] = A.view[threadIdx.x];
}

}  // namespace sge
