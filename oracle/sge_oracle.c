/*
 * CPU oracle for per-pixel stochastic gradient estimation through a plain
 * rasterizer (Deliot, Heitz, Belcour 2024).  TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it to check
 * and to time the GPU path; the library itself never calls it.
 *
 * It is written to be read against the paper, not to be fast:
 *   - every render loops over every triangle and every pixel of its bounding box;
 *   - every sign is recomputed from the counter-based hash when it is needed;
 *   - losses, loss differences and gradient sums are accumulated in double.
 *
 * Precision.  The paper's perturbation shader stores the perturbed parameters
 * theta +- s*eps as floats (Algorithm 1), so perturbed parameters are rounded
 * to float here too.  The steps whose float results decide integers (the
 * snapped screen position, the depth that picks the visible triangle, the UV
 * that picks texels) are evaluated in float, one rounding per written
 * operation, in the order written (compile with -ffp-contract=off).
 * Everything after that (colours, losses, sums, the descent step) is double.
 *
 * No code, header, table or constant is shared with the CUDA implementation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_TEX 8

enum { OR_ROLE_ALBEDO = 0, OR_ROLE_NORMAL = 1, OR_ROLE_ROUGHNESS = 2, OR_ROLE_METALLIC = 3 };
enum { OR_UNLIT = 0, OR_LAMBERT = 1, OR_GGX = 2, OR_TRANSPARENT = 3 };
#define OR_LAYERS 4 /* fragments a pixel's deep ID buffer keeps (transparent geometry) */
enum { OR_FOOT_BILINEAR = 0, OR_FOOT_NEAREST = 1 };

/* Everything describing one scene; mirrors the ctypes Structure in __init__.py. */
typedef struct {
    int32_t n_vertices, n_triangles, n_uvs, n_textures;
    const float *positions;   /* [V,3] welded vertex positions (parameters)          */
    const int32_t *pos_idx;   /* [T,3]                                                */
    const float *uvs;         /* [Vt,2]                                               */
    const int32_t *uv_idx;    /* [T,3]                                                */
    const float *tex[OR_MAX_TEX];   /* [H,W,C] texels (parameters)                    */
    int32_t tex_w[OR_MAX_TEX], tex_h[OR_MAX_TEX], tex_c[OR_MAX_TEX], tex_role[OR_MAX_TEX];
    float eps_tex[OR_MAX_TEX];
    float eps_pos;
    const float *eps_vec;     /* optional [d]: one magnitude per parameter (Table 1)  */
    int32_t n_views, width, height;
    const float *mvp;         /* [n_views,4,4] row-major, clip = M * (x,y,z,1)        */
    const float *cam_pos;     /* [n_views,3]                                          */
    float near_w;             /* vertices need clip w > near_w                        */
    const float *targets;     /* [n_views,H,W,3] target image I                       */
    float background[3];
    int32_t shading;
    float light_dir[3], light_rgb[3], ambient;
    int32_t footprint;
} or_scene;

/* ------------------------------------------------------------------ signs (Alg. 1)
 * The paper draws s_i with "a random hash function" (Algorithm 1) and does not
 * say which.  This oracle uses SplitMix64 (Steele, Lea & Flood, OOPSLA 2014):
 * or_mix64 is its output function and or_splitmix_next its generator step.
 * The key of one estimate chains four generator steps over (seed, iteration,
 * view, pair); s_i is bit (i mod 64) of the (floor(i / 64) + 1)-th output of the
 * generator seeded with that key (bit 0 -> +1, bit 1 -> -1): each 64-bit output
 * gives the signs of 64 consecutive parameters, one bit each.                      */
#define OR_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One step of the generator: advance the state, return the mixed state. */
uint64_t or_splitmix_next(uint64_t *state)
{
    *state += OR_GAMMA;
    return or_mix64(*state);
}

uint64_t or_pair_key(uint64_t seed, uint32_t iter, uint32_t view, uint32_t pair)
{
    uint64_t st = seed;
    uint64_t k = or_splitmix_next(&st);
    st = k ^ (uint64_t)iter;
    k = or_splitmix_next(&st);
    st = k ^ (uint64_t)view;
    k = or_splitmix_next(&st);
    st = k ^ (uint64_t)pair;
    return or_splitmix_next(&st);
}

/* s_i for parameter i under key k: +1 or -1, each with probability 1/2 (Eq. 4). */
int or_sign(uint64_t key, uint64_t i)
{
    uint64_t st = key + (i / 64) * OR_GAMMA; /* floor(i / 64) steps of the generator ... */
    uint64_t out = or_splitmix_next(&st);    /* ... then the next output                 */
    return ((out >> (i % 64)) & 1) ? -1 : 1;
}

/* The views of one iteration (Section 5 draws the view of each estimate at random): a
 * Fisher-Yates shuffle of 0..n-1 of which the first `count` entries are kept.  Step i swaps
 * entry i with entry i + (r_i mod (n - i)), r_i the (i+1)-th generator output from the key
 * (seed, iteration, view ~0, pair ~0).                                               */
int or_draw_views(uint64_t seed, uint32_t iter, int32_t n, int32_t count, int32_t *out)
{
    if (n < 1 || count < 1 || count > n) return 1;
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!a) return 2;
    for (int32_t i = 0; i < n; ++i) a[i] = i;
    uint64_t st = or_pair_key(seed, iter, 0xFFFFFFFFu, 0xFFFFFFFFu);
    for (int32_t i = 0; i < count; ++i) {
        uint64_t r = or_splitmix_next(&st);
        int32_t j = i + (int32_t)(r % (uint64_t)(n - i));
        int32_t t = a[i];
        a[i] = a[j];
        a[j] = t;
        out[i] = a[i];
    }
    free(a);
    return 0;
}

/* ------------------------------------------------------------------ parameters */
static int64_t or_n_pos(const or_scene *s) { return 3 * (int64_t)s->n_vertices; }

static int64_t or_tex_offset(const or_scene *s, int k)
{
    int64_t o = or_n_pos(s);
    for (int j = 0; j < k; ++j) o += (int64_t)s->tex_w[j] * s->tex_h[j] * s->tex_c[j];
    return o;
}

int64_t or_n_params(const or_scene *s) { return or_tex_offset(s, s->n_textures); }

static float or_eps(const or_scene *s, int64_t i, int group)
{
    if (s->eps_vec) return s->eps_vec[i];
    return group < 0 ? s->eps_pos : s->eps_tex[group];
}

/* theta_i + side * s_i * eps_i, stored as a float like the output of shader P. */
static float or_perturbed(const or_scene *s, float theta, int64_t i, int group,
                          uint64_t key, int side)
{
    if (side == 0) return theta;
    float e = or_eps(s, i, group);
    float d = (side * or_sign(key, (uint64_t)i) > 0) ? e : -e;
    return theta + d;
}

/* ------------------------------------------------------------------ projection
 * clip = M (x,y,z,1); x_ndc = clip.x / clip.w; screen x = (x_ndc/2 + 1/2) W,
 * screen y = (1/2 - y_ndc/2) H (row 0 at the top); both snapped to 1/256 pixel
 * (24.8 fixed point, round half to even).  A vertex needs clip.w > near_w and
 * |screen| < 2^15 pixels; a triangle with a vertex failing either is dropped. */
#define OR_GUARD 8388608.0f /* 2^23 fixed-point units = 2^15 pixels */

typedef struct { int ok; int32_t X, Y; float z, iw; } or_vtx;

static or_vtx or_project(const float *m, float px, float py, float pz, int W, int H, float near_w)
{
    or_vtx v;
    float cx = ((m[0] * px + m[1] * py) + m[2] * pz) + m[3];
    float cy = ((m[4] * px + m[5] * py) + m[6] * pz) + m[7];
    float cz = ((m[8] * px + m[9] * py) + m[10] * pz) + m[11];
    float cw = ((m[12] * px + m[13] * py) + m[14] * pz) + m[15];
    v.ok = cw > near_w;
    v.iw = 1.0f / cw;
    float xn = cx * v.iw, yn = cy * v.iw;
    v.z = cz * v.iw;
    float xs = (xn * 0.5f + 0.5f) * (float)W;
    float ys = (0.5f - yn * 0.5f) * (float)H;
    float xf = xs * 256.0f, yf = ys * 256.0f;
    if (!(fabsf(xf) < OR_GUARD) || !(fabsf(yf) < OR_GUARD)) v.ok = 0;
    v.X = v.ok ? (int32_t)nearbyintf(xf) : 0;
    v.Y = v.ok ? (int32_t)nearbyintf(yf) : 0;
    return v;
}

/* ------------------------------------------------------------------ triangles */
typedef struct {
    int ok;
    int32_t X[3], Y[3];
    float z[3], iw[3];
    float p[3][3];           /* perturbed world positions */
    int64_t area;            /* twice the signed screen area, made positive */
    int sgn;                 /* orientation of the projected triangle        */
    int tl[3];               /* edge k (opposite vertex k) is a top or left edge */
} or_tri;

/* Edge function of the edge opposite vertex k at fixed-point point (px,py):
 * E_k = (Xb-Xa)(py-Ya) - (Yb-Ya)(px-Xa) with a = k+1, b = k+2 (mod 3).
 * E_0 + E_1 + E_2 is twice the signed area; E_k / area is vertex k's weight. */
static int64_t or_edge(const or_tri *t, int k, int64_t px, int64_t py)
{
    int a = (k + 1) % 3, b = (k + 2) % 3;
    return ((int64_t)t->X[b] - t->X[a]) * (py - t->Y[a])
         - ((int64_t)t->Y[b] - t->Y[a]) * (px - t->X[a]);
}

/* Perturb, project and set up triangle `tri` for one side of one estimate. */
static void or_setup(const or_scene *s, int view, uint64_t key, int side, int tri, or_tri *t)
{
    const float *m = s->mvp + 16 * view;
    t->ok = 1;
    for (int k = 0; k < 3; ++k) {
        int vi = s->pos_idx[3 * tri + k];
        float q[3];
        for (int c = 0; c < 3; ++c) {
            int64_t i = 3 * (int64_t)vi + c;
            q[c] = or_perturbed(s, s->positions[i], i, -1, key, side);
            t->p[k][c] = q[c];
        }
        or_vtx v = or_project(m, q[0], q[1], q[2], s->width, s->height, s->near_w);
        if (!v.ok) t->ok = 0;
        t->X[k] = v.X; t->Y[k] = v.Y; t->z[k] = v.z; t->iw[k] = v.iw;
    }
    if (!t->ok) return;
    int64_t area = or_edge(t, 2, t->X[2], t->Y[2]);
    if (area == 0) { t->ok = 0; return; }
    t->sgn = area > 0 ? 1 : -1;
    t->area = area > 0 ? area : -area;
    for (int k = 0; k < 3; ++k) {
        int a = (k + 1) % 3, b = (k + 2) % 3;
        /* inward normal of the edge, in the positive orientation */
        int64_t nx = (int64_t)t->sgn * ((int64_t)t->Y[a] - t->Y[b]);
        int64_t ny = (int64_t)t->sgn * ((int64_t)t->X[b] - t->X[a]);
        /* y grows downwards: a left edge has the inside on +x, a top edge on +y */
        t->tl[k] = nx > 0 || (nx == 0 && ny > 0);
    }
}

/* Coverage of the pixel centre at fixed-point (px,py), top-left fill rule. */
static int or_inside(const or_tri *t, int64_t px, int64_t py, int64_t e[3])
{
    for (int k = 0; k < 3; ++k) {
        e[k] = t->sgn * or_edge(t, k, px, py);
        if (!(e[k] > 0 || (e[k] == 0 && t->tl[k]))) return 0;
    }
    return 1;
}

static void or_lambda(const or_tri *t, const int64_t e[3], float l[3])
{
    float inv_area = 1.0f / (float)t->area;
    for (int k = 0; k < 3; ++k) l[k] = (float)e[k] * inv_area;
}

static uint32_t or_ordered(float z)
{
    uint32_t b;
    memcpy(&b, &z, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

/* Depth|ID key of a covered pixel: smaller is nearer; equal depths keep the lower id. */
static uint64_t or_key(const or_tri *t, const int64_t e[3], int tri)
{
    float l[3];
    or_lambda(t, e, l);
    float z = ((l[0] * t->z[0]) + (l[1] * t->z[1])) + (l[2] * t->z[2]);
    return ((uint64_t)or_ordered(z) << 32) | (uint32_t)tri;
}

static int64_t or_floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

/* Pixels whose centres (256 px + 128 in fixed point) lie in the triangle's bounding box,
 * clipped to the image: [pxa, pxb] x [pya, pyb].                                */
static void or_pixel_box(const or_tri *t, int W, int H, int64_t *pxa, int64_t *pxb, int64_t *pya, int64_t *pyb)
{
    int32_t x0 = t->X[0], x1 = t->X[0], y0 = t->Y[0], y1 = t->Y[0];
    for (int k = 1; k < 3; ++k) {
        if (t->X[k] < x0) x0 = t->X[k];
        if (t->X[k] > x1) x1 = t->X[k];
        if (t->Y[k] < y0) y0 = t->Y[k];
        if (t->Y[k] > y1) y1 = t->Y[k];
    }
    *pxa = -or_floordiv(-((int64_t)x0 - 128), 256);
    *pxb = or_floordiv((int64_t)x1 - 128, 256);
    *pya = -or_floordiv(-((int64_t)y0 - 128), 256);
    *pyb = or_floordiv((int64_t)y1 - 128, 256);
    if (*pxa < 0) *pxa = 0;
    if (*pya < 0) *pya = 0;
    if (*pxb > W - 1) *pxb = W - 1;
    if (*pyb > H - 1) *pyb = H - 1;
}

/* ------------------------------------------------------------------ rasterizer R
 * Rasterize one (perturbed) scene into a depth|ID buffer (Section 4.4, opaque
 * geometry): for every triangle and every pixel centre of its bounding box,
 * keep the smallest key.  Background pixels keep ~0.                          */
static void or_raster(const or_scene *s, int view, uint64_t key, int side, uint64_t *keys)
{
    int W = s->width, H = s->height;
    for (int64_t p = 0; p < (int64_t)W * H; ++p) keys[p] = ~0ULL;
    for (int tri = 0; tri < s->n_triangles; ++tri) {
        or_tri t;
        or_setup(s, view, key, side, tri, &t);
        if (!t.ok) continue;
        int64_t pxa, pxb, pya, pyb;
        or_pixel_box(&t, W, H, &pxa, &pxb, &pya, &pyb);
        for (int64_t py = pya; py <= pyb; ++py)
            for (int64_t px = pxa; px <= pxb; ++px) {
                int64_t e[3];
                if (!or_inside(&t, 256 * px + 128, 256 * py + 128, e)) continue;
                uint64_t k = or_key(&t, e, tri);
                if (k < keys[py * W + px]) keys[py * W + px] = k;
            }
    }
}

/* ------------------------------------------------------------------ deep rasterizer (transparent geometry)
 * Section 4.4, transparent geometry: the raster pass outputs a deep ID buffer, the
 * front-to-back list of the triangles a pixel sees.  Here every pixel keeps the
 * OR_LAYERS smallest keys (depth bits, triangle id) among the triangles covering its
 * centre, in ascending order; unused slots hold ~0.  deep is [OR_LAYERS][H][W].   */
static void or_raster_deep(const or_scene *s, int view, uint64_t key, int side, uint64_t *deep)
{
    int W = s->width, H = s->height;
    int64_t npx = (int64_t)W * H;
    for (int64_t i = 0; i < OR_LAYERS * npx; ++i) deep[i] = ~0ULL;
    for (int tri = 0; tri < s->n_triangles; ++tri) {
        or_tri t;
        or_setup(s, view, key, side, tri, &t);
        if (!t.ok) continue;
        int64_t pxa, pxb, pya, pyb;
        or_pixel_box(&t, W, H, &pxa, &pxb, &pya, &pyb);
        for (int64_t py = pya; py <= pyb; ++py)
            for (int64_t px = pxa; px <= pxb; ++px) {
                int64_t e[3];
                if (!or_inside(&t, 256 * px + 128, 256 * py + 128, e)) continue;
                /* insert into the pixel's ascending list; the largest key falls off the end */
                uint64_t k = or_key(&t, e, tri);
                for (int j = 0; j < OR_LAYERS; ++j) {
                    uint64_t *slot = deep + j * npx + py * W + px;
                    if (k < *slot) {
                        uint64_t tmp = *slot;
                        *slot = k;
                        k = tmp;
                    }
                }
            }
    }
}

/* ------------------------------------------------------------------ UV buffer
 * Perspective-correct UV of the visible triangle (Section 4.4, textures):
 * q_k = lambda_k / w_k,  uv = sum q_k uv_k / sum q_k.                          */
typedef struct { float u, v; double b[3]; } or_uvs;

static or_uvs or_uv(const or_scene *s, const or_tri *t, int tri, int64_t px, int64_t py)
{
    int64_t e[3];
    for (int k = 0; k < 3; ++k) e[k] = t->sgn * or_edge(t, k, px, py);
    float l[3], q[3];
    or_lambda(t, e, l);
    for (int k = 0; k < 3; ++k) q[k] = l[k] * t->iw[k];
    float qs = (q[0] + q[1]) + q[2];
    const float *uv0 = s->uvs + 2 * s->uv_idx[3 * tri + 0];
    const float *uv1 = s->uvs + 2 * s->uv_idx[3 * tri + 1];
    const float *uv2 = s->uvs + 2 * s->uv_idx[3 * tri + 2];
    or_uvs r;
    r.u = (((q[0] * uv0[0]) + (q[1] * uv1[0])) + (q[2] * uv2[0])) / qs;
    r.v = (((q[0] * uv0[1]) + (q[1] * uv1[1])) + (q[2] * uv2[1])) / qs;
    for (int k = 0; k < 3; ++k) r.b[k] = (double)q[k] / (double)qs;
    return r;
}

/* ------------------------------------------------------------------ texture footprint
 * Texel centres sit at half-integer coordinates: x = u W - 1/2, x0 = floor(x),
 * fx = x - x0 (float).  u wraps, v clamps; row 0 is v = 0.  The bilinear
 * footprint is the 2x2 block (x0..x0+1, y0..y0+1); "nearest" is the single
 * texel (floor(u W), floor(v H)) whose square holds the sample point.          */
typedef struct { int n; int32_t tx[4], ty[4]; double w[4]; } or_foot;

static int or_wrap(int64_t i, int n) { int64_t r = i % n; return (int)(r < 0 ? r + n : r); }
static int or_clamp(int64_t i, int n) { return (int)(i < 0 ? 0 : (i > n - 1 ? n - 1 : i)); }

static void or_bilinear(float u, float v, int W, int H, or_foot *f)
{
    float x = u * (float)W - 0.5f, y = v * (float)H - 0.5f;
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    int64_t ix = (int64_t)xf, iy = (int64_t)yf;
    f->n = 4;
    for (int j = 0; j < 4; ++j) {
        int dx = j & 1, dy = j >> 1;
        f->tx[j] = or_wrap(ix + dx, W);
        f->ty[j] = or_clamp(iy + dy, H);
        f->w[j] = (dx ? (double)fx : 1.0 - (double)fx) * (dy ? (double)fy : 1.0 - (double)fy);
    }
}

static void or_nearest(float u, float v, int W, int H, or_foot *f)
{
    float x = u * (float)W, y = v * (float)H;
    f->n = 1;
    f->tx[0] = or_wrap((int64_t)floorf(x), W);
    f->ty[0] = or_clamp((int64_t)floorf(y), H);
    f->w[0] = 1.0;
}

/* Bilinear sample of perturbed texture k (all its channels, up to 4). */
static void or_sample(const or_scene *s, int k, const or_foot *f, uint64_t key, int side, double out[4])
{
    int W = s->tex_w[k], C = s->tex_c[k];
    int64_t off = or_tex_offset(s, k);
    for (int c = 0; c < 4; ++c) out[c] = 0.0;
    for (int j = 0; j < f->n; ++j) {
        int64_t t = (int64_t)f->ty[j] * W + f->tx[j];
        for (int c = 0; c < C; ++c) {
            int64_t i = off + t * C + c;
            out[c] += f->w[j] * (double)or_perturbed(s, s->tex[k][t * C + c], i, k, key, side);
        }
    }
    for (int c = C; c < 4; ++c) out[c] = (C == 1 && c < 3) ? out[0] : 0.0;
}

/* ------------------------------------------------------------------ shading */
static int or_find_role(const or_scene *s, int role)
{
    for (int k = 0; k < s->n_textures; ++k)
        if (s->tex_role[k] == role) return k;
    return -1;
}

/* Does the shading model read texture k (and so does k contribute to pixels)? */
static int or_reads(const or_scene *s, int k)
{
    int r = s->tex_role[k];
    if (or_find_role(s, r) != k) return 0; /* only the first texture of a role is read */
    if (s->shading == OR_UNLIT || s->shading == OR_TRANSPARENT) return r == OR_ROLE_ALBEDO;
    if (s->shading == OR_LAMBERT) return r == OR_ROLE_ALBEDO || r == OR_ROLE_NORMAL;
    return 1;
}

static double or_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void or_cross(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static void or_normalize(double a[3])
{
    double n = sqrt(or_dot(a, a));
    if (n > 0.0) { a[0] /= n; a[1] /= n; a[2] /= n; }
}

/* Shading normal: the normal map's tangent-space vector 2 t - 1 carried into the
 * frame (T, B, N) of the triangle's own perturbed geometry and UVs: N is the face
 * normal, T the direction of +u (Gram-Schmidt against N), B = N x T.            */
static void or_normal(const or_scene *s, const or_tri *t, int tri, const double nm[4], double n[3])
{
    double e1[3], e2[3], N[3], T[3], B[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = (double)t->p[1][c] - t->p[0][c];
        e2[c] = (double)t->p[2][c] - t->p[0][c];
    }
    or_cross(e1, e2, N);
    or_normalize(N);
    const float *uv0 = s->uvs + 2 * s->uv_idx[3 * tri + 0];
    const float *uv1 = s->uvs + 2 * s->uv_idx[3 * tri + 1];
    const float *uv2 = s->uvs + 2 * s->uv_idx[3 * tri + 2];
    double du1 = (double)uv1[0] - uv0[0], dv1 = (double)uv1[1] - uv0[1];
    double du2 = (double)uv2[0] - uv0[0], dv2 = (double)uv2[1] - uv0[1];
    double det = du1 * dv2 - du2 * dv1;
    for (int c = 0; c < 3; ++c) T[c] = det != 0.0 ? (e1[c] * dv2 - e2[c] * dv1) / det : e1[c];
    double nt = or_dot(N, T);
    for (int c = 0; c < 3; ++c) T[c] -= N[c] * nt;
    or_normalize(T);
    or_cross(N, T, B);
    double m[3] = { 2.0 * nm[0] - 1.0, 2.0 * nm[1] - 1.0, 2.0 * nm[2] - 1.0 };
    for (int c = 0; c < 3; ++c) n[c] = T[c] * m[0] + B[c] * m[1] + N[c] * m[2];
    if (or_dot(n, n) == 0.0) for (int c = 0; c < 3; ++c) n[c] = N[c];
    or_normalize(n);
}

/* Colour of a covered pixel seen through triangle `tri` on one side. */
static void or_shade(const or_scene *s, int view, const or_tri *t, int tri, const or_uvs *uv,
                     uint64_t key, int side, double rgb[3])
{
    double alb[4] = { 1, 1, 1, 1 }, nm[4] = { 0.5, 0.5, 1, 0 }, rough[4] = { 0.5, 0, 0, 0 },
           metal[4] = { 0, 0, 0, 0 };
    for (int k = 0; k < s->n_textures; ++k) {
        if (!or_reads(s, k)) continue;
        or_foot f;
        or_bilinear(uv->u, uv->v, s->tex_w[k], s->tex_h[k], &f);
        double *dst = s->tex_role[k] == OR_ROLE_ALBEDO ? alb
                    : s->tex_role[k] == OR_ROLE_NORMAL ? nm
                    : s->tex_role[k] == OR_ROLE_ROUGHNESS ? rough : metal;
        or_sample(s, k, &f, key, side, dst);
    }
    if (s->shading == OR_UNLIT) {
        for (int c = 0; c < 3; ++c) rgb[c] = alb[c];
        return;
    }
    double n[3], L[3] = { s->light_dir[0], s->light_dir[1], s->light_dir[2] };
    or_normal(s, t, tri, nm, n);
    double ndl = or_dot(n, L);
    if (ndl < 0.0) ndl = 0.0;
    if (s->shading == OR_LAMBERT) {
        for (int c = 0; c < 3; ++c) rgb[c] = alb[c] * (s->ambient + s->light_rgb[c] * ndl);
        return;
    }
    /* Cook-Torrance: GGX distribution, Smith-Schlick geometry (k = alpha/2),
     * Schlick Fresnel with F0 = 0.04 (1 - metallic) + albedo * metallic.        */
    double P[3], V[3], Hh[3];
    const float *cp = s->cam_pos + 3 * view;
    for (int c = 0; c < 3; ++c)
        P[c] = uv->b[0] * t->p[0][c] + uv->b[1] * t->p[1][c] + uv->b[2] * t->p[2][c];
    for (int c = 0; c < 3; ++c) V[c] = (double)cp[c] - P[c];
    or_normalize(V);
    for (int c = 0; c < 3; ++c) Hh[c] = L[c] + V[c];
    or_normalize(Hh);
    double ndv = or_dot(n, V), ndh = or_dot(n, Hh), vdh = or_dot(V, Hh);
    if (ndv < 1e-4) ndv = 1e-4;
    if (ndh < 0.0) ndh = 0.0;
    if (vdh < 0.0) vdh = 0.0;
    double r = rough[0] < 0.02 ? 0.02 : (rough[0] > 1.0 ? 1.0 : rough[0]);
    double a = r * r, a2 = a * a;
    double dd = ndh * ndh * (a2 - 1.0) + 1.0;
    double D = a2 / (M_PI * dd * dd);
    double kk = 0.5 * a;
    double G = (ndl / (ndl * (1.0 - kk) + kk)) * (ndv / (ndv * (1.0 - kk) + kk));
    double mt = metal[0], om = 1.0 - vdh;
    double om5 = om * om * om * om * om;
    for (int c = 0; c < 3; ++c) {
        double F0 = 0.04 * (1.0 - mt) + alb[c] * mt;
        double F = F0 + (1.0 - F0) * om5;
        double diff = (1.0 - F) * (1.0 - mt) * alb[c] * ndl / M_PI;
        double spec = D * G * F / (4.0 * ndv);
        rgb[c] = s->light_rgb[c] * (diff + spec) + s->ambient * alb[c];
    }
}

/* ------------------------------------------------------------------ transparent compositing
 * Section 4.4, transparent geometry: front-to-back rendering of the pixel's deep list.
 * Listed fragment j is unlit, with colour rgb_j and opacity a_j = clamp(alpha, 0, 1)
 * from the RGBA albedo sampled (bilinear) at its UV; with transmittance T_0 = 1,
 *   C = sum_j T_j a_j rgb_j + T_n background,   T_{j+1} = T_j (1 - a_j).
 * Fragments beyond the list are not drawn.  Returns the number n of listed
 * fragments; tris[j] and uvs[j] are fragment j's triangle and UV.               */
static int or_composite(const or_scene *s, int view, uint64_t key, int side, const uint64_t *deep, int64_t npx,
                        int64_t px, int64_t py, double rgb[3], int tris[OR_LAYERS], or_uvs uvs[OR_LAYERS])
{
    int ka = or_find_role(s, OR_ROLE_ALBEDO);
    int64_t p = py * s->width + px;
    double T = 1.0;
    int n = 0;
    for (int c = 0; c < 3; ++c) rgb[c] = 0.0;
    for (int j = 0; j < OR_LAYERS && ka >= 0; ++j) {
        uint64_t k = deep[j * npx + p];
        if (k == ~0ULL) break;
        int tri = (int)(k & 0xFFFFFFFFu);
        or_tri t;
        or_setup(s, view, key, side, tri, &t);
        uvs[j] = or_uv(s, &t, tri, 256 * px + 128, 256 * py + 128);
        or_foot f;
        or_bilinear(uvs[j].u, uvs[j].v, s->tex_w[ka], s->tex_h[ka], &f);
        double a[4];
        or_sample(s, ka, &f, key, side, a);
        double al = a[3] < 0.0 ? 0.0 : (a[3] > 1.0 ? 1.0 : a[3]);
        for (int c = 0; c < 3; ++c) rgb[c] += T * al * a[c];
        T *= 1.0 - al;
        tris[j] = tri;
        n++;
    }
    for (int c = 0; c < 3; ++c) rgb[c] += T * s->background[c];
    return n;
}

/* ------------------------------------------------------------------ public: deep render
 * The deep ID buffer of one render (see or_raster_deep), [OR_LAYERS][H][W], and with
 * rgb != NULL (transparent scenes only) its front-to-back composite [H][W][3].    */
int oracle_render_deep(const or_scene *s, int view, uint64_t seed, uint32_t iter, uint32_t pair, int side,
                       uint64_t *deep, double *rgb)
{
    if (view < 0 || view >= s->n_views || side < -1 || side > 1) return 1;
    if (rgb && s->shading != OR_TRANSPARENT) return 1;
    uint64_t key = or_pair_key(seed, iter, (uint32_t)view, pair);
    int64_t npx = (int64_t)s->width * s->height;
    or_raster_deep(s, view, key, side, deep);
    if (rgb)
        for (int64_t py = 0; py < s->height; ++py)
            for (int64_t px = 0; px < s->width; ++px) {
                int tris[OR_LAYERS];
                or_uvs uvs[OR_LAYERS];
                or_composite(s, view, key, side, deep, npx, px, py, rgb + 3 * (py * s->width + px), tris, uvs);
            }
    return 0;
}

int oracle_layers(void) { return OR_LAYERS; }

/* ------------------------------------------------------------------ public: render
 * One render of the scene theta + side * s * eps (side -1, 0 or +1) for the
 * estimate keyed by (seed, iter, view, pair): depth|ID keys, UV buffer (0 on
 * background) and colour (the background colour on background).  A transparent
 * scene gives its front fragment's key and UV and the composite colour.      */
int oracle_render(const or_scene *s, int view, uint64_t seed, uint32_t iter, uint32_t pair, int side,
                  uint64_t *keys, float *uv, double *rgb)
{
    if (view < 0 || view >= s->n_views || side < -1 || side > 1) return 1;
    uint64_t key = or_pair_key(seed, iter, (uint32_t)view, pair);
    int W = s->width, H = s->height;
    if (s->shading == OR_TRANSPARENT) {
        int64_t npx = (int64_t)W * H;
        uint64_t *deep = malloc(sizeof(uint64_t) * OR_LAYERS * npx);
        if (!deep) return 2;
        or_raster_deep(s, view, key, side, deep);
        for (int64_t py = 0; py < H; ++py)
            for (int64_t px = 0; px < W; ++px) {
                int64_t p = py * W + px;
                int tris[OR_LAYERS];
                or_uvs uvs[OR_LAYERS];
                double col[3];
                int n = or_composite(s, view, key, side, deep, npx, px, py, col, tris, uvs);
                keys[p] = deep[p];
                if (uv) { uv[2 * p] = n ? uvs[0].u : 0.0f; uv[2 * p + 1] = n ? uvs[0].v : 0.0f; }
                if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * p + c] = col[c];
            }
        free(deep);
        return 0;
    }
    or_raster(s, view, key, side, keys);
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            int64_t p = py * W + px;
            if (keys[p] == ~0ULL) {
                if (uv) uv[2 * p] = uv[2 * p + 1] = 0.0f;
                if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * p + c] = s->background[c];
                continue;
            }
            int tri = (int)(keys[p] & 0xFFFFFFFFu);
            or_tri t;
            or_setup(s, view, key, side, tri, &t);
            or_uvs u = or_uv(s, &t, tri, 256 * px + 128, 256 * py + 128);
            if (uv) { uv[2 * p] = u.u; uv[2 * p + 1] = u.v; }
            if (rgb) or_shade(s, view, &t, tri, &u, key, side, rgb + 3 * p);
        }
    return 0;
}

/* ------------------------------------------------------------------ contributor set
 * The parameters a pixel credits (Algorithm 2's loop "for each parameter
 * contributing to pixel (w,h)").  The algorithm reads one ID buffer, but an
 * estimate renders two scenes; the pixel credits the union over both sides of
 * (a) the three welded vertices of the visible triangle, x, y and z each, and
 * (b) the texels of the footprint of every texture the shading reads, all
 * channels.  Each parameter appears once per pixel.  In a transparent scene the
 * pixel credits this for every fragment of each side's deep list (Section 4.4: G
 * walks the list and treats each listed triangle as the opaque case does).     */
#define OR_MAX_CONTRIB 1024

typedef struct { int n; int64_t idx[OR_MAX_CONTRIB]; int group[OR_MAX_CONTRIB]; } or_set;

static void or_set_add(or_set *k, int64_t i, int group)
{
    for (int j = 0; j < k->n; ++j)
        if (k->idx[j] == i) return;
    if (k->n < OR_MAX_CONTRIB) { k->idx[k->n] = i; k->group[k->n] = group; k->n++; }
}

static void or_contributors(const or_scene *s, int tri, const or_uvs *uv, or_set *K)
{
    for (int k = 0; k < 3; ++k) {
        int vi = s->pos_idx[3 * tri + k];
        for (int c = 0; c < 3; ++c) or_set_add(K, 3 * (int64_t)vi + c, -1);
    }
    for (int k = 0; k < s->n_textures; ++k) {
        if (!or_reads(s, k)) continue;
        or_foot f;
        if (s->footprint == OR_FOOT_NEAREST) or_nearest(uv->u, uv->v, s->tex_w[k], s->tex_h[k], &f);
        else or_bilinear(uv->u, uv->v, s->tex_w[k], s->tex_h[k], &f);
        int64_t off = or_tex_offset(s, k);
        for (int j = 0; j < f.n; ++j) {
            int64_t t = (int64_t)f.ty[j] * s->tex_w[k] + f.tx[j];
            for (int c = 0; c < s->tex_c[k]; ++c) or_set_add(K, off + t * s->tex_c[k] + c, k);
        }
    }
}

/* ------------------------------------------------------------------ public: estimate
 * Per-pixel stochastic finite differences (Eq. 8), repeated over views and
 * pairs (Eq. 9).  For every listed view and every pair n < pairs:
 *   s = sign vector of key (seed, iter, view, n);  render theta + s eps and theta - s eps;
 *   f+-_p = || I_p(theta +- s eps) - I_p ||^2 per pixel (Table 1);
 *   for i in K(p):  S_i += (f+_p - f-_p) * s_i,  C_i += 1.
 * S is the numerator of Eq. 8 summed over pixels and estimates (s_i = 1/s_i);
 * the estimate of Eq. 9 is S_i / (2 eps_i N), N = views * pairs.
 * loss[j] = sum over pixels of the mean over pairs of (f+ + f-)/2.
 * Optional per-pixel outputs, each [n_views][pairs][H][W]: delta_f = f+ - f-,
 * fmax = max(f+, f-), cond = sum_c (|a_c| + |b_c|)(|I+_c| + |I-_c| + 2|I_c|) with
 * a = I+ - I-, b = I+ + I- - 2 I (the size of the terms in f+ - f-).
 * Transparent scenes render each side through its deep list (or_raster_deep,
 * or_composite).                                                                */
int oracle_estimate(const or_scene *s, uint64_t seed, uint32_t iter, const int32_t *view_ids,
                    int n_views, int pairs, double *S, uint64_t *C, double *loss,
                    double *delta_f, double *fmax, double *cond)
{
    int W = s->width, H = s->height;
    int64_t npx = (int64_t)W * H;
    /* transparent scenes keep a deep list per pixel (Section 4.4) and credit every listed fragment */
    int deep = s->shading == OR_TRANSPARENT;
    int64_t nbuf = deep ? OR_LAYERS * npx : npx;
    uint64_t *kp = malloc(sizeof(uint64_t) * nbuf), *km = malloc(sizeof(uint64_t) * nbuf);
    or_set *K = malloc(sizeof(or_set));
    if (!kp || !km || !K) { free(kp); free(km); free(K); return 2; }
    for (int j = 0; j < n_views; ++j) {
        int view = view_ids[j];
        if (view < 0 || view >= s->n_views) { free(kp); free(km); free(K); return 1; }
        const float *tgt = s->targets + (int64_t)view * npx * 3;
        if (loss) loss[j] = 0.0;
        for (int n = 0; n < pairs; ++n) {
            uint64_t key = or_pair_key(seed, iter, (uint32_t)view, (uint32_t)n);
            if (deep) {
                or_raster_deep(s, view, key, +1, kp);
                or_raster_deep(s, view, key, -1, km);
            } else {
                or_raster(s, view, key, +1, kp);
                or_raster(s, view, key, -1, km);
            }
            for (int64_t py = 0; py < H; ++py)
                for (int64_t px = 0; px < W; ++px) {
                    int64_t p = py * W + px;
                    double col[2][3];
                    or_uvs uvl[2][OR_LAYERS];
                    int tris[2][OR_LAYERS], nl[2];
                    K->n = 0;
                    for (int sd = 0; sd < 2; ++sd) {
                        const uint64_t *buf = sd == 0 ? kp : km;
                        int side = sd == 0 ? +1 : -1;
                        if (deep) {
                            nl[sd] = or_composite(s, view, key, side, buf, npx, px, py, col[sd], tris[sd], uvl[sd]);
                            continue;
                        }
                        nl[sd] = 0;
                        if (buf[p] == ~0ULL) {
                            for (int c = 0; c < 3; ++c) col[sd][c] = s->background[c];
                            continue;
                        }
                        nl[sd] = 1;
                        tris[sd][0] = (int)(buf[p] & 0xFFFFFFFFu);
                        or_tri t;
                        or_setup(s, view, key, side, tris[sd][0], &t);
                        uvl[sd][0] = or_uv(s, &t, tris[sd][0], 256 * px + 128, 256 * py + 128);
                        or_shade(s, view, &t, tris[sd][0], &uvl[sd][0], key, side, col[sd]);
                    }
                    double fp = 0.0, fm = 0.0, cd = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        double T = tgt[3 * p + c];
                        fp += (col[0][c] - T) * (col[0][c] - T);
                        fm += (col[1][c] - T) * (col[1][c] - T);
                        double a = col[0][c] - col[1][c], b = col[0][c] + col[1][c] - 2.0 * T;
                        cd += (fabs(a) + fabs(b)) * (fabs(col[0][c]) + fabs(col[1][c]) + 2.0 * fabs(T));
                    }
                    double df = fp - fm;
                    int64_t o = ((int64_t)j * pairs + n) * npx + p;
                    if (delta_f) delta_f[o] = df;
                    if (fmax) fmax[o] = fp > fm ? fp : fm;
                    if (cond) cond[o] = cd;
                    if (loss) loss[j] += 0.5 * (fp + fm) / pairs;
                    for (int sd = 0; sd < 2; ++sd)
                        for (int j = 0; j < nl[sd]; ++j) or_contributors(s, tris[sd][j], &uvl[sd][j], K);
                    for (int q = 0; q < K->n; ++q) {
                        int64_t i = K->idx[q];
                        S[i] += df * or_sign(key, (uint64_t)i);
                        C[i] += 1;
                    }
                }
        }
    }
    free(kp);
    free(km);
    free(K);
    return 0;
}

/* ------------------------------------------------------------------ public: full-image estimate
 * The stochastic finite difference of Eq. 4 with the whole-image error f (the estimator the
 * per-pixel formulation replaces; Section 6.1 compares the two).  For every listed view and
 * pair n < pairs: s = sign vector of key (seed, iter, view, n); render theta + s eps and
 * theta - s eps; dF = f(theta + s eps) - f(theta - s eps) = sum_p (f+_p - f-_p) (Table 1);
 * then for EVERY parameter i: S_i += dF * s_i, C_i += 1.  The estimate is S_i / (2 eps_i N).
 * Per estimate e = j * pairs + n also: dF[e], and for error bounds sum_p |f+_p - f-_p|,
 * sum_p max(f+_p, f-_p), sum_p cond_p (cond as in oracle_estimate).                        */
int oracle_estimate_full_image(const or_scene *s, uint64_t seed, uint32_t iter, const int32_t *view_ids,
                               int n_views, int pairs, double *S, uint64_t *C, double *dF, double *sum_abs,
                               double *sum_fmax, double *sum_cond)
{
    int W = s->width, H = s->height;
    int64_t npx = (int64_t)W * H, d = or_n_params(s);
    if (s->shading == OR_TRANSPARENT) return 3; /* the whole-image form is written for opaque scenes */
    uint64_t *kp = malloc(sizeof(uint64_t) * npx), *km = malloc(sizeof(uint64_t) * npx);
    if (!kp || !km) { free(kp); free(km); return 2; }
    for (int j = 0; j < n_views; ++j) {
        int view = view_ids[j];
        if (view < 0 || view >= s->n_views) { free(kp); free(km); return 1; }
        const float *tgt = s->targets + (int64_t)view * npx * 3;
        for (int n = 0; n < pairs; ++n) {
            uint64_t key = or_pair_key(seed, iter, (uint32_t)view, (uint32_t)n);
            or_raster(s, view, key, +1, kp);
            or_raster(s, view, key, -1, km);
            double F = 0.0, A = 0.0, M = 0.0, K = 0.0;
            for (int64_t py = 0; py < H; ++py)
                for (int64_t px = 0; px < W; ++px) {
                    int64_t p = py * W + px;
                    double col[2][3];
                    for (int sd = 0; sd < 2; ++sd) {
                        uint64_t k = sd == 0 ? kp[p] : km[p];
                        int side = sd == 0 ? +1 : -1;
                        if (k == ~0ULL) {
                            for (int c = 0; c < 3; ++c) col[sd][c] = s->background[c];
                            continue;
                        }
                        int tri = (int)(k & 0xFFFFFFFFu);
                        or_tri t;
                        or_setup(s, view, key, side, tri, &t);
                        or_uvs uv = or_uv(s, &t, tri, 256 * px + 128, 256 * py + 128);
                        or_shade(s, view, &t, tri, &uv, key, side, col[sd]);
                    }
                    double fp = 0.0, fm = 0.0, cd = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        double T = tgt[3 * p + c];
                        fp += (col[0][c] - T) * (col[0][c] - T);
                        fm += (col[1][c] - T) * (col[1][c] - T);
                        double a = col[0][c] - col[1][c], b = col[0][c] + col[1][c] - 2.0 * T;
                        cd += (fabs(a) + fabs(b)) * (fabs(col[0][c]) + fabs(col[1][c]) + 2.0 * fabs(T));
                    }
                    F += fp - fm;
                    A += fabs(fp - fm);
                    M += fp > fm ? fp : fm;
                    K += cd;
                }
            int64_t e = (int64_t)j * pairs + n;
            if (dF) dF[e] = F;
            if (sum_abs) sum_abs[e] = A;
            if (sum_fmax) sum_fmax[e] = M;
            if (sum_cond) sum_cond[e] = K;
            for (int64_t i = 0; i < d; ++i) {
                S[i] += F * or_sign(key, (uint64_t)i);
                C[i] += 1;
            }
        }
    }
    free(kp);
    free(km);
    return 0;
}

/* ------------------------------------------------------------------ public: full-image loss
 * f(theta) = sum_p || I_p(theta) - I_p ||^2 of the unperturbed scene (Table 1). */
double oracle_loss(const or_scene *s, int view)
{
    int64_t npx = (int64_t)s->width * s->height;
    uint64_t *keys = malloc(sizeof(uint64_t) * npx);
    double *rgb = malloc(sizeof(double) * 3 * npx);
    if (!keys || !rgb) { free(keys); free(rgb); return -1.0; }
    oracle_render(s, view, 0, 0, 0, 0, keys, NULL, rgb);
    const float *tgt = s->targets + (int64_t)view * npx * 3;
    double f = 0.0;
    for (int64_t i = 0; i < 3 * npx; ++i) f += (rgb[i] - tgt[i]) * (rgb[i] - tgt[i]);
    free(keys);
    free(rgb);
    return f;
}

/* ------------------------------------------------------------------ public: descent step
 * Gradient estimate g_i = S_i / (2 eps_i N) (Eq. 9), then one step per parameter:
 *   kind 0, SGD:  theta -= lr_i g_i
 *   kind 1, Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *           theta -= lr_i (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + adam_eps)
 *   kind 2, SGD on the per-pixel mean: g_i = S_i / (2 eps_i max(C_i, 1)).
 * The paper runs Adam with b1 = 0.9, b2 = 0.999 and lr_i = eps_i (Section 5).  */
void oracle_step(int kind, int64_t d, const float *theta, const double *S, const uint64_t *C,
                 const float *eps, const float *lr, int64_t n_total, double b1, double b2,
                 double adam_eps, int t, const float *m_in, const float *v_in,
                 double *theta_out, double *m_out, double *v_out)
{
    for (int64_t i = 0; i < d; ++i) {
        double g;
        if (kind == 2) g = S[i] / (2.0 * (double)eps[i] * (double)(C[i] > 0 ? C[i] : 1));
        else g = S[i] / (2.0 * (double)eps[i] * (double)n_total);
        if (kind == 1) {
            double m = b1 * (double)m_in[i] + (1.0 - b1) * g;
            double v = b2 * (double)v_in[i] + (1.0 - b2) * g * g;
            double mh = m / (1.0 - pow(b1, t)), vh = v / (1.0 - pow(b2, t));
            theta_out[i] = (double)theta[i] - (double)lr[i] * mh / (sqrt(vh) + adam_eps);
            m_out[i] = m;
            v_out[i] = v;
        } else {
            theta_out[i] = (double)theta[i] - (double)lr[i] * g;
        }
    }
}
