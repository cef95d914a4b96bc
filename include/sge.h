/*
 * sge.h -- C ABI of a GB300 (sm_103a) implementation of per-pixel stochastic
 * gradient estimation through a plain rasterizer (Deliot, Heitz, Belcour,
 * "Transforming a Non-Differentiable Rasterizer into a Differentiable One with
 * Stochastic Gradient Estimation", 2024).
 *
 * One optimisation iteration of the paper (Section 5) is
 *     repeat N times:  P (perturb, Algorithm 1) -> R (rasterize theta + s eps and
 *                      theta - s eps, Section 4.3) -> G (per-pixel loss difference,
 *                      scattered to the contributing parameters, Algorithm 2, Eq. 8)
 *     then D (descent step on the averaged estimate, Eq. 9, Section 5).
 * Here sge_estimate_grad runs all N estimates of one iteration (several views,
 * several antithetic pairs per view) in one persistent launch and
 * sge_step runs D; sge_render_idb exposes one render of R with its ID and UV
 * buffers (Section 4.4).
 *
 * Conventions shared by every call
 *  - Every pointer named "device" is CUDA device memory owned by the caller; the
 *    library borrows it for the lifetime of the scene and never frees it.
 *  - The library never allocates device memory: scratch lives in a caller-owned
 *    workspace of sge_workspace_size() bytes.
 *  - Calls are asynchronous and ordered on the stream given (a cudaStream_t,
 *    NULL = legacy default stream).  They never synchronise; errors detected by
 *    kernels (bin overflow, bad indices) land in a device status word that
 *    sge_status() reads.
 *  - Return value: SGE_OK or an sge_result code; sge_last_error() gives a
 *    thread-local message for the last failing call of the calling thread.
 *  - Parameter vector theta (Table 1): all vertex coordinates first (vertex-major
 *    x,y,z), then each texture in order, row-major (y, x, channel).
 *  - A scene is not thread-safe: calls on one scene must be serialised by the caller,
 *    across streams too.  Every call on a scene uses its one workspace (bins, work lists,
 *    counters), so work enqueued on two streams (or a replayed CUDA graph and an eager call on
 *    another stream) must be ordered by the caller with events or a synchronisation.
 */
#ifndef SGE_H
#define SGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGE_MAX_TEXTURES 8
#define SGE_MAX_VIEWS_PER_CALL 64
#define SGE_MAX_BATCH 64        /* assets of one sge_estimate_grad_batch call */
#define SGE_MAX_BATCH_VIEWS 8   /* views per asset of one batched call        */

typedef enum {
    SGE_OK = 0,
    SGE_ERR_INVALID_ARG = 1,   /* a bad argument or descriptor (message says which) */
    SGE_ERR_CUDA = 2,          /* a CUDA runtime call failed                         */
    SGE_ERR_BIN_OVERFLOW = 3,  /* (device status) tile bins exceeded bin_capacity    */
    SGE_ERR_BAD_INDEX = 4,     /* (device status) an index buffer entry out of range */
    SGE_ERR_UNSUPPORTED = 5,   /* a valid request the library does not implement     */
    SGE_ERR_WORKSPACE = 6,     /* workspace missing, too small or misaligned         */
    SGE_ERR_BOUNDS = 7         /* (device status, checked build) an index failed its
                                  range check; that access was skipped               */
} sge_result;

/* Texture roles: what the shading model reads a texture as. */
enum { SGE_ROLE_ALBEDO = 0, SGE_ROLE_NORMAL = 1, SGE_ROLE_ROUGHNESS = 2, SGE_ROLE_METALLIC = 3 };
/* Shading models: unlit albedo; Lambert + normal map; GGX (Cook-Torrance) + 4 maps;
 * transparent geometry (Section 4.4): unlit RGBA fragments composited front to back.
 * A transparent scene's raster pass keeps a deep ID buffer: for every pixel the
 * SGE_MAX_LAYERS covering fragments with the smallest (depth bits << 32 | triangle id)
 * keys, ascending; farther fragments are not drawn.  Fragment j has colour rgb_j and
 * opacity a_j = clamp(alpha_j, 0, 1) from the bilinear RGBA albedo (4 channels required)
 * and the pixel is C = sum_j T_j a_j rgb_j + T_n background, T_0 = 1, T_{j+1} = T_j (1 - a_j).
 * Its contributor set is every listed fragment's three vertices and albedo footprint, on
 * both sides.  Transparent scenes take sge_estimate_grad, sge_loss, sge_render_deep,
 * sge_gradient and sge_step; the other estimate and render calls return
 * SGE_ERR_UNSUPPORTED for them. */
enum { SGE_SHADE_UNLIT = 0, SGE_SHADE_LAMBERT = 1, SGE_SHADE_GGX = 2, SGE_SHADE_TRANSPARENT = 3 };
#define SGE_MAX_LAYERS 4 /* fragments per pixel of a transparent scene's deep ID buffer */
/* Descent steps (Section 5).  MEAN divides each sum by its count instead of 2 eps N. */
enum { SGE_STEP_SGD = 0, SGE_STEP_ADAM = 1, SGE_STEP_SGD_MEAN = 2 };

typedef struct CUstream_st *sge_stream_t; /* identical to cudaStream_t */

/* One texture parameter group (texels are parameters theta_i, Table 1). */
typedef struct {
    float *texels;          /* device, [height][width][channels] float32, row-major      */
    int32_t width, height;  /* >= 1, width*height < 2^28                                  */
    int32_t channels;       /* 1..4                                                       */
    float eps;              /* perturbation magnitude eps_i of every texel channel        */
    int32_t role;           /* SGE_ROLE_*; only the first texture of each role is read    */
} sge_texture;

/* Scene: a triangle mesh (opaque, or transparent with SGE_SHADE_TRANSPARENT) with textures
 * seen from n_views cameras. */
typedef struct {
    float *positions;       /* device, [n_vertices][3] float32 (parameters)               */
    int32_t n_vertices;     /* >= 3, < 2^28                                                */
    float eps_pos;          /* perturbation magnitude of every vertex coordinate          */
    const int32_t *pos_idx; /* device, [n_triangles][3] into positions (welded vertices)  */
    int32_t n_triangles;    /* >= 1                                                        */
    const float *uvs;       /* device, [n_uvs][2] float32                                 */
    int32_t n_uvs;
    const int32_t *uv_idx;  /* device, [n_triangles][3] into uvs                          */
    int32_t n_textures;     /* 0..SGE_MAX_TEXTURES                                        */
    sge_texture textures[SGE_MAX_TEXTURES];
    const float *mvp;       /* device, [n_views][4][4] row-major; clip = M (x,y,z,1)      */
    const float *cam_pos;   /* device, [n_views][3] eye positions (GGX view vector)       */
    int32_t n_views;
    int32_t width, height;  /* render size, 1..16384                                      */
    float near_w;           /* a vertex needs clip w > near_w, else its triangle drops    */
    const float *targets;   /* device, [n_views][height][width][3] target images I        */
    float background[3];    /* colour of uncovered pixels                                 */
    int32_t shading;        /* SGE_SHADE_*; the textures must include the roles it reads:
                               unlit albedo; Lambert albedo, normal; GGX all four;
                               transparent a 4-channel (RGBA) albedo                     */
    float light_dir[3];     /* unit vector towards the light, world space                 */
    float light_rgb[3];
    float ambient;
} sge_scene_desc;

/* Tuning knobs; zero-initialise for defaults. */
typedef struct {
    int32_t max_views_per_call; /* views per estimate call the workspace is sized for (default n_views, <= 64) */
    int64_t bin_capacity;       /* triangle-tile bin entries over those views (default (6 n_triangles + 8 tiles) * views) */
    int32_t pairs_per_item;     /* antithetic pairs one CTA runs per (view, tile) item (default 8, <= 64) */
    int32_t blocks_per_sm;      /* persistent CTAs per SM (default: as many as fit) */
    int32_t max_pairs_per_call; /* pairs per view projected at once (default 64); more run in blocks */
    int32_t footprint;          /* texels a pixel credits (SGE_FOOT_*; default bilinear)           */
} sge_config;

/* Texels a pixel credits for each texture the shading reads (Algorithm 2's contributor set).
 * Rendering samples bilinearly either way.  SGE_FOOT_BILINEAR credits the 2x2 bilinear
 * footprint, which makes Eq. 8 unbiased for textures the image depends on linearly;
 * SGE_FOOT_NEAREST credits the single texel whose square holds the sample point,
 * (floor(u W) wrapped, floor(v H) clamped), as Section 4.4 ("Textures") describes. */
#define SGE_FOOT_BILINEAR 0
#define SGE_FOOT_NEAREST 1

typedef struct {
    int32_t kind;                       /* SGE_STEP_*                                   */
    float lr_pos;                       /* learning rate of vertex coordinates          */
    float lr_tex[SGE_MAX_TEXTURES];     /* learning rate of each texture                */
    float beta1, beta2, adam_eps;       /* Adam (Kingma & Ba 2015); paper: 0.9, 0.999   */
    int32_t t;                          /* Adam step number, >= 1 (bias correction)     */
} sge_opt;

typedef struct sge_scene sge_scene;

/* Bytes of device workspace a scene needs: scratch for bins and tile lists, the
 * projected perturbed vertices of max_views_per_call x max_pairs_per_call
 * estimates (32 B + 1 B per vertex each), and the staged buffers of
 * sge_render_idb (Section 4.4). */
int sge_workspace_size(const sge_scene_desc *desc, const sge_config *cfg, size_t *bytes);

/* Validate desc (host-side checks only: sizes, pointers, enums) and create a scene
 * that borrows every device pointer in desc and uses `workspace` (device, 256-byte
 * aligned, >= sge_workspace_size bytes) as scratch.  *out receives a host object to
 * release with sge_destroy_scene.  Index buffers are checked on the device by
 * sge_validate (status SGE_ERR_BAD_INDEX). */
int sge_create_scene(const sge_scene_desc *desc, const sge_config *cfg, void *workspace,
                     size_t workspace_bytes, sge_scene **out);

/* Number of parameters d of the scene (Table 1). */
int sge_num_params(const sge_scene *scene, int64_t *d);

/* Point the scene at new target images (device, same layout as desc->targets). */
int sge_set_targets(sge_scene *scene, const float *targets);

/* Enqueue a range check of pos_idx / uv_idx; failures set SGE_ERR_BAD_INDEX. */
int sge_validate(sge_scene *scene, sge_stream_t stream);

/* Rasterize one perturbed scene (Section 4.3, R; ID and UV buffers, Section 4.4):
 * theta + side * s eps with s the sign vector of estimate (seed, iter, view, pair)
 * and side in {-1, 0, +1} (0 = unperturbed).  Outputs (device, any may be NULL):
 *   depth_id [height][width] uint64: (ordered depth bits << 32) | triangle id of the
 *            visible triangle (smallest depth, then lowest id), ~0 on background;
 *   uv       [height][width][2] float32 perspective-correct UV, 0 on background;
 *   rgb      [height][width][3] float32 shaded colour, background colour where uncovered. */
int sge_render_idb(sge_scene *scene, int32_t view, uint64_t seed, uint32_t iter, uint32_t pair,
                   int32_t side, uint64_t *depth_id, float *uv, float *rgb, sge_stream_t stream);

/* Transparent geometry (Section 4.4): one render's deep ID buffer and its front-to-back
 * composite, for a scene of shading SGE_SHADE_TRANSPARENT (else SGE_ERR_UNSUPPORTED).
 * The render is theta + side * s * eps (side -1, 0 or +1) with s drawn for
 * (seed, iter, view, pair) as sge_estimate_grad draws it.  deep_ids (device
 * [SGE_MAX_LAYERS][height][width] uint64, or NULL) receives each pixel's ascending
 * (depth bits << 32 | triangle id) keys, ~0 in unused slots; rgb (device
 * [height][width][3] float32, or NULL) the composite colour. */
int sge_render_deep(sge_scene *scene, int32_t view, uint64_t seed, uint32_t iter, uint32_t pair, int32_t side,
                    uint64_t *deep_ids, float *rgb, sge_stream_t stream);

/* All estimates of one iteration (Eq. 9): for each of the n_views views in view_ids
 * (host array, distinct indices < desc->n_views, n_views <= max_views_per_call) and
 * each pair n < pairs_per_view, render theta +- s eps with s drawn from
 * (seed, iter, view, n) and, per pixel p, add (f+_p - f-_p) s_i to grad_sums[i]
 * and 1 to counts[i] for every parameter i contributing to p on either side
 * (Algorithm 2, Eq. 8; the three welded vertices of the visible triangle and the
 * bilinear 2x2 texel footprint of every texture the shading reads).
 * grad_sums [d] float32 and counts [d] uint32 (device) ACCUMULATE: zero them
 * before the first call (sge_step zeroes them).  The estimate of Eq. 9 is
 * grad_sums[i] / (2 eps_i N) with N = n_views * pairs_per_view.
 * loss_out (device [n_views] float32 or NULL) ACCUMULATES, per view, the sum
 * over pixels of the mean over pairs of (f+ + f-)/2.
 * delta_f_out (device [n_views][pairs_per_view][height][width] float32 or NULL)
 * receives f+ - f- per pixel (a debugging output; it costs bandwidth). */
int sge_estimate_grad(sge_scene *scene, uint64_t seed, uint32_t iter, const int32_t *view_ids,
                      int32_t n_views, int32_t pairs_per_view, float *grad_sums, uint32_t *counts,
                      float *loss_out, float *delta_f_out, sge_stream_t stream);

/* Same results as sge_estimate_grad, computed the plain way: for every (view, pair)
 * separate launches render both sides into ID/UV buffers, form f+ - f- per pixel
 * and scatter with global atomics, one estimate after another (the paper's
 * P -> R -> G loop of Section 5).  Kept as the baseline the batched path is
 * measured against. */
int sge_estimate_grad_plain(sge_scene *scene, uint64_t seed, uint32_t iter, const int32_t *view_ids,
                            int32_t n_views, int32_t pairs_per_view, float *grad_sums,
                            uint32_t *counts, float *loss_out, sge_stream_t stream);

/* The full-image estimator the per-pixel form replaces (Eq. 4 with the whole-image error;
 * Section 6.1 compares the two): for each of the n_views views in view_ids and each pair
 * n < pairs_per_view, with s drawn from (seed, iter, view, n) exactly as sge_estimate_grad
 * draws it, dF = f(theta + s eps) - f(theta - s eps) summed over the whole image, then EVERY
 * parameter i gets grad_sums[i] += dF s_i and counts[i] += 1 (ACCUMULATE, as in
 * sge_estimate_grad; the estimate is grad_sums[i] / (2 eps_i N)).  image_df (device
 * [n_views][pairs_per_view] float32, required) receives each estimate's dF.  Runs the renders
 * one estimate at a time (staged ID/UV buffers); n_views * pairs_per_view <= 4096. */
int sge_estimate_grad_full_image(sge_scene *scene, uint64_t seed, uint32_t iter, const int32_t *view_ids,
                                 int32_t n_views, int32_t pairs_per_view, float *grad_sums, uint32_t *counts,
                                 float *image_df, sge_stream_t stream);

/* Control-mesh optimisation through a subdivision (linear or Catmull-Clark; the paper tessellates
 * a Catmull-Clark surface on the fly and credits each tessellated triangle to its control mesh,
 * Section 6.3): the subdivided mesh's vertices are a fixed linear map of the control vertices,
 * fine = R control, so the control vertices' gradient is R^T times the fine vertices' one, and
 * R^T applied to the sums of sge_estimate_grad (the first 3 V_fine entries) gives sums whose
 * Eq. 9 estimate (/ 2 eps N) is that of the control coordinates.  sge_refine computes, for
 * every row r of a CSR matrix A (device row_ptr [n_rows + 1], col [nnz], w [nnz] float32),
 * y[3r + k] = sum_j w_j x[3 col_j + k] for k = 0, 1, 2 (x, y device float32; accumulate != 0
 * adds to y instead of overwriting it), summing each row in order.  Pass R to refine
 * positions (fine = R control) and R^T's CSR to map sums (control += R^T fine). */
int sge_refine(const int32_t *row_ptr, const int32_t *col, const float *w, int32_t n_rows, const float *x,
               float *y, int32_t accumulate, sge_stream_t stream);

/* Image error of the unperturbed scene, f(theta) = sum over pixels of
 * || I_p(theta) - I_p ||^2 (Table 1), per view: loss_out[j] (device [n_views]
 * float32) ACCUMULATES view view_ids[j]'s error.  The forward value of the
 * autograd form whose backward is sge_estimate_grad + sge_gradient. */
int sge_loss(sge_scene *scene, const int32_t *view_ids, int32_t n_views, float *loss_out, sge_stream_t stream);

/* The gradient estimate of Eq. 9 from accumulated sums: out[i] = scale *
 * grad_sums[i] / (2 eps_i n_pairs_total) (device [d] float32; scale is a device
 * float32 scalar, NULL for 1).  Leaves grad_sums untouched. */
int sge_gradient(sge_scene *scene, const float *grad_sums, int64_t n_pairs_total, const float *scale, float *out,
                 sge_stream_t stream);

/* Descent step D (Section 5) on every parameter group, then zero grad_sums and
 * counts.  g_i = grad_sums[i] / (2 eps_i n_pairs_total) (Eq. 9; for
 * SGE_STEP_SGD_MEAN, / (2 eps_i max(counts[i], 1))).  SGD: theta -= lr g.  Adam:
 * m, v (device [d] float32, caller-zeroed before step 1) updated in place,
 * theta -= lr mhat / (sqrt(vhat) + adam_eps).  The paper uses Adam with
 * lr = eps (Section 5). */
int sge_step(sge_scene *scene, const sge_opt *opt, float *grad_sums, uint32_t *counts,
             int64_t n_pairs_total, float *adam_m, float *adam_v, sge_stream_t stream);

/* Optimizer loop captured once in a CUDA graph.  Section 5 draws fresh signs for every
 * estimate (Eq. 9 averages independent ones) and runs one Adam step per iteration, so a
 * replayed graph must not bake the iteration index or Adam's step number into its launch
 * arguments.  These forms read both from a small state object in device memory when their
 * kernels run, and sge_iter_advance moves it on: capture estimate -> step -> advance once,
 * then every replay is the next iteration.  The state is caller-owned device memory
 * (8 bytes, 4-byte aligned); initialise it (e.g. {iter0, 1}) before the first replay. */
typedef struct {
    uint32_t iter;   /* iteration index whose sign vectors the next estimate draws          */
    int32_t t;       /* Adam step number of the next step, >= 1                             */
} sge_iter_state;

/* sge_estimate_grad with the iteration index read from state->iter (device) by the kernels
 * at run time; every other argument, output and error is that of sge_estimate_grad, and the
 * result equals sge_estimate_grad(..., state->iter, ...) at that moment. */
int sge_estimate_grad_state(sge_scene *scene, uint64_t seed, const sge_iter_state *state, const int32_t *view_ids,
                            int32_t n_views, int32_t pairs_per_view, float *grad_sums, uint32_t *counts,
                            float *loss_out, float *delta_f_out, sge_stream_t stream);

/* sge_step with Adam's step number read from state->t (device) at run time (opt->t is
 * ignored); the bias corrections 1 - beta^t are formed on the device in float32.  SGD and
 * the per-pixel mean do not read the state. */
int sge_step_state(sge_scene *scene, const sge_opt *opt, const sge_iter_state *state, float *grad_sums,
                   uint32_t *counts, int64_t n_pairs_total, float *adam_m, float *adam_v, sge_stream_t stream);

/* One device thread adds d_iter to state->iter and d_t to state->t, stream-ordered after the
 * work enqueued before it (an iteration's last node in a captured loop). */
int sge_iter_advance(sge_iter_state *state, int32_t d_iter, int32_t d_t, sge_stream_t stream);

/* Host memory of one optimizer iteration run by sge_iterate_host; any member may be NULL
 * (that copy is skipped).  Pinned (page-locked) host memory lets the copies run
 * asynchronously; pageable memory works too, with the copies staged by the driver. */
typedef struct {
    const float *theta_in;   /* host [d]: theta in gradient order (positions vertex-major xyz,
                                then each texture [height][width][channels]), copied into the
                                scene's parameter arrays before the estimate                 */
    const float *targets_in; /* host [n_views of the scene][height][width][3]: copied into the
                                scene's target images before the estimate                   */
    float *theta_out;        /* host [d]: the updated theta, copied out after the step       */
    float *loss_out;         /* host [n_views of the call]: each listed view's image error
                                (as loss_out of sge_estimate_grad), copied out after the step */
} sge_host_io;

/* One iteration of Section 5's loop (N = n_views x pairs_per_view estimates, Eq. 9, then one
 * descent step) for a caller whose parameters and targets live in host memory: copies
 * io->theta_in and io->targets_in into the device arrays the scene borrows (its positions,
 * textures and targets: these are overwritten), zeroes loss_dev, then runs
 * sge_estimate_grad_state, sge_step_state (n_pairs_total = N) and sge_iter_advance(state, 1, 1),
 * and copies the updated theta to io->theta_out and loss_dev to io->loss_out.  Every copy and
 * kernel is enqueued on `stream` in that order (one cudaMemcpyAsync per array); nothing
 * synchronises, so the host buffers must stay valid until the stream has passed the call.
 * grad_sums, counts (zeroed by the step), adam_m, adam_v, state: device memory, as in those
 * calls; loss_dev: device [n_views] float32, required when io->loss_out is set (else may be
 * NULL).  Errors: SGE_ERR_INVALID_ARG for a NULL scene, io, opt, state, grad_sums or counts,
 * a bad view list, pairs_per_view < 1, loss_out without loss_dev, a bad step kind, Adam without
 * m and v, or an eps <= 0 (all checked before anything is enqueued); the errors of the calls it
 * runs; SGE_ERR_CUDA when a copy cannot be enqueued. */
int sge_iterate_host(sge_scene *scene, uint64_t seed, sge_iter_state *state, const int32_t *view_ids,
                     int32_t n_views, int32_t pairs_per_view, const sge_opt *opt, float *grad_sums,
                     uint32_t *counts, float *adam_m, float *adam_v, float *loss_dev, const sge_host_io *io,
                     sge_stream_t stream);

/* One asset of a batched call: a scene with its views and its own outputs. */
typedef struct {
    sge_scene *scene;          /* distinct within one call                                  */
    const int32_t *view_ids;   /* host, n_views distinct view indices of this scene         */
    int32_t n_views;           /* 1..SGE_MAX_BATCH_VIEWS and <= its max_views_per_call      */
    float *grad_sums;          /* device [d of this scene] float32, accumulates             */
    uint32_t *counts;          /* device [d] uint32, accumulates                            */
    float *loss_out;           /* device [n_views] float32 or NULL, accumulates             */
} sge_batch_entry;

/* Launch shape of a batched call; zero fields take the defaults.  sge_autotune_batch
 * measures the choices and returns the fastest. */
typedef struct {
    int32_t pairs_per_item;    /* antithetic pairs one CTA runs per (view, tile) item (default 8, <= 64) */
    int32_t blocks_per_sm;     /* persistent CTAs per SM of the fast kernel (default: as many as fit)    */
    int32_t light_bin;         /* tiles whose bin holds at most this many triangles take the fast
                                  kernel, the rest the general one (default and maximum 256)             */
} sge_batch_tuning;

/* sge_estimate_grad for several scenes (assets of different sizes, textures and
 * view counts) in one call: every estimate of every entry, pairs_per_view pairs per
 * view, from (seed, iter, view, pair) exactly as sge_estimate_grad would draw them
 * for that scene, each entry's sums, counts and losses into its own buffers.  The
 * estimates of all entries with the same shading model run in one persistent
 * launch of each estimator kernel (per block of max_pairs_per_call pairs, the
 * smallest of the entries'); binning and vertex passes are per entry.  Results
 * equal sge_estimate_grad's per entry up to the order of float additions.  The
 * paper runs one asset at a time; batching is this library's addition.  The first
 * batched call of a scene (and the first after sge_set_targets) also writes the
 * scene's launch descriptor into its workspace on `stream`. */
int sge_estimate_grad_batch(const sge_batch_entry *entries, int32_t n_entries, uint64_t seed, uint32_t iter,
                            int32_t pairs_per_view, const sge_batch_tuning *tuning, sge_stream_t stream);

/* sge_estimate_grad_batch with the iteration index read from state->iter (device) when the
 * kernels run (see sge_iter_state); results, outputs and errors as sge_estimate_grad_batch's. */
int sge_estimate_grad_batch_state(const sge_batch_entry *entries, int32_t n_entries, uint64_t seed,
                                  const sge_iter_state *state, int32_t pairs_per_view,
                                  const sge_batch_tuning *tuning, sge_stream_t stream);

/* Autotuner of sge_estimate_grad_batch's launch shape (no counterpart in the paper,
 * which runs one asset at a time) for these entries: times
 * candidate shapes (pairs per item 1..64, 1 or 2 CTAs per SM, light-bin limit
 * 64/128/256; a coordinate search from the defaults), each as one untimed call then
 * the mean of `repeats` calls (CUDA events on `stream`), and returns the fastest in
 * *out and its time in *best_ms (may be NULL).  Runs real estimates into the
 * entries' buffers and zeroes grad_sums, counts and loss_out before returning.
 * Synchronises `stream`; not for use under stream capture. */
int sge_autotune_batch(const sge_batch_entry *entries, int32_t n_entries, int32_t pairs_per_view, int32_t repeats,
                       sge_batch_tuning *out, float *best_ms, sge_stream_t stream);

/* Synchronise `stream`, return the device status word (SGE_OK or the first
 * device-side error) in *device_status and clear it. */
int sge_status(sge_scene *scene, sge_stream_t stream, int32_t *device_status);

/* Allocation-free render, for callers that cannot allocate device memory: code
 * embedded in a host application that owns the whole device-memory budget, or
 * that must not let cudaMalloc / cudaFree synchronise the device mid-frame, and so
 * cannot provide the workspace the other entry points need.  The paper has no
 * counterpart; the result equals sge_render_idb's for the same arguments.
 * Takes the scene description directly (no sge_scene, no workspace; targets may
 * be NULL).  Its scratch is a fixed array in the library's device memory,
 * SGE_STATIC_SCRATCH limits below, held on every GPU that loads the library until
 * the process exits; requests beyond the limits return SGE_ERR_INVALID_ARG and
 * launch nothing, and transparent scenes SGE_ERR_UNSUPPORTED; the descriptor is
 * checked exactly as sge_create_scene checks it.  The first call on a device (that
 * device current) looks up the array's address; make it before any stream capture.
 * The address is kept per device and CUDA context: the first call after a
 * cudaDeviceReset looks it up again, so it too should precede any capture.  All calls share the
 * array: calls that overlap on the GPU (other streams or threads) race; order
 * them on one stream.  device_status (device int32, or NULL) receives SGE_OK or
 * SGE_ERR_BIN_OVERFLOW (tiles whose lists did not fit render as background).
 * Allocates nothing and calls no allocating library routine.  Errors return their
 * code and leave a message for sge_last_error, as the other calls do. */
#define SGE_STATIC_MAX_TRIANGLES 131072
#define SGE_STATIC_MAX_PIXELS (2048 * 2048)
#define SGE_STATIC_BIN_ENTRIES (1 << 21)
int sge_render_idb_static(const sge_scene_desc *desc, int32_t view, uint64_t seed, uint32_t iter,
                          uint32_t pair, int32_t side, uint64_t *depth_id, float *uv, float *rgb,
                          int32_t *device_status, sge_stream_t stream);

/* Throughput probe of global float atomics, for benchmarks (the paper has no counterpart; it
 * measures the ceiling of Algorithm 2's per-contribution AtomicAdd).  Enqueues n_threads device
 * threads that each add 1.0f per_thread times to buf[i mod n_addr] (device float32 [n_addr],
 * caller-owned; its contents grow by the additions), as fire-and-forget reductions.  Time it with
 * CUDA events on `stream`: n_threads * per_thread reductions.  n_addr = n_threads gives one
 * address per thread; small n_addr gives 1-of-n_addr hot addresses. */
int sge_atomic_bench(float *buf, int64_t n_addr, int64_t n_threads, int32_t per_thread, sge_stream_t stream);

/* ---- checked build (the library compiled with SGE_CHECKED=1, libsge_checked.so) ----
 * Stand-in for a memory checker: every kernel range-checks the indices it takes from the
 * caller's data or computes into the workspace before it uses them: vertex and UV indices read
 * from pos_idx / uv_idx (against n_positions / n_uvs), bin entries (against bin_capacity),
 * texel sign-plane words (against one estimate's plane size), parameter indices of the gradient
 * sums and counts (against sge_num_params), and the direct slots of the fast estimator's
 * shared-memory texel table.  A failing check does not make the access (a read yields element
 * 0 or nothing, a write or credit is dropped) and records SGE_ERR_BOUNDS in the device status
 * word (sge_status); nothing traps.  Results of a call that recorded it are meaningless. */

/* 1 if this library is the checked build, else 0. */
int sge_checked_build(void);

/* Which range sge_check_limit lowers. */
enum {
    SGE_LIMIT_VERTICES = 0,     /* vertex indices read from pos_idx        */
    SGE_LIMIT_UVS = 1,          /* UV indices read from uv_idx             */
    SGE_LIMIT_BIN_ENTRIES = 2,  /* bin entries (bin_capacity)              */
    SGE_LIMIT_SIGN_WORDS = 3,   /* words of one estimate's sign planes     */
    SGE_LIMIT_PARAMS = 4        /* parameter indices of grad_sums / counts */
};

/* Checked build only (else SGE_ERR_UNSUPPORTED): set the bound that the checks of `which`
 * compare against to `limit` (0 <= limit <= the true size), or back to the true size
 * (limit < 0).  It changes no allocation and no logic of the library, only what the checks
 * treat as the end of the range, so that a test can make the range too small from the host and
 * see the checks fire without any access leaving its buffer.  SGE_ERR_INVALID_ARG for a bad
 * `which` or a limit above the true size. */
int sge_check_limit(sge_scene *scene, int32_t which, int64_t limit);

/* Checked build only (else SGE_ERR_UNSUPPORTED): synchronise `stream`, then give the site of the
 * first range check that failed since the last call (0: none; otherwise the source file's id
 * times 100000 plus the line: 1 k_bin.cu, 2 k_deep.cu, 3 k_estimate.cu, 4 k_fast.cu,
 * 5 k_staged.cu, 6 k_vertex.cu, 9 sge_device.cuh) and the low 32 bits of its index, and clear
 * both.  site, index: host. */
int sge_check_report(sge_scene *scene, sge_stream_t stream, int32_t *site, int64_t *index);

/* Timing of the estimator kernels, for benchmarks (the paper has no counterpart).
 * While enabled, each sge_estimate_grad call records CUDA events on its stream right
 * before and right after each launch of its fast estimator kernel (the one that runs
 * tiles with light bins) and after the following heavy-bin kernel, up to 256 launches
 * between reads.  sge_kernel_time synchronises on those events and returns the total
 * milliseconds of the fast launches, of the heavy ones (heavy_ms may be NULL) and the
 * number of launches timed, then starts a new count.  Enabling creates the events
 * (host objects, no device memory); disabling (and sge_destroy_scene) releases them.
 * Calls made under stream capture must not be timed. */
int sge_kernel_timing(sge_scene *scene, int32_t enable);
int sge_kernel_time(sge_scene *scene, float *total_ms, float *heavy_ms, int32_t *launches);

/* Work list of the scene's last estimate call (after its binning and pruning; a
 * diagnostic with no counterpart in the paper):
 * tiles x views taken by the fast kernel (light_items), by the heavy-bin kernel
 * (heavy_items) and the triangle-tile bin entries before pruning.  Synchronises
 * `stream`.  For tuning sge_batch_tuning.light_bin and for diagnostics. */
int sge_bin_stats(sge_scene *scene, sge_stream_t stream, int64_t *light_items, int64_t *heavy_items,
                  int64_t *bin_entries);

/* The views of one iteration (Section 5 picks the view of each estimate at random): the first
 * `count` entries of a Fisher-Yates shuffle of 0..n_views-1 whose i-th step swaps slot i with
 * slot i + (r_i mod (n_views - i)), r_i the (i+1)-th SplitMix64 output from the key
 * pair_key(seed, iter, 0xFFFFFFFF, 0xFFFFFFFF) (the same generator family as the signs; no
 * estimate uses that key).  Host-only, deterministic; out: host [count] distinct view indices.
 * Needs 1 <= count <= n_views and count <= SGE_MAX_VIEWS_PER_CALL. */
int sge_draw_views(uint64_t seed, uint32_t iter, int32_t n_views, int32_t count, int32_t *out);

/* Release the host object (never the borrowed device memory). */
void sge_destroy_scene(sge_scene *scene);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *sge_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGE_H */
