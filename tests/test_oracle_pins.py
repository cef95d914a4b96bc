"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle to something the paper or the
mathematics determines: published hash outputs, exact pixel counts of the
top-left fill rule, a library bilinear interpolator, a ray-plane intersection,
finite differences (Eq. 3) that equal the per-pixel estimator (Eq. 8) in the
one-parameter case, the exact expectation over all sign vectors, and a
statistical test of unbiasedness (Eq. 9).
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests.tiny import flat_scene, square_quad, to_world

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BG = np.uint64(0xFFFFFFFFFFFFFFFF)
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def covered(scene, view=0):
    keys, _, _ = oracle.render(oracle.OracleScene(scene), view)
    return keys != BG, keys


def coverage_count(scene_tris, W, H, **kw):
    """How many triangles cover each pixel, rendering each triangle alone."""
    cnt = np.zeros((H, W), np.int64)
    for t in scene_tris:
        m, _ = covered(flat_scene([t], W, H, **kw))
        cnt += m
    return cnt


# ------------------------------------------------------------------ sign hash (Alg. 1)
def test_splitmix64_known_answers():
    """The generator under the sign hash reproduces SplitMix64's published outputs."""
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not l.startswith("#")]
    want = [int(l, 16) for l in lines if l.strip()]
    got = [oracle.mix64((k * GAMMA) & M64) for k in range(1, len(want) + 1)]
    assert got == want


def test_sign_is_a_bit_of_the_splitmix_stream():
    """s_i is bit (i mod 64) of the (floor(i / 64) + 1)-th generator output."""
    key = oracle.pair_key(7, 3, 2, 5)
    for i in (0, 1, 2, 63, 64, 65, 1000, 2**26 + 3):
        out = oracle.mix64((key + (i // 64 + 1) * GAMMA) & M64)
        assert oracle.sign(key, i) == (-1 if (out >> (i % 64)) & 1 else 1)


def test_signs_within_one_output_are_uncorrelated():
    """Neighbouring parameters take neighbouring bits of one output: their signs (and those one
    output apart) must be uncorrelated over 10^6 draws (within 5 sigma)."""
    L = oracle.lib()
    key = oracle.pair_key(3, 1, 4, 1)
    n = 1_000_000
    s = np.fromiter((L.or_sign(key, i) for i in range(n + 64)), np.int64, n + 64)
    for lag in (1, 2, 31, 32, 63, 64):
        assert abs((s[:n] * s[lag:lag + n]).sum()) < 5 * math.sqrt(n), lag


def test_sign_balance_and_independence():
    """Rademacher signs (Eq. 4): balanced within 5 sigma over 10^6 draws; two pairs uncorrelated."""
    k1, k2 = oracle.pair_key(0, 0, 0, 0), oracle.pair_key(0, 0, 0, 1)
    n = 1_000_000
    L = oracle.lib()
    s1 = np.fromiter((L.or_sign(k1, i) for i in range(n)), np.int64, n)
    s2 = np.fromiter((L.or_sign(k2, i) for i in range(0, n, 10)), np.int64, n // 10)
    assert abs(s1.sum()) < 5 * math.sqrt(n)
    assert abs((s1[::10] * s2).sum()) < 5 * math.sqrt(n // 10)
    keys = {oracle.pair_key(s, it, v, p) for s in range(3) for it in range(3) for v in range(3)
            for p in range(3)}
    assert len(keys) == 81


# ------------------------------------------------------------------ coverage (Section 4.4, R)
def test_square_through_pixel_centres_counts_each_pixel_once():
    """Edges through pixel centres: left/top included, right/bottom excluded -> L^2 pixels."""
    W = H = 64
    for L in (1, 5, 32):
        a = 8.5
        cnt = coverage_count(square_quad(a, a, a + L, a + L), W, H)
        assert cnt.max() == 1
        assert cnt.sum() == L * L
        assert cnt[8:8 + L, 8:8 + L].all()


def test_right_triangles_top_left_counts():
    """Legs L through pixel centres: upper-left half L(L+1)/2 pixels, lower-right L(L-1)/2."""
    W = H = 64
    for L in (1, 2, 7, 20):
        a = 10.5
        ul = [[(a, a), (a + L, a), (a, a + L)]]
        lr = [[(a + L, a + L), (a, a + L), (a + L, a)]]
        assert coverage_count(ul, W, H).sum() == L * (L + 1) // 2
        assert coverage_count(lr, W, H).sum() == L * (L - 1) // 2
        # reversing the winding changes nothing (no back-face culling)
        assert coverage_count([ul[0][::-1]], W, H).sum() == L * (L + 1) // 2


def test_fan_covers_every_pixel_exactly_once():
    """A closed fan around a pixel centre, edges through lattice points, tiles the screen."""
    W = H = 32
    c = (15.5, 16.5)
    dirs = [(1, 0), (2, 1), (1, 1), (1, 2), (0, 1), (-1, 3), (-1, 1), (-3, 1), (-1, 0),
            (-2, -1), (-1, -1), (0, -1), (1, -3), (3, -2)]
    R = 40  # lattice multiples keep the rim vertices on pixel centres' grid
    rim = [(c[0] + R * dx, c[1] + R * dy) for dx, dy in dirs]
    tris = [[c, rim[k], rim[(k + 1) % len(rim)]] for k in range(len(rim))]
    cnt = coverage_count(tris, W, H)
    assert (cnt == 1).all()


def test_degenerate_and_behind_triangles_are_dropped():
    W = H = 16
    line = [[(2.5, 2.5), (8.5, 8.5), (12.5, 12.5)]]
    assert coverage_count(line, W, H).sum() == 0
    behind = flat_scene([[(2, 2, 0.5), (12, 2, 0.5), (2, 12, 0.5)]], W, H)
    behind.mvp[0, 3, 3] = 0.05  # clip w below the near limit 0.1
    assert covered(behind)[0].sum() == 0


# ------------------------------------------------------------------ visibility (ID buffer)
def test_nearest_wins_and_equal_depth_keeps_lower_id():
    W = H = 16
    big = [(0, 0), (16, 0), (0, 16)]
    tris = [[(x, y, 0.6) for x, y in big], [(x, y, 0.3) for x, y in big], [(x, y, 0.3) for x, y in big]]
    m, keys = covered(flat_scene(tris, W, H))
    ids = (keys[m] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert m.sum() > 0 and (ids == 1).all()
    # the winner's depth is the interpolated 0.3 (a few ulps of rounding in the weights)
    depth = ((keys[m] >> np.uint64(32)) & np.uint64(0x7FFFFFFF)).astype(np.uint32).view(np.float32)
    assert np.abs(depth - np.float32(0.3)).max() <= 4 * np.spacing(np.float32(0.3))
    # swap the order: the nearer triangle still wins, whatever its id
    m2, keys2 = covered(flat_scene(tris[::-1], W, H))
    assert ((keys2[m2] & np.uint64(0xFFFFFFFF)) == 0).all()


def test_sphere_silhouette_matches_projected_disk():
    """Unit sphere at distance 3, fov 45: silhouette radius tan(asin(1/3))/tan(22.5 deg) * W/2."""
    W = 256
    mesh = synth.uv_sphere(256, 128)
    sc = synth.Scene("s", mesh.positions, mesh.pos_idx, mesh.uvs, mesh.uv_idx,
                     [synth.Texture(synth.constant_texture(2, 2, 3, 1.0), 0.0, 0)], 0.0,
                     synth.mvp_matrix((0, 0, 3), W, W)[None], np.zeros((1, 3), np.float32), W, W)
    m, _ = covered(sc)
    r = math.tan(math.asin(1 / 3)) / math.tan(math.radians(22.5)) * W / 2
    assert abs(m.sum() / (math.pi * r * r) - 1) < 0.005
    ys, xs = np.nonzero(m)
    assert abs(xs.mean() + 0.5 - W / 2) < 0.5 and abs(ys.mean() + 0.5 - W / 2) < 0.5


# ------------------------------------------------------------------ UV buffer and texture sampling
def test_bilinear_sampling_matches_scipy():
    """Affine screen-filling quad with uv = screen/size: colour = bilinear sample (scipy, order 1)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    W = H = 32
    tex = synth.sinusoid_texture(8, 8, 3, seed=5)
    sc = flat_scene(square_quad(0, 0, W, H), W, H,
                    textures=[synth.Texture(tex, 0.0, synth.ROLE_ALBEDO)])
    _, uv, rgb = oracle.render(oracle.OracleScene(sc), 0)
    px = (np.arange(W) + 0.5) / W
    assert np.array_equal(uv[..., 0], np.broadcast_to(px.astype(np.float32), (H, W)))
    x = uv[..., 0].astype(np.float64) * 8 - 0.5
    y = uv[..., 1].astype(np.float64) * 8 - 0.5
    inner = (y >= 0) & (y <= 7)  # away from the clamped v edges
    for c in range(3):
        ref = ndimage.map_coordinates(tex[..., c].astype(np.float64), [y, x], order=1, mode="grid-wrap")
        assert np.abs(rgb[..., c] - ref)[inner].max() < 1e-6


def test_perspective_correct_uv_matches_ray_plane_intersection():
    """UV of a tilted textured quad equals the UV of the 3D point hit by the pixel's ray."""
    W = H = 64
    eye = np.array([0.4, 0.3, 3.0])
    mvp = synth.mvp_matrix(eye, W, H).astype(np.float64)
    P0, Pu, Pv = np.array([-1.0, -1.0, -0.8]), np.array([2.0, 0.0, 1.2]), np.array([0.0, 2.0, 0.3])
    corners = [P0, P0 + Pu, P0 + Pu + Pv, P0 + Pv]
    uvc = [(0, 0), (1, 0), (1, 1), (0, 1)]
    pos = np.array(corners, np.float32)
    sc = synth.Scene("q", pos, np.array([[0, 1, 2], [0, 2, 3]], np.int32),
                     np.array(uvc, np.float32), np.array([[0, 1, 2], [0, 2, 3]], np.int32),
                     [synth.Texture(synth.constant_texture(2, 2, 3, 1.0), 0.0, 0)], 0.0,
                     mvp.astype(np.float32)[None], eye[None].astype(np.float32), W, H)
    keys, uv, _ = oracle.render(oracle.OracleScene(sc), 0)
    inv = np.linalg.inv(mvp)
    n = np.cross(Pu, Pv)
    errs = []
    for py in range(0, H, 3):
        for px in range(0, W, 3):
            if keys[py, px] == BG:
                continue
            xn, yn = 2 * (px + 0.5) / W - 1, 1 - 2 * (py + 0.5) / H
            a = inv @ np.array([xn, yn, 0.0, 1.0])
            b = inv @ np.array([xn, yn, 1.0, 1.0])
            a, b = a[:3] / a[3], b[:3] / b[3]
            t = n @ (P0 - a) / (n @ (b - a))
            X = a + t * (b - a) - P0
            u, v = np.linalg.lstsq(np.stack([Pu, Pv], 1), X, rcond=None)[0]
            errs.append(max(abs(u - uv[py, px, 0]), abs(v - uv[py, px, 1])))
    assert len(errs) > 50
    # vertices snap to 1/256 pixel: the UV moves by at most ~(1/256) px / (quad size in px)
    assert max(errs) < 2e-4


# ------------------------------------------------------------------ shading special cases
def test_lambert_flat_normal_map_is_cosine_law():
    W = H = 16
    alb = synth.constant_texture(4, 4, 3, 0.6)
    for ld in ((0.0, 0.0, 1.0), (0.6, 0.0, 0.8), (0.0, -0.8, 0.6)):
        sc = flat_scene(square_quad(0, 0, W, H, True), W, H, shading=synth.SHADE_LAMBERT, light_dir=ld,
                        ambient=0.1, textures=[synth.Texture(alb, 0.0, synth.ROLE_ALBEDO),
                                               synth.Texture(synth.flat_normal_texture(4, 4), 0.0,
                                                             synth.ROLE_NORMAL)])
        _, _, rgb = oracle.render(oracle.OracleScene(sc), 0)
        assert np.allclose(rgb, 0.6 * (0.1 + max(0.0, ld[2])), atol=1e-7)


def test_normal_map_tangent_frame_orientation():
    """Tangent-space (1,0,0) maps to +u's direction, (0,1,0) to N x T."""
    W = H = 16
    alb = synth.constant_texture(4, 4, 3, 1.0)
    for nt, ld, want in (((1, 0, 0), (1, 0, 0), 1.0), ((1, 0, 0), (-1, 0, 0), 0.0),
                         ((0, 1, 0), (0, 1, 0), 1.0), ((0, 0, 1), (0, 0, 1), 1.0)):
        nm = np.empty((4, 4, 3), np.float32)
        nm[...] = 0.5 + 0.5 * np.array(nt, np.float32)
        sc = flat_scene(square_quad(0, 0, W, H, True), W, H, shading=synth.SHADE_LAMBERT, light_dir=ld,
                        textures=[synth.Texture(alb, 0.0, synth.ROLE_ALBEDO),
                                  synth.Texture(nm, 0.0, synth.ROLE_NORMAL)])
        _, _, rgb = oracle.render(oracle.OracleScene(sc), 0)
        # u grows with screen x = world +x; v grows down the screen = world -y, so N x T = +y
        assert np.allclose(rgb, want, atol=1e-7), (nt, ld)


def test_ggx_normal_incidence_closed_form():
    """L = V = N, roughness 1 (D = 1/pi), metallic 0: c = light (0.96 a + 0.01)/pi + ambient a."""
    W = H = 16
    a = 0.7
    texs = [synth.Texture(synth.constant_texture(2, 2, 3, a), 0.0, synth.ROLE_ALBEDO),
            synth.Texture(synth.constant_texture(2, 2, 3, 1.0), 0.0, synth.ROLE_ROUGHNESS),
            synth.Texture(synth.constant_texture(2, 2, 3, 0.0), 0.0, synth.ROLE_METALLIC),
            synth.Texture(synth.flat_normal_texture(2, 2), 0.0, synth.ROLE_NORMAL)]
    sc = flat_scene(square_quad(0, 0, W, H, True), W, H, shading=synth.SHADE_GGX, textures=texs,
                    light_dir=(0.0, 0.0, 1.0), ambient=0.05, cam_pos=(0.0, 0.0, 1e6))
    sc.light_rgb = (2.0, 2.0, 2.0)
    _, _, rgb = oracle.render(oracle.OracleScene(sc), 0)
    want = 2.0 * (0.96 * a + 0.04 * 1.0 * 1.0 / 4.0) / math.pi + 0.05 * a
    assert np.allclose(rgb, want, rtol=1e-6, atol=0)


# ------------------------------------------------------------------ estimator (Eq. 3, 8, 9)
def _plain_small(render=64):
    sc = synth.config_plain(render=render)
    tgt = oracle.render_targets(sc, synth.target_scene(sc))
    return sc, tgt


def test_zero_perturbation_gives_zero_sums_but_counts():
    sc, tgt = _plain_small()
    sc.eps_pos = 0.0
    sc.textures[0].eps = 0.0
    osc = oracle.OracleScene(sc, tgt)
    S, Cn, _ = oracle.estimate(osc, 3, 0, [0], 2)
    assert np.all(S == 0.0)
    keys, _, _ = oracle.render(osc, 0)
    assert Cn[:osc.n_params].sum() > 0
    # every covered pixel credits at least 9 vertex coordinates and 3 texel channels per pair
    assert Cn.sum() >= 2 * 12 * (keys != BG).sum()


@pytest.mark.parametrize("which", ["vertex", "texel"])
def test_one_parameter_estimate_equals_central_difference(which):
    """Only theta_i perturbed: sum over impacted pixels of Eq. 8 equals Eq. 3 (same two renders)."""
    sc, tgt = _plain_small(96)
    # textured initial state, so moving a vertex moves texture across pixels
    sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(256, 256, 3, seed=4)])
    osc0 = oracle.OracleScene(sc, tgt)
    keys, uv, _ = oracle.render(osc0, 0)
    tri = int(keys[48, 50] & np.uint64(0xFFFFFFFF))
    if which == "vertex":
        i = 3 * int(sc.pos_idx[tri, 0]) + 0
        eps = 1e-2
    else:
        u, v = uv[48, 50]
        x, y = int(math.floor(u * 256 - 0.5)), int(math.floor(v * 256 - 0.5))
        i = sc.n_pos_params + (y * 256 + x) * 3 + 1
        eps = 1.0 / 64.0
    eps_vec = np.zeros(sc.n_params, np.float32)
    eps_vec[i] = eps
    for pair in range(3):
        S, Cn, _ = oracle.estimate(oracle.OracleScene(sc, tgt, eps_vec=eps_vec), 11, 0, [0], 1)
        assert Cn[i] > 0
        est = S[i] / (2 * eps)

        def f_at(delta):
            pos = sc.positions.copy().ravel()
            tex = sc.textures[0].data.copy().ravel()
            if i < sc.n_pos_params:
                pos[i] = np.float32(pos[i] + np.float32(delta))
            else:
                tex[i - sc.n_pos_params] = np.float32(tex[i - sc.n_pos_params] + np.float32(delta))
            s2 = synth.with_params(sc, pos.reshape(-1, 3), [tex.reshape(256, 256, 3)])
            return oracle.loss(oracle.OracleScene(s2, tgt), 0)

        fd = (f_at(eps) - f_at(-eps)) / (2 * eps)
        assert fd != 0.0
        assert abs(est - fd) <= 1e-9 * max(1.0, abs(fd)), (pair, est, fd)


def _quad_texture_scene(footprint_nearest=False, n=4, W=16):
    rng = np.random.default_rng(9)
    # multiples of 1/256, so theta +- eps and the finite-difference steps are exact in float32
    tex = (np.round(rng.uniform(0.2, 0.8, size=(n, n, 3)) * 256) / 256).astype(np.float32)
    sc = flat_scene(square_quad(0, 0, W, W), W, W,
                    textures=[synth.Texture(tex, 1.0 / 64.0, synth.ROLE_ALBEDO)])
    tgt = rng.uniform(0.0, 1.0, size=(1, W, W, 3)).astype(np.float32)
    return sc, tgt


def _exact_texel_gradient(sc, tgt):
    """f is quadratic in the texels of an unlit scene, so a central difference is exact."""
    tex = sc.textures[0].data
    g = np.zeros(tex.size)
    h = 0.25
    for j in range(tex.size):
        vals = []
        for d in (h, -h):
            t2 = tex.copy().ravel()
            t2[j] += d
            s2 = synth.with_params(sc, sc.positions, [t2.reshape(tex.shape)])
            vals.append(oracle.loss(oracle.OracleScene(s2, tgt), 0))
        g[j] = (vals[0] - vals[1]) / (2 * h)
    return g


def test_expectation_over_all_sign_vectors_is_the_gradient():
    """Averaging Eq. 8 over all 2^d sign vectors of a 2x2 RGB texture gives the exact gradient."""
    sc, tgt = _quad_texture_scene(n=2, W=8)
    d_pos = sc.n_pos_params
    d = sc.n_params
    eps = sc.textures[0].eps
    key = oracle.pair_key(5, 0, 0, 0)
    s_hash = np.array([oracle.sign(key, i) for i in range(d)], np.float32)
    total = np.zeros(d - d_pos)
    n_tex = d - d_pos
    for mask in range(1 << n_tex):
        sigma = np.array([1.0 if (mask >> j) & 1 else -1.0 for j in range(n_tex)], np.float32)
        eps_vec = np.zeros(d, np.float32)
        # perturbation s_i * eps_vec_i = sigma_i * eps, so the hash's signs cancel out
        eps_vec[d_pos:] = sigma * s_hash[d_pos:] * eps
        S, _, _ = oracle.estimate(oracle.OracleScene(sc, tgt, eps_vec=eps_vec), 5, 0, [0], 1)
        total += S[d_pos:] / (2.0 * eps_vec[d_pos:])
    mean = total / (1 << n_tex)
    g = _exact_texel_gradient(sc, tgt)
    assert np.allclose(mean, g, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("nearest", [False, True])
def test_statistical_unbiasedness_bilinear_not_nearest(nearest):
    """Eq. 9 over 10^5 pairs on a bilinearly textured quad: the bilinear footprint is unbiased
    (every texel's z-score small, chi^2 consistent); the paper's nearest-texel footprint is not."""
    sc, tgt = _quad_texture_scene()
    osc = oracle.OracleScene(sc, tgt, footprint=oracle.FOOT_NEAREST if nearest else 0)
    d_pos = sc.n_pos_params
    eps = sc.textures[0].eps
    n_pairs = 100_000
    L = oracle.lib()
    s1 = np.zeros(osc.n_params)
    s2 = np.zeros(osc.n_params)
    S = np.zeros(osc.n_params)
    Cn = np.zeros(osc.n_params, np.uint64)
    views = np.zeros(1, np.int32)
    chunk = 1000
    for it in range(n_pairs // chunk):
        # one pair per call, so every estimate's variance is visible
        for p in range(chunk):
            S[:] = 0.0
            L.oracle_estimate(osc.ref, 77, it * chunk + p, views.ctypes.data, 1, 1, S.ctypes.data,
                              Cn.ctypes.data, None, None, None, None)
            est = S / (2 * eps)
            s1 += est
            s2 += est * est
    mean = s1[d_pos:] / n_pairs
    var = s2[d_pos:] / n_pairs - mean * mean
    se = np.sqrt(var / n_pairs)
    g = _exact_texel_gradient(sc, tgt)
    z = (mean - g) / se
    if nearest:
        assert np.abs(z).max() > 10
    else:
        assert np.abs(z).max() < 4.5, z
        assert abs(np.mean(z * z) - 1.0) < 0.5


# ------------------------------------------------------------------ descent step (Section 5)
def test_sgd_step_is_scaled_estimate():
    rng = np.random.default_rng(0)
    th = rng.normal(size=50).astype(np.float32)
    S = rng.normal(size=50)
    Cn = rng.integers(0, 9, size=50).astype(np.uint64)
    e = float(np.float32(0.01))  # magnitudes are float32 parameters
    out, _, _ = oracle.step(0, th, S, Cn, 0.01, 0.5, 8)
    assert np.allclose(out, th.astype(np.float64) - 0.5 * S / (2 * e * 8), rtol=0, atol=1e-12)
    out2, _, _ = oracle.step(2, th, S, Cn, 0.01, 0.5, 8)
    want = th.astype(np.float64) - 0.5 * S / (2 * e * np.maximum(Cn, 1).astype(np.float64))
    assert np.allclose(out2, want, rtol=0, atol=1e-12)


def test_sgd_step_normalisation_gives_the_exact_gradient_step():
    """Eq. 9's normalisation inside the SGD step, pinned by mathematics: feeding the step the
    sums of Eq. 8 over all 2^d sign vectors of a 2x2 RGB texture (N = 2^d estimates) must move
    theta by exactly lr times the true gradient (f is quadratic in the texels).  A wrong 2,
    eps or N in the step's scale fails this; Adam's scale invariance would hide it."""
    sc, tgt = _quad_texture_scene(n=2, W=8)
    d_pos, d = sc.n_pos_params, sc.n_params
    eps = sc.textures[0].eps
    key = oracle.pair_key(5, 0, 0, 0)
    s_hash = np.array([oracle.sign(key, i) for i in range(d)], np.float64)
    n_tex = d - d_pos
    S_all = np.zeros(d)
    C_all = np.zeros(d, np.uint64)
    for mask in range(1 << n_tex):
        sigma = np.array([1.0 if (mask >> j) & 1 else -1.0 for j in range(n_tex)])
        eps_vec = np.zeros(d, np.float32)
        eps_vec[d_pos:] = (sigma * s_hash[d_pos:] * eps).astype(np.float32)
        S, Cn, _ = oracle.estimate(oracle.OracleScene(sc, tgt, eps_vec=eps_vec), 5, 0, [0], 1)
        # the sums a step sees when the perturbation of parameter i is sigma_i eps (not s_i eps)
        S_all[d_pos:] += S[d_pos:] * sigma * s_hash[d_pos:]
        C_all += Cn
    theta = sc.textures[0].data.ravel().astype(np.float32)
    lr = 0.125
    out, _, _ = oracle.step(0, theta, S_all[d_pos:], C_all[d_pos:], eps, lr, 1 << n_tex)
    g = _exact_texel_gradient(sc, tgt)
    assert np.allclose(out, theta.astype(np.float64) - lr * g, rtol=0, atol=1e-9)
    # the same sums counted as twice as many estimates halve the step
    out2, _, _ = oracle.step(0, theta, S_all[d_pos:], C_all[d_pos:], eps, lr, 2 << n_tex)
    assert np.allclose(theta - out2, 0.5 * lr * g, rtol=0, atol=1e-9)


@pytest.mark.parametrize("kind", [0, 2])
def test_sgd_steps_match_torch_sgd(kind):
    """The SGD step (kind 0, Eq. 9's 1 / (2 eps N)) and the per-pixel-mean step (kind 2,
    1 / (2 eps max(C, 1)), zero counts included) against torch.optim.SGD fed those gradients."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    d, N = 64, 12
    th = rng.normal(size=d).astype(np.float32)
    eps = rng.choice([1e-3, 1.0 / 255.0], size=d).astype(np.float32)
    lr = rng.uniform(0.05, 0.5, size=d).astype(np.float32)
    S = rng.normal(size=d) * 0.01
    Cn = rng.integers(0, 20, size=d).astype(np.uint64)
    Cn[:5] = 0
    out, _, _ = oracle.step(kind, th, S, Cn, eps, lr, N)
    scale = N if kind == 0 else np.maximum(Cn, 1).astype(np.float64)
    grad = S / (2.0 * eps.astype(np.float64) * scale)
    for i in range(d):
        p = torch.tensor([float(th[i])], dtype=torch.float64, requires_grad=True)
        opt = torch.optim.SGD([p], lr=float(lr[i]))
        p.grad = torch.tensor([grad[i]], dtype=torch.float64)
        opt.step()
        assert abs(out[i] - float(p.detach()[0])) <= 1e-12 * max(1.0, abs(out[i])), (kind, i)


def test_adam_step_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    d = 64
    th = rng.normal(size=d).astype(np.float32)
    eps = np.full(d, 1e-3, np.float32)
    lr = eps.copy()
    p = torch.tensor(th.astype(np.float64), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(d, np.float32)
    v = np.zeros(d, np.float32)
    cur = th
    for t in range(1, 6):
        S = rng.normal(size=d)
        out, m64, v64 = oracle.step(1, cur, S, np.ones(d, np.uint64), eps, lr, 4, t=t, m=m, v=v)
        p.grad = torch.tensor(S / (2 * 1e-3 * 4))
        opt.step()
        assert np.allclose(out, p.detach().numpy(), rtol=0, atol=5e-6 * 1e-3 + 1e-7)
        # carry the state in float32 as the device does; torch keeps float64, so re-sync
        cur = p.detach().numpy().astype(np.float32)
        p.data = torch.tensor(cur.astype(np.float64))
        st = opt.state[p]
        m = st["exp_avg"].numpy().astype(np.float32)
        v = st["exp_avg_sq"].numpy().astype(np.float32)
        st["exp_avg"].copy_(torch.tensor(m.astype(np.float64)))
        st["exp_avg_sq"].copy_(torch.tensor(v.astype(np.float64)))


def test_view_draw_is_a_uniform_choice_of_distinct_views():
    """Section 5's random view per estimate: distinct views, each view equally likely (5 sigma
    over 16,000 draws), a full draw is a permutation, and the draw is a function of (seed, iter)."""
    import collections
    for n, k in ((8, 8), (8, 3), (1, 1), (20, 5)):
        v = oracle.draw_views(3, 7, n, k)
        assert len(v) == k and len(set(v)) == k and all(0 <= x < n for x in v)
    assert sorted(oracle.draw_views(11, 2, 8, 8)) == list(range(8))
    assert oracle.draw_views(5, 9, 8, 4) == oracle.draw_views(5, 9, 8, 4)
    assert oracle.draw_views(5, 9, 8, 4) != oracle.draw_views(5, 10, 8, 4)
    n, draws = 8, 16000
    c = collections.Counter(oracle.draw_views(1, it, n, 1)[0] for it in range(draws))
    sd = (draws * (1 / n) * (1 - 1 / n)) ** 0.5
    assert all(abs(c[v] - draws / n) < 5 * sd for v in range(n)), c
    # second position: uniform over the views other than the first
    c2 = collections.Counter(tuple(oracle.draw_views(2, it, 4, 2)) for it in range(12000))
    assert len(c2) == 12 and all(abs(x - 1000) < 5 * (12000 * (1 / 12) * (11 / 12)) ** 0.5 for x in c2.values())


# ------------------------------------------------------------- full-image estimator (Eq. 4)

def test_full_image_difference_is_the_loss_of_two_explicit_scenes():
    """dF of Eq. 4 is f(theta + s eps) - f(theta - s eps): rebuild both scenes explicitly from
    the published signs and take the difference of their whole-image errors."""
    sc, tgt = _quad_texture_scene(n=4, W=16)
    sc = synth.with_params(sc, sc.positions + np.float32(0.0), [sc.textures[0].data])
    osc = oracle.OracleScene(sc, tgt)
    seed, it = 8, 3
    S, Cn, dF, A, M, K = oracle.estimate_full_image(osc, seed, it, [0], 1)
    key = oracle.pair_key(seed, it, 0, 0)
    d = sc.n_params
    s = np.array([oracle.sign(key, i) for i in range(d)], np.float64)
    eps = np.concatenate([np.full(sc.n_pos_params, sc.eps_pos), np.full(d - sc.n_pos_params, sc.textures[0].eps)])
    theta = np.concatenate([sc.positions.ravel(), sc.textures[0].data.ravel()]).astype(np.float32)

    def f_of(sign):
        th = (theta + (sign * s * eps).astype(np.float32)).astype(np.float32)
        s2 = synth.with_params(sc, th[:sc.n_pos_params].reshape(-1, 3),
                               [th[sc.n_pos_params:].reshape(sc.textures[0].data.shape)])
        return oracle.loss(oracle.OracleScene(s2, tgt), 0)

    want = f_of(+1) - f_of(-1)
    assert want != 0.0 and abs(dF[0] - want) <= 1e-9 * max(1.0, abs(want))
    # every parameter is credited: S = dF * s, one count each
    assert np.allclose(S, dF[0] * s, rtol=0, atol=1e-12 * max(1.0, abs(dF[0])))
    assert (Cn == 1).all()
    assert A[0] >= abs(dF[0]) and M[0] > 0 and K[0] > 0


def test_full_image_expectation_over_all_sign_vectors_is_the_gradient():
    """Eq. 4 averaged over all 2^d sign vectors of a 2x2 RGB texture gives the exact gradient
    (f is quadratic in the texels), like the per-pixel form."""
    sc, tgt = _quad_texture_scene(n=2, W=8)
    d_pos, d = sc.n_pos_params, sc.n_params
    eps = sc.textures[0].eps
    key = oracle.pair_key(5, 0, 0, 0)
    s_hash = np.array([oracle.sign(key, i) for i in range(d)], np.float32)
    n_tex = d - d_pos
    total = np.zeros(n_tex)
    for mask in range(1 << n_tex):
        sigma = np.array([1.0 if (mask >> j) & 1 else -1.0 for j in range(n_tex)], np.float32)
        eps_vec = np.zeros(d, np.float32)
        eps_vec[d_pos:] = sigma * s_hash[d_pos:] * eps
        S = oracle.estimate_full_image(oracle.OracleScene(sc, tgt, eps_vec=eps_vec), 5, 0, [0], 1)[0]
        total += S[d_pos:] / (2.0 * eps_vec[d_pos:])
    g = _exact_texel_gradient(sc, tgt)
    assert np.allclose(total / (1 << n_tex), g, rtol=1e-9, atol=1e-9)


def test_per_pixel_estimate_has_less_variance_than_full_image():
    """Section 4.2's motivation, measured: on a textured quad the per-pixel estimator (Eq. 8) of a
    texel's gradient varies far less than the full-image one (Eq. 4), whose every texel carries
    the whole image's difference; both are unbiased here, so their means agree."""
    sc, tgt = _quad_texture_scene(n=4, W=16)
    osc = oracle.OracleScene(sc, tgt)
    d_pos, eps = sc.n_pos_params, sc.textures[0].eps
    n = 1500
    pp = np.zeros((n, sc.n_params - d_pos))
    fi = np.zeros_like(pp)
    for it in range(n):
        pp[it] = oracle.estimate(osc, 13, it, [0], 1)[0][d_pos:] / (2 * eps)
        fi[it] = oracle.estimate_full_image(osc, 13, it, [0], 1)[0][d_pos:] / (2 * eps)
    var_pp, var_fi = pp.var(0), fi.var(0)
    assert np.median(var_fi / var_pp) > 3.0, np.median(var_fi / var_pp)
    se = np.sqrt((var_pp + var_fi) / n)
    assert np.median(np.abs(pp.mean(0) - fi.mean(0)) / se) < 1.0


def test_linear_refine_matrix_reproduces_the_subdivision():
    """The refine matrix of midpoint subdivision maps control positions to the subdivided mesh's
    positions (every row sums to 1: a subdivided vertex is an affine combination)."""
    c = synth.uv_sphere(12, 8)
    for levels in (1, 2):
        f = synth.subdivide_linear(c, levels)
        R = synth.linear_refine_matrix(c, levels)
        assert R.shape == (len(f.positions), len(c.positions))
        assert np.allclose(np.asarray(R.sum(1)).ravel(), 1.0)
        got = (R @ c.positions.astype(np.float64)).astype(np.float32)
        assert np.abs(got - f.positions).max() <= 2 * np.finfo(np.float32).eps
