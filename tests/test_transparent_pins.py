"""Pins of the oracle's transparent-geometry mode (Section 4.4: a deep ID buffer, front-to-back
rendering, G walking each pixel's list), each against a fact that does not come from the mode
itself.

- Two overlapping constant RGBA quads at different depths: every pixel is the closed form of
  front-to-back "over" compositing, whatever order the triangles are listed in.
- Opaque texels (alpha = 1): the composite is the opaque unlit render, and the front entry of the
  deep list is the opaque ID buffer.
- The deep list of a stack of six triangles is, pixel by pixel, the four smallest of the keys
  each triangle gets when it is rasterized alone.
- One perturbed parameter (a vertex coordinate, a colour channel, an opacity): the sum of Eq. 8
  over the pixels that credit it equals the central difference of the whole-image error (Eq. 3)
  exactly, as in the opaque case: every pixel whose colour changes lists the parameter.
- Hidden layers are credited: a parameter of a back face no opaque render shows gets counts.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.tiny import flat_scene, square_quad

BG = np.uint64(0xFFFFFFFFFFFFFFFF)
LAYERS = 4


def _two_quads(front_first=True, a_front=0.25, a_back=0.5):
    W = H = 16
    # texel (0,0) and (1,0) of a 2x2 RGBA texture, sampled at their centres (u = 1/4, 3/4; v = 1/4)
    tex = np.zeros((2, 2, 4), np.float32)
    tex[0, 0] = (0.875, 0.25, 0.125, a_front)
    tex[0, 1] = (0.125, 0.5, 0.75, a_back)
    A = [[(x, y, 0.25) for x, y in t] for t in square_quad(2, 2, 10, 10)]
    B = [[(x, y, 0.625) for x, y in t] for t in square_quad(6, 6, 14, 14)]
    uvA = [[(0.25, 0.25)] * 3] * 2
    uvB = [[(0.75, 0.25)] * 3] * 2
    tris, uvs = (A + B, uvA + uvB) if front_first else (B + A, uvB + uvA)
    bg = (0.25, 0.125, 0.0625)
    sc = flat_scene(tris, W, H, uv_tris=uvs, shading=synth.SHADE_TRANSPARENT, background=bg,
                    textures=[synth.Texture(tex, 0.0, synth.ROLE_ALBEDO)])
    return sc, tex[0, 0], tex[0, 1], np.asarray(bg)


@pytest.mark.parametrize("front_first", [True, False])
def test_two_quads_composite_front_to_back(front_first):
    sc, f, b, bg = _two_quads(front_first)
    deep, rgb = oracle.render_deep(oracle.OracleScene(sc), 0)
    over = lambda c, a, under: a * c[:3] + (1.0 - a) * under
    only_f = over(f, f[3], bg)
    only_b = over(b, b[3], bg)
    both = over(f, f[3], over(b, b[3], bg))
    want = np.tile(bg, (16, 16, 1))
    want[2:10, 2:10] = only_f
    want[10:14, 6:14] = only_b
    want[6:10, 10:14] = only_b
    want[6:10, 6:10] = both
    assert np.allclose(rgb, want, rtol=0, atol=1e-12)
    n = (deep != BG).sum(0)
    assert n[7, 7] == 2 and n[3, 3] == 1 and n[12, 12] == 1 and n[0, 0] == 0
    # the list is ascending: the front quad (depth 0.25) first
    front_ids = {0, 1} if front_first else {2, 3}
    assert int(deep[0, 7, 7] & np.uint64(0xFFFFFFFF)) in front_ids


def test_swapping_depths_swaps_the_composite():
    sc, f, b, bg = _two_quads()
    sc.positions[:, 2] = np.where(sc.positions[:, 2] < 0.5, 0.625, 0.25).astype(np.float32)
    _, rgb = oracle.render_deep(oracle.OracleScene(sc), 0)
    want = b[3] * b[:3] + (1 - b[3]) * (f[3] * f[:3] + (1 - f[3]) * bg)
    assert np.allclose(rgb[7, 7], want, rtol=0, atol=1e-12)


def _rgba_sphere(alpha=None, render=64):
    sc = synth.config_plain(render=render)
    tex = synth.rgba_texture(256, 256, seed=4)
    if alpha is not None:
        tex[..., 3] = alpha
    return synth.with_params(sc, sc.positions, [tex])


def test_opaque_texels_reduce_to_the_opaque_render():
    import dataclasses
    sc = _rgba_sphere(alpha=1.0)
    tr = dataclasses.replace(sc, shading=synth.SHADE_TRANSPARENT, background=(0.2, 0.3, 0.4))
    op = dataclasses.replace(sc, shading=synth.SHADE_UNLIT, background=(0.2, 0.3, 0.4))
    deep, rgb_t = oracle.render_deep(oracle.OracleScene(tr), 0)
    keys, _, rgb_o = oracle.render(oracle.OracleScene(op), 0)
    assert (deep[0] == keys).all()
    assert np.array_equal(rgb_t, rgb_o)
    # a sphere seen from outside: its back faces form the second layer where the front covers
    assert ((deep[1] != BG) == (keys != BG)).mean() > 0.99


def test_deep_list_is_the_smallest_single_triangle_keys():
    W = H = 16
    rng = np.random.default_rng(3)
    tris = []
    for k in range(6):  # six large triangles over the centre, depths in random order
        z = float(rng.uniform(0.1, 0.9))
        c = rng.uniform(6.0, 10.0, size=2)
        r = 9.0
        tris.append([(c[0] - r, c[1] - r, z), (c[0] + r, c[1] - r * 0.2, z), (c[0] - r * 0.1, c[1] + r, z)])
    sc = flat_scene(tris, W, H)
    deep, _ = oracle.render_deep(oracle.OracleScene(sc), 0, with_rgb=False)
    per_tri = []
    for i in range(len(tris)):
        alone = sc.positions.copy()
        for j in range(len(tris)):
            if j != i:
                alone[3 * j:3 * j + 3] = alone[3 * j]  # zero area: dropped, ids unchanged
        keys, _, _ = oracle.render(oracle.OracleScene(synth.with_params(sc, alone, [sc.textures[0].data])), 0)
        per_tri.append(keys)
    allk = np.sort(np.stack(per_tri), axis=0)  # ~0 (not covered) sorts last
    assert (deep == allk[:LAYERS]).all()
    assert (allk[LAYERS] != BG).any()  # some pixels see more fragments than the list keeps


@pytest.mark.parametrize("which", ["vertex", "colour", "opacity", "back_vertex", "back_opacity"])
def test_one_parameter_estimate_equals_central_difference(which):
    """The back_* cases take a parameter of the second fragment of the pixel: a back face that only
    the deep list shows."""
    import dataclasses
    sc0 = _rgba_sphere(render=96)
    sc = dataclasses.replace(sc0, shading=synth.SHADE_TRANSPARENT, background=(0.3, 0.3, 0.3))
    tgt = np.random.default_rng(5).uniform(0.0, 1.0, size=(1, 96, 96, 3)).astype(np.float32)
    osc0 = oracle.OracleScene(sc, tgt)
    keys, uv, _ = oracle.render(osc0, 0)
    deep, _ = oracle.render_deep(osc0, 0, with_rgb=False)
    tri = int(keys[48, 50] & np.uint64(0xFFFFFFFF))
    back = int(deep[1, 48, 50] & np.uint64(0xFFFFFFFF))
    if which == "vertex":
        i, eps = 3 * int(sc.pos_idx[tri, 0]) + 1, 1e-2
    elif which == "back_vertex":
        i, eps = 3 * int(sc.pos_idx[back, 2]) + 0, 1e-2
    elif which == "back_opacity":
        # the back fragment's UV at the pixel: render with the front triangle dropped (zero area)
        pidx = sc.pos_idx.copy()
        pidx[tri] = pidx[tri, 0]
        k2, uv2, _ = oracle.render(oracle.OracleScene(dataclasses.replace(sc, pos_idx=pidx), tgt), 0)
        assert int(k2[48, 50] & np.uint64(0xFFFFFFFF)) == back
        u, v = uv2[48, 50]
        x, y = int(math.floor(u * 256 - 0.5)), int(math.floor(v * 256 - 0.5))
        i, eps = sc.n_pos_params + (y * 256 + x) * 4 + 3, 1.0 / 64.0
    else:
        u, v = uv[48, 50]
        x, y = int(math.floor(u * 256 - 0.5)), int(math.floor(v * 256 - 0.5))
        i = sc.n_pos_params + (y * 256 + x) * 4 + (0 if which == "colour" else 3)
        eps = 1.0 / 64.0
    eps_vec = np.zeros(sc.n_params, np.float32)
    eps_vec[i] = eps
    S, Cn, _ = oracle.estimate(oracle.OracleScene(sc, tgt, eps_vec=eps_vec), 11, 0, [0], 1)
    assert Cn[i] > 0

    def f_at(delta):
        pos = sc.positions.copy().ravel()
        tex = sc.textures[0].data.copy().ravel()
        if i < sc.n_pos_params:
            pos[i] = np.float32(pos[i] + np.float32(delta))
        else:
            tex[i - sc.n_pos_params] = np.float32(tex[i - sc.n_pos_params] + np.float32(delta))
        s2 = synth.with_params(sc, pos.reshape(-1, 3), [tex.reshape(256, 256, 4)])
        return oracle.loss(oracle.OracleScene(s2, tgt), 0)

    fd = (f_at(eps) - f_at(-eps)) / (2 * eps)
    assert fd != 0.0
    assert abs(S[i] / (2 * eps) - fd) <= 1e-9 * max(1.0, abs(fd)), (S[i] / (2 * eps), fd)


def test_hidden_layers_are_credited_and_zero_eps_gives_zero_sums():
    import dataclasses
    sc0 = _rgba_sphere(render=64)
    tgt = np.zeros((1, 64, 64, 3), np.float32)
    tr = dataclasses.replace(sc0, shading=synth.SHADE_TRANSPARENT, eps_pos=0.0,
                             textures=[synth.Texture(sc0.textures[0].data, 0.0, synth.ROLE_ALBEDO)])
    op = dataclasses.replace(tr, shading=synth.SHADE_UNLIT)
    S_t, C_t, _ = oracle.estimate(oracle.OracleScene(tr, tgt), 2, 0, [0], 1)
    S_o, C_o, _ = oracle.estimate(oracle.OracleScene(op, tgt), 2, 0, [0], 1)
    assert np.all(S_t == 0.0) and np.all(S_o == 0.0)
    npos = tr.n_pos_params
    # every vertex the opaque render credits is credited, and the back faces' vertices too
    assert np.all(C_t[:npos][C_o[:npos] > 0] >= C_o[:npos][C_o[:npos] > 0])
    hidden = (C_t[:npos] > 0) & (C_o[:npos] == 0)
    assert hidden.sum() > 0.2 * (C_o[:npos] > 0).sum()


def test_whole_image_form_refuses_transparent_scenes():
    sc, _, _, _ = _two_quads()
    with pytest.raises(ValueError):
        oracle.estimate_full_image(oracle.OracleScene(sc, np.zeros((1, 16, 16, 3), np.float32)), 0, 0, [0], 1)
