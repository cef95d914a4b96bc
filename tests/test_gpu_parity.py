"""GPU path (through the C ABI) against the CPU oracle on the same seeded inputs.

Sizes are small enough for the oracle to finish in seconds and still span many
16x16 tiles, ragged right/bottom tails and several pairs per work item.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.parity import BG, U32, assert_parity, color_k, gpu_scene, run_both, torch_keys_to_u64
from tests.tiny import flat_scene, square_quad

pytestmark = pytest.mark.gpu


def _with_targets(sc):
    return oracle.render_targets(sc, synth.target_scene(sc))


def _sphere(n_lon, n_lat, tex, render_w, render_h, eyes, textured_init=False):
    sc = synth.sphere_scene("t", n_lon, n_lat, tex, render_w, eyes)
    sc.width, sc.height = render_w, render_h
    sc.mvp = np.stack([synth.mvp_matrix(e, render_w, render_h) for e in eyes]).astype(np.float32)
    if textured_init:
        sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(tex, tex, 3, seed=4)])
    return sc


def _lambert_small():
    return synth.config_autograd(n_views=2, pairs=2, render=96, tex=64)


def _lambert_mixed_sizes():
    """Albedo 64^2 RGBA and normal map 32^2: footprints differ per texture (no texel groups)."""
    import dataclasses
    sc = synth.config_autograd(n_views=2, pairs=2, render=96, tex=64)
    nrm = synth.Texture(synth.flat_normal_texture(32, 32), sc.textures[1].eps, synth.ROLE_NORMAL)
    return dataclasses.replace(sc, textures=[sc.textures[0], nrm],
                               target_textures=[sc.target_textures[0], synth.normal_map_texture(32, 32, seed=6)])


def _unlit_channels(c, tw, th):
    """Unlit sphere whose albedo has c channels at tw x th texels (a size whose sign planes end
    mid-word: 8 texels per plane word)."""
    import dataclasses
    sc = _sphere(64, 64, 128, 96, 80, synth.random_eyes(2, 9))
    tex = synth.Texture(synth.constant_texture(tw, th, c, 0.5), sc.textures[0].eps, synth.ROLE_ALBEDO)
    return dataclasses.replace(sc, textures=[tex], target_textures=[synth.sinusoid_texture(tw, th, c, seed=8)])


def _ggx_small():
    return synth.config_scale(n_views=2, pairs=2, render=96, tex=64, n_lon=64, n_lat=32)


RENDER_CASES = {
    "plain_256": lambda: synth.config_plain(256),
    "sphere8k_ragged_70x45": lambda: _sphere(64, 64, 128, 70, 45, synth.random_eyes(3, 2), True),
    "lambert_subdiv": _lambert_small,
    "ggx_grid": _ggx_small,
}


@pytest.mark.parametrize("case", list(RENDER_CASES))
def test_render_idb_bit_exact(case):
    import torch
    sc = RENDER_CASES[case]()
    g = gpu_scene(sc, None)
    osc = oracle.OracleScene(sc)
    for view in range(sc.n_views):
        for pair, side in ((0, 0), (1, 1), (1, -1), (7, -1)):
            keys, uv, rgb = g.render_idb(view, seed=5, it=3, pair=pair, side=side)
            torch.cuda.synchronize()
            ok, ouv, orgb = oracle.render(osc, view, 5, 3, pair, side)
            k = torch_keys_to_u64(keys)
            assert np.array_equal(k, ok), f"view {view} pair {pair} side {side}: {(k != ok).sum()} keys differ"
            cov = ok != BG
            assert cov.sum() > 50
            assert np.array_equal(uv.cpu().numpy()[cov].view(np.uint32), ouv[cov].view(np.uint32))
            diff = np.abs(rgb.cpu().numpy().astype(np.float64) - orgb)
            assert (diff <= color_k(sc) * U32 * (1.0 + np.abs(orgb))).all(), diff.max()
    assert g.status() == 0


def test_render_tiny_edge_cases():
    """Fan tiling the screen with edges through pixel centres; a ragged 37x23 image."""
    import torch
    W, H = 37, 23
    c = (15.5, 11.5)
    dirs = [(1, 0), (2, 1), (1, 1), (1, 2), (0, 1), (-1, 3), (-1, 1), (-3, 1), (-1, 0), (-2, -1), (-1, -1),
            (0, -1), (1, -3), (3, -2)]
    rim = [(c[0] + 40 * dx, c[1] + 40 * dy) for dx, dy in dirs]
    tris = [[c, rim[k], rim[(k + 1) % len(rim)]] for k in range(len(rim))]
    # W, H not powers of two: place the vertices through the camera matrix instead
    sc = flat_scene(tris, 64, 64)
    sc.width, sc.height = W, H
    sc.mvp = np.array([[[64 / W, 0, 0, 64 / W - 1], [0, 64 / H, 0, 1 - 64 / H], [0, 0, 1, 0], [0, 0, 0, 1]]],
                      np.float32)
    g = gpu_scene(sc, None)
    keys, uv, _ = g.render_idb(0)
    torch.cuda.synchronize()
    ok, ouv, _ = oracle.render(oracle.OracleScene(sc), 0)
    assert np.array_equal(torch_keys_to_u64(keys), ok)
    cov = ok != BG
    assert np.array_equal(uv.cpu().numpy()[cov].view(np.uint32), ouv[cov].view(np.uint32))


ESTIMATE_CASES = {
    "plain_256_1view": (lambda: synth.config_plain(256), [0], 3, {}),
    "sphere8k_3views_ragged": (lambda: _sphere(64, 64, 128, 70, 45, synth.random_eyes(3, 2), True),
                               [2, 0, 1], 5, {"pairs_per_item": 2}),
    "sphere8k_128": (lambda: _sphere(64, 64, 512, 128, 128, synth.random_eyes(4, 2)), [0, 1, 2, 3], 4, {}),
    "lambert_subdiv": (_lambert_small, [0, 1], 2, {}),
    "lambert_mixed_sizes": (_lambert_mixed_sizes, [1, 0], 2, {}),
    "ggx_grid": (_ggx_small, [1, 0], 2, {"pairs_per_item": 1}),
    # 32K triangles at 48x48: bins far above the fast path's limit (the general kernel)
    "dense_heavy_bins": (lambda: _sphere(128, 128, 64, 48, 48, synth.random_eyes(2, 5), True), [0, 1], 3, {}),
    # 8K triangles at 96x96: light and heavy bins mixed, pixels with more candidates than kept
    "dense_mixed_bins": (lambda: _sphere(64, 64, 64, 96, 96, synth.random_eyes(2, 6), True), [1, 0], 3,
                         {"pairs_per_item": 2}),
    # 32K triangles at 160^2 (unlit), 32K at 256^2 (Lambert), 64K at 256^2 (GGX): dense meshes whose
    # tiles mix light bins and bins of more than 256 live triangles (the general kernel)
    "dense_unlit": (lambda: _sphere(128, 128, 64, 160, 160, synth.random_eyes(2, 8), True), [0, 1], 2, {}),
    "dense_lambert": (lambda: synth.config_autograd(n_views=2, pairs=2, render=256, tex=64), [1, 0], 2, {}),
    "dense_ggx": (lambda: synth.config_scale(n_views=2, pairs=2, render=256, tex=64, n_lon=256, n_lat=128),
                  [0, 1], 2, {"pairs_per_item": 1}),
    # one- and two-channel albedo of ragged sizes (every channel count of the texel sign planes)
    "albedo_1ch_37x29": (lambda: _unlit_channels(1, 37, 29), [0, 1], 3, {}),
    "albedo_2ch_50x21": (lambda: _unlit_channels(2, 50, 21), [1, 0], 3, {"pairs_per_item": 2}),
    # 5 pairs projected in blocks of 2 (max_pairs_per_call): three launches of each estimator kernel
    "pair_blocks": (lambda: _sphere(64, 64, 128, 96, 96, synth.random_eyes(2, 7)), [0, 1], 5,
                    {"max_pairs_per_call": 2, "pairs_per_item": 2}),
}


@pytest.mark.parametrize("case", list(ESTIMATE_CASES))
def test_estimate_grad_matches_oracle(case):
    make, views, pairs, kw = ESTIMATE_CASES[case]
    sc = make()
    tg = _with_targets(sc)
    r = run_both(sc, tg, seed=11, it=2, views=views, pairs=pairs, gpu_kwargs=kw)
    assert_parity(sc, r)
    assert r["C"].sum() > 0 and np.abs(r["S"]).sum() > 0
    if case in ("dense_unlit", "dense_lambert", "dense_ggx"):
        light, heavy, _ = r["bins"]
        assert light > 0 and heavy > 0, r["bins"]


@pytest.mark.parametrize("case", ["plain_256_1view", "sphere8k_3views_ragged", "lambert_subdiv"])
def test_estimate_grad_plain_matches_oracle(case):
    make, views, pairs, kw = ESTIMATE_CASES[case]
    sc = make()
    tg = _with_targets(sc)
    r = run_both(sc, tg, seed=11, it=2, views=views, pairs=pairs, plain=True)
    assert_parity(sc, r)


NEAREST_CASES = {
    # fast kernel (light bins), several pairs per item, a ragged image
    "fast_ragged": ("sphere8k_3views_ragged", False),
    # the general kernel's bins and the fast one's mixed
    "mixed_bins": ("dense_mixed_bins", False),
    # texel groups (Lambert: albedo and normal map of one size) in both kernels
    "lambert_groups": ("dense_lambert", False),
    # the plain path (staged renders, global scatter)
    "plain_path": ("plain_256_1view", True),
}


@pytest.mark.parametrize("case", list(NEAREST_CASES))
def test_nearest_texel_footprint_matches_oracle(case):
    """Section 4.4's contributor set (the nearest texel, not the bilinear 2x2) on the GPU against
    the oracle's nearest-footprint estimate: counts bit-exact, sums within the tolerance."""
    from paper_2404_09758_gb300 import FOOT_NEAREST
    name, plain = NEAREST_CASES[case]
    make, views, pairs, kw = ESTIMATE_CASES[name]
    sc = make()
    tg = _with_targets(sc)
    r = run_both(sc, tg, seed=13, it=1, views=views, pairs=pairs, plain=plain, footprint=oracle.FOOT_NEAREST,
                 gpu_kwargs=dict(kw, footprint=FOOT_NEAREST))
    assert_parity(sc, r)
    # fewer texel credits than the bilinear footprint would give, and some
    tex = slice(sc.n_pos_params, None)
    assert 0 < r["C"][tex].sum()
    rb = run_both(sc, tg, seed=13, it=1, views=views, pairs=pairs, plain=plain, gpu_kwargs=kw, want_df=False)
    assert r["C"][tex].sum() < rb["C"][tex].sum()


def test_small_table_and_many_chunks_still_match():
    """One pair per work item and a scene whose tiles touch many texels (texture 4x the render)."""
    sc = _sphere(32, 32, 1024, 64, 64, np.array([[0.0, 0.0, 3.0]], np.float32), True)
    tg = _with_targets(sc)
    r = run_both(sc, tg, seed=1, it=0, views=[0], pairs=3, gpu_kwargs={"pairs_per_item": 1})
    assert_parity(sc, r)


def test_zero_eps_gives_zero_sums():
    sc = synth.config_plain(128)
    sc.eps_pos = 0.0
    sc.textures[0].eps = 0.0
    tg = _with_targets(sc)
    r = run_both(sc, tg, seed=3, it=0, views=[0], pairs=2)
    assert np.all(r["grad"] == 0.0)
    assert np.array_equal(r["counts"], r["C"]) and r["C"].sum() > 0


def test_view_that_sees_nothing():
    import torch
    sc = synth.config_plain(64)
    sc.mvp = synth.mvp_matrix((0.0, 0.0, 3.0), 64, 64)[None].copy()
    sc.mvp[0] = synth.perspective(45, 1, 0.1, 10).astype(np.float32) @ synth.look_at((0, 0, 3), (0, 0, 10)).astype(np.float32)
    tg = np.random.default_rng(0).uniform(size=(1, 64, 64, 3)).astype(np.float32)
    r = run_both(sc, tg, seed=3, it=0, views=[0], pairs=2)
    assert r["C"].sum() == 0 and np.all(r["counts"] == 0) and np.all(r["grad"] == 0)
    assert np.isclose(r["loss"][0], (tg.astype(np.float64) ** 2).sum(), rtol=1e-5)


def test_bin_overflow_is_reported_not_silent():
    import torch
    sc = synth.config_plain(64)
    g = gpu_scene(sc, _with_targets(sc), bin_capacity=16)
    grad, counts = g.new_grad_buffers()
    g.estimate_grad(1, 0, [0], 1, grad, counts)
    from paper_2404_09758_gb300 import ERR_BIN_OVERFLOW
    assert g.status() == ERR_BIN_OVERFLOW
    assert g.status() == 0  # reading clears it
    assert counts.sum().item() == 0
    keys, _, _ = g.render_idb(0)  # tiles whose list did not fit render as background
    assert g.status() == ERR_BIN_OVERFLOW
    assert (keys == -1).sum().item() > 0


def test_bad_index_is_reported():
    sc = synth.config_plain(64)
    sc.pos_idx = sc.pos_idx.copy()
    sc.pos_idx[5, 1] = sc.positions.shape[0] + 7
    g = gpu_scene(sc, None)
    from paper_2404_09758_gb300 import ERR_BAD_INDEX
    assert g.validate() == ERR_BAD_INDEX


def test_invalid_arguments_raise():
    from paper_2404_09758_gb300 import SGEError
    sc = synth.config_plain(64)
    g = gpu_scene(sc, None)
    grad, counts = g.new_grad_buffers()
    with pytest.raises(SGEError):
        g.estimate_grad(1, 0, [0, 0], 1, grad, counts)   # view listed twice
    with pytest.raises(SGEError):
        g.estimate_grad(1, 0, [3], 1, grad, counts)      # no such view
    with pytest.raises(SGEError):
        g.estimate_grad(1, 0, [0], 0, grad, counts)      # no pairs
    with pytest.raises(SGEError):
        g.render_idb(0, side=2)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_step_matches_oracle(kind):
    import torch
    sc = synth.config_plain(64)
    g = gpu_scene(sc, None)
    rng = np.random.default_rng(kind)
    d = g.n_params
    S = rng.normal(size=d).astype(np.float32)
    Cn = rng.integers(0, 20, size=d).astype(np.int32)
    m0 = (0.01 * rng.normal(size=d)).astype(np.float32)
    v0 = (0.001 * rng.uniform(size=d)).astype(np.float32)
    theta0 = np.concatenate([p.detach().cpu().numpy().ravel() for p in g.param_groups()])
    eps = np.concatenate([np.full(sc.n_pos_params, sc.eps_pos, np.float32),
                          np.full(sc.textures[0].data.size, sc.textures[0].eps, np.float32)])
    lr = np.concatenate([np.full(sc.n_pos_params, 1e-3, np.float32),
                         np.full(sc.textures[0].data.size, 2e-3, np.float32)])
    grad = torch.tensor(S, device=g.device)
    counts = torch.tensor(Cn, device=g.device)
    m = torch.tensor(m0, device=g.device)
    v = torch.tensor(v0, device=g.device)
    g.step(kind, grad, counts, 8, 1e-3, [2e-3], m=m, v=v, t=3)
    torch.cuda.synchronize()
    # the device receives beta1, beta2 as float32: give the oracle the same values
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    th, mo, vo = oracle.step(kind, theta0, S.astype(np.float64), Cn.astype(np.uint64), eps, lr, 8, t=3, m=m0, v=v0,
                             b1=b1, b2=b2)
    got = np.concatenate([p.detach().cpu().numpy().ravel() for p in g.param_groups()]).astype(np.float64)
    assert np.abs(got - th).max() <= 1e-6 * (1 + np.abs(th).max())
    if kind == 1:
        # float32 moments: g carries <= 2 roundings, g^2 <= 5, then a product and a sum
        g = S.astype(np.float64) / (2 * eps.astype(np.float64) * 8)
        assert (np.abs(m.cpu().numpy() - mo) <= 8 * U32 * (np.abs(b1 * m0) + np.abs((1 - b1) * g))).all()
        assert (np.abs(v.cpu().numpy() - vo) <= 16 * U32 * (np.abs(b2 * v0) + np.abs((1 - b2) * g * g))).all()
    assert grad.abs().sum().item() == 0 and counts.abs().sum().item() == 0
