"""Transparent geometry (Section 4.4) through the C ABI against the oracle: three overlapping
semi-transparent spheres (up to six fragments a pixel, the deep ID buffer keeps four) on a
ragged 100 x 100 render.  Deep ID buffers bit-exact and composites within the colour
tolerance; sge_estimate_grad's sums, counts, loss and per-pixel loss differences; the image
error of sge_loss; the calls a transparent scene does not take; a scene without an RGBA
albedo is refused."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests.parity import BG, U32, assert_parity, color_k, gpu_scene

pytestmark = pytest.mark.gpu

SEED, ITER = 21, 4


def _scene(render=100, views=2, pairs=3):
    sc = synth.config_transparent(n_views=views, pairs=pairs, render=render, tex=64, n_lon=16, n_lat=16)
    return sc, oracle.render_targets(sc, synth.target_scene(sc))


def test_deep_render_matches_oracle():
    sc, tg = _scene()
    g = gpu_scene(sc, tg)
    osc = oracle.OracleScene(sc, tg)
    k = color_k(sc)
    deepest = 0
    for view, pair, side in [(0, 0, 1), (0, 0, -1), (1, 2, 0), (1, 1, 1)]:
        deep, rgb = g.render_deep(view, seed=SEED, it=ITER, pair=pair, side=side)
        od, orgb = oracle.render_deep(osc, view, SEED, ITER, pair, side)
        got = deep.cpu().numpy().view(np.uint64)
        assert (got == od).all(), f"view {view} pair {pair} side {side}: {(got != od).sum()} keys differ"
        err = np.abs(rgb.cpu().numpy().astype(np.float64) - orgb)
        assert (err <= k * U32 * (1.0 + np.abs(orgb))).all(), err.max()
        deepest = max(deepest, int((od != BG).sum(0).max()))
    assert deepest == synth_layers()
    assert g.status() == 0


def synth_layers():
    from paper_2404_09758_gb300 import MAX_LAYERS
    return MAX_LAYERS


# 100 x 100: tiles whose bins fit one staged chunk of 128 triangles (credits pre-summed in shared
# memory) beside larger ones; 32 x 32: the three spheres' 1,536 triangles over four tiles, every
# bin larger than a chunk (credits straight to the global sums)
@pytest.mark.parametrize("render,views,pairs", [(100, 2, 3), (48, 1, 5), (32, 1, 2)])
def test_estimate_matches_oracle(render, views, pairs):
    import torch
    sc, tg = _scene(render, views, pairs)
    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    vids = list(range(views))
    df = torch.empty(views, pairs, sc.height, sc.width, device=g.device)
    loss = torch.zeros(views, device=g.device)
    g.estimate_grad(SEED, ITER, vids, pairs, grad, counts, loss=loss, delta_f=df)
    st = g.status()
    torch.cuda.synchronize()
    S, Cn, oloss, odf, fmax, cond = oracle.estimate(oracle.OracleScene(sc, tg), SEED, ITER, vids, pairs,
                                                    per_pixel=True)
    assert_parity(sc, dict(status=st, grad=grad.cpu().numpy().astype(np.float64),
                           counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                           loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss,
                           df=df.cpu().numpy().astype(np.float64), odf=odf, fmax=fmax, cond=cond))
    assert (odf != 0).sum() > 100


def test_estimate_with_nearest_texel_footprint_matches_oracle():
    """Every listed fragment credits only its nearest texel (Section 4.4's footprint)."""
    import torch
    from paper_2404_09758_gb300 import FOOT_NEAREST
    sc, tg = _scene(64, 2, 3)
    g = gpu_scene(sc, tg, footprint=FOOT_NEAREST)
    grad, counts = g.new_grad_buffers()
    loss = torch.zeros(2, device=g.device)
    g.estimate_grad(SEED, ITER, [0, 1], 3, grad, counts, loss=loss)
    st = g.status()
    torch.cuda.synchronize()
    S, Cn, oloss = oracle.estimate(oracle.OracleScene(sc, tg, footprint=oracle.FOOT_NEAREST), SEED, ITER, [0, 1], 3)
    assert_parity(sc, dict(status=st, grad=grad.cpu().numpy().astype(np.float64),
                           counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                           loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss))
    assert Cn[sc.n_pos_params:].sum() > 0


def test_loss_and_targets_match_oracle():
    import torch
    sc, tg = _scene()
    g = gpu_scene(sc, tg)
    loss = g.loss([0, 1])
    osc = oracle.OracleScene(sc, tg)
    want = np.array([oracle.loss(osc, 0), oracle.loss(osc, 1)])
    assert np.allclose(loss.cpu().numpy(), want, rtol=1e-5)
    # targets rendered on the GPU from the target scene agree with the oracle's
    t = gpu_scene(synth.target_scene(sc), None).render_targets()
    torch.cuda.synchronize()
    assert np.abs(t.cpu().numpy() - tg).max() <= color_k(sc) * U32 * 2.0


def test_calls_a_transparent_scene_does_not_take():
    import torch
    from paper_2404_09758_gb300 import Batch, SGEError
    sc, tg = _scene(render=32, views=1)
    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    with pytest.raises(SGEError, match="transparent"):
        g.render_idb(0)
    with pytest.raises(SGEError, match="transparent"):
        g.estimate_grad_plain(0, 0, [0], 1, grad, counts)
    with pytest.raises(SGEError, match="transparent"):
        g.estimate_grad_full_image(0, 0, [0], 1, grad, counts)
    with pytest.raises(SGEError, match="transparent"):
        Batch([(g, [0], grad, counts)]).estimate_grad(0, 0, 1)
    opaque = gpu_scene(synth.config_plain(render=32), None)
    with pytest.raises(SGEError, match="not transparent"):
        opaque.render_deep(0)
    rgb = dataclasses.replace(sc, textures=[synth.Texture(sc.textures[0].data[..., :3].copy(), 0.01,
                                                          synth.ROLE_ALBEDO)])
    with pytest.raises(SGEError, match="RGBA"):
        gpu_scene(rgb, tg)
    torch.cuda.synchronize()
    assert g.status() == 0
