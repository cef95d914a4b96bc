"""sge_render_idb_static, the render entry point for callers that cannot allocate
device memory (it uses a fixed scratch array in the library instead of a
caller-allocated workspace), must give what sge_render_idb gives.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.parity import BG, U32, color_k

pytestmark = pytest.mark.gpu


def _static_render(desc, view, seed, it, pair, side, H, W, device):
    import torch
    from paper_2404_09758_gb300 import _abi
    keys = torch.full((H, W), 7, dtype=torch.int64, device=device)
    uv = torch.full((H, W, 2), 7.0, dtype=torch.float32, device=device)
    rgb = torch.full((H, W, 3), 7.0, dtype=torch.float32, device=device)
    status = torch.full((1,), -1, dtype=torch.int32, device=device)
    rc = _abi.load().sge_render_idb_static(ctypes.byref(desc), view, seed, it, pair, side, keys.data_ptr(),
                                           uv.data_ptr(), rgb.data_ptr(), status.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    return rc, keys, uv, rgb, status


def _assert_same_as_workspace_render(g, sc, view, pair, side, seed=9, it=4):
    import torch
    k_ref, uv_ref, rgb_ref = g.render_idb(view, seed=seed, it=it, pair=pair, side=side)
    rc, k, uv, rgb, status = _static_render(g._desc, view, seed, it, pair, side, sc.height, sc.width, g.device)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(status.item()) == 0
    assert torch.equal(k, k_ref)
    assert torch.equal(uv.view(torch.int32), uv_ref.view(torch.int32))
    # same kernel, same inputs: the colours agree within the colour tolerance (in fact exactly)
    diff = (rgb.double() - rgb_ref.double()).abs()
    assert (diff <= color_k(sc) * U32 * (1 + rgb_ref.double().abs())).all()
    return k_ref


def test_static_scratch_render_matches_workspace_render_twice():
    from paper_2404_09758_gb300 import Scene
    sc = synth.config_batched(n_views=3, pairs=2, render=160)
    sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(512, 512, 3, seed=4)])
    g = Scene.from_arrays(sc)
    # two calls in a row (the second finds the first one's scratch contents)
    for view, pair, side in ((2, 3, 1), (0, 5, -1)):
        k_ref = _assert_same_as_workspace_render(g, sc, view, pair, side)
        assert (k_ref != -1).sum().item() > 1000


@pytest.mark.parametrize("shading", ["lambert", "ggx"])
def test_static_scratch_render_lit_scenes(shading):
    """Lit models read more textures (normal, roughness, metallic): the static call builds the
    same device view of them as the workspace path."""
    from paper_2404_09758_gb300 import Scene
    if shading == "lambert":
        sc = synth.config_autograd(n_views=2, pairs=2, render=96, tex=64)
    else:
        sc = synth.config_scale(n_views=2, pairs=2, render=96, tex=64, n_lon=64, n_lat=32)
    g = Scene.from_arrays(sc)
    for view, pair, side in ((1, 2, 1), (0, 1, -1)):
        k_ref = _assert_same_as_workspace_render(g, sc, view, pair, side, seed=3, it=1)
        assert (k_ref != -1).sum().item() > 500


def test_static_scratch_larger_then_smaller_scene_match_oracle():
    """A large scene, then a smaller one with a ragged image: the second call must not read the
    first call's bins, tile counts or status.  Both against the oracle's render."""
    from paper_2404_09758_gb300 import Scene
    big = synth.config_batched(n_views=2, pairs=1, render=208)
    big = synth.with_params(big, big.positions, [synth.sinusoid_texture(512, 512, 3, seed=4)])
    small = synth.config_plain(render=72)
    small.width, small.height = 72, 41
    small.mvp = np.stack([synth.mvp_matrix(e, 72, 41) for e in small.cam_pos]).astype(np.float32)
    small = synth.with_params(small, small.positions, [synth.sinusoid_texture(256, 256, 3, seed=5)])
    for sc, view, pair, side in ((big, 1, 2, 1), (small, 0, 3, -1), (big, 0, 1, 0)):
        g = Scene.from_arrays(sc)
        rc, k, uv, rgb, status = _static_render(g._desc, view, 5, 2, pair, side, sc.height, sc.width, g.device)
        import torch
        torch.cuda.synchronize()
        assert rc == 0 and int(status.item()) == 0
        ok, ouv, orgb = oracle.render(oracle.OracleScene(sc), view, 5, 2, pair, side)
        assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
        assert np.array_equal(uv.cpu().numpy().view(np.uint32), ouv.view(np.uint32))
        got = rgb.cpu().numpy().astype(np.float64)
        assert (np.abs(got - orgb) <= color_k(sc) * U32 * (1 + np.abs(orgb))).all()
        assert (ok != BG).sum() > 300


def _big_triangles(n, render, seed=3):
    """n triangles of circumradius 0.3 (clip units: a third of the image) at seeded positions
    and depths: far more tile-bin entries than the static scratch holds."""
    sc, _ = synth.triangle_soup(n, render, seed=seed)
    p = sc.positions.reshape(n, 3, 3).copy()
    c = p.mean(axis=1, keepdims=True)
    p[..., :2] = c[..., :2] + (p[..., :2] - c[..., :2]) * (0.3 / (3.0 / np.sqrt(n)))
    return synth.with_params(sc, p.reshape(-1, 3).astype(np.float32), [sc.textures[0].data])


def test_static_scratch_bin_overflow_drops_whole_tiles():
    """Within the triangle limit but past the fixed bin capacity: the call succeeds, reports
    SGE_ERR_BIN_OVERFLOW in device_status, and every tile either matches a render with enough
    capacity or is left entirely as background."""
    import torch
    from paper_2404_09758_gb300 import ERR_BIN_OVERFLOW, Scene, _abi
    n, R, T = 3000, 2048, 16
    sc = _big_triangles(n, R)
    g = Scene.from_arrays(sc, bin_capacity=12_000_000)
    k_ref, _, _ = g.render_idb(0, seed=1, it=0, pair=0, side=1)
    assert g.status() == 0
    rc, k, _, _, status = _static_render(g._desc, 0, 1, 0, 0, 1, R, R, g.device)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(status.item()) == ERR_BIN_OVERFLOW
    a = k.cpu().numpy().view(np.uint64).reshape(R // T, T, R // T, T).transpose(0, 2, 1, 3)
    b = k_ref.cpu().numpy().view(np.uint64).reshape(R // T, T, R // T, T).transpose(0, 2, 1, 3)
    same = (a == b).all(axis=(2, 3))
    dropped = (a == BG).all(axis=(2, 3))
    assert (same | dropped).all()
    assert (dropped & ~(b == BG).all(axis=(2, 3))).any(), "no covered tile was dropped"
    assert (same & ~(b == BG).all(axis=(2, 3))).any(), "no covered tile was kept"
    # the next call within capacity starts from a clean status
    small = synth.config_plain(render=64)
    gs = Scene.from_arrays(small)
    _assert_same_as_workspace_render(gs, small, 0, 0, 1)


def test_static_scratch_rejects_sizes_beyond_its_limits():
    from paper_2404_09758_gb300 import Scene, _abi
    sc = synth.config_plain(64)
    g = Scene.from_arrays(sc)
    big = _abi.SceneDesc.from_buffer_copy(g._desc)
    big.width, big.height = 4096, 4096
    rc, *_ = _static_render(big, 0, 0, 0, 0, 0, 1, 1, g.device)
    assert rc == _abi.ERR_INVALID_ARG
