"""sge_render_idb_static, the render entry point for callers that cannot allocate
device memory (it uses a fixed scratch array in the library instead of a
caller-allocated workspace), must give what sge_render_idb gives.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

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


def test_static_scratch_render_matches_workspace_render_twice():
    import torch
    from paper_2404_09758_gb300 import Scene
    sc = synth.config_batched(n_views=3, pairs=2, render=160)
    sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(512, 512, 3, seed=4)])
    g = Scene.from_arrays(sc)
    # two calls in a row (the second finds the first one's scratch contents)
    for view, pair, side in ((2, 3, 1), (0, 5, -1)):
        k_ref, uv_ref, rgb_ref = g.render_idb(view, seed=9, it=4, pair=pair, side=side)
        rc, k, uv, rgb, status = _static_render(g._desc, view, 9, 4, pair, side, sc.height, sc.width, g.device)
        torch.cuda.synchronize()
        assert rc == 0
        assert int(status.item()) == 0
        assert torch.equal(k, k_ref)
        assert (k_ref != -1).sum().item() > 1000
        assert torch.equal(uv.view(torch.int32), uv_ref.view(torch.int32))
        # same kernel, same inputs: the colours agree within the colour tolerance (in fact exactly)
        diff = (rgb.double() - rgb_ref.double()).abs()
        assert (diff <= 8 * 2.0 ** -24 * (1 + rgb_ref.double().abs())).all()


def test_static_scratch_rejects_sizes_beyond_its_limits():
    from paper_2404_09758_gb300 import Scene, _abi
    sc = synth.config_plain(64)
    g = Scene.from_arrays(sc)
    big = _abi.SceneDesc.from_buffer_copy(g._desc)
    big.width, big.height = 4096, 4096
    rc, *_ = _static_render(big, 0, 0, 0, 0, 0, 1, 1, g.device)
    assert rc == _abi.ERR_INVALID_ARG
