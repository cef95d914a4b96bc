"""Host-side argument checks of the Python binding (no GPU needed)."""
import pytest


def test_batch_size_is_checked_before_any_call():
    from paper_2404_09758_gb300 import Batch
    with pytest.raises(ValueError):
        Batch([])
    with pytest.raises(ValueError):
        Batch([None] * 65)


def test_no_cpu_path_without_a_gpu():
    """The library has no CPU fallback: without a CUDA device a scene cannot be made."""
    import torch
    import synth
    from paper_2404_09758_gb300 import Scene
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA"):
        Scene.from_arrays(synth.config_plain(render=32))


def test_new_entry_points_check_their_arguments_on_the_host():
    """NULL scenes and negative sizes are refused before anything is launched."""
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    assert L.sge_render_deep(None, 0, 0, 0, 0, 0, None, None, None) == _abi.ERR_INVALID_ARG
    assert b"scene" in L.sge_last_error()
    assert L.sge_refine(None, None, None, 0, None, None, 0, None) == _abi.ERR_INVALID_ARG
    import ctypes as C
    dummy = C.c_int32(0)
    p = C.addressof(dummy)
    assert L.sge_refine(p, p, p, -1, p, p, 0, None) == _abi.ERR_INVALID_ARG
    assert b"n_rows" in L.sge_last_error()


def test_catmull_clark_control_scene_shapes():
    """The teaser-style configuration: the scene's positions are R times the control positions."""
    import numpy as np
    import synth
    sc, ctl, R, tgt = synth.config_control(n_views=2, pairs=2, render=64, tex=32)
    assert R.shape == (len(sc.positions), len(ctl.positions))
    assert np.abs((R @ ctl.positions.astype(np.float64)) - sc.positions).max() <= 1e-6
    assert np.abs((R @ tgt.astype(np.float64)) - sc.target_positions).max() <= 1e-6
    assert len(sc.pos_idx) == 47616
