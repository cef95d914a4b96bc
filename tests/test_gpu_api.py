"""The library's diagnostic calls: CUDA-event timing of the estimator kernels and the work
split of the last call."""
import pytest

import synth
from tests.parity import gpu_scene

pytestmark = pytest.mark.gpu


def test_kernel_timing_and_bin_stats():
    import torch
    sc = synth.config_plain(128)
    g = gpu_scene(sc, None)
    grad, counts = g.new_grad_buffers()
    g.kernel_timing(True)
    for it in range(3):
        g.estimate_grad(1, it, [0], 2, grad, counts)
    fast_ms, heavy_ms, n = g.kernel_time(with_heavy=True)
    assert n == 3 and fast_ms > 0.0 and heavy_ms >= 0.0
    assert g.kernel_time() == (0.0, 0)  # read and cleared
    g.kernel_timing(False)
    g.estimate_grad(1, 9, [0], 2, grad, counts)
    assert g.kernel_time() == (0.0, 0)  # timing off records nothing
    light, heavy, entries = g.bin_stats()
    tiles = ((sc.width + 15) // 16) * ((sc.height + 15) // 16)
    assert 0 < light + heavy <= tiles and entries >= light + heavy
    torch.cuda.synchronize()
