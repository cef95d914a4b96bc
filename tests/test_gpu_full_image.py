"""The full-image estimator (Eq. 4 with the whole-image error, Section 6.1's comparison) against
the oracle.  Tolerances from the arithmetic: each estimate's dF is a float32 sum of the per-pixel
differences, so |dF_gpu - dF_oracle| <= sum_p (per-pixel bound of tests/parity.py) + 64 u
sum_p |f+_p - f-_p|; every parameter's sum adds the estimates' dF with signs, so its bound is the
sum of those plus n u sum_e |dF_e| for the float32 accumulation over the n estimates."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import U32, color_k, gpu_scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["unlit", "lambert"])
def test_full_image_estimate_matches_oracle(case):
    import torch
    if case == "unlit":
        sc, views, pairs = synth.config_plain(96), [0], 3
    else:
        sc, views, pairs = synth.config_autograd(n_views=2, pairs=2, render=80, tex=32), [1, 0], 2
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    dF = g.estimate_grad_full_image(4, 2, views, pairs, grad, counts)
    assert g.status() == 0
    torch.cuda.synchronize()
    S, Cn, odF, A, M, K = oracle.estimate_full_image(oracle.OracleScene(sc, tg), 4, 2, views, pairs)
    n = len(views) * pairs
    got = dF.cpu().numpy().astype(np.float64).ravel()
    bound = 1e-5 * M + color_k(sc) * U32 * K + 64 * U32 * A
    assert (np.abs(got - odF) <= bound).all(), (got, odF, bound)
    assert np.abs(odF).max() > 0
    assert (counts.cpu().numpy() == n).all()
    sb = bound.sum() + n * U32 * np.abs(odF).sum()
    gs = grad.cpu().numpy().astype(np.float64)
    assert (np.abs(gs - S) <= sb).all(), np.abs(gs - S).max() / sb
