"""Section 6.1's experiment on the GPU: a soup of 1,024 independent triangles (12 parameters
each: three vertices and an RGB colour) fitted to a smooth image with Adam, once with the
per-pixel estimator (Eq. 8, sge_estimate_grad) and once with the full-image one (Eq. 4,
sge_estimate_grad_full_image), the same number of estimates per iteration.  The first iterations
of both loops follow the oracle's own loops; after 60 iterations the per-pixel form has removed
most of the error (the oracle's loop: 94 %) and the full-image form far less (oracle: 41 %)."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import gpu_scene

pytestmark = pytest.mark.gpu

N, RENDER, ITERS, PAIRS, N_CHECK = 1024, 128, 60, 4, 4


def _oracle_losses(sc, tg, kind, n):
    pos, tex = sc.positions.copy(), sc.textures[0].data.copy()
    d = pos.size + tex.size
    m, v = np.zeros(d, np.float32), np.zeros(d, np.float32)
    eps = np.concatenate([np.full(pos.size, sc.eps_pos, np.float32),
                          np.full(tex.size, np.float32(sc.textures[0].eps))])
    losses = []
    for it in range(n):
        osc = oracle.OracleScene(synth.with_params(sc, pos, [tex]), tg)
        losses.append(oracle.loss(osc, 0))
        if kind == "per_pixel":
            S, C, _ = oracle.estimate(osc, 1, it, [0], PAIRS)
        else:
            S, C = oracle.estimate_full_image(osc, 1, it, [0], PAIRS)[:2]
        th = np.concatenate([pos.ravel(), tex.ravel()])
        th, m, v = oracle.step(1, th, S, C, eps, eps, PAIRS, t=it + 1, m=m, v=v)
        th, m, v = th.astype(np.float32), m.astype(np.float32), v.astype(np.float32)
        pos, tex = th[:pos.size].reshape(pos.shape), th[pos.size:].reshape(tex.shape)
    return np.array(losses)


def _gpu_losses(sc, tg, kind):
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM
    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=g.device)
    v = torch.zeros(g.n_params, device=g.device)
    losses = []
    for it in range(ITERS):
        losses.append(float(g.loss([0]).item()))
        if kind == "per_pixel":
            g.estimate_grad(1, it, [0], PAIRS, grad, counts)
        else:
            g.estimate_grad_full_image(1, it, [0], PAIRS, grad, counts)
        g.step(STEP_ADAM, grad, counts, PAIRS, sc.eps_pos, [sc.textures[0].eps], m=m, v=v, t=it + 1)
    losses.append(float(g.loss([0]).item()))
    assert g.status() == 0
    return np.array(losses)


def test_per_pixel_estimator_outpaces_the_full_image_one():
    sc, tg = synth.triangle_soup(N, RENDER, seed=0)
    red = {}
    for kind in ("per_pixel", "full_image"):
        got = _gpu_losses(sc, tg, kind)
        want = _oracle_losses(sc, tg, kind, N_CHECK)
        assert np.allclose(got[:N_CHECK], want, rtol=1e-3), (kind, got[:N_CHECK], want)
        red[kind] = got[-1] / got[0]
    assert red["per_pixel"] < 0.15, red
    assert red["full_image"] > 0.4, red
    print(f"error left after {ITERS} iterations: per-pixel {red['per_pixel']:.3f}, "
          f"full-image {red['full_image']:.3f}")
