"""The plain configuration's optimisation loop (Section 5): one view, one antithetic pair per
iteration, the paper's Adam (beta1 0.9, beta2 0.999, learning rate = eps per group), from the
undisplaced sphere and a gray texture towards the displaced, textured target.

The GPU loop (sge_estimate_grad + sge_step) and the oracle's own loop (estimate + step in
float64, parameters rounded to float32 between iterations) run side by side for the first
iterations: their image errors and parameters must agree.  The GPU loop then runs the full 200
iterations and must cut the image error by more than 80 %.  (Plain SGD with one pair per
iteration diverges at any rate that moves the texels visibly: every texel's estimate carries
the position parameters' much larger gradients as noise, scaled by eps_pos / eps_tex.  Adam's
per-parameter normalisation is why the paper uses it.)"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED = 3
N_CHECK = 8


def _oracle_loop(sc, tg, n):
    pos, tex = sc.positions.copy(), sc.textures[0].data.copy()
    d = pos.size + tex.size
    m, v = np.zeros(d, np.float32), np.zeros(d, np.float32)
    eps = np.concatenate([np.full(pos.size, sc.eps_pos, np.float32),
                          np.full(tex.size, np.float32(sc.textures[0].eps))])
    losses = []
    for it in range(n):
        osc = oracle.OracleScene(synth.with_params(sc, pos, [tex]), tg)
        losses.append(oracle.loss(osc, 0))
        S, C, _ = oracle.estimate(osc, SEED, it, [0], 1)
        theta = np.concatenate([pos.ravel(), tex.ravel()])
        th, m, v = oracle.step(1, theta, S, C, eps, eps, 1, t=it + 1, m=m, v=v)
        th, m, v = th.astype(np.float32), m.astype(np.float32), v.astype(np.float32)
        pos, tex = th[:pos.size].reshape(pos.shape), th[pos.size:].reshape(tex.shape)
    osc = oracle.OracleScene(synth.with_params(sc, pos, [tex]), tg)
    losses.append(oracle.loss(osc, 0))
    return np.array(losses), np.concatenate([pos.ravel(), tex.ravel()])


def test_plain_configuration_adam_loop_matches_oracle_and_converges():
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM
    from tests.parity import gpu_scene
    sc = synth.config_plain()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    o_loss, o_theta = _oracle_loop(sc, tg, N_CHECK)

    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=g.device)
    v = torch.zeros(g.n_params, device=g.device)
    eps_tex = [t[1] for t in g.textures]
    losses = []
    for it in range(200):
        losses.append(float(g.loss([0]).item()))
        if it == N_CHECK:
            theta = torch.cat([p.detach().reshape(-1) for p in g.param_groups()]).cpu().numpy()
        g.estimate_grad(SEED, it, [0], 1, grad, counts)
        g.step(STEP_ADAM, grad, counts, 1, sc.eps_pos, eps_tex, m=m, v=v, t=it + 1)
    losses.append(float(g.loss([0]).item()))
    assert g.status() == 0
    # the first iterations follow the oracle's loop
    assert np.allclose(losses[:N_CHECK + 1], o_loss, rtol=1e-3), (losses[:N_CHECK + 1], o_loss)
    close = np.abs(theta - o_theta) <= 1e-5 + 1e-5 * np.abs(o_theta)
    assert close.mean() > 0.999, f"{(~close).sum()} of {close.size} parameters differ"
    # and the full loop converges
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    print(f"image error {losses[0]:.1f} -> {losses[-1]:.1f} after 200 iterations")
