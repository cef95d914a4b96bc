"""An optimizer loop captured once in a CUDA graph (Section 5: fresh sign vectors for every
estimate, one Adam step per iteration) must equal the same loop run eagerly.  The iteration
index and Adam's step number live in device memory (sge_iter_state): the captured estimate and
step read them when they run and the captured advance moves them on, so replay k is
iteration k."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import group_slices, rel_l2

pytestmark = pytest.mark.gpu

SEED = 11


def _capture(fn, stream):
    import torch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    stream.synchronize()
    return g


def test_graph_replays_draw_the_next_iterations_signs():
    """Estimate-only graph: replay k gives exactly the eager estimate of iteration it0 + k
    (counts bit-exact, sums within the parity tolerance), and the state ends at it0 + K."""
    import torch
    from paper_2404_09758_gb300 import IterState
    from tests.parity import gpu_scene
    sc = synth.config_batched(n_views=3, pairs=4, render=96)
    sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(512, 512, 3, seed=4)])
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    g = gpu_scene(sc, tg)
    views, pairs, it0, K = [0, 1, 2], 4, 40, 4
    grad, counts = g.new_grad_buffers()
    eager = []
    for k in range(K):
        grad.zero_()
        counts.zero_()
        g.estimate_grad(SEED, it0 + k, views, pairs, grad, counts)
        eager.append((grad.double().cpu().numpy(), counts.cpu().numpy().copy()))
    st = torch.cuda.Stream(device=g.device)
    state = IterState(it0, 1, device=g.device)
    snaps = torch.zeros(K, 2, g.n_params, dtype=torch.float64, device=g.device)
    slot = torch.zeros(1, dtype=torch.int64, device=g.device)

    def body():
        grad.zero_()
        counts.zero_()
        g.estimate_grad(SEED, state, views, pairs, grad, counts, stream=st)
        snaps.index_copy_(0, slot, torch.stack([grad.double(), counts.double()])[None])
        slot.add_(1)
        state.advance(1, 0, stream=st)

    torch.cuda.synchronize()
    graph = _capture(body, st)
    for _ in range(K):
        graph.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    assert state.value() == (it0 + K, 1)
    for k in range(K):
        S, Cn = eager[k]
        got_S, got_C = snaps[k, 0].cpu().numpy(), snaps[k, 1].cpu().numpy()
        assert np.array_equal(got_C.astype(np.int64), Cn.astype(np.int64)), f"replay {k}: counts differ"
        for sl in group_slices(sc):
            if np.linalg.norm(S[sl]) > 0:
                assert rel_l2(got_S[sl], S[sl]) <= 1e-4, f"replay {k}"
    # the replays really differ from one another (fresh signs per iteration)
    assert rel_l2(snaps[1, 0].cpu().numpy(), snaps[0, 0].cpu().numpy()) > 0.1


def test_graph_adam_loop_equals_eager_loop():
    """Estimate + Adam step + advance captured once, replayed K times, against the eager loop
    with iteration it and t = it + 1: the per-iteration image errors agree, and the parameters
    agree as closely as two eager runs agree with each other (float atomics sum in a different
    order on every run; where a sum is near zero Adam's sign of the step can flip)."""
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM, IterState
    from tests.parity import gpu_scene
    sc = synth.config_batched(n_views=2, pairs=4, render=96)
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    views, pairs, K = [0, 1], 4, 6
    runs = []
    for mode in ("eager", "graph", "eager"):
        g = gpu_scene(sc, tg)
        grad, counts = g.new_grad_buffers()
        m = torch.zeros(g.n_params, device=g.device)
        v = torch.zeros(g.n_params, device=g.device)
        loss = torch.zeros(len(views), device=g.device)
        losses = torch.zeros(K, device=g.device)
        eps_tex = [t[1] for t in g.textures]
        st = torch.cuda.Stream(device=g.device)
        if mode == "eager":
            with torch.cuda.stream(st):
                for k in range(K):
                    loss.zero_()
                    g.estimate_grad(SEED, k, views, pairs, grad, counts, loss=loss, stream=st)
                    losses[k] = loss.sum()
                    g.step(STEP_ADAM, grad, counts, len(views) * pairs, sc.eps_pos, eps_tex, m=m, v=v, t=k + 1,
                           stream=st)
        else:
            state = IterState(0, 1, device=g.device)
            slot = torch.zeros(1, dtype=torch.int64, device=g.device)

            def body():
                loss.zero_()
                g.estimate_grad(SEED, state, views, pairs, grad, counts, loss=loss, stream=st)
                losses.index_copy_(0, slot, loss.sum()[None])
                slot.add_(1)
                g.step(STEP_ADAM, grad, counts, len(views) * pairs, sc.eps_pos, eps_tex, m=m, v=v, t=state,
                       stream=st)
                state.advance(1, 1, stream=st)

            torch.cuda.synchronize()
            graph = _capture(body, st)
            for _ in range(K):
                graph.replay()
            assert state.value() == (K, K + 1)
        torch.cuda.synchronize()
        assert g.status() == 0
        theta = torch.cat([p.detach().reshape(-1) for p in g.param_groups()]).cpu().numpy().astype(np.float64)
        runs.append((losses.cpu().numpy().astype(np.float64), theta))
    (le, te), (lg, tgr), (le2, te2) = runs
    assert np.allclose(lg, le, rtol=1e-4), (lg, le)
    assert le[-1] < le[0]

    def differ(a, b):
        return float((np.abs(a - b) > 1e-6 + 1e-6 * np.abs(b)).mean())

    d_graph, d_eager = differ(tgr, te), differ(te2, te)
    assert d_graph <= 2.0 * d_eager + 1e-3, (d_graph, d_eager)
    assert d_graph < 0.01, d_graph
    # the loop moved the parameters the views see (about a third of them here)
    assert differ(tgr, _initial_theta(sc)) > 0.2


def _initial_theta(sc):
    return np.concatenate([sc.positions.ravel(), sc.textures[0].data.ravel()]).astype(np.float64)


def test_graph_plain_configuration_loop_follows_oracle():
    """The plain configuration's Adam loop (one view, one pair per iteration) captured once and
    replayed: its first iterations follow the oracle's own loop, as the eager loop does."""
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM, IterState
    from tests.parity import gpu_scene
    from tests.test_gpu_optimize import N_CHECK, SEED as OSEED, _oracle_loop
    sc = synth.config_plain()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    o_loss, o_theta = _oracle_loop(sc, tg, N_CHECK)
    g = gpu_scene(sc, tg)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=g.device)
    v = torch.zeros(g.n_params, device=g.device)
    eps_tex = [t[1] for t in g.textures]
    st = torch.cuda.Stream(device=g.device)
    state = IterState(0, 1, device=g.device)
    img = torch.zeros(N_CHECK + 1, device=g.device)
    slot = torch.zeros(1, dtype=torch.int64, device=g.device)
    err = torch.zeros(1, device=g.device)

    def body():
        err.zero_()
        g.loss([0], out=err, stream=st)
        img.index_copy_(0, slot, err)
        slot.add_(1)
        g.estimate_grad(OSEED, state, [0], 1, grad, counts, stream=st)
        g.step(STEP_ADAM, grad, counts, 1, sc.eps_pos, eps_tex, m=m, v=v, t=state, stream=st)
        state.advance(1, 1, stream=st)

    torch.cuda.synchronize()
    graph = _capture(body, st)
    for _ in range(N_CHECK):
        graph.replay()
    torch.cuda.synchronize()
    theta = torch.cat([p.detach().reshape(-1) for p in g.param_groups()]).cpu().numpy()
    img[N_CHECK] = g.loss([0]).sum()
    torch.cuda.synchronize()
    assert g.status() == 0
    losses = img.cpu().numpy().astype(np.float64)
    assert np.allclose(losses, o_loss, rtol=1e-3), (losses, o_loss)
    close = np.abs(theta - o_theta) <= 1e-5 + 1e-5 * np.abs(o_theta)
    assert close.mean() > 0.999, f"{(~close).sum()} of {close.size} parameters differ"
