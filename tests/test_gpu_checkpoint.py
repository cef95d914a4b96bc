"""Checkpoint and resume of an optimisation (Section 5's loop: estimate, Adam step): a run saved
after some iterations and resumed in a fresh scene credits the next iteration's counts bit for bit
as the uninterrupted run does (the signs depend only on seed, iteration, view, pair and parameter),
and its sums and updated parameters agree to the order of the atomic additions."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, VIEWS, PAIRS = 21, [0, 1], 3


def _setup():
    import torch
    from paper_2404_09758_gb300 import Scene
    sc = synth.sphere_scene("ck", 32, 32, 128, 96, synth.random_eyes(2, 3))
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    g = Scene.from_arrays(sc, targets=tg)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, dtype=torch.float32, device=g.device)
    v = torch.zeros_like(m)
    return sc, g, grad, counts, m, v


def _iteration(sc, g, grad, counts, m, v, it, t):
    """One iteration; returns (counts, sums) as the estimate left them, before the step."""
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM
    g.estimate_grad(SEED, it, VIEWS, PAIRS, grad, counts)
    torch.cuda.synchronize()
    out = counts.cpu().numpy().copy(), grad.cpu().numpy().astype(np.float64)
    g.step(STEP_ADAM, grad, counts, len(VIEWS) * PAIRS, sc.eps_pos, [t_[1] for t_ in g.textures], m=m, v=v, t=t)
    return out


def _theta(g):
    return np.concatenate([p.detach().cpu().numpy().ravel() for p in g.param_groups()]).astype(np.float64)


@pytest.mark.parametrize("with_state", [False, True])
def test_resume_reproduces_the_next_iteration(tmp_path, with_state):
    import torch
    from paper_2404_09758_gb300 import IterState, load_checkpoint, save_checkpoint
    sc, g, grad, counts, m, v = _setup()
    for it in range(3):
        _iteration(sc, g, grad, counts, m, v, it, it + 1)
    path = tmp_path / "run.pt"
    if with_state:
        save_checkpoint(path, g, SEED, IterState(3, 4, device=g.device), m=m, v=v)
    else:
        save_checkpoint(path, g, SEED, 3, 4, m=m, v=v)
    theta_saved = _theta(g)
    c_ref, s_ref = _iteration(sc, g, grad, counts, m, v, 3, 4)
    theta_ref = _theta(g)

    # a fresh scene (initial parameters), then the checkpoint
    sc2, g2, grad2, counts2, m2, v2 = _setup()
    assert not np.array_equal(_theta(g2), theta_saved)
    st = IterState(0, 1, device=g2.device) if with_state else None
    seed, it, t = load_checkpoint(path, g2, m=m2, v=v2, iter_state=st)
    assert (seed, it, t) == (SEED, 3, 4)
    if with_state:
        assert st.value() == (3, 4)
    assert np.array_equal(_theta(g2), theta_saved)
    saved = torch.load(path, weights_only=True)
    assert np.array_equal(m2.cpu().numpy(), saved["m"].numpy()) and np.array_equal(v2.cpu().numpy(), saved["v"].numpy())
    c, s = _iteration(sc2, g2, grad2, counts2, m2, v2, it, t)
    assert np.array_equal(c, c_ref), f"{(c != c_ref).sum()} counts differ"
    assert c.sum() > 0
    assert np.linalg.norm(s - s_ref) <= 1e-5 * np.linalg.norm(s_ref)
    # Adam's step divides by sqrt(v): a parameter first credited now whose sum is at the level of
    # the rounding of its additions may step the other way; every other one agrees closely
    moved = np.abs(_theta(g2) - theta_ref) > 1e-6
    assert moved.mean() < 1e-3, f"{moved.sum()} of {moved.size} parameters differ by more than 1e-6"
    assert g.status() == 0 and g2.status() == 0
