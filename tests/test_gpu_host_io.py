"""An optimizer iteration run from host memory (sge_iterate_host): the parameters and targets
are copied in from CPU tensors, the estimate, the Adam step and the iteration advance run on the
device, and the updated parameters and the estimate's loss come back to CPU tensors (Section 5's
loop: N estimates with fresh signs, then one step).

The plain configuration's loop run this way starts from device arrays that hold nothing useful
(zero parameters, constant targets), so every input has to come through the host copies; its
parameters must then follow the oracle's own loop, and its losses the same loop run eagerly on
the device."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_optimize import N_CHECK, SEED, _oracle_loop

pytestmark = pytest.mark.gpu


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).pin_memory()


def test_host_iteration_loop_follows_oracle_and_eager_loop():
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM, IterState
    from tests.parity import gpu_scene
    sc = synth.config_plain()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    o_loss, o_theta = _oracle_loop(sc, tg, N_CHECK)

    # the same loop eagerly on the device (the estimate's losses of each iteration)
    g = gpu_scene(sc, tg)
    eps_tex = [t[1] for t in g.textures]
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=g.device)
    v = torch.zeros(g.n_params, device=g.device)
    loss = torch.zeros(1, device=g.device)
    eager = []
    for it in range(N_CHECK):
        loss.zero_()
        g.estimate_grad(SEED, it, [0], 1, grad, counts, loss=loss)
        eager.append(float(loss.item()))
        g.step(STEP_ADAM, grad, counts, 1, sc.eps_pos, eps_tex, m=m, v=v, t=it + 1)
    torch.cuda.synchronize()

    h = gpu_scene(sc, tg)
    theta0 = _pinned(np.concatenate([sc.positions.ravel(), sc.textures[0].data.ravel()]))
    targets = _pinned(tg)
    with torch.no_grad():
        for p in h.param_groups():
            p.zero_()
        h.targets.fill_(7.0)
    grad, counts = h.new_grad_buffers()
    m = torch.zeros(h.n_params, device=h.device)
    v = torch.zeros(h.n_params, device=h.device)
    loss_dev = torch.zeros(1, device=h.device)
    state = IterState(0, 1, device=h.device)
    theta_out = torch.empty(h.n_params, dtype=torch.float32).pin_memory()
    losses = torch.zeros(N_CHECK, 1, dtype=torch.float32).pin_memory()
    st = torch.cuda.Stream(device=h.device)
    torch.cuda.synchronize()
    for it in range(N_CHECK):
        first, last = it == 0, it == N_CHECK - 1
        h.iterate_host(SEED, state, [0], 1, grad, counts, m, v, sc.eps_pos, eps_tex, kind=STEP_ADAM,
                       loss_dev=loss_dev, theta_in=theta0 if first else None, targets_in=targets if first else None,
                       theta_out=theta_out if last else None, loss_out=losses[it], stream=st)
    st.synchronize()
    assert h.status(st) == 0
    assert state.value() == (N_CHECK, N_CHECK + 1)
    got = losses.numpy()[:, 0].astype(np.float64)
    assert np.allclose(got, eager, rtol=1e-4), (got, eager)
    theta = theta_out.numpy()
    close = np.abs(theta - o_theta) <= 1e-5 + 1e-5 * np.abs(o_theta)
    assert close.mean() > 0.999, f"{(~close).sum()} of {close.size} parameters differ"
    # the parameters came back through the host copy: the device arrays hold the same values
    dev = torch.cat([p.detach().reshape(-1) for p in h.param_groups()]).cpu()
    assert torch.equal(dev, theta_out)


def test_host_iteration_refuses_loss_out_without_device_loss():
    import torch
    from paper_2404_09758_gb300 import IterState
    from paper_2404_09758_gb300._abi import SGEError
    from tests.parity import gpu_scene
    sc = synth.config_plain(render=64)
    g = gpu_scene(sc, oracle.render_targets(sc, synth.target_scene(sc)))
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=g.device)
    v = torch.zeros(g.n_params, device=g.device)
    with pytest.raises(SGEError):
        g.iterate_host(1, IterState(0, 1, device=g.device), [0], 1, grad, counts, m, v, sc.eps_pos,
                       [t[1] for t in g.textures], loss_out=torch.zeros(1).pin_memory())
