"""Control-mesh optimisation through subdivision (linear, and Catmull-Clark as in Section 6.3):
the subdivided mesh is R times the control mesh, so R^T maps the subdivided vertices' sums to the
control vertices.  sge_refine (one CSR row per thread) against scipy's sparse products of the
oracle's sums."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, gpu_scene, rel_l2

pytestmark = pytest.mark.gpu


def _csr(M, device):
    import torch
    M = M.tocsr()
    M.sort_indices()
    return (torch.tensor(M.indptr.astype(np.int32), device=device),
            torch.tensor(M.indices.astype(np.int32), device=device),
            torch.tensor(M.data.astype(np.float32), device=device))


def _subdivide(kind, control):
    if kind == "linear":
        return synth.subdivide_linear(control, 2), synth.linear_refine_matrix(control, 2)
    return synth.subdivide_catmull_clark(control, 2)


@pytest.mark.parametrize("kind", ["linear", "catmull_clark"])
def test_control_mesh_sums_through_the_refine_matrix(kind):
    import torch
    from paper_2404_09758_gb300 import refine
    control = synth.uv_sphere(16, 16)
    ctl_pos = synth.radial_displace(control.positions, seed=3, amplitude=0.04)
    control = dataclasses.replace(control, positions=ctl_pos)
    fine, R = _subdivide(kind, control)
    base = synth.sphere_scene("t", 16, 16, 64, 96, synth.random_eyes(2, 4))
    tgt_ctl = synth.radial_displace(synth.uv_sphere(16, 16).positions, seed=5, amplitude=0.06)
    sc = dataclasses.replace(base, positions=fine.positions, pos_idx=fine.pos_idx, uvs=fine.uvs,
                             uv_idx=fine.uv_idx,
                             target_positions=(R @ tgt_ctl.astype(np.float64)).astype(np.float32))
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    g = gpu_scene(sc, tg)
    dev = g.device
    # refine: the subdivided positions from the control positions
    x = torch.tensor(control.positions, device=dev)
    y = refine(_csr(R, dev), x)
    want = R @ control.positions.astype(np.float64)
    # a row of k terms summed in float32, with weights rounded to float32: error below
    # (k + 1) units of 2^-24 of the sum of |w x|
    bound = abs(R) @ np.abs(control.positions.astype(np.float64))
    k = np.diff(R.indptr)[:, None]
    assert (np.abs(y.cpu().numpy() - want) <= (k + 1) * 2.0 ** -24 * bound + 1e-30).all()
    # estimate on the subdivided mesh, then the control vertices' sums through R^T
    grad, counts = g.new_grad_buffers()
    loss = torch.zeros(2, device=dev)
    g.estimate_grad(6, 1, [0, 1], 3, grad, counts, loss=loss)
    st = g.status()
    nf = 3 * len(fine.positions)
    ctl = refine(_csr(R.T, dev), grad[:nf].reshape(-1, 3))
    torch.cuda.synchronize()
    S, Cn, oloss = oracle.estimate(oracle.OracleScene(sc, tg), 6, 1, [0, 1], 3)
    assert_parity(sc, dict(status=st, grad=grad.cpu().numpy().astype(np.float64),
                           counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                           loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss))
    want_c = (R.T @ S[:nf].reshape(-1, 3))
    assert np.linalg.norm(want_c) > 0
    assert rel_l2(ctl.cpu().numpy().astype(np.float64).ravel(), want_c.ravel()) <= 1e-4


N_CHECK = 6


def _cc_loop_scene():
    """A 12 x 12 control sphere under two Catmull-Clark levels (6,336 triangles), the texture
    already the target's: only the control vertices have to move (radial displacement 0.08)."""
    ctl = synth.uv_sphere(12, 12)
    fine, R = synth.subdivide_catmull_clark(ctl, 2)
    tgt_ctl = synth.radial_displace(ctl.positions, seed=5, amplitude=0.08)
    base = synth.sphere_scene("cc", 12, 12, 64, 128, np.array([[0.0, 0.0, 3.0]], np.float32))
    sc = dataclasses.replace(base, positions=fine.positions, pos_idx=fine.pos_idx, uvs=fine.uvs,
                             uv_idx=fine.uv_idx,
                             textures=[dataclasses.replace(base.textures[0], data=base.target_textures[0].copy())],
                             target_positions=(R @ tgt_ctl.astype(np.float64)).astype(np.float32))
    return ctl, R, sc


def _oracle_control_loop(ctl, R, sc, tg, n, seed):
    """The same loop in the oracle: fine = R control (float64, rounded), the oracle's estimate on
    the fine scene, R^T on its position sums, the oracle's Adam step on the control parameters."""
    pos, tex = ctl.positions.copy(), sc.textures[0].data.copy()
    d = pos.size + tex.size
    m, v = np.zeros(d, np.float32), np.zeros(d, np.float32)
    eps = np.concatenate([np.full(pos.size, sc.eps_pos, np.float32),
                          np.full(tex.size, np.float32(sc.textures[0].eps))])
    nf = 3 * R.shape[0]
    losses = []
    for it in range(n + 1):
        fpos = (R @ pos.astype(np.float64)).astype(np.float32)
        osc = oracle.OracleScene(synth.with_params(sc, fpos, [tex]), tg)
        losses.append(oracle.loss(osc, 0))
        if it == n:
            break
        S, C, _ = oracle.estimate(osc, seed, it, [0], 1)
        Sc = np.concatenate([(R.T @ S[:nf].reshape(-1, 3)).ravel(), S[nf:]])
        th = np.concatenate([pos.ravel(), tex.ravel()])
        th, m, v = oracle.step(1, th, Sc, np.zeros(d, np.uint64), eps, eps, 1, t=it + 1, m=m, v=v)
        th, m, v = th.astype(np.float32), m.astype(np.float32), v.astype(np.float32)
        pos, tex = th[:pos.size].reshape(pos.shape), th[pos.size:].reshape(tex.shape)
    return np.array(losses), np.concatenate([pos.ravel(), tex.ravel()])


def test_control_mesh_adam_loop_through_catmull_clark():
    """Section 6.3's control-mesh optimisation: refine, estimate on the subdivided surface, R^T
    to the control vertices, Adam on the control parameters.  The first iterations follow the
    oracle's loop; 200 iterations cut the image error by more than 80 %."""
    import torch
    from paper_2404_09758_gb300 import STEP_ADAM, ControlMesh
    ctl, R, sc = _cc_loop_scene()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    o_loss, o_theta = _oracle_control_loop(ctl, R, sc, tg, N_CHECK, 3)
    g = gpu_scene(sc, tg)
    cm = ControlMesh(g, ctl, R)
    gf, cf = g.new_grad_buffers()
    gc, cc = cm.new_grad_buffers()
    m = torch.zeros(cm.params.n_params, device=g.device)
    v = torch.zeros(cm.params.n_params, device=g.device)
    losses = []
    for it in range(200):
        cm.refine()
        losses.append(float(g.loss([0]).item()))
        if it == N_CHECK:
            theta = torch.cat([p.detach().reshape(-1) for p in cm.params.param_groups()]).cpu().numpy()
        g.estimate_grad(3, it, [0], 1, gf, cf)
        cm.control_sums(gf, gc)
        cm.params.step(STEP_ADAM, gc, cc, 1, sc.eps_pos, [sc.textures[0].eps], m=m, v=v, t=it + 1)
        gf.zero_()
        cf.zero_()
    cm.refine()
    losses.append(float(g.loss([0]).item()))
    assert g.status() == 0 and cm.params.status() == 0
    assert np.allclose(losses[:N_CHECK + 1], o_loss, rtol=1e-3), (losses[:N_CHECK + 1], o_loss)
    # float32 sums differ from the oracle's float64 ones in their last bits; where a sum is near
    # zero Adam's step can take the other sign, and after the next refine a moved vertex can snap
    # differently, so a few parameters drift apart (a wrong refinement, R^T or step would move most)
    close = np.abs(theta - o_theta) <= 1e-5 + 1e-5 * np.abs(o_theta)
    assert close.mean() > 0.995, f"{(~close).sum()} of {close.size} parameters differ"
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    print(f"image error {losses[0]:.1f} -> {losses[-1]:.1f} after 200 iterations")
