"""Control-mesh optimisation through linear subdivision: the subdivided mesh is R times the
control mesh, so R^T maps the subdivided vertices' sums to the control vertices.  sge_refine
(one CSR row per thread) against scipy's sparse products of the oracle's sums."""
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


def test_control_mesh_sums_through_the_refine_matrix():
    import torch
    from paper_2404_09758_gb300 import refine
    control = synth.uv_sphere(16, 16)
    ctl_pos = synth.radial_displace(control.positions, seed=3, amplitude=0.04)
    control = dataclasses.replace(control, positions=ctl_pos)
    R = synth.linear_refine_matrix(control, 2)
    fine = synth.subdivide_linear(control, 2)
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
    assert np.abs(y.cpu().numpy() - want).max() <= 4 * np.finfo(np.float32).eps * np.abs(want).max()
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
