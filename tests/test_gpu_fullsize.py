"""Parity at the benchmark's full size and launch configuration: the unlit 8,192-triangle
sphere, 512^2 texture and render, 8 views x 64 antithetic pairs in one batched call.

The oracle computes the whole job (512 estimates) in a pool of spawned processes, one
view per worker; counts must match exactly, sums within 1e-4 relative L2 per group;
the per-pixel loss differences are compared on sampled (view, pair) images.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import U32, assert_parity, gpu_scene, group_slices, rel_l2

pytestmark = pytest.mark.gpu

SEED, ITER, PAIRS = 1, 0, 64


def _oracle_view(args):
    view, targets, per_pixel_pairs = args
    sc = synth.config_batched()
    osc = oracle.OracleScene(sc, targets)
    S, C, loss = oracle.estimate(osc, SEED, ITER, [view], PAIRS)
    dfs = None
    if per_pixel_pairs:
        r = oracle.estimate(osc, SEED, ITER, [view], per_pixel_pairs, per_pixel=True)
        dfs = (r[3][0], r[4][0], r[5][0])
    return view, S, C, loss[0], dfs


def test_full_size_batched_estimate_matches_oracle():
    import torch
    sc = synth.config_batched()
    targets = oracle.render_targets(sc, synth.target_scene(sc))
    sampled = {0: 2, 5: 2}  # views whose first pairs' per-pixel differences are compared
    ctx = mp.get_context("spawn")
    n_proc = min(len(sc.mvp), max(1, os.cpu_count() or 1))
    with ctx.Pool(n_proc) as pool:
        jobs = pool.map_async(_oracle_view, [(v, targets, sampled.get(v, 0)) for v in range(sc.n_views)])
        g = gpu_scene(sc, targets)
        grad, counts = g.new_grad_buffers()
        loss = torch.zeros(sc.n_views, device=g.device)
        df = torch.empty(sc.n_views, PAIRS, sc.height, sc.width, device=g.device)
        g.estimate_grad(SEED, ITER, list(range(sc.n_views)), PAIRS, grad, counts, loss=loss, delta_f=df)
        st = g.status()
        torch.cuda.synchronize()
        res = jobs.get()
    S = np.zeros(sc.n_params)
    C = np.zeros(sc.n_params, np.uint64)
    oloss = np.zeros(sc.n_views)
    for view, Sv, Cv, lv, dfs in res:
        S += Sv
        C += Cv
        oloss[view] = lv
    r = dict(status=st, grad=grad.cpu().numpy().astype(np.float64),
             counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
             loss=loss.cpu().numpy().astype(np.float64), S=S, C=C, oloss=oloss)
    assert_parity(sc, r)
    assert C.sum() > 10**9  # the whole job: about 1.9 G contributions
    for view, _, _, _, dfs in res:
        if dfs is None:
            continue
        odf, fmax, cond = dfs
        got = df[view, :odf.shape[0]].cpu().numpy().astype(np.float64)
        tol = 1e-5 * np.maximum(fmax, 1e-6) + 8 * U32 * cond
        assert (np.abs(got - odf) <= tol).all(), f"view {view}: loss differences out of tolerance"
