"""Parity at the scale configuration's full size: 1,048,576-triangle displaced grid sphere,
four 2048^2 RGB maps (albedo, roughness, metallic, normal), GGX with one light, 2048^2
render.  The whole 16 views x 16 pairs call runs in the benchmark's launch configuration
with its per-pixel loss differences kept; the oracle recomputes sampled (view, pair)
images one by one.  Gradient sums and counts are compared on a call over two views and
two pairs of the same scene (the oracle's cost grows with every estimate)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import U32, assert_parity, color_k, gpu_scene

pytestmark = pytest.mark.gpu

SEED, ITER = 5, 1
SAMPLED = [(0, 0), (9, 1)]  # (view, pair) images whose loss differences the oracle recomputes
GRAD_VIEWS, GRAD_PAIRS = [3, 12], 2


def _scene():
    return synth.config_scale()


def _oracle_targets(views):
    sc = _scene()
    tsc = synth.target_scene(sc)
    osc = oracle.OracleScene(tsc, None)
    return {v: oracle.render(osc, v)[2].astype(np.float32) for v in views}


def _oracle_job(args):
    kind, view, pair, targets = args
    sc = _scene()
    tg = np.zeros((sc.n_views, sc.height, sc.width, 3), np.float32)
    for v, img in targets.items():
        tg[v] = img
    osc = oracle.OracleScene(sc, tg)
    if kind == "df":
        # the per-pixel differences of pair `pair` alone: an estimate of pairs 0..pair keeps
        # every pair's image, so ask for exactly that many
        r = oracle.estimate(osc, SEED, ITER, [view], pair + 1, per_pixel=True)
        return kind, view, pair, (r[3][0][pair], r[4][0][pair], r[5][0][pair])
    S, C, loss = oracle.estimate(osc, SEED, ITER, GRAD_VIEWS, GRAD_PAIRS)
    return kind, view, pair, (S, C, loss)


def test_scale_full_call_matches_oracle_on_samples():
    import torch
    sc = _scene()
    views_needed = sorted({v for v, _ in SAMPLED} | set(GRAD_VIEWS))
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(4, max(1, os.cpu_count() or 1))) as pool:
        # targets of the views the oracle uses come from the oracle; the others from the GPU
        per_view = pool.map(_oracle_targets, [[v] for v in views_needed])
        otg = {v: img for d in per_view for v, img in d.items()}
        jobs = pool.map_async(_oracle_job, [("df", v, p, otg) for v, p in SAMPLED] + [("grad", -1, -1, otg)])
        tscene = gpu_scene(synth.target_scene(sc), None)
        targets = tscene.render_targets()
        torch.cuda.synchronize()
        del tscene
        for v, img in otg.items():
            targets[v] = torch.from_numpy(img).to(targets.device)
        g = gpu_scene(sc, targets, max_pairs_per_call=sc.pairs_per_view)
        grad, counts = g.new_grad_buffers()
        views = list(range(sc.n_views))
        df = torch.empty(sc.n_views, sc.pairs_per_view, sc.height, sc.width, device=g.device)
        loss = torch.zeros(sc.n_views, device=g.device)
        g.estimate_grad(SEED, ITER, views, sc.pairs_per_view, grad, counts, loss=loss, delta_f=df)
        st_full = g.status()
        torch.cuda.synchronize()
        total = int(counts.to(torch.int64).sum().item())
        grad.zero_()
        counts.zero_()
        loss2 = torch.zeros(len(GRAD_VIEWS), device=g.device)
        g.estimate_grad(SEED, ITER, GRAD_VIEWS, GRAD_PAIRS, grad, counts, loss=loss2)
        st = g.status()
        torch.cuda.synchronize()
        got = dict(grad=grad.cpu().numpy().astype(np.float64),
                   counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                   loss=loss2.cpu().numpy().astype(np.float64))
        res = jobs.get()
    assert st_full == 0 and st == 0
    assert total > 10**9  # the full call credits billions of contributions
    for kind, view, pair, out in res:
        if kind == "df":
            odf, fmax, cond = out
            d = df[view, pair].cpu().numpy().astype(np.float64)
            tol = 1e-5 * np.maximum(fmax, 1e-6) + color_k(sc) * U32 * cond
            bad = np.abs(d - odf) > tol
            if bad.any():
                r = np.abs(d - odf) / tol
                y, x = np.unravel_index(int(np.argmax(r)), r.shape)
                raise AssertionError(
                    f"view {view} pair {pair}: {bad.sum()} loss differences out of tolerance; worst at (x {x}, "
                    f"y {y}): gpu {d[y, x]!r} oracle {odf[y, x]!r} tolerance {tol[y, x]!r} (x{r[y, x]:.2f}), "
                    f"f max {fmax[y, x]!r}, cond {cond[y, x]!r}")
            assert (odf != 0).sum() > 10**5
        else:
            S, C, oloss = out
            assert_parity(sc, dict(status=st, S=S, C=C, oloss=oloss, **got))
