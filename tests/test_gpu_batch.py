"""Batched estimator over several assets (sge_estimate_grad_batch): assets of uneven
triangle counts and texture sizes, each with its own views and outputs, in one
persistent launch per estimator kernel.  Every asset's sums and counts must match
the oracle's estimate of that asset alone (counts exactly, sums within 1e-4
relative L2 per group), whatever launch shape the call uses."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, gpu_scene

pytestmark = pytest.mark.gpu

SEED, ITER = 17, 3


def _small_assets():
    # triangle counts 200..20,000 at 96^2: the larger assets have bins above the light limit
    return synth.config_uneven(n_assets=5, n_views=3, pairs=3, render=96, tri_lo=200, tri_hi=20_000,
                               tex_choices=(32, 64, 128))


def _views_of(k):
    return [k % 3, (k + 1) % 3]


def _run_batch(scs, targets, pairs, tuning=None, autotune=False, max_pairs=0):
    import torch
    from paper_2404_09758_gb300 import Batch
    gs, bufs, entries = [], [], []
    for k, (sc, tg) in enumerate(zip(scs, targets)):
        g = gpu_scene(sc, tg, max_views_per_call=2, max_pairs_per_call=max_pairs)
        grad, counts = g.new_grad_buffers()
        loss = torch.zeros(2, device=g.device)
        gs.append(g)
        bufs.append((grad, counts, loss))
        entries.append((g, _views_of(k), grad, counts, loss))
    b = Batch(entries)
    if autotune:
        b.autotune(pairs, repeats=1)
    if tuning:
        for name, v in tuning.items():
            setattr(b.tuning, name, v)
    b.estimate_grad(SEED, ITER, pairs)
    sts = [g.status() for g in gs]
    torch.cuda.synchronize()
    return gs, bufs, sts, b


def _check_against_oracle(scs, targets, bufs, sts, pairs):
    for k, (sc, tg) in enumerate(zip(scs, targets)):
        S, Cn, oloss = oracle.estimate(oracle.OracleScene(sc, tg), SEED, ITER, _views_of(k), pairs)
        grad, counts, loss = bufs[k]
        r = dict(status=sts[k], grad=grad.cpu().numpy().astype(np.float64),
                 counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                 loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss)
        assert_parity(sc, r)


@pytest.fixture(scope="module")
def small():
    scs = _small_assets()
    targets = [oracle.render_targets(sc, synth.target_scene(sc)) for sc in scs]
    return scs, targets


def test_batch_default_shape_matches_oracle(small):
    scs, targets = small
    _, bufs, sts, _ = _run_batch(scs, targets, 3)
    _check_against_oracle(scs, targets, bufs, sts, 3)


@pytest.mark.parametrize("tuning", [dict(pairs_per_item=1, blocks_per_sm=1, light_bin=64),
                                    dict(pairs_per_item=2, light_bin=128)])
def test_batch_other_shapes_match_oracle(small, tuning):
    scs, targets = small
    _, bufs, sts, _ = _run_batch(scs, targets, 3, tuning=tuning)
    _check_against_oracle(scs, targets, bufs, sts, 3)


def test_batch_pair_blocks_and_autotune_match_oracle(small):
    """Pairs in blocks of 2 (max_pairs_per_call) after the autotuner picked the shape."""
    scs, targets = small
    _, bufs, sts, b = _run_batch(scs, targets, 3, autotune=True, max_pairs=2)
    assert 1 <= b.tuning.pairs_per_item <= 64 and b.tuning.light_bin in (64, 128, 256)
    _check_against_oracle(scs, targets, bufs, sts, 3)


def test_autotune_cache_reuses_the_stored_shape(small, tmp_path):
    """With a cache file, the first autotune times and stores its shape; a second batch of the
    same assets takes it from the file without timing (the same shape and the stored ms), and
    its estimate still matches the oracle."""
    import json
    import torch
    from paper_2404_09758_gb300 import Batch
    scs, targets = small
    cache = str(tmp_path / "tune.json")
    shapes = []
    for rep in range(2):
        gs, bufs, entries = [], [], []
        for k, (sc, tg) in enumerate(zip(scs, targets)):
            g = gpu_scene(sc, tg, max_views_per_call=2)
            grad, counts = g.new_grad_buffers()
            loss = torch.zeros(2, device=g.device)
            gs.append(g)
            bufs.append((grad, counts, loss))
            entries.append((g, _views_of(k), grad, counts, loss))
        b = Batch(entries)
        ms = b.autotune(3, repeats=1, cache=cache)
        shapes.append((b.tuning.pairs_per_item, b.tuning.blocks_per_sm, b.tuning.light_bin, ms))
    assert shapes[0] == shapes[1]
    assert len(json.load(open(cache))) == 1
    b.estimate_grad(SEED, ITER, 3)
    sts = [g.status() for g in gs]
    torch.cuda.synchronize()
    _check_against_oracle(scs, targets, bufs, sts, 3)


def test_batch_equals_single_scene_calls(small):
    """Same estimates as one sge_estimate_grad per asset: counts exactly, sums to float order."""
    import torch
    scs, targets = small
    gs, bufs, sts, _ = _run_batch(scs, targets, 3)
    assert all(s == 0 for s in sts)
    for k, g in enumerate(gs):
        grad, counts = g.new_grad_buffers()
        loss = torch.zeros(2, device=g.device)
        g.estimate_grad(SEED, ITER, _views_of(k), 3, grad, counts, loss=loss)
        torch.cuda.synchronize()
        assert torch.equal(counts, bufs[k][1])
        assert torch.allclose(grad, bufs[k][0], rtol=1e-4, atol=1e-5 * float(grad.abs().max()))
        assert torch.allclose(loss, bufs[k][2], rtol=1e-5)


def test_lit_batch_matches_oracle():
    """Two Lambert assets (one with textures of one size, one with albedo and normal map of
    different sizes) in one batched call: the lit estimator kernels of the batched form."""
    import dataclasses
    import torch
    from paper_2404_09758_gb300 import Batch
    a = synth.config_autograd(n_views=2, pairs=2, render=96, tex=64)
    nrm = synth.Texture(synth.flat_normal_texture(32, 32), a.textures[1].eps, synth.ROLE_NORMAL)
    b = dataclasses.replace(a, textures=[a.textures[0], nrm],
                            target_textures=[a.target_textures[0], synth.normal_map_texture(32, 32, seed=6)])
    scs = [a, b]
    targets = [oracle.render_targets(sc, synth.target_scene(sc)) for sc in scs]
    views = [[0, 1], [1]]
    gs, bufs, entries = [], [], []
    for sc, tg, vw in zip(scs, targets, views):
        g = gpu_scene(sc, tg)
        grad, counts = g.new_grad_buffers()
        loss = torch.zeros(len(vw), device=g.device)
        gs.append(g)
        bufs.append((grad, counts, loss))
        entries.append((g, vw, grad, counts, loss))
    Batch(entries).estimate_grad(SEED, ITER, 2)
    sts = [g.status() for g in gs]
    torch.cuda.synchronize()
    for k, (sc, tg, vw) in enumerate(zip(scs, targets, views)):
        S, Cn, oloss = oracle.estimate(oracle.OracleScene(sc, tg), SEED, ITER, vw, 2)
        grad, counts, loss = bufs[k]
        assert_parity(sc, dict(status=sts[k], grad=grad.cpu().numpy().astype(np.float64),
                               counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                               loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss))


def test_batch_rejects_bad_entries(small):
    import torch
    from paper_2404_09758_gb300 import Batch, SGEError
    scs, targets = small
    g = gpu_scene(scs[0], targets[0], max_views_per_call=2)
    grad, counts = g.new_grad_buffers()
    with pytest.raises(SGEError):  # the same scene twice
        Batch([(g, [0], grad, counts), (g, [1], grad, counts)]).estimate_grad(0, 0, 1)
    with pytest.raises(SGEError):  # a view out of range
        Batch([(g, [7], grad, counts)]).estimate_grad(0, 0, 1)
    with pytest.raises(SGEError):  # more views than the scene's workspace holds
        Batch([(g, [0, 1, 2], grad, counts)]).estimate_grad(0, 0, 1)
    torch.cuda.synchronize()


# ---------------------------------------------------------------- full uneven configuration

FULL_PAIRS = 8


def _oracle_targets(k):
    sc = synth.uneven_asset(k)
    return oracle.render_targets(sc, synth.target_scene(sc))


def _oracle_asset(args):
    k, tg = args
    sc = synth.uneven_asset(k)
    S, Cn, oloss = oracle.estimate(oracle.OracleScene(sc, tg), SEED, ITER, list(range(sc.n_views)), FULL_PAIRS)
    return k, S, Cn, oloss


def test_full_uneven_batch_matches_oracle_on_sampled_assets():
    """32 assets (1K..200K triangles, 256^2..2048^2 textures), 512^2, 4 views x 8 pairs each,
    one batched call with the autotuned shape.  The smallest, a middle and the largest asset
    are checked against the oracle; every asset's counts equal its single-scene call's."""
    import torch
    from paper_2404_09758_gb300 import Batch
    scs = synth.config_uneven()
    nts = [len(sc.pos_idx) for sc in scs]
    order = np.argsort(nts)
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(sample), max(1, os.cpu_count() or 1))) as pool:
        # the sampled assets' targets come from the oracle (its inputs never come from the GPU)
        targets = dict(zip(sample, pool.map(_oracle_targets, sample)))
        jobs = pool.map_async(_oracle_asset, [(k, targets[k]) for k in sample])
        gs, bufs, entries = [], [], []
        for k, sc in enumerate(scs):
            if k in targets:
                tg = targets[k]
            else:
                tscene = gpu_scene(synth.target_scene(sc), None, max_pairs_per_call=FULL_PAIRS)
                tg = tscene.render_targets()
                torch.cuda.synchronize()
                del tscene
            g = gpu_scene(sc, tg, max_pairs_per_call=FULL_PAIRS)
            grad, counts = g.new_grad_buffers()
            loss = torch.zeros(sc.n_views, device=g.device)
            gs.append(g)
            bufs.append((grad, counts, loss))
            entries.append((g, list(range(sc.n_views)), grad, counts, loss))
        b = Batch(entries)
        b.autotune(FULL_PAIRS, repeats=1)
        b.estimate_grad(SEED, ITER, FULL_PAIRS)
        sts = [g.status() for g in gs]
        torch.cuda.synchronize()
        # every asset: the same counts as its own single-scene call
        for k, g in enumerate(gs):
            grad, counts = g.new_grad_buffers()
            g.estimate_grad(SEED, ITER, list(range(scs[k].n_views)), FULL_PAIRS, grad, counts)
            torch.cuda.synchronize()
            assert torch.equal(counts, bufs[k][1]), f"asset {k}"
        res = jobs.get()
    assert all(s == 0 for s in sts), [(k, s) for k, s in enumerate(sts) if s]
    for k, S, Cn, oloss in res:
        grad, counts, loss = bufs[k]
        r = dict(status=sts[k], grad=grad.cpu().numpy().astype(np.float64),
                 counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
                 loss=loss.cpu().numpy().astype(np.float64), S=S, C=Cn, oloss=oloss)
        assert_parity(scs[k], r)
