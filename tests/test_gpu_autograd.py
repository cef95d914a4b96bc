"""The autograd form: forward = render + L2 (sge_loss), backward = the per-pixel
stochastic estimate of Eq. 9 (sge_estimate_grad + sge_gradient)."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import gpu_scene, group_slices, rel_l2

pytestmark = pytest.mark.gpu


def _small():
    sc = synth.config_autograd(n_views=3, pairs=2, render=96, tex=64)
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    return sc, tg


def test_forward_loss_matches_oracle():
    import torch
    sc, tg = _small()
    g = gpu_scene(sc, tg)
    got = g.loss([2, 0, 1]).cpu().numpy().astype(np.float64)
    osc = oracle.OracleScene(sc, tg)
    want = np.array([oracle.loss(osc, v) for v in (2, 0, 1)])
    assert np.allclose(got, want, rtol=1e-5)


def test_backward_is_the_scaled_estimate_and_matches_oracle():
    import torch
    from paper_2404_09758_gb300 import sge_loss
    sc, tg = _small()
    g = gpu_scene(sc, tg)
    views, pairs, seed, it = [0, 2], 2, 21, 5
    loss = sge_loss(g, seed, it, views, pairs)
    (3.0 * loss).backward()
    got = np.concatenate([p.grad.detach().cpu().numpy().ravel() for p in g.param_groups()]).astype(np.float64)
    # the same sums straight from the oracle, for the same seeds
    S, C, _ = oracle.estimate(oracle.OracleScene(sc, tg), seed, it, views, pairs)
    eps = np.concatenate([np.full(sc.n_pos_params, sc.eps_pos)] +
                         [np.full(t.data.size, np.float32(t.eps)) for t in sc.textures])
    # the forward sums the views' errors: per-view estimates (N = pairs) summed over views
    want = 3.0 * S / (2.0 * eps.astype(np.float32).astype(np.float64) * pairs)
    for k, sl in enumerate(group_slices(sc)):
        assert rel_l2(got[sl], want[sl]) <= 1e-4, k
    # forward value is the summed image error of the listed views
    osc = oracle.OracleScene(sc, tg)
    assert np.isclose(loss.item(), sum(oracle.loss(osc, v) for v in views), rtol=1e-5)


def test_estimate_agrees_with_central_differences_on_sampled_parameters():
    """Full autograd configuration (32,768 triangles, 1024^2 RGBA albedo + normal map, Lambert,
    1024^2 render, 16 views x 16 pairs): the mean of repeated backward passes against central
    differences with h = eps on 1,000 sampled parameters.  The reference sums the per-pixel
    differences of two renders in float64, since a float32 whole-image loss cannot resolve the
    change one parameter makes."""
    import torch
    from paper_2404_09758_gb300 import Scene
    sc = synth.config_autograd()
    tscene = Scene.from_arrays(synth.target_scene(sc))
    targets = tscene.render_targets()
    torch.cuda.synchronize()
    del tscene
    g = Scene.from_arrays(sc, targets=targets)
    views = list(range(sc.n_views))
    pairs = sc.pairs_per_view
    grad, counts = g.new_grad_buffers()
    g.estimate_grad(0, 0, views, pairs, grad, counts)
    touched = (counts > 0).nonzero().flatten().cpu().numpy()
    offs = sc.param_offsets() + [sc.n_params]
    rng = np.random.default_rng(0)
    picks = []
    for k, n in ((0, 200), (1, 500), (2, 300)):  # vertex coordinates, albedo texels, normal-map texels
        cand = touched[(touched >= offs[k]) & (touched < offs[k + 1])]
        picks.append(rng.choice(cand, size=n, replace=False))
    picks = np.concatenate(picks)
    # estimator: mean and standard error over repeated iterations
    R = 24
    est = np.zeros((R, picks.size))
    idx = torch.tensor(picks, device=g.device)
    for r in range(R):
        grad.zero_()
        counts.zero_()
        g.estimate_grad(7, 1000 + r, views, pairs, grad, counts)
        # estimate of the gradient of the summed error of all views: per-view Eq. 9, summed
        est[r] = g.gradient(grad, pairs)[idx].double().cpu().numpy()
    mean, se = est.mean(0), est.std(0, ddof=1) / np.sqrt(R)
    # central differences, per-pixel float64 sums
    groups = g.param_groups()
    tgt64 = targets.double()

    def image_error_diff():
        out = torch.zeros((), dtype=torch.float64, device=g.device)
        for v in views:
            _, _, rgb = g.render_idb(v)
            out += ((rgb.double() - tgt64[v]) ** 2).sum()
        return out

    fd = np.zeros(picks.size)
    for n, i in enumerate(picks):
        k = int(np.searchsorted(offs, i, side="right") - 1)
        flat = groups[k].detach().view(-1)
        li = int(i - offs[k])
        h = sc.eps_pos if k == 0 else sc.textures[k - 1].eps
        old = flat[li].item()
        flat[li] = float(np.float32(old + h))
        fp = image_error_diff()
        flat[li] = float(np.float32(old - h))
        fm = image_error_diff()
        flat[li] = old
        fd[n] = ((fp - fm) / (2.0 * h)).item()
    z = (mean - fd) / np.maximum(se, 1e-30)
    alb = slice(200, 700)
    rgb = ((picks[alb] - offs[1]) % 4) < 3  # the albedo's alpha channel does not reach the image
    kinds = {"vertex": (slice(0, 200), None), "albedo rgb": (alb, rgb), "albedo alpha": (alb, ~rgb),
             "normal": (slice(700, 1000), None)}
    stats = {}
    for name, (sl, m) in kinds.items():
        zz, mm, ff = z[sl], mean[sl], fd[sl]
        if m is not None:
            zz, mm, ff = zz[m], mm[m], ff[m]
        c = np.corrcoef(mm, ff)[0, 1] if ff.std() > 0 else float("nan")
        stats[name] = (c, np.median(np.abs(zz)), np.mean(np.abs(zz) < 4))
        print(f"{name}: n {zz.size} corr {c:.4f} median|z| {stats[name][1]:.3f} frac|z|<4 {stats[name][2]:.3f}")
    # albedo enters the image linearly: the estimate is unbiased, z ~ N(0, 1) (median |z| 0.674).
    # (Its correlation with the differences is limited by noise: the standard error of 24
    # iterations is about the size of a texel's gradient.)
    for name in ("albedo rgb", "albedo alpha"):
        assert stats[name][1] < 1.0 and stats[name][2] > 0.95, name
    # the normal map enters through normalisation and clamping, vertices also through
    # visibility: the estimate and the central difference carry different O(eps^2) terms;
    # they must agree in direction and scale
    assert stats["normal"][1] < 1.0 and stats["normal"][0] > 0.6
    assert stats["vertex"][1] < 2.0 and stats["vertex"][0] > 0.85
    assert np.corrcoef(mean, fd)[0, 1] > 0.9
