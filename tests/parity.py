"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare them with the tolerances stated here.

Tolerances (derived from the arithmetic of each side):
  - depth|ID keys, UV buffer, counts: bit-exact (integers, or floats whose
    rounding sequence is fixed on both sides);
  - loss differences f+ - f-: |diff| <= 1e-5 max(f+, f-, 1e-6) + k u cond with
    u = 2^-24 (float32 unit roundoff) and cond = sum_c (|a_c| + |b_c|)(|I+_c| +
    |I-_c| + 2|I_c|), a = I+ - I-, b = I+ + I- - 2I: a float32 colour carries
    about k u of relative error, which the product a*b carries into f+ - f-.
    k = 8 for unlit and Lambert shading (a bilinear sum and a dot product);
    k = 4096 for GGX, whose distribution term divides by (n.h^2 (alpha^2 - 1) + 1)^2
    and so amplifies rounding by up to 1/alpha^2, on top of three normalisations and the
    view and light terms that vanish at grazing and barely lit pixels: on the 1M-triangle
    GGX scene at 2048^2 the float32 colour of a pixel whose n.l is near zero on one side
    was measured 1.06e-4 (about 1,800 u) from the float64 oracle, the same in a plain
    render as in the fused estimator;
    k = 32 for transparent geometry: up to four bilinear fragments, each weighted by a
    running product of (1 - alpha) factors, summed front to back;
  - colours of one render: |diff| <= k u (1 + |I|) with the same k;
  - gradient sums: relative L2 error <= 1e-4 per parameter group against the
    oracle's float64 sums.
"""
import numpy as np

import oracle

U32 = 2.0 ** -24
BG = np.uint64(0xFFFFFFFFFFFFFFFF)


def gpu_scene(sc, targets, **kw):
    from paper_2404_09758_gb300 import Scene
    return Scene.from_arrays(sc, targets=targets, **kw)


def torch_keys_to_u64(t):
    return t.cpu().numpy().view(np.uint64)


def group_slices(sc):
    offs = sc.param_offsets() + [sc.n_params]
    return [slice(offs[k], offs[k + 1]) for k in range(len(offs) - 1)]


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def run_both(sc, targets, seed, it, views, pairs, plain=False, footprint=0, gpu_kwargs=None, want_df=True):
    import torch
    g = gpu_scene(sc, targets, **(gpu_kwargs or {}))
    grad, counts = g.new_grad_buffers()
    loss = torch.zeros(len(views), device=g.device)
    df = None
    if plain:
        g.estimate_grad_plain(seed, it, views, pairs, grad, counts, loss=loss)
    else:
        if want_df:
            df = torch.empty(len(views), pairs, sc.height, sc.width, device=g.device)
        g.estimate_grad(seed, it, views, pairs, grad, counts, loss=loss, delta_f=df)
    st = g.status()
    bins = g.bin_stats() if not plain else None
    torch.cuda.synchronize()
    osc = oracle.OracleScene(sc, targets, footprint=footprint)
    res = oracle.estimate(osc, seed, it, views, pairs, per_pixel=want_df and not plain)
    out = dict(status=st, grad=grad.cpu().numpy().astype(np.float64),
               counts=counts.cpu().numpy().astype(np.int64).astype(np.uint64),
               loss=loss.cpu().numpy().astype(np.float64), S=res[0], C=res[1], oloss=res[2], bins=bins)
    if df is not None:
        out.update(df=df.cpu().numpy().astype(np.float64), odf=res[3], fmax=res[4], cond=res[5])
    return out


def color_k(sc):
    import synth
    return {synth.SHADE_GGX: 4096.0, synth.SHADE_TRANSPARENT: 32.0}.get(sc.shading, 8.0)


def assert_parity(sc, r, grad_tol=1e-4):
    assert r["status"] == 0
    assert np.array_equal(r["counts"], r["C"]), \
        f"counts differ at {np.flatnonzero(r['counts'] != r['C'])[:10]}"
    for k, sl in enumerate(group_slices(sc)):
        if np.linalg.norm(r["S"][sl]) > 0:
            e = rel_l2(r["grad"][sl], r["S"][sl])
            assert e <= grad_tol, f"group {k}: relative L2 error {e:.3g}"
        else:
            assert np.all(r["grad"][sl] == 0.0)
    assert np.allclose(r["loss"], r["oloss"], rtol=1e-5, atol=1e-6)
    if "df" in r:
        tol = 1e-5 * np.maximum(r["fmax"], 1e-6) + color_k(sc) * U32 * r["cond"]
        bad = np.abs(r["df"] - r["odf"]) > tol
        assert not bad.any(), f"{bad.sum()} loss differences out of tolerance"
