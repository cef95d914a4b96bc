"""Cases for the range-checked build (run as a child process with SGE_CHECKED=1, so that the
package loads libsge_checked.so): prints one JSON object with what each case observed.

Every case makes its bad input on the host.  Lowered bounds (Scene.check_limit) change only what
the checks compare against, never an allocation, so an access a check misses still stays inside
its buffer.  The one real out-of-range input (a pos_idx entry past the vertex array) is read only
through the checked index helpers, which read it as vertex 0.
"""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def _scene():
    sc = synth.config_plain(96)
    sc = synth.with_params(sc, sc.positions, [synth.sinusoid_texture(256, 256, 3, seed=4)])
    return sc, oracle.render_targets(sc, synth.target_scene(sc))


def _estimate(g, views=(0,), pairs=3, plain=False):
    import torch
    grad, counts = g.new_grad_buffers()
    if plain:
        g.estimate_grad_plain(5, 1, list(views), pairs, grad, counts)
    else:
        g.estimate_grad(5, 1, list(views), pairs, grad, counts)
    torch.cuda.synchronize()
    return g.status(), grad.cpu().numpy(), counts.cpu().numpy()


def main():
    import torch
    import paper_2404_09758_gb300 as sge
    from tests.parity import assert_parity, run_both
    torch.cuda.set_device(0)
    out = {"checked": sge.checked_build()}
    sc, tg = _scene()

    # no false alarms: a valid scene gives status 0 and the oracle's counts and sums
    r = run_both(sc, tg, seed=5, it=1, views=[0], pairs=3)
    assert_parity(sc, r)
    out["parity_status"] = r["status"]

    g = sge.Scene.from_arrays(sc, targets=tg)
    st0, grad0, cnt0 = _estimate(g)
    out["clean_status"] = st0
    n_params = int(g.n_params)
    limits = {"vertices": (sge.LIMIT_VERTICES, sc.positions.shape[0] // 2),
              "uvs": (sge.LIMIT_UVS, sc.uvs.shape[0] // 2),
              "bin_entries": (sge.LIMIT_BIN_ENTRIES, 10),
              "sign_words": (sge.LIMIT_SIGN_WORDS, 5),
              "params": (sge.LIMIT_PARAMS, n_params // 2)}
    for name, (which, lim) in limits.items():
        g.check_limit(which, lim)
        st, _, _ = _estimate(g)
        stp, _, _ = _estimate(g, plain=True)
        g.check_limit(which, -1)
        st_after, grad1, cnt1 = _estimate(g)
        # counts are integers (bit-exact); the float sums differ only by the order of the atomics
        out[name] = {"status": st, "plain_status": stp, "status_after_restore": st_after,
                     "counts_same_after_restore": bool(np.array_equal(cnt1, cnt0)),
                     "sums_rel_diff_after_restore": float(np.linalg.norm(grad1 - grad0) / np.linalg.norm(grad0))}
    try:
        g.check_limit(sge.LIMIT_PARAMS, n_params + 1)
        out["limit_above_true_size"] = "accepted"
    except sge.SGEError as e:
        out["limit_above_true_size"] = e.code

    # a real out-of-range vertex index, not validated: every kernel reads it as vertex 0
    bad = synth.with_params(sc, sc.positions, [t.data for t in sc.textures])
    bad.pos_idx = sc.pos_idx.copy()
    bad.pos_idx[5, 1] = sc.positions.shape[0] + 7
    gb = sge.Scene.from_arrays(bad, targets=tg)
    out["bad_index_estimate"] = _estimate(gb)[0]
    out["bad_index_plain"] = _estimate(gb, plain=True)[0]
    gb.render_idb(0)
    torch.cuda.synchronize()
    out["bad_index_render"] = gb.status()
    keys = torch.empty((bad.height, bad.width), dtype=torch.int64, device=gb.device)
    uv = torch.empty((bad.height, bad.width, 2), dtype=torch.float32, device=gb.device)
    rgb = torch.empty((bad.height, bad.width, 3), dtype=torch.float32, device=gb.device)
    status = torch.full((1,), -1, dtype=torch.int32, device=gb.device)
    rc = sge._abi.load().sge_render_idb_static(ctypes.byref(gb._desc), 0, 5, 1, 0, 0, keys.data_ptr(),
                                               uv.data_ptr(), rgb.data_ptr(), status.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out["bad_index_static"] = [rc, int(status.item())]
    out["bad_index_validate"] = gb.validate()

    # transparent scenes (the deep estimator) check their sign-plane words and credits too
    tsc = synth.config_transparent(n_views=2, pairs=2, render=64, tex=64, n_lon=16, n_lat=16)
    ttg = oracle.render_targets(tsc, synth.target_scene(tsc))
    gt = sge.Scene.from_arrays(tsc, targets=ttg)
    gt.check_limit(sge.LIMIT_SIGN_WORDS, 3)
    out["transparent_sign_words"] = _estimate(gt, views=(0, 1), pairs=2)[0]
    gt.check_limit(sge.LIMIT_SIGN_WORDS, -1)
    gt.check_limit(sge.LIMIT_PARAMS, 100)
    out["transparent_params"] = _estimate(gt, views=(0, 1), pairs=2)[0]
    gt.check_limit(sge.LIMIT_PARAMS, -1)
    out["transparent_clean"] = _estimate(gt, views=(0, 1), pairs=2)[0]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
