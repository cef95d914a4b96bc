"""Pins of the subdivision refine matrices the control-mesh form uses (Section 6.3's Catmull-Clark
surfaces): each is checked against results fixed by the mathematics, not against a retyping
of its own rules.

- A cube's first level: vertex points at 5/9 of the corners, edge points at (0, 3/4, 3/4),
  face points at the face centres (the worked cube of the subdivision literature).
- The limit position: repeated levels drive a cube corner to the Catmull-Clark limit mask
  (n^2 P + 4 sum e_j + sum f_j) / (n (n + 5)) of Halstead, Kass and DeRose (1993), which is 1/2
  of the corner for the cube.
- A regular quad grid (a torus: every vertex of valence 4): Catmull-Clark is tensor-product
  cubic B-spline subdivision there, so its vertex, edge and face masks are the outer products
  of the one-dimensional masks (1/8, 3/4, 1/8) and (1/2, 1/2).
- The sphere control mesh: a closed, consistently oriented triangle mesh whose Euler
  characteristic the subdivision keeps; 24 fine triangles per control triangle after two
  levels (the paper's 2K control triangles and 50K surface triangles); affine rows.
"""
import itertools

import numpy as np
import pytest

import synth


def _cube():
    P = np.array(list(itertools.product((-1.0, 1.0), repeat=3)))
    idx = {tuple(p): k for k, p in enumerate(P)}
    faces = []
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            u, v = [a for a in range(3) if a != axis]
            corners = []
            for a, b in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                p = [0.0] * 3
                p[axis], p[u], p[v] = sgn, a, b
                corners.append(idx[tuple(p)])
            # counter-clockwise seen from outside: flip the faces whose (u, v, axis) frame
            # is left-handed
            n = np.cross(P[corners[1]] - P[corners[0]], P[corners[2]] - P[corners[1]])
            if np.dot(n, P[corners].mean(0)) < 0:
                corners = corners[::-1]
            faces.append(corners)
    return P, faces


def test_cube_first_level_points():
    P, faces = _cube()
    R, quads = synth.catmull_clark_faces(len(P), faces, 1)
    assert R.shape == (8 + 12 + 6, 8) and quads.shape == (24, 4)
    X = R @ P
    assert np.allclose(X[:8], P * 5.0 / 9.0, atol=1e-15)
    # edge points: the edge's midpoint pulled to 3/4 along both other axes
    E = X[8:20]
    assert np.allclose(np.sort(np.abs(E), axis=1), np.tile([0.0, 0.75, 0.75], (12, 1)))
    assert len({tuple(np.round(e, 12)) for e in E}) == 12
    F = X[20:]
    assert np.allclose(np.sort(np.abs(F), axis=1), np.tile([0.0, 0.0, 1.0], (6, 1)))
    assert np.allclose(F.sum(0), 0.0)


def test_cube_corner_converges_to_the_limit_mask():
    P, faces = _cube()
    corner = 7  # (1, 1, 1): valence 3, edge neighbours sum to (1,1,1), diagonals to (-1,-1,-1)
    n = 3
    e = [k for k in range(8) if np.abs(P[k] - P[corner]).sum() == 2.0]
    f = [k for k in range(8) if np.abs(P[k] - P[corner]).sum() == 4.0]
    limit = (n * n * P[corner] + 4 * P[e].sum(0) + P[f].sum(0)) / (n * (n + 5))
    assert np.allclose(limit, 0.5)
    errs = []
    for levels in range(1, 6):
        R, _ = synth.catmull_clark_faces(len(P), faces, levels)
        errs.append(np.abs((R @ P)[corner] - limit).max())
    assert errs[-1] < 1e-4
    assert all(b < 0.25 * a for a, b in zip(errs, errs[1:]))  # geometric convergence


def test_regular_grid_masks_are_cubic_bspline_tensor_products():
    m, n = 7, 6  # a torus of m x n quads, every vertex of valence 4
    vid = lambda i, j: (i % m) * n + (j % n)
    faces = [[vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)] for i in range(m) for j in range(n)]
    R, quads = synth.catmull_clark_faces(m * n, faces, 1)
    nv, ne, nf = m * n, 2 * m * n, m * n
    assert R.shape == (nv + ne + nf, nv)
    b3 = {-1: 1 / 8, 0: 3 / 4, 1: 1 / 8}
    b2 = {0: 1 / 2, 1: 1 / 2}
    R = R.toarray()

    def mask(wi, wj, i0, j0):
        want = np.zeros(nv)
        for (di, a), (dj, b) in itertools.product(wi.items(), wj.items()):
            want[vid(i0 + di, j0 + dj)] += a * b
        return want

    for i, j in itertools.product(range(m), range(n)):
        assert np.allclose(R[vid(i, j)], mask(b3, b3, i, j), atol=1e-15)
    # every edge row is one of the two edge masks at one edge, every face row the face mask
    edge_masks = {}
    for i, j in itertools.product(range(m), range(n)):
        edge_masks[tuple(np.round(mask(b2, b3, i, j), 12))] = ("i", i, j)
        edge_masks[tuple(np.round(mask(b3, b2, i, j), 12))] = ("j", i, j)
    seen = {edge_masks[tuple(np.round(R[r], 12))] for r in range(nv, nv + ne)}
    assert len(seen) == ne
    faces_seen = set()
    for r in range(nv + ne, nv + ne + nf):
        hit = [(i, j) for i, j in itertools.product(range(m), range(n))
               if np.allclose(R[r], mask(b2, b2, i, j), atol=1e-15)]
        assert len(hit) == 1
        faces_seen.add(hit[0])
    assert len(faces_seen) == nf


def _closed_oriented(tris):
    directed = {}
    for t in tris.tolist():
        for c in range(3):
            e = (t[c], t[(c + 1) % 3])
            directed[e] = directed.get(e, 0) + 1
    return all(v == 1 for v in directed.values()) and all((b, a) in directed for a, b in directed)


@pytest.mark.parametrize("n_lon,n_lat", [(16, 16), (32, 32)])
def test_sphere_control_mesh(n_lon, n_lat):
    c = synth.uv_sphere(n_lon, n_lat)
    nondeg = int(((c.pos_idx[:, 0] != c.pos_idx[:, 1]) & (c.pos_idx[:, 1] != c.pos_idx[:, 2])
                  & (c.pos_idx[:, 2] != c.pos_idx[:, 0])).sum())
    fine, R = synth.subdivide_catmull_clark(c, 2)
    assert fine.n_triangles == 24 * nondeg
    if (n_lon, n_lat) == (32, 32):
        assert 1900 < nondeg and 45000 < fine.n_triangles < 55000
    assert _closed_oriented(fine.pos_idx)
    V, F = len(fine.positions), fine.n_triangles
    assert V - (3 * F // 2) + F == 2  # genus 0 kept
    assert R.shape == (V, len(c.positions))
    assert (R.data >= 0).all() and np.allclose(np.asarray(R.sum(1)).ravel(), 1.0)
    assert np.abs((R @ c.positions.astype(np.float64)) - fine.positions).max() <= np.finfo(np.float32).eps
    # a smoothing scheme: the fine vertices stay inside the control sphere, and close to it
    r = np.linalg.norm(fine.positions, axis=1)
    assert r.max() <= 1.0 + 1e-6 and r.min() > 0.95
    assert fine.uvs.min() >= 0.0 and fine.uvs.max() <= 1.0
    assert fine.uv_idx.shape == fine.pos_idx.shape and fine.uv_idx.max() < len(fine.uvs)


def test_open_meshes_are_refused():
    with pytest.raises(ValueError):
        synth.catmull_clark_faces(4, [[0, 1, 2], [0, 2, 3]], 1)
