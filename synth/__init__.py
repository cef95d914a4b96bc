"""Seeded synthetic inputs: meshes, textures, cameras and whole scene configurations.

This module is the one piece shared by the CPU oracle's tests, the GPU tests and
the benchmark.  It holds none of the method's arithmetic (no projection,
rasterisation, shading, perturbation or estimation): it only builds the arrays a
caller hands to either side, every one of them from an explicit seed.

The workloads stand in for the paper's assets (the teaser's displaced,
normal-mapped subdivision surface and the Table 2 cow/skull meshes, whose
files and target images are not available): UV spheres with welded positions,
smooth random textures, and cameras on a sphere of radius 3 looking at the origin.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Texture roles (what the shading model reads a texture as).
ROLE_ALBEDO = 0
ROLE_NORMAL = 1
ROLE_ROUGHNESS = 2
ROLE_METALLIC = 3

# Shading models.
SHADE_UNLIT = 0
SHADE_LAMBERT = 1
SHADE_GGX = 2
SHADE_TRANSPARENT = 3  # unlit RGBA fragments composited front to back (deep ID buffer)


# --------------------------------------------------------------------------- meshes
@dataclasses.dataclass
class Mesh:
    positions: np.ndarray  # [V,3] float32, welded (one entry per distinct 3D point)
    pos_idx: np.ndarray    # [T,3] int32 into positions
    uvs: np.ndarray        # [Vt,2] float32
    uv_idx: np.ndarray     # [T,3] int32 into uvs

    @property
    def n_triangles(self) -> int:
        return int(self.pos_idx.shape[0])


def uv_sphere(n_lon: int, n_lat: int, radius: float = 1.0) -> Mesh:
    """Latitude/longitude sphere: n_lon x n_lat quads, two triangles each.

    Positions are welded: the two poles are single vertices and the u seam
    shares its column, so a perturbed position can never open a crack.  UVs
    live on their own (n_lon+1) x (n_lat+1) grid.  The quads touching a pole
    yield one zero-area triangle each (two corners are the pole).  Winding is
    counter-clockwise seen from outside.  The seam (u=0/1) faces -z, so a
    camera on +z sees the middle of the texture.
    """
    pole_n = 0
    pole_s = 1 + (n_lat - 1) * n_lon
    pos = np.zeros((pole_s + 1, 3), dtype=np.float64)
    pos[pole_n] = (0.0, radius, 0.0)
    pos[pole_s] = (0.0, -radius, 0.0)
    jj, ii = np.meshgrid(np.arange(1, n_lat), np.arange(n_lon), indexing="ij")
    phi = math.pi * jj / n_lat
    lam = 2.0 * math.pi * ii / n_lon - math.pi
    ring = np.stack([radius * np.sin(phi) * np.sin(lam), radius * np.cos(phi),
                     radius * np.sin(phi) * np.cos(lam)], axis=-1)
    pos[1:pole_s] = ring.reshape(-1, 3)

    jg, ig = np.meshgrid(np.arange(n_lat + 1), np.arange(n_lon + 1), indexing="ij")
    uvs = np.stack([ig / n_lon, jg / n_lat], axis=-1).reshape(-1, 2)

    def pid(i, j):
        inner = 1 + (j - 1) * n_lon + (i % n_lon)
        return np.where(j == 0, pole_n, np.where(j == n_lat, pole_s, inner))

    def tid(i, j):
        return j * (n_lon + 1) + i

    j, i = np.meshgrid(np.arange(n_lat), np.arange(n_lon), indexing="ij")
    i, j = i.ravel(), j.ravel()
    a, b, c, d = (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)
    # two triangles per quad, (a, c, b) then (b, c, d), interleaved quad by quad
    p1 = np.stack([pid(*a), pid(*c), pid(*b)], axis=-1)
    p2 = np.stack([pid(*b), pid(*c), pid(*d)], axis=-1)
    t1 = np.stack([tid(*a), tid(*c), tid(*b)], axis=-1)
    t2 = np.stack([tid(*b), tid(*c), tid(*d)], axis=-1)
    pidx = np.stack([p1, p2], axis=1).reshape(-1, 3)
    tidx = np.stack([t1, t2], axis=1).reshape(-1, 3)
    return Mesh(pos.astype(np.float32), pidx.astype(np.int32),
                uvs.astype(np.float32), tidx.astype(np.int32))


def subdivide_linear(mesh: Mesh, levels: int = 1) -> Mesh:
    """Midpoint (linear) subdivision, 1 triangle -> 4 per level, welded midpoints."""
    pos = mesh.positions.astype(np.float64)
    uvs = mesh.uvs.astype(np.float64)
    pidx, tidx = mesh.pos_idx, mesh.uv_idx
    for _ in range(levels):
        pos_list, uv_list = list(pos), list(uvs)
        pmid, tmid = {}, {}

        def mid(cache, store, a, b):
            if a == b:
                return a
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                cache[key] = len(store)
                store.append(0.5 * (store[a] + store[b]))
            return cache[key]

        npi, nti = [], []
        for (p0, p1, p2), (t0, t1, t2) in zip(pidx.tolist(), tidx.tolist()):
            m01, m12, m20 = (mid(pmid, pos_list, p0, p1), mid(pmid, pos_list, p1, p2),
                             mid(pmid, pos_list, p2, p0))
            n01, n12, n20 = (mid(tmid, uv_list, t0, t1), mid(tmid, uv_list, t1, t2),
                             mid(tmid, uv_list, t2, t0))
            npi += [[p0, m01, m20], [m01, p1, m12], [m20, m12, p2], [m01, m12, m20]]
            nti += [[t0, n01, n20], [n01, t1, n12], [n20, n12, t2], [n01, n12, n20]]
        pos, uvs = np.asarray(pos_list), np.asarray(uv_list)
        pidx, tidx = np.asarray(npi, np.int32), np.asarray(nti, np.int32)
    return Mesh(pos.astype(np.float32), pidx, uvs.astype(np.float32), tidx)


def linear_refine_matrix(mesh: Mesh, levels: int = 1):
    """Refine matrix of subdivide_linear(mesh, levels): a scipy CSR matrix R (fine vertices x
    control vertices) with the fine positions = R @ mesh.positions; a midpoint row is half of
    each end of its edge, in the order subdivide_linear creates them."""
    import scipy.sparse as sp
    R = sp.identity(len(mesh.positions), format="csr", dtype=np.float64)
    pidx = mesh.pos_idx
    for _ in range(levels):
        n = R.shape[0]
        ends, cache, npi = [], {}, []

        def mid(a, b):
            if a == b:
                return a
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                cache[key] = n + len(ends)
                ends.append((a, b))
            return cache[key]

        for p0, p1, p2 in pidx.tolist():
            m01, m12, m20 = mid(p0, p1), mid(p1, p2), mid(p2, p0)
            npi += [[p0, m01, m20], [m01, p1, m12], [m20, m12, p2], [m01, m12, m20]]
        k = len(ends)
        cols = np.asarray(ends, np.int64).ravel()
        M = sp.csr_matrix((np.full(2 * k, 0.5), (np.repeat(np.arange(k), 2), cols)), shape=(k, n))
        R = sp.vstack([R, M @ R]).tocsr()
        pidx = np.asarray(npi, np.int32)
    R.sort_indices()
    return R


def catmull_clark_faces(n_vertices: int, faces, levels: int = 1):
    """Catmull-Clark subdivision (Catmull & Clark 1978) of a closed polygon mesh, as a matrix.

    faces: polygons (sequences of vertex indices, counter-clockwise seen from outside); every
    edge must be shared by exactly two faces.  Returns (R, quads): R is a scipy CSR matrix
    (fine vertices x control vertices) with the subdivided positions = R @ control positions,
    and quads the subdivided faces, [F, 4] int32.  Each level maps
      face point   = mean of the face's corners,
      edge point   = (both ends + the two adjacent face points) / 4,
      vertex point = (Q + 2 M + (n - 3) P) / n,
    with n the vertex's valence, Q the mean of its adjacent face points and M the mean of its
    incident edges' midpoints.  Fine vertices are numbered vertex points, then edge points (in
    order of first appearance), then face points; each face of k corners becomes k quads
    (corner, edge point, face point, edge point)."""
    import scipy.sparse as sp
    R = sp.identity(n_vertices, format="csr", dtype=np.float64)
    faces = [tuple(int(v) for v in f) for f in faces]
    for _ in range(levels):
        n = R.shape[0]
        edge_id, edge_ends, edge_faces = {}, [], []
        for fi, f in enumerate(faces):
            k = len(f)
            for c in range(k):
                a, b = f[c], f[(c + 1) % k]
                key = (a, b) if a < b else (b, a)
                if key not in edge_id:
                    edge_id[key] = len(edge_ends)
                    edge_ends.append(key)
                    edge_faces.append([])
                edge_faces[edge_id[key]].append(fi)
        if any(len(fs) != 2 for fs in edge_faces):
            raise ValueError("Catmull-Clark subdivision here takes closed manifold meshes only")
        ne, nf = len(edge_ends), len(faces)
        rows, cols, vals = [], [], []

        def put(r, c, w):
            rows.append(r)
            cols.append(c)
            vals.append(w)

        # face points: rows n + ne + fi
        for fi, f in enumerate(faces):
            for v in f:
                put(n + ne + fi, v, 1.0 / len(f))

        def put_face_point(r, fi, w):
            f = faces[fi]
            for v in f:
                put(r, v, w / len(f))

        # edge points
        for e, (a, b) in enumerate(edge_ends):
            put(n + e, a, 0.25)
            put(n + e, b, 0.25)
            for fi in edge_faces[e]:
                put_face_point(n + e, fi, 0.25)
        # vertex points: Q / n + 2 M / n + (n - 3) / n P, with M = mean of (P + other end) / 2
        inc_edges = [[] for _ in range(n)]
        for e, (a, b) in enumerate(edge_ends):
            inc_edges[a].append(e)
            inc_edges[b].append(e)
        inc_faces = [[] for _ in range(n)]
        for fi, f in enumerate(faces):
            for v in f:
                inc_faces[v].append(fi)
        for v in range(n):
            val = len(inc_edges[v])
            if val == 0:
                put(v, v, 1.0)  # a vertex no face uses stays where it is
                continue
            for fi in inc_faces[v]:
                put_face_point(v, fi, 1.0 / (len(inc_faces[v]) * val))
            for e in inc_edges[v]:
                a, b = edge_ends[e]
                put(v, a, 1.0 / (val * val))
                put(v, b, 1.0 / (val * val))
            put(v, v, (val - 3.0) / val)
        M = sp.csr_matrix((vals, (rows, cols)), shape=(n + ne + nf, n))  # duplicates are summed
        R = (M @ R).tocsr()
        quads = []
        for fi, f in enumerate(faces):
            k = len(f)
            for c in range(k):
                a, b, p = f[c], f[(c + 1) % k], f[c - 1]
                e_next = edge_id[(a, b) if a < b else (b, a)]
                e_prev = edge_id[(p, a) if p < a else (a, p)]
                quads.append((a, n + e_next, n + ne + fi, n + e_prev))
        faces = quads
    R.sum_duplicates()
    R.sort_indices()
    return R, np.asarray(faces, np.int32).reshape(-1, 4)


def subdivide_catmull_clark(mesh: Mesh, levels: int = 1):
    """Catmull-Clark subdivision of a closed triangle mesh (zero-area triangles, such as a UV
    sphere's pole slivers, are dropped from the control mesh first), returned as a triangle mesh
    and its refine matrix: (fine Mesh, R) with fine.positions = R @ mesh.positions (rounded to
    float32).  Each fine quad (a, b, c, d) is split into (a, b, c) and (a, c, d).  UVs are
    subdivided linearly per face (face point UV = mean of the face's corner UVs, edge point UV
    = midpoint of the edge's UVs on that face), so texture seams stay seams."""
    keep = ((mesh.pos_idx[:, 0] != mesh.pos_idx[:, 1]) & (mesh.pos_idx[:, 1] != mesh.pos_idx[:, 2])
            & (mesh.pos_idx[:, 2] != mesh.pos_idx[:, 0]))
    faces = mesh.pos_idx[keep].tolist()
    uv_faces = mesh.uv_idx[keep].tolist()
    R, quads = catmull_clark_faces(len(mesh.positions), faces, levels)
    # the same face order and corner order as catmull_clark_faces, on the UV indices
    uvs = [tuple(u) for u in mesh.uvs.astype(np.float64)]
    for _ in range(levels):
        mids, new_faces = {}, []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mids:
                mids[key] = len(uvs)
                uvs.append(tuple(0.5 * (np.asarray(uvs[a]) + np.asarray(uvs[b]))))
            return mids[key]

        for f in uv_faces:
            k = len(f)
            centre = len(uvs)
            uvs.append(tuple(np.mean([uvs[t] for t in f], axis=0)))
            for c in range(k):
                a, b, p = f[c], f[(c + 1) % k], f[c - 1]
                new_faces.append((a, mid(a, b), centre, mid(p, a)))
        uv_faces = new_faces
    uq = np.asarray(uv_faces, np.int32).reshape(-1, 4)
    tri = lambda q: np.stack([q[:, [0, 1, 2]], q[:, [0, 2, 3]]], axis=1).reshape(-1, 3)
    pos = (R @ mesh.positions.astype(np.float64)).astype(np.float32)
    fine = Mesh(pos, tri(quads).astype(np.int32), np.asarray(uvs, np.float32), tri(uq).astype(np.int32))
    return fine, R


def radial_displace(positions: np.ndarray, seed: int, amplitude: float = 0.05,
                    n_terms: int = 4) -> np.ndarray:
    """Seeded low-frequency radial displacement: p <- p * (1 + a * g(p)), |g| <= 1."""
    rng = np.random.default_rng(seed)
    p = positions.astype(np.float64)
    g = np.zeros(p.shape[0])
    for _ in range(n_terms):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        f = rng.uniform(1.0, 3.0)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        g += np.sin(f * (p @ d) + ph) / n_terms
    return (p * (1.0 + amplitude * g)[:, None]).astype(np.float32)


def gaussian_displace(positions: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (positions.astype(np.float64)
            + rng.normal(scale=sigma, size=positions.shape)).astype(np.float32)


# --------------------------------------------------------------------------- textures
def sinusoid_texture(width: int, height: int, channels: int, seed: int,
                     n_terms: int = 8) -> np.ndarray:
    """Smooth random texture in [0,1]: 0.5 + 0.5 * mean of n_terms scaled sinusoids.

    Horizontal frequencies are integers so the texture is periodic in u (the
    sampler wraps u).
    """
    rng = np.random.default_rng(seed)
    x = (np.arange(width) + 0.5) / width
    y = (np.arange(height) + 0.5) / height
    out = np.zeros((height, width, channels))
    for c in range(channels):
        acc = np.zeros((height, width))
        for _ in range(n_terms):
            fx = rng.integers(1, 7)
            fy = rng.uniform(0.5, 6.0)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            a = rng.uniform(0.5, 1.0)
            acc += a * np.sin(2.0 * math.pi * (fx * x[None, :] + fy * y[:, None]) + ph)
        out[..., c] = 0.5 + 0.5 * acc / n_terms
    return out.astype(np.float32)


def constant_texture(width: int, height: int, channels: int, value: float) -> np.ndarray:
    return np.full((height, width, channels), value, dtype=np.float32)


def normal_map_texture(width: int, height: int, seed: int, strength: float = 0.3) -> np.ndarray:
    """Tangent-space normal map stored as 0.5 + 0.5 * n, n = normalize(gx, gy, 1)."""
    g = sinusoid_texture(width, height, 2, seed, n_terms=6).astype(np.float64)
    gx = strength * (2.0 * g[..., 0] - 1.0)
    gy = strength * (2.0 * g[..., 1] - 1.0)
    n = np.stack([gx, gy, np.ones_like(gx)], axis=-1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return (0.5 + 0.5 * n).astype(np.float32)


def flat_normal_texture(width: int, height: int) -> np.ndarray:
    out = np.empty((height, width, 3), np.float32)
    out[...] = (0.5, 0.5, 1.0)
    return out


# --------------------------------------------------------------------------- cameras
def look_at(eye, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0])
    if abs(f @ up) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def perspective(fov_y_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    """Projection with depth z/w in [0,1] between the near and far planes and w = -z_view."""
    fy = 1.0 / math.tan(math.radians(fov_y_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0] = fy / aspect
    p[1, 1] = fy
    p[2, 2] = far / (near - far)
    p[2, 3] = near * far / (near - far)
    p[3, 2] = -1.0
    return p


def mvp_matrix(eye, width: int, height: int, fov_y_deg: float = 45.0,
               near: float = 0.1, far: float = 10.0) -> np.ndarray:
    return (perspective(fov_y_deg, width / height, near, far) @ look_at(eye)).astype(np.float32)


def random_eyes(n: int, seed: int, radius: float = 3.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (radius * d).astype(np.float32)


# --------------------------------------------------------------------------- scenes
@dataclasses.dataclass
class Texture:
    data: np.ndarray   # [H,W,C] float32
    eps: float
    role: int


@dataclasses.dataclass
class Scene:
    """Everything one side of the comparison needs; plain numpy arrays."""
    name: str
    positions: np.ndarray
    pos_idx: np.ndarray
    uvs: np.ndarray
    uv_idx: np.ndarray
    textures: List[Texture]
    eps_pos: float
    mvp: np.ndarray          # [n_views,4,4] float32, row-major, column-vector convention
    cam_pos: np.ndarray      # [n_views,3] float32
    width: int
    height: int
    near: float = 0.1
    shading: int = SHADE_UNLIT
    light_dir: tuple = (0.0, 0.0, 1.0)
    light_rgb: tuple = (1.0, 1.0, 1.0)
    ambient: float = 0.0
    background: tuple = (0.0, 0.0, 0.0)
    # target parameters (the image to match is rendered from these)
    target_positions: Optional[np.ndarray] = None
    target_textures: Optional[List[np.ndarray]] = None
    pairs_per_view: int = 1

    @property
    def n_views(self) -> int:
        return int(self.mvp.shape[0])

    @property
    def n_pos_params(self) -> int:
        return int(self.positions.size)

    @property
    def n_params(self) -> int:
        return self.n_pos_params + sum(int(t.data.size) for t in self.textures)

    def param_offsets(self) -> List[int]:
        """Start of each group in the flat parameter vector: positions, then textures."""
        offs, o = [0], self.n_pos_params
        for t in self.textures:
            offs.append(o)
            o += int(t.data.size)
        return offs


def _views(eyes: np.ndarray, w: int, h: int):
    mvp = np.stack([mvp_matrix(e, w, h) for e in eyes]).astype(np.float32)
    return mvp, eyes.astype(np.float32)


def sphere_scene(name: str, n_lon: int, n_lat: int, tex_size: int, render: int,
                 eyes: np.ndarray, seed_asset: int = 0, seed_target: int = 1,
                 pairs_per_view: int = 1) -> Scene:
    """Unlit textured UV sphere: the first two workload configurations.

    Initial state: the undisplaced sphere with a 0.5 gray RGB texture.  Target:
    the sphere with Gaussian vertex noise (sigma 0.02) and a smooth random texture.
    """
    mesh = uv_sphere(n_lon, n_lat)
    del seed_asset  # the sphere itself is deterministic
    tex0 = constant_texture(tex_size, tex_size, 3, 0.5)
    tgt_pos = gaussian_displace(mesh.positions, 0.02, seed_target)
    tgt_tex = sinusoid_texture(tex_size, tex_size, 3, seed_target)
    mvp, cam = _views(eyes, render, render)
    return Scene(name, mesh.positions, mesh.pos_idx, mesh.uvs, mesh.uv_idx,
                 [Texture(tex0, 1.0 / 255.0, ROLE_ALBEDO)], 1e-3, mvp, cam, render, render,
                 target_positions=tgt_pos, target_textures=[tgt_tex],
                 pairs_per_view=pairs_per_view)


def config_plain(render: int = 256) -> Scene:
    """UV sphere 32x32 (2,048 triangles), 256^2 RGB texture, 256^2 render, camera (0,0,3)."""
    return sphere_scene("sphere2k_tex256_r256", 32, 32, 256, render,
                        np.array([[0.0, 0.0, 3.0]], np.float32))


def config_batched(n_views: int = 8, pairs: int = 64, render: int = 512) -> Scene:
    """UV sphere 64x64 (8,192 triangles), 512^2 RGB texture, 512^2 render, 8 views x 64 pairs."""
    return sphere_scene("sphere8k_tex512_r512", 64, 64, 512, render,
                        random_eyes(n_views, seed=2), pairs_per_view=pairs)


def config_autograd(n_views: int = 16, pairs: int = 16, render: int = 1024,
                    tex: int = 1024) -> Scene:
    """2,048-triangle control sphere, 2x linear subdivision (32,768 triangles), displaced;
    RGBA albedo + tangent-space normal map; Lambert with one directional light."""
    mesh = subdivide_linear(uv_sphere(32, 32), 2)
    pos0 = radial_displace(mesh.positions, seed=0, amplitude=0.05)
    tgt_pos = radial_displace(mesh.positions, seed=1, amplitude=0.08)
    alb0 = constant_texture(tex, tex, 4, 0.5)
    nrm0 = flat_normal_texture(tex, tex)
    tgt_alb = sinusoid_texture(tex, tex, 4, seed=1)
    tgt_nrm = normal_map_texture(tex, tex, seed=1)
    mvp, cam = _views(random_eyes(n_views, seed=2), render, render)
    ld = np.array([0.3, 0.6, 0.74])
    ld /= np.linalg.norm(ld)
    return Scene("subdiv32k_rgba1024_nrm1024_r1024", pos0, mesh.pos_idx, mesh.uvs, mesh.uv_idx,
                 [Texture(alb0, 1.0 / 255.0, ROLE_ALBEDO), Texture(nrm0, 1.0 / 255.0, ROLE_NORMAL)],
                 1e-3, mvp, cam, render, render, shading=SHADE_LAMBERT,
                 light_dir=tuple(float(x) for x in ld), ambient=0.1,
                 target_positions=tgt_pos, target_textures=[tgt_alb, tgt_nrm],
                 pairs_per_view=pairs)


def config_control(n_views: int = 16, pairs: int = 16, render: int = 1024, tex: int = 1024):
    """The autograd configuration as the paper's teaser builds it (Section 6.3): a 2,048-triangle
    control sphere (1,984 after its pole slivers are dropped) under two Catmull-Clark levels
    (47,616 triangles), the control vertices displaced; RGBA albedo + tangent-space normal map;
    Lambert with one directional light.  Returns (scene, control Mesh, R, target control
    positions), the scene's positions R @ the control positions."""
    ctl = uv_sphere(32, 32)
    fine, R = subdivide_catmull_clark(ctl, 2)
    ctl0 = radial_displace(ctl.positions, seed=0, amplitude=0.05)
    tgt_ctl = radial_displace(ctl.positions, seed=1, amplitude=0.08)
    lift = lambda p: (R @ p.astype(np.float64)).astype(np.float32)
    base = config_autograd(n_views, pairs, render, tex)
    sc = dataclasses.replace(base, name=f"catmullclark48k_rgba{tex}_nrm{tex}_r{render}", positions=lift(ctl0),
                             pos_idx=fine.pos_idx, uvs=fine.uvs, uv_idx=fine.uv_idx,
                             target_positions=lift(tgt_ctl))
    return sc, dataclasses.replace(ctl, positions=ctl0), R, tgt_ctl


def merge_meshes(meshes: List[Mesh], offsets) -> Mesh:
    """One mesh from several, mesh k translated by offsets[k]; indices renumbered."""
    pos, pidx, uvs, tidx = [], [], [], []
    nv = nt = 0
    for m, off in zip(meshes, offsets):
        pos.append(m.positions + np.asarray(off, np.float32))
        pidx.append(m.pos_idx + nv)
        uvs.append(m.uvs)
        tidx.append(m.uv_idx + nt)
        nv += len(m.positions)
        nt += len(m.uvs)
    return Mesh(np.concatenate(pos).astype(np.float32), np.concatenate(pidx).astype(np.int32),
                np.concatenate(uvs).astype(np.float32), np.concatenate(tidx).astype(np.int32))


def rgba_texture(width: int, height: int, seed: int, alpha_lo: float = 0.25, alpha_hi: float = 0.75) -> np.ndarray:
    """Smooth random RGBA texture: sinusoid colours, opacity remapped into [alpha_lo, alpha_hi]."""
    t = sinusoid_texture(width, height, 4, seed)
    t[..., 3] = alpha_lo + (alpha_hi - alpha_lo) * t[..., 3]
    return t.astype(np.float32)


def config_transparent(n_views: int = 8, pairs: int = 16, render: int = 512, tex: int = 512,
                       n_lon: int = 32, n_lat: int = 32) -> Scene:
    """Transparent geometry (Section 4.4): three overlapping semi-transparent UV spheres
    (radius 0.6, 3 x 2,048 triangles) in a row, so a pixel sees up to six fragments (each
    sphere's front and back), more than the deep ID buffer keeps; one RGBA albedo (opacity in
    [0.25, 0.75]), composited front to back over a gray background.  Target: Gaussian vertex
    noise (sigma 0.02) and another RGBA texture."""
    sph = uv_sphere(n_lon, n_lat, radius=0.6)
    mesh = merge_meshes([sph, sph, sph], [(-0.45, 0.0, -0.3), (0.0, 0.05, 0.0), (0.45, -0.05, 0.3)])
    tgt_pos = gaussian_displace(mesh.positions, 0.02, 1)
    mvp, cam = _views(random_eyes(n_views, seed=2), render, render)
    return Scene(f"transparent3x{2 * n_lon * n_lat // 1000}k_rgba{tex}_r{render}", mesh.positions, mesh.pos_idx,
                 mesh.uvs, mesh.uv_idx, [Texture(rgba_texture(tex, tex, seed=0), 1.0 / 255.0, ROLE_ALBEDO)],
                 1e-3, mvp, cam, render, render, shading=SHADE_TRANSPARENT, background=(0.3, 0.3, 0.3),
                 target_positions=tgt_pos, target_textures=[rgba_texture(tex, tex, seed=1)],
                 pairs_per_view=pairs)


def triangle_soup(n: int, render: int = 512, seed: int = 0):
    """Section 6.1's experiment: n independent triangles with 12 parameters each (three vertices,
    one RGB colour) fitted to an image.  Identity camera (clip = world: x, y in [-1, 1] span the
    image, z in (0, 1) orders the triangles).  Colour i is texel i of an n x 1 RGB texture, named
    by the triangle's three UVs (the texel's centre).  Initial state: triangles of circumradius
    3 / sqrt(n) world units at uniform positions and orientations (the soup covers the image
    about three times over), colours uniform in [0.25, 0.75]; eps_pos is one pixel, the colour
    eps 2/255.  Returns (scene, target image [1, render, render, 3]): a smooth random image."""
    rng = np.random.default_rng(seed)
    c = np.concatenate([rng.uniform(-1.0, 1.0, size=(n, 2)), rng.uniform(0.2, 0.8, size=(n, 1))], axis=1)
    R = 3.0 / math.sqrt(n)
    ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 1)) + np.array([0.0, 2.0, 4.0]) * math.pi / 3.0
    pos = np.repeat(c[:, None, :], 3, axis=1)
    pos[..., 0] += R * np.cos(ang)
    pos[..., 1] += R * np.sin(ang)
    pidx = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    uv = np.stack([np.repeat((np.arange(n) + 0.5) / n, 3), np.full(3 * n, 0.5)], axis=1)
    tex = rng.uniform(0.25, 0.75, size=(1, n, 3)).astype(np.float32)
    target = sinusoid_texture(render, render, 3, seed + 1)[None]
    sc = Scene(f"soup{n}_r{render}", pos.reshape(-1, 3).astype(np.float32), pidx, uv.astype(np.float32),
               pidx.copy(), [Texture(tex, 2.0 / 255.0, ROLE_ALBEDO)], 2.0 / render,
               np.eye(4, dtype=np.float32)[None], np.array([[0.0, 0.0, 3.0]], np.float32), render, render)
    return sc, target.astype(np.float32)


def config_uneven(n_assets: int = 32, n_views: int = 4, pairs: int = 8, render: int = 512,
                  tri_lo: int = 1000, tri_hi: int = 200_000,
                  tex_choices=(256, 512, 1024, 2048)) -> List[Scene]:
    """Assets with triangle counts log-uniform in [tri_lo, tri_hi] and square RGB textures."""
    return [uneven_asset(k, n_views, pairs, render, tri_lo, tri_hi, tex_choices) for k in range(n_assets)]


def uneven_asset(k: int, n_views: int = 4, pairs: int = 8, render: int = 512, tri_lo: int = 1000,
                 tri_hi: int = 200_000, tex_choices=(256, 512, 1024, 2048)) -> Scene:
    """Asset k of config_uneven (each asset has its own seeds, so it can be made alone)."""
    rng = np.random.default_rng(100 + k)
    t = math.exp(rng.uniform(math.log(tri_lo), math.log(tri_hi)))
    n_lat = max(2, int(round(math.sqrt(t / 4.0))))
    tex = int(rng.choice(tex_choices))
    return sphere_scene(f"asset{k}_lat{n_lat}_tex{tex}", 2 * n_lat, n_lat, tex, render,
                        random_eyes(n_views, seed=1000 + k), seed_target=100 + k, pairs_per_view=pairs)


def config_scale(n_views: int = 16, pairs: int = 16, render: int = 2048, tex: int = 2048,
                 n_lon: int = 1024, n_lat: int = 512) -> Scene:
    """1,048,576-triangle displaced grid sphere, four 2048^2 RGB maps, GGX with one light."""
    mesh = uv_sphere(n_lon, n_lat)
    pos0 = radial_displace(mesh.positions, seed=0, amplitude=0.03)
    tgt_pos = radial_displace(mesh.positions, seed=1, amplitude=0.05)
    texs = [Texture(constant_texture(tex, tex, 3, 0.5), 1.0 / 255.0, ROLE_ALBEDO),
            Texture(constant_texture(tex, tex, 3, 0.5), 1.0 / 255.0, ROLE_ROUGHNESS),
            Texture(constant_texture(tex, tex, 3, 0.0), 1.0 / 255.0, ROLE_METALLIC),
            Texture(flat_normal_texture(tex, tex), 1.0 / 255.0, ROLE_NORMAL)]
    tgt = [sinusoid_texture(tex, tex, 3, seed=1),
           0.2 + 0.7 * sinusoid_texture(tex, tex, 3, seed=2),
           sinusoid_texture(tex, tex, 3, seed=3),
           normal_map_texture(tex, tex, seed=4)]
    mvp, cam = _views(random_eyes(n_views, seed=2), render, render)
    ld = np.array([0.3, 0.6, 0.74])
    ld /= np.linalg.norm(ld)
    return Scene("gridsphere1m_4x2048_r2048", pos0, mesh.pos_idx, mesh.uvs, mesh.uv_idx, texs,
                 1e-3, mvp, cam, render, render, shading=SHADE_GGX,
                 light_dir=tuple(float(x) for x in ld), light_rgb=(3.0, 3.0, 3.0), ambient=0.05,
                 target_positions=tgt_pos, target_textures=[t.astype(np.float32) for t in tgt],
                 pairs_per_view=pairs)


def with_params(scene: Scene, positions: np.ndarray, textures: List[np.ndarray]) -> Scene:
    """Copy of `scene` whose parameter arrays are replaced (e.g. by the target's)."""
    texs = [Texture(np.ascontiguousarray(d, np.float32), t.eps, t.role)
            for d, t in zip(textures, scene.textures)]
    return dataclasses.replace(scene, positions=np.ascontiguousarray(positions, np.float32),
                               textures=texs)


def target_scene(scene: Scene) -> Scene:
    return with_params(scene, scene.target_positions, scene.target_textures)
