"""CPU oracle for per-pixel stochastic gradient estimation (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the library under ``paper_2404_09758_gb300`` never imports it and it
never imports that library.  The arithmetic lives in ``sge_oracle.c`` (plain C,
fp64 accumulation); this file compiles it with gcc and marshals numpy arrays.

Scenes are passed as any object with the attributes of ``synth.Scene``
(positions, pos_idx, uvs, uv_idx, textures[.data/.eps/.role], eps_pos, mvp,
cam_pos, width, height, near, shading, light_dir, light_rgb, ambient,
background); target images are passed separately.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sge_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
MAX_TEX = 8
FOOT_BILINEAR, FOOT_NEAREST = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so float steps round as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int32), ("n_triangles", C.c_int32), ("n_uvs", C.c_int32),
        ("n_textures", C.c_int32),
        ("positions", C.c_void_p), ("pos_idx", C.c_void_p), ("uvs", C.c_void_p),
        ("uv_idx", C.c_void_p),
        ("tex", C.c_void_p * MAX_TEX),
        ("tex_w", C.c_int32 * MAX_TEX), ("tex_h", C.c_int32 * MAX_TEX),
        ("tex_c", C.c_int32 * MAX_TEX), ("tex_role", C.c_int32 * MAX_TEX),
        ("eps_tex", C.c_float * MAX_TEX),
        ("eps_pos", C.c_float),
        ("eps_vec", C.c_void_p),
        ("n_views", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
        ("mvp", C.c_void_p), ("cam_pos", C.c_void_p),
        ("near_w", C.c_float),
        ("targets", C.c_void_p),
        ("background", C.c_float * 3),
        ("shading", C.c_int32),
        ("light_dir", C.c_float * 3), ("light_rgb", C.c_float * 3), ("ambient", C.c_float),
        ("footprint", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, U64, I32, U32, I64 = C.c_void_p, C.c_uint64, C.c_int, C.c_uint32, C.c_int64
            L.or_mix64.restype, L.or_mix64.argtypes = U64, [U64]
            L.or_pair_key.restype, L.or_pair_key.argtypes = U64, [U64, U32, U32, U32]
            L.or_sign.restype, L.or_sign.argtypes = I32, [U64, U64]
            L.or_draw_views.restype, L.or_draw_views.argtypes = I32, [U64, U32, I32, I32, P]
            L.or_n_params.restype, L.or_n_params.argtypes = I64, [P]
            L.oracle_render.restype = I32
            L.oracle_render.argtypes = [P, I32, U64, U32, U32, I32, P, P, P]
            L.oracle_render_deep.restype = I32
            L.oracle_render_deep.argtypes = [P, I32, U64, U32, U32, I32, P, P]
            L.oracle_layers.restype, L.oracle_layers.argtypes = I32, []
            L.oracle_estimate.restype = I32
            L.oracle_estimate.argtypes = [P, U64, U32, P, I32, I32, P, P, P, P, P, P]
            L.oracle_loss.restype, L.oracle_loss.argtypes = C.c_double, [P, I32]
            L.oracle_estimate_full_image.restype = I32
            L.oracle_estimate_full_image.argtypes = [P, U64, U32, P, I32, I32, P, P, P, P, P, P]
            L.oracle_step.restype = None
            L.oracle_step.argtypes = [I32, I64, P, P, P, P, P, I64, C.c_double, C.c_double,
                                      C.c_double, I32, P, P, P, P, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleScene:
    """Marshalled scene: keeps every array it points to alive."""

    def __init__(self, scene, targets=None, eps_vec=None, footprint=FOOT_BILINEAR):
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        s = _Scene()
        pos = arr(scene.positions, np.float32)
        s.n_vertices = pos.shape[0]
        s.positions = _ptr(pos)
        pidx = arr(scene.pos_idx, np.int32)
        s.n_triangles = pidx.shape[0]
        s.pos_idx = _ptr(pidx)
        uvs = arr(scene.uvs, np.float32)
        s.n_uvs = uvs.shape[0]
        s.uvs = _ptr(uvs)
        s.uv_idx = _ptr(arr(scene.uv_idx, np.int32))
        if len(scene.textures) > MAX_TEX:
            raise ValueError("too many textures")
        s.n_textures = len(scene.textures)
        self.tex_shapes = []
        for k, t in enumerate(scene.textures):
            d = arr(t.data, np.float32)
            if d.ndim == 2:
                d = d[..., None]
            s.tex[k] = _ptr(d)
            s.tex_h[k], s.tex_w[k], s.tex_c[k] = d.shape
            s.tex_role[k] = t.role
            s.eps_tex[k] = t.eps
            self.tex_shapes.append(d.shape)
        s.eps_pos = scene.eps_pos
        if eps_vec is not None:
            s.eps_vec = _ptr(arr(eps_vec, np.float32))
        mvp = arr(scene.mvp, np.float32)
        s.n_views = mvp.shape[0]
        s.mvp = _ptr(mvp)
        s.cam_pos = _ptr(arr(scene.cam_pos, np.float32))
        s.width, s.height = scene.width, scene.height
        s.near_w = scene.near
        if targets is None:
            targets = np.zeros((s.n_views, scene.height, scene.width, 3), np.float32)
        s.targets = _ptr(arr(targets, np.float32))
        for c in range(3):
            s.background[c] = scene.background[c]
            s.light_dir[c] = scene.light_dir[c]
            s.light_rgb[c] = scene.light_rgb[c]
        s.shading = scene.shading
        s.ambient = scene.ambient
        s.footprint = footprint
        self.s = s
        self.width, self.height, self.n_views = scene.width, scene.height, s.n_views
        self.n_params = int(lib().or_n_params(C.byref(s)))

    @property
    def ref(self):
        return C.byref(self.s)


# ------------------------------------------------------------------ functions
def mix64(z: int) -> int:
    return int(lib().or_mix64(z & 0xFFFFFFFFFFFFFFFF))


def pair_key(seed: int, it: int, view: int, pair: int) -> int:
    return int(lib().or_pair_key(seed, it, view, pair))


def sign(key: int, i: int) -> int:
    return int(lib().or_sign(key, i))


def draw_views(seed: int, it: int, n_views: int, count: int):
    """The `count` distinct views of iteration `it` (a random view per estimate, Section 5)."""
    out = np.empty(count, np.int32)
    if lib().or_draw_views(seed, it, n_views, count, _ptr(out)):
        raise ValueError("need 1 <= count <= n_views")
    return [int(v) for v in out]


def render(osc: OracleScene, view: int, seed: int = 0, it: int = 0, pair: int = 0, side: int = 0):
    """Depth|ID keys [H,W] uint64, UV [H,W,2] float32, colour [H,W,3] float64."""
    H, W = osc.height, osc.width
    keys = np.empty((H, W), np.uint64)
    uv = np.empty((H, W, 2), np.float32)
    rgb = np.empty((H, W, 3), np.float64)
    rc = lib().oracle_render(osc.ref, view, seed, it, pair, side, _ptr(keys), _ptr(uv), _ptr(rgb))
    if rc:
        raise ValueError(f"oracle_render failed ({rc})")
    return keys, uv, rgb


def render_deep(osc: OracleScene, view: int, seed: int = 0, it: int = 0, pair: int = 0, side: int = 0,
                with_rgb: bool = True):
    """Deep ID buffer [LAYERS,H,W] uint64 (ascending keys, ~0 = empty; Section 4.4, transparent
    geometry) and, for a transparent scene, its front-to-back composite [H,W,3] float64."""
    H, W = osc.height, osc.width
    deep = np.empty((lib().oracle_layers(), H, W), np.uint64)
    rgb = np.empty((H, W, 3), np.float64) if with_rgb else None
    rc = lib().oracle_render_deep(osc.ref, view, seed, it, pair, side, _ptr(deep), _ptr(rgb) if with_rgb else None)
    if rc:
        raise ValueError(f"oracle_render_deep failed ({rc})")
    return deep, rgb


def estimate(osc: OracleScene, seed: int, it: int, view_ids, pairs: int, per_pixel: bool = False):
    """Sums S [d] float64, counts C [d] uint64, loss [n_views] float64 (+ per-pixel arrays)."""
    views = np.ascontiguousarray(view_ids, np.int32)
    S = np.zeros(osc.n_params, np.float64)
    Cn = np.zeros(osc.n_params, np.uint64)
    loss = np.zeros(len(views), np.float64)
    shape = (len(views), pairs, osc.height, osc.width)
    df = np.zeros(shape) if per_pixel else None
    fm = np.zeros(shape) if per_pixel else None
    cd = np.zeros(shape) if per_pixel else None
    rc = lib().oracle_estimate(osc.ref, seed, it, _ptr(views), len(views), pairs, _ptr(S), _ptr(Cn),
                               _ptr(loss), _ptr(df) if per_pixel else None,
                               _ptr(fm) if per_pixel else None, _ptr(cd) if per_pixel else None)
    if rc:
        raise ValueError(f"oracle_estimate failed ({rc})")
    if per_pixel:
        return S, Cn, loss, df, fm, cd
    return S, Cn, loss


def estimate_full_image(osc: OracleScene, seed: int, it: int, view_ids, pairs: int):
    """Eq. 4 with the whole-image error: sums S [d] float64, counts C [d] uint64, and per
    estimate (view-major) dF, sum |f+ - f-|, sum max(f+, f-), sum cond (float64 arrays)."""
    views = np.ascontiguousarray(view_ids, np.int32)
    S = np.zeros(osc.n_params, np.float64)
    Cn = np.zeros(osc.n_params, np.uint64)
    ne = len(views) * pairs
    dF, A, M, K = (np.zeros(ne) for _ in range(4))
    rc = lib().oracle_estimate_full_image(osc.ref, seed, it, _ptr(views), len(views), pairs, _ptr(S), _ptr(Cn),
                                          _ptr(dF), _ptr(A), _ptr(M), _ptr(K))
    if rc:
        raise ValueError(f"oracle_estimate_full_image failed ({rc})")
    return S, Cn, dF, A, M, K


def loss(osc: OracleScene, view: int) -> float:
    return float(lib().oracle_loss(osc.ref, view))


def step(kind: int, theta, S, Cn, eps, lr, n_total: int, t: int = 1, m=None, v=None,
         b1: float = 0.9, b2: float = 0.999, adam_eps: float = 1e-8):
    """One descent step (kind 0 SGD, 1 Adam, 2 SGD on the per-pixel mean); float64 outputs."""
    theta = np.ascontiguousarray(theta, np.float32)
    d = theta.size
    S = np.ascontiguousarray(S, np.float64)
    Cn = np.ascontiguousarray(Cn, np.uint64)
    eps = np.ascontiguousarray(np.broadcast_to(eps, (d,)), np.float32)
    lr = np.ascontiguousarray(np.broadcast_to(lr, (d,)), np.float32)
    m = np.zeros(d, np.float32) if m is None else np.ascontiguousarray(m, np.float32)
    v = np.zeros(d, np.float32) if v is None else np.ascontiguousarray(v, np.float32)
    th_o, m_o, v_o = np.empty(d), np.empty(d), np.empty(d)
    lib().oracle_step(kind, d, _ptr(theta), _ptr(S), _ptr(Cn), _ptr(eps), _ptr(lr), n_total, b1, b2,
                      adam_eps, t, _ptr(m), _ptr(v), _ptr(th_o), _ptr(m_o), _ptr(v_o))
    return th_o, m_o, v_o


def render_targets(scene, target) -> np.ndarray:
    """Target images [n_views,H,W,3] float32: unperturbed renders of the target scene."""
    osc = OracleScene(target)
    out = np.empty((osc.n_views, osc.height, osc.width, 3), np.float32)
    for v in range(osc.n_views):
        out[v] = render(osc, v)[2].astype(np.float32)
    return out
