"""Tiny hand-built scenes for the oracle pins and the GPU edge cases.

With the identity camera matrix, clip = (x, y, z, 1), so a vertex at screen
pixel coordinate (sx, sy) of a W x H image has x = 2 sx / W - 1 and
y = 1 - 2 sy / H; with W, H powers of two and sx, sy multiples of 1/256 these
are exact in float32 and land exactly on the rasterizer's fixed-point grid.
"""
import numpy as np

import synth


def to_world(sx, sy, W, H):
    return 2.0 * np.asarray(sx, np.float64) / W - 1.0, 1.0 - 2.0 * np.asarray(sy, np.float64) / H


def flat_scene(screen_tris, W, H, z=0.5, uv_tris=None, textures=None, eps_pos=0.0,
               shading=synth.SHADE_UNLIT, light_dir=(0.0, 0.0, 1.0), ambient=0.0,
               cam_pos=(0.0, 0.0, 3.0), mvp=None, background=(0.0, 0.0, 0.0)):
    """Triangle soup given in screen pixels: screen_tris [T,3,2] (or [T,3,3] with depth)."""
    st = np.asarray(screen_tris, np.float64)
    T = st.shape[0]
    pos = np.zeros((T * 3, 3))
    x, y = to_world(st[..., 0], st[..., 1], W, H)
    pos[:, 0], pos[:, 1] = x.ravel(), y.ravel()
    pos[:, 2] = st[..., 2].ravel() if st.shape[-1] == 3 else z
    pidx = np.arange(T * 3, dtype=np.int32).reshape(T, 3)
    if uv_tris is None:
        uv = np.zeros((T * 3, 2), np.float32)
        uv[:, 0] = (st[..., 0] / W).ravel()
        uv[:, 1] = (st[..., 1] / H).ravel()
    else:
        uv = np.asarray(uv_tris, np.float32).reshape(-1, 2)
    if textures is None:
        textures = [synth.Texture(synth.constant_texture(2, 2, 3, 1.0), 0.0, synth.ROLE_ALBEDO)]
    M = np.eye(4, dtype=np.float32)[None] if mvp is None else np.asarray(mvp, np.float32)[None]
    return synth.Scene("tiny", pos.astype(np.float32), pidx, uv.astype(np.float32), pidx.copy(),
                       textures, eps_pos, M, np.asarray([cam_pos], np.float32), W, H,
                       shading=shading, light_dir=light_dir, ambient=ambient,
                       background=background)


def square_quad(x0, y0, x1, y1, facing_camera=False):
    """Two triangles covering the axis-aligned rectangle, split along (x0,y0)-(x1,y1).

    Screen y grows downwards while world y grows upwards, so the default
    winding has a -z face normal (cross(e1, e2) in world space);
    facing_camera=True reverses it so the face normal is +z.
    """
    tris = [[(x0, y0), (x1, y0), (x1, y1)], [(x0, y0), (x1, y1), (x0, y1)]]
    return [t[::-1] for t in tris] if facing_camera else tris
