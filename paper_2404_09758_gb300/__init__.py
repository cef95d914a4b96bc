"""Per-pixel stochastic gradient estimation through a plain rasterizer, on GB300.

Python binding of the C ABI in include/sge.h (libsge.so, built from csrc/):
tensors provide device memory and streams, every step of the method runs in
the library's CUDA kernels.  There is no CPU path: the calls raise if the
library or a CUDA device is missing.

    scene = Scene.from_arrays(arrays, targets)      # borrows torch CUDA tensors
    scene.estimate_grad(seed, it, views, pairs, grad, counts)   # Eq. 9 sums
    scene.step(opt, grad, counts, n_total, m, v)                # Adam / SGD, Section 5
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

from . import _abi
from ._abi import (ERR_BIN_OVERFLOW, ERR_BAD_INDEX, ERR_BOUNDS, LIMIT_VERTICES, LIMIT_UVS, LIMIT_BIN_ENTRIES,
                   LIMIT_SIGN_WORDS, LIMIT_PARAMS, FOOT_BILINEAR, FOOT_NEAREST, MAX_LAYERS, MAX_TEXTURES, MAX_VIEWS_PER_CALL, OK,
                   SHADE_GGX, SHADE_LAMBERT, SHADE_TRANSPARENT, SHADE_UNLIT, STEP_ADAM, STEP_SGD, STEP_SGD_MEAN,
                   SGEError)
from ._build import build

__all__ = ["Scene", "Batch", "ControlMesh", "IterState", "save_checkpoint", "load_checkpoint", "draw_views", "refine", "SGEError", "SGEFunction", "sge_loss", "build", "load", "STEP_SGD", "STEP_ADAM",
           "STEP_SGD_MEAN", "FOOT_BILINEAR", "FOOT_NEAREST", "OK", "ERR_BIN_OVERFLOW", "ERR_BAD_INDEX", "ERR_BOUNDS",
           "LIMIT_VERTICES", "LIMIT_UVS", "LIMIT_BIN_ENTRIES", "LIMIT_SIGN_WORDS", "LIMIT_PARAMS", "checked_build",
           "MAX_VIEWS_PER_CALL"]


def load(build_if_missing: bool = False):
    return _abi.load(build_if_missing)


def checked_build() -> bool:
    """Is the loaded library the range-checked build (SGE_CHECKED=1)?"""
    return bool(_abi.load().sge_checked_build())


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class Scene:
    """A scene on the GPU: borrows the tensors it is built from (keep them alive).

    positions [V,3] and every texture [H,W,C] (float32, CUDA, contiguous) are the
    parameters theta that sge_step updates in place.
    """

    def __init__(self, positions, pos_idx, uvs, uv_idx, textures, eps_pos: float, mvp, cam_pos,
                 width: int, height: int, targets=None, near: float = 0.1, shading: int = 0,
                 light_dir=(0.0, 0.0, 1.0), light_rgb=(1.0, 1.0, 1.0), ambient: float = 0.0,
                 background=(0.0, 0.0, 0.0), max_views_per_call: int = 0, bin_capacity: int = 0,
                 pairs_per_item: int = 0, blocks_per_sm: int = 0, max_pairs_per_call: int = 0,
                 footprint: int = 0, device=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("sge needs a CUDA device; there is no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        L = _abi.load()

        def dev(x, dtype):
            t = torch.as_tensor(x).to(device=self.device, dtype=dtype)
            return t.contiguous()

        self.positions = dev(positions, torch.float32)
        self.pos_idx = dev(pos_idx, torch.int32)
        self.uvs = dev(uvs, torch.float32)
        self.uv_idx = dev(uv_idx, torch.int32)
        self.textures = []  # list of (tensor [H,W,C], eps, role)
        for t in textures:
            data = dev(t[0], torch.float32)
            if data.dim() == 2:
                data = data.unsqueeze(-1).contiguous()
            self.textures.append((data, float(t[1]), int(t[2])))
        self.mvp = dev(mvp, torch.float32).reshape(-1, 4, 4).contiguous()
        self.cam_pos = dev(cam_pos, torch.float32).reshape(-1, 3).contiguous()
        self.n_views = int(self.mvp.shape[0])
        self.width, self.height = int(width), int(height)
        if targets is None:
            targets = torch.zeros(self.n_views, self.height, self.width, 3)
        self.targets = dev(targets, torch.float32)
        if len(self.textures) > MAX_TEXTURES:
            raise ValueError(f"at most {MAX_TEXTURES} textures")

        d = _abi.SceneDesc()
        d.positions = _ptr(self.positions)
        d.n_vertices = int(self.positions.shape[0])
        d.eps_pos = float(eps_pos)
        d.pos_idx = _ptr(self.pos_idx)
        d.n_triangles = int(self.pos_idx.shape[0])
        d.uvs = _ptr(self.uvs)
        d.n_uvs = int(self.uvs.shape[0])
        d.uv_idx = _ptr(self.uv_idx)
        d.n_textures = len(self.textures)
        for k, (data, eps, role) in enumerate(self.textures):
            d.textures[k].texels = _ptr(data)
            d.textures[k].height, d.textures[k].width, d.textures[k].channels = (int(x) for x in data.shape)
            d.textures[k].eps = eps
            d.textures[k].role = role
        d.mvp = _ptr(self.mvp)
        d.cam_pos = _ptr(self.cam_pos)
        d.n_views = self.n_views
        d.width, d.height = self.width, self.height
        d.near_w = float(near)
        d.targets = _ptr(self.targets)
        for c in range(3):
            d.background[c] = float(background[c])
            d.light_dir[c] = float(light_dir[c])
            d.light_rgb[c] = float(light_rgb[c])
        d.shading = int(shading)
        d.ambient = float(ambient)
        self._desc = d
        cfg = _abi.Config(int(max_views_per_call), int(bin_capacity), int(pairs_per_item), int(blocks_per_sm),
                          int(max_pairs_per_call), int(footprint))
        self._cfg = cfg
        nbytes = C.c_size_t()
        _abi.check(L.sge_workspace_size(C.byref(d), C.byref(cfg), C.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        base = _ptr(self.workspace)
        off = (-base) % 256
        handle = C.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(L.sge_create_scene(C.byref(d), C.byref(cfg), base + off, int(nbytes.value),
                                          C.byref(handle)))
        self._h = handle
        n = C.c_int64()
        _abi.check(L.sge_num_params(self._h, C.byref(n)))
        self.n_params = int(n.value)

    # ------------------------------------------------------------------ construction helpers
    @classmethod
    def from_arrays(cls, s, targets=None, **kw) -> "Scene":
        """From any object with synth.Scene's attributes (numpy arrays)."""
        return cls(s.positions, s.pos_idx, s.uvs, s.uv_idx, [(t.data, t.eps, t.role) for t in s.textures],
                   s.eps_pos, s.mvp, s.cam_pos, s.width, s.height, targets=targets, near=s.near,
                   shading=s.shading, light_dir=s.light_dir, light_rgb=s.light_rgb, ambient=s.ambient,
                   background=s.background, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _abi.load().sge_destroy_scene(h)
            except Exception:
                pass
            self._h = None

    # ------------------------------------------------------------------ parameters
    def param_groups(self) -> List:
        return [self.positions] + [t[0] for t in self.textures]

    def group_offsets(self) -> List[int]:
        offs, o = [], 0
        for g in self.param_groups():
            offs.append(o)
            o += g.numel()
        return offs

    def new_grad_buffers(self):
        torch = _torch()
        return (torch.zeros(self.n_params, dtype=torch.float32, device=self.device),
                torch.zeros(self.n_params, dtype=torch.int32, device=self.device))

    def set_targets(self, targets) -> None:
        torch = _torch()
        t = torch.as_tensor(targets).to(device=self.device, dtype=torch.float32).contiguous()
        if tuple(t.shape) != (self.n_views, self.height, self.width, 3):
            raise ValueError(f"targets must be [{self.n_views},{self.height},{self.width},3]")
        self.targets = t
        _abi.check(_abi.load().sge_set_targets(self._h, _ptr(t)))

    # ------------------------------------------------------------------ calls
    def validate(self, stream=None) -> int:
        L = _abi.load()
        _abi.check(L.sge_validate(self._h, _stream_ptr(stream)))
        return self.status(stream)

    def check_limit(self, which: int, limit: int = -1) -> None:
        """Checked build only: lower the bound the range checks of `which` (LIMIT_*) compare
        against (limit < 0: back to the true size); no allocation or logic changes."""
        _abi.check(_abi.load().sge_check_limit(self._h, which, limit))

    def check_report(self, stream=None):
        """Checked build only: (site, index) of the first range check that failed since the last
        report (site 0: none), cleared by reading."""
        site, index = C.c_int32(), C.c_int64()
        _abi.check(_abi.load().sge_check_report(self._h, _stream_ptr(stream), C.byref(site), C.byref(index)))
        return int(site.value), int(index.value)

    def status(self, stream=None) -> int:
        v = C.c_int32()
        _abi.check(_abi.load().sge_status(self._h, _stream_ptr(stream), C.byref(v)))
        return int(v.value)

    def render_idb(self, view: int, seed: int = 0, it: int = 0, pair: int = 0, side: int = 0,
                   keys=None, uv=None, rgb=None, stream=None):
        """One render (Section 4.3 R): depth|ID [H,W] int64 (bit pattern of uint64), UV, RGB."""
        torch = _torch()
        H, W = self.height, self.width
        keys = torch.empty(H, W, dtype=torch.int64, device=self.device) if keys is None else keys
        uv = torch.empty(H, W, 2, dtype=torch.float32, device=self.device) if uv is None else uv
        rgb = torch.empty(H, W, 3, dtype=torch.float32, device=self.device) if rgb is None else rgb
        _abi.check(_abi.load().sge_render_idb(self._h, int(view), int(seed), int(it), int(pair), int(side),
                                              _ptr(keys), _ptr(uv), _ptr(rgb), _stream_ptr(stream)))
        return keys, uv, rgb

    def render_deep(self, view: int, seed: int = 0, it: int = 0, pair: int = 0, side: int = 0,
                    deep=None, rgb=None, stream=None):
        """One render of a transparent scene (Section 4.4): deep ID buffer [MAX_LAYERS,H,W] int64
        (bit patterns of the ascending uint64 keys, -1 = empty) and the composite [H,W,3]."""
        torch = _torch()
        H, W = self.height, self.width
        deep = torch.empty(_abi.MAX_LAYERS, H, W, dtype=torch.int64, device=self.device) if deep is None else deep
        rgb = torch.empty(H, W, 3, dtype=torch.float32, device=self.device) if rgb is None else rgb
        _abi.check(_abi.load().sge_render_deep(self._h, int(view), int(seed), int(it), int(pair), int(side),
                                               _ptr(deep), _ptr(rgb), _stream_ptr(stream)))
        return deep, rgb

    def render_targets(self, stream=None):
        """Unperturbed renders of every view, [n_views,H,W,3] (e.g. of a target scene)."""
        torch = _torch()
        out = torch.empty(self.n_views, self.height, self.width, 3, dtype=torch.float32, device=self.device)
        for v in range(self.n_views):
            if self._desc.shading == SHADE_TRANSPARENT:
                self.render_deep(v, side=0, rgb=out[v], stream=stream)
            else:
                self.render_idb(v, side=0, rgb=out[v], stream=stream)
        return out

    @staticmethod
    def _views(view_ids: Sequence[int]):
        arr = (C.c_int32 * len(view_ids))(*[int(v) for v in view_ids])
        return arr, len(view_ids)

    def estimate_grad(self, seed: int, it, view_ids: Sequence[int], pairs_per_view: int, grad, counts,
                      loss=None, delta_f=None, stream=None) -> None:
        """Accumulate Eq. 9's numerators into grad [d] and counts [d] (batched, one launch).
        `it` is the iteration index, or an IterState whose device word the kernels read when
        they run (a loop captured once in a CUDA graph)."""
        arr, n = self._views(view_ids)
        L = _abi.load()
        if isinstance(it, IterState):
            _abi.check(L.sge_estimate_grad_state(self._h, int(seed), it.ptr, arr, n, int(pairs_per_view),
                                                 _ptr(grad), _ptr(counts), _ptr(loss), _ptr(delta_f),
                                                 _stream_ptr(stream)))
            return
        _abi.check(L.sge_estimate_grad(self._h, int(seed), int(it), arr, n, int(pairs_per_view),
                                       _ptr(grad), _ptr(counts), _ptr(loss), _ptr(delta_f), _stream_ptr(stream)))

    def estimate_grad_plain(self, seed: int, it: int, view_ids: Sequence[int], pairs_per_view: int, grad,
                            counts, loss=None, stream=None) -> None:
        """Same sums, one estimate at a time with separate R and G launches (the baseline path)."""
        arr, n = self._views(view_ids)
        _abi.check(_abi.load().sge_estimate_grad_plain(self._h, int(seed), int(it), arr, n, int(pairs_per_view),
                                                       _ptr(grad), _ptr(counts), _ptr(loss), _stream_ptr(stream)))

    def kernel_timing(self, enable: bool) -> None:
        """Record CUDA events around each fast-estimator launch of estimate_grad (benchmarks)."""
        _abi.check(_abi.load().sge_kernel_timing(self._h, 1 if enable else 0))

    def kernel_time(self, with_heavy: bool = False):
        """(total ms, launches) of the fast estimator since the last read (synchronises);
        with_heavy: (fast ms, heavy-bin kernel ms, launches)."""
        ms, hms, n = C.c_float(0.0), C.c_float(0.0), C.c_int32(0)
        _abi.check(_abi.load().sge_kernel_time(self._h, C.byref(ms), C.byref(hms), C.byref(n)))
        if with_heavy:
            return float(ms.value), float(hms.value), int(n.value)
        return float(ms.value), int(n.value)

    def bin_stats(self, stream=None):
        """(light items, heavy items, bin entries) of the last estimate call (synchronises)."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _abi.check(_abi.load().sge_bin_stats(self._h, _stream_ptr(stream), C.byref(a), C.byref(b), C.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def estimate_grad_full_image(self, seed: int, it: int, view_ids: Sequence[int], pairs_per_view: int, grad,
                                 counts, image_df=None, stream=None):
        """Eq. 4 with the whole-image error (the estimator Section 6.1 compares with): every
        parameter gets dF s_i per estimate.  Returns image_df [views, pairs] (each estimate's dF)."""
        torch = _torch()
        if image_df is None:
            image_df = torch.empty(len(view_ids), int(pairs_per_view), dtype=torch.float32, device=self.device)
        arr, n = self._views(view_ids)
        _abi.check(_abi.load().sge_estimate_grad_full_image(self._h, int(seed), int(it), arr, n, int(pairs_per_view),
                                                            _ptr(grad), _ptr(counts), _ptr(image_df),
                                                            _stream_ptr(stream)))
        return image_df

    def iterate_host(self, seed: int, state: "IterState", view_ids: Sequence[int], pairs_per_view: int, grad,
                     counts, m, v, lr_pos: float, lr_tex: Sequence[float], kind: int = _abi.STEP_ADAM,
                     loss_dev=None, theta_in=None, targets_in=None, theta_out=None, loss_out=None,
                     beta1: float = 0.9, beta2: float = 0.999, adam_eps: float = 1e-8, stream=None) -> None:
        """One optimizer iteration from host memory (sge_iterate_host): theta_in [d] and
        targets_in (CPU float32 tensors, pinned for asynchronous copies) into the scene's device
        arrays, the estimate of the state's iteration, the step with the state's t, the
        advance, then the updated theta into theta_out and the loss into loss_out.  Nothing
        synchronises: keep the host tensors alive until the stream has passed the call."""
        o = _abi.Opt()
        o.kind = int(kind)
        o.lr_pos = float(lr_pos)
        for k, lr in enumerate(lr_tex):
            o.lr_tex[k] = float(lr)
        o.beta1, o.beta2, o.adam_eps, o.t = float(beta1), float(beta2), float(adam_eps), 1
        io = _abi.HostIO(_host_ptr(theta_in), _host_ptr(targets_in), _host_ptr(theta_out), _host_ptr(loss_out))
        arr, n = self._views(view_ids)
        _abi.check(_abi.load().sge_iterate_host(self._h, int(seed), state.ptr, arr, n, int(pairs_per_view),
                                                C.byref(o), _ptr(grad), _ptr(counts), _ptr(m), _ptr(v),
                                                _ptr(loss_dev), C.byref(io), _stream_ptr(stream)))

    def loss(self, view_ids: Sequence[int], out=None, stream=None):
        """Image error f(theta) of the unperturbed scene per listed view (Table 1), [n] float32."""
        torch = _torch()
        out = torch.zeros(len(view_ids), dtype=torch.float32, device=self.device) if out is None else out
        arr, n = self._views(view_ids)
        _abi.check(_abi.load().sge_loss(self._h, arr, n, _ptr(out), _stream_ptr(stream)))
        return out

    def gradient(self, grad, n_pairs_total: int, scale=None, out=None, stream=None):
        """Eq. 9's estimate from accumulated sums: scale * grad / (2 eps N), flat [d] float32."""
        torch = _torch()
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device) if out is None else out
        _abi.check(_abi.load().sge_gradient(self._h, _ptr(grad), int(n_pairs_total), _ptr(scale), _ptr(out),
                                            _stream_ptr(stream)))
        return out

    def step(self, kind: int, grad, counts, n_pairs_total: int, lr_pos: float, lr_tex: Sequence[float],
             m=None, v=None, t=1, beta1: float = 0.9, beta2: float = 0.999, adam_eps: float = 1e-8,
             stream=None) -> None:
        """Descent step D on every group (Section 5); zeroes grad and counts.  `t` is Adam's step
        number, or an IterState whose device word the step reads when it runs."""
        o = _abi.Opt()
        o.kind = int(kind)
        o.lr_pos = float(lr_pos)
        for k, lr in enumerate(lr_tex):
            o.lr_tex[k] = float(lr)
        L = _abi.load()
        if isinstance(t, IterState):
            o.beta1, o.beta2, o.adam_eps, o.t = float(beta1), float(beta2), float(adam_eps), 1
            _abi.check(L.sge_step_state(self._h, C.byref(o), t.ptr, _ptr(grad), _ptr(counts), int(n_pairs_total),
                                        _ptr(m), _ptr(v), _stream_ptr(stream)))
            return
        o.beta1, o.beta2, o.adam_eps, o.t = float(beta1), float(beta2), float(adam_eps), int(t)
        _abi.check(L.sge_step(self._h, C.byref(o), _ptr(grad), _ptr(counts), int(n_pairs_total),
                              _ptr(m), _ptr(v), _stream_ptr(stream)))


def _host_ptr(t):
    """Address of a host (CPU) tensor's data, or None."""
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous() or t.dtype != _torch().float32:
        raise ValueError("host buffers must be contiguous float32 CPU tensors")
    return t.data_ptr()


class IterState:
    """The (iteration index, Adam step number) of an optimizer loop in device memory
    (sge_iter_state): estimate_grad and step read it when their kernels run, and advance()
    enqueues its increment, so a loop captured once in a CUDA graph draws fresh signs and takes
    the next Adam step on every replay (Section 5)."""

    def __init__(self, it: int = 0, t: int = 1, device=None):
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.tensor = torch.tensor([int(it), int(t)], dtype=torch.int32, device=dev)

    @property
    def ptr(self) -> int:
        return int(self.tensor.data_ptr())

    def advance(self, d_iter: int = 1, d_t: int = 1, stream=None) -> None:
        _abi.check(_abi.load().sge_iter_advance(self.ptr, int(d_iter), int(d_t), _stream_ptr(stream)))

    def value(self):
        """(iteration, t) as they stand (synchronises)."""
        it, t = (int(x) for x in self.tensor.tolist())
        return it & 0xFFFFFFFF, t


CHECKPOINT_FORMAT = "sge-checkpoint-1"


def save_checkpoint(path, scene, seed: int, it, t=None, m=None, v=None) -> None:
    """Save an optimisation's state with torch.save: theta (every parameter group of `scene`:
    positions, then each texture), Adam's first and second moments m and v (or None for SGD), the
    seed, the iteration index and Adam's step number t.  `it` may be an IterState (then it also
    gives t).  Synchronises the device first.  The sign generator is counter-based (seed,
    iteration, view, pair, parameter), so these determine every later estimate: a resumed run
    draws the same signs and credits the same counts."""
    torch = _torch()
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if isinstance(it, IterState):
        it, t = it.value()
    if t is None:
        raise ValueError("save_checkpoint: t (Adam's step number) is required")
    state = {"format": CHECKPOINT_FORMAT, "seed": int(seed), "iter": int(it), "t": int(t),
             "n_params": int(scene.n_params),
             "groups": [g.detach().to("cpu", copy=True) for g in scene.param_groups()],
             "m": None if m is None else m.detach().to("cpu", copy=True),
             "v": None if v is None else v.detach().to("cpu", copy=True)}
    torch.save(state, path)


def load_checkpoint(path, scene, m=None, v=None, iter_state=None):
    """Restore a save_checkpoint file into `scene`'s own parameter tensors (in place: the
    library keeps their device addresses), into m and v (when the file has them), and, given one,
    into an IterState.  Returns (seed, iteration, t).  Raises ValueError if the file is not a
    checkpoint of a scene with the same parameter groups."""
    torch = _torch()
    state = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(state, dict) or state.get("format") != CHECKPOINT_FORMAT:
        raise ValueError(f"{path}: not a {CHECKPOINT_FORMAT} file")
    groups = scene.param_groups()
    if state["n_params"] != scene.n_params or len(state["groups"]) != len(groups) or \
            any(tuple(a.shape) != tuple(b.shape) for a, b in zip(state["groups"], groups)):
        raise ValueError(f"{path}: parameter groups differ from the scene's")
    for dst, src in zip(groups, state["groups"]):
        dst.copy_(src)
    for dst, key in ((m, "m"), (v, "v")):
        if dst is not None and state[key] is not None:
            if dst.numel() != state[key].numel():
                raise ValueError(f"{path}: {key} has {state[key].numel()} entries, the buffer {dst.numel()}")
            dst.copy_(state[key].reshape(dst.shape))
    if iter_state is not None:
        it = state["iter"] - (1 << 32) if state["iter"] >= (1 << 31) else state["iter"]  # uint32 in an int32 word
        iter_state.tensor.copy_(torch.tensor([it, state["t"]], dtype=torch.int32))
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    return state["seed"], state["iter"], state["t"]


def draw_views(seed: int, it: int, n_views: int, count: int) -> List[int]:
    """Views of iteration `it` (Section 5: a random view per estimate), `count` distinct ones."""
    out = (C.c_int32 * int(count))()
    _abi.check(_abi.load().sge_draw_views(int(seed), int(it), int(n_views), int(count), out))
    return [int(v) for v in out]


def refine(matrix, x, y=None, accumulate: bool = False, stream=None):
    """y (+)= A x for xyz rows: A a CSR triple (row_ptr int32, col int32, w float32; CUDA tensors),
    x [n_cols, 3] float32.  With A = R, the refine matrix of a subdivision, y = fine positions;
    with A = R^T, y accumulates the control vertices' sums from the fine ones (chain rule)."""
    torch = _torch()
    row_ptr, col, w = matrix
    n_rows = int(row_ptr.numel()) - 1
    if y is None:
        y = torch.zeros(n_rows, 3, dtype=torch.float32, device=x.device)
    _abi.check(_abi.load().sge_refine(_ptr(row_ptr), _ptr(col), _ptr(w), n_rows, _ptr(x), _ptr(y),
                                      1 if accumulate else 0, _stream_ptr(stream)))
    return y


def csr_tensors(matrix, device):
    """A scipy sparse matrix as the CSR triple refine takes (row_ptr, col int32; w float32)."""
    torch = _torch()
    M = matrix.tocsr()
    M.sort_indices()
    return (torch.tensor(M.indptr.astype("int32"), device=device),
            torch.tensor(M.indices.astype("int32"), device=device),
            torch.tensor(M.data.astype("float32"), device=device))


class ControlMesh:
    """A control mesh behind a subdivided scene (Section 6.3: the rendered surface is the
    control mesh's subdivision; the parameters optimised are the control vertices and the
    textures).  R is the fixed refine matrix (scipy sparse, fine vertices x control vertices,
    e.g. synth.subdivide_catmull_clark's): fine = R control, so the control coordinates' sums
    are R^T times the fine vertices' sums.  `params` is a scene over the control vertices and
    the fine scene's own texture tensors; its step updates both in place.

        cm = ControlMesh(fine_scene, control, R)       # control: positions, pos_idx, uvs, uv_idx
        cm.refine()                                    # fine positions = R control
        fine_scene.estimate_grad(seed, it, views, pairs, g_fine, c_fine)
        cm.control_sums(g_fine, g_ctl)                 # positions through R^T, texture sums copied
        cm.params.step(STEP_ADAM, g_ctl, c_ctl, n_pairs, ...)
    """

    def __init__(self, fine: Scene, control, R):
        if R.shape != (int(fine.positions.shape[0]), int(len(control.positions))):
            raise ValueError(f"refine matrix {R.shape} does not map {len(control.positions)} control "
                             f"vertices to the scene's {int(fine.positions.shape[0])}")
        self.fine = fine
        self.R = csr_tensors(R, fine.device)
        self.RT = csr_tensors(R.T, fine.device)
        d = fine._desc
        self.params = Scene(control.positions, control.pos_idx, control.uvs, control.uv_idx,
                            [(t, eps, role) for t, eps, role in fine.textures], d.eps_pos, fine.mvp,
                            fine.cam_pos, fine.width, fine.height, targets=fine.targets, near=d.near_w,
                            shading=d.shading, light_dir=tuple(d.light_dir), light_rgb=tuple(d.light_rgb),
                            ambient=d.ambient, background=tuple(d.background), device=fine.device)
        self.positions = self.params.positions
        self.n_fine = 3 * int(fine.positions.shape[0])
        self.n_control = 3 * int(self.positions.shape[0])
        if self.params.n_params - self.n_control != fine.n_params - self.n_fine:
            raise RuntimeError("control and fine scenes disagree on the texture parameters")

    def new_grad_buffers(self):
        return self.params.new_grad_buffers()

    def refine(self, stream=None) -> None:
        """The fine scene's positions from the control positions (sge_refine with R)."""
        refine(self.R, self.positions, self.fine.positions, stream=stream)

    def control_sums(self, grad_fine, grad_control, stream=None) -> None:
        """grad_control = the control parameters' sums: R^T on the position block, the texture
        block copied (the textures are the same parameters in both scenes)."""
        torch = _torch()
        refine(self.RT, grad_fine[:self.n_fine].view(-1, 3), grad_control[:self.n_control].view(-1, 3),
               stream=stream)
        s = torch.cuda.current_stream(self.fine.device) if stream is None else stream
        with torch.cuda.stream(s):
            grad_control[self.n_control:].copy_(grad_fine[self.n_fine:], non_blocking=True)


class Batch:
    """Several scenes (assets) estimated together: sge_estimate_grad_batch runs every
    estimate of every asset in one persistent launch per estimator kernel, each
    asset's sums into its own buffers.

        b = Batch([(scene, views, grad, counts), ...])       # or (scene, views, grad, counts, loss)
        b.autotune(pairs)                                     # optional: pick the launch shape
        b.estimate_grad(seed, it, pairs)
    """

    def __init__(self, entries):
        if not 1 <= len(entries) <= _abi.MAX_BATCH:
            raise ValueError(f"a batch holds 1..{_abi.MAX_BATCH} entries")
        self.scenes = []
        self._keep = []
        self._arr = (_abi.BatchEntry * len(entries))()
        for i, e in enumerate(entries):
            scene, views, grad, counts = e[:4]
            loss = e[4] if len(e) > 4 else None
            varr, n = Scene._views(views)
            self._keep.append((varr, grad, counts, loss))
            self.scenes.append(scene)
            E = self._arr[i]
            E.scene, E.view_ids, E.n_views = scene._h.value, C.addressof(varr), n
            E.grad_sums, E.counts, E.loss_out = _ptr(grad), _ptr(counts), _ptr(loss)
        self.tuning = _abi.BatchTuning()

    def estimate_grad(self, seed: int, it, pairs_per_view: int, stream=None) -> None:
        """Every entry's estimates in one persistent launch per kernel; `it` is the iteration
        index or an IterState read on the device (a loop captured in a CUDA graph)."""
        L = _abi.load()
        if isinstance(it, IterState):
            _abi.check(L.sge_estimate_grad_batch_state(self._arr, len(self.scenes), int(seed), it.ptr,
                                                       int(pairs_per_view), C.byref(self.tuning),
                                                       _stream_ptr(stream)))
            return
        _abi.check(L.sge_estimate_grad_batch(self._arr, len(self.scenes), int(seed), int(it),
                                             int(pairs_per_view), C.byref(self.tuning), _stream_ptr(stream)))

    def autotune(self, pairs_per_view: int, repeats: int = 2, stream=None, cache: Optional[str] = None) -> float:
        """Pick the launch shape for these entries (zeroes their buffers); returns its ms.
        With `cache` (a JSON file path), a launch shape stored there for the same GPU, render
        sizes, triangle-count buckets and pairs is reused without timing, and a new one is
        stored."""
        key = None
        if cache is not None:
            torch = _torch()
            dev = self.scenes[0].device
            key = tuning_key(torch.cuda.get_device_name(dev),
                             [(sc.width, sc.height, int(sc.pos_idx.shape[0])) for sc in self.scenes],
                             pairs_per_view)
            hit = tuning_cache_load(cache, key)
            if hit is not None:
                self.tuning, ms = hit
                return ms
        t = _abi.BatchTuning()
        ms = C.c_float(0.0)
        _abi.check(_abi.load().sge_autotune_batch(self._arr, len(self.scenes), int(pairs_per_view), int(repeats),
                                                  C.byref(t), C.byref(ms), _stream_ptr(stream)))
        self.tuning = t
        if key is not None:
            tuning_cache_store(cache, key, t, float(ms.value))
        return float(ms.value)


def tuning_key(gpu: str, assets, pairs_per_view: int) -> str:
    """Key of a batch's launch shape in the tuning cache: the GPU's name, each asset's render
    size and triangle count rounded up to a power of two (in the batch's order), and the pairs per
    view.  assets: [(width, height, n_triangles), ...]."""
    parts = [f"{int(w)}x{int(h)}:T{1 << max(0, int(t) - 1).bit_length()}" for w, h, t in assets]
    return f"{gpu}|{int(pairs_per_view)}|" + ",".join(parts)


def tuning_cache_load(path: str, key: str):
    """(BatchTuning, ms) stored under key, or None (no file, no entry, or an unreadable file)."""
    import json
    import os
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            e = json.load(f).get(key)
        if e is None:
            return None
        return _abi.BatchTuning(int(e["pairs_per_item"]), int(e["blocks_per_sm"]), int(e["light_bin"])), float(e["ms"])
    except (OSError, ValueError, KeyError, TypeError, AttributeError):
        return None


def tuning_cache_store(path: str, key: str, t, ms: float) -> None:
    """Store a launch shape under key (the file is rewritten whole, through a temporary file)."""
    import json
    import os
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
            if not isinstance(data, dict):
                data = {}
        except (OSError, ValueError):
            data = {}
    data[key] = {"pairs_per_item": int(t.pairs_per_item), "blocks_per_sm": int(t.blocks_per_sm),
                 "light_bin": int(t.light_bin), "ms": float(ms)}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _make_function():
    torch = _torch()

    class SGEFunction(torch.autograd.Function):
        """f(theta) = sum over views of the image error (forward: render + L2 in the library);
        backward: per view, the per-pixel stochastic estimate of Eq. 9 over `pairs`
        antithetic pairs for (seed, iteration), summed over the views
        (sge_estimate_grad + sge_gradient), times the incoming gradient.  `params` must
        be the scene's own parameter tensors."""

        @staticmethod
        def forward(ctx, scene, spec, *params):
            for p, q in zip(params, scene.param_groups()):
                if p.data_ptr() != q.data_ptr():
                    raise ValueError("SGEFunction: params must be the scene's own parameter tensors")
            ctx.scene, ctx.spec = scene, spec
            return scene.loss(spec["views"]).sum()

        @staticmethod
        def backward(ctx, grad_out):
            scene, spec = ctx.scene, ctx.spec
            grad, counts = scene.new_grad_buffers()
            scene.estimate_grad(spec["seed"], spec["iter"], spec["views"], spec["pairs"], grad, counts)
            scale = grad_out.reshape(1).to(dtype=torch.float32).contiguous()
            # the forward sums the views' errors, so its gradient sums the per-view estimates:
            # Eq. 9 averaged over the pairs of each view only
            flat = scene.gradient(grad, spec["pairs"], scale=scale)
            outs, o = [], 0
            for g in scene.param_groups():
                outs.append(flat[o:o + g.numel()].view_as(g))
                o += g.numel()
            return (None, None, *outs)

    return SGEFunction


_fn_cache = {}


def __getattr__(name):
    if name == "SGEFunction":
        if "f" not in _fn_cache:
            _fn_cache["f"] = _make_function()
        return _fn_cache["f"]
    raise AttributeError(name)


def sge_loss(scene: Scene, seed: int, it: int, views: Sequence[int], pairs: int):
    """Differentiable image error: forward renders, backward estimates (Eq. 9) with the given seeds."""
    fn = __getattr__("SGEFunction")
    params = scene.param_groups()
    for p in params:
        p.requires_grad_(True)
    return fn.apply(scene, {"seed": int(seed), "iter": int(it), "views": list(views), "pairs": int(pairs)}, *params)
