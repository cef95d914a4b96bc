"""The C ABI library loads on a machine without a GPU and exports every symbol
include/sge.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sge.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char \*)\s*\*?\s*(sge_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sge_create_scene", "sge_render_idb", "sge_estimate_grad", "sge_step"):
        assert want in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_2404_09758_gb300 import _abi, build
    path = build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(_abi.EXPORTS)


def test_structure_layouts_match_the_header():
    """Compile a tiny C program against sge.h and compare sizes/offsets with the ctypes mirror."""
    import subprocess
    import tempfile
    from paper_2404_09758_gb300 import _abi
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "sge.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(sge_texture), sizeof(sge_scene_desc), sizeof(sge_config), sizeof(sge_opt));
  printf("%zu %zu %zu %zu\n", offsetof(sge_scene_desc, textures), offsetof(sge_scene_desc, mvp),
         offsetof(sge_scene_desc, targets), offsetof(sge_scene_desc, ambient));
  printf("%zu %zu %zu\n", offsetof(sge_opt, beta1), offsetof(sge_opt, t), offsetof(sge_config, max_pairs_per_call));
  printf("%zu %zu %zu\n", sizeof(sge_host_io), offsetof(sge_host_io, targets_in), offsetof(sge_host_io, loss_out));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    got = [int(x) for x in out]
    S = _abi.SceneDesc
    want = [ctypes.sizeof(_abi.Texture), ctypes.sizeof(S), ctypes.sizeof(_abi.Config), ctypes.sizeof(_abi.Opt),
            S.textures.offset, S.mvp.offset, S.targets.offset, S.ambient.offset,
            _abi.Opt.beta1.offset, _abi.Opt.t.offset, _abi.Config.max_pairs_per_call.offset,
            ctypes.sizeof(_abi.HostIO), _abi.HostIO.targets_in.offset, _abi.HostIO.loss_out.offset]
    assert got == want


def test_host_iteration_checks_its_arguments_before_enqueueing():
    """sge_iterate_host refuses a NULL scene, io, opt or state with SGE_ERR_INVALID_ARG before it
    copies or launches anything (no GPU is touched here)."""
    from paper_2404_09758_gb300 import _abi
    L = _abi.load()
    io, opt = _abi.HostIO(), _abi.Opt()
    state = ctypes.c_int32 * 2
    st = state()
    cases = ((None, ctypes.byref(st), ctypes.byref(opt), ctypes.byref(io)),
             (ctypes.c_void_p(8), ctypes.byref(st), ctypes.byref(opt), None),
             (ctypes.c_void_p(8), ctypes.byref(st), None, ctypes.byref(io)),
             (ctypes.c_void_p(8), None, ctypes.byref(opt), ctypes.byref(io)))
    for scene, stp, optp, iop in cases:
        rc = L.sge_iterate_host(scene, 1, stp, None, 0, 1, optp, None, None, None, None, None, iop, None)
        assert rc == _abi.ERR_INVALID_ARG, L.sge_last_error()
    # the step's own argument checks, also before the scene is looked at
    buf = (ctypes.c_float * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    scene, stp, iop = ctypes.c_void_p(8), ctypes.byref(st), ctypes.byref(io)
    rc = L.sge_iterate_host(scene, 1, stp, None, 1, 1, ctypes.byref(opt), None, p, p, p, None, iop, None)
    assert rc == _abi.ERR_INVALID_ARG and b"grad_sums" in L.sge_last_error()
    bad = _abi.Opt()
    bad.kind = 7
    rc = L.sge_iterate_host(scene, 1, stp, None, 1, 1, ctypes.byref(bad), p, p, p, p, None, iop, None)
    assert rc == _abi.ERR_INVALID_ARG and b"kind" in L.sge_last_error()
    adam = _abi.Opt()
    adam.kind = _abi.STEP_ADAM
    rc = L.sge_iterate_host(scene, 1, stp, None, 1, 1, ctypes.byref(adam), p, p, None, p, None, iop, None)
    assert rc == _abi.ERR_INVALID_ARG and b"Adam" in L.sge_last_error()


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2404_09758_gb300 import Scene
    with pytest.raises(RuntimeError):
        Scene(np.zeros((3, 3)), np.zeros((1, 3)), np.zeros((3, 2)), np.zeros((1, 3)), [], 1e-3,
              np.eye(4), np.zeros(3), 8, 8)


def test_descriptor_checks_run_on_the_host():
    """sge_workspace_size validates a scene description without touching a GPU: the textures
    must include every role the shading model reads."""
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    d = _abi.SceneDesc()
    fake = 0x1000  # never dereferenced by the host checks
    d.positions, d.n_vertices, d.eps_pos = fake, 3, 1e-3
    d.pos_idx, d.n_triangles, d.uvs, d.n_uvs, d.uv_idx = fake, 1, fake, 3, fake
    d.mvp, d.cam_pos, d.n_views, d.width, d.height, d.near_w, d.targets = fake, fake, 1, 32, 32, 0.1, fake
    nbytes = C.c_size_t()
    for shading, roles, ok in ((0, [0], True), (0, [], False), (1, [0], False), (1, [0, 1], True),
                               (2, [0, 1, 2], False), (2, [0, 1, 2, 3], True)):
        d.shading, d.n_textures = shading, len(roles)
        for k, role in enumerate(roles):
            d.textures[k].texels, d.textures[k].width, d.textures[k].height = fake, 4, 4
            d.textures[k].channels, d.textures[k].eps, d.textures[k].role = 3, 1.0 / 255.0, role
        rc = L.sge_workspace_size(C.byref(d), None, C.byref(nbytes))
        assert (rc == _abi.OK) == ok, (shading, roles, L.sge_last_error())
        if not ok:
            assert rc == _abi.ERR_INVALID_ARG and b"role" in L.sge_last_error()
    # transparent geometry reads one albedo, which must carry an opacity channel (RGBA)
    d.shading, d.n_textures = 3, 1
    d.textures[0].role = 0
    for channels, ok in ((4, True), (3, False), (1, False)):
        d.textures[0].channels = channels
        rc = L.sge_workspace_size(C.byref(d), None, C.byref(nbytes))
        assert (rc == _abi.OK) == ok, (channels, L.sge_last_error())
        if not ok:
            assert rc == _abi.ERR_INVALID_ARG and b"RGBA" in L.sge_last_error()


def test_view_draw_equals_the_oracle():
    """sge_draw_views (host code of the library) against the oracle's independent restatement."""
    import oracle
    from paper_2404_09758_gb300 import SGEError, draw_views
    for seed, it, n, k in ((0, 0, 8, 8), (7, 3, 8, 2), (123456789, 42, 64, 64), (5, 1, 100, 10), (9, 9, 1, 1)):
        assert draw_views(seed, it, n, k) == oracle.draw_views(seed, it, n, k)
    with pytest.raises(SGEError):
        draw_views(0, 0, 4, 5)


def _valid_desc():
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    d = _abi.SceneDesc()
    fake = 0x1000  # never dereferenced by the host checks
    d.positions, d.n_vertices, d.eps_pos = fake, 3, 1e-3
    d.pos_idx, d.n_triangles, d.uvs, d.n_uvs, d.uv_idx = fake, 1, fake, 3, fake
    d.mvp, d.cam_pos, d.n_views, d.width, d.height, d.near_w, d.targets = fake, fake, 2, 32, 24, 0.1, fake
    d.shading, d.n_textures = 0, 1
    t = d.textures[0]
    t.texels, t.width, t.height, t.channels, t.eps, t.role = fake, 4, 4, 3, 1.0 / 255.0, 0
    return d


@pytest.mark.parametrize("field, value", [
    ("n_vertices", 2), ("n_triangles", 0), ("n_views", 0), ("width", 0), ("height", 20000),
    ("eps_pos", -1.0), ("eps_pos", float("nan")), ("near_w", 0.0), ("shading", 4), ("n_textures", 9),
    ("positions", None), ("targets", None), ("tex_channels", 5), ("tex_role", 4), ("tex_eps", -1.0),
    ("tex_texels", None)])
def test_invalid_descriptions_are_rejected_on_the_host(field, value):
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    d = _valid_desc()
    n = C.c_size_t()
    assert L.sge_workspace_size(C.byref(d), None, C.byref(n)) == _abi.OK and n.value > 0
    if field.startswith("tex_"):
        setattr(d.textures[0], field[4:], value)
    else:
        setattr(d, field, value)
    assert L.sge_workspace_size(C.byref(d), None, C.byref(n)) == _abi.ERR_INVALID_ARG
    assert L.sge_last_error()  # a message says which
    # the allocation-free render checks the description with the same code (it reads no targets)
    rc = L.sge_render_idb_static(C.byref(d), 0, 0, 0, 0, 0, None, None, None, None, None)
    if field == "targets":
        assert rc != _abi.ERR_INVALID_ARG or b"targets" not in L.sge_last_error()
    else:
        assert rc == _abi.ERR_INVALID_ARG, (field, value, L.sge_last_error())


def test_static_render_checks_roles_and_its_own_limits_on_the_host():
    """A lit description without the textures its model reads, and a request one triangle over
    the fixed scratch's limit, are refused before any device call."""
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    d = _valid_desc()
    d.shading = 1  # Lambert without a normal map
    rc = L.sge_render_idb_static(C.byref(d), 0, 0, 0, 0, 0, None, None, None, None, None)
    assert rc == _abi.ERR_INVALID_ARG and b"role" in L.sge_last_error()
    d = _valid_desc()
    header = open(os.path.join(ROOT, "include", "sge.h")).read()
    limit = int(re.search(r"#define SGE_STATIC_MAX_TRIANGLES (\d+)", header).group(1))
    d.n_triangles = limit + 1
    n = C.c_size_t()
    assert L.sge_workspace_size(C.byref(d), None, C.byref(n)) == _abi.OK  # fine for a workspace
    rc = L.sge_render_idb_static(C.byref(d), 0, 0, 0, 0, 0, None, None, None, None, None)
    assert rc == _abi.ERR_INVALID_ARG and b"SGE_STATIC_MAX_TRIANGLES" in L.sge_last_error()
    d = _valid_desc()
    for view, side in ((2, 0), (-1, 0), (0, 2)):
        rc = L.sge_render_idb_static(C.byref(d), view, 0, 0, 0, side, None, None, None, None, None)
        assert rc == _abi.ERR_INVALID_ARG


def test_workspace_grows_with_views_and_pairs():
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    d = _valid_desc()
    sizes = []
    for views, pairs in ((1, 1), (2, 1), (2, 8)):
        cfg = _abi.Config(views, 0, 0, 0, pairs)
        n = C.c_size_t()
        assert L.sge_workspace_size(C.byref(d), C.byref(cfg), C.byref(n)) == _abi.OK
        sizes.append(n.value)
    assert sizes[0] < sizes[1] < sizes[2]
    cfg = _abi.Config(0, 1 << 33, 0, 0, 0)  # bin capacity must stay below 2^32 entries
    assert L.sge_workspace_size(C.byref(d), C.byref(cfg), C.byref(C.c_size_t())) == _abi.ERR_INVALID_ARG
    # the texel footprint is bilinear or nearest
    for foot, rc in ((_abi.FOOT_BILINEAR, _abi.OK), (_abi.FOOT_NEAREST, _abi.OK), (2, _abi.ERR_INVALID_ARG)):
        cfg = _abi.Config(0, 0, 0, 0, 0, foot)
        assert L.sge_workspace_size(C.byref(d), C.byref(cfg), C.byref(C.c_size_t())) == rc


def test_static_render_refuses_transparent_scenes_on_the_host():
    """The allocation-free render is written for one visible triangle a pixel: a transparent
    description is refused as unsupported before any device call."""
    import ctypes as C
    from paper_2404_09758_gb300 import _abi
    L = _abi.load(build_if_missing=True)
    d = _valid_desc()
    d.shading = 3
    d.textures[0].channels = 4
    rc = L.sge_render_idb_static(C.byref(d), 0, 0, 0, 0, 0, None, None, None, None, None)
    assert rc == _abi.ERR_UNSUPPORTED and b"sge_render_deep" in L.sge_last_error()
