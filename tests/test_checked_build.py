"""Host-side checks of the range-checked build (SGE_CHECKED=1): every index the kernels take from
the caller's index buffers or compute into a workspace buffer or the gradient sums goes through a
range check, and the two libraries answer the checked-build entry points as documented."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2404_09758_gb300", "csrc")


def _sources():
    out = {}
    for p in sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))):
        out[os.path.basename(p)] = open(p).read().splitlines()
    return out


def test_index_buffers_are_read_only_through_the_checked_helpers():
    """pos_idx / uv_idx entries reach no kernel except through vert_of / uv_of (which check them
    against the vertex and UV counts) and k_validate (which only compares them)."""
    raw = re.compile(r"\bS\.(pidx|uvidx)\b(?!\s*=[^=])|\.pidx\s*\[|\.uvidx\s*\[")  # reads, not the host's set-up
    bad = []
    for name, lines in _sources().items():
        fn = None
        for i, line in enumerate(lines):
            m = re.match(r"\s*(?:__device__|__global__)[^(]*?\b(\w+)\(", line)
            if m:
                fn = m.group(1)
            if raw.search(line) and fn not in ("vert_of", "uv_of", "k_validate"):
                bad.append(f"{name}:{i + 1}: {line.strip()}")
    assert not bad, "\n".join(bad)


def test_every_gradient_credit_and_bin_write_is_range_checked():
    credit = re.compile(r"atomicAdd\((a\.)?grad\s*\+")
    bins = re.compile(r"ws\.bins\[")
    bad = []
    for name, lines in _sources().items():
        for i, line in enumerate(lines):
            window = " ".join(lines[max(0, i - 2):i + 1])
            if credit.search(line) and "CHK(S, " not in window:
                bad.append(f"{name}:{i + 1}: {line.strip()}")
            if bins.search(line) and "CHK(S, " not in line and "bin_at" not in window:
                bad.append(f"{name}:{i + 1}: {line.strip()}")
    assert not bad, "\n".join(bad)


def test_sign_plane_reads_and_writes_are_range_checked():
    src = _sources()
    dev = "\n".join(src["sge_device.cuh"])
    assert re.search(r"texel_signs\(.*?\{.*?CHK_H\(\*ps\.S, w, ps\.S->chk\.sign_words\)", dev, re.S)
    fast = "\n".join(src["k_fast.cu"])
    assert re.search(r"plane_nibble\(.*?\{.*?CHK\(S, w, S\.chk\.sign_words\)", fast, re.S)
    assert "CHK(S, w, S.chk.sign_words)) out[w] = bits;" in "\n".join(src["k_vertex.cu"])


def test_both_libraries_answer_the_checked_entry_points():
    from paper_2404_09758_gb300 import _abi, _build
    plain = ctypes.CDLL(_build.build())
    checked = ctypes.CDLL(_build.build(checked=True))
    for L in (plain, checked):
        L.sge_check_limit.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]
        L.sge_check_limit.restype = ctypes.c_int32
        L.sge_checked_build.restype = ctypes.c_int32
    assert plain.sge_checked_build() == 0 and checked.sge_checked_build() == 1
    assert plain.sge_check_limit(None, _abi.LIMIT_PARAMS, 0) == _abi.ERR_UNSUPPORTED
    assert checked.sge_check_limit(None, _abi.LIMIT_PARAMS, 0) == _abi.ERR_INVALID_ARG
