"""Compile the CUDA sources under csrc/ into the in-tree shared library libsge.so (sm_103a), and
the same sources with SGE_CHECKED=1 (every kernel range-checks its indices into the device status
word) into libsge_checked.so."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libsge.so")
OUT_CHECKED = os.path.join(HERE, "libsge_checked.so")
BUILD = os.path.join(HERE, "_build")
BUILD_CHECKED = os.path.join(HERE, "_build", "checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libsge.so (libsge_checked.so with checked=True) if any source or header is newer than
    it; return its path."""
    out, bdir = (OUT_CHECKED, BUILD_CHECKED) if checked else (OUT, BUILD)
    extra = ["-DSGE_CHECKED=1"] if checked else []
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest(sources + headers):
        return out
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    hdr_time = _newest(headers)

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time):
            cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(sources)) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = out + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> None:
    """Both libraries, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(build, force, False, c) for c in (False, True)]:
            f.result()


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, verbose=True, checked=True))
