"""Build ``libqmpm.so`` in-tree with nvcc for sm_103a (B300).

``python -m paper_2207_04658_b300.build [--force]``.  Each source is compiled to an object
under ``_build/`` (in parallel) and linked into ``paper_2207_04658_b300/libqmpm.so``.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libqmpm.so")
SOURCES = ["api.cu", "step.cu", "sort.cu", "scheme.cpp"]
HEADERS = ["device_common.cuh", "qmpm_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]


def _sources():
    extra = [f for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cpp")) and f not in SOURCES]
    return SOURCES + extra


def _newest_header():
    paths = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    paths.append(os.path.join(ROOT, "include", "qmpm.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(src, force, verbose):
    obj = os.path.join(BUILD, src + ".o")
    src_path = os.path.join(CSRC, src)
    if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src_path)
            and os.path.getmtime(obj) >= _newest_header()):
        return obj
    cmd = [NVCC] + _flags() + ["-c", src_path, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose), srcs))
    if (force or not os.path.exists(LIB)
            or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lnvrtc"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
