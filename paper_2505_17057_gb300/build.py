"""In-tree build of libmmfd.so for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel; the shared library lands in
paper_2505_17057_gb300/_build/libmmfd.so.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmmfd.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmmfd")
    return cand


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _headers_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()


def _obj_stale(src: str, obj: str, digest_file: str, digest: str) -> bool:
    if not os.path.exists(obj):
        return True
    if os.path.getmtime(obj) < os.path.getmtime(src):
        return True
    try:
        with open(digest_file) as fh:
            return fh.read().strip() != digest
    except OSError:
        return True


def build(verbose: bool = False, jobs: int | None = None, extra_flags=None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    home = _cuda_home(nvcc)
    cu, cpp = _sources()
    digest = _headers_digest() + " ".join(extra_flags or [])
    digest_file = os.path.join(BUILD, "headers.sha")
    common_inc = ["-I", CSRC, "-I", INCLUDE]
    cmds = []
    objs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f[:-3] + ".o")
        objs.append(obj)
        if _obj_stale(src, obj, digest_file, digest):
            cmds.append([nvcc, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
                         "-Xptxas", "-O3", "--expt-relaxed-constexpr", *common_inc,
                         *(extra_flags or []), "-c", src, "-o", obj])
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f[:-4] + ".o")
        objs.append(obj)
        if _obj_stale(src, obj, digest_file, digest):
            cmds.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function",
                         "-I", os.path.join(home, "include"), *common_inc, "-c", src, "-o", obj])
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 4))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        if verbose and p.stderr:
            print(p.stderr, file=sys.stderr)
        return p

    if cmds:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            list(ex.map(run, cmds))
    need_link = bool(cmds) or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
    if need_link:
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-Xlinker", "-z,defs"])
        os.replace(tmp, LIB)
    with open(digest_file, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
