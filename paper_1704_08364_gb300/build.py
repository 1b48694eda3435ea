"""In-tree build of libbst.so (the C-ABI library) and libbstsynth.so (the
device-side input generator) for sm_103a with nvcc.

Each translation unit compiles in its own nvcc process (in parallel), then one
link step produces the shared library next to this file.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]

LIBS = {
    "bst": (os.path.join(HERE, "csrc"), ["plan.cu", "fbp.cu", "adjoint.cu", "brute.cu", "noalloc.cu", "host.cu", "ragged.cu", "kb.cu", "fbp_pad1.cu", "fbp_pad2.cu"],
            os.path.join(HERE, "libbst.so")),
    "bstsynth": (os.path.join(ROOT, "synth", "csrc"), ["synth.cu"],
                 os.path.join(ROOT, "synth", "libbstsynth.so")),
}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def _stale(out: str, inputs) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(i) > t for i in inputs)


def build_lib(name: str, force: bool = False, extra_flags=()) -> str:
    src_dir, sources, out = LIBS[name]
    build_dir = os.path.join(ROOT, "_build", name)
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(src_dir, f) for f in os.listdir(src_dir) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in sources:
        src = os.path.join(src_dir, s)
        obj = os.path.join(build_dir, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-I", os.path.join(ROOT, "include"),
                         "-c", src, "-o", obj])
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(_run, jobs))
    if force or jobs or _stale(out, objs):
        _run([nvcc, *ARCH, "-shared", "-o", out, *objs])
    return out


def build_all(force: bool = False) -> list[str]:
    with ThreadPoolExecutor(max_workers=2) as ex:
        return list(ex.map(lambda n: build_lib(n, force), list(LIBS)))


if __name__ == "__main__":
    for p in build_all(force="--force" in sys.argv):
        print(p)
