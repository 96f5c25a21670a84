"""Build libdsr.so (sm_103a) in-tree with nvcc: one object per .cu file,
compiled in parallel, then linked against the shared CUDA runtime."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdsr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or install the CUDA toolkit)")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.cuh"))
            + [os.path.abspath(__file__)])


def _elf_machine(path: str) -> int:
    with open(path, "rb") as f:
        head = f.read(20)
    return int.from_bytes(head[18:20], "little") if head[:4] == b"\x7fELF" else -1


def _host_machine() -> int:
    return _elf_machine(sys.executable)


def _stale() -> bool:
    if not os.path.exists(LIB) or _elf_machine(LIB) != _host_machine():
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def compile_flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC, "--expt-relaxed-constexpr"] + list(extra)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every csrc/*.cu and link libdsr.so; returns its path."""
    with _lock:
        if not (force or ptxas_info or _stale()):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        cc = nvcc()
        extra = ["-Xptxas", "-v"] if ptxas_info else []

        def one(src):
            obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
            cmd = [cc, "-c", src, "-o", obj] + compile_flags(extra)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
            return obj, r.stderr

        srcs = _sources()
        with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
            results = list(ex.map(one, srcs))
        logs = "".join(r[1] for r in results)
        if verbose or ptxas_info:
            sys.stderr.write(logs)
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [cc, "-shared", "-o", tmp] + [r[0] for r in results] + ARCH + ["-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
        return LIB


def build_user(sources, out: str, force: bool = False, ptxas_info: bool = False) -> str:
    """Compile region programs written against include/dsr_device.cuh (the
    .cu files `sources`) into the shared library `out`, linked with
    libdsr.so (built first if needed); returns `out`. A program's kernels
    are instantiated in its own library, from the same templates as the
    built-in programs'."""
    lib = build()
    sources = [os.path.abspath(x) for x in sources]
    with _lock:
        deps = sources + _deps() + [lib]
        fresh = (os.path.exists(out) and _elf_machine(out) == _host_machine()
                 and all(os.path.getmtime(p) <= os.path.getmtime(out) for p in deps))
        if fresh and not (force or ptxas_info):
            return out
        cc = nvcc()
        extra = ["-Xptxas", "-v"] if ptxas_info else []
        objs = []
        os.makedirs(BUILD, exist_ok=True)
        for src in sources:
            obj = os.path.join(BUILD, "user_" + os.path.basename(src)[:-3] + ".o")
            r = subprocess.run([cc, "-c", src, "-o", obj] + compile_flags(extra),
                               capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
            if ptxas_info:
                sys.stderr.write(r.stderr)
            objs.append(obj)
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ([cc, "-shared", "-o", tmp] + objs + ARCH
               + ["-cudart", "shared", "-L", PKG, "-ldsr", "-Xlinker", "-rpath=" + PKG,
                  "-Xlinker", "-rpath=/usr/local/cuda/lib64"])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, out)
        return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
