"""Build libcootgb.so in-tree with nvcc (sm_103a).

Steps:
  1. embed the device headers (csrc/dev/*.cuh, *.h) as string literals in
     csrc/_embedded.inc -- NVRTC compiles them per expression tree at run time;
  2. compile the host sources (csrc/*.cpp) with nvcc in parallel and link them
     with the static CUDA runtime and NVRTC into libcootgb.so;
  3. compile csrc/dev_check.cu, which instantiates every kernel family of the
     device headers, with nvcc -gencode arch=compute_103a,code=sm_103a, so a
     header error fails the build rather than the first run (its register and
     shared-memory report lands in _build/ptxas.log).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
DEV = os.path.join(CSRC, "dev")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcootgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(os.path.realpath(nv)))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _dev_headers():
    return sorted(glob.glob(os.path.join(DEV, "*.cuh")) + glob.glob(os.path.join(DEV, "*.h")))


def _sources():
    cu = [p for p in glob.glob(os.path.join(CSRC, "*.cu")) if not os.path.basename(p).startswith("dev_check")]
    return sorted(glob.glob(os.path.join(CSRC, "*.cpp")) + cu)


def _inputs():
    return (_dev_headers() + _sources() + glob.glob(os.path.join(CSRC, "*.h"))
            + [os.path.join(ROOT, "include", "coot.h"), os.path.join(CSRC, "dev_check.cu"),
               os.path.join(CSRC, "dev_check_gm.cu"), __file__])


def embed_headers() -> str:
    out = os.path.join(CSRC, "_embedded.inc")
    parts = ["// generated by build.py from csrc/dev -- do not edit\n",
             "struct CootHeader { const char* name; const char* text; };\n",
             "static const CootHeader k_headers[] = {\n"]
    for h in _dev_headers():
        text = open(h).read()
        delim = "COOT_RAW_"
        assert (")" + delim + '"') not in text
        # split into chunks below the compiler's literal limit
        chunks = [text[i:i + 12000] for i in range(0, len(text), 12000)] or [""]
        lit = "\n".join('R"%s(%s)%s"' % (delim, c, delim) for c in chunks)
        parts.append('  {"%s", %s},\n' % (os.path.basename(h), lit))
    parts.append("};\nstatic const int k_n_headers = %d;\n" % len(_dev_headers()))
    new = "".join(parts)
    if not os.path.exists(out) or open(out).read() != new:
        with open(out, "w") as f:
            f.write(new)
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs() if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    embed_headers()
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(home, "include")]
    common = ARCH + ["-std=c++17", "-O2", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-Wall,-fvisibility=hidden"] + inc
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        procs.append((src, subprocess.Popen([nvcc, "-x", "cu"] + common + ["-c", src, "-o", obj],
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    chk = os.path.join(CSRC, "dev_check.cu")
    chk_obj = os.path.join(BUILD, "dev_check.o")
    procs.append((chk, subprocess.Popen([nvcc] + ARCH + ["-std=c++17", "-O3", "-fmad=false", "-Xptxas", "-v",
                                                         "-I", DEV, "-c", chk, "-o", chk_obj],
                                        stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    # the same kernels in the bounds-check build (COOT_DEBUG_BOUNDS)
    procs.append((chk + " (bounds)", subprocess.Popen(
        [nvcc] + ARCH + ["-std=c++17", "-O3", "-fmad=false", "-DCOOT_DEBUG_BOUNDS=1", "-I", DEV, "-c", chk, "-o",
                         os.path.join(BUILD, "dev_check_bounds.o")],
        stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    # kernels that write a general output (their own translation unit: the
    # output kind is a define of the whole program)
    chk_gm = os.path.join(CSRC, "dev_check_gm.cu")
    procs.append((chk_gm, subprocess.Popen(
        [nvcc] + ARCH + ["-std=c++17", "-O3", "-fmad=false", "-I", DEV, "-c", chk_gm, "-o",
                         os.path.join(BUILD, "dev_check_gm.o")],
        stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if src == chk:
            with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
                f.write(text)
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip() and src != chk:
            print(text)
    if failed:
        msg = "\n".join("== %s\n%s" % (s, t[-6000:]) for s, t in failed)
        raise RuntimeError("libcootgb build failed:\n" + msg)
    tmp = LIB + ".%d.tmp" % os.getpid()
    libdir = os.path.join(home, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(home, "lib")
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-L", libdir, "-lnvrtc", "-cudart", "static",
        "-Xlinker", "-rpath", "-Xlinker", libdir]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libcootgb link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
