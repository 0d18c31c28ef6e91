"""Builds libfgadmm.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel; the FP64 sweep is built with
-fmad=false (every product rounded on its own), the FP32 sweep with FMA
contraction allowed.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfgadmm.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _units():
    """(source, extra flags) for every translation unit of the library."""
    nv = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    units = [
        ("sweep_f32.cu", nv),
        ("sweep_f64.cu", nv + ["-fmad=false"]),
        ("sweep_tile.cu", nv),
        ("sweep_hinge.cu", nv),
        ("mpc_batch.cu", nv),
        ("mpc_warp.cu", nv),
        ("mpc_noalloc.cu", nv),
        ("mpc_horizon.cu", nv),
        ("mlp.cu", nv),
        ("fga_graph.cpp", None),
        ("fga_tile.cpp", None),
        ("fga_hinge.cpp", None),
        ("fga_batch.cpp", None),
        ("fga_mlp.cpp", None),
        ("fga_user.cpp", None),
    ]
    return [(s, f) for s, f in units if os.path.exists(os.path.join(CSRC, s))]


def _stale(objs):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    srcs.append(os.path.join(INCLUDE, "fgadmm.h"))
    srcs.append(os.path.abspath(__file__))
    return any(os.path.getmtime(s) > t for s in srcs if os.path.exists(s))


def build(force=False, verbose=False):
    """Compiles every translation unit and links libfgadmm.so; returns its path."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    units = _units()
    objs = [os.path.join(OUT, os.path.splitext(s)[0] + ".o") for s, _ in units]
    if not force and not _stale(objs):
        return LIB
    procs = []
    for (src, flags), obj in zip(units, objs):
        path = os.path.join(CSRC, src)
        if flags is None:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC,
                   "-I", os.path.join(cuda, "include"), "-c", path, "-o", obj]
        else:
            cmd = [nvcc] + ARCH + flags + ["-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("libfgadmm build failed:\n" + msg)
    tmp = LIB + ".%d.tmp" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-ldl"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libfgadmm link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
