"""Builds libbigmeans.so in-tree with nvcc for sm_103a (no cmake, no torch).

Each translation unit compiles in parallel; the shared library lands next to
this file, where the ctypes binding loads it.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libbigmeans.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


# Build variants: the product library, and two checking builds of the same
# sources that the tests load in child processes (never the product path):
#   guards: device index guards compiled in (BM_DEBUG_GUARDS; an access outside
#           its buffer is skipped and reported as BM_EGUARD);
#   asan:   host code instrumented with AddressSanitizer and
#           UndefinedBehaviorSanitizer (the process must preload their
#           runtimes).
VARIANTS = {
    "release": ([], [], "libbigmeans.so"),
    "guards": (["-DBM_DEBUG_GUARDS"], [], "libbigmeans_guards.so"),
    # (nvcc splits -Xcompiler values at commas: one flag per option)
    "asan": (["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
              "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize=vptr"],
             ["-lasan", "-lubsan"], "libbigmeans_asan.so"),
}


def variant_path(variant):
    """Where build(variant=...) puts that variant's library."""
    name = VARIANTS[variant][2]
    return LIB if variant == "release" else os.path.join(BUILD, variant, name)


def _compile(src, extra, outdir):
    obj = os.path.join(outdir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(verbose=False, ptxas_info=False, variant="release"):
    """Compile every .cu under csrc/ and link the variant's library (the
    in-tree libbigmeans.so for "release"); returns its path."""
    cflags, libs, _ = VARIANTS[variant]
    outdir = BUILD if variant == "release" else os.path.join(BUILD, variant)
    os.makedirs(outdir, exist_ok=True)
    extra = list(cflags) + (["-Xptxas", "-v"] if ptxas_info else [])
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, outdir), srcs))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    lib = variant_path(variant)
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", *libs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
