"""Build the in-tree shared library ``libdgwave.so`` (C ABI of include/dgwave.h)
for sm_103a with nvcc.  Translation units compile in parallel; the link step
produces ``paper_1304_5546_gb300/libdgwave.so``.  ``build(checked=True)``
builds the same sources with DGW_DEVICE_CHECKS into ``libdgwave_checked.so``:
the stage kernels then test the face connection codes and block-table
entries they read before using them, and report DG_ERR_INDEX instead of
faulting."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdgwave.so")
LIB_CHECKED = os.path.join(PKG, "libdgwave_checked.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    names = (["host_setup.cpp", "api.cu"] + ["kernels_N%d.cu" % n for n in range(1, 8)]
             + ["kernels_tc_N%d.cu" % n for n in range(1, 8)]
             + ["kernels_tcp_N%d.cu" % n for n in range(1, 8)]
             + ["kernels_ept_N%d.cu" % n for n in range(1, 6)]
             + ["kernels_batch_s1.cu", "kernels_batch_s2.cu", "batch.cu", "server.cu", "checkpoint.cu",
                  "partition.cu"])
    return [os.path.join(CSRC, n) for n in names]


def _deps():
    return ([os.path.join(CSRC, f) for f in os.listdir(CSRC)]
            + [os.path.join(INCLUDE, "dgwave.h"), os.path.abspath(__file__)])


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False, extra_flags=(), checked=False):
    """Compile and link the library (the checked build with checked=True);
    returns its path."""
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    if checked:
        extra_flags = tuple(extra_flags) + ("-DDGW_DEVICE_CHECKS",)
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *COMMON, *ARCH, *extra_flags, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++", *COMMON, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    workers = min(len(sources()), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib



# Source files that define each stage-kernel family (kernel_source_hash)
KERNEL_FAMILIES = {
    "tc": lambda n: (n.startswith("kernels_tc") or n == "kernels.cuh"
                     or n in ("launch.h", "ptx.cuh")),
    "ept": lambda n: (n.startswith("kernels_ept") or n == "kernels.cuh"
                      or n in ("launch.h", "ptx.cuh")),
}


def kernel_source_hash(family=None):
    """Short hash of the kernel sources (code only: // comments, trailing
    blanks and empty lines are left out); profiles record it so that stale
    counter captures are not reported for a changed kernel.  family: only
    the files of one stage-kernel family (KERNEL_FAMILIES: the tensor-core
    kernel "tc", the element-thread kernel "ept"); None: every kernel
    source."""
    import hashlib
    import re
    h = hashlib.sha256()
    pick = KERNEL_FAMILIES[family] if family else (
        lambda n: n.startswith("kernels") or n in ("launch.h", "ptx.cuh"))
    for name in sorted(os.listdir(CSRC)):
        if pick(name):
            with open(os.path.join(CSRC, name), encoding="utf-8") as f:
                lines = (re.sub(r"//.*$", "", line).rstrip() for line in f)
                code = "\n".join(line for line in lines if line)
            h.update(name.encode() + code.encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
