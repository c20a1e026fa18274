"""Build libbbfmm.so (the CUDA library behind include/bbfmm.h) in-tree.

Every translation unit under csrc/ is compiled by nvcc for sm_103a only, in
parallel, then linked into ``paper_1903_02153_gb300/_lib/libbbfmm.so``.  A
hash of the sources and flags skips the work when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libbbfmm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC,-fopenmp,-O3", "-I", os.path.join(ROOT, "include"), "-I", BUILD]
# headers whose text the library embeds for run-time compilation (NVRTC) of
# user-supplied kernels, in include order
NVRTC_HEADERS = ["morton.cuh", "p2p_kernels.cuh"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _digest():
    h = hashlib.sha256()
    h.update(" ".join(NVCC_FLAGS).encode())
    for f in sorted(os.listdir(CSRC)) + [os.path.join("..", "..", "include", "bbfmm.h")]:
        path = os.path.join(CSRC, f)
        h.update(f.encode())
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _c_string(text):
    out = []
    for line in text.splitlines(True):
        esc = line.replace("\\", "\\\\").replace('"', '\\"').replace("\n", "\\n")
        out.append('"%s"' % esc)
    return "\n".join(out) if out else '""'


def write_nvrtc_headers():
    """Write _build/nvrtc_headers.inc: the {name, text} of every header in
    NVRTC_HEADERS, as C string literals."""
    parts = ["// generated by build.py from csrc/ (do not edit)",
             "struct NvrtcHeader { const char *name, *text; };",
             "static const NvrtcHeader kNvrtcHeaders[] = {"]
    for name in NVRTC_HEADERS:
        with open(os.path.join(CSRC, name)) as fh:
            parts.append('    {"%s",\n%s},' % (name, _c_string(fh.read())))
    parts.append("};")
    path = os.path.join(BUILD, "nvrtc_headers.inc")
    with open(path, "w") as fh:
        fh.write("\n".join(parts) + "\n")
    return path


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()
    write_nvrtc_headers()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu"] + NVCC_FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
