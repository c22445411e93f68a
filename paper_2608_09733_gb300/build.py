"""Builds libsv.so in-tree for sm_103a (nvcc, one -gencode, parallel compiles).

    python -m paper_2608_09733_gb300.build [--force]

The library lands in ``paper_2608_09733_gb300/_build/libsv.so`` (git-ignored).
A stamp of the source contents and flags skips the build when nothing changed.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsv.so")

SOURCES = ["sv_plan.cpp", "sv_program.cpp", "sv_api.cpp", "sv_adjoint_host.cpp", "sv_serve.cpp", "sv_jit.cpp",
           "sv_sweep.cu", "sv_reduce.cu", "sv_adjoint.cu", "sv_noalloc.cu", "sv_sample.cu",
           "sv_hostcopy.cu"]
# Device headers the run-time compiled pass kernels include (sv_jit.cpp): their
# text is embedded in the library, so a kernel compiled at run time is built
# from the same code as the library's own pass kernel.
JIT_HEADERS = ["sv_prog_layout.h", "sv_pass_ops.cuh", "sv_tma_pass.cuh", "sv_batch_layout.h", "sv_batch_ops.cuh"]
HEADERS = ["sv_internal.h", "sv_adjoint.h"] + JIT_HEADERS
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + OUT]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsv.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stamp(extra=()) -> str:
    h = hashlib.sha256()
    for f in _sources() + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "include", "sv.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


# Sources that decide what the pass kernel does (the kernel, the program
# builder, the planner and the shared structures).
SWEEP_SOURCES = ["sv_sweep.cu", "sv_program.cpp", "sv_plan.cpp", "sv_internal.h", "sv_jit.cpp", "sv_prog_layout.h",
                 "sv_pass_ops.cuh", "sv_tma_pass.cuh"]


def sweep_stamp() -> str:
    """Hash of the pass kernel's sources and flags: ncu counters recorded
    for one stamp say nothing about another."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    # flags without the include directory: that path differs between checkouts
    # of the same sources, so it must not change the stamp
    h.update(" ".join(ARCH + [f for f in FLAGS if not f.startswith("-I")]).encode())
    return h.hexdigest()


def write_jit_headers() -> None:
    """Writes _build/sv_jit_headers.inc: the device headers as string
    literals (names and texts) for the run-time compiler."""
    names, texts = [], []
    for f in JIT_HEADERS:
        with open(os.path.join(CSRC, f)) as fh:
            body = fh.read()
        if ")svjit\"" in body:
            raise RuntimeError("%s holds the raw-string delimiter" % f)
        names.append('"%s"' % f)
        texts.append('R"svjit(' + body + ')svjit"')
    out = ("// written by build.py from " + ", ".join(JIT_HEADERS) + "\n"
           "static const char* const kJitHeaderNames[] = {" + ", ".join(names) + "};\n"
           "static const char* const kJitHeaderTexts[] = {\n" + ",\n".join(texts) + "};\n")
    path = os.path.join(OUT, "sv_jit_headers.inc")
    old = None
    if os.path.exists(path):
        with open(path) as fh:
            old = fh.read()
    if old != out:
        with open(path, "w") as fh:
            fh.write(out)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    write_jit_headers()
    stamp_file = os.path.join(OUT, "libsv.stamp")
    stamp = _stamp(extra_flags)
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return LIB
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + ARCH + FLAGS + list(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
