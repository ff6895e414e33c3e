"""Builds libgrins_racipe.so in this folder with nvcc for sm_103a.

Each CUDA translation unit is compiled in parallel, then linked into one
shared library.  Host code is compiled without floating-point contraction
(the half-functional median table must be reproducible bit for bit).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgrins_racipe.so")

SOURCES = ["api.cu", "sample.cu", "integrate_generic.cu", "integrate_grp2.cu", "integrate_grp4.cu",
           "integrate_grp6.cu", "integrate_grp8.cu", "integrate_grp12.cu", "polish.cu", "unique.cu",
           "jit.cu", "integrate_batch.cu", "levels.cu", "ising.cu", "tail.cu", "rates.cu"]

# Sources the run-time compile of the lane-group kernel needs (jit.cu embeds
# them as string literals): (include name, path).
JIT_SOURCES = [("grins_racipe.h", os.path.join(INCLUDE, "grins_racipe.h")),
               ("common.cuh", os.path.join(CSRC, "common.cuh")),
               ("integrate.cuh", os.path.join(CSRC, "integrate.cuh")),
               ("dd.cuh", os.path.join(CSRC, "dd.cuh")),
               ("integrate_grp.cuh", os.path.join(CSRC, "integrate_grp.cuh")),
               ("integrate_rr.cuh", os.path.join(CSRC, "integrate_rr.cuh")),
               ("integrate_rr_layout.inc", os.path.join(CSRC, "integrate_rr_layout.inc")),
               ("integrate_plan.cuh", os.path.join(CSRC, "integrate_plan.cuh"))]


def write_jit_sources(bdir):
    """jit_sources.inc: the JIT_SOURCES files as C++ raw string literals."""
    parts = []
    for name, path in JIT_SOURCES:
        text = open(path).read()
        assert ")GRINSJIT\"" not in text
        parts.append('R"GRINSJIT(' + text + ')GRINSJIT"')
    inc = ("static const int kJitSourceCount = %d;\n" % len(JIT_SOURCES)
           + "static const char *const kJitSourceNames[] = {"
           + ", ".join('"%s"' % n for n, _ in JIT_SOURCES) + "};\n"
           + "static const char *const kJitSources[] = {\n" + ",\n".join(parts) + "};\n")
    path = os.path.join(bdir, "jit_sources.inc")
    if not os.path.exists(path) or open(path).read() != inc:
        with open(path, "w") as f:
            f.write(inc)

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(INCLUDE, "grins_racipe.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


LIB_CHECKED = os.path.join(HERE, "libgrins_racipe_checked.so")


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    return os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime()


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          checked: bool = False) -> str:
    """Builds the library; `checked` builds the index/alignment-checked
    variant libgrins_racipe_checked.so (-DGRINS_CHECKED) used by the tests."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return lib
    bdir = BUILD + ("_checked" if checked else "")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    write_jit_sources(bdir)
    flags = NVCC_FLAGS + ["-I" + bdir] + (["-DGRINS_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    # longest translation units first so the parallel build ends sooner
    order = sorted(SOURCES, key=lambda s: 0 if "grp" in s else 1)
    with ThreadPoolExecutor(jobs or min(len(order), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, order))
    tmp = lib + ".tmp.%d" % os.getpid()
    subprocess.check_call([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-o", tmp] + objs + ["-ldl"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
