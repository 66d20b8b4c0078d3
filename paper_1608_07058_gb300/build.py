"""Build the CUDA library libmatleap.so in-tree for sm_103a.

Each kernel variant is its own translation unit (precision x table capacity), compiled
in parallel; the reference-precision units get -fmad=false so that no multiply-add is
contracted.  Objects go to _build/ next to this file; the library next to this file.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmatleap.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
N_THREAD_VARIANTS = 4


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


# The generic thread variant (8 species x 16 reactions) is large: its kernels are
# compiled as separate units (ML_PART) so that they build in parallel.
SPLIT_VARIANTS = (N_THREAD_VARIANTS - 1,)


def _thread_units(name, flags, v, parts):
    if v not in SPLIT_VARIANTS:
        return [("kern_thread.cu", f"kt_{name}_{v}.o", flags)]
    return [("kern_thread.cu", f"kt_{name}_{v}_p{k}.o", flags + [f"-DML_PART={k}"])
            for k in parts]


def _units():
    u = []
    for fast in (0, 1):
        for v in range(N_THREAD_VARIANTS):
            u += _thread_units("fast" if fast else "ref", [f"-DML_FAST={fast}", f"-DML_VARIANT={v}"]
                               + ([] if fast else ["-fmad=false"]), v, (0, 1, 2, 3))
        if fast:
            for v in range(N_THREAD_VARIANTS):
                u += _thread_units("fastocc", ["-DML_FAST=1", f"-DML_VARIANT={v}",
                                               "-DML_THREAD_MIN_BLOCKS=2"], v, (0, 1, 3))
        u.append(("kern_warp.cu", f"kw_{'fast' if fast else 'ref'}.o",
                  [f"-DML_FAST={fast}"] + ([] if fast else ["-fmad=false"])))
    u.append(("api.cu", "api.o", []))
    u.append(("jit.cu", "jit.o", []))
    u.append(("noalloc.cu", "noalloc.o", []))
    u.append(("server.cu", "server.o", []))
    u.append(("bayes.cu", "bayes.o", ["-fmad=false"]))
    u.append(("metrics.cu", "metrics.o", ["-fmad=false"]))
    u.append(("peaks.cu", "peaks.o", []))
    return u


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "matleap.h")]


# Headers compiled again at run time for the model-specialized kernels (jit.cu): embedded
# into the library as strings, so the library does not need its source tree at run time.
JIT_HEADERS = [("thread_core.cuh", CSRC), ("dev_common.cuh", CSRC), ("ml_internal.h", CSRC),
               ("matleap.h", INCLUDE)]


def _write_jit_sources():
    out = ["// Generated by build.py: kernel headers for runtime compilation.", "#pragma once",
           f"constexpr int kJitHeaderCount = {len(JIT_HEADERS)};"]
    names, texts = [], []
    for name, d in JIT_HEADERS:
        text = open(os.path.join(d, name)).read()
        assert ")MLJIT\"" not in text
        names.append(f'"{name}"')
        texts.append('R"MLJIT(' + text + ')MLJIT"')
    out.append("static const char* const kJitHeaderName[] = {" + ", ".join(names) + "};")
    out.append("static const char* const kJitHeaderText[] = {\n" + ",\n".join(texts) + "};")
    path = os.path.join(BUILD, "jit_sources.h")
    text = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)


def _cuda_lib_dir(nvcc):
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for d in (os.path.join(root, "lib64"), os.path.join(root, "lib")):
        if os.path.exists(os.path.join(d, "libnvrtc.so")):
            return d
    raise RuntimeError(f"libnvrtc.so not found next to {nvcc}")


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_sources()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, "-I", BUILD]
    jobs = []
    for src, obj, flags in _units():
        cmd = common + flags + ["-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    # the generic variant's units take longest: start them first
    heavy = [f"-DML_VARIANT={v}" for v in SPLIT_VARIANTS]
    jobs.sort(key=lambda c: 0 if any(h in c for h in heavy) else 1)
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, res in zip(jobs, results):
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{res.stderr}")
    objs = [os.path.join(BUILD, o) for _, o, _ in _units()]
    tmp = LIB + ".tmp"
    libdir = _cuda_lib_dir(nvcc)
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-L", libdir, "-lnvrtc",
            "-Xlinker", "-rpath", "-Xlinker", libdir]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
