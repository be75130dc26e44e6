"""Build of libmadflow_gb.so for sm_103a (in-tree, into ``_build/``).

The device headers under ``csrc/device`` are embedded into the library as
strings (NVRTC compiles the per-process kernels at run time from them); the
host library and the Vegas kernels are compiled with nvcc for sm_103a.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmadflow_gb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
EMBED = ["mf_common.cuh", "mf_dual.cuh", "mf_kinematics.cuh", "mf_helas.cuh", "mf_kparams.h", "mf_kernel.cuh",
         "mf_helas_adj.cuh", "mf_grad.cuh", "mf_tc.cuh", "mf_channels.cuh"]
SOURCES = ["mf_api.cu", "mf_colour.cu", "mf_peaks.cu", "mf_codegen.cpp", "mf_jit.cpp", "mf_lhe.cpp",
           "mf_channels.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _embed() -> str:
    out = ["// generated by build.py: device headers for run-time compilation"]
    names, bodies = [], []
    for name in EMBED:
        with open(os.path.join(CSRC, "device", name)) as fh:
            text = fh.read()
        if ")MFSRC\"" in text:
            raise RuntimeError("delimiter clash")
        names.append(f'"{name}"')
        bodies.append('R"MFSRC(' + text + ')MFSRC"')
    out.append(f"static const int kNumHeaders = {len(EMBED)};")
    out.append("static const char *kHeaderNames[] = {" + ", ".join(names) + "};")
    out.append("static const char *kHeaderSources[] = {\n" + ",\n".join(bodies) + "\n};")
    return "\n".join(out) + "\n"


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    inc = os.path.join(BUILD, "_embedded_sources.inc")
    text = _embed()
    if force or not os.path.exists(inc) or open(inc).read() != text:
        with open(inc, "w") as fh:
            fh.write(text)
    nvcc = _nvcc()
    home = _cuda_home(nvcc)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    headers += [os.path.join(CSRC, "device", f) for f in os.listdir(os.path.join(CSRC, "device"))]
    headers += [os.path.join(os.path.dirname(HERE), "include", "madflow_gb.h"), inc]
    lib64 = os.path.join(home, "lib64")
    if not os.path.isdir(lib64):
        lib64 = os.path.join(home, "lib")
    nvrtc = [f for f in sorted(os.listdir(lib64)) if f.startswith("libnvrtc.so.") and f.count(".") == 2]
    nvrtc_path = os.path.join(lib64, nvrtc[0]) if nvrtc else "libnvrtc.so.13"
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "-I", BUILD, "-I", CSRC,
              "-I", os.path.join(home, "include"), f'-DMF_NVRTC_DEFAULT="{nvrtc_path}"']
    objs, jobs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        path = os.path.join(CSRC, src)
        if force or _stale(obj, [path] + headers):
            jobs.append([nvcc, *ARCH, *common, "-c", path, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            if res.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-L", lib64, "-ldl", "-lpthread", "-cudart", "shared",
               "-Xlinker", f"-rpath={lib64}"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or res.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
        if res.returncode:
            raise RuntimeError("link of libmadflow_gb.so failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
