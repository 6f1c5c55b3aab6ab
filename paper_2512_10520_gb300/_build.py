"""Build libmt.so in-tree for sm_103a with nvcc (no CMake, no torch extension machinery)."""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
from typing import List, Optional

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
OBJ_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libmt.so")
SOURCES = ["api.cu", "transport.cu", "compact.cu", "noalloc.cu", "adjoint.cu", "batched.cu", "offline.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or cand)


def _cuda_lib_dir() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "lib64")


def _stale(target: str, deps: List[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: Optional[List[str]] = None,
          out_path: Optional[str] = None, obj_dir: Optional[str] = None) -> str:
    """Compile every CUDA translation unit (in parallel) and link libmt.so; returns its path.

    ``out_path`` / ``obj_dir`` / ``extra_flags`` (e.g. ``-DMT_PASS_MIN_BLOCKS=5``) build a
    tuning variant of the library elsewhere without touching the default one."""
    lib_path = out_path or LIB_PATH
    odir = obj_dir or OBJ_DIR
    os.makedirs(odir, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    flags = ARCH + ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-Xcompiler", "-Wall"] + (extra_flags or [])
    if verbose:
        flags += ["-Xptxas", "-v"]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(odir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + flags + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    logs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for out in ex.map(run, jobs):
            logs.append(out)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        libdir = _cuda_lib_dir()
        logs.append(run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs +
                        ["-cudart", "shared", "-Xlinker", f"-rpath,{libdir}"]))
        os.replace(tmp, lib_path)
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return lib_path
