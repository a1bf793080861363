"""Builds the CUDA library libpm_gb300.so in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
SOURCES = ["pm_api.cu", "pm_sweep_f32_t0.cu", "pm_sweep_f32_t1.cu", "pm_sweep_f32_t2.cu", "pm_sweep_f64_t0.cu",
           "pm_sweep_f32_tr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def lib_path() -> str:
    return os.path.join(HERE, "_lib", f"libpm_gb300_{platform.machine()}.so")


def _newest_source_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(ROOT, "include", "poremaps_gb.h"))
    return max(os.path.getmtime(p) for p in paths)


def _nvcc() -> str:
    nvcc = os.environ.get("NVCC", "nvcc")
    if not os.path.isabs(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
        nvcc = "/usr/local/cuda/bin/nvcc"
    return nvcc


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every translation unit (in parallel) and links the shared library."""
    from concurrent.futures import ThreadPoolExecutor

    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_source_mtime():
        return out
    objdir = os.path.join(HERE, "_lib", f"obj_{platform.machine()}_{os.getpid()}")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", *objs, "-o", tmp], check=True)
    os.replace(tmp, out)
    for o in objs:
        os.remove(o)
    os.rmdir(objdir)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
