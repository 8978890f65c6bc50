"""In-tree build of libemc.so with nvcc for sm_103a (no cmake, no torch
extension machinery): the translation units compile in parallel and link into
``paper_1707_09073_gb300/_build/libemc.so``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libemc.so")
UNITS = ["emc.cu", "inst_f32.cu", "inst_f64.cu", "mlp.cu", "thermal.cu"]
HEADERS = ["common.cuh", "kernels.cuh", "phonon.cuh", "trace.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
# the float (production) kernels use approximate division and square root;
# the double (parity) kernels and the host/Poisson unit stay IEEE
UNIT_FLAGS = {"inst_f32.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


BUILD_CHECKED = os.path.join(HERE, "_build_checked")


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile libemc.so.  checked=True builds the checked variant (array
    indices and positions verified in the kernels, a violation reported
    through the device error word) into _build_checked/ instead; load it by
    setting EMC_LIBRARY to the returned path before the first library call."""
    bdir = BUILD_CHECKED if checked else BUILD
    lib_path = os.path.join(bdir, "libemc.so")
    extra = ["-DEMC_CHECKED"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    deps_common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "emc.h")]
    nvcc = _nvcc()

    def one(unit: str) -> str:
        src = os.path.join(CSRC, unit)
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        if force or _stale(obj, [src] + deps_common):
            cmd = [nvcc] + ARCH + FLAGS + extra + UNIT_FLAGS.get(unit, []) + ["-c", src, "-o", obj + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
            os.replace(obj + ".tmp", obj)
            if verbose:
                print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    if force or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
