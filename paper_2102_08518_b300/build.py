"""Build the native library libls.so in-tree (nvcc, sm_103a).

The library holds the C ABI (include/lattice_spline.h), the code generator, the
NVRTC driver and the spline-independent kernels.  Spline kernels are generated
and compiled by the library itself at ls_spline_create (or ls_spline_precompile).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libls.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cpp", ".cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    deps.append(os.path.join(ROOT, "include", "lattice_spline.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [os.path.join(CUDA, "bin", "nvcc"), "-shared", "-Xcompiler", "-fPIC", *ARCH, "-lineinfo", "-O3",
           "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-o", tmp, *sources(),
           f"-L{CUDA}/lib64", "-lnvrtc", f"-Xlinker=-rpath,{CUDA}/lib64", "-Xptxas", "-v" if verbose else "-O3"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
