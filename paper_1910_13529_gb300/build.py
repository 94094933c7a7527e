"""Compile libpic.so (the CUDA path) for sm_103a with nvcc, in-tree.

The translation units are compiled in parallel and linked with the static CUDA runtime;
the output goes to paper_1910_13529_gb300/_lib/libpic.so (git-ignored).
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libpic.so")
SOURCES = ["pic_api.cu", "field_kernels.cu", "particle_kernels.cu", "diag_kernels.cu", "adjoint_kernels.cu",
           "current_kernels.cu", "kspace_kernels.cu", "host_math.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _cufft_dir():
    """Directory of the toolkit's libcufft.so next to nvcc, or None (the k-space solvers are then
    built as stubs that refuse)."""
    import glob
    import shutil
    nvcc = shutil.which(NVCC)
    if not nvcc:
        return None
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for d in [os.path.join(root, "lib64")] + sorted(glob.glob(os.path.join(root, "targets", "*", "lib"))):
        if os.path.exists(os.path.join(d, "libcufft.so")) and os.path.exists(os.path.join(root, "include", "cufft.h")):
            return d
    return None


def _flags():
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "-I", os.path.join(HERE, "..", "include")]
    if _cufft_dir():
        f += ["-DPIC_HAVE_CUFFT"]
    return f


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "pic.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [NVCC] + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    fft = _cufft_dir()
    if fft:
        cmd += ["-L", fft, "-lcufft", "-Xlinker", "-rpath", "-Xlinker", fft]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
