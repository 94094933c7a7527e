"""Build the FP64 CPU oracle (test infrastructure only) with plain gcc.

The oracle is a checker for the CUDA path; building it is not using it.  Only
tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
load the resulting library.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pic_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into oracle/_build/liboracle.so (portable flags, no -march)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", SRC, "-o", tmp]
    # OpenMP (for the all-cores CPU baseline) when the compiler has it; plain otherwise
    r = subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
