"""Build the FP64 CPU oracle shared library (test infrastructure only).

    python oracle/build.py            # writes oracle/librtlb_oracle.so
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rtlb_oracle.c")
LIB = os.path.join(HERE, "librtlb_oracle.so")


def build(force: bool = False) -> str:
    """Compile rtlb_oracle.c with gcc -O2 -fopenmp; returns the library path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
