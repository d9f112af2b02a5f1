"""Build the CPU oracle shared library (test infrastructure only).

Compiles ``drtopk_oracle.cpp`` with the host C++ compiler into
``oracle/_build/liboracle.so``. Plain portable C++17 with OpenMP (used only
by the chunked multi-core variant): no architecture flags, so the same
source builds on x86_64 and aarch64.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "drtopk_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-fopenmp", "-shared", SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
