"""Builds the FP64 oracle (test infrastructure) as oracle/_build/libpbng_oracle.so.

Plain portable C++17 (no architecture flags) so the same source builds on the
x86 development host and the Arm GPU host.  OpenMP is used when the compiler
supports it; the results do not depend on it.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pbng_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpbng_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "pbng_oracle.h")))):
        return LIB
    cxx = os.environ.get("CXX", "g++")
    base = [cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", SRC, "-o", LIB + ".tmp"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            break
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
