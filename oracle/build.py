"""Build the C oracle (``numa_oracle.c``) into ``liboracle_numa.so`` beside it.

Test infrastructure only: the oracle is a plain FP64 CPU statement of the
element volume term and is never part of the GPU product path.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "numa_oracle.c")
LIB = os.path.join(HERE, "liboracle_numa.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc; rebuild when the source is newer."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
            "-ffp-contract=off", "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # No OpenMP runtime: the pragmas are ignored and O2 runs on one thread.
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
