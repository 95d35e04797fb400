"""Build step of the oracle (test infrastructure): compiles soma_oracle.c into
liboracle.so with the host C compiler.  FP contraction is switched off so the
FP64 arithmetic is the same on x86-64 and AArch64 hosts."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose: bool = False) -> str:
    src = os.path.join(_HERE, "soma_oracle.c")
    out = os.path.join(_HERE, "liboracle.so")
    tmp = f"{out}.tmp{os.getpid()}"   # concurrent builds (parallel test workers) do not collide
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
