"""Build the CPU oracle (test infrastructure) into oracle/liboracle.so.

Compiled with -ffp-contract=off so that the same source gives the same roundings on x86-64 and
on aarch64 (gcc contracts a*b+c into fused multiply-adds by default on aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["oracle.cpp"]
HEADERS = ["dual.hpp", "systems.hpp", "tableaux.hpp"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def compile_lib(src_dir: str, out: str) -> str:
    """Compile the oracle sources found in src_dir into the shared library `out`."""
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", out + ".tmp"] + [os.path.join(src_dir, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    if not force and not _stale():
        return LIB
    return compile_lib(HERE, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
