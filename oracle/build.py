"""Build the C oracle into oracle/_build/liboracle.so.

The oracle is test infrastructure: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py load it.  Compiled with plain gcc (OpenMP for the
per-cell / per-ordinate loops), no fast-math, so IEEE double rounding holds.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oci_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, src: str = SRC, out: str = LIB, extra_flags=()) -> str:
    """Compile `src` to the shared library `out` if it is missing or stale."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-Wall", "-Wno-unknown-pragmas",
           *extra_flags, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force=True))
