"""Compile oracle.c into an in-tree shared library (gcc, no GPU).

Part of the test infrastructure: building the checker is not using it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
OUT = os.path.join(HERE, "_build", "liborc_bsde.so")


def build(force=False):
    """Return the path of the compiled oracle, rebuilding it when stale."""
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    stale = force or not os.path.exists(OUT) or any(
        os.path.getmtime(f) > os.path.getmtime(OUT) for f in (SRC, HDR, __file__))
    if stale:
        tmp = OUT + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
