"""Compile the CPU oracle (plain C, single-threaded) into a shared library.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg load the result.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sw_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "libsw_oracle.so")


def build(force: bool = False) -> str:
    """Build oracle/_build/libsw_oracle.so if missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [SRC, os.path.join(HERE, "sw_oracle.h")]
    if not force and os.path.exists(OUT):
        if os.path.getmtime(OUT) >= max(os.path.getmtime(d) for d in deps):
            return OUT
    tmp = OUT + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
