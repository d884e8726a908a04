"""Build the CPU oracle (plain C, FP64) into oracle/_build/libsrfmg_oracle.so.

The oracle is test infrastructure: only the tests, the package smoke check and
the benchmark's CPU-baseline leg load it.  It is compiled with
-ffp-contract=off so that no fused multiply-add changes its rounding on any
host (gcc contracts by default on aarch64).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "srfmg_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsrfmg_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
