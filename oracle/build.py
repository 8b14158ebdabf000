"""Build the FP64 CPU oracle (test infrastructure) as oracle/liborc.so.

Plain gcc, -O2, OpenMP across bundles only; no SIMD intrinsics, no
architecture flags, so the same source builds on x86_64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "orc.c")]
OUT = os.path.join(HERE, "liborc.so")


def build(force=False, verbose=False):
    hdr = os.path.join(HERE, "orc.h")
    if not force and os.path.exists(OUT):
        newest = max(os.path.getmtime(p) for p in SRC + [hdr, __file__])
        if os.path.getmtime(OUT) >= newest:
            return OUT
    tmp = OUT + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-Wall", "-Wextra", "-o", tmp] + SRC + ["-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
