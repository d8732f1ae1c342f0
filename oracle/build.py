"""Compile the C oracle into oracle/_build/liboracle.so (test infrastructure only).

Plain gcc, no architecture-specific flags, so the same source builds on x86-64 and on
the Arm hosts that carry the GPUs.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["ring.c", "transforms.c", "zx.c", "sn.c"]
LIB = os.path.join(HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr, __file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-Wno-unused-parameter", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
