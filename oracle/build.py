"""Compile the CPU oracle into oracle/_build/liboracle.so with gcc.

Test infrastructure: the oracle is built so the test suite, the smoke check
and the benchmark's CPU-baseline leg can load it.  Plain C11, no
architecture-specific flags (the same source builds on x86_64 and aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c")]


def needs_build() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    lib_mtime = os.path.getmtime(LIB_PATH)
    deps = SOURCES + [os.path.join(HERE, "oracle.h")]
    return any(os.path.getmtime(p) > lib_mtime for p in deps)


def build(force: bool = False) -> str:
    if not force and not needs_build():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", tmp] + SOURCES + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
