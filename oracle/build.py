"""Compiles the CPU oracle (sw_oracle.c, discovery_oracle.c, filter_oracle.c) into
oracle/_build/liboracle.so.

Test infrastructure only: the product path never loads this library.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "sw_oracle.c"), os.path.join(HERE, "discovery_oracle.c"),
        os.path.join(HERE, "filter_oracle.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def command():
    return ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
            "-Wall", "-Wextra", "-o", LIB, *SRCS]


def build(force=False):
    """Builds the library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(src) for src in SRCS)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    subprocess.run(command(), check=True)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
