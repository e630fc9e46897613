"""Compile the oracle's plain C into oracle/liboracle.so (gcc, -O2, no FP contraction).

Test infrastructure: building the checker is not using it. Run directly or via
__graft_entry__.build().
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liboracle.so")
SRCS = [os.path.join(HERE, "icarus_oracle.c"), os.path.join(HERE, "conv3d_oracle.c")]


def compile_so(srcs, out: str) -> str:
    """gcc the given C sources into the shared library `out` with the oracle's flags."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-std=gnu11", "-o", out + ".tmp"] + list(srcs) + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    srcs = [s for s in SRCS if os.path.exists(s)]
    if not force and os.path.exists(SO) and all(os.path.getmtime(SO) >= os.path.getmtime(s) for s in srcs):
        return SO
    return compile_so(srcs, SO)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
