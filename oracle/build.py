"""Build the C oracle into oracle/liboracle.so with gcc.

Test infrastructure only: the product library never links or loads it.
``-ffp-contract=off`` keeps every floating-point operation a separately
rounded IEEE operation in source order.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "helk_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
           "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp, SRC, "-lm",
           "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
