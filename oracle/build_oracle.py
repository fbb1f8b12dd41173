"""Compile the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain gcc, -ffp-contract=off so that no multiply-add is fused: every expression
is evaluated as written on x86_64 and aarch64 alike. Built with OpenMP when the compiler
has it: a step's actions may then be valued on several threads (orc_set_threads), which
changes no result.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fmdp_oracle.c")
HDR = os.path.join(HERE, "fmdp_oracle.h")
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")


def stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in (SRC, HDR, __file__))


def build(force: bool = False) -> str:
    if force or stale():
        os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wextra", "-Wno-unused-parameter", SRC, "-o", tmp, "-lm"]
        # OpenMP (for the multi-core timing of the CPU baseline) when the compiler has it
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
