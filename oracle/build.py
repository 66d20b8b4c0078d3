"""Build the CPU oracle (test infrastructure) into oracle/libml_oracle.so.

Plain gcc, single translation unit, -ffp-contract=off so that no multiply-add is fused
and every floating-point operation rounds once, in source order.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ml_oracle.c")
LIB = os.path.join(HERE, "libml_oracle.so")


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    out = LIB if not extra_flags else os.path.join(
        HERE, "libml_oracle_" + "_".join(f.strip("-").replace("=", "") for f in extra_flags) + ".so")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "ml_oracle.h")))):
        return out
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wextra", *extra_flags, SRC, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
