"""Compile the serial CPU oracle (test infrastructure only).

Two shared libraries are built from ``tdse_oracle.c`` with plain gcc:
``liboracle_f64.so`` (REAL = double) and ``liboracle_fld.so`` (REAL = long
double, the rounding-floor instrument).  ``-ffp-contract=off`` keeps the
evaluation order as written, so x86 and Arm builds round identically.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tdse_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
FLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
VARIANTS = {"f64": [], "fld": ["-DORC_LONG_DOUBLE"]}


def lib_path(precision: str) -> str:
    return os.path.join(OUT_DIR, f"liboracle_{precision}.so")


def build(force: bool = False) -> None:
    os.makedirs(OUT_DIR, exist_ok=True)
    for name, extra in VARIANTS.items():
        out = lib_path(name)
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(SRC)):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", *FLAGS, *extra, "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print("oracle built in", OUT_DIR)
