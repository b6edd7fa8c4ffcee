"""Compile the oracle's C helper (oracle/kmvm64.c) into oracle/lib/liboracle64.so.

TEST INFRASTRUCTURE ONLY (see krr_oracle.py).  gcc with OpenMP when available, else a
serial build; a content hash avoids rebuilding an unchanged source.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kmvm64.c")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "liboracle64.so")


def build(force: bool = False) -> str:
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle helper")
    with open(SRC, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    stamp = os.path.join(LIBDIR, "liboracle64.sha256")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = LIB + ".tmp"
    base = [cc, "-O2", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    res = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
    if res.returncode != 0:
        res = subprocess.run(base, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"oracle helper build failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
