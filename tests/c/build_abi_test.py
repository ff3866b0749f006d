"""Builds tests/c/dock_abi_test (a plain C11 client of include/dock.h) against libdock.so."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(HERE, "dock_abi_test.c")
OUT = os.path.join(HERE, "_build", "dock_abi_test")


def build(lib_path: str) -> str:
    """Compiles the test client with gcc (C11, warnings as errors) and links it to `lib_path`."""
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC, os.path.join(ROOT, "include", "dock.h"), lib_path]
    if not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in deps):
        lib_dir = os.path.dirname(lib_path)
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", "-I",
                               os.path.join(ROOT, "include"), SRC, "-o", tmp, "-L", lib_dir, "-ldock",
                               f"-Wl,-rpath,{lib_dir}"])
        os.replace(tmp, OUT)
    return OUT
