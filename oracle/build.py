"""Compiles the C oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain IEEE arithmetic: no fast-math and no floating-point contraction, so that
every product and sum in the oracle rounds exactly as written.
"""
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SOURCES = [os.path.join(HERE, "dpr1_oracle.c"), os.path.join(HERE, "quad_ref.c")]
_LOCK = threading.Lock()


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SOURCES + [__file__])


def build_oracle(force=False):
    """Builds the oracle library if it is missing or older than its sources; returns its path.
    Safe to call from several threads and processes at once: one thread of a process builds, and
    each build writes a file of its own that replaces the library in one step."""
    with _LOCK:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        tmp = LIB + ".%d.%d.tmp" % (os.getpid(), threading.get_ident())
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp] + SOURCES + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
