"""Builds the FP64 CPU oracle (plain C) into oracle/_build/.

Test infrastructure: the oracle is the checker for the CUDA library and is
never linked into it.  `build()` compiles the default oracle; `build(mutant=k)`
compiles a copy with one planted mistake (see ORC_MUTANT in pic_oracle.c),
which the oracle's own self-test uses to show that its pins catch such
mistakes.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "pic_oracle.c")
SRCS = [SRC, os.path.join(HERE, "pic_oracle_adj.c")]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so"
    return os.path.join(BUILD_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    out = lib_path(mutant)
    hdr = os.path.join(HERE, "pic_oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max([os.path.getmtime(s) for s in SRCS] + [os.path.getmtime(hdr)])):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           f"-DORC_MUTANT={int(mutant)}", *SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


MT_SRCS = [SRC, os.path.join(HERE, "pic_oracle_mt.c")]


def build_mt(force: bool = False) -> str:
    """The multi-threaded CPU baseline (OpenMP): the serial oracle's functions
    plus pic_oracle_mt.c, in a library of its own."""
    out = os.path.join(BUILD_DIR, "liboracle_mt.so")
    hdr = os.path.join(HERE, "pic_oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max([os.path.getmtime(s) for s in MT_SRCS] + [os.path.getmtime(hdr)])):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", *MT_SRCS, "-o", tmp,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
