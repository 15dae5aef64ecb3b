"""Build the FP64 CPU oracle shared libraries (test infrastructure only).

The oracle is plain C compiled without floating-point contraction so that the
same source gives the same bits on x86_64 and aarch64 hosts.  Two builds of the
one source:
  liblbe_oracle.so      single-threaded: the parity reference of the tests;
  liblbe_oracle_omp.so  the same source with -fopenmp, its per-node loops
                        spread over the host cores: the timed CPU baseline.
Both give the same numbers (each node's arithmetic is unchanged; the one
reduction, the plane flux, stays serial).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["lbe_oracle.c"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbe_oracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liblbe_oracle_omp.so")


def _build_one(out, extra, force):
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.abspath(__file__)])
        if os.path.getmtime(out) >= newest:
            return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + extra + \
          ["-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False, openmp: bool = False) -> str:
    """Path of the single-threaded oracle library, or of the OpenMP timing build."""
    if openmp:
        return _build_one(LIB_OMP, ["-fopenmp"], force)
    return _build_one(LIB, [], force)


if __name__ == "__main__":
    f = "--force" in sys.argv
    print(build(force=f))
    print(build(force=f, openmp=True))
