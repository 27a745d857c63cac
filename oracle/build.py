"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liblhmm_oracle.so.

Plain gcc, OpenMP over boxes.  No flags that tie the object to one CPU
family, so the same source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["micro_oracle.c", "sph_oracle.c", "mlp_oracle.c"]
LIB = os.path.join(HERE, "liblhmm_oracle.so")


def build_oracle(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "lhmm_oracle.h")]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in deps)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-fopenmp", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
