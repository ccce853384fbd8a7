"""Pipe-throughput probe of the GPU (FP64 / FP32 FMA, integer multiply-add,
shared-memory atomics): builds diag/pipes_probe.cu with nvcc and runs it.
Used to decide how the numeric phase accumulates (float64 FMA vs float32
pairs); prints one line per pipe."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    src = os.path.join(HERE, "pipes_probe.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "pipes_probe")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
