"""Build and run the pipe-throughput probe (csrc/probe_pipes.cu) on GPU 0."""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    src = os.path.join(HERE, "csrc", "probe_pipes.cu")
    exe = os.path.join(HERE, "probe_pipes")
    subprocess.run(["/usr/local/cuda/bin/nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
