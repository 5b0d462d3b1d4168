"""Build and run the GB300 throughput probe (csrc/probe_peaks.cu): python -m paper_1912_10596_gb300.probe"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(HERE, "_build", "probe_peaks")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "csrc", "probe_peaks.cu")], check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
