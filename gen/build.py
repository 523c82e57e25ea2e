"""Compile the workload generator (host + sm_103a kernels) into gen/libmpsm_gen.so."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def command():
    return ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
            os.path.join(HERE, "gen.cu"), "-o", os.path.join(HERE, "libmpsm_gen.so")]


def build():
    subprocess.run(command(), check=True)


if __name__ == "__main__":
    build()
