"""Compile the CPU oracle (plain C++17, host compiler only) into oracle/liboracle.so."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def command():
    return ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
            os.path.join(HERE, "oracle.cpp"), "-o", os.path.join(HERE, "liboracle.so")]


def build():
    subprocess.run(command(), check=True)


if __name__ == "__main__":
    build()
