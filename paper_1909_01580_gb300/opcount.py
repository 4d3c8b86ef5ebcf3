"""Counts the arithmetic of the hot path per unit of work by compiling
csrc/opcount.cpp (the device templates instantiated on the host with a
counting scalar) and running it.  A measurement tool: prints JSON."""
import json
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def counts() -> dict:
    src = os.path.join(HERE, "csrc", "opcount.cpp")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "opcount")
        subprocess.run(["g++", "-std=c++17", "-O1", "-I/usr/local/cuda/include", src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


if __name__ == "__main__":
    print(json.dumps(counts(), indent=1))
