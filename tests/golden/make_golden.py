"""Write the oracle's stored expected values under tests/golden/.

Calls only ``oracle/``.  Run from the repository root:
    python tests/golden/make_golden.py
A change to any file this writes needs a commit message naming the passage of
the paper (or the reading of it) that justifies the change.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402


def write(name, header, values, fmt):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(header.rstrip() + "\n")
        for v in values:
            f.write(fmt(v) + "\n")


def main():
    # single stream of the default set, seed 0x12345678, Weyl on: first 1024 words
    g = O.Xorgens.param_set(0).seed(0x12345678)
    write("xorgens_128_95_seed12345678_u32_first1024.txt",
          "# oracle: param set (128,95,17,12,13,15), Weyl on, seed 0x12345678; "
          "output words 0..1023 (hex)", g.u32(1024), lambda v: f"{int(v):08x}")
    # the paper's set, seed 1 (first block id), first 256 words
    g = O.Xorgens.param_set(1).seed(1)
    write("xorgens_128_65_seed1_u32_first256.txt",
          "# oracle: param set (128,65,15,14,12,17), Weyl on, seed 1; "
          "output words 0..255 (hex)", g.u32(256), lambda v: f"{int(v):08x}")
    # FP64 normals of the default set, seed 7
    g = O.Xorgens.param_set(0).seed(7)
    write("xorgens_128_95_seed7_normal64_first256.txt",
          "# oracle: param set (128,95,17,12,13,15), Weyl on, seed 7; "
          "Box-Muller FP64 normals 0..255 (repr)", g.normal64(256), lambda v: repr(float(v)))


if __name__ == "__main__":
    main()
