"""Writes the stored expected values under tests/golden/ from the CPU oracle
alone (no CUDA code is imported).  Run: python tests/golden/make_golden.py"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def main():
    wl = synth.make_workload("block_20x20x10")
    d = oracle.forward(wl.mesh, wl.survey, wl.m)
    np.savetxt(os.path.join(HERE, "block_20x20x10_forward.txt"), d, fmt="%.17e",
               header="oracle forward d = G m (mGal), block_20x20x10 workload, station order of synth.grid_survey")


if __name__ == "__main__":
    main()
