"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

The paper prints no worked example (its spectra figures carry no data), so every
stored value here is the oracle's, written by this script and nothing else:

    python tests/golden/make_golden.py

conv4_k3_n8_sigma.txt: the 256 singular values of the 4->4 3x3 layer on the 8x8
torus (seed 1, N(0, 1/(c_in k^2)) weights from lfa_workloads), one frequency per
line in row-major order f = j*8 + l, descending within a line, computed by the
per-frequency FP64 LAPACK SVD (Algorithm 1) and checked here against the dense
256x256 operator's LAPACK SVD (the definition) before writing.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lfa_workloads as W  # noqa: E402
import oracle as O  # noqa: E402


def main():
    lay = W.layers("conv4_k3_n8")[0]
    w = W.weights(lay)
    s = O.lfa_svd(w, lay.n, lay.m, compute_uv=False)
    dense = np.sort(O.dense_svd(w, lay.n, lay.m))[::-1]
    assert np.max(np.abs(np.sort(s.ravel())[::-1] - dense)) <= 1e-12 * dense[0]
    path = os.path.join(HERE, "conv4_k3_n8_sigma.txt")
    with open(path, "w") as fh:
        fh.write("# sigma of the 4->4 3x3 periodic conv on 8x8 (seed 1); row f = j*8 + l, descending\n")
        for row in s:
            fh.write(" ".join(f"{v:.17e}" for v in row) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
