"""The stored oracle values in tests/golden/ still match the oracle and the dense definition."""
import os

import numpy as np

import lfa_workloads as W
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "conv4_k3_n8_sigma.txt")


def test_conv4_golden_matches_dense_definition():
    lay = W.layers("conv4_k3_n8")[0]
    w = W.weights(lay)
    s = np.loadtxt(GOLD)
    assert s.shape == (64, 4)
    dense = np.sort(O.dense_svd(w, lay.n, lay.m))[::-1]
    np.testing.assert_allclose(np.sort(s.ravel())[::-1], dense, atol=1e-12 * dense[0])
    np.testing.assert_allclose(s, O.lfa_svd(w, lay.n, lay.m, compute_uv=False), atol=1e-14)
