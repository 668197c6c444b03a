"""Periodic (LFA) versus zero-padded (Dirichlet) spectra, the boundary-condition comparison of the
convolution section: 16 -> 16 3x3 layers, three seeded weight tensors, n = 4, 8, 16.

The GPU computes the LFA spectra; the Dirichlet spectra come from the oracle's dense zero-padded
operator (LAPACK, the only route for non-periodic boundaries). Checks:
  * interlacing: the zero-padded operator on n x n is a compression of the periodic one on the
    (n + 2) x (n + 2) torus, so sigma_i(Dirichlet) <= sigma_i(LFA on the (n+2)-torus) for every i
    (the GPU spectrum, within the 1e-5 sigma_max parity tolerance);
  * the boundary effect shrinks with n: the mean distance between the sorted periodic and
    Dirichlet spectra on the same n x n grid, relative to sigma_max, falls by at least a third
    each time n doubles (it scales like the boundary's share of the grid, ~1/n)."""
import numpy as np
import pytest
import torch

import lfa_workloads as W
import oracle as O

from test_gpu_parity import gpu_svd, SIG_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_periodic_vs_dirichlet_spectra(seed):
    lay = W.Layer(16, 16, 3, 3, 4, 4, "normal", 2.0, seed)
    w = W.weights(lay)
    dist = []
    for n in (4, 8, 16):
        plan, (sp, _, _), st, _ = gpu_svd(w, n, n, vectors=False)
        plan.close()
        plan2, (sp2, _, _), st2, _ = gpu_svd(w, n + 2, n + 2, vectors=False)
        plan2.close()
        assert st == 0 and st2 == 0
        sd = np.sort(np.linalg.svd(O.dense_operator_dirichlet(w, n, n), compute_uv=False))[::-1]
        sp = np.sort(sp.ravel().astype(np.float64))[::-1]
        sp2 = np.sort(sp2.ravel().astype(np.float64))[::-1]
        assert sd.size == sp.size
        assert np.all(sd <= sp2[: sd.size] + SIG_TOL * sp2[0])
        dist.append(float(np.mean(np.abs(sp - sd)) / sp[0]))
    assert dist[1] < 0.67 * dist[0] and dist[2] < 0.67 * dist[1], dist
