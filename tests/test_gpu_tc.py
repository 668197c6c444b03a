"""The tensor-core contractions of the blocked Jacobi route (tcgen05, 3xTF32) against FP64.

Y = 64 columns (two blocks of 32, in a scattered order) of column-major complex planes. The Gram
H = Y^* Y must match numpy's FP64 product to 1e-6 |y_p| |y_q| off the diagonal and 1e-5 on it. The
tensor core's FP32 accumulation is not correctly rounded: on GB300 the error grows with K, from
1.8e-7 (off) / 6.5e-7 (diagonal) at K = 32 rows to 5.4e-7 / 5.9e-6 at K = 512 (a sum of positive
terms on the diagonal). The Jacobi test compares |h_pq| with tol sqrt(h_pp h_qq), so the route
keeps tol well above the off-diagonal level (tol = 4 sqrt(M) 2^-24 = 5.4e-6 at M = 512); the
diagonal only sets the scale of that test (sigma comes from the column norms on the CUDA cores).
The update Y Q (Q unitary) is formed as Y + Y (Q - I), the second term on the tensor cores: its
error scales with |Q - I|, 2e-6 of the largest column for a random unitary Q (measured 1.2-1.4e-6)
and 2e-7 for the near-identity rotations of the late sweeps. A one-pass TF32 product would miss
these bounds by ~3 orders of magnitude, which the tests would catch."""
import numpy as np
import pytest
import torch

from paper_2506_05617_gb300 import lfa as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build()


def _planes(ncols, rows, ld, seed, spread=True):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((ncols, rows)) + 1j * rng.standard_normal((ncols, rows))
    if spread:                                      # column norms over four decades
        Y *= np.logspace(0, -4, ncols)[rng.permutation(ncols)][:, None]
    Xr = np.zeros((ncols, ld), np.float32)
    Xi = np.zeros((ncols, ld), np.float32)
    Xr[:, :rows] = Y.real
    Xi[:, :rows] = Y.imag
    return Xr, Xi


@pytest.mark.parametrize("rows,ld", [(64, 64), (512, 512), (192, 196), (512, 516)])
def test_tc_gram_matches_fp64(rows, ld):
    ncols = 192
    Xr, Xi = _planes(ncols, rows, ld, seed=rows + ld)
    cols = np.random.default_rng(1).permutation(ncols)[:64].astype(np.int32)
    dXr, dXi, dc = (torch.from_numpy(a).cuda() for a in (Xr, Xi, cols))
    D = torch.full((64, 64, 2), float("nan"), device="cuda")
    st = C.lfa_debug_tc_gram(dXr.data_ptr(), dXi.data_ptr(), ld, rows, dc.data_ptr(), D.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    Y = (Xr[cols, :rows].astype(np.float64) + 1j * Xi[cols, :rows].astype(np.float64)).T   # rows x 64
    H = np.conj(Y.T) @ Y
    Hg = D.cpu().numpy().astype(np.float64)
    Hg = Hg[..., 0] + 1j * Hg[..., 1]
    nrm = np.sqrt(np.real(np.diag(H)))
    rel = np.abs(Hg - H) / np.outer(nrm, nrm)
    off = rel[~np.eye(64, dtype=bool)].max()
    diag = np.diag(rel).max()
    print(f"gram rows={rows}: off-diagonal {off:.2e}, diagonal {diag:.2e}")
    assert off <= 1e-6, off          # the entries the rotation test compares with tol
    assert diag <= 1e-5, diag        # column norms: only the scale of that test


@pytest.mark.parametrize("rows,near_identity", [(128, False), (512, False), (512, True)])
def test_tc_update_matches_fp64(rows, near_identity):
    ncols, ld = 160, rows + 4
    Pr, Pi = _planes(ncols, rows, ld, seed=7 * rows)
    cols = np.random.default_rng(2).permutation(ncols)[:64].astype(np.int32)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    if near_identity:
        # a late-sweep block rotation: Q = exp(i K), K Hermitian with entries ~1e-3
        K = 1e-3 * (G + np.conj(G.T)) / 2
        lam, E = np.linalg.eigh(K)
        Q = (E * np.exp(1j * lam)) @ np.conj(E.T)
    else:
        Q, _ = np.linalg.qr(G)
    Qc = np.stack([Q.real, Q.imag], -1).astype(np.float32)
    dPr, dPi, dc, dQ = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (Pr, Pi, cols, Qc))
    Or, Oi = dPr.clone(), dPi.clone()
    st = C.lfa_debug_tc_update(dPr.data_ptr(), dPi.data_ptr(), Or.data_ptr(), Oi.data_ptr(), ld, rows,
                               dc.data_ptr(), dQ.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    Y = (Pr[cols, :rows].astype(np.float64) + 1j * Pi[cols, :rows].astype(np.float64)).T
    Qd = Qc[..., 0].astype(np.float64) + 1j * Qc[..., 1].astype(np.float64)
    ref = Y @ Qd                                                  # rows x 64
    out = Or.cpu().numpy().astype(np.float64) + 1j * Oi.cpu().numpy().astype(np.float64)
    got = out[cols, :rows].T
    colnorm = np.linalg.norm(Y, axis=0).max()
    err = np.max(np.linalg.norm(got - ref, axis=0)) / colnorm
    print(f"update rows={rows} near_identity={near_identity}: {err:.2e}")
    assert err <= (2e-7 if near_identity else 2e-6), err
    others = np.setdiff1d(np.arange(ncols), cols)                  # untouched columns
    assert np.array_equal(out[others], Pr[others] + 1j * Pi[others])
