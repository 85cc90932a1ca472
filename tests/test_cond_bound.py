"""The condition bound the coefficient stage compares with cond_threshold:
kappa = 8 tr(G_PP) / (1 - K/N) >= cond_2(G_PP) for every block shape and
point set (Sec. 2.2: G is the pseudo-inverse of A = -L, whose eigenvalues
lie in [0, 8]; so c^T G_PP c >= |E_P c - mean|^2 / 8 >= (1 - K/N) |c|^2 / 8,
and lambda_max <= tr).  Checked against numpy's symmetric eigensolver on the
oracle's FP64 Green's matrices, with the block operator's spectrum from the
dense matrix (not from the oracle), and the largest bound any shape can
reach is below the default threshold 1e6."""
import numpy as np
import pytest

import oracle
from test_oracle_block import _block_neg_laplacian


@pytest.mark.parametrize("w,h", [(16, 16), (16, 8), (11, 16), (5, 3), (1, 16), (2, 2)])
def test_bound_holds(w, h):
    rng = np.random.default_rng(w * 31 + h)
    N = w * h
    A = _block_neg_laplacian(w, h)
    assert np.linalg.eigvalsh(A).max() <= 8 + 1e-12  # Gershgorin: degree <= 4
    G = oracle.green_matrix(w, h)
    ks = sorted({1, 2, max(1, N // 4), max(1, N // 2), N - 1})
    for K in ks:
        for _ in range(4):
            P = np.sort(rng.choice(N, K, replace=False))
            Gp = G[np.ix_(P, P)]
            ev = np.linalg.eigvalsh(Gp)
            assert ev[0] >= (1 - K / N) / 8 * (1 - 1e-9), (w, h, K)
            assert 8 * np.trace(Gp) / (1 - K / N) >= ev[-1] / ev[0] * (1 - 1e-9), (w, h, K)


def test_clustered_blocks_are_well_conditioned():
    """25 points in a 5 x 5 window (the stress set's worst case)."""
    G = oracle.green_matrix(16, 16)
    P = np.array([y * 16 + x for y in range(5) for x in range(5)])
    ev = np.linalg.eigvalsh(G[np.ix_(P, P)])
    assert ev[0] >= (1 - 25 / 256) / 8
    assert ev[-1] / ev[0] < 1e3


def test_largest_bound_below_default_threshold():
    """For each shape the bound is largest with the K largest diagonal
    entries of G and K = N - 1; over all 256 shapes it stays below 4e5."""
    worst = 0.0
    for w in range(1, 17):
        for h in range(1, 17):
            N = w * h
            if N < 2:
                continue
            d = np.sort(np.diag(oracle.green_matrix(w, h)))[::-1]
            K = np.arange(1, N)
            worst = max(worst, float((8 * np.cumsum(d)[: N - 1] / (1 - K / N)).max()))
    assert 3e5 < worst < 4e5
