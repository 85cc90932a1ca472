"""Pins of the oracle's residual correction: block-based pseudodifferential
inpainting with the harmonic operator (Sec. 2.2, Eqs. 2-4; Sec. 2.3).

Independent anchors:
* hand-derived Green's matrices (tests/golden/green_*.txt);
* the defining property of G: A G = I - 11^T/N with A the block's mirrored
  5-point operator, G symmetric (Sec. 2.2);
* the eigenvalues of A against numpy's symmetric eigensolver;
* the DCT-II route of Eq. (4) via scipy.fft against the explicit sum;
* brute force: the Green's route equals the block's own homogeneous
  diffusion inpainting (Eq. 1 on the block) solved as a dense system;
* special cases: K = 0 (zero), K = 1 and equal values (constant),
  interpolation at the points, a single row (piecewise linear).
"""
import numpy as np
import pytest
import scipy.fft

from conftest import read_golden
from workload import make_residual


def _block_neg_laplacian(w, h):
    """Dense A = -L on a w x h block, missing neighbours contribute nothing."""
    N = w * h
    A = np.zeros((N, N))
    for y in range(h):
        for x in range(w):
            i = y * w + x
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < w and 0 <= yy < h:
                    A[i, i] += 1.0
                    A[i, yy * w + xx] -= 1.0
    return A


def _dense_block_inpaint(w, h, pos, v):
    """Eq. (1) on the block itself (the brute-force counterpart)."""
    A = _block_neg_laplacian(w, h)
    M = np.zeros(w * h, bool)
    M[pos] = True
    S = np.where(M[:, None], np.eye(w * h), A)
    rhs = np.zeros(w * h)
    rhs[pos] = v
    return np.linalg.solve(S, rhs).reshape(h, w)


@pytest.mark.parametrize("name", ["green_2x1.txt", "green_2x2.txt"])
def test_golden_green_matrices(oracle_lib, name):
    (w, h), tags = read_golden(name)
    assert np.abs(oracle_lib.green_matrix(w, h) - np.array(tags["row"])).max() < 1e-15


@pytest.mark.parametrize("w,h", [(16, 16), (16, 8), (6, 16), (5, 3), (1, 7), (16, 12), (11, 16)])
def test_green_is_pseudo_inverse(oracle_lib, w, h):
    G = oracle_lib.green_matrix(w, h)
    N = w * h
    assert np.abs(G - G.T).max() < 1e-13
    A = _block_neg_laplacian(w, h)
    assert np.abs(A @ G - (np.eye(N) - np.ones((N, N)) / N)).max() < 1e-12
    assert np.abs(G.sum(axis=1)).max() < 1e-11  # constants are in the null space


@pytest.mark.parametrize("w,h", [(4, 3), (16, 16), (7, 1)])
def test_eigenvalues_match_dense_operator(oracle_lib, w, h):
    mus = sorted(oracle_lib.block_eigenvalue(w, h, p, q) for q in range(h) for p in range(w))
    ref = np.linalg.eigvalsh(_block_neg_laplacian(w, h))
    assert np.abs(np.array(mus) - ref).max() < 1e-12


def test_golden_single_row_block(oracle_lib):
    (w, h), tags = read_golden("block_row_5.txt")
    pts = tags["point"]
    r, c, a = oracle_lib.block_solve(w, h, [int(p) for p, _ in pts], [v for _, v in pts])
    assert np.abs(r.reshape(-1) - np.array(tags["row"][0])).max() < 1e-12


@pytest.mark.parametrize("seed,w,h,K", [(0, 16, 16, 8), (1, 16, 8, 3), (2, 6, 16, 12), (3, 5, 3, 14),
                                        (4, 16, 16, 1), (5, 16, 16, 48), (6, 11, 16, 30), (7, 16, 16, 255)])
def test_brute_force_block_eq1(oracle_lib, seed, w, h, K):
    rng = np.random.default_rng(seed)
    pos = np.sort(rng.choice(w * h, K, replace=False))
    v = rng.integers(-64, 65, K).astype(np.float64)
    r, c, a = oracle_lib.block_solve(w, h, pos, v)
    ref = _dense_block_inpaint(w, h, pos, v)
    assert np.abs(r - ref).max() < 1e-9
    assert abs(c.sum()) < 1e-10  # coefficients sum to zero
    assert np.abs(r.reshape(-1)[pos] - v).max() < 1e-9  # interpolation at the points
    assert r.min() >= v.min() - 1e-9 and r.max() <= v.max() + 1e-9  # maximum principle


def test_dct_route_equals_explicit_sum(oracle_lib):
    """Eq. (4): u = C^-1 diag(lambda) C (M c) + a with the orthonormal
    DCT-II and lambda = 1/mu (0 for the constant mode)."""
    rng = np.random.default_rng(9)
    for w, h, K in [(16, 16, 10), (16, 12, 5), (9, 16, 20)]:
        pos = np.sort(rng.choice(w * h, K, replace=False))
        v = rng.integers(-64, 65, K).astype(np.float64)
        r, c, a = oracle_lib.block_solve(w, h, pos, v)
        img = np.zeros(h * w)
        img[pos] = c
        spec = scipy.fft.dctn(img.reshape(h, w), type=2, norm="ortho")
        p = np.arange(w)[None, :]
        q = np.arange(h)[:, None]
        mu = 4 * np.sin(np.pi * p / (2 * w)) ** 2 + 4 * np.sin(np.pi * q / (2 * h)) ** 2
        lam = np.where(mu > 0, 1.0 / np.where(mu > 0, mu, 1.0), 0.0)
        r_dct = scipy.fft.idctn(lam * spec, type=2, norm="ortho") + a
        assert np.abs(r_dct - r).max() < 1e-10


def test_special_cases(oracle_lib):
    rng = np.random.default_rng(11)
    r, c, a = oracle_lib.block_solve(16, 16, [37], [25.0])
    assert np.abs(r - 25.0).max() < 1e-11 and abs(c[0]) < 1e-11
    pos = np.sort(rng.choice(256, 9, replace=False))
    r, c, a = oracle_lib.block_solve(16, 16, pos, np.full(9, -13.0))
    assert np.abs(r + 13.0).max() < 1e-10
    r, _, _ = oracle_lib.block_solve(16, 16, [], [])
    assert np.all(r == 0.0)


def test_saddle_matrix_conditioning_bound(oracle_lib):
    """Derived fact the GPU path relies on: G_PP is SPD with
    lambda_min >= (1 - K/N)/8 (G's nonzero eigenvalues are >= 1/8 and E_P x
    has mean-free energy >= |x|^2 (1 - K/N))."""
    rng = np.random.default_rng(12)
    G = oracle_lib.green_matrix(16, 16)
    for K in (2, 8, 32, 64, 128, 200):
        pos = np.sort(rng.choice(256, K, replace=False))
        lmin = np.linalg.eigvalsh(G[np.ix_(pos, pos)])[0]
        assert lmin >= (1 - K / 256) / 8 - 1e-12


def test_plane_with_ragged_edges(oracle_lib):
    """Every block, including cropped edge blocks, is an independent image."""
    rng = np.random.default_rng(13)
    W, H, B = 37, 21, 16
    res = make_residual(rng, W, H, B, 5.0, 64)
    r = oracle_lib.block_residual(res)
    nbx = -(-W // B)
    for b in range(res.n_blocks):
        bx, by = b % nbx, b // nbx
        w, h = min(B, W - bx * B), min(B, H - by * B)
        lo, hi = res.block_ptr[b], res.block_ptr[b + 1]
        blk = r[by * B: by * B + h, bx * B: bx * B + w]
        if hi == lo:
            assert np.all(blk == 0.0)
            continue
        ref = _dense_block_inpaint(w, h, res.pos[lo:hi].astype(int), res.val[lo:hi].astype(float))
        assert np.abs(blk - ref).max() < 1e-9


def test_invalid_blocks(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.block_solve(2, 2, [0, 1, 2, 3], [1, 2, 3, 4])  # K = N
    with pytest.raises(ValueError):
        oracle_lib.block_solve(4, 4, [5, 3], [1, 2])  # unsorted
    with pytest.raises(ValueError):
        oracle_lib.block_solve(4, 2, [9], [1])  # outside the block
