"""Pins of the oracle's next rows: the biharmonic operator (Sec. 2.2: the
operator is defined by the eigenvalues of the Green's functions) and the
coefficient mode of the residual decoder (Sec. 2.2, 2.3: the decoder
receives the dead-zone quantised coefficients and the constant and only
evaluates Eq. 3).

Independent anchors:
* the defining property A^2 G = I - 11^T/N with A the block's mirrored
  5-point operator built densely here (not by the oracle);
* brute force: the Green's route equals the block's biharmonic inpainting
  ((A^2 u)_i = 0 off the points, u = v at them) solved as a dense system;
* the paper's transform route of Eq. 4 for the coefficient mode,
  r = C^-1 diag(lambda) C (M c) + a, with scipy's orthonormal DCT-II;
* the values mode: coefficients with sum zero, evaluated at the points,
  must be recovered by the oracle's own (K+1) solve (uniqueness);
* the condition bound with the biharmonic spectrum (eigenvalues <= 64).
"""
import numpy as np
import pytest
import scipy.fft

import oracle
from test_oracle_block import _block_neg_laplacian
from workload import CoefResidual, make_coef_residual


def _dense_biharmonic_inpaint(w, h, pos, v):
    A = _block_neg_laplacian(w, h)
    B = A @ A
    N = w * h
    S, rhs = B.copy(), np.zeros(N)
    for p, x in zip(pos, v):
        S[p, :] = 0.0
        S[p, p] = 1.0
        rhs[p] = x
    return np.linalg.solve(S, rhs)


@pytest.mark.parametrize("w,h", [(16, 16), (16, 8), (5, 3), (1, 7), (2, 2)])
def test_biharmonic_green_definition(w, h):
    N = w * h
    A = _block_neg_laplacian(w, h)
    G = oracle.green_matrix(w, h, op=1)
    assert np.allclose(G, G.T, atol=1e-10)
    assert np.allclose((A @ A) @ G, np.eye(N) - np.ones((N, N)) / N, atol=1e-8 * max(1.0, np.abs(G).max()))
    assert np.allclose(G @ np.ones(N), 0.0, atol=1e-8 * max(1.0, np.abs(G).max()))


@pytest.mark.parametrize("w,h,K,seed", [(16, 16, 8, 0), (16, 16, 30, 1), (11, 16, 5, 2), (5, 3, 4, 3), (1, 16, 3, 4)])
def test_biharmonic_block_equals_dense_inpainting(w, h, K, seed):
    rng = np.random.default_rng(seed)
    pos = np.sort(rng.choice(w * h, K, replace=False)).astype(np.uint8)
    v = rng.integers(-64, 65, K).astype(np.float64)
    r, c, a = oracle.block_solve(w, h, pos, v, G=oracle.green_matrix(w, h, op=1))
    u = _dense_biharmonic_inpaint(w, h, pos.astype(int), v)
    assert np.abs(r.reshape(-1) - u).max() <= 1e-7 * max(1.0, np.abs(u).max())
    assert np.abs(r.reshape(-1)[pos] - v).max() <= 1e-8
    assert abs(c.sum()) <= 1e-8 * max(1.0, np.abs(c).max())


def test_biharmonic_special_cases():
    G = oracle.green_matrix(16, 16, op=1)
    r, c, a = oracle.block_solve(16, 16, np.array([37], np.uint8), np.array([12.0]), G=G)
    assert np.allclose(r, 12.0) and abs(a - 12.0) < 1e-12
    pos = np.array([3, 70, 200], np.uint8)
    r, c, a = oracle.block_solve(16, 16, pos, np.full(3, -5.0), G=G)
    assert np.allclose(r, -5.0, atol=1e-9)


@pytest.mark.parametrize("w,h", [(16, 16), (16, 8), (5, 3)])
def test_biharmonic_condition_bound(w, h):
    """lambda_min(G_PP) >= (1 - K/N) / 64 (the eigenvalues of A^2 are at most
    64), so 64 tr(G_PP) / (1 - K/N) bounds cond_2(G_PP)."""
    rng = np.random.default_rng(w + 7 * h)
    N = w * h
    A = _block_neg_laplacian(w, h)
    assert np.linalg.eigvalsh(A @ A).max() <= 64 + 1e-9
    G = oracle.green_matrix(w, h, op=1)
    for K in sorted({1, 2, N // 4, N // 2, N - 1}):
        if K < 1:
            continue
        P = np.sort(rng.choice(N, K, replace=False))
        ev = np.linalg.eigvalsh(G[np.ix_(P, P)])
        assert ev[0] >= (1 - K / N) / 64 * (1 - 1e-9)
        assert 64 * ev.sum() / (1 - K / N) >= ev[-1] / ev[0] * (1 - 1e-9)


def test_dequantise():
    for step, off in ((1.0, 0.5), (0.25, 0.0), (3.0, 0.375)):
        assert oracle.dequantise(0, step, off) == 0.0
        for q in (1, 2, 17, 127):
            d = oracle.dequantise(q, step, off)
            assert d == (q + off) * step
            assert oracle.dequantise(-q, step, off) == -d
        vals = [oracle.dequantise(q, step, off) for q in range(-127, 128)]
        assert all(b > a for a, b in zip(vals, vals[1:]))


def _dct_route(w, h, pos, c, a, op):
    """Eq. 4: r = C^-1 diag(lambda) C (M c) + a, orthonormal DCT-II."""
    m = np.zeros((h, w))
    for p, x in zip(pos, c):
        m[p // w, p % w] += x
    Cm = scipy.fft.dctn(m, type=2, norm="ortho")
    qq, pp = np.mgrid[0:h, 0:w]
    mu = 4 * np.sin(np.pi * pp / (2 * w)) ** 2 + 4 * np.sin(np.pi * qq / (2 * h)) ** 2
    lam = np.zeros_like(mu)
    nz = mu > 0
    lam[nz] = 1.0 / (mu[nz] if op == 0 else mu[nz] ** 2)
    return scipy.fft.idctn(lam * Cm, type=2, norm="ortho") + a


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("W,H,B,seed", [(48, 32, 16, 0), (37, 21, 16, 1), (20, 13, 8, 2)])
def test_coef_mode_plane_equals_transform_route(op, W, H, B, seed):
    rng = np.random.default_rng(seed)
    res = make_coef_residual(rng, W, H, B, 6.0, step=0.75, offset=0.5)
    r = oracle.block_residual_coef(res, op)
    nbx = -(-W // B)
    for b in range(res.n_blocks):
        bx, by = b % nbx, b // nbx
        w, h = min(B, W - bx * B), min(B, H - by * B)
        s, e = int(res.block_ptr[b]), int(res.block_ptr[b + 1])
        c = [oracle.dequantise(int(q), res.step, res.offset) for q in res.q[s:e]]
        want = _dct_route(w, h, res.pos[s:e].astype(int), c, float(res.a[b]), op)
        got = r[by * B:by * B + h, bx * B:bx * B + w]
        assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max()), b


@pytest.mark.parametrize("op", [0, 1])
def test_coef_mode_matches_values_mode(op):
    """Coefficients with sum zero (c = q step exactly, offset 0) and a
    constant: their Eq. 3 evaluation at the points, solved again by the
    values mode, gives back the same c, a and residual."""
    rng = np.random.default_rng(5 + op)
    w = h = 16
    G = oracle.green_matrix(w, h, op)
    for K in (1, 5, 20, 48):
        pos = np.sort(rng.choice(w * h, K, replace=False)).astype(np.uint8)
        half = rng.integers(-60, 61, K // 2)
        q = np.concatenate([half, -rng.permutation(half), np.zeros(K % 2, np.int64)])
        res = CoefResidual(w, h, 16, np.array([0, K], np.uint32), pos, q.astype(np.int8),
                           np.array([3.25], np.float32), step=0.25, offset=0.0)
        rc = oracle.block_residual_coef(res, op)
        v = rc.reshape(-1)[pos.astype(int)]
        rv, c, a = oracle.block_solve(w, h, pos, v, G=G)
        assert np.abs(rv - rc).max() <= 1e-7 * max(1.0, np.abs(rc).max())
        assert np.abs(c - q * 0.25).max() <= 1e-6 * max(1.0, np.abs(q).max())
        assert abs(a - 3.25) <= 1e-6 * max(1.0, np.abs(rc).max())


def test_coef_mode_special_cases():
    W = H = 16
    # K = 0 everywhere: r = a per block
    res = CoefResidual(W, H, 16, np.array([0, 0], np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.int8),
                       np.array([-7.5], np.float32))
    assert np.all(oracle.block_residual_coef(res) == -7.5)
    # all indices zero: the dead zone reconstructs as zero, r = a
    res = CoefResidual(W, H, 16, np.array([0, 3], np.uint32), np.array([1, 2, 3], np.uint8), np.zeros(3, np.int8),
                       np.array([2.0], np.float32))
    assert np.all(oracle.block_residual_coef(res) == 2.0)
    # linear in the coefficients (offset 0)
    rng = np.random.default_rng(9)
    pos = np.sort(rng.choice(256, 10, replace=False)).astype(np.uint8)
    q1, q2 = rng.integers(-50, 51, 10), rng.integers(-50, 51, 10)
    mk = lambda q, a: CoefResidual(W, H, 16, np.array([0, 10], np.uint32), pos, q.astype(np.int8),
                                   np.array([a], np.float32), step=0.5, offset=0.0)
    r12 = oracle.block_residual_coef(mk(q1 + q2, 1.0))
    assert np.allclose(r12, oracle.block_residual_coef(mk(q1, 0.5)) + oracle.block_residual_coef(mk(q2, 0.5)),
                       atol=1e-9)
    # index -128 is outside the quantiser's range
    bad = CoefResidual(W, H, 16, np.array([0, 1], np.uint32), np.array([5], np.uint8), np.array([-128], np.int8),
                       np.array([0.0], np.float32))
    with pytest.raises(ValueError):
        oracle.block_residual_coef(bad)
