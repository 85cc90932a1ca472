"""Pins of the oracle's intra prediction: homogeneous diffusion inpainting,
Sec. 2.1, Eq. (1) with A = -L and reflecting boundary conditions.

Each pin is fixed by the paper or by mathematics, not by the oracle itself:
hand-solved instances (tests/golden), closed forms (linear interpolation in
1-D, discrete-harmonic polynomials), invariants (constants, symmetry, the
maximum principle) and a brute-force dense solve of the whole N x N system.
"""
import numpy as np
import pytest

from conftest import read_golden


def _golden_case(oracle, name):
    (W, H), tags = read_golden(name)
    mask = tags["mask"]
    idx = np.array([int(y) * W + int(x) for x, y, _ in mask], np.uint32)
    val = np.array([v for _, _, v in mask])
    order = np.argsort(idx)
    u, res, _, _ = oracle.inpaint(W, H, idx[order], val[order], 1e-13)
    return u, np.array(tags["row"])


@pytest.mark.parametrize("name", ["inpaint_3x2.txt", "inpaint_2x2.txt", "inpaint_1d_9.txt"])
def test_hand_solved_instances(oracle_lib, name):
    u, expect = _golden_case(oracle_lib, name)
    assert np.abs(u - expect).max() < 1e-11


def test_constant_image_is_exact(oracle_lib):
    rng = np.random.default_rng(3)
    W, H = 37, 23
    idx = np.sort(rng.choice(W * H, 20, replace=False)).astype(np.uint32)
    u, _, _, _ = oracle_lib.inpaint(W, H, idx, np.full(20, 77.0), 1e-12)
    assert np.all(u == 77.0)


def test_mask_values_bit_exact_and_residual(oracle_lib):
    rng = np.random.default_rng(4)
    W, H = 64, 40
    idx = np.sort(rng.choice(W * H, 100, replace=False)).astype(np.uint32)
    val = rng.integers(0, 256, 100).astype(np.float64)
    u, res, _, st = oracle_lib.inpaint(W, H, idx, val, 1e-10)
    assert st == 0
    assert np.array_equal(u.reshape(-1)[idx], val)
    assert res <= 1e-10


def test_maximum_principle_and_mirror_symmetry(oracle_lib):
    rng = np.random.default_rng(5)
    W, H = 41, 29
    idx = np.sort(rng.choice(W * H, 60, replace=False)).astype(np.uint32)
    val = rng.integers(0, 256, 60).astype(np.float64)
    u, _, _, _ = oracle_lib.inpaint(W, H, idx, val, 1e-12)
    assert u.min() >= val.min() - 1e-9 and u.max() <= val.max() + 1e-9
    # mirror the image left-right: the solution mirrors too
    x, y = idx % W, idx // W
    midx = (y * W + (W - 1 - x)).astype(np.uint32)
    o = np.argsort(midx)
    um, _, _, _ = oracle_lib.inpaint(W, H, midx[o], val[o], 1e-12)
    assert np.abs(um[:, ::-1] - u).max() < 1e-9
    # transpose (swap axes): the 5-point operator is isotropic
    tidx = (x * H + y).astype(np.uint32)
    o = np.argsort(tidx)
    ut, _, _, _ = oracle_lib.inpaint(H, W, tidx[o], val[o], 1e-12)
    assert np.abs(ut.T - u).max() < 1e-9


def test_linear_between_masked_columns(oracle_lib):
    """Columns x=0 and x=W-1 masked with values a and b in every row: the
    solution is a + (b-a) x/(W-1) in every row (uses the reflecting boundary
    at the top and bottom rows)."""
    W, H, a, b = 13, 7, 20.0, 200.0
    idx = np.array(sorted([y * W for y in range(H)] + [y * W + W - 1 for y in range(H)]), np.uint32)
    val = np.where(idx % W == 0, a, b).astype(np.float64)
    u, _, _, _ = oracle_lib.inpaint(W, H, idx, val, 1e-13)
    expect = a + (b - a) * np.arange(W) / (W - 1)
    assert np.abs(u - expect[None, :]).max() < 1e-10


@pytest.mark.parametrize("poly", ["x2-y2", "xy"])
def test_discrete_harmonic_polynomials(oracle_lib, poly):
    """x^2 - y^2 and x*y satisfy the 5-point Laplace equation exactly; with
    the outer ring masked the interior must reproduce them."""
    W, H = 11, 9
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    f = xs * xs - ys * ys if poly == "x2-y2" else xs * ys
    f = f + 100.0
    ring = (xs == 0) | (ys == 0) | (xs == W - 1) | (ys == H - 1)
    idx = np.flatnonzero(ring.reshape(-1)).astype(np.uint32)
    u, _, _, _ = oracle_lib.inpaint(W, H, idx, f.reshape(-1)[idx], 1e-13)
    assert np.abs(u - f).max() < 1e-10


def _dense_eq1(W, H, idx, val):
    """Brute force: assemble Eq. (1) as a dense N x N system and LU-solve."""
    N = W * H
    Amat = np.zeros((N, N))
    rhs = np.zeros(N)
    mask = np.zeros(N, bool)
    mask[idx] = True
    for y in range(H):
        for x in range(W):
            i = y * W + x
            if mask[i]:
                Amat[i, i] = 1.0
                rhs[i] = val[list(idx).index(i)]
                continue
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < W and 0 <= yy < H:
                    Amat[i, yy * W + xx] += 1.0
                    Amat[i, i] -= 1.0
    return np.linalg.solve(Amat, rhs).reshape(H, W)


@pytest.mark.parametrize("seed,W,H,K", [(0, 20, 20, 9), (1, 17, 11, 3), (2, 1, 30, 2), (3, 25, 16, 1)])
def test_brute_force_dense_solve(oracle_lib, seed, W, H, K):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(W * H, K, replace=False)).astype(np.uint32)
    val = rng.uniform(0, 255, K)
    u, _, _, _ = oracle_lib.inpaint(W, H, idx, val, 1e-13)
    ref = _dense_eq1(W, H, idx, val)
    assert np.abs(u - ref).max() < 1e-10


def test_invalid_inputs(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle_lib.inpaint(4, 4, np.array([3, 3], np.uint32), np.array([1.0, 2.0]))
    with pytest.raises(RuntimeError):
        oracle_lib.inpaint(4, 4, np.array([16], np.uint32), np.array([1.0]))
    with pytest.raises(RuntimeError):
        oracle_lib.inpaint(4, 4, np.zeros(0, np.uint32), np.zeros(0))


# ---------------------------------------------------------------------------
# the residual of Eq. (1), max over unknown pixels of |(L u)_i|, pinned by
# fields whose 5-point Laplacian with reflecting boundaries is known by hand
# ---------------------------------------------------------------------------
def test_residual_of_a_parabola_is_two(oracle_lib):
    """u = x^2 with columns 0 and W-1 on the mask: every unknown pixel has
    both horizontal neighbours, (x+1)^2 + (x-1)^2 - 2x^2 = 2, and u is
    constant along y, so the vertical terms vanish even at the reflecting
    top and bottom edges.  The residual is exactly 2."""
    W, H = 9, 5
    u = np.tile((np.arange(W, dtype=np.float64) ** 2)[None, :], (H, 1))
    idx = np.array([y * W + x for y in range(H) for x in (0, W - 1)], np.uint32)
    assert oracle_lib.inpaint_residual(u, idx) == 2.0
    # a parabola along y with rows 0 and H-1 masked: the same by symmetry
    v = np.tile((np.arange(H, dtype=np.float64) ** 2)[:, None], (1, W))
    idy = np.array([y * W + x for y in (0, H - 1) for x in range(W)], np.uint32)
    assert oracle_lib.inpaint_residual(v, idy) == 2.0


@pytest.mark.parametrize("x,y,expect", [(4, 2, 4.0), (0, 2, 3.0), (0, 0, 2.0), (8, 4, 2.0)])
def test_residual_of_a_unit_spike_counts_neighbours(oracle_lib, x, y, expect):
    """u = 1 at one unknown pixel, 0 elsewhere: there (L u) = -(number of
    in-image neighbours), 4 inside, 3 on an edge, 2 in a corner (a missing
    neighbour contributes nothing under reflecting boundaries); each
    neighbour sees +1.  With the spike itself on the mask only the
    neighbours count: the residual drops to 1."""
    W, H = 9, 5
    u = np.zeros((H, W))
    u[y, x] = 1.0
    far = np.array([0 if (x, y) != (0, 0) else W * H - 1], np.uint32)  # a mask point away from the spike
    if (x, y) == (8, 4):
        far = np.array([0], np.uint32)
    assert oracle_lib.inpaint_residual(u, far) == expect
    on = np.array([y * W + x], np.uint32)
    assert oracle_lib.inpaint_residual(u, on) == 1.0


def test_residual_ignores_masked_pixels_and_sees_the_worst_unknown(oracle_lib):
    """A harmonic field (x^2 - y^2 has L u = 0 off the boundary) masked on
    its whole border has residual 0; lifting one unknown pixel by d makes
    the residual 4 d (at that pixel), while lifting a mask pixel by d
    changes only its unknown neighbours, by d."""
    W, H = 7, 6
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = xx ** 2 - yy ** 2
    border = np.array([y * W + x for y in range(H) for x in range(W)
                       if x in (0, W - 1) or y in (0, H - 1)], np.uint32)
    assert oracle_lib.inpaint_residual(u, border) == 0.0
    d = 0.375
    up = u.copy()
    up[3, 3] += d
    assert oracle_lib.inpaint_residual(up, border) == 4 * d
    um = u.copy()
    um[0, 3] += d  # a mask pixel on the top edge: its unknown neighbour (3, 1) sees +d
    assert oracle_lib.inpaint_residual(um, border) == d
