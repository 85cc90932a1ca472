"""Seeded synthetic decoder inputs (numpy ``Generator(PCG64(seed))``).

Recipes (sizes, distributions) follow the workloads the paper measures on
(Sec. 3: FullHD video, 32-frame tests, piecewise smooth content) with
synthetic stand-ins, since no video data is available:

* source frames: a constant base + a linear gradient + isotropic Gaussian
  blobs, moved between frames by a small rotation + translation, rendered
  analytically (no interpolation);
* intra masks: uniformly random pixel subsets (sorted linear indices);
  chroma uses one mask for both chroma channels at half the luma density
  (Sec. 2.3 takes half the mask points for chroma and one shared mask);
* backward flow: the exact backward displacement of the scene motion
  (GOP workloads) or a sum of random vector sinusoids (single P-frame);
* residual data per B x B block: a Poisson number of distinct random
  positions and uniform random integer values (Sec. 2.2/2.3 block mask).

Nothing here performs inpainting, warping or any other decoding step.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Residual:
    """Sparse block residual data of one plane.

    Blocks tile the plane in raster order with edge ``block``; edge blocks are
    cropped to the plane.  Block ``b`` owns points ``block_ptr[b] ..
    block_ptr[b+1]-1``; ``pos`` is the point's index ``ly*w + lx`` inside the
    block's own width ``w`` (strictly increasing within a block); ``val`` is
    the integer residual value at that point.
    """

    width: int
    height: int
    block: int
    block_ptr: np.ndarray  # uint32 [n_blocks + 1]
    pos: np.ndarray  # uint8  [n_points]
    val: np.ndarray  # int16  [n_points]

    @property
    def n_blocks(self) -> int:
        return int(self.block_ptr.shape[0] - 1)

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class CoefResidual:
    """Block residual of one plane in coefficient mode (Sec. 2.2, 2.3): per
    point a dead-zone quantisation index ``q`` in [-127, 127] of its Green's
    coefficient, per block the constant ``a``; the plane's quantiser step
    and reconstruction offset.  Blocks and positions as in :class:`Residual`."""

    width: int
    height: int
    block: int
    block_ptr: np.ndarray  # uint32 [n_blocks + 1]
    pos: np.ndarray  # uint8  [n_points]
    q: np.ndarray  # int8   [n_points]
    a: np.ndarray  # float32 [n_blocks]
    step: float = 1.0
    offset: float = 0.5

    @property
    def n_blocks(self) -> int:
        return int(self.block_ptr.shape[0] - 1)

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class IFrame:
    width: int
    height: int
    chroma: bool
    y_idx: np.ndarray  # uint32 sorted linear indices (y*W + x)
    y_val: np.ndarray  # uint8
    c_idx: Optional[np.ndarray] = None  # uint32, shared by Cb and Cr
    cb_val: Optional[np.ndarray] = None
    cr_val: Optional[np.ndarray] = None
    res: Optional[List[Residual]] = None  # None, or one Residual per plane
    rct: bool = False  # 4:4:4 RCT planes (chroma values int16 in [-255, 255])


@dataclass
class PFrame:
    flow: np.ndarray  # float32 [H, W, 2], (dx, dy): pred(x) = ref(x + flow(x))
    res: List[Residual]  # one per plane


@dataclass
class PFrameCoef:
    flow: np.ndarray  # float32 [H, W, 2]
    res: List[CoefResidual]  # one per plane


@dataclass
class Gop:
    width: int
    height: int
    chroma: bool
    block: int
    iframe: IFrame
    pframes: List[PFrame]
    sources: List[Tuple[np.ndarray, ...]] = field(default_factory=list)
    rct: bool = False  # 4:4:4 RCT planes Y, U, V (Sec. 2.3)

    @property
    def n_frames(self) -> int:
        return 1 + len(self.pframes)


def chroma_size(width: int, height: int) -> Tuple[int, int]:
    """4:2:0 chroma plane size."""
    return (width + 1) // 2, (height + 1) // 2


def block_grid(width: int, height: int, block: int):
    """Block counts and the per-block (w, h) of a raster block tiling."""
    nbx = -(-width // block)
    nby = -(-height // block)
    bw = np.minimum(block, width - block * np.arange(nbx))
    bh = np.minimum(block, height - block * np.arange(nby))
    w = np.tile(bw, nby)
    h = np.repeat(bh, nbx)
    return nbx, nby, w.astype(np.int64), h.astype(np.int64)


# ----------------------------------------------------------------------------
# residual data
# ----------------------------------------------------------------------------
def _positions_from_counts(rng, w, h, block, k):
    """Distinct uniform positions per block, sorted, concatenated."""
    n = w.shape[0]
    cells = block * block
    keys = rng.random((n, cells))
    valid = np.arange(cells)[None, :] < (w * h)[:, None]
    keys[~valid] = 2.0
    order = np.argsort(keys, axis=1, kind="stable")
    take = np.arange(cells)[None, :] < k[:, None]
    sel = np.where(take, order, cells + 1)
    sel.sort(axis=1)
    return sel[take]


def _clustered_positions(rng, w, h, k, window):
    """K distinct positions inside one random window x window square."""
    out = []
    for b in range(w.shape[0]):
        wb, hb, kb = int(w[b]), int(h[b]), int(k[b])
        ww, wh = min(window, wb), min(window, hb)
        x0 = int(rng.integers(0, wb - ww + 1))
        y0 = int(rng.integers(0, hb - wh + 1))
        cand = np.array([(y0 + j) * wb + (x0 + i) for j in range(wh) for i in range(ww)])
        kb = min(kb, cand.size, wb * hb - 1)
        k[b] = kb
        out.append(np.sort(rng.choice(cand, size=kb, replace=False)))
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def make_residual(
    rng: np.random.Generator,
    width: int,
    height: int,
    block: int,
    lam: float,
    vmax: int,
    kmax: Optional[int] = None,
    empty_frac: float = 0.0,
    positions_from: Optional[Residual] = None,
    shared_layouts: int = 0,
    shared_frac: float = 0.0,
    clustered_frac: float = 0.0,
    cluster_window: int = 5,
    cluster_kmax: int = 25,
) -> Residual:
    """Random block residual: K_b ~ Poisson(lam) distinct positions per block
    (clipped to ``[0, min(kmax, w*h - 1)]``), values uniform in
    ``[-vmax, vmax]``.

    ``positions_from`` reuses another plane's layout (shared chroma mask) and
    draws fresh values.  ``shared_layouts``/``shared_frac`` make that fraction
    of the full-size blocks draw one of a few common layouts.
    ``clustered_frac`` puts that fraction of blocks' points inside a small
    window (the clustered stress set).
    """
    if positions_from is not None:
        bp = positions_from.block_ptr.copy()
        pos = positions_from.pos.copy()
        val = rng.integers(-vmax, vmax + 1, size=pos.shape[0]).astype(np.int16)
        return Residual(width, height, block, bp, pos, val)

    nbx, nby, w, h = block_grid(width, height, block)
    n = nbx * nby
    cap = w * h - 1
    if kmax is not None:
        cap = np.minimum(cap, kmax)
    k = np.minimum(rng.poisson(lam, size=n), cap).astype(np.int64)
    if empty_frac > 0:
        k[rng.random(n) < empty_frac] = 0
    pos_parts = None
    if shared_layouts > 0 and shared_frac > 0:
        full = (w == block) & (h == block) & (k > 0)
        layouts = []
        for _ in range(shared_layouts):
            kl = int(min(max(rng.poisson(lam), 1), block * block - 1, kmax or 10**9))
            layouts.append(np.sort(rng.choice(block * block, size=kl, replace=False)))
        pick = full & (rng.random(n) < shared_frac)
        which = rng.integers(0, shared_layouts, size=n)
        k[pick] = [layouts[i].size for i in which[pick]]
        base = _positions_from_counts(rng, w, h, block, np.where(pick, 0, k))
        parts, off = [], 0
        for b in range(n):
            if pick[b]:
                parts.append(layouts[which[b]])
            else:
                parts.append(base[off : off + k[b]])
                off += k[b]
        pos_parts = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    elif clustered_frac > 0:
        clus = rng.random(n) < clustered_frac
        kc = np.minimum(k, cluster_kmax)
        k = np.where(clus, kc, k)
        base = _positions_from_counts(rng, w, h, block, np.where(clus, 0, k))
        kcl = k[clus].copy()
        cl = _clustered_positions(rng, w[clus], h[clus], kcl, cluster_window)
        k[clus] = kcl
        parts, off, offc, ic = [], 0, 0, 0
        for b in range(n):
            if clus[b]:
                parts.append(cl[offc : offc + k[b]])
                offc += k[b]
            else:
                parts.append(base[off : off + k[b]])
                off += k[b]
        pos_parts = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    else:
        pos_parts = _positions_from_counts(rng, w, h, block, k)

    bp = np.zeros(n + 1, np.uint32)
    np.cumsum(k, out=bp[1:])
    val = rng.integers(-vmax, vmax + 1, size=int(bp[-1])).astype(np.int16)
    return Residual(width, height, block, bp, pos_parts.astype(np.uint8), val)


def make_coef_residual(
    rng: np.random.Generator,
    width: int,
    height: int,
    block: int,
    lam: float,
    qmax: int = 127,
    zero_frac: float = 0.4,
    amax: float = 8.0,
    step: float = 1.0,
    offset: float = 0.5,
    kmax: Optional[int] = None,
    positions_from: Optional[CoefResidual] = None,
) -> CoefResidual:
    """Random coefficient-mode residual: positions as :func:`make_residual`
    (K ~ Poisson(lam), clipped), indices uniform in [-qmax, qmax] with a
    ``zero_frac`` share of zeros (the dead zone's mass), constants uniform in
    [-amax, amax].  ``positions_from`` reuses another plane's layout."""
    if positions_from is not None:
        bp = positions_from.block_ptr.copy()
        pos = positions_from.pos.copy()
    else:
        nbx, nby, w, h = block_grid(width, height, block)
        cap = w * h - 1
        if kmax is not None:
            cap = np.minimum(cap, kmax)
        k = np.minimum(rng.poisson(lam, size=nbx * nby), cap).astype(np.int64)
        pos = _positions_from_counts(rng, w, h, block, k).astype(np.uint8)
        bp = np.zeros(nbx * nby + 1, np.uint32)
        np.cumsum(k, out=bp[1:])
    n = int(pos.shape[0])
    q = rng.integers(-qmax, qmax + 1, size=n)
    q[rng.random(n) < zero_frac] = 0
    a = rng.uniform(-amax, amax, size=bp.shape[0] - 1).astype(np.float32)
    return CoefResidual(width, height, block, bp, pos, q.astype(np.int8), a, float(step), float(offset))


def coef_frame_residuals(rng, width, height, chroma, block, lam_y=8.0, lam_c=4.0, rct=False,
                         **kw) -> List[CoefResidual]:
    """Coefficient-mode residuals of one frame; Cr shares the Cb layout."""
    ry = make_coef_residual(rng, width, height, block, lam_y, **kw)
    if not chroma:
        return [ry]
    cw, ch = (width, height) if rct else chroma_size(width, height)
    rcb = make_coef_residual(rng, cw, ch, block, lam_c, **kw)
    rcr = make_coef_residual(rng, cw, ch, block, lam_c, positions_from=rcb, **kw)
    return [ry, rcb, rcr]


def empty_residual(width: int, height: int, block: int) -> Residual:
    nbx, nby, _, _ = block_grid(width, height, block)
    return Residual(
        width, height, block,
        np.zeros(nbx * nby + 1, np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.int16),
    )


# ----------------------------------------------------------------------------
# source frames
# ----------------------------------------------------------------------------
@dataclass
class _Texture:
    base: float
    grad: np.ndarray  # (2,) grey levels per pixel of texture coordinate
    centers: np.ndarray  # (n, 2)
    sigmas: np.ndarray  # (n,)
    amps: np.ndarray  # (n,)
    signed: bool = False  # an RCT chroma plane: int16 in [-255, 255]


def _random_texture(rng, width, height, n_blobs, amp, grad_span, base=128.0):
    span = np.array([width, height], float)
    centers = rng.uniform(-0.1, 1.1, size=(n_blobs, 2)) * span
    sigmas = rng.uniform(8.0, 40.0, size=n_blobs) * max(1.0, min(width, height) / 144.0) ** 0.5
    amps = rng.uniform(-amp, amp, size=n_blobs)
    direction = rng.normal(size=2)
    direction /= np.linalg.norm(direction) + 1e-12
    grad = direction * (2.0 * grad_span / max(width, height))
    return _Texture(base, grad, centers, sigmas, amps)


def _render(tex: _Texture, xs: np.ndarray, ys: np.ndarray, rot: float, shift, center):
    """Texture sampled at frame coordinates, texture coords p = R(rot)(x-c)+c+shift.

    Isotropic blobs stay isotropic under rotation, so each blob is an outer
    product of two 1-D Gaussians centred at the blob's frame position.
    """
    c, s = np.cos(rot), np.sin(rot)
    R = np.array([[c, -s], [s, c]])
    img = np.full((ys.size, xs.size), tex.base)
    # gradient term g . p
    gx, gy = R.T @ tex.grad
    off = tex.grad @ (np.asarray(center) - R @ np.asarray(center) + np.asarray(shift))
    img += gx * xs[None, :] + gy * ys[:, None] + off
    for (cx, cy), sg, a in zip(tex.centers, tex.sigmas, tex.amps):
        # frame position x of the blob centre: R(x - c) + c + shift = centre
        fx, fy = R.T @ (np.array([cx, cy]) - np.asarray(center) - np.asarray(shift)) + np.asarray(center)
        ex = np.exp(-((xs - fx) ** 2) / (2 * sg * sg))
        ey = np.exp(-((ys - fy) ** 2) / (2 * sg * sg))
        img += a * np.outer(ey, ex)
    if tex.signed:
        return np.clip(np.floor(img + 0.5), -255, 255).astype(np.int16)
    return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)


def make_flow_sinusoids(rng, width, height, n=3, vmax=4.0) -> np.ndarray:
    """Smooth flow: sum of ``n`` random vector sinusoids, max |v| = vmax."""
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    v = np.zeros((height, width, 2))
    for _ in range(n):
        lam = rng.uniform(0.25, 1.0) * max(width, height)
        ang = rng.uniform(0, 2 * np.pi)
        k = (2 * np.pi / lam) * np.array([np.cos(ang), np.sin(ang)])
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.normal(size=2)
        v += a[None, None, :] * np.sin(k[0] * xs + k[1] * ys + ph)[:, :, None]
    m = np.sqrt((v ** 2).sum(-1)).max()
    if m > 0:
        v *= vmax / m
    return v.astype(np.float32)


def _mask(rng, n_pixels, frac):
    k = int(round(frac * n_pixels))
    k = max(1, min(k, n_pixels))
    return np.sort(rng.choice(n_pixels, size=k, replace=False)).astype(np.uint32)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def make_config1(seed: int = 0, width: int = 256, height: int = 144):
    """Tiny plain-method workload: grey, one I-frame (4% mask) + one P-frame
    (sinusoid flow |v| <= 4 px, 16x16 residual blocks, Poisson(6), values in
    [-32, 32]).  Returns (source uint8 [H, W], IFrame, PFrame)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tex = _random_texture(rng, width, height, 12, 60.0, 30.0)
    xs = np.arange(width, dtype=np.float64)
    ys = np.arange(height, dtype=np.float64)
    src = _render(tex, xs, ys, 0.0, (0.0, 0.0), (width / 2, height / 2))
    idx = _mask(rng, width * height, 0.04)
    ifr = IFrame(width, height, False, idx, src.reshape(-1)[idx].copy())
    flow = make_flow_sinusoids(rng, width, height, 3, 4.0)
    res = make_residual(rng, width, height, 16, 6.0, 32)
    return src, ifr, PFrame(flow, [res])


def make_iframe_only(seed: int, width: int, height: int, mask_frac: float,
                     chroma: bool = False, chroma_mask_frac: Optional[float] = None,
                     residual: Optional[dict] = None, block: int = 16):
    """One intra frame of a random scene at the given mask density."""
    rng = np.random.Generator(np.random.PCG64(seed))
    planes = _scene_planes(rng, width, height, chroma)
    srcs = tuple(_render(t, xs, ys, 0.0, (0.0, 0.0), c) for (t, xs, ys, c) in planes)
    ifr = _intra(rng, width, height, chroma, srcs, mask_frac,
                 chroma_mask_frac if chroma_mask_frac is not None else mask_frac / 2)
    if residual is not None:
        ifr.res = _frame_residuals(rng, width, height, chroma, block, **residual)
    return srcs, ifr


def _scene_planes(rng, width, height, chroma, rct=False):
    center = (width / 2.0, height / 2.0)
    out = [(_random_texture(rng, width, height, 12, 60.0, 30.0),
            np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64), center)]
    if chroma and rct:
        # 4:4:4 planes of the reversible colour transform: U = B - G and
        # V = R - G are signed (Sec. 2.3)
        for _ in range(2):
            tex = _random_texture(rng, width, height, 12, 60.0, 20.0, base=0.0)
            tex.signed = True
            out.append((tex, np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64), center))
    elif chroma:
        cw, ch = chroma_size(width, height)
        xs = 2.0 * np.arange(cw) + 0.5
        ys = 2.0 * np.arange(ch) + 0.5
        for _ in range(2):
            out.append((_random_texture(rng, width, height, 12, 40.0, 20.0), xs, ys, center))
    return out


def _intra(rng, width, height, chroma, srcs, frac, cfrac, rct=False):
    idx = _mask(rng, width * height, frac)
    ifr = IFrame(width, height, chroma, idx, srcs[0].reshape(-1)[idx].copy())
    ifr.rct = bool(rct and chroma)
    if chroma:
        cw, ch = (width, height) if rct else chroma_size(width, height)
        cidx = _mask(rng, cw * ch, cfrac)
        ifr.c_idx = cidx
        ifr.cb_val = srcs[1].reshape(-1)[cidx].copy()
        ifr.cr_val = srcs[2].reshape(-1)[cidx].copy()
    return ifr


def _frame_residuals(rng, width, height, chroma, block, lam_y=8.0, lam_c=4.0, vmax=64, rct=False,
                     **kw) -> List[Residual]:
    ry = make_residual(rng, width, height, block, lam_y, vmax, **kw)
    if not chroma:
        return [ry]
    cw, ch = (width, height) if rct else chroma_size(width, height)
    kwc = {k: v for k, v in kw.items() if k not in ("shared_layouts", "shared_frac")}
    rcb = make_residual(rng, cw, ch, block, lam_c, vmax, **kwc)
    rcr = make_residual(rng, cw, ch, block, lam_c, vmax, positions_from=rcb)
    return [ry, rcb, rcr]


def make_gop(
    seed: int = 0,
    width: int = 1920,
    height: int = 1080,
    n_frames: int = 30,
    chroma: bool = True,
    mask_frac: float = 0.03,
    chroma_mask_frac: float = 0.015,
    block: int = 16,
    lam_y: float = 8.0,
    lam_c: float = 4.0,
    vmax: int = 64,
    iframe_residual: bool = False,
    with_sources: bool = True,
    max_shift: float = 3.0,
    max_rot_deg: float = 0.2,
    residual_kw: Optional[dict] = None,
    coef_mode: bool = False,
    coef_kw: Optional[dict] = None,
    rct: bool = False,
) -> Gop:
    """A GOP of one intra frame and ``n_frames - 1`` inter frames of a moving
    synthetic scene (FullHD 4:2:0 by default).  The flow of inter frame t is
    the exact backward displacement from frame t to frame t-1.  With
    ``coef_mode`` the inter frames carry coefficient-mode residuals
    (:class:`PFrameCoef`); with ``rct`` the colour planes are the 4:4:4
    planes Y, U, V of the reversible colour transform (Sec. 2.3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rct = bool(rct and chroma)
    planes = _scene_planes(rng, width, height, chroma, rct)
    center = (width / 2.0, height / 2.0)
    rots = [0.0]
    shifts = [np.zeros(2)]
    for _ in range(n_frames - 1):
        rots.append(rots[-1] + np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg)))
        shifts.append(shifts[-1] + rng.uniform(-max_shift, max_shift, size=2))

    def render_frame(t):
        return tuple(_render(tex, xs, ys, rots[t], shifts[t], c) for (tex, xs, ys, c) in planes)

    src0 = render_frame(0)
    sources = [src0] if with_sources else []
    ifr = _intra(rng, width, height, chroma, src0, mask_frac, chroma_mask_frac, rct)
    rkw = dict(lam_y=lam_y, lam_c=lam_c, vmax=vmax, rct=rct, **(residual_kw or {}))
    if iframe_residual:
        ifr.res = _frame_residuals(rng, width, height, chroma, block, **rkw)

    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    cx, cy = center
    pframes = []
    for t in range(1, n_frames):
        # x' = c + R(-rot_{t-1}) (R(rot_t)(x - c) + shift_t - shift_{t-1})
        ct, st = np.cos(rots[t]), np.sin(rots[t])
        cp, sp = np.cos(rots[t - 1]), np.sin(rots[t - 1])
        dxs, dys = xs - cx, ys - cy
        px = ct * dxs - st * dys + shifts[t][0] - shifts[t - 1][0]
        py = st * dxs + ct * dys + shifts[t][1] - shifts[t - 1][1]
        qx = cp * px + sp * py + cx
        qy = -sp * px + cp * py + cy
        flow = np.stack([qx - xs, qy - ys], axis=-1).astype(np.float32)
        if coef_mode:
            res = coef_frame_residuals(rng, width, height, chroma, block, lam_y=lam_y, lam_c=lam_c, rct=rct,
                                       **(coef_kw or {}))
            pframes.append(PFrameCoef(flow, res))
        else:
            pframes.append(PFrame(flow, _frame_residuals(rng, width, height, chroma, block, **rkw)))
        if with_sources:
            sources.append(render_frame(t))
    return Gop(width, height, chroma, block, ifr, pframes, sources, rct)


# ----------------------------------------------------------------------------
# side information: rectangular subdivision trees (Sec. 2.3)
# ----------------------------------------------------------------------------
def _pack_bits(bits: List[int]) -> np.ndarray:
    """LSB-first in 32-bit words."""
    n = len(bits)
    words = np.zeros(max(1, (n + 31) // 32), np.uint32)
    if n:
        b = np.asarray(bits, np.uint64)
        idx = np.arange(n)
        np.bitwise_or.at(words, idx >> 5, (b << (idx & 31).astype(np.uint64)).astype(np.uint32))
    return words


def _random_tree_bits(rng, w: int, h: int, n_leaves: int) -> List[int]:
    """Breadth-first split bits of a random subdivision of a w x h rectangle
    with about n_leaves leaves: random leaves (of two or more pixels) are
    split until the count is reached.  A split halves the longer side (the
    first part is the larger one); the format is the decoder's input, the
    tree itself is not kept."""
    children = {}
    rect = {0: (w, h)}
    leaves = [0]
    nxt = 1
    target = max(1, min(int(n_leaves), w * h))
    while len(leaves) < target:
        k = -1
        for _ in range(32):  # a random leaf of two or more pixels
            j = int(rng.integers(len(leaves)))
            if rect[leaves[j]][0] * rect[leaves[j]][1] >= 2:
                k = j
                break
        if k < 0:
            cand = [i for i, l in enumerate(leaves) if rect[l][0] * rect[l][1] >= 2]
            if not cand:
                break
            k = cand[int(rng.integers(len(cand)))]
        node = leaves[k]
        leaves[k] = leaves[-1]
        leaves.pop()
        cw, ch = rect[node]
        if cw >= ch:
            rect[nxt], rect[nxt + 1] = (cw - cw // 2, ch), (cw // 2, ch)
        else:
            rect[nxt], rect[nxt + 1] = (cw, ch - ch // 2), (cw, ch // 2)
        children[node] = (nxt, nxt + 1)
        leaves += [nxt, nxt + 1]
        nxt += 2
    bits, queue, qi = [], [0], 0
    while qi < len(queue):
        node = queue[qi]
        qi += 1
        if node in children:
            bits.append(1)
            queue += list(children[node])
        else:
            bits.append(0)
    return bits


def make_flow_tree(rng, width: int, height: int, n_leaves: int = 400, vmax: float = 4.0):
    """A piecewise-constant backward flow as its side information: the
    breadth-first split bits of a random subdivision (packed words, bit
    count) and one (dx, dy) per leaf, uniform in [-vmax, vmax]."""
    bits = _random_tree_bits(rng, width, height, n_leaves)
    n = sum(1 for b in bits if b == 0)
    values = rng.uniform(-vmax, vmax, size=(n, 2)).astype(np.float32)
    return _pack_bits(bits), len(bits), values


def make_block_trees(rng, width: int, height: int, block: int, lam: float = 8.0):
    """Residual mask side information: per block of the plane (raster
    order, edge blocks cropped) the split bits of a random subdivision with
    Poisson(lam) leaves (at least one), concatenated; tree_ptr[b] is the
    first bit of block b."""
    nbx, nby, w, h = block_grid(width, height, block)
    allbits, ptr = [], [0]
    for b in range(nbx * nby):
        k = max(1, int(rng.poisson(lam)))
        allbits += _random_tree_bits(rng, int(w[b]), int(h[b]), k)
        ptr.append(len(allbits))
    return _pack_bits(allbits), len(allbits), np.asarray(ptr, np.uint32)
