"""FP64 CPU oracle of the decoder reconstruction (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The CUDA decoder never calls it and shares no code
with it; its inputs come from :mod:`workload`.

The arithmetic lives in ``hivc_oracle.c`` (plain loops, double precision),
compiled with gcc into ``oracle/_build``.  This module adds the frame and GOP
composition of Sec. 2: prediction (diffusion inpainting for intra frames,
backward warping for inter frames) plus the block residual correction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hivc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhivc_oracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, INVALID = 0, 1, -1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i16p = ctypes.POINTER(ctypes.c_int16)
            f32p = ctypes.POINTER(ctypes.c_float)
            ip = ctypes.POINTER(ctypes.c_int)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            L.oracle_inpaint.argtypes = [c_int, c_int, u32p, dp, c_int, c_double, c_int, dp, dp, ip]
            L.oracle_inpaint.restype = c_int
            L.oracle_inpaint_residual.argtypes = [c_int, c_int, u8p, dp]
            L.oracle_inpaint_residual.restype = c_double
            L.oracle_warp.argtypes = [c_int, c_int, dp, dp, dp]
            L.oracle_warp.restype = None
            L.oracle_chroma_flow.argtypes = [c_int, c_int, f32p, c_int, c_int, dp]
            L.oracle_chroma_flow.restype = None
            L.oracle_block_eigenvalue.argtypes = [c_int, c_int, c_int, c_int]
            L.oracle_block_eigenvalue.restype = c_double
            L.oracle_green_matrix.argtypes = [c_int, c_int, dp]
            L.oracle_green_matrix.restype = None
            L.oracle_block_solve.argtypes = [c_int, c_int, dp, c_int, u8p, dp, dp, dp, dp]
            L.oracle_block_solve.restype = c_int
            L.oracle_block_residual.argtypes = [c_int, c_int, c_int, u32p, u8p, i16p, dp]
            L.oracle_block_residual.restype = c_int
            L.oracle_green_matrix_op.argtypes = [c_int, c_int, c_int, dp]
            L.oracle_green_matrix_op.restype = None
            L.oracle_block_residual_op.argtypes = [c_int, c_int, c_int, c_int, u32p, u8p, i16p, dp]
            L.oracle_block_residual_op.restype = c_int
            u32p_ = ctypes.POINTER(ctypes.c_uint32)
            lp = ctypes.POINTER(ctypes.c_long)
            L.oracle_tree_leaves.argtypes = [c_int, c_int, c_int, c_int, u32p_, ctypes.c_long, ctypes.c_long, ip,
                                             c_int, ip, lp]
            L.oracle_tree_leaves.restype = c_int
            L.oracle_flow_from_tree.argtypes = [c_int, c_int, u32p_, ctypes.c_long, f32p, c_int, f32p]
            L.oracle_flow_from_tree.restype = c_int
            L.oracle_masks_from_trees.argtypes = [c_int, c_int, c_int, u32p_, u32p_, u32p_, u8p, ctypes.c_long]
            L.oracle_masks_from_trees.restype = c_int
            L.oracle_intra_mask_from_tree.argtypes = [c_int, c_int, u32p_, ctypes.c_long, u32p_, ip]
            L.oracle_intra_mask_from_tree.restype = c_int
            L.oracle_inverse_rct.argtypes = [c_int, dp, dp, dp, u8p]
            L.oracle_inverse_rct.restype = None
            L.oracle_dequantise.argtypes = [c_int, c_double, c_double]
            L.oracle_dequantise.restype = c_double
            L.oracle_block_residual_coef.argtypes = [c_int, c_int, c_int, c_int, u32p, u8p,
                                                     ctypes.POINTER(ctypes.c_int8), f32p, c_double, c_double, dp]
            L.oracle_block_residual_coef.restype = c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ----------------------------------------------------------------------------
# single steps
# ----------------------------------------------------------------------------
def inpaint(width: int, height: int, idx, val, tol: float = 1e-12,
            max_iter: int = 200000, check: bool = True):
    """Diffusion inpainting of one plane (Sec. 2.1, Eq. 1).

    Returns ``(u, residual, iterations, status)``, ``u`` float64 [H, W]."""
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    u = np.empty((height, width), np.float64)
    res = ctypes.c_double(0.0)
    its = ctypes.c_int(0)
    st = lib().oracle_inpaint(width, height, _p(idx, ctypes.c_uint32), _p(val, ctypes.c_double),
                              int(idx.size), tol, max_iter, _p(u, ctypes.c_double),
                              ctypes.byref(res), ctypes.byref(its))
    if check and st != OK:
        raise RuntimeError(f"oracle_inpaint status {st} (residual {res.value:.3e})")
    return u, res.value, its.value, st


def inpaint_residual(u: np.ndarray, idx) -> float:
    """max over unknown pixels of |(L u)_i| (Eq. 1 residual)."""
    h, w = u.shape
    mask = np.zeros(h * w, np.uint8)
    mask[np.asarray(idx, np.int64)] = 1
    u = np.ascontiguousarray(u, np.float64)
    return lib().oracle_inpaint_residual(w, h, _p(mask, ctypes.c_uint8), _p(u, ctypes.c_double))


def warp(ref: np.ndarray, flow: np.ndarray) -> np.ndarray:
    """Backward bilinear warp pred(x) = ref(x + flow(x)), sample clamped."""
    h, w = ref.shape
    ref = np.ascontiguousarray(ref, np.float64)
    fl = np.ascontiguousarray(flow, np.float64)
    assert fl.shape == (h, w, 2)
    out = np.empty((h, w), np.float64)
    lib().oracle_warp(w, h, _p(ref, ctypes.c_double), _p(fl, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def chroma_flow(flow: np.ndarray, cw: int, ch: int) -> np.ndarray:
    """4:2:0 chroma flow: half the mean of the 2x2 co-sited luma vectors."""
    h, w, _ = flow.shape
    fl = np.ascontiguousarray(flow, np.float32)
    out = np.empty((ch, cw, 2), np.float64)
    lib().oracle_chroma_flow(w, h, _p(fl, ctypes.c_float), cw, ch, _p(out, ctypes.c_double))
    return out


def block_eigenvalue(w: int, h: int, p: int, q: int) -> float:
    return lib().oracle_block_eigenvalue(w, h, p, q)


def green_matrix(w: int, h: int, op: int = 0) -> np.ndarray:
    """Green's matrix on a w x h block (pixel index y*w + x) of the harmonic
    operator A = -L (op 0) or the biharmonic A = L^2 (op 1)."""
    G = np.empty((w * h, w * h), np.float64)
    lib().oracle_green_matrix_op(w, h, op, _p(G, ctypes.c_double))
    return G


def block_solve(w: int, h: int, pos, v, G: Optional[np.ndarray] = None):
    """One block: returns ``(r [h, w], c [K], a)`` (Sec. 2.2, Eqs. 2-3)."""
    if G is None:
        G = green_matrix(w, h)
    pos = np.ascontiguousarray(pos, np.uint8)
    v = np.ascontiguousarray(v, np.float64)
    K = int(pos.size)
    r = np.empty(w * h, np.float64)
    c = np.empty(max(K, 1), np.float64)
    a = ctypes.c_double(0.0)
    st = lib().oracle_block_solve(w, h, _p(np.ascontiguousarray(G), ctypes.c_double), K,
                                  _p(pos, ctypes.c_uint8), _p(v, ctypes.c_double),
                                  _p(r, ctypes.c_double), _p(c, ctypes.c_double), ctypes.byref(a))
    if st != OK:
        raise ValueError(f"oracle_block_solve status {st}")
    return r.reshape(h, w), c[:K], a.value


def block_residual(res, op: int = 0) -> np.ndarray:
    """Residual plane (float64 [H, W]) from a :class:`workload.Residual`
    (values at the points; the decoder solves Eq. 2 per block)."""
    r = np.empty((res.height, res.width), np.float64)
    bp = np.ascontiguousarray(res.block_ptr, np.uint32)
    pos = np.ascontiguousarray(res.pos, np.uint8)
    val = np.ascontiguousarray(res.val, np.int16)
    if pos.size == 0:
        pos = np.zeros(1, np.uint8)
        val = np.zeros(1, np.int16)
    st = lib().oracle_block_residual_op(res.width, res.height, res.block, op, _p(bp, ctypes.c_uint32),
                                        _p(pos, ctypes.c_uint8), _p(val, ctypes.c_int16),
                                        _p(r, ctypes.c_double))
    if st != OK:
        raise ValueError(f"oracle_block_residual status {st}")
    return r


def dequantise(q: int, step: float, offset: float) -> float:
    """Dead-zone reconstruction of one coefficient index (Sec. 2.3)."""
    return lib().oracle_dequantise(int(q), float(step), float(offset))


def block_residual_coef(res, op: int = 0) -> np.ndarray:
    """Residual plane (float64 [H, W]) from a :class:`workload.CoefResidual`
    (coefficient mode: dequantised c and the constant a per block, Eq. 3)."""
    r = np.empty((res.height, res.width), np.float64)
    bp = np.ascontiguousarray(res.block_ptr, np.uint32)
    pos = np.ascontiguousarray(res.pos, np.uint8)
    q = np.ascontiguousarray(res.q, np.int8)
    a = np.ascontiguousarray(res.a, np.float32)
    if pos.size == 0:
        pos = np.zeros(1, np.uint8)
        q = np.zeros(1, np.int8)
    st = lib().oracle_block_residual_coef(res.width, res.height, res.block, op, _p(bp, ctypes.c_uint32),
                                          _p(pos, ctypes.c_uint8), _p(q, ctypes.c_int8), _p(a, ctypes.c_float),
                                          float(res.step), float(res.offset), _p(r, ctypes.c_double))
    if st != OK:
        raise ValueError(f"oracle_block_residual_coef status {st}")
    return r


def to_uint8(recon: np.ndarray) -> np.ndarray:
    """Output rounding (reading): round half up of the clamped value."""
    return np.floor(np.clip(recon, 0.0, 255.0) + 0.5).astype(np.uint8)


# ----------------------------------------------------------------------------
# frames and GOPs (Sec. 2: prediction + correction, closed loop)
# ----------------------------------------------------------------------------
def tree_leaves(width: int, height: int, bits: np.ndarray, nbits: int) -> np.ndarray:
    """Leaves (x0, y0, w, h), breadth-first, of a subdivision tree over a
    width x height rectangle (Sec. 2.3; bit format in hivc_oracle.c)."""
    words = np.ascontiguousarray(bits, np.uint32)
    rects = np.empty((width * height, 4), np.int32)
    nl, used = ctypes.c_int(0), ctypes.c_long(0)
    st = lib().oracle_tree_leaves(0, 0, width, height, _p(words, ctypes.c_uint32), 0, int(nbits),
                                  _p(rects, ctypes.c_int), width * height, ctypes.byref(nl), ctypes.byref(used))
    if st != OK or used.value != nbits:
        raise ValueError("invalid subdivision tree")
    return rects[:nl.value].copy()


def flow_from_tree(width: int, height: int, bits: np.ndarray, nbits: int, values: np.ndarray) -> np.ndarray:
    """Dense flow (float32 [H, W, 2]) from a subdivision tree and one
    vector per leaf (Sec. 2.3: each region gets its average value)."""
    words = np.ascontiguousarray(bits, np.uint32)
    vals = np.ascontiguousarray(values, np.float32).reshape(-1)
    flow = np.zeros((height, width, 2), np.float32)
    st = lib().oracle_flow_from_tree(width, height, _p(words, ctypes.c_uint32), int(nbits), _p(vals, ctypes.c_float),
                                     vals.size // 2, _p(flow, ctypes.c_float))
    if st != OK:
        raise ValueError("invalid subdivision tree")
    return flow


def masks_from_trees(width: int, height: int, block: int, bits: np.ndarray, tree_ptr: np.ndarray):
    """Residual mask positions (block_ptr, pos) from one subdivision tree
    per block (Sec. 2.3)."""
    words = np.ascontiguousarray(bits, np.uint32)
    tp = np.ascontiguousarray(tree_ptr, np.uint32)
    nb = tp.size - 1
    bp = np.zeros(nb + 1, np.uint32)
    cap = width * height
    pos = np.zeros(max(cap, 1), np.uint8)
    st = lib().oracle_masks_from_trees(width, height, block, _p(words, ctypes.c_uint32), _p(tp, ctypes.c_uint32),
                                       _p(bp, ctypes.c_uint32), _p(pos, ctypes.c_uint8), cap)
    if st != OK:
        raise ValueError("invalid subdivision trees")
    return bp, pos[:int(bp[-1])].copy()


def intra_mask_from_tree(width: int, height: int, bits: np.ndarray, nbits: int) -> np.ndarray:
    """Intra mask indices (sorted uint32, y*W + x): the leaf centres of a
    subdivision tree over the plane (Sec. 2.3)."""
    words = np.ascontiguousarray(bits, np.uint32)
    idx = np.zeros(width * height, np.uint32)
    n = ctypes.c_int(0)
    st = lib().oracle_intra_mask_from_tree(width, height, _p(words, ctypes.c_uint32), int(nbits),
                                           _p(idx, ctypes.c_uint32), ctypes.byref(n))
    if st != OK:
        raise ValueError("invalid subdivision tree")
    return idx[:n.value].copy()


def inverse_rct(y: np.ndarray, u: np.ndarray, v: np.ndarray) -> List[np.ndarray]:
    """R, G, B uint8 planes from reconstructed RCT planes (Sec. 2.3)."""
    h, w = y.shape
    out = np.empty(3 * h * w, np.uint8)
    yy, uu, vv = (np.ascontiguousarray(a, np.float64) for a in (y, u, v))
    lib().oracle_inverse_rct(h * w, _p(yy, ctypes.c_double), _p(uu, ctypes.c_double), _p(vv, ctypes.c_double),
                             _p(out, ctypes.c_uint8))
    return [out[k * h * w:(k + 1) * h * w].reshape(h, w) for k in range(3)]


def plane_sizes(width: int, height: int, chroma: bool, rct: bool = False) -> List[Tuple[int, int]]:
    if not chroma:
        return [(width, height)]
    if rct:
        return [(width, height)] * 3
    cw, ch = (width + 1) // 2, (height + 1) // 2
    return [(width, height), (cw, ch), (cw, ch)]


class OracleDecoder:
    """Reference decoder state: the previous reconstruction of each plane,
    kept unrounded (clamped float64) as the inter-frame reference."""

    def __init__(self, width: int, height: int, chroma: bool, block: int = 16,
                 iframe_tol: float = 1e-12, op: int = 0, rct: bool = False):
        """``rct``: the colour path of Sec. 2.3 (4:4:4 RCT planes Y, U, V;
        U and V clamped to [-255, 255]; the output is R, G, B)."""
        self.width, self.height, self.chroma, self.block = width, height, chroma, block
        self.iframe_tol = iframe_tol
        self.op = op
        self.rct = bool(rct) and bool(chroma)
        self.ref: Optional[List[np.ndarray]] = None
        self.last_inpaint: List[Tuple[float, int]] = []

    def decode_iframe(self, ifr):
        sizes = plane_sizes(self.width, self.height, self.chroma, self.rct)
        preds = []
        self.last_inpaint = []
        u, res, its, _ = inpaint(sizes[0][0], sizes[0][1], ifr.y_idx, ifr.y_val, self.iframe_tol)
        preds.append(u)
        self.last_inpaint.append((res, its))
        if self.chroma:
            for vals in (ifr.cb_val, ifr.cr_val):
                u, res, its, _ = inpaint(sizes[1][0], sizes[1][1], ifr.c_idx, vals, self.iframe_tol)
                preds.append(u)
                self.last_inpaint.append((res, its))
        return self._correct(preds, ifr.res)

    def decode_pframe(self, pfr):
        if self.ref is None:
            raise RuntimeError("inter frame before any intra frame")
        sizes = plane_sizes(self.width, self.height, self.chroma, self.rct)
        preds = [warp(self.ref[0], pfr.flow)]
        if self.chroma:
            cf = pfr.flow.astype(np.float64) if self.rct else chroma_flow(pfr.flow, sizes[1][0], sizes[1][1])
            preds += [warp(self.ref[1], cf), warp(self.ref[2], cf)]
        return self._correct(preds, pfr.res)

    def decode_pframe_coef(self, pfr):
        """Inter frame whose residual comes in coefficient mode
        (:class:`workload.PFrameCoef`)."""
        if self.ref is None:
            raise RuntimeError("inter frame before any intra frame")
        sizes = plane_sizes(self.width, self.height, self.chroma, self.rct)
        preds = [warp(self.ref[0], pfr.flow)]
        if self.chroma:
            cf = pfr.flow.astype(np.float64) if self.rct else chroma_flow(pfr.flow, sizes[1][0], sizes[1][1])
            preds += [warp(self.ref[1], cf), warp(self.ref[2], cf)]
        return self._correct(preds, pfr.res, coef=True)

    def _correct(self, preds, residuals, coef: bool = False):
        recon = []
        for k, p in enumerate(preds):
            if residuals is None:
                r = 0.0
            elif coef:
                r = block_residual_coef(residuals[k], self.op)
            else:
                r = block_residual(residuals[k], self.op)
            lo = -255.0 if (self.rct and k > 0) else 0.0
            recon.append(np.clip(p + r, lo, 255.0))
        self.ref = recon
        if self.rct:
            return recon, inverse_rct(*recon)
        return recon, [to_uint8(x) for x in recon]


def decode_gop(gop, n_frames: Optional[int] = None, iframe_tol: float = 1e-12, op: int = 0):
    """Decode the first ``n_frames`` frames of a :class:`workload.Gop`
    (inter frames in values or coefficient mode).  Returns the list of
    (recon float64 planes, uint8 planes) per frame."""
    dec = OracleDecoder(gop.width, gop.height, gop.chroma, gop.block, iframe_tol, op=op,
                        rct=getattr(gop, "rct", False))
    n = gop.n_frames if n_frames is None else n_frames
    out = [dec.decode_iframe(gop.iframe)]
    for t in range(1, n):
        pf = gop.pframes[t - 1]
        out.append(dec.decode_pframe_coef(pf) if hasattr(pf.res[0], "q") else dec.decode_pframe(pf))
    return out


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """10 log10(255^2 / MSE) (reading: the paper reports MSE, Sec. 3)."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)
