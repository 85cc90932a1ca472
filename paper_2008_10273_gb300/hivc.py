"""Thin ctypes binding of libhivc (include/hivc.h).

Argument marshalling only: every decoding step runs in the library's CUDA
kernels.  Device arrays are passed as torch CUDA tensors (their
``data_ptr()``); streams as ``torch.cuda.Stream`` or raw handles.  There is
no fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhivc.so")

HIVC_OK = 0
HIVC_E_INVALID = -1
HIVC_E_NOMEM = -2
HIVC_E_CUDA = -3
HIVC_E_NOT_CONVERGED = -4
HIVC_E_NO_REFERENCE = -5
HIVC_E_BUDGET = -6
HIVC_E_TIMEOUT = -7
STAT_KERNELS = 8
KERNEL_FAMILIES = ("intra_setup", "intra_sweeps", "intra_residual", "block_coef",
                   "inter_pixels", "block_eval", "warp_add", "intra_coarse_sweeps")

c_i32, c_u32, c_f64, c_f32, c_vp, c_sz = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_double,
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t)


class Config(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("chroma", c_i32), ("block", c_i32),
                ("op", c_i32), ("precision", c_i32), ("iframe_tol", c_f64), ("max_cycles", c_i32),
                ("cond_threshold", c_f64), ("stream", c_vp), ("layout_groups", c_i32),
                ("batch_frames", c_i32), ("fused_residual", c_i32), ("flat_start", c_i32)]


class Points(ctypes.Structure):
    _fields_ = [("n", c_i32), ("idx", c_vp), ("val", c_vp)]


class Residual(ctypes.Structure):
    _fields_ = [("block_ptr", c_vp), ("pos", c_vp), ("val", c_vp), ("n_points", c_i32)]


class CoefResidual(ctypes.Structure):
    _fields_ = [("block_ptr", c_vp), ("pos", c_vp), ("q", c_vp), ("a", c_vp), ("n_points", c_i32),
                ("step", c_f32), ("offset", c_f32)]


class IFrame(ctypes.Structure):
    _fields_ = [("y", Points), ("c_n", c_i32), ("c_idx", c_vp), ("cb_val", c_vp), ("cr_val", c_vp),
                ("res", ctypes.POINTER(Residual)), ("cu_val", c_vp), ("cv_val", c_vp)]


class PFrame(ctypes.Structure):
    _fields_ = [("flow", c_vp), ("res", Residual * 3)]


class PFrameCoef(ctypes.Structure):
    _fields_ = [("flow", c_vp), ("res", CoefResidual * 3)]


class Out(ctypes.Structure):
    _fields_ = [("plane", c_vp * 3), ("pitch", c_i32 * 3)]


class Frame(ctypes.Structure):
    _fields_ = [("type", c_i32), ("i", ctypes.POINTER(IFrame)), ("p", ctypes.POINTER(PFrame))]


class Stats(ctypes.Structure):
    _fields_ = [("resid", c_f64 * 3), ("cycles", c_i32), ("sweeps", c_i32), ("fp64_blocks", c_i32),
                ("large_blocks", c_i32), ("max_cond", c_f32), ("device_flags", c_u32),
                ("frames", c_i32), ("launches", c_i32), ("kernel_ms", c_f32 * STAT_KERNELS),
                ("kernel_launches", c_i32 * STAT_KERNELS), ("kernel_pixels", ctypes.c_int64 * STAT_KERNELS),
                ("group_blocks", c_i32), ("layout_groups", c_i32)]


_lib = None

# (name, restype, argtypes) for every function include/hivc.h declares
PROTOTYPES = [
    ("hivc_config_default", None, [ctypes.POINTER(Config)]),
    ("hivc_decoder_create", c_i32, [ctypes.POINTER(Config), ctypes.POINTER(c_vp)]),
    ("hivc_decoder_bytes", c_sz, [ctypes.POINTER(Config)]),
    ("hivc_decode_iframe", c_i32, [c_vp, ctypes.POINTER(IFrame), ctypes.POINTER(Out)]),
    ("hivc_decode_pframe", c_i32, [c_vp, ctypes.POINTER(PFrame), ctypes.POINTER(Out)]),
    ("hivc_decode_batch", c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(Frame), c_i32, ctypes.POINTER(Out)]),
    ("hivc_decode_pframe_coef", c_i32, [c_vp, ctypes.POINTER(PFrameCoef), ctypes.POINTER(Out)]),
    ("hivc_block_residual_coef", c_i32, [c_i32, c_i32, c_i32, c_i32, ctypes.POINTER(CoefResidual), c_vp, c_i32,
                                         c_vp, c_vp]),
    ("hivc_decoder_sync", c_i32, [c_vp, ctypes.POINTER(Stats)]),
    ("hivc_decoder_set_timing", c_i32, [c_vp, c_i32]),
    ("hivc_decoder_reset", c_i32, [c_vp]),
    ("hivc_set_sor_variant", c_i32, [c_i32]),
    ("hivc_decoder_reference", c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_i32),
                                       ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    ("hivc_decoder_intra_solution", c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp),
                                            ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    ("hivc_decoder_stream", c_vp, [c_vp]),
    ("hivc_tune_lookup", c_i32, [ctypes.c_char_p]),
    ("hivc_tune_record", c_i32, [ctypes.c_char_p, c_i32]),
    ("hivc_decoder_destroy", None, [c_vp]),
    ("hivc_status_str", ctypes.c_char_p, [c_i32]),
    ("hivc_block_residual_workspace_bytes", c_sz, [c_i32, c_i32, c_i32, c_i32]),
    ("hivc_block_residual", c_i32, [c_i32, c_i32, c_i32, ctypes.POINTER(Residual), c_vp, c_i32, c_vp, c_sz,
                                    c_vp, c_vp]),
    ("hivc_block_residual_static", c_i32, [c_i32, c_i32, c_i32, ctypes.POINTER(Residual), c_vp, c_i32, c_vp,
                                           c_vp]),
    ("hivc_warp", c_i32, [c_i32, c_i32, c_vp, c_i32, c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp]),
    ("hivc_flow_from_tree_workspace_bytes", c_sz, [ctypes.c_int64]),
    ("hivc_flow_from_tree", c_i32, [c_i32, c_i32, c_vp, ctypes.c_int64, c_vp, c_i32, c_vp, c_vp, c_sz, c_vp, c_vp]),
    ("hivc_masks_from_trees", c_i32, [c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp]),
    ("hivc_intra_mask_from_tree_workspace_bytes", c_sz, [c_i32, c_i32, ctypes.c_int64]),
    ("hivc_intra_mask_from_tree", c_i32, [c_i32, c_i32, c_vp, ctypes.c_int64, c_vp, ctypes.c_int64, c_vp, c_vp, c_sz,
                                          c_vp, c_vp]),
]


def lib():
    """Load libhivc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhivc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in PROTOTYPES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HivcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().hivc_status_str(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def check(status: int, what: str = "") -> int:
    if status != HIVC_OK:
        raise HivcError(status, what)
    return status


def _ptr(t) -> int:
    """Device pointer of a tensor (0 for None or an empty tensor)."""
    if t is None:
        return 0
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("device (CUDA) tensor expected")
        if not t.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return t.data_ptr() if t.numel() > 0 else 0
    return int(t)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def config_default() -> Config:
    c = Config()
    lib().hivc_config_default(ctypes.byref(c))
    return c


def coef_residual_struct(r) -> CoefResidual:
    """``r``: the dict of :func:`device_coef_residual`."""
    c = CoefResidual()
    c.block_ptr = _ptr(r["block_ptr"])
    c.pos = _ptr(r["pos"])
    c.q = _ptr(r["q"])
    c.a = _ptr(r["a"])
    c.n_points = int(r["pos"].numel())
    c.step = float(r["step"])
    c.offset = float(r["offset"])
    return c


def residual_struct(block_ptr, pos, val) -> Residual:
    r = Residual()
    r.block_ptr = _ptr(block_ptr)
    r.pos = _ptr(pos)
    r.val = _ptr(val)
    r.n_points = int(pos.numel()) if pos is not None else 0
    return r


class _DeviceArray:
    """Exposes a raw device pointer to torch via __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr, strides=None):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": strides}


class Decoder:
    """Owns one ``hivc_decoder``.  Frames are dicts of torch CUDA tensors
    (see :func:`device_iframe` / :func:`device_pframe`)."""

    def __init__(self, width: int, height: int, chroma: bool = True, block: int = 16,
                 iframe_tol: float = 1e-8, max_cycles: int = 40, precision: int = 0,
                 stream=None, timing: bool = False, cond_threshold: float = 1e6, op: int = 0,
                 layout_groups: Optional[bool] = None, batch_frames: int = 0, fused_residual: bool = False,
                 flat_start: bool = False):
        cfg = config_default()
        # chroma: False/0 grey, True/1 4:2:0, 2 the 4:4:4 RCT colour path
        cfg.width, cfg.height, cfg.chroma, cfg.block = width, height, int(chroma), block
        cfg.iframe_tol, cfg.max_cycles, cfg.precision = iframe_tol, max_cycles, precision
        cfg.cond_threshold = cond_threshold
        cfg.op = op
        if layout_groups is not None:
            cfg.layout_groups = int(bool(layout_groups))
        cfg.batch_frames = int(batch_frames)
        cfg.fused_residual = int(bool(fused_residual))
        cfg.flat_start = int(bool(flat_start))
        cfg.stream = _stream_handle(stream)
        self.cfg = cfg
        self.width, self.height, self.chroma, self.block = width, height, bool(chroma), block
        self.rct = int(chroma) == 2
        h = c_vp()
        check(lib().hivc_decoder_create(ctypes.byref(cfg), ctypes.byref(h)), "hivc_decoder_create")
        self.handle = h
        self._keep = []
        if timing:
            check(lib().hivc_decoder_set_timing(self.handle, 1))

    # -- lifetime ------------------------------------------------------------
    def reset(self):
        """Forget the reference frame: the next frame must be an intra frame."""
        check(lib().hivc_decoder_reset(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().hivc_decoder_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream_handle(self) -> int:
        return lib().hivc_decoder_stream(self.handle) or 0

    @staticmethod
    def bytes_for(width, height, chroma=True, block=16) -> int:
        cfg = config_default()
        # chroma: False/0 grey, True/1 4:2:0, 2 the 4:4:4 RCT colour path
        cfg.width, cfg.height, cfg.chroma, cfg.block = width, height, int(chroma), block
        return int(lib().hivc_decoder_bytes(ctypes.byref(cfg)))

    # -- decoding --------------------------------------------------------------
    def _out(self, out) -> Out:
        o = Out()
        for k, t in enumerate(out):
            o.plane[k] = _ptr(t)
            o.pitch[k] = int(t.stride(0))
        return o

    def iframe_struct(self, f) -> IFrame:
        s = IFrame()
        s.y.n = int(f["y_idx"].numel())
        s.y.idx = _ptr(f["y_idx"])
        s.y.val = _ptr(f["y_val"])
        if self.chroma:
            s.c_n = int(f["c_idx"].numel())
            s.c_idx = _ptr(f["c_idx"])
            if "cu_val" in f:  # 4:4:4 RCT planes: signed chroma values
                s.cu_val = _ptr(f["cu_val"])
                s.cv_val = _ptr(f["cv_val"])
            else:
                s.cb_val = _ptr(f["cb_val"])
                s.cr_val = _ptr(f["cr_val"])
        if f.get("res") is not None:
            arr = (Residual * 3)(*[residual_struct(*r) for r in f["res"]])
            s.res = ctypes.cast(arr, ctypes.POINTER(Residual))
            self._keep.append(arr)
        return s

    def pframe_struct(self, f) -> PFrame:
        s = PFrame()
        s.flow = _ptr(f["flow"])
        for k, r in enumerate(f["res"]):
            s.res[k] = residual_struct(*r)
        return s

    def decode_iframe(self, f, out, allow_not_converged: bool = False) -> int:
        s = self.iframe_struct(f)
        st = lib().hivc_decode_iframe(self.handle, ctypes.byref(s), ctypes.byref(self._out(out)))
        self._keep.clear()
        if not (allow_not_converged and st == HIVC_E_NOT_CONVERGED):
            check(st, "hivc_decode_iframe")
        return st

    def decode_pframe(self, f, out) -> int:
        s = self.pframe_struct(f)
        return check(lib().hivc_decode_pframe(self.handle, ctypes.byref(s), ctypes.byref(self._out(out))),
                     "hivc_decode_pframe")

    def decode_pframe_coef(self, f, out) -> int:
        """Inter frame with a coefficient-mode residual (``f`` from
        :func:`device_pframe_coef`)."""
        s = PFrameCoef()
        s.flow = _ptr(f["flow"])
        for k, r in enumerate(f["res"]):
            s.res[k] = coef_residual_struct(r)
        return check(lib().hivc_decode_pframe_coef(self.handle, ctypes.byref(s), ctypes.byref(self._out(out))),
                     "hivc_decode_pframe_coef")

    def sync(self, raise_on_error: bool = True) -> Stats:
        st = Stats()
        s = lib().hivc_decoder_sync(self.handle, ctypes.byref(st))
        if raise_on_error:
            check(s, "hivc_decoder_sync")
        self.last_status = s
        return st

    def reference(self, plane: int):
        """Copy of the current FP32 reference plane as a torch tensor."""
        import torch

        p, w, h, pitch = c_vp(), c_i32(), c_i32(), c_i32()
        check(lib().hivc_decoder_reference(self.handle, plane, ctypes.byref(p), ctypes.byref(w),
                                           ctypes.byref(h), ctypes.byref(pitch)), "hivc_decoder_reference")
        arr = _DeviceArray(p.value, (h.value, w.value), "<f4", (pitch.value * 4, 4))
        torch.cuda.synchronize()
        return torch.as_tensor(arr, device="cuda").clone()


    def intra_solution(self, plane: int):
        """Copies (hi, lo) of the last intra frame's diffusion iterate of one
        plane as FP32 torch tensors (lo is None in FP32-only mode); the
        solution is hi + lo."""
        import torch

        hi, lo, w, h, pitch = c_vp(), c_vp(), c_i32(), c_i32(), c_i32()
        check(lib().hivc_decoder_intra_solution(self.handle, plane, ctypes.byref(hi), ctypes.byref(lo),
                                                ctypes.byref(w), ctypes.byref(h), ctypes.byref(pitch)),
              "hivc_decoder_intra_solution")
        torch.cuda.synchronize()
        get = lambda p: torch.as_tensor(_DeviceArray(p, (h.value, w.value), "<f4", (pitch.value * 4, 4)),
                                        device="cuda").clone()
        return get(hi.value), (get(lo.value) if lo.value else None)


def decode_batch(decoders: Sequence[Decoder], frames, outs) -> int:
    """Decode frames[k] (('i'|'p', dict)) on decoders[k] into outs[k]."""
    n = len(decoders)
    handles = (c_vp * n)(*[d.handle for d in decoders])
    fr = (Frame * n)()
    keep = []
    for k, (d, (kind, f)) in enumerate(zip(decoders, frames)):
        if kind == "i":
            s = d.iframe_struct(f)
            keep.append(s)
            fr[k].type = 0
            fr[k].i = ctypes.pointer(s)
        else:
            s = d.pframe_struct(f)
            keep.append(s)
            fr[k].type = 1
            fr[k].p = ctypes.pointer(s)
    oa = (Out * n)(*[d._out(o) for d, o in zip(decoders, outs)])
    st = lib().hivc_decode_batch(handles, fr, n, oa)
    for d in decoders:
        d._keep.clear()
    if st not in (HIVC_OK, HIVC_E_NOT_CONVERGED):
        check(st, "hivc_decode_batch")
    return st


# ----------------------------------------------------------------------------
# step entry points
# ----------------------------------------------------------------------------
def block_residual(width, height, block, block_ptr, pos, val, r, workspace=None, flags=None, stream=None):
    res = residual_struct(block_ptr, pos, val)
    need = lib().hivc_block_residual_workspace_bytes(width, height, block, res.n_points)
    if workspace is None:
        import torch

        workspace = torch.empty(need, dtype=torch.uint8, device=r.device)
    return check(lib().hivc_block_residual(width, height, block, ctypes.byref(res), _ptr(r), int(r.stride(0)),
                                           _ptr(workspace), int(workspace.numel()), _ptr(flags),
                                           _stream_handle(stream)), "hivc_block_residual")


def block_residual_static(width, height, block, block_ptr, pos, val, r, flags=None, stream=None):
    """hivc_block_residual_static: the residual plane with the library's
    fixed scratch array (no device allocation anywhere); see include/hivc.h
    for its limits and the rule that calls must not overlap on the GPU."""
    res = residual_struct(block_ptr, pos, val)
    return check(lib().hivc_block_residual_static(width, height, block, ctypes.byref(res), _ptr(r), int(r.stride(0)),
                                                  _ptr(flags), _stream_handle(stream)), "hivc_block_residual_static")


def warp(ref, flow, pred, chroma_flow: bool = False, stream=None):
    h, w = pred.shape
    fh, fw = flow.shape[0], flow.shape[1]
    return check(lib().hivc_warp(w, h, _ptr(ref), int(ref.stride(0)), _ptr(flow), fw, fh, int(chroma_flow),
                                 _ptr(pred), int(pred.stride(0)), _stream_handle(stream)), "hivc_warp")


# ----------------------------------------------------------------------------
# host -> device marshalling of workload objects (numpy -> torch CUDA)
# ----------------------------------------------------------------------------
def _dev(a, device="cuda"):
    import numpy as np
    import torch

    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(device)


def device_residual(res, device="cuda"):
    return (_dev(res.block_ptr, device), _dev(res.pos, device), _dev(res.val, device))


def device_coef_residual(res, device="cuda"):
    """A :class:`workload.CoefResidual` on the device."""
    return {"block_ptr": _dev(res.block_ptr, device), "pos": _dev(res.pos, device), "q": _dev(res.q, device),
            "a": _dev(res.a, device), "step": res.step, "offset": res.offset}


def device_pframe_coef(pfr, device="cuda"):
    return {"flow": _dev(pfr.flow, device), "res": [device_coef_residual(r, device) for r in pfr.res]}


def block_residual_coef(width, height, block, op, res, r, flags=None, stream=None):
    """hivc_block_residual_coef: ``res`` from :func:`device_coef_residual`."""
    c = coef_residual_struct(res)
    return check(lib().hivc_block_residual_coef(width, height, block, op, ctypes.byref(c), _ptr(r),
                                                int(r.stride(0)), _ptr(flags), _stream_handle(stream)),
                 "hivc_block_residual_coef")


def flow_from_tree(width, height, bits, nbits, values, flow, flags=None, workspace=None, stream=None):
    """hivc_flow_from_tree: ``bits`` (int32/uint32 words), ``values``
    (float32 [n, 2]) and ``flow`` (float32 [H, W, 2]) are CUDA tensors."""
    need = lib().hivc_flow_from_tree_workspace_bytes(int(nbits))
    if workspace is None:
        import torch

        workspace = torch.empty(need, dtype=torch.uint8, device=flow.device)
    return check(lib().hivc_flow_from_tree(width, height, _ptr(bits), int(nbits), _ptr(values), int(values.shape[0]),
                                           _ptr(flow), _ptr(workspace), int(workspace.numel()), _ptr(flags),
                                           _stream_handle(stream)), "hivc_flow_from_tree")


def intra_mask_from_tree(width, height, bits, nbits, idx, n_points, flags=None, workspace=None, stream=None):
    """hivc_intra_mask_from_tree: sorted indices into ``idx`` (capacity =
    its length), their count into ``n_points`` (one int32)."""
    need = lib().hivc_intra_mask_from_tree_workspace_bytes(width, height, int(nbits))
    if workspace is None:
        import torch

        workspace = torch.empty(need, dtype=torch.uint8, device=idx.device)
    return check(lib().hivc_intra_mask_from_tree(width, height, _ptr(bits), int(nbits), _ptr(idx), int(idx.numel()),
                                                 _ptr(n_points), _ptr(workspace), int(workspace.numel()), _ptr(flags),
                                                 _stream_handle(stream)), "hivc_intra_mask_from_tree")


def masks_from_trees(width, height, block, bits, tree_ptr, block_ptr, pos, flags=None, stream=None):
    """hivc_masks_from_trees: block_ptr (nblocks + 1) and pos (capacity =
    its length) are written."""
    return check(lib().hivc_masks_from_trees(width, height, block, _ptr(bits), _ptr(tree_ptr), _ptr(block_ptr),
                                             _ptr(pos), int(pos.numel()), _ptr(flags), _stream_handle(stream)),
                 "hivc_masks_from_trees")


def device_iframe(ifr, device="cuda"):
    f = {"y_idx": _dev(ifr.y_idx, device), "y_val": _dev(ifr.y_val, device)}
    if ifr.chroma and getattr(ifr, "rct", False):
        f.update(c_idx=_dev(ifr.c_idx, device), cu_val=_dev(ifr.cb_val, device), cv_val=_dev(ifr.cr_val, device))
    elif ifr.chroma:
        f.update(c_idx=_dev(ifr.c_idx, device), cb_val=_dev(ifr.cb_val, device), cr_val=_dev(ifr.cr_val, device))
    if ifr.res is not None:
        f["res"] = [device_residual(r, device) for r in ifr.res]
    return f


def device_pframe(pfr, device="cuda", shared_chroma: bool = True):
    res = [device_residual(r, device) for r in pfr.res]
    if shared_chroma and len(res) == 3:
        import numpy as np

        if np.array_equal(pfr.res[1].pos, pfr.res[2].pos) and np.array_equal(pfr.res[1].block_ptr,
                                                                              pfr.res[2].block_ptr):
            res[2] = (res[1][0], res[1][1], res[2][2])
    return {"flow": _dev(pfr.flow, device), "res": res}


def _map_tensors(obj, fn):
    """obj with every tensor t (in dicts, lists, tuples) replaced by fn(t)."""
    import torch

    if isinstance(obj, torch.Tensor):
        return fn(obj)
    if isinstance(obj, dict):
        return {k: _map_tensors(v, fn) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return type(obj)(_map_tensors(v, fn) for v in obj)
    return obj


class FramePack:
    """The inputs of several frames in one pinned host buffer and one device
    buffer of the same layout (every array at a 256-byte offset), so that a
    single host-to-device copy moves all of them.

    ``frames`` are ``("i" | "p", frame dict)`` as made by :func:`device_iframe`
    and :func:`device_pframe` (tensors on any device).  :meth:`frames` gives
    the same dicts with every tensor a view of the device buffer; an array
    that several planes share (a shared chroma layout) stays one array, so
    the decoder still sees the shared layout."""

    def __init__(self, frames, device="cuda"):
        import torch

        place = {}
        off = 0

        def note(t):
            nonlocal off
            if id(t) not in place:
                place[id(t)] = (t, off)
                off += -(-t.numel() * t.element_size() // 256) * 256
            return t

        _map_tensors(list(frames), note)
        self.nbytes = off
        self.host = torch.empty(max(off, 256), dtype=torch.uint8)
        if torch.cuda.is_available():
            self.host = self.host.pin_memory()
        self.device = torch.empty(max(off, 256), dtype=torch.uint8, device=device)
        views = {}
        for key, (t, o) in place.items():
            n = t.numel() * t.element_size()
            self.host[o:o + n].view(t.dtype).copy_(t.reshape(-1).cpu())
            views[key] = self.device[o:o + n].view(t.dtype).view(t.shape)
        self._frames = [(kind, _map_tensors(f, lambda t: views[id(t)])) for kind, f in frames]

    def upload(self):
        """One host-to-device copy of every input, on the current stream."""
        self.device[:self.nbytes].copy_(self.host[:self.nbytes], non_blocking=True)

    def frames(self):
        return self._frames


def alloc_out_block(n, width, height, chroma=True, device="cuda"):
    """Output planes of n frames (as :func:`alloc_out`) as views of one
    uint8 device buffer (planes at 256-byte offsets), so that one
    device-to-host copy brings all of them back.  Returns (buffer, outs)."""
    import torch

    cw, ch = (width + 1) // 2, (height + 1) // 2
    shapes = [(height, width)]
    if int(chroma) == 2:
        shapes += [(height, width)] * 2
    elif chroma:
        shapes += [(ch, cw)] * 2
    sizes = [-(-h * w // 256) * 256 for h, w in shapes]
    per = sum(sizes)
    buf = torch.empty(max(n * per, 256), dtype=torch.uint8, device=device)
    outs = []
    for k in range(n):
        o, planes = k * per, []
        for (h, w), sz in zip(shapes, sizes):
            planes.append(buf[o:o + h * w].view(h, w))
            o += sz
        outs.append(planes)
    return buf[:n * per], outs


def alloc_out(width, height, chroma=True, device="cuda"):
    """uint8 output planes: Y (+ Cb, Cr at 4:2:0); chroma=2: R, G, B."""
    import torch

    planes = [torch.empty((height, width), dtype=torch.uint8, device=device)]
    if int(chroma) == 2:
        planes += [torch.empty((height, width), dtype=torch.uint8, device=device) for _ in range(2)]
    elif chroma:
        cw, ch = (width + 1) // 2, (height + 1) // 2
        planes += [torch.empty((ch, cw), dtype=torch.uint8, device=device) for _ in range(2)]
    return planes
