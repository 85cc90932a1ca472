"""GB300 (sm_103a) decoder for the inpainting-based video codec of Andris
et al., "Inpainting-based Video Compression in FullHD".

The compute path is libhivc.so (hand-written CUDA behind the C ABI in
include/hivc.h); :mod:`.hivc` is its thin ctypes binding and :mod:`.build`
compiles it.
"""
from . import hivc  # noqa: F401
from .hivc import Decoder, decode_batch, block_residual, warp  # noqa: F401
