"""Helpers for the GPU parity tests (imported by test modules marked gpu)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def hivc_module():
    torch_cuda()
    from paper_2008_10273_gb300 import build, hivc

    build.build()
    hivc.lib()
    return hivc


def to_np(t):
    return t.detach().cpu().numpy()


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)


# Parity bar: |GPU - oracle| <= 0.5 grey levels before uint8 rounding, PSNR
# within 0.01 dB, mask pixels bit-exact.  The per-step bounds below are the
# FP32 arithmetic error of each kernel (far inside the bar), so a regression
# shows long before the bar is crossed.
TOL_RECON = 0.5
TOL_PSNR_DB = 0.01
TOL_WARP = 1e-3      # bilinear in FP32 of values <= 255
TOL_BLOCK = 1e-2     # Green's solve + DCT evaluation in FP32, |v| <= 64, K <= 48
TOL_INTRA = 1e-3     # FP64-corrected solve to residual 1e-8
