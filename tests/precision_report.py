"""Precision report: the error of each result against the FP64 oracle at
FullHD 4:2:0.

* Intra frames at 1%, 3% and 8% luma masks (chroma mask at half the
  density, shared by Cb and Cr), diffusion inpainting (Sec. 2.1, Eq. 1)
  solved to max |Lu| <= 1e-10 over the unknown pixels with FP32 sweeps and
  a float-float residual correction.
* An inter frame whose residual blocks are 20% clustered (K <= 25 points
  inside a 5 x 5 window), block solves (Sec. 2.2, Eq. 2) with the default
  condition threshold and with every block re-solved in FP64.

Per plane: max |GPU FP32 reference - oracle| before uint8 rounding, the
PSNR difference against the source, and whether the intra mask pixels of
the uint8 output equal their values.  Run on a GPU machine:

    python tests/precision_report.py > report.json

``tests/test_gpu_precision.py`` runs the same report and checks the bars.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
from workload import make_gop, make_iframe_only  # noqa: E402


def precision_report(seed: int = 0, width: int = 1920, height: int = 1080, fracs=(0.01, 0.03, 0.08)) -> dict:
    import torch

    from paper_2008_10273_gb300 import hivc

    W, H = width, height
    rep = {"intra": [], "blocks": []}

    def planes(dec, n):
        return [dec.reference(p).cpu().numpy().astype(np.float64) for p in range(n)]

    for frac in fracs:
        src, ifr = make_iframe_only(seed + 11, W, H, frac, chroma=True)
        dec = hivc.Decoder(W, H, chroma=True, iframe_tol=1e-10)
        out = hivc.alloc_out(W, H)
        dfr = hivc.device_iframe(ifr)
        s = torch.cuda.ExternalStream(dec.stream_handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        dec.decode_iframe(dfr, out)
        e1.record(s)
        st = dec.sync()
        g = planes(dec, 3)
        rec, _ = oracle.OracleDecoder(W, H, True, iframe_tol=1e-10).decode_iframe(ifr)
        idx = [ifr.y_idx, ifr.c_idx, ifr.c_idx]
        vals = [ifr.y_val, ifr.cb_val, ifr.cr_val]
        rep["intra"].append({
            "mask": frac, "tol": 1e-10, "resid": [float(x) for x in st.resid], "cycles": int(st.cycles),
            "sweeps": int(st.sweeps), "gpu_ms": e0.elapsed_time(e1),
            "max_abs_err": [float(np.abs(g[p] - rec[p]).max()) for p in range(3)],
            "dpsnr_db": [float(oracle.psnr(g[p], src[p]) - oracle.psnr(rec[p], src[p])) for p in range(3)],
            "mask_exact": bool(all(np.array_equal(out[p].cpu().numpy().reshape(-1)[idx[p].astype(np.int64)],
                                                  vals[p]) for p in range(3)))})
        dec.close()
    gop = make_gop(seed + 21, W, H, n_frames=2,
                   residual_kw={"clustered_frac": 0.2, "cluster_window": 5, "cluster_kmax": 25})
    rec = oracle.decode_gop(gop)[-1][0]
    for thr in (1e6, 0.0):
        dec = hivc.Decoder(W, H, chroma=True, cond_threshold=thr)
        out = hivc.alloc_out(W, H)
        dec.decode_iframe(hivc.device_iframe(gop.iframe), out)
        dec.sync()
        dec.decode_pframe(hivc.device_pframe(gop.pframes[0]), out)
        st = dec.sync()
        g = planes(dec, 3)
        rep["blocks"].append({
            "cond_threshold": thr, "fp64_blocks": int(st.fp64_blocks), "max_cond_bound": float(st.max_cond),
            "max_abs_err": [float(np.abs(g[p] - rec[p]).max()) for p in range(3)],
            "dpsnr_db": [float(oracle.psnr(g[p], gop.sources[-1][p]) - oracle.psnr(rec[p], gop.sources[-1][p]))
                         for p in range(3)]})
        dec.close()
    rep["workload"] = (f"{W}x{H} 4:2:0 intra frames ({'/'.join(f'{100 * f:g}' for f in fracs)}% luma masks, "
                       "half-density shared chroma mask) to max |Lu| <= 1e-10; an inter frame with 20% of the "
                       "residual blocks clustered (K <= 25 in a 5 x 5 window); FP32 references against the "
                       "FP64 oracle, per plane (Y, Cb, Cr)")
    return rep


if __name__ == "__main__":
    print(json.dumps(precision_report(), indent=1))
