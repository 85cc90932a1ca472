"""Parity of the benchmarked workload: the FullHD 4:2:0 GOP of 30 frames
(seed 0: 1 intra frame with a 3% luma / 1.5% shared chroma mask solved to
max |Lu| <= 1e-8, then 29 inter frames with dense backward flow and 16 x 16
residual blocks) decoded through hivc_decode_batch exactly as the benchmark
decodes it, frame by frame against the FP64 oracle (Sec. 2: prediction +
correction in a closed loop, so every inter frame inherits the drift of the
frames before it).

Per frame and plane: the max |GPU FP32 reference - oracle| before uint8
rounding, PSNR(GPU) - PSNR(oracle) against the synthetic source, the uint8
outputs' largest difference and the share of pixels that differ (rounding
ties), and, for the intra frame, whether the mask pixels are bit-exact.

Each frame's FP32 reference comes from a batch call on the GOP's first
t + 1 frames (the reference after a call is its last frame's); the uint8
outputs come from one call on the whole GOP, the benchmark's call, and must
equal the prefix calls' outputs bit for bit.  Run on a GPU machine:

    python tests/gop_parity_report.py > report.json
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
from workload import make_gop  # noqa: E402


def gop_parity(seed: int = 0, width: int = 1920, height: int = 1080, n_frames: int = 30,
               iframe_tol: float = 1e-8) -> dict:
    from paper_2008_10273_gb300 import hivc

    W, H = width, height
    gop = make_gop(seed, W, H, n_frames=n_frames)
    want = oracle.decode_gop(gop)  # FP64, intra solved to 1e-12
    frames = [("i", hivc.device_iframe(gop.iframe))] + [("p", hivc.device_pframe(p)) for p in gop.pframes]
    dec = hivc.Decoder(W, H, chroma=True, iframe_tol=iframe_tol)
    # the benchmark's call: the whole GOP in one batch, one output per frame
    outs = [hivc.alloc_out(W, H) for _ in range(n_frames)]
    hivc.decode_batch([dec] * n_frames, frames, outs)
    st = dec.sync()
    full_u8 = [[o.cpu().numpy() for o in out] for out in outs]
    rows = []
    for t in range(n_frames):
        dec.reset()
        out = [hivc.alloc_out(W, H) for _ in range(t + 1)]
        hivc.decode_batch([dec] * (t + 1), frames[:t + 1], out)
        dec.sync()
        g = [dec.reference(p).cpu().numpy().astype(np.float64) for p in range(3)]
        u8 = [o.cpu().numpy() for o in out[t]]
        rec, o8 = want[t]
        src = gop.sources[t]
        row = {"frame": t, "type": "intra" if t == 0 else "inter",
               "max_abs_err": [float(np.abs(g[p] - rec[p]).max()) for p in range(3)],
               "dpsnr_db": [float(oracle.psnr(g[p], src[p]) - oracle.psnr(rec[p], src[p])) for p in range(3)],
               "u8_max_diff": [int(np.abs(u8[p].astype(int) - o8[p].astype(int)).max()) for p in range(3)],
               "u8_diff_share": [float(np.mean(u8[p] != o8[p])) for p in range(3)],
               "batch_equals_prefix": bool(all(np.array_equal(u8[p], full_u8[t][p]) for p in range(3)))}
        if t == 0:
            idx = [gop.iframe.y_idx, gop.iframe.c_idx, gop.iframe.c_idx]
            vals = [gop.iframe.y_val, gop.iframe.cb_val, gop.iframe.cr_val]
            row["mask_exact"] = bool(all(
                np.array_equal(g[p].reshape(-1)[idx[p].astype(np.int64)], vals[p].astype(np.float64)) and
                np.array_equal(u8[p].reshape(-1)[idx[p].astype(np.int64)], vals[p]) for p in range(3)))
        rows.append(row)
    dec.close()
    return {"workload": f"{W}x{H} 4:2:0 GOP of {n_frames} frames, seed {seed} (the benchmark's), "
                        f"hivc_decode_batch with iframe_tol {iframe_tol:g}, against the FP64 oracle",
            "intra_resid": [float(x) for x in st.resid], "frames": rows,
            "max_abs_err": max(max(r["max_abs_err"]) for r in rows),
            "max_abs_dpsnr_db": max(max(abs(x) for x in r["dpsnr_db"]) for r in rows)}


if __name__ == "__main__":
    print(json.dumps(gop_parity(), indent=1))
