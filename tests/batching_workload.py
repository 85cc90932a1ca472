"""The batching workload of the benchmark, runnable on its own for a
profiler: four FullHD 4:2:0 inter frames (luma blocks with Poisson(8)
points clipped to 0..48, 10% empty, 30% of the full blocks on 8 shared
layouts per frame) decoded by hivc_decode_batch after their intra frame,
``--reps`` times, with or without layout groups.

    python tests/batching_workload.py [--groups] [--reps N]
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--groups", action="store_true", help="group blocks that share a mask layout")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--seed", type=int, default=3)
    a = p.parse_args(argv)
    import torch

    from paper_2008_10273_gb300 import hivc
    from workload import make_gop

    W, H = 1920, 1080
    g = make_gop(a.seed, W, H, n_frames=5, with_sources=False,
                 residual_kw={"kmax": 48, "empty_frac": 0.1, "shared_layouts": 8, "shared_frac": 0.3})
    dec = hivc.Decoder(W, H, chroma=True, layout_groups=a.groups)
    out = hivc.alloc_out(W, H)
    ifr = hivc.device_iframe(g.iframe)
    pfs = [hivc.device_pframe(f) for f in g.pframes]
    for _ in range(a.reps):
        dec.decode_iframe(ifr, out)
        hivc.decode_batch([dec] * 4, [("p", f) for f in pfs], [out] * 4)
        st = dec.sync()
    torch.cuda.synchronize()
    print(f"groups {int(a.groups)}: {st.layout_groups} layout groups, {st.group_blocks} blocks in them")
    dec.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
