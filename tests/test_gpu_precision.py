"""Precision workloads: intra frames solved to max |Lu| <= 1e-10 at 1%, 3%
and 8% masks (FP32 sweeps, float-float outer correction), and block
residuals on the clustered stress set (points of a block inside a 5 x 5
window), each against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_BLOCK, TOL_RECON, hivc_module, to_np, torch_cuda
from workload import make_iframe_only, make_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


@pytest.mark.parametrize("frac", [0.01, 0.03, 0.08])
def test_intra_to_1e10(hv, frac):
    W, H = 480, 270
    _, ifr = make_iframe_only(11, W, H, frac, chroma=True)
    dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-10)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    st = dec.sync()
    assert all(r <= 1e-10 for r in st.resid)
    rec, _ = oracle.OracleDecoder(W, H, True, iframe_tol=1e-10).decode_iframe(ifr)
    for p in range(3):
        g = to_np(dec.reference(p)).astype(np.float64)
        # the reference plane is FP32: the solve is as exact as the storage
        assert np.abs(g - rec[p]).max() <= 1e-4, p
        assert np.abs(g - rec[p]).max() <= TOL_RECON


@pytest.mark.parametrize("frac,seed", [(0.2, 12), (1.0, 13)])
def test_clustered_blocks(hv, frac, seed):
    """K <= 25 points inside a 5 x 5 window: G_PP stays far from singular
    (lambda_min >= (1 - K/N) / 8), so FP32 keeps the block bound."""
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    W, H = 256, 192
    res = make_residual(rng, W, H, 16, 8.0, 64, clustered_frac=frac, cluster_window=5, cluster_kmax=25)
    r = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    bp, pos, val = hv.device_residual(res)
    hv.block_residual(W, H, 16, bp, pos, val, r)
    torch.cuda.synchronize()
    assert np.abs(to_np(r).astype(np.float64) - oracle.block_residual(res)).max() <= TOL_BLOCK
