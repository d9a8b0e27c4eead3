"""The tile weights of the scans, exp(lw - k ln 2): the subtraction of the tile
reference k ln 2 is error-free (TwoSum against a float pair), its remainder
enters to first order, and the exponential is expf (whose stated error is 2
ulp).  Against the exact (FP64) exponential: within 3e-7 relative wherever
the weight is a normal float (2 ulp plus the first-order correction), within
3e-7 of the largest weight in absolute terms everywhere, zero for -inf."""
import numpy as np
import pytest

from paper_1202_6163_gb300 import pf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("k", [0, 1, -1, 7, -40, 150, -150, 5000, -100000, 1 << 20])
def test_tile_weights_against_exact_exp(k):
    pf.load()
    ref = k * np.log(2.0)
    rng = np.random.default_rng(abs(k) + 3)
    # log-weights from the tile's reference down to 160 below it (weights 1 .. e^-160), float32
    d = np.concatenate([-np.logspace(-8, np.log10(160.0), 200000), -rng.uniform(0, 30, 200000), [0.0]])
    lw = (ref + d).astype(np.float32)
    lw = lw[lw <= np.float32(ref) + np.float32(0.7)]  # at most ~1 (the scans take k >= max lw log2 e)
    lw = np.concatenate([lw, np.array([-np.inf], np.float32)])
    d_lw = torch.from_numpy(lw).cuda()
    out = torch.empty_like(d_lw)
    pf.pf_debug_tile_weights(d_lw, lw.size, k, out)
    torch.cuda.synchronize()
    w = out.cpu().numpy().astype(np.float64)
    exact = np.exp(lw.astype(np.float64) - ref)
    assert w[-1] == 0.0 and exact[-1] == 0.0
    assert np.all(np.abs(w - exact) <= 3e-7 * max(1.0, exact.max()))
    big = exact >= 2.0 ** -125
    assert np.all(np.abs(w[big] / exact[big] - 1.0) <= 3e-7)
