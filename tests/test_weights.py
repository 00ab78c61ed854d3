"""The committed warm-start network file: its layout matches the network the
oracle defines (seven 3x3x3 convolutions of the U-Net, then the 16-weight
head), it runs at a supported stride, and every parameter is finite.  A
corrupted or mismatched file would otherwise surface only on the GPU."""
import os

import numpy as np

from oracle import net_oracle

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1504_02264_gb300",
                       "weights", "warmstart.npz")


def test_warmstart_file_layout():
    z = np.load(WEIGHTS)
    theta = z["params"]
    n_conv = sum(27 * ci * co for ci, co in zip(net_oracle.CIN, net_oracle.COUT))
    assert theta.dtype == np.float32
    assert theta.shape == (n_conv + net_oracle.HEAD,)
    assert int(z["stride"]) in (1, 2, 4, 8)
    assert np.all(np.isfinite(theta))
    ws, head = net_oracle.unflatten(theta.astype(np.float64))
    assert len(ws) == 7 and head.shape == (net_oracle.HEAD,)
    assert all(np.abs(w).max() > 0 for w in ws)          # every layer trained / initialised


def test_coarse_residual_params_compute_the_scaled_residual():
    """The non-learned coarse correction expressed as network weights: under
    the network oracle they give y = mask * r / rms(r) (at stride 1 on a
    ragged grid, and the block-mean pooled residual prolongated at stride 2)."""
    from paper_1504_02264_gb300 import train
    n = sum(27 * a * b for a, b in zip(net_oracle.CIN, net_oracle.COUT)) + net_oracle.HEAD
    theta = train.coarse_residual_params(n).astype(np.float64)
    rng = np.random.default_rng(0)
    shape = (6, 9, 13)
    m = (rng.random(shape) < 0.8).astype(np.float64)
    r = rng.standard_normal(shape) * m
    y = net_oracle.forward_strided(theta, r, m, 1)
    rms = np.sqrt((m * r * r).sum() / m.sum())
    assert np.abs(y - m * r / rms).max() <= 1e-14
    # stride 2: pooled residual and mask, scaled by the pooled RMS, prolongated
    y2 = net_oracle.forward_strided(theta, r, m, 2)
    assert np.all(y2[m == 0] == 0.0)
    assert np.corrcoef(y2[m > 0], r[m > 0])[0, 1] > 0.3
