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
