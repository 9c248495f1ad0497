"""Host-side logic of the serving loop (no GPU): device footprints used for
admission and the one-at-a-time FIFO baseline."""
import numpy as np

import paper_2501_01461_gb300 as cg
from paper_2501_01461_gb300 import serve


def test_fft_footprint_counts_the_grids():
    g = serve.footprint_bytes(1024, (2048, 2048), 10000, (2, 2), 50)
    f = serve.footprint_bytes(1024, (2048, 2048), 10000, (2, 2), 50, cg.FB_FFT)
    L = 2048  # smallest even 2-3-5-7-smooth size >= 2 * 1024 - 1
    # kernel spectrum, the column work area (image rows only), the round's
    # components (4 tiles x K 50), both twiddle tables, the round-start residual
    # twiddles of 2048 = 8 x 8 x 8 x 4: the L roots, then r Ns entries a stage
    tw = L + 8 + 64 + 512 + 2048
    assert f - g == (8 * L * (L // 2 + 1) + 8 * 1024 * (L // 2 + 1) + 24 * 4 * 50 + 16
                     + 2 * 8 * tw + 4 * 1024 * 1024)
    assert serve.footprint_bytes(512, (1024, 1024), 100, (1, 1), 50, cg.FB_FFT) == \
        serve.footprint_bytes(512, (1024, 1024), 100, (1, 1), 50)


def test_fifo_latencies():
    # arrivals 0, 1, 1.5 with service 2, 1, 1: finishes at 2, 3, 4
    lat = serve.fifo_latencies([0.0, 1.0, 1.5], [2.0, 1.0, 1.0])
    assert np.allclose(lat, [2.0, 2.0, 2.5])
    # unsorted input is served in arrival order
    assert np.allclose(sorted(serve.fifo_latencies([1.0, 0.0], [1.0, 1.0])), [1.0, 1.0])
