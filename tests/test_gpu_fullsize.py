"""The headline workload at full size (4096^2 image, 8192^2 PSF, 4 x 4 tiles,
K = 50, 50000 iterations, gain 0.1) in the launch configuration bench.py
times.

* The first two rounds (1600 minor iterations and both feedbacks, the second
  round replayed from the two-round CUDA graph) equal the float32 oracle bit
  for bit over the whole image.
* The whole run satisfies what holds at any size: 50000 components, at most
  K per tile per round, every component inside its own tile, the model equal
  to the float32 sum of the list in list order, and the identity
  model (*) PSF + residual = dirty (Section 3) on a random sample of pixels,
  evaluated one by one in float64.
"""
import numpy as np
import pytest

import oracle
import paper_2501_01461_gb300 as cg
import synth
from gpu_helpers import assert_bit_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    import torch
    w = synth.workload("tiled-4096")
    data = w.build(threshold=0.0)
    d_psf = torch.from_numpy(data["psf"]).cuda()
    d_dirty = torch.from_numpy(data["dirty"]).cuda()
    return w, data, d_psf, d_dirty


def _run(w, d_psf, d_dirty, max_rounds):
    with cg.Plan(d_psf, w.n, w.n, gain=w.gain, niter=w.niter, threshold=0.0, tiles=w.tiles,
                 feedback_interval=w.feedback_interval) as p:
        p.run(d_dirty, max_rounds=max_rounds)
        r, m, _ = p.get()
        comps = p.components_with_rounds()
        return dict(residual=r.cpu().numpy(), model=m.cpu().numpy(), comps=comps,
                    n=len(comps["y"]), stats=p.stats())


def test_first_two_rounds_bit_exact(workload):
    w, data, d_psf, d_dirty = workload
    g = _run(w, d_psf, d_dirty, 2)
    assert g["stats"]["graph_launches"] == 1     # the pair of rounds came from a graph
    o = oracle.clean_f32(data["dirty"], data["psf"], w.gain, w.niter, 0.0, w.tiles,
                         w.feedback_interval, max_rounds=2)
    assert o.n == 2 * 16 * w.feedback_interval
    assert_bit_exact(g, o, "4096^2 first two rounds")


def test_full_run_properties(workload):
    w, data, d_psf, d_dirty = workload
    g = _run(w, d_psf, d_dirty, -1)
    c = g["comps"]
    ty, tx = w.tiles
    n = w.n
    assert g["n"] == w.niter
    # at most K components per tile per round, each inside its own tile
    key = c["round"].astype(np.int64) * (ty * tx) + c["tile"]
    assert np.bincount(key).max() <= w.feedback_interval
    i, j = c["tile"] // tx, c["tile"] % tx
    assert np.all((c["y"] >= i * n // ty) & (c["y"] < (i + 1) * n // ty))
    assert np.all((c["x"] >= j * n // tx) & (c["x"] < (j + 1) * n // tx))
    # model = float32 sum of the list, in list order
    model = np.zeros((n, n), np.float32)
    np.add.at(model, (c["y"], c["x"]), c["flux"])
    assert np.array_equal(model.view(np.uint32), g["model"].view(np.uint32))
    # identity on 4096 sampled pixels, float64, one pixel at a time
    rng = np.random.default_rng(5)
    qy, qx = rng.integers(0, n, 4096), rng.integers(0, n, 4096)
    nz = np.flatnonzero(g["model"])
    py, px = nz // n, nz % n
    f = g["model"].ravel()[nz].astype(np.float64)
    psf = data["psf"].astype(np.float64)
    cy, cx = psf.shape[0] // 2, psf.shape[1] // 2
    conv = np.array([np.dot(f, psf[y - py + cy, x - px + cx]) for y, x in zip(qy, qx)])
    err = np.abs(conv + g["residual"][qy, qx] - data["dirty"][qy, qx].astype(np.float64))
    bound = 8 * w.niter * 2.0 ** -24 * np.abs(data["dirty"]).max()
    assert err.max() <= bound, (err.max(), bound)
