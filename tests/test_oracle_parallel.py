"""The multi-core CPU baseline (oracle/clean_parallel.c) equals the float32
oracle bit for bit: components, residual, model and rounds, on one thread
and on several, over grids, intervals, thresholds and ragged tiles."""
import numpy as np
import pytest

import oracle
import synth

CASES = [
    # (n, tiles, K, threshold, niter)
    (40, (2, 2), 5, 0.0, 700),
    (37, (3, 2), 1, 0.01, 600),
    (64, (4, 4), 7, 0.0, 900),
    (30, (1, 1), 0, 0.0, 500),
    (33, (2, 3), 0, 0.0, 500),
    (50, (5, 3), 11, 2e-3, 1200),
]


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-t{c[1][0]}x{c[1][1]}-K{c[2]}" for c in CASES])
def test_parallel_equals_oracle(case, threads):
    n, tiles, K, thr, niter = case
    rng = np.random.default_rng(n + 7 * K)
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 10, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    oracle.parallel_threads(threads)
    a = oracle.clean_f32(dirty, psf, 0.1, niter, thr, tiles, K)
    b = oracle.parallel_clean_f32(dirty, psf, 0.1, niter, thr, tiles, K)
    assert a.n == b.n and a.rounds == b.rounds
    for k in ("y", "x", "tile", "round"):
        assert np.array_equal(a.comps[k], b.comps[k]), k
    assert np.array_equal(a.comps["flux"].view(np.uint32), b.comps["flux"].view(np.uint32))
    assert np.array_equal(a.residual.view(np.uint32), b.residual.view(np.uint32))
    assert np.array_equal(a.model.view(np.uint32), b.model.view(np.uint32))


def test_parallel_max_rounds_and_errors():
    rng = np.random.default_rng(2)
    n = 32
    psf = synth.make_psf(2 * n, 2 * n)
    dirty = synth.random_image(n, n, rng)
    a = oracle.clean_f32(dirty, psf, 0.2, 400, 0.0, (2, 2), 3, max_rounds=4)
    b = oracle.parallel_clean_f32(dirty, psf, 0.2, 400, 0.0, (2, 2), 3, max_rounds=4)
    assert a.n == b.n == 48 and np.array_equal(a.residual, b.residual)
    with pytest.raises(ValueError):
        oracle.parallel_clean_f32(dirty, psf, 1.5, 10)
