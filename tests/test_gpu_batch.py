"""Batched deconvolution: many images of uneven sizes in shared launches.

Each image's component list, residual and model must equal its own solo run
(clean_plan + clean_run) bit for bit -- batching only changes which CTA
serves which tile -- and the small ones must equal the CPU oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2501_01461_gb300 as cg
import synth
from gpu_helpers import assert_bit_exact, gpu_clean

pytestmark = pytest.mark.gpu

JOBS = [
    # (n, tiles, K, niter, threshold, freq_scale)
    (128, (2, 2), 10, 400, 0.0, 1.0),      # tiles resident in shared memory
    (250, (4, 4), 7, 900, 1e-3, 1.3),      # ragged tiles
    (512, (2, 2), 20, 600, 0.0, 1.6),      # streamed tiles
    (96, (3, 2), 0, 300, 0.0, 1.1),        # no feedback (independent tiles)
    (1024, (4, 4), 50, 1600, 5e-3, 2.0),   # larger, with a threshold
    (200, (1, 1), 25, 500, 0.0, 1.8),      # a single tile
]


def _job(n, fs, seed):
    rng = np.random.default_rng(seed)
    psf = synth.make_psf(2 * n, 2 * n, freq_scale=fs)
    ys, xs, fl = synth.make_sky(n, 10, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    return psf, dirty


def test_batch_equals_solo_runs():
    import torch
    data = [_job(n, fs, 100 + i) for i, (n, tiles, K, niter, thr, fs) in enumerate(JOBS)]
    d_psfs = [torch.from_numpy(p).cuda() for p, _ in data]
    d_dirties = [torch.from_numpy(d).cuda() for _, d in data]
    jobs = [dict(psf=d_psfs[i], ny=n, nx=n, gain=0.1, niter=niter, threshold=thr, tiles=tiles,
                 feedback_interval=K) for i, (n, tiles, K, niter, thr, fs) in enumerate(JOBS)]
    with cg.Batch(jobs) as b:
        # rounds replayed from CUDA graphs, then launched one by one; the
        # second run must also start clean
        for rep, graphs in enumerate((True, False)):
            before = b.graphs(graphs)
            b.run(d_dirties)
            assert (b.graphs() > before) == graphs
            for i, (n, tiles, K, niter, thr, fs) in enumerate(JOBS):
                res, mod, comps = b.get(i)
                solo = gpu_clean(data[i][1], data[i][0], 0.1, niter, thr, tiles, K)
                assert len(comps) == solo["n"], (i, rep)
                assert np.array_equal(comps["y"], solo["comps"]["y"])
                assert np.array_equal(comps["x"], solo["comps"]["x"])
                assert np.array_equal(comps["flux"].view(np.uint32),
                                      solo["comps"]["flux"].view(np.uint32))
                assert np.array_equal(res.cpu().numpy().view(np.uint32),
                                      solo["residual"].view(np.uint32)), (i, rep)
                assert np.array_equal(mod.cpu().numpy().view(np.uint32),
                                      solo["model"].view(np.uint32)), (i, rep)
        st = b.stats()
        assert st["n_components"] == sum(len(b.get(i)[2]) for i in range(len(JOBS)))


def test_batch_small_images_equal_oracle_and_resume():
    import torch
    picks = [0, 1, 3]
    data = [_job(JOBS[i][0], JOBS[i][5], 200 + i) for i in picks]
    jobs = []
    for (psf, dirty), i in zip(data, picks):
        n, tiles, K, niter, thr, fs = JOBS[i]
        jobs.append(dict(psf=torch.from_numpy(psf).cuda(), ny=n, nx=n, gain=0.1, niter=niter,
                         threshold=thr, tiles=tiles, feedback_interval=K))
    dirties = [torch.from_numpy(d).cuda() for _, d in data]
    with cg.Batch(jobs) as b:
        b.run(dirties, max_rounds=2)   # stop early, then continue
        b.run(None)
        for k, ((psf, dirty), i) in enumerate(zip(data, picks)):
            n, tiles, K, niter, thr, fs = JOBS[i]
            o = oracle.clean_f32(dirty, psf, 0.1, niter, thr, tiles, K)
            res, mod, comps = b.get(k)
            assert len(comps) == o.n
            assert np.array_equal(comps["flux"].view(np.uint32), o.comps["flux"].view(np.uint32))
            assert np.array_equal(res.cpu().numpy().view(np.uint32), o.residual.view(np.uint32))
            assert np.array_equal(mod.cpu().numpy().view(np.uint32), o.model.view(np.uint32))


def test_batch_rejects_untiled_mode():
    import torch
    psf = torch.from_numpy(synth.make_psf(128, 128)).cuda()
    with pytest.raises(cg.CleanError):
        cg.Batch([dict(psf=psf, ny=64, nx=64, niter=10, mode=cg.UNTILED_GRID)])


def test_batch_with_fft_feedback_equals_solo_runs():
    """FFT-feedback images share the minor-loop launches with gather images
    and run their own transforms; each equals its solo run bit for bit
    (same kernels, same cuFFT plans), with graphs on and off."""
    import torch
    cases = [(256, (2, 2), 10, 600, cg.FB_FFT), (300, (3, 3), 7, 900, cg.FB_GATHER),
             (512, (4, 4), 20, 1600, cg.FB_FFT), (128, (2, 2), 5, 300, cg.FB_AUTO)]
    data = [_job(n, 1.0 + 0.1 * i, 400 + i) for i, (n, *_r) in enumerate(cases)]
    jobs = [dict(psf=torch.from_numpy(p).cuda(), ny=n, nx=n, gain=0.1, niter=niter,
                 threshold=0.0, tiles=tiles, feedback_interval=K, feedback_mode=mode)
            for (p, _), (n, tiles, K, niter, mode) in zip(data, cases)]
    dirties = [torch.from_numpy(d).cuda() for _, d in data]
    with cg.Batch(jobs) as b:
        for graphs in (True, False):
            b.graphs(graphs)
            b.run(dirties)
            for i, (n, tiles, K, niter, mode) in enumerate(cases):
                res, mod, comps = b.get(i)
                solo = gpu_clean(data[i][1], data[i][0], 0.1, niter, 0.0, tiles, K,
                                 feedback_mode=mode)
                assert len(comps) == solo["n"], (i, graphs)
                assert np.array_equal(comps["flux"].view(np.uint32),
                                      solo["comps"]["flux"].view(np.uint32)), (i, graphs)
                assert np.array_equal(res.cpu().numpy().view(np.uint32),
                                      solo["residual"].view(np.uint32)), (i, graphs)
                assert np.array_equal(mod.cpu().numpy().view(np.uint32),
                                      solo["model"].view(np.uint32)), (i, graphs)


def test_batch_with_flux_trigger_equals_oracle():
    import torch
    data = [_job(n, 1.0, 300 + n) for n in (96, 160)]
    jobs = [dict(psf=torch.from_numpy(p).cuda(), ny=p.shape[0] // 2, nx=p.shape[0] // 2,
                 gain=0.1, niter=500, threshold=0.0, tiles=(2, 2), feedback_interval=0,
                 feedback_trigger=0.5) for p, _ in data]
    with cg.Batch(jobs) as b:
        b.run([torch.from_numpy(d).cuda() for _, d in data])
        for i, (psf, dirty) in enumerate(data):
            o = oracle.clean_f32(dirty, psf, 0.1, 500, 0.0, (2, 2), 0, trigger=0.5)
            res, mod, comps = b.get(i)
            assert len(comps) == o.n
            assert np.array_equal(comps["flux"].view(np.uint32), o.comps["flux"].view(np.uint32))
            assert np.array_equal(res.cpu().numpy().view(np.uint32), o.residual.view(np.uint32))


def test_batch_streamed_pipeline_groups_equal_solo_runs():
    """Tiles too large for resident slabs run as 16 streaming CTAs of the
    batched TMA pipeline (2048^2 in one tile, 1536^2 in 1 x 2 tiles);
    every image still equals its solo run bit for bit."""
    import torch
    cases = [(2048, (1, 1), 0, 300), (1536, (1, 2), 25, 400), (256, (2, 2), 10, 300)]
    data = [_job(n, 1.0 + 0.2 * i, 300 + i) for i, (n, tiles, K, niter) in enumerate(cases)]
    jobs = [dict(psf=torch.from_numpy(p).cuda(), ny=n, nx=n, gain=0.1, niter=niter,
                 threshold=0.0, tiles=tiles, feedback_interval=K)
            for (p, _), (n, tiles, K, niter) in zip(data, cases)]
    dirties = [torch.from_numpy(d).cuda() for _, d in data]
    with cg.Batch(jobs) as b:
        b.run(dirties)
        for i, (n, tiles, K, niter) in enumerate(cases):
            res, mod, comps = b.get(i)
            solo = gpu_clean(data[i][1], data[i][0], 0.1, niter, 0.0, tiles, K)
            assert len(comps) == solo["n"] == niter
            assert np.array_equal(comps["flux"].view(np.uint32),
                                  solo["comps"]["flux"].view(np.uint32)), i
            assert np.array_equal(res.cpu().numpy().view(np.uint32),
                                  solo["residual"].view(np.uint32)), i


def test_batch_tile_pairs_with_idle_tiles_equal_oracle():
    """Persistent tile-pair units (512^2 in 2 x 2 tiles: two pairs of
    256-pixel-wide tiles) beside single-tile units, where every left tile
    stays under the threshold from the start: each image equals the oracle
    bit for bit."""
    import torch
    from gpu_helpers import one_sided_job
    cases = [(512, (2, 2), 20, 700, 0.01), (640, (2, 2), 0, 500, 0.01),
             (512, (1, 1), 15, 300, 0.0)]
    data = [one_sided_job(n, 10, 500 + i) for i, (n, *_rest) in enumerate(cases)]
    jobs = [dict(psf=torch.from_numpy(p).cuda(), ny=n, nx=n, gain=0.1, niter=niter,
                 threshold=thr, tiles=tiles, feedback_interval=K)
            for (p, _), (n, tiles, K, niter, thr) in zip(data, cases)]
    dirties = [torch.from_numpy(d).cuda() for _, d in data]
    with cg.Batch(jobs) as b:
        for rep in range(2):
            b.run(dirties)
            for i, (n, tiles, K, niter, thr) in enumerate(cases):
                res, mod, comps = b.get(i)
                o = oracle.clean_f32(data[i][1], data[i][0], 0.1, niter, thr, tiles, K)
                assert len(comps) == o.n, (i, rep)
                assert np.array_equal(comps["y"], o.comps["y"]), (i, rep)
                assert np.array_equal(comps["x"], o.comps["x"]), (i, rep)
                assert np.array_equal(comps["flux"].view(np.uint32),
                                      o.comps["flux"].view(np.uint32)), (i, rep)
                assert np.array_equal(res.cpu().numpy().view(np.uint32),
                                      o.residual.view(np.uint32)), (i, rep)
                assert np.array_equal(mod.cpu().numpy().view(np.uint32),
                                      o.model.view(np.uint32)), (i, rep)


def test_batch_non_square_tile_pairs_equal_solo_runs():
    """Non-square images whose tiles run as pairs in the persistent launch
    (a 1 x 2 grid of 500-pixel-wide tiles: ragged column halves; 2 x 2 of
    384 x 256 tiles; 3 x 2 of ragged 233/234-row tiles), beside a
    single-tile image: each equals its solo run bit for bit."""
    import torch
    cases = [(520, 1000, (1, 2), 13, 700), (512, 768, (2, 2), 25, 900),
             (700, 600, (3, 2), 12, 900), (300, 200, (1, 1), 20, 300)]
    data = []
    for i, (ny, nx, tiles, K, niter) in enumerate(cases):
        rng = np.random.default_rng(700 + i)
        psf = synth.make_psf(2 * ny, 2 * nx)
        n = min(ny, nx)
        ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
        d = synth.make_dirty(psf[ny - n:ny + n, nx - n:nx + n], n, ys, xs, fl, 1e-3, rng)
        dirty = synth.random_image(ny, nx, rng, 1e-3)
        dirty[:n, :n] += d
        data.append((psf, dirty))
    jobs = [dict(psf=torch.from_numpy(p).cuda(), ny=ny, nx=nx, gain=0.1, niter=niter,
                 threshold=0.0, tiles=tiles, feedback_interval=K)
            for (p, _), (ny, nx, tiles, K, niter) in zip(data, cases)]
    with cg.Batch(jobs) as b:
        b.run([torch.from_numpy(d).cuda() for _, d in data])
        for i, (ny, nx, tiles, K, niter) in enumerate(cases):
            res, mod, comps = b.get(i)
            solo = gpu_clean(data[i][1], data[i][0], 0.1, niter, 0.0, tiles, K)
            assert len(comps) == solo["n"] == niter, i
            assert np.array_equal(comps["flux"].view(np.uint32),
                                  solo["comps"]["flux"].view(np.uint32)), i
            assert np.array_equal(res.cpu().numpy().view(np.uint32),
                                  solo["residual"].view(np.uint32)), i
            assert np.array_equal(mod.cpu().numpy().view(np.uint32),
                                  solo["model"].view(np.uint32)), i
