"""Continuous batching: jobs that arrive while others run join at the next
step and run in the same launches; each job's result must be identical to
its solo run (clean_plan + clean_run), bit for bit, alone and in the mix."""
import numpy as np
import pytest

import paper_2501_01461_gb300 as cg
from paper_2501_01461_gb300 import serve
import synth
from gpu_helpers import gpu_clean

pytestmark = pytest.mark.gpu


def _data(n, seed, n_src=10):
    rng = np.random.default_rng(seed)
    psf = synth.make_psf(2 * n, 2 * n, freq_scale=1.0 + (seed % 7) / 7)
    ys, xs, fl = synth.make_sky(n, n_src, 0.05, 2.1, rng)
    return psf, synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)


def _same(result, solo):
    res, mod, comps = result
    assert len(comps) == solo["n"]
    assert np.array_equal(comps["flux"].view(np.uint32), solo["comps"]["flux"].view(np.uint32))
    assert np.array_equal(comps["y"], solo["comps"]["y"]) and np.array_equal(comps["x"], solo["comps"]["x"])
    assert np.array_equal(res.cpu().numpy().view(np.uint32), solo["residual"].view(np.uint32))
    assert np.array_equal(mod.cpu().numpy().view(np.uint32), solo["model"].view(np.uint32))


def test_jobs_joining_midway_equal_solo_runs():
    import torch
    specs = [(256, (2, 2), 20, 800), (512, (2, 2), 50, 1500), (128, (1, 1), 10, 300),
             (1024, (4, 4), 50, 2000), (200, (3, 3), 7, 600)]
    data = [_data(n, 40 + i) for i, (n, *_r) in enumerate(specs)]
    srv = serve.Server(max_jobs=8)
    jobs = {}
    try:
        # two jobs start; the others join one at a time while they run
        for i in range(len(specs)):
            n, tiles, K, niter = specs[i]
            psf, dirty = data[i]
            job = serve.Job(psf=torch.from_numpy(psf).cuda(), dirty=torch.from_numpy(dirty).cuda(),
                            niter=niter, tiles=tiles, feedback_interval=K)
            jobs[srv.add(job)] = (i, job)
            if i >= 1:
                srv.step(1)
        while srv.step(3) > 0:
            pass
        finished = srv.done()
        assert sorted(finished) == sorted(jobs)
        for jid in finished:
            i, job = jobs[jid]
            n, tiles, K, niter = specs[i]
            r = srv.get(jid, (n, n))
            _same(r, gpu_clean(data[i][1], data[i][0], 0.1, niter, 0.0, tiles, K))
            srv.remove(jid)
    finally:
        srv.close()


def test_serve_loop_results_and_latencies():
    import torch
    rng = np.random.default_rng(5)
    specs = []
    for k in range(10):
        n = int(rng.choice([128, 256, 512]))
        specs.append((n, (2, 2) if n > 128 else (1, 1), int(rng.integers(5, 40)),
                      int(rng.integers(200, 1200)), float(k) * 0.002))
    data = [_data(n, 70 + k) for k, (n, *_r) in enumerate(specs)]
    jobs = [serve.Job(psf=torch.from_numpy(p).cuda(), dirty=torch.from_numpy(d).cuda(), niter=nit,
                      tiles=t, feedback_interval=K, arrival=a)
            for (p, d), (n, t, K, nit, a) in zip(data, specs)]
    stats = serve.serve(jobs, budget_bytes=2e9, rounds_per_step=2)
    assert stats["jobs"] == 10 and stats["p99_s"] >= stats["p50_s"] > 0
    for (p, d), (n, t, K, nit, a), job in zip(data, specs, jobs):
        assert job.admitted >= a - 1e-9 and job.finished >= job.admitted
        _same(job.result, gpu_clean(d, p, 0.1, nit, 0.0, t, K))


def test_remove_running_job_and_memory_budget_admission():
    import torch
    psf, dirty = _data(256, 3)
    srv = serve.Server(max_jobs=2)
    try:
        job = serve.Job(psf=torch.from_numpy(psf).cuda(), dirty=torch.from_numpy(dirty).cuda(),
                        niter=5000, tiles=(2, 2), feedback_interval=10)
        a = srv.add(job)
        srv.step(1)
        srv.remove(a)                     # leaves mid-run
        b = srv.add(job)
        c = srv.add(job)
        with pytest.raises(cg.CleanError) as e:
            srv.add(job)                  # no free slot
        assert e.value.status == 3
        while srv.step(4) > 0:
            pass
        assert sorted(srv.done()) == sorted([b, c])
    finally:
        srv.close()
    # a budget smaller than two jobs admits them one after the other
    jobs = [serve.Job(psf=torch.from_numpy(psf).cuda(), dirty=torch.from_numpy(dirty).cuda(),
                      niter=400, tiles=(2, 2), feedback_interval=20, arrival=0.0) for _ in range(3)]
    serve.serve(jobs, budget_bytes=jobs[0].footprint() * 1.5, keep_results=False)
    order = sorted(jobs, key=lambda j: j.admitted)
    assert order[1].admitted >= order[0].finished - 1e-9


def test_served_fft_job_equals_solo_fft_run():
    """A job asking for FFT feedback, served beside gather jobs, equals its
    solo FFT run bit for bit."""
    import torch
    rng = np.random.default_rng(17)
    specs = [(256, (2, 2), 800, cg.FB_FFT, 0.0), (192, (2, 2), 500, cg.FB_GATHER, 0.002)]
    jobs = []
    for n, tiles, niter, mode, arrival in specs:
        psf = synth.make_psf(2 * n, 2 * n)
        ys, xs, fl = synth.make_sky(n, 10, 0.05, 2.1, rng)
        dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
        jobs.append(serve.Job(psf=torch.from_numpy(psf).cuda(), dirty=torch.from_numpy(dirty).cuda(),
                              niter=niter, tiles=tiles, feedback_interval=10, feedback_mode=mode,
                              arrival=arrival))
    serve.serve(jobs, budget_bytes=4e9)
    for j, (n, tiles, niter, mode, _) in zip(jobs, specs):
        res, mod, comps = j.result
        solo = gpu_clean(j.dirty.cpu().numpy(), j.psf.cpu().numpy(), 0.1, niter, 0.0, tiles, 10,
                         feedback_mode=mode)
        assert len(comps) == solo["n"]
        assert np.array_equal(res.cpu().numpy().view(np.uint32), solo["residual"].view(np.uint32))
        assert np.array_equal(comps["flux"].view(np.uint32), solo["comps"]["flux"].view(np.uint32))



def test_serving_stream_non_power_of_two_jobs_equal_solo_runs():
    """Jobs of the serving stream's kind (sides log-uniform, rounded to
    multiples of 64, so mostly not powers of two; each its own sky and dirty
    image; crops of one large PSF) served together in real time equal their
    solo runs bit for bit, and the one-at-a-time baseline server runs the
    same jobs in arrival order."""
    import torch
    psf_full = synth.make_psf(1024, 1024)
    specs = synth.serving_stream(psf_full, n_jobs=6, seed=77, lo=192, hi=512, step=64)
    sides = [sp["n"] for sp in specs]
    assert all(n % 64 == 0 and 192 <= n <= 512 for n in sides)
    assert any(n & (n - 1) for n in sides)             # a side that is not a power of two
    jobs = [serve.Job(psf=sp["psf"], dirty=sp["dirty"], niter=min(sp["niter"], 1500),
                      tiles=sp["tiles"], feedback_interval=sp["K"], arrival=0.003 * i)
            for i, sp in enumerate(specs)]
    serve.serve(jobs, budget_bytes=4e9)
    for j in jobs:
        _same(j.result, gpu_clean(j.dirty.cpu().numpy(), j.psf.cpu().numpy(), 0.1, j.niter, 0.0,
                                  j.tiles, j.feedback_interval))
    ran = []

    def run(job):
        with cg.Plan(job.psf, job.n, job.n, niter=job.niter, tiles=(1, 1)) as p:
            p.run(job.dirty)
            torch.cuda.synchronize()
        ran.append(job.arrival)
    st = serve.serve_one_at_a_time(jobs, run)
    assert ran == sorted(ran) and st["jobs"] == len(jobs)
    assert all(j.finished >= j.admitted >= j.arrival - 1e-9 for j in jobs)


def test_saturated_stream_of_tile_pair_jobs_equals_solo_runs():
    """Jobs whose tiles run as pairs in the persistent minor-loop launch
    (even tile counts, tiles at least 256 pixels wide), all arriving at once
    under a memory budget that admits a few at a time: the others join as
    jobs finish, so the pair units of new jobs run beside those of jobs in
    later rounds.  In one job the left tiles never have an iteration (their
    keys are 0 from the first step).  Each result equals its solo run bit
    for bit."""
    import torch
    from gpu_helpers import one_sided_job
    specs = [(576, (2, 2), 900, 0.0), (768, (2, 2), 1200, 0.0), (1088, (4, 4), 1600, 0.0),
             (640, (2, 2), 700, 0.0), (1024, (2, 2), 1000, 0.0), (1536, (4, 4), 1600, 0.0)]
    data = [_data(n, 300 + i, n_src=25) for i, (n, *_r) in enumerate(specs)]
    specs.append((512, (2, 2), 600, 0.01))
    data.append(one_sided_job(512, 10, 901))
    jobs = [serve.Job(psf=torch.from_numpy(p).cuda(), dirty=torch.from_numpy(d).cuda(), niter=nit,
                      threshold=thr, tiles=tiles, feedback_interval=50, arrival=0.0)
            for (p, d), (n, tiles, nit, thr) in zip(data, specs)]
    fp = sorted(j.footprint() for j in jobs)
    st = serve.serve(jobs, budget_bytes=1.1 * (fp[-1] + fp[-2]), rounds_per_step=2)
    assert st["jobs"] == len(jobs)
    assert max(j.admitted for j in jobs) >= min(j.finished for j in jobs)  # later jobs joined
    for j, (p, d), (n, tiles, nit, thr) in zip(jobs, data, specs):
        _same(j.result, gpu_clean(d, p, 0.1, nit, thr, tiles, 50))
