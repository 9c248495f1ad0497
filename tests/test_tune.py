"""Autotuner: candidate generation and the cache on CPU; on the GPU, the
tuned plan reproduces the oracle bit for bit and a tuned interval K keeps
the restored image in the paper's band of the untiled run."""
import os
import tempfile

import numpy as np
import pytest

import paper_2501_01461_gb300 as cg
from paper_2501_01461_gb300 import tune


def test_candidates_cover_paths_and_barriers():
    c = tune.candidates((4, 4), 152)
    assert c[0] == tune.Choice()                      # the library's own choice first
    kinds = {(x.group_sync, x.minor_path, x.feedback_path, x.feedback_mode) for x in c}
    assert any(k[0] == cg.SYNC_GRID for k in kinds)
    assert any(k[0] == cg.SYNC_CLUSTER for k in kinds)
    assert 1 in {x.feedback_path for x in c}
    assert any(not x.minor_pairs for x in c) and any(not x.minor_tmem for x in c)
    assert all(x.feedback_mode == cg.FB_GATHER for x in c)   # exact unless FFT allowed
    assert any(x.feedback_mode == cg.FB_FFT for x in tune.candidates((4, 4), 152, allow_fft=True))
    assert len(c) == len({tuple(vars(x).items()) for x in c})
    # grid groups never exceed one CTA per SM per tile share
    assert all(x.group_ctas <= 152 // 16 for x in c if x.group_sync == cg.SYNC_GRID)
    # untiled: no FFT candidate even when allowed (nothing to feed back)
    assert not any(x.feedback_mode == cg.FB_FFT for x in tune.candidates((1, 1), 152, True))


def test_cache_roundtrip():
    key = tune.problem_key(1024, 1024, (2048, 2048), (2, 2), 50, 152)
    assert key == "1024x1024|psf2048x2048|t2x2|K50|sm152|fft0"
    r = tune.TuneResult(key=key, choice=tune.Choice(group_ctas=9, group_sync=cg.SYNC_GRID,
                                                    minor_path=2), K=50, ms_per_round=1.25,
                        trials=[{"choice": {}, "ms_per_round": 1.25}])
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sub", "tune.json")
        assert tune.load_cache(path) == {}
        tune.save_cache(path, {key: r.to_json()})
        back = tune.TuneResult.from_json(tune.load_cache(path)[key])
    assert back == r


@pytest.mark.gpu
def test_tuned_plan_is_bit_exact():
    import torch
    import oracle
    import synth
    from gpu_helpers import assert_bit_exact
    rng = np.random.default_rng(77)
    n = 256
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 15, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "t.json")
        res = tune.tune_launch(d_psf, d_dirty, 0.1, 2000, 0.0, (2, 2), 10, rounds=2,
                               cache_path=cache)
        assert res.ms_per_round > 0 and len(res.trials) >= 5
        again = tune.tune_launch(d_psf, d_dirty, 0.1, 2000, 0.0, (2, 2), 10, cache_path=cache)
        assert again.choice == res.choice            # served from the cache
    o = oracle.clean_f32(dirty, psf, 0.1, 2000, 0.0, (2, 2), 10)
    with tune.tuned_plan(res, d_psf, n, n, 0.1, 2000, 0.0, (2, 2)) as p:
        p.run(d_dirty)
        r, m, _ = p.get()
        comps = p.components_with_rounds()
        g = {"residual": r.cpu().numpy(), "model": m.cpu().numpy(), "comps": comps,
             "n": len(comps["y"])}
    assert_bit_exact(g, o, "tuned")


@pytest.mark.gpu
def test_tuned_interval_stays_in_paper_band():
    import torch
    import synth
    w = synth.workload("tiled-1024")
    data = w.build()
    beam = synth.fit_beam(data["psf"])
    d_psf, d_dirty = torch.from_numpy(data["psf"]).cuda(), torch.from_numpy(data["dirty"]).cuda()
    res = tune.tune(d_psf, d_dirty, w.gain, w.niter, data["threshold"], w.tiles, 50,
                    k_candidates=[10, 50, 200], beam=beam, rounds=2, use_cache=False)
    assert [t["K"] for t in res.k_trials] == [10, 50, 200]
    chosen = [t for t in res.k_trials if t["K"] == res.K]
    assert chosen and chosen[0]["in_band"]
    for t in res.k_trials:
        assert t["in_band"] == (tune.PAPER_BAND[0] <= t["min_diff"] and
                                t["max_diff"] <= tune.PAPER_BAND[1])
