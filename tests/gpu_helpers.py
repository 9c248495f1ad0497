"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
compare it with the CPU oracle on the same seeded inputs."""
import numpy as np

import oracle
import paper_2501_01461_gb300 as cg


def gpu_clean(dirty, psf, gain, niter, threshold=0.0, tiles=(1, 1), K=0, max_rounds=-1,
              mode=cg.TILED, group_ctas=0, group_sync=cg.SYNC_AUTO, feedback_path=0, minor_path=0,
              feedback_mode=cg.FB_GATHER, trigger=0.0, minor_tmem=None, minor_pair=None):
    import torch
    d_psf = torch.from_numpy(np.ascontiguousarray(psf, np.float32)).cuda()
    d_dirty = torch.from_numpy(np.ascontiguousarray(dirty, np.float32)).cuda()
    ny, nx = dirty.shape
    with cg.Plan(d_psf, ny, nx, gain=gain, niter=niter, threshold=threshold, tiles=tiles,
                 feedback_interval=K, mode=mode, group_ctas=group_ctas,
                 group_sync=group_sync, feedback_mode=feedback_mode,
                 feedback_trigger=trigger) as plan:
        if feedback_path:
            plan.debug_set(cg.DEBUG_FEEDBACK_PATH, feedback_path)
        if minor_path:
            plan.debug_set(cg.DEBUG_MINOR_PATH, minor_path)
        if minor_tmem is not None:
            plan.debug_set(cg.DEBUG_MINOR_TMEM, int(minor_tmem))
        if minor_pair is not None:
            plan.debug_set(cg.DEBUG_MINOR_PAIR, int(minor_pair))
        plan.run(d_dirty, max_rounds=max_rounds)
        res, mod, _ = plan.get()
        comps = plan.components_with_rounds()
        stats = plan.stats()
        torch.cuda.synchronize()
        return dict(residual=res.cpu().numpy(), model=mod.cpu().numpy(), comps=comps,
                    n=len(comps["y"]), stats=stats)


def assert_bit_exact(g, o, what=""):
    """GPU run g equals oracle run o: component list, residual, model."""
    assert g["n"] == o.n, f"{what}: {g['n']} vs {o.n} components"
    for key in ("y", "x", "tile", "round"):
        if not np.array_equal(g["comps"][key], o.comps[key]):
            i = int(np.flatnonzero(g["comps"][key] != o.comps[key])[0])
            raise AssertionError(f"{what}: component {key} differs first at {i}")
    gf, of = g["comps"]["flux"].view(np.uint32), o.comps["flux"].view(np.uint32)
    assert np.array_equal(gf, of), f"{what}: flux bits differ at {np.flatnonzero(gf != of)[:5]}"
    dr = g["residual"].view(np.uint32) != o.residual.view(np.uint32)
    assert not dr.any(), f"{what}: residual differs at {np.argwhere(dr)[:5].tolist()}"
    dm = g["model"].view(np.uint32) != o.model.view(np.uint32)
    assert not dm.any(), f"{what}: model differs at {np.argwhere(dm)[:5].tolist()}"


def one_sided_job(n, n_sources, seed):
    """An n x n dirty image whose sources all sit in the right half, over a
    narrow Gaussian PSF (2n x 2n, sigma 1.5 pixels, peak 1 at the centre) and
    noise of 1 mJy: with a threshold of 10 mJy no left-half tile ever has an
    iteration, so its key is 0 from the first step while its right-hand
    neighbour runs."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[-n:n, -n:n].astype(np.float64)
    psf = np.exp(-(yy * yy + xx * xx) / (2 * 1.5 ** 2)).astype(np.float32)
    ys = rng.integers(8, n - 8, size=n_sources)
    xs = rng.choice(np.arange(n // 2 + 8, n - 8), size=n_sources, replace=False)
    fl = np.exp(rng.uniform(np.log(0.05), np.log(2.1), size=n_sources))
    import synth
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    return psf, dirty
