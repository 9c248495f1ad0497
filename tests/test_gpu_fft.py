"""FFT feedback (tolerance-exact alternative to the gather).

Section 3 defines the cross-coupling image as a tile's components placed on
a full-size image and convolved with the full PSF; the FFT path evaluates
that convolution with transforms and subtracts it, so it matches the float64
evaluation of the same component list to float32 transform accuracy, not
bit for bit.  Gates: the residual after every round within 1e-4 Jy of the
float64 replay of the GPU's own component list; model * PSF + residual =
dirty within 1e-4 Jy; and on the 1024^2 workload the restored image within
the paper's -0.1 .. +0.04 Jy band of the exact (gather) run.
"""
import numpy as np
import pytest

import oracle
import paper_2501_01461_gb300 as cg
import synth
from gpu_helpers import gpu_clean

pytestmark = pytest.mark.gpu

CASES = [
    # (ny, nx, psf, tiles, K, niter)
    (256, 256, (512, 512), (2, 2), 20, 1200),
    (200, 260, (400, 520), (3, 2), 15, 1500),    # non-square, ragged tiles
    (192, 192, (160, 200), (2, 3), 10, 600),     # PSF smaller than 2N: clipped kernel
    (195, 230, (390, 460), (3, 2), 12, 900),     # odd rows (a last half pair), nx not a multiple of 4
    (1024, 1024, (2048, 2048), (2, 2), 25, 1000),  # 2048-point radix-16 axes
]


def _sky(ny, nx, psf_shape, rng, n_src=12):
    psf = synth.make_psf(*psf_shape)
    n = min(ny, nx)
    ys, xs, fl = synth.make_sky(n, n_src, 0.05, 2.1, rng)
    d = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    dirty = synth.random_image(ny, nx, rng, 1e-3)
    dirty[:n, :n] += d
    return dirty, psf


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}-psf{c[2][0]}x{c[2][1]}-t{c[3][0]}x{c[3][1]}"
                                             for c in CASES])
def test_fft_rounds_match_float64_replay(case):
    ny, nx, ps, tiles, K, niter = case
    rng = np.random.default_rng(ny * 7 + nx)
    dirty, psf = _sky(ny, nx, ps, rng)
    for R in (1, 3, -1):
        g = gpu_clean(dirty, psf, 0.1, niter, 0.0, tiles, K, max_rounds=R,
                      feedback_mode=cg.FB_FFT)
        assert g["stats"]["feedback_mode"] == cg.FB_FFT
        rep = oracle.clean_f64(dirty, psf, 0.1, niter, 0.0, tiles, K, max_rounds=R,
                               replay=g["comps"])
        assert rep.n == g["n"]
        err_r = np.abs(g["residual"].astype(np.float64) - rep.residual).max()
        err_m = np.abs(g["model"].astype(np.float64) - rep.model).max()
        assert err_r <= 1e-4, (R, err_r)
        assert err_m <= 1e-4, (R, err_m)
    ident = oracle.psf_convolve(g["model"], psf) + g["residual"] - dirty
    assert np.abs(ident).max() <= 1e-4


def test_fft_with_tile_pairs_and_tmem():
    """FFT feedback behind the streamed minor loop with tile pairs and TMEM
    chunks: within 1e-4 Jy of the float64 replay after every round, and bit
    for bit the same as one group per tile (the minor loops agree exactly and
    the FFT path is deterministic)."""
    rng = np.random.default_rng(4242)
    dirty, psf = _sky(512, 512, (1024, 1024), rng, n_src=20)
    kw = dict(feedback_mode=cg.FB_FFT, group_ctas=2, group_sync=cg.SYNC_GRID, minor_path=2)
    for R in (1, 3, -1):
        g = gpu_clean(dirty, psf, 0.1, 1200, 0.0, (1, 2), 20, max_rounds=R, **kw)
        st = g["stats"]
        assert st["feedback_mode"] == cg.FB_FFT and st["minor_pairs"] == 1 and st["minor_tmem"] == 1
        rep = oracle.clean_f64(dirty, psf, 0.1, 1200, 0.0, (1, 2), 20, max_rounds=R,
                               replay=g["comps"])
        assert rep.n == g["n"]
        assert np.abs(g["residual"].astype(np.float64) - rep.residual).max() <= 1e-4, R
        assert np.abs(g["model"].astype(np.float64) - rep.model).max() <= 1e-4, R
    single = gpu_clean(dirty, psf, 0.1, 1200, 0.0, (1, 2), 20, minor_pair=0, **kw)
    assert single["stats"]["minor_pairs"] == 0
    assert np.array_equal(single["residual"].view(np.uint32), g["residual"].view(np.uint32))
    assert np.array_equal(single["model"].view(np.uint32), g["model"].view(np.uint32))
    for k in ("y", "x", "tile", "round"):
        assert np.array_equal(single["comps"][k], g["comps"][k])


@pytest.mark.slow
def test_fft_paper_band_1024():
    """1024^2, 2 x 2 tiles, K = 50, threshold 5 mJy: FFT feedback vs the exact
    gather, restored images within the paper's band; both vs untiled too."""
    import torch
    w = synth.workload("tiled-1024").build()
    psf, dirty = w["psf"], w["dirty"]
    beam = synth.fit_beam(psf)
    exact = gpu_clean(dirty, psf, 0.1, 10000, 5e-3, (2, 2), 50)
    fft = gpu_clean(dirty, psf, 0.1, 10000, 5e-3, (2, 2), 50, feedback_mode=cg.FB_FFT)
    std = gpu_clean(dirty, psf, 0.1, 10000, 5e-3, mode=cg.UNTILED_GRID)
    r_exact = oracle.restore(exact["model"], exact["residual"], *beam)
    r_fft = oracle.restore(fft["model"], fft["residual"], *beam)
    r_std = oracle.restore(std["model"], std["residual"], *beam)
    for a, b in ((r_fft, r_exact), (r_fft, r_std)):
        diff = a - b
        assert diff.min() >= -0.1 and diff.max() <= 0.04
    rep = oracle.clean_f64(dirty, psf, 0.1, 10000, 5e-3, (2, 2), 50, replay=fft["comps"])
    assert np.abs(fft["residual"] - rep.residual).max() <= 1e-4


def test_auto_picks_fft_for_large_rounds_and_gather_for_small():
    import torch
    psf = torch.from_numpy(synth.make_psf(1024, 1024)).cuda()
    with cg.Plan(psf, 512, 512, niter=20000, tiles=(4, 4), feedback_interval=500,
                 feedback_mode=cg.FB_AUTO) as p:
        assert p.stats()["feedback_mode"] == cg.FB_FFT
    with cg.Plan(psf, 128, 128, niter=2000, tiles=(2, 2), feedback_interval=1,
                 feedback_mode=cg.FB_AUTO) as p:
        assert p.stats()["feedback_mode"] == cg.FB_GATHER


def test_force_feedback_environment(monkeypatch):
    """CLEANGB_FORCE_FEEDBACK overrides a plan's feedback mode."""
    import torch
    psf = torch.zeros((256, 256), dtype=torch.float32, device="cuda")
    psf[128, 128] = 1.0
    for env, want in (("fft", cg.FB_FFT), ("gather", cg.FB_GATHER)):
        monkeypatch.setenv("CLEANGB_FORCE_FEEDBACK", env)
        mode = cg.FB_GATHER if env == "fft" else cg.FB_FFT
        with cg.Plan(psf, 128, 128, gain=0.1, niter=100, tiles=(2, 2), feedback_interval=5,
                     feedback_mode=mode) as p:
            assert p.stats()["feedback_mode"] == want
