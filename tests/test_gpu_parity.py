"""Parity of the CUDA path with the CPU oracle (bit-exact in float32: the
component list, the residual and the model image), element by element on
seeded inputs.  Every call goes through the C ABI of libcleangb.so.

Sizes span several tiles and CTA slabs and include ragged tiles (sizes not
divisible by the grid), clipped PSFs, tie-heavy integer images, thresholds,
every feedback interval kind (none, 1, small, larger than the budget), both
group barriers (cluster, grid) and both residual placements (shared memory,
global memory).
"""
import numpy as np
import pytest

import oracle
import paper_2501_01461_gb300 as cg
import synth
from gpu_helpers import assert_bit_exact, gpu_clean

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cg.build()
    cg.lib()


SMALL = [
    # (ny, nx, psf, tiles, K, niter, threshold, kind)
    (16, 16, (32, 32), (1, 1), 0, 40, 0.0, "rand"),
    (16, 16, (32, 32), (2, 2), 1, 60, 0.0, "tie"),
    (16, 16, (32, 32), (4, 4), 3, 90, 0.05, "rand"),
    (33, 47, (66, 94), (3, 2), 7, 200, 0.0, "rand"),
    (64, 64, (128, 128), (2, 2), 50, 400, 0.0, "sky"),
    (64, 64, (40, 50), (2, 3), 5, 300, 0.0, "rand"),     # clipped PSF
    (250, 250, (500, 500), (4, 4), 10, 800, 0.0, "sky"),  # ragged 62/63-pixel tiles
    (250, 250, (500, 500), (4, 4), 0, 800, 1e-3, "sky"),  # independent tiles
    (128, 96, (256, 192), (1, 1), 20, 300, 0.0, "sky"),   # 1x1 grid with rounds
    (96, 128, (192, 256), (3, 5), 1000, 900, 0.0, "tie"), # K larger than the budget
]


def _inputs(ny, nx, psf_shape, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "sky":
        psf = synth.make_psf(*psf_shape)
        ys, xs, fl = synth.make_sky(min(ny, nx), 8, 0.05, 2.1, rng)
        d = synth.make_dirty(psf, min(ny, nx), ys, xs, fl, 1e-3, rng)
        dirty = np.zeros((ny, nx), np.float32)
        dirty[:d.shape[0], :d.shape[1]] = d
        dirty += synth.random_image(ny, nx, rng, 1e-3)
        return dirty, psf
    psf = synth.random_psf(*psf_shape, rng)
    img = synth.tie_image(ny, nx, rng) if kind == "tie" else synth.random_image(ny, nx, rng)
    return img, psf


@pytest.mark.parametrize("case", SMALL, ids=[f"{c[0]}x{c[1]}-t{c[3][0]}x{c[3][1]}-K{c[4]}-{c[7]}"
                                             for c in SMALL])
@pytest.mark.parametrize("sync", [cg.SYNC_CLUSTER, cg.SYNC_GRID])
def test_small_bit_exact(case, sync):
    ny, nx, ps, tiles, K, niter, thr, kind = case
    dirty, psf = _inputs(ny, nx, ps, kind, seed=hash(case) % 2 ** 31)
    o = oracle.clean_f32(dirty, psf, 0.2, niter, thr, tiles, K)
    g = gpu_clean(dirty, psf, 0.2, niter, thr, tiles, K, group_sync=sync)
    assert_bit_exact(g, o, str(case))


@pytest.mark.parametrize("G", [1, 2, 3, 8, 16])
def test_group_sizes_cluster(G):
    """Every cluster size splits the tile rows differently; results agree."""
    dirty, psf = _inputs(120, 100, (240, 200), "sky", 5)
    o = oracle.clean_f32(dirty, psf, 0.1, 600, 0.0, (2, 2), 9)
    g = gpu_clean(dirty, psf, 0.1, 600, 0.0, (2, 2), 9, group_ctas=G,
                  group_sync=cg.SYNC_CLUSTER)
    assert g["stats"]["group_ctas"] == G
    assert_bit_exact(g, o, f"G={G}")


@pytest.mark.parametrize("G", [1, 5, 37])
def test_group_sizes_grid(G):
    dirty, psf = _inputs(120, 100, (240, 200), "sky", 6)
    o = oracle.clean_f32(dirty, psf, 0.1, 600, 0.0, (2, 2), 9)
    g = gpu_clean(dirty, psf, 0.1, 600, 0.0, (2, 2), 9, group_ctas=G, group_sync=cg.SYNC_GRID)
    assert g["stats"]["group_ctas"] == G and g["stats"]["group_sync"] == cg.SYNC_GRID
    assert_bit_exact(g, o, f"G={G}")


@pytest.mark.parametrize("sync", [cg.SYNC_CLUSTER, cg.SYNC_GRID])
@pytest.mark.parametrize("minor_path", [1, 2])
def test_streamed_residual(sync, minor_path):
    """Tiles whose CTA slabs exceed shared memory keep the residual in global
    memory for the round (plain loads, and the bulk-copy pipeline)."""
    dirty, psf = _inputs(512, 512, (1024, 1024), "sky", 7)
    o = oracle.clean_f32(dirty, psf, 0.1, 300, 0.0, (1, 2), 25)
    g = gpu_clean(dirty, psf, 0.1, 300, 0.0, (1, 2), 25, group_ctas=1, group_sync=sync,
                  minor_path=minor_path)
    assert g["stats"]["resident"] == 0
    assert g["stats"]["minor_pipe"] == (1 if minor_path == 2 else 0)
    assert_bit_exact(g, o, "streamed")


MINOR_CASES = [
    # (ny, nx, psf, tiles, K, niter, G, sync): resident and streamed slabs,
    # ragged tiles, clipped PSFs, every group barrier
    (128, 128, (256, 256), (2, 2), 7, 500, 4, cg.SYNC_CLUSTER),
    (200, 240, (400, 480), (3, 4), 11, 900, 3, cg.SYNC_GRID),
    (96, 160, (64, 80), (2, 2), 5, 400, 2, cg.SYNC_CLUSTER),     # clipped PSF rows/columns
    (1024, 1024, (2048, 2048), (2, 2), 20, 600, 1, cg.SYNC_CLUSTER),  # streamed slabs
    (300, 600, (600, 1200), (1, 1), 0, 500, 16, cg.SYNC_GRID),   # untiled-style group
    (96, 96, (192, 192), (3, 3), 6, 500, 2, cg.SYNC_GRID),       # 32-pixel-wide tiles
    (90, 152, (180, 304), (2, 3), 4, 400, 2, cg.SYNC_CLUSTER),   # 50-51 wide: per-pixel path
    (520, 1000, (1040, 2000), (1, 2), 13, 400, 3, cg.SYNC_GRID), # ragged 128-column chunks
]


@pytest.mark.parametrize("case", MINOR_CASES, ids=[f"{c[0]}x{c[1]}-t{c[3][0]}x{c[3][1]}-G{c[6]}-s{c[7]}"
                                                   for c in MINOR_CASES])
def test_minor_paths_bit_exact(case):
    """Plain-load and bulk-copy-pipeline minor loops give the oracle's bits."""
    ny, nx, ps, tiles, K, niter, G, sync = case
    rng = np.random.default_rng(ny + nx)
    psf = synth.make_psf(*ps) if ps[0] >= 2 * ny else synth.random_psf(*ps, rng)
    if ps[0] >= 2 * ny:
        ys, xs, fl = synth.make_sky(min(ny, nx), 10, 0.05, 2.1, rng)
        d = synth.make_dirty(psf, min(ny, nx), ys, xs, fl, 1e-3, rng)
        dirty = synth.random_image(ny, nx, rng, 1e-3)
        dirty[:d.shape[0], :d.shape[1]] += d
    else:
        dirty = synth.random_image(ny, nx, rng)
    o = oracle.clean_f32(dirty, psf, 0.1, niter, 0.0, tiles, K)
    for path in (1, 2):
        g = gpu_clean(dirty, psf, 0.1, niter, 0.0, tiles, K, group_ctas=G, group_sync=sync,
                      minor_path=path)
        assert g["stats"]["minor_pipe"] == (1 if path == 2 else 0)
        assert_bit_exact(g, o, f"{case} path={path}")


TMEM_CASES = [
    # (ny, nx, psf, tiles, K, niter, G, threshold, expect_flag): streamed
    # pipeline slabs whose leading full 128 x 60 chunks live in tensor memory
    (512, 512, (1024, 1024), (1, 1), 0, 400, 2, 0.0, 1),     # 8 TMEM chunks a CTA
    (512, 512, (900, 1024), (1, 1), 0, 400, 4, 0.0, 0),      # only the middle CTAs qualify
    (512, 600, (1024, 1200), (1, 1), 0, 300, 2, 0.0, 1),     # ragged 88-column chunk ends the run
    (1024, 1024, (2048, 2048), (2, 2), 20, 600, 2, 0.0, 1),  # feedback between launches
    (512, 512, (1024, 1024), (1, 2), 1, 120, 1, 0.0, 1),     # one iteration a launch
    (512, 512, (1024, 1024), (1, 1), 0, 4000, 2, 0.05, 1),   # threshold stops mid-launch
]


@pytest.mark.parametrize("case", TMEM_CASES, ids=[f"{c[0]}x{c[1]}-psf{c[2][0]}x{c[2][1]}-t{c[3][0]}x{c[3][1]}-K{c[4]}-G{c[6]}"
                                                  for c in TMEM_CASES])
def test_minor_tmem_bit_exact(case):
    """The pipeline with each CTA's leading chunks in tensor memory gives the
    oracle's bits, as does the same pipeline streaming every chunk; CTAs whose
    windows can leave the PSF array stream all their chunks."""
    ny, nx, ps, tiles, K, niter, G, thr, flag = case
    rng = np.random.default_rng(ny * 7 + nx + G)
    if ps[0] >= 2 * ny and ps[1] >= 2 * nx:
        psf = synth.make_psf(*ps)
        ys, xs, fl = synth.make_sky(min(ny, nx), 12, 0.05, 2.1, rng)
        d = synth.make_dirty(psf, min(ny, nx), ys, xs, fl, 1e-3, rng)
        dirty = synth.random_image(ny, nx, rng, 1e-3)
        dirty[:d.shape[0], :d.shape[1]] += d
    else:
        psf = synth.random_psf(*ps, rng)
        dirty = synth.random_image(ny, nx, rng)
    o = oracle.clean_f32(dirty, psf, 0.1, niter, thr, tiles, K)
    for tm in (1, 0):
        g = gpu_clean(dirty, psf, 0.1, niter, thr, tiles, K, group_ctas=G,
                      group_sync=cg.SYNC_GRID, minor_path=2, minor_tmem=tm)
        st = g["stats"]
        assert st["minor_pipe"] == 1 and st["resident"] == 0
        assert st["minor_tmem"] == (flag if tm else 0), st
        assert_bit_exact(g, o, f"{case} tmem={tm}")
    if thr > 0:
        assert o.n < niter  # the threshold, not the budget, ended the run


PAIR_CASES = [
    # (ny, nx, psf, tiles, K, niter, G, threshold, pairs): tile pairs served
    # by groups of 2G CTAs (streamed rows, grid groups, an even tile count)
    (512, 512, (1024, 1024), (1, 2), 0, 400, 2, 0.0, 1),      # one pair, TMEM chunks
    (1024, 1024, (2048, 2048), (2, 2), 20, 600, 2, 0.0, 1),   # two pairs, feedback
    (520, 1000, (1040, 2000), (1, 2), 13, 401, 3, 0.0, 1),    # ragged halves, odd budget
    (512, 512, (600, 700), (2, 2), 10, 600, 1, 0.0, 1),       # clipped windows: scalar path
    (512, 512, (1024, 1024), (1, 2), 1, 120, 2, 0.0, 1),      # one iteration a launch
    (512, 512, (1024, 1024), (2, 2), 0, 4000, 1, 0.05, 1),    # tiles stop at different times
    (768, 512, (1536, 1024), (3, 1), 10, 300, 2, 0.0, 0),     # odd tile count: one group a tile
    (1024, 512, (2048, 1024), (2, 1), 15, 500, 2, 0.0, 1),    # a vertical pair
    (700, 600, (1400, 1200), (3, 2), 12, 900, 1, 0.0, 1),     # three pairs, ragged heights
]


@pytest.mark.parametrize("case", PAIR_CASES, ids=[f"{c[0]}x{c[1]}-psf{c[2][0]}x{c[2][1]}-t{c[3][0]}x{c[3][1]}-K{c[4]}-G{c[6]}"
                                                  for c in PAIR_CASES])
def test_minor_tile_pairs_bit_exact(case):
    """Groups of 2G CTAs alternating between two tiles give the oracle's
    bits, as does one group per tile."""
    ny, nx, ps, tiles, K, niter, G, thr, pairs = case
    rng = np.random.default_rng(ny * 3 + nx + G + K)
    if ps[0] >= 2 * ny and ps[1] >= 2 * nx:
        psf = synth.make_psf(*ps)
        ys, xs, fl = synth.make_sky(min(ny, nx), 12, 0.05, 2.1, rng)
        d = synth.make_dirty(psf, min(ny, nx), ys, xs, fl, 1e-3, rng)
        dirty = synth.random_image(ny, nx, rng, 1e-3)
        dirty[:d.shape[0], :d.shape[1]] += d
    else:
        psf = synth.random_psf(*ps, rng)
        dirty = synth.random_image(ny, nx, rng)
    o = oracle.clean_f32(dirty, psf, 0.1, niter, thr, tiles, K)
    for pr in (1, 0):
        g = gpu_clean(dirty, psf, 0.1, niter, thr, tiles, K, group_ctas=G,
                      group_sync=cg.SYNC_GRID, minor_path=2, minor_pair=pr)
        st = g["stats"]
        assert st["minor_pipe"] == 1 and st["resident"] == 0
        assert st["minor_pairs"] == (pairs if pr else 0), st
        assert_bit_exact(g, o, f"{case} pairs={pr}")


def test_tile_pairs_with_an_idle_tile_bit_exact():
    """Tile pairs whose left tile never has an iteration: its key is 0 from
    the first step, so the producer posts two keys before the consumers wait
    for the first (one key barrier per buffer keeps the waits exact)."""
    from gpu_helpers import one_sided_job
    psf, dirty = one_sided_job(512, 12, 77)
    # (tiles, K, G): G row bands a tile, streamed (a 256-wide slab of 256
    # rows does not fit in shared memory beside the ring)
    for tiles, K, G in (((1, 2), 10, 2), ((2, 2), 0, 1), ((2, 2), 25, 1)):
        o = oracle.clean_f32(dirty, psf, 0.1, 800, 0.01, tiles, K)
        assert 0 < o.n < 800 and set(o.comps["tile"].tolist()) <= {1, 3}
        g = gpu_clean(dirty, psf, 0.1, 800, 0.01, tiles, K, group_ctas=G,
                      group_sync=cg.SYNC_GRID, minor_path=2, minor_pair=1)
        assert g["stats"]["minor_pairs"] == 1 and g["stats"]["resident"] == 0, (tiles, g["stats"])
        assert_bit_exact(g, o, f"idle left tiles {tiles} K {K}")


def test_tile_pairs_with_ties_everywhere_bit_exact():
    """A delta PSF over an integer-valued image: each iteration changes only
    the peak pixel, so every later peak is a tie among thousands of pixels of
    |R| = 3 spread over chunks, lanes, warps and CTAs, and must still be the
    lowest index (the pair body's per-chunk tracking reads the tied chunks
    back)."""
    rng = np.random.default_rng(2024)
    for (ny, nx), tiles, K, G in (((512, 512), (1, 2), 10, 2), ((512, 512), (2, 2), 0, 1),
                                  ((520, 1000), (1, 2), 13, 3)):
        psf = np.zeros((2 * ny, 2 * nx), np.float32)
        psf[ny, nx] = 1.0
        dirty = synth.tie_image(ny, nx, rng)
        o = oracle.clean_f32(dirty, psf, 0.1, 400, 0.0, tiles, K)
        assert o.n == 400
        g = gpu_clean(dirty, psf, 0.1, 400, 0.0, tiles, K, group_ctas=G,
                      group_sync=cg.SYNC_GRID, minor_path=2, minor_pair=1)
        assert g["stats"]["minor_pairs"] == 1 and g["stats"]["resident"] == 0, g["stats"]
        assert_bit_exact(g, o, f"ties {ny}x{nx} {tiles} K {K}")


def test_untiled_grid_256():
    """Plain Hogbom CLEAN on the whole GPU: 256^2 image, 512^2 PSF, 20
    sources, gain 0.1, 2000 iterations, threshold 5 mJy."""
    w = synth.workload("untiled-256").build()
    o = oracle.clean_f32(w["dirty"], w["psf"], 0.1, 2000, 5e-3)
    g = gpu_clean(w["dirty"], w["psf"], 0.1, 2000, 5e-3, mode=cg.UNTILED_GRID)
    assert g["stats"]["group_sync"] == cg.SYNC_GRID
    assert_bit_exact(g, o, "untiled-256")


def test_automatic_group_choice():
    """One tile of up to 2^17 pixels runs as a 16-CTA cluster, larger tiles
    on a grid group of about one CTA per 8192 pixels (at most all SMs); the
    256^2 workload still matches the oracle bit for bit."""
    w = synth.workload("untiled-256").build()
    o = oracle.clean_f32(w["dirty"], w["psf"], 0.1, 2000, 5e-3)
    g = gpu_clean(w["dirty"], w["psf"], 0.1, 2000, 5e-3)
    assert g["stats"]["group_sync"] == cg.SYNC_CLUSTER and g["stats"]["group_ctas"] == 16
    assert_bit_exact(g, o, "untiled-256 auto")
    import torch
    for n, want in ((512, 32), (1024, 128)):
        psf = torch.zeros((2 * n, 2 * n), dtype=torch.float32, device="cuda")
        psf[n, n] = 1.0
        with cg.Plan(psf, n, n, gain=0.1, niter=10) as p:
            st = p.stats()
        sms = st["sm_count"]
        assert st["group_sync"] == cg.SYNC_GRID and st["group_ctas"] == min(want, sms), (n, st)


@pytest.mark.slow
@pytest.mark.parametrize("thr", [0.0, 5e-3])
def test_tiled_1024(thr, record_property):
    """1024^2 image, 2048^2 PSF, 2x2 tiles, K = 50, 10000 iterations: the
    float32 lists and images are identical; the model is within 1e-4 Jy of
    the float64 replay of the same list at every pixel.  The independent
    float64 run (its own trajectory) is reported, not gated: where its list
    first departs from the float32 one and the largest model difference."""
    w = synth.workload("tiled-1024").build()
    o = oracle.clean_f32(w["dirty"], w["psf"], 0.1, 10000, thr, (2, 2), 50)
    g = gpu_clean(w["dirty"], w["psf"], 0.1, 10000, thr, (2, 2), 50)
    assert_bit_exact(g, o, f"tiled-1024 thr={thr}")
    rep = oracle.clean_f64(w["dirty"], w["psf"], 0.1, 10000, thr, (2, 2), 50, replay=g["comps"])
    assert np.abs(g["model"].astype(np.float64) - rep.model).max() <= 1e-4
    if thr > 0:
        ind = oracle.clean_f64(w["dirty"], w["psf"], 0.1, 10000, thr, (2, 2), 50)
        m = min(ind.n, g["n"])
        same = (ind.comps["y"][:m] == g["comps"]["y"][:m]) & (ind.comps["x"][:m] == g["comps"]["x"][:m])
        first = int(np.flatnonzero(~same)[0]) if not same.all() else m
        diff = float(np.abs(g["model"].astype(np.float64) - ind.model).max())
        record_property("fp64_independent_first_divergence", first)
        record_property("fp64_independent_max_model_diff_jy", diff)
        print(f"independent float64 run: lists agree for the first {first} of {m} components; "
              f"max model difference {diff:.3g} Jy")


def test_resume_and_step_equal_single_run():
    """run(D, 3 rounds) + run(continue) == run(D); step/feedback == run."""
    import torch
    dirty, psf = _inputs(96, 96, (192, 192), "sky", 8)
    full = gpu_clean(dirty, psf, 0.1, 400, 0.0, (2, 2), 10)
    d_psf = torch.from_numpy(psf).cuda()
    d_dirty = torch.from_numpy(dirty).cuda()
    with cg.Plan(d_psf, 96, 96, gain=0.1, niter=400, tiles=(2, 2), feedback_interval=10) as p:
        p.run(d_dirty, max_rounds=3)
        assert p.n_components() == 3 * 4 * 10
        p.run(None)
        r, m, _ = p.get()
        assert np.array_equal(r.cpu().numpy(), full["residual"])
        assert np.array_equal(m.cpu().numpy(), full["model"])
        # the same rounds driven one step at a time
        p.run(d_dirty, max_rounds=0)
        for _ in range(10):
            p.step()
            p.feedback()
        p.feedback()  # nothing pending: no-op
        r2, m2, _ = p.get()
        assert np.array_equal(r2.cpu().numpy(), full["residual"])
        assert p.n_components() == 400


def test_truncated_rounds_match_oracle():
    dirty, psf = _inputs(200, 200, (400, 400), "sky", 9)
    for R in (1, 2, 5):
        o = oracle.clean_f32(dirty, psf, 0.1, 2000, 0.0, (3, 3), 7, max_rounds=R)
        g = gpu_clean(dirty, psf, 0.1, 2000, 0.0, (3, 3), 7, max_rounds=R)
        assert_bit_exact(g, o, f"rounds={R}")


def test_host_buffers_match_device_path():
    dirty, psf = _inputs(128, 128, (256, 256), "sky", 10)
    dev = gpu_clean(dirty, psf, 0.1, 500, 0.0, (2, 2), 20)
    with cg.Plan(None, 128, 128, gain=0.1, niter=500, tiles=(2, 2), feedback_interval=20,
                 psf_shape=psf.shape) as p:
        res = np.empty_like(dirty)
        mod = np.empty_like(dirty)
        comps = np.empty(500, dtype=cg.COMPONENT_DTYPE)
        for _ in range(2):
            n = p.deconvolve_host(dirty, psf, res, mod, comps)
            assert n == 500
            assert np.array_equal(res, dev["residual"]) and np.array_equal(mod, dev["model"])
            assert np.array_equal(comps["flux"], dev["comps"]["flux"])


def test_empty_budget_and_zero_image():
    dirty, psf = _inputs(32, 32, (64, 64), "rand", 11)
    g = gpu_clean(dirty, psf, 0.1, 0, 0.0, (2, 2), 3)
    assert g["n"] == 0 and np.array_equal(g["residual"], dirty)
    z = np.zeros((32, 32), np.float32)
    g = gpu_clean(z, psf, 0.1, 100, 0.0, (2, 2), 3)
    assert g["n"] == 0 and not g["model"].any()


def test_restore_matches_oracle():
    import torch
    w = synth.workload("untiled-256").build()
    psf, dirty = w["psf"], w["dirty"]
    bmaj, bmin, bpa = (float(np.float32(v)) for v in synth.fit_beam(psf))
    bpa = float(np.float32(0.3))
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    with cg.Plan(d_psf, 256, 256, gain=0.1, niter=2000, threshold=5e-3, tiles=(2, 2),
                 feedback_interval=30) as p:
        p.run(d_dirty)
        out = p.restore(bmaj, bmin * 0.8, bpa).cpu().numpy()
        r, m, _ = p.get()
        want = oracle.restore(m.cpu().numpy(), r.cpu().numpy(), bmaj, bmin * 0.8, bpa)
        assert np.abs(out - want).max() <= 1e-5 * max(1.0, np.abs(want).max())


FB_CASES = [
    # (ny, nx, psf, tiles, K, niter)
    (250, 250, (500, 500), (4, 4), 10, 800),    # ragged tiles, full PSF
    (200, 300, (150, 180), (3, 2), 6, 400),     # PSF smaller than the image: clipped windows
    (256, 256, (512, 512), (2, 2), 300, 1200),  # more components than one staged chunk
    (300, 260, (600, 520), (5, 3), 40, 3000),
    (256, 256, (512, 512), (3, 3), 200, 3600),  # more than 1024 components a round
    (512, 1000, (1024, 2000), (2, 2), 25, 1200),  # ragged 500-wide tiles: 4 blocks, the last 116
    (512, 512, (600, 700), (2, 2), 10, 600),      # 256-wide tiles, clipped windows
]


@pytest.mark.parametrize("case", FB_CASES, ids=[f"{c[0]}x{c[1]}-psf{c[2][0]}x{c[2][1]}-t{c[3][0]}x{c[3][1]}-K{c[4]}"
                                                for c in FB_CASES])
def test_feedback_paths_bit_exact(case):
    """Plain-load and TMA feedback kernels give the oracle's bits."""
    ny, nx, ps, tiles, K, niter = case
    rng = np.random.default_rng(sum(case[:2]))
    psf = synth.make_psf(*ps) if ps[0] >= 2 * ny else synth.random_psf(*ps, rng)
    dirty = synth.random_image(ny, nx, rng)
    o = oracle.clean_f32(dirty, psf, 0.1, niter, 0.0, tiles, K)
    for path in (1, 2):
        g = gpu_clean(dirty, psf, 0.1, niter, 0.0, tiles, K, feedback_path=path)
        assert g["stats"]["feedback_tma"] == (1 if path == 2 else 0)
        assert_bit_exact(g, o, f"{case} path={path}")


def test_psf_narrower_than_tma_box_uses_plain_loads():
    """A PSF narrower than the TMA window box (132 floats) cannot be tiled by
    the tensor map: the plan falls back to plain loads, with the oracle's
    bits, even when the TMA kernel is requested."""
    rng = np.random.default_rng(330)
    psf = synth.random_psf(100, 120, rng)
    dirty = synth.random_image(130, 200, rng)
    o = oracle.clean_f32(dirty, psf, 0.1, 400, 0.0, (3, 2), 6)
    for path in (0, 2):
        g = gpu_clean(dirty, psf, 0.1, 400, 0.0, (3, 2), 6, feedback_path=path)
        assert g["stats"]["feedback_tma"] == 0
        assert_bit_exact(g, o, f"narrow PSF path={path}")


def test_plans_with_different_shared_memory_coexist():
    """A plan created later with a smaller shared-memory need must not break
    launches of an earlier plan that needs more (kernel attributes are
    process-wide)."""
    import torch
    dirty, psf = _inputs(200, 256, (400, 512), "sky", 12)
    big_ref = oracle.clean_f32(dirty, psf, 0.1, 300, 0.0, (1, 1), 10)
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    big = cg.Plan(d_psf, 200, 256, gain=0.1, niter=300, tiles=(1, 1), feedback_interval=10,
                  group_ctas=1, group_sync=cg.SYNC_CLUSTER)
    # about 200 KB of shared memory either way: a resident slab, or the ring of
    # the pipelined kernel
    small_dirty, small_psf = _inputs(32, 32, (64, 64), "rand", 13)
    small = cg.Plan(torch.from_numpy(small_psf).cuda(), 32, 32, niter=50, tiles=(2, 2),
                    feedback_interval=3)
    small.run(torch.from_numpy(small_dirty).cuda())
    big.run(d_dirty)
    r, m, _ = big.get()
    assert np.array_equal(r.cpu().numpy().view(np.uint32), big_ref.residual.view(np.uint32))
    big.close()
    small.close()


TRIGGER_CASES = [
    # (n, tiles, K, niter, threshold, trigger)
    (128, (2, 2), 0, 600, 1e-3, 0.5),     # rounds end on flux alone
    (250, (4, 4), 20, 1500, 0.0, 0.3),    # interval and trigger, ragged tiles
    (512, (2, 2), 0, 800, 0.0, 0.8),      # streamed slabs
]


@pytest.mark.parametrize("case", TRIGGER_CASES, ids=[f"{c[0]}-t{c[1][0]}x{c[1][1]}-K{c[2]}-trig{c[5]}"
                                                     for c in TRIGGER_CASES])
def test_flux_trigger_bit_exact(case):
    """Flux-triggered feedback rounds (Section 3) equal the oracle."""
    n, tiles, K, niter, thr, trig = case
    dirty, psf = _inputs(n, n, (2 * n, 2 * n), "sky", n + K)
    o = oracle.clean_f32(dirty, psf, 0.1, niter, thr, tiles, K, trigger=trig)
    assert o.rounds > 1
    g = gpu_clean(dirty, psf, 0.1, niter, thr, tiles, K, trigger=trig)
    assert_bit_exact(g, o, str(case))
    g = gpu_clean(dirty, psf, 0.1, niter, thr, tiles, K, trigger=trig, feedback_path=1,
                  minor_path=1)
    assert_bit_exact(g, o, str(case) + " plain paths")


def test_graph_replay_equals_direct_launches():
    """Rounds replayed from two-round CUDA graphs give the same bits as
    kernels launched one by one, and the graphs are really used."""
    import torch
    rng = np.random.default_rng(4242)
    n = 300
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    out = {}
    for graphs in (1, 0):
        with cg.Plan(d_psf, n, n, gain=0.1, niter=2400, tiles=(3, 3), feedback_interval=7) as p:
            p.debug_set(cg.DEBUG_GRAPHS, graphs)
            p.run(d_dirty)
            r, m, c = p.get()
            out[graphs] = (r.cpu().numpy(), m.cpu().numpy(), c, p.stats())
    assert out[1][3]["graph_launches"] > 0 and out[0][3]["graph_launches"] == 0
    assert out[1][3]["rounds_launched"] == out[0][3]["rounds_launched"]
    for a, b in zip(out[1][:2], out[0][:2]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(out[1][2], out[0][2])
    o = oracle.clean_f32(dirty, psf, 0.1, 2400, 0.0, (3, 3), 7)
    assert np.array_equal(out[1][0].view(np.uint32), o.residual.view(np.uint32))


@pytest.mark.parametrize("mode", [cg.FB_GATHER, cg.FB_FFT])
def test_checkpoint_resume_equals_uninterrupted_run(mode):
    """A run stopped after three rounds, checkpointed to host memory and
    resumed in a new plan ends exactly as the uninterrupted run."""
    import torch
    rng = np.random.default_rng(99)
    n = 260
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 15, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    kw = dict(gain=0.1, niter=3000, threshold=1e-3, tiles=(3, 3), feedback_interval=9,
              feedback_mode=mode)

    def result(p):
        r, m, _ = p.get()
        return r.cpu().numpy(), m.cpu().numpy(), p.components_with_rounds()

    with cg.Plan(d_psf, n, n, **kw) as p:
        p.run(d_dirty)
        want = result(p)
    with cg.Plan(d_psf, n, n, **kw) as p:
        p.run(d_dirty, max_rounds=3)
        blob = p.checkpoint()
    with cg.Plan(d_psf, n, n, **kw) as q:
        q.resume(blob)
        q.run(None)
        got = result(q)
        with pytest.raises(cg.CleanError):
            q.resume(blob[:-4])                 # truncated
        bad = bytearray(blob)
        bad[0] ^= 1
        with pytest.raises(cg.CleanError):
            q.resume(bytes(bad))                # not a checkpoint
    with cg.Plan(d_psf, n, n, **dict(kw, niter=2999)) as other:
        with pytest.raises(cg.CleanError):
            other.resume(blob)                  # another problem
    for a, b in zip(got[:2], want[:2]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    for k in ("y", "x", "tile", "round"):
        assert np.array_equal(got[2][k], want[2][k])
    assert np.array_equal(got[2]["flux"].view(np.uint32), want[2]["flux"].view(np.uint32))


def test_checkpoint_resume_with_tile_pairs():
    """Checkpoint and resume under tile pairs (streamed rows, grid groups of
    2G CTAs, TMEM chunks): the resumed run restarts the exchange count and
    ends exactly as the uninterrupted run and the oracle."""
    import torch
    rng = np.random.default_rng(123)
    n = 1024
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 30, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    d_psf, d_dirty = torch.from_numpy(psf).cuda(), torch.from_numpy(dirty).cuda()
    kw = dict(gain=0.1, niter=900, tiles=(2, 2), feedback_interval=25, group_ctas=2,
              group_sync=cg.SYNC_GRID)
    o = oracle.clean_f32(dirty, psf, 0.1, 900, 0.0, (2, 2), 25)
    with cg.Plan(d_psf, n, n, **kw) as p:
        p.debug_set(cg.DEBUG_MINOR_PATH, 2)
        p.run(d_dirty, max_rounds=3)
        assert p.stats()["minor_pairs"] == 1 and p.stats()["minor_tmem"] == 1
        blob = p.checkpoint()
    with cg.Plan(d_psf, n, n, **kw) as q:
        q.debug_set(cg.DEBUG_MINOR_PATH, 2)
        q.resume(blob)
        q.run(None)
        r, m, _ = q.get()
        comps = q.components_with_rounds()
        g = dict(residual=r.cpu().numpy(), model=m.cpu().numpy(), comps=comps,
                 n=len(comps["y"]))
    assert_bit_exact(g, o, "resumed under tile pairs")


DEGENERATE = [
    # (ny, nx, psf, tiles, K, niter, threshold): one-pixel images and tiles,
    # strips, a one-pixel PSF, budgets smaller than the tile count, a single
    # iteration, a threshold above every pixel
    (1, 1, (1, 1), (1, 1), 0, 5, 0.0),
    (1, 40, (1, 80), (1, 4), 2, 30, 0.0),
    (40, 1, (80, 1), (5, 1), 3, 30, 0.0),
    (8, 8, (16, 16), (8, 8), 1, 100, 0.0),
    (30, 30, (1, 1), (3, 3), 2, 200, 0.0),
    (20, 20, (40, 40), (4, 4), 2, 7, 0.0),
    (20, 20, (40, 40), (2, 2), 2, 50, 100.0),
    (16, 16, (32, 32), (2, 2), 1, 1, 0.0),
]


@pytest.mark.parametrize("case", DEGENERATE, ids=[f"{c[0]}x{c[1]}-psf{c[2][0]}x{c[2][1]}-t{c[3][0]}x{c[3][1]}-n{c[5]}"
                                                  for c in DEGENERATE])
def test_degenerate_bit_exact(case):
    ny, nx, ps, tiles, K, niter, thr = case
    rng = np.random.default_rng(ny * 131 + nx)
    psf = synth.random_psf(*ps, rng) if ps[0] * ps[1] > 1 else np.ones((1, 1), np.float32)
    dirty = synth.random_image(ny, nx, rng)
    o = oracle.clean_f32(dirty, psf, 0.3, niter, thr, tiles, K)
    g = gpu_clean(dirty, psf, 0.3, niter, thr, tiles, K)
    assert_bit_exact(g, o, str(case))
    if thr >= 100.0:
        assert g["n"] == 0 and np.array_equal(g["residual"], dirty)
