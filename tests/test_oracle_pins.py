"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics,
independent of the oracle's own code.

* hand-derived worked examples (exact dyadic arithmetic), tests/golden/
* single point source: closed form S (1 - g)^n for the peak residual,
  g S (1 - g)^(k-1) for component k (Section 3, both equations)
* identity: model convolved with the PSF plus residual equals the dirty
  image (Section 3: the components record every PSF subtracted); holds after
  the final feedback of a tiled run, fails without feedback (Fig. 1(b))
* a 1 x 1 tile grid with any feedback interval equals plain CLEAN
* delta PSF and non-interacting tiles: tiled equals untiled bit for bit
* brute force: a literal NumPy restatement (full shifted-PSF images, explicit
  cross-coupling subtraction) on tiny images over many grids and intervals
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _golden():
    g = json.load(open(GOLDEN))
    psf = np.zeros(g["psf"]["shape"], np.float32)
    for y, x, v in g["psf"]["nonzero"]:
        psf[y, x] = v
    return g, psf, np.array(g["dirty"], np.float32)


def _comp_rows(r):
    c = r.comps
    return [[int(c["y"][i]), int(c["x"][i]), float(c["flux"][i]), int(c["tile"][i]),
             int(c["round"][i])] for i in range(r.n)]


@pytest.mark.parametrize("fn", [oracle.clean_f32, oracle.clean_f64])
def test_worked_examples(fn):
    g, psf, dirty = _golden()
    for case in g["cases"]:
        r = fn(dirty, psf, case["gain"], case["niter"], case["threshold"],
               tuple(case["tiles"]), case["K"], trigger=case.get("trigger", 0.0))
        assert _comp_rows(r) == case["components"], case["name"]
        assert np.array_equal(r.residual, np.array(case["residual"])), case["name"]
        assert r.rounds == case["rounds"], case["name"]


def test_worked_examples_brute():
    g, psf, dirty = _golden()
    for case in g["cases"]:
        r = oracle.brute_clean(dirty, psf, case["gain"], case["niter"], case["threshold"],
                               tuple(case["tiles"]), case["K"], trigger=case.get("trigger", 0.0))
        assert _comp_rows(r) == case["components"], case["name"]
        assert np.array_equal(r.residual, np.array(case["residual"])), case["name"]


def _point_source(n, S, gain, pos, psf_n=None):
    psf = synth.make_psf(psf_n or 2 * n, psf_n or 2 * n)
    ys, xs = np.array([pos[0]]), np.array([pos[1]])
    dirty = synth.make_dirty(psf, n, ys, xs, np.array([S]), 0.0, 0)
    return psf, dirty


@pytest.mark.parametrize("S", [2.1, -0.75, 2.0, -0.5])
def test_point_source_closed_form_f64(S):
    n, g, iters = 48, 0.1, 60
    psf, dirty = _point_source(n, S, g, (17, 30))
    S32 = float(dirty[17, 30])          # the dirty image holds S rounded to float32
    r = oracle.clean_f64(dirty, psf, g, iters)
    g32 = float(np.float32(g))
    assert r.n == iters
    assert np.all(r.comps["y"] == 17) and np.all(r.comps["x"] == 30)
    k = np.arange(1, iters + 1)
    want = g32 * S32 * (1 - g32) ** (k - 1)
    assert np.allclose(r.comps["flux"], want, rtol=0, atol=1e-12 * abs(S32))
    assert abs(r.residual[17, 30] - S32 * (1 - g32) ** iters) <= 1e-12 * abs(S32)
    assert abs(r.comps["flux"].sum() - S32 * (1 - (1 - g32) ** iters)) <= 1e-12 * abs(S32)
    if S in (2.0, -0.5):
        # S * P is exact in float32 for a power of two, so the closed form
        # holds until (1 - g)^n nears float64 resolution: the sum tends to S
        n_long = 200
        r2 = oracle.clean_f64(dirty, psf, g, n_long)
        assert np.all(r2.comps["y"] == 17) and np.all(r2.comps["x"] == 30)
        err = abs(r2.model[17, 30] - S32 * (1 - (1 - g32) ** n_long))
        assert err <= 1e-12 * abs(S32)
        assert abs(r2.model[17, 30] - S32) <= abs(S32) * (1 - g32) ** n_long * 1.001


def test_point_source_closed_form_f32():
    n, g, S, iters = 48, 0.1, 2.1, 60
    psf, dirty = _point_source(n, S, g, (5, 40))
    r = oracle.clean_f32(dirty, psf, g, iters)
    S32, g32 = float(dirty[5, 40]), float(np.float32(g))
    assert np.all(r.comps["y"] == 5) and np.all(r.comps["x"] == 40)
    bound = iters * 2.0 ** -23 * S32
    assert abs(float(r.residual[5, 40]) - S32 * (1 - g32) ** iters) <= bound
    assert abs(float(r.model[5, 40]) - S32 * (1 - (1 - g32) ** iters)) <= bound


def _identity_err(r, dirty, psf):
    rebuilt = oracle.psf_convolve(r.model, psf) + np.asarray(r.residual, np.float64)
    return np.abs(rebuilt - dirty.astype(np.float64)).max()


@pytest.mark.parametrize("tiles,K", [((1, 1), 0), ((2, 2), 5), ((3, 2), 1), ((4, 4), 3)])
def test_identity_f64(tiles, K):
    rng = np.random.default_rng(7)
    n = 40
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    r = oracle.clean_f64(dirty, psf, 0.1, 800, 0.0, tiles, K)
    assert r.n == 800
    assert _identity_err(r, dirty, psf) <= 1e-9 * np.abs(dirty).max()


@pytest.mark.parametrize("tiles,K", [((1, 1), 0), ((2, 2), 7)])
def test_identity_f32(tiles, K):
    rng = np.random.default_rng(8)
    n = 40
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    r = oracle.clean_f32(dirty, psf, 0.1, 800, 0.0, tiles, K)
    bound = 8 * r.n * 2.0 ** -24 * np.abs(dirty).max()
    assert _identity_err(r, dirty, psf) <= bound


def test_identity_fails_without_feedback():
    """Independent tiles (Fig. 1(b)): lobes of other tiles' sources stay."""
    rng = np.random.default_rng(9)
    n = 40
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    r = oracle.clean_f64(dirty, psf, 0.1, 800, 0.0, (2, 2), 0)
    assert _identity_err(r, dirty, psf) > 1e-2


@pytest.mark.parametrize("K", [1, 4, 50])
def test_single_tile_equals_untiled(K):
    rng = np.random.default_rng(10)
    n = 32
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 8, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    for fn in (oracle.clean_f32, oracle.clean_f64):
        a = fn(dirty, psf, 0.1, 300, 1e-3, (1, 1), 0)
        b = fn(dirty, psf, 0.1, 300, 1e-3, (1, 1), K)
        assert a.n == b.n
        assert np.array_equal(a.residual, b.residual)
        assert np.array_equal(a.model, b.model)
        for key in ("y", "x", "flux"):
            assert np.array_equal(a.comps[key], b.comps[key])


def test_delta_psf_tiled_equals_untiled():
    rng = np.random.default_rng(11)
    n = 16
    psf = np.zeros((2 * n, 2 * n), np.float32)
    psf[n, n] = 1.0
    dirty = synth.random_image(n, n, rng)
    for fn in (oracle.clean_f32, oracle.clean_f64):
        u = fn(dirty, psf, 0.25, 10 ** 6, 0.01, (1, 1), 0)
        for tiles, K in (((2, 2), 3), ((4, 4), 1), ((3, 5), 0)):
            t = fn(dirty, psf, 0.25, 10 ** 6, 0.01, tiles, K)
            assert np.array_equal(u.model, t.model)
            assert np.array_equal(u.residual, t.residual)
        assert np.abs(u.residual).max() <= np.float32(0.01)


def test_non_interacting_tiles():
    """PSF support radius 3; sources at least 3 pixels from every tile edge."""
    n, r = 32, 3
    yy, xx = np.mgrid[-n:n, -n:n]
    rng = np.random.default_rng(12)
    # a truncated Gaussian (positive definite, so CLEAN converges to the
    # threshold)
    psf = np.where(yy * yy + xx * xx <= r * r,
                   np.exp(-(yy * yy + xx * xx) / 3.0), 0.0).astype(np.float32)
    psf[n, n] = 1.0
    # 2 x 2 tiles of 16 x 16; keep sources in [3, 12] of each tile
    pos = []
    for t in range(4):
        oy, ox = (t // 2) * 16, (t % 2) * 16
        for _ in range(3):
            pos.append((oy + int(rng.integers(r, 16 - r)), ox + int(rng.integers(r, 16 - r))))
    pos = sorted(set(pos))
    ys = np.array([p[0] for p in pos]); xs = np.array([p[1] for p in pos])
    fl = rng.uniform(0.2, 2.0, len(pos)) * rng.choice([-1, 1], len(pos))
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 0.0, 0)
    for fn in (oracle.clean_f32, oracle.clean_f64):
        u = fn(dirty, psf, 0.2, 10 ** 5, 1e-3, (1, 1), 0)
        assert u.n < 10 ** 5 and np.abs(u.residual).max() <= np.float32(1e-3)
        for K in (1, 5, 0):
            t = fn(dirty, psf, 0.2, 10 ** 5, 1e-3, (2, 2), K)
            assert np.array_equal(u.model, t.model)
            assert np.array_equal(u.residual, t.residual)
            # each tile's picks are its subsequence of the untiled picks
            for tile in range(4):
                i, j = divmod(tile, 2)
                sel = (u.comps["y"] // 16 == i) & (u.comps["x"] // 16 == j)
                mine = t.comps["tile"] == tile
                assert np.array_equal(u.comps["y"][sel], t.comps["y"][mine])
                assert np.array_equal(u.comps["flux"][sel], t.comps["flux"][mine])


BRUTE_CASES = [(tiles, K) for tiles in ((1, 1), (2, 2), (4, 4), (2, 3))
               for K in (1, 3, 7, 0)]


@pytest.mark.parametrize("tiles,K", BRUTE_CASES)
def test_brute_force_16(tiles, K):
    rng = np.random.default_rng(abs(hash((tiles, K))) % 2 ** 31)
    ny, nx = 16, 13 if tiles == (2, 3) else 16
    psf = synth.random_psf(2 * ny, 2 * nx, rng)
    for dirty, thr in ((synth.random_image(ny, nx, rng), 0.05),
                       (synth.tie_image(ny, nx, rng), 0.0)):
        for dt, fn in ((np.float32, oracle.clean_f32), (np.float64, oracle.clean_f64)):
            a = fn(dirty, psf, 0.3, 45, thr, tiles, K)
            b = oracle.brute_clean(dirty, psf, 0.3, 45, thr, tiles, K, dtype=dt)
            assert a.n == b.n and a.rounds == b.rounds
            assert np.array_equal(a.residual, b.residual)
            assert np.array_equal(a.model, b.model)
            for key in ("y", "x", "flux", "tile", "round"):
                assert np.array_equal(a.comps[key], b.comps[key]), key


def test_brute_force_clipped_psf():
    """PSF smaller than the image: pixels off the PSF array are untouched."""
    rng = np.random.default_rng(13)
    psf = synth.random_psf(7, 5, rng)
    dirty = synth.random_image(12, 15, rng)
    for tiles, K in (((1, 1), 0), ((3, 2), 2)):
        a = oracle.clean_f32(dirty, psf, 0.5, 30, 0.0, tiles, K)
        b = oracle.brute_clean(dirty, psf, 0.5, 30, 0.0, tiles, K)
        assert np.array_equal(a.residual, b.residual)
        assert np.array_equal(a.comps["flux"], b.comps["flux"])


def test_replay_matches_independent_f64_when_no_near_ties():
    """Replaying the float32 list in float64 reproduces the float64 run when
    the two trajectories pick the same pixels."""
    rng = np.random.default_rng(14)
    n = 24
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 4, 0.3, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 0.0, rng)
    a = oracle.clean_f32(dirty, psf, 0.1, 120, 0.0, (2, 2), 5)
    b = oracle.clean_f64(dirty, psf, 0.1, 120, 0.0, (2, 2), 5)
    rep = oracle.clean_f64(dirty, psf, 0.1, 120, 0.0, (2, 2), 5, replay=a.comps)
    same = np.array_equal(a.comps["y"], b.comps["y"]) and np.array_equal(a.comps["x"], b.comps["x"])
    assert np.array_equal(rep.comps["y"], a.comps["y"])
    assert np.array_equal(rep.comps["round"], a.comps["round"])
    assert np.abs(rep.model - a.model).max() < 1e-5
    if same:
        assert np.array_equal(rep.model, b.model)
        assert np.array_equal(rep.residual, b.residual)


def test_budget_split_and_rounds():
    """niter = 7 over 4 tiles gives budgets 2, 2, 2, 1; K = 1 needs 2 rounds."""
    rng = np.random.default_rng(15)
    psf = synth.random_psf(16, 16, rng)
    dirty = synth.random_image(8, 8, rng)
    r = oracle.clean_f32(dirty, psf, 0.2, 7, 0.0, (2, 2), 1)
    assert r.rounds == 2
    assert np.bincount(r.comps["tile"], minlength=4).tolist() == [2, 2, 2, 1]
    assert r.comps["tile"].tolist() == [0, 1, 2, 3, 0, 1, 2]


@pytest.mark.parametrize("tiles,K,trigger", [((2, 2), 0, 0.5), ((4, 4), 3, 0.3), ((2, 3), 0, 0.9),
                                             ((1, 1), 0, 0.5)])
def test_brute_force_flux_trigger(tiles, K, trigger):
    """Flux-triggered rounds (Section 3): literal restatement agrees."""
    rng = np.random.default_rng(int(trigger * 100) + K)
    ny, nx = 16, 15 if tiles == (2, 3) else 16
    psf = synth.random_psf(2 * ny, 2 * nx, rng)
    for dirty in (synth.random_image(ny, nx, rng), synth.tie_image(ny, nx, rng)):
        for dt, fn in ((np.float32, oracle.clean_f32), (np.float64, oracle.clean_f64)):
            a = fn(dirty, psf, 0.3, 60, 0.02, tiles, K, trigger=trigger)
            b = oracle.brute_clean(dirty, psf, 0.3, 60, 0.02, tiles, K, dtype=dt, trigger=trigger)
            assert a.n == b.n and a.rounds == b.rounds
            assert np.array_equal(a.residual, b.residual)
            for key in ("y", "x", "flux", "tile", "round"):
                assert np.array_equal(a.comps[key], b.comps[key]), key


def test_flux_trigger_identity_and_progress():
    """Every round makes progress and the final feedback keeps
    model * PSF + residual = dirty."""
    rng = np.random.default_rng(17)
    n = 40
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 12, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    r = oracle.clean_f64(dirty, psf, 0.1, 600, 1e-3, (2, 2), 0, trigger=0.5)
    assert r.n == 600 or np.abs(r.residual).max() <= np.float32(1e-3) * 1.0000001
    assert len(np.unique(r.comps["round"])) == r.rounds
    assert _identity_err(r, dirty, psf) <= 1e-9 * np.abs(dirty).max()
