"""Pins for the oracle's auxiliary functions and the beam fit.

* restore: a unit component restores to the clean beam, whose value is 1/2
  at half the FWHM along each axis (the definition of FWHM), whose axes turn
  with the position angle, and whose pixel sum is the Gaussian integral
  2 pi sigma_maj sigma_min
* psf_convolve: FFT evaluation equals a brute-force double loop on tiny
  inputs, and a delta model gives the shifted PSF
* fit_beam: recovers the FWHMs and angle of a sampled elliptical Gaussian
"""
import math

import numpy as np
import pytest

import oracle
import synth

K_FWHM = 2.0 * math.sqrt(2.0 * math.log(2.0))


def test_restore_half_maximum_and_axes():
    n = 64
    model = np.zeros((n, n))
    model[32, 32] = 1.0
    res = np.zeros((n, n))
    out = oracle.restore(model, res, 8.0, 6.0, 0.0)      # major axis along +x
    assert out[32, 32] == pytest.approx(1.0)
    assert out[32, 36] == pytest.approx(0.5, rel=1e-12)  # +bmaj/2 along x
    assert out[32, 28] == pytest.approx(0.5, rel=1e-12)
    assert out[35, 32] == pytest.approx(0.5, rel=1e-12)  # +bmin/2 along y
    rot = oracle.restore(model, res, 8.0, 6.0, math.pi / 2)   # major axis along +y
    assert rot[36, 32] == pytest.approx(0.5, rel=1e-12)
    assert rot[32, 35] == pytest.approx(0.5, rel=1e-12)


def test_restore_flux_integral_and_residual():
    n = 96
    model = np.zeros((n, n))
    model[48, 40] = 2.5
    rng = np.random.default_rng(0)
    res = rng.normal(0, 1e-3, (n, n))
    bmaj, bmin = 9.0, 5.5
    out = oracle.restore(model, res, bmaj, bmin, 0.4)
    integral = 2.5 * 2 * math.pi * (bmaj / K_FWHM) * (bmin / K_FWHM)
    assert (out - res).sum() == pytest.approx(integral, rel=1e-6)
    far = out.copy()
    far[48 - 20:48 + 21, 40 - 20:40 + 21] = res[48 - 20:48 + 21, 40 - 20:40 + 21]
    assert np.array_equal(far, res)   # nothing beyond the truncation radius


def test_psf_convolve_matches_brute_force():
    rng = np.random.default_rng(1)
    model = np.where(rng.random((9, 11)) < 0.2, rng.normal(size=(9, 11)), 0.0)
    psf = rng.normal(size=(7, 10))
    cy, cx = 7 // 2, 10 // 2
    want = np.zeros((9, 11))
    for qy in range(9):
        for qx in range(11):
            s = 0.0
            for py in range(9):
                for px in range(11):
                    iy, ix = qy - py + cy, qx - px + cx
                    if 0 <= iy < 7 and 0 <= ix < 10:
                        s += model[py, px] * psf[iy, ix]
            want[qy, qx] = s
    assert np.allclose(oracle.psf_convolve(model, psf), want, atol=1e-12)
    delta = np.zeros((9, 11))
    delta[4, 6] = 3.0
    got = oracle.psf_convolve(delta, psf)
    assert got[4 - 1, 6 + 2] == pytest.approx(3.0 * psf[cy - 1, cx + 2])


@pytest.mark.parametrize("bmaj,bmin,pa", [(10.0, 6.0, 0.0), (12.0, 7.0, 0.6), (8.0, 8.0, 0.0)])
def test_fit_beam_recovers_gaussian(bmaj, bmin, pa):
    n = 128
    yy, xx = np.mgrid[-n // 2:n // 2, -n // 2:n // 2].astype(np.float64)
    psf = oracle.gaussian_beam(bmaj, bmin, pa, yy, xx).astype(np.float32)
    fmaj, fmin, fpa = synth.fit_beam(psf)
    assert fmaj == pytest.approx(bmaj, rel=0.03)
    assert fmin == pytest.approx(bmin, rel=0.03)
    if bmaj > bmin:
        d = (fpa - pa + math.pi / 2) % math.pi - math.pi / 2
        assert abs(d) < 0.05
