"""The paper's accuracy band on the 1024 x 1024, 2 x 2 tile workload.

Section 4 (and the abstract): with 4 tiles on a 1024 x 1024 image holding
sources up to 2.1 Jy, the tiled-feedback reconstruction agreed with standard
Hogbom CLEAN to within -0.1 Jy .. +0.04 Jy over the whole image.  The
reconstructed image is read as the restored image (model convolved with a
Gaussian clean beam fitted to the PSF main lobe, plus the residual); the
difference is tiled minus standard.  This is statistical evidence on
synthetic data, not an exact pin.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.slow
def test_paper_band_tiled_vs_untiled_1024():
    w = synth.workload("tiled-1024").build()
    psf, dirty = w["psf"], w["dirty"]
    beam = synth.fit_beam(psf)
    std = oracle.clean_f32(dirty, psf, 0.1, 10000, 5e-3, (1, 1), 0)
    til = oracle.clean_f32(dirty, psf, 0.1, 10000, 5e-3, (2, 2), 50)
    diff = oracle.restore(til.model, til.residual, *beam) - \
        oracle.restore(std.model, std.residual, *beam)
    assert diff.min() >= -0.1 and diff.max() <= 0.04
    # both runs stopped on the threshold, not on the budget
    assert std.n < 10000 and til.n < 10000
    assert np.abs(std.residual).max() <= np.float32(5e-3)
