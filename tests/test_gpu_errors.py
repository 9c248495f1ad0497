"""Error conventions of the C ABI on a GPU.  Nothing here faults, traps or
hangs the device: failures are made on the host (bad inputs, an allocation
cap) or by a bounded device wait that is made to expire."""
import numpy as np
import pytest

import paper_2501_01461_gb300 as cg
import synth

pytestmark = pytest.mark.gpu


def _psf(n=64):
    return synth.make_psf(2 * n, 2 * n)


def test_nonfinite_dirty():
    import torch
    psf = torch.from_numpy(_psf()).cuda()
    d = np.zeros((64, 64), np.float32)
    d[3, 5] = np.nan
    with cg.Plan(psf, 64, 64, niter=10, tiles=(2, 2), feedback_interval=2) as p:
        with pytest.raises(cg.CleanError) as e:
            p.run(torch.from_numpy(d).cuda())
        assert e.value.status == 2
        d[3, 5] = 0.0
        d[10, 10] = np.inf
        with pytest.raises(cg.CleanError) as e:
            p.run(torch.from_numpy(d).cuda())
        assert e.value.status == 2
        d[10, 10] = 1.0
        p.run(torch.from_numpy(d).cuda())   # the plan is still usable
        assert p.n_components() == 10


def test_nonfinite_psf_and_offcentre_psf():
    import torch
    bad = _psf()
    bad[5, 7] = np.nan
    with pytest.raises(cg.CleanError) as e:
        cg.Plan(torch.from_numpy(bad).cuda(), 64, 64, niter=10)
    assert e.value.status == 2
    off = _psf()
    off[0, 0] = 1.5
    with pytest.raises(cg.CleanError) as e:
        cg.Plan(torch.from_numpy(off).cuda(), 64, 64, niter=10)
    assert e.value.status == 1


def test_alloc_cap_gives_oom():
    import torch
    psf = torch.from_numpy(_psf()).cuda()
    cg.lib().clean_debug_alloc_limit(1000)
    try:
        with pytest.raises(cg.CleanError) as e:
            cg.Plan(psf, 64, 64, niter=10)
        assert e.value.status == 3
    finally:
        cg.lib().clean_debug_alloc_limit(-1)
    cg.Plan(psf, 64, 64, niter=10).close()


def test_grid_barrier_timeout_is_bounded_and_poisons():
    """The first grid-barrier wait waits for an arrival that never comes; it
    expires after 20 ms, the kernel returns, the plan reports TIMEOUT from
    then on, and the device stays usable for a new plan."""
    import time
    import torch
    psf = torch.from_numpy(_psf()).cuda()
    d = torch.from_numpy(synth.random_image(64, 64, 1)).cuda()
    p = cg.Plan(psf, 64, 64, niter=50, tiles=(1, 1), mode=cg.UNTILED_GRID, group_ctas=8)
    p.debug_set(cg.DEBUG_SPIN_LIMIT_NS, 20_000_000)
    p.debug_set(cg.DEBUG_FORCE_TIMEOUT, 1)
    t0 = time.time()
    with pytest.raises(cg.CleanError) as e:
        p.run(d)
    assert e.value.status == 5
    assert time.time() - t0 < 30
    with pytest.raises(cg.CleanError) as e:
        p.run(d)
    assert e.value.status == 5
    p.close()
    q = cg.Plan(psf, 64, 64, niter=50, mode=cg.UNTILED_GRID, group_ctas=8)
    q.run(d)
    assert q.n_components() == 50
    q.close()


def test_bad_calls():
    import torch
    psf = torch.from_numpy(_psf()).cuda()
    with cg.Plan(psf, 64, 64, niter=10) as p:
        with pytest.raises(cg.CleanError):
            p.run(None)          # nothing to continue
        with pytest.raises(cg.CleanError):
            p.step()
        with pytest.raises(ValueError):
            p.run(torch.zeros((32, 32), device="cuda"))
    with pytest.raises(cg.CleanError) as e:
        cg.Plan(psf, 64, 64, niter=10, feedback_mode=9)
    assert e.value.status == 1


def test_forced_grid_timeout_with_tile_pairs():
    """Tile pairs: an exchange poll that expires (a mark no CTA writes) sets
    CLEAN_ERR_TIMEOUT, stops both tiles of every pair and returns within
    bounded time; the plan stays poisoned and a new plan runs normally."""
    import time
    import torch
    n = 512
    psf = torch.from_numpy(synth.make_psf(2 * n, 2 * n)).cuda()
    d = torch.from_numpy(synth.random_image(n, n, 3)).cuda()
    kw = dict(niter=400, tiles=(1, 2), feedback_interval=10, group_ctas=2,
              group_sync=cg.SYNC_GRID)
    p = cg.Plan(psf, n, n, **kw)
    p.debug_set(cg.DEBUG_MINOR_PATH, 2)
    assert p.stats()["minor_pairs"] == 1
    p.debug_set(cg.DEBUG_SPIN_LIMIT_NS, 20_000_000)
    p.debug_set(cg.DEBUG_FORCE_TIMEOUT, 1)
    t0 = time.time()
    with pytest.raises(cg.CleanError) as e:
        p.run(d)
    assert e.value.status == 5
    assert time.time() - t0 < 30
    p.close()
    q = cg.Plan(psf, n, n, **kw)
    q.debug_set(cg.DEBUG_MINOR_PATH, 2)
    q.run(d)
    assert q.n_components() == 400 and q.stats()["minor_pairs"] == 1
    q.close()
