"""clean_hogbom_noalloc: Hogbom CLEAN for callers that cannot allocate.

A pipeline that reserves all of its device memory up front, or code running
inside a framework that owns every allocation, cannot let a library call
cudaMalloc mid-run.  clean_hogbom_noalloc takes caller-owned inputs and
outputs and keeps its own small working state in a fixed array compiled
into the library.  These checks call it through the C ABI, twice in a row on
different inputs (so state left by the first call must not leak into the
second), and compare every output bit for bit with the plan-based untiled
path (clean_plan + clean_run with CLEAN_UNTILED_GRID), the tolerance all GPU
parity tests here use.  The file runs last and also passes on its own.
"""
import ctypes

import numpy as np
import pytest

import paper_2501_01461_gb300 as cg
import synth

pytestmark = pytest.mark.gpu


def _reference(dirty, psf, gain, niter, thr):
    import torch
    ny, nx = dirty.shape
    d_psf = torch.from_numpy(psf).cuda()
    with cg.Plan(d_psf, ny, nx, gain=gain, niter=niter, threshold=thr,
                 mode=cg.UNTILED_GRID) as p:
        p.run(torch.from_numpy(dirty).cuda())
        r, m, comps = p.get()
        torch.cuda.synchronize()
        return r.cpu().numpy(), m.cpu().numpy(), comps


def _noalloc(dirty, psf, gain, niter, thr, alias=False, check_free=False):
    """Runs the entry point on caller-owned buffers.  alias: the residual is
    written over the dirty image's buffer.  check_free: after a first call
    (which loads the kernels), a second call must leave the device's free
    memory exactly as it was."""
    import torch
    ny, nx = dirty.shape
    # the caller owns every buffer; the library allocates nothing
    d_dirty = torch.from_numpy(dirty).cuda()
    d_psf = torch.from_numpy(psf).cuda()
    d_res = d_dirty if alias else torch.empty_like(d_dirty)
    d_mod = torch.empty_like(d_dirty)
    d_comps = torch.empty((max(niter, 1), 4), dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    stream = torch.cuda.current_stream()

    def call(src):
        return cg.lib().clean_hogbom_noalloc(
            ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(d_psf.data_ptr()),
            ny, nx, psf.shape[0], psf.shape[1], float(gain), int(niter), float(thr),
            ctypes.c_void_p(d_res.data_ptr()), ctypes.c_void_p(d_mod.data_ptr()),
            ctypes.c_void_p(d_comps.data_ptr()), ctypes.byref(n),
            ctypes.c_void_p(stream.cuda_stream))

    if check_free:
        src = d_dirty.clone()                   # the aliased run overwrites d_dirty
        assert call(src) == 0
        torch.cuda.synchronize()
        if alias:
            d_dirty.copy_(src)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = call(d_dirty)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
    else:
        rc = call(d_dirty)
    assert rc == 0, cg.STATUS.get(rc, rc)
    c = d_comps[:n.value].cpu().numpy()
    return d_res.cpu().numpy(), d_mod.cpu().numpy(), c, n.value


def _same(noalloc_out, ref):
    r1, m1, c1, n1 = noalloc_out
    r0, m0, c0 = ref
    assert n1 == len(c0) > 0
    assert np.array_equal(c1[:, 0], c0["y"]) and np.array_equal(c1[:, 1], c0["x"])
    assert np.array_equal(c1[:, 2], c0["flux"].view(np.int32))
    assert np.array_equal(r1.view(np.uint32), r0.view(np.uint32))
    assert np.array_equal(m1.view(np.uint32), m0.view(np.uint32))


def test_noalloc_matches_plan_path_twice_in_a_row():
    cg.build()
    rng = np.random.default_rng(77)
    cases = []
    # 1: the untiled workload's shape and law: 256^2 image, 512^2 PSF
    w = synth.workload("untiled-256").build()
    cases.append((w["dirty"], w["psf"], 0.1, 2000, 5e-3))
    # 2: a different, non-square image right after, threshold 0
    psf = synth.make_psf(2 * 160, 2 * 160)
    ys, xs, fl = synth.make_sky(160, 12, 0.05, 2.1, rng)
    d = synth.make_dirty(psf, 160, ys, xs, fl, 1e-3, rng)
    dirty = np.ascontiguousarray(np.concatenate([d, d[:40] * 0.5], axis=0))
    cases.append((dirty, psf, 0.15, 700, 0.0))
    for dirty, psf, gain, niter, thr in cases:
        _same(_noalloc(dirty, psf, gain, niter, thr), _reference(dirty, psf, gain, niter, thr))


def test_noalloc_short_image_aliased_and_allocation_free():
    """An image with fewer rows than SMs (48 x 300: one CTA per row), the
    residual written over the dirty image's own buffer, equal to the plan
    path bit for bit; a warmed-up call leaves the device's free memory
    unchanged."""
    cg.build()
    rng = np.random.default_rng(78)
    psf = synth.random_psf(96, 600, rng)
    dirty = synth.random_image(48, 300, rng)
    ref = _reference(dirty, psf, 0.1, 500, 0.0)
    _same(_noalloc(dirty, psf, 0.1, 500, 0.0, alias=True, check_free=True), ref)


def test_noalloc_rejects_bad_arguments():
    cg.build()
    L = cg.lib()
    rc = L.clean_hogbom_noalloc(None, None, 16, 16, 32, 32, 0.1, 10, 0.0, None, None, None,
                                None, None)
    assert rc == 1
    rc = L.clean_hogbom_noalloc(None, None, 0, 16, 32, 32, 0.1, 10, 0.0, None, None, None,
                                None, None)
    assert rc == 1
