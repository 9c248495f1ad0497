"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/cleangb.h declares, and rejects bad
parameters before touching a device."""
import ctypes
import os
import re

import pytest

import paper_2501_01461_gb300 as cg

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cleangb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(clean_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    cg.build()
    return cg.lib()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(cg.EXPORTED_SYMBOLS)


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror(lib):
    for code, name in cg.STATUS.items():
        assert lib.clean_strerror(code)
    assert lib.clean_strerror(99) == b"unknown status"


def _params(**kw):
    base = dict(ny=64, nx=64, psf_shape=(128, 128), gain=0.1, niter=100, threshold=0.0,
                tiles=(2, 2), feedback_interval=5)
    base.update(kw)
    psf_shape = base.pop("psf_shape")
    return cg.make_params(base.pop("ny"), base.pop("nx"), psf_shape, **base)


def test_params_check_accepts_valid(lib):
    assert lib.clean_params_check(ctypes.byref(_params())) == 0
    assert lib.clean_params_check(ctypes.byref(_params(mode=cg.UNTILED_GRID, tiles=(1, 1)))) == 0


@pytest.mark.parametrize("bad", [
    dict(ny=0), dict(nx=-1), dict(psf_shape=(0, 5)), dict(gain=0.0), dict(gain=1.5),
    dict(gain=float("nan")), dict(threshold=-1.0), dict(threshold=float("inf")),
    dict(niter=-1), dict(tiles=(0, 1)), dict(tiles=(65, 1)), dict(tiles=(1, 65)),
    dict(ny=4, tiles=(5, 1)), dict(feedback_interval=-1), dict(feedback_mode=7),
    dict(mode=3), dict(mode=cg.UNTILED_GRID, tiles=(2, 1)), dict(group_ctas=-2),
    dict(group_sync=9), dict(group_sync=cg.SYNC_CLUSTER, group_ctas=32),
    dict(ny=50000, nx=50000), dict(feedback_trigger=1.0), dict(feedback_trigger=-0.1),
    dict(feedback_trigger=float("nan")),
])
def test_params_check_rejects(lib, bad):
    assert lib.clean_params_check(ctypes.byref(_params(**bad))) == 1


def test_reserved_must_be_zero(lib):
    p = _params()
    p.reserved[2] = 1
    assert lib.clean_params_check(ctypes.byref(p)) == 1


def test_plan_rejects_bad_params_before_any_cuda_call(lib):
    h = ctypes.c_void_p(123)
    assert lib.clean_plan(ctypes.byref(h), ctypes.byref(_params(gain=2.0)), None, None) == 1
    assert h.value is None
    assert lib.clean_plan(None, ctypes.byref(_params()), None, None) == 1


def test_null_plan_calls(lib):
    assert lib.clean_run(None, None, -1, None) == 1
    assert lib.clean_step(None, None) == 1
    assert lib.clean_feedback(None, None) == 1
    assert lib.clean_get(None, None, None, None, 0, None, None) == 1
    lib.clean_destroy(None)


def test_checkpoint_resume_reject_without_a_plan(lib):
    n = ctypes.c_int64(0)
    assert lib.clean_checkpoint(None, None, 0, ctypes.byref(n), None) == 1
    assert lib.clean_resume(None, b"x" * 64, 64, None) == 1


def test_no_oracle_in_product():
    """The product package never imports, links or reads the oracle."""
    pkg = os.path.dirname(cg.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "clean_oracle" not in txt and "liboracle" not in txt, f
