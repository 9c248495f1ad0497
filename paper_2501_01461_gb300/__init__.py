"""Tiled Hogbom CLEAN with feedback on a GB300 GPU (arXiv 2501.01461).

A thin ctypes binding over ``libcleangb.so`` (C ABI in include/cleangb.h).
Every step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory and streams.  There is no
CPU fallback: without the compiled library every call raises.

    import torch, paper_2501_01461_gb300 as cg
    plan = cg.Plan(psf_cuda, ny=1024, nx=1024, gain=0.1, niter=10000,
                   threshold=5e-3, tiles=(2, 2), feedback_interval=50)
    plan.run(dirty_cuda)
    residual, model, comps = plan.get()
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["CleanError", "Plan", "Batch", "lib", "library_path", "build", "STATUS",
           "FB_GATHER", "FB_FFT", "FB_AUTO", "TILED", "UNTILED_GRID",
           "SYNC_AUTO", "SYNC_CLUSTER", "SYNC_GRID", "COMPONENT_DTYPE",
           "DEBUG_SPIN_LIMIT_NS", "DEBUG_FORCE_TIMEOUT", "DEBUG_TIMING", "DEBUG_FEEDBACK_PATH", "DEBUG_MINOR_PATH",
           "DEBUG_PIPE_CHUNK_PX", "DEBUG_PIPE_STAGES", "DEBUG_GRAPHS", "DEBUG_MINOR_TMEM",
           "DEBUG_MINOR_PAIR", "probe_l2_read",
           "EXPORTED_SYMBOLS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
FB_GATHER, FB_FFT, FB_AUTO = 0, 1, 2
TILED, UNTILED_GRID = 0, 1
SYNC_AUTO, SYNC_CLUSTER, SYNC_GRID = 0, 1, 2
DEBUG_SPIN_LIMIT_NS, DEBUG_FORCE_TIMEOUT, DEBUG_TIMING = 1, 2, 3
DEBUG_FEEDBACK_PATH, DEBUG_MINOR_PATH, DEBUG_PIPE_CHUNK_PX, DEBUG_PIPE_STAGES = 4, 5, 6, 7
DEBUG_GRAPHS, DEBUG_MINOR_TMEM, DEBUG_MINOR_PAIR = 8, 9, 10
STATUS = {0: "CLEAN_OK", 1: "CLEAN_ERR_INVALID_ARG", 2: "CLEAN_ERR_NONFINITE",
          3: "CLEAN_ERR_OOM", 4: "CLEAN_ERR_CUDA", 5: "CLEAN_ERR_TIMEOUT",
          6: "CLEAN_ERR_UNSUPPORTED"}
COMPONENT_DTYPE = np.dtype([("y", np.int32), ("x", np.int32), ("flux", np.float32),
                            ("tile", np.int32)])


class CleanError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Params(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("psf_ny", ctypes.c_int32), ("psf_nx", ctypes.c_int32),
                ("gain", ctypes.c_float), ("threshold", ctypes.c_float),
                ("niter", ctypes.c_int64),
                ("tiles_y", ctypes.c_int32), ("tiles_x", ctypes.c_int32),
                ("feedback_interval", ctypes.c_int32), ("feedback_mode", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("group_ctas", ctypes.c_int32),
                ("group_sync", ctypes.c_int32), ("feedback_trigger", ctypes.c_float),
                ("reserved", ctypes.c_int32 * 4)]


class Stats(ctypes.Structure):
    _fields_ = [("n_components", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("rounds_launched", ctypes.c_int64), ("group_ctas", ctypes.c_int32),
                ("group_sync", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("feedback_mode", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("feedback_tma", ctypes.c_int32), ("minor_pipe", ctypes.c_int32),
                ("minor_tmem", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("minor_launches", ctypes.c_int64), ("feedback_launches", ctypes.c_int64),
                ("minor_ms", ctypes.c_double), ("feedback_ms", ctypes.c_double),
                ("graph_launches", ctypes.c_int64), ("minor_pairs", ctypes.c_int64),
                ("host_in_ms", ctypes.c_double), ("host_run_ms", ctypes.c_double),
                ("host_out_ms", ctypes.c_double)]


# name -> (restype, argtypes); the C ABI of include/cleangb.h
_vp, _i32, _i64, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
_SIGS = {
    "clean_params_default": (ctypes.c_int, [_vp]),
    "clean_params_check": (ctypes.c_int, [_vp]),
    "clean_plan": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "clean_set_psf": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "clean_run": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "clean_step": (ctypes.c_int, [_vp, _vp]),
    "clean_feedback": (ctypes.c_int, [_vp, _vp]),
    "clean_restore": (ctypes.c_int, [_vp, _f32, _f32, _f32, _vp, _vp]),
    "clean_get": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "clean_get_rounds": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "clean_deconvolve_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "clean_checkpoint": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "clean_resume": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "clean_stats": (ctypes.c_int, [_vp, _vp, _vp]),
    "clean_destroy": (None, [_vp]),
    "clean_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "clean_debug_set": (ctypes.c_int, [_vp, _i32, _i64]),
    "clean_debug_alloc_limit": (None, [_i64]),
    "clean_hogbom_noalloc": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32, _i32, _f32, _i64, _f32,
                                            _vp, _vp, _vp, _vp, _vp]),
    "clean_batch_create": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "clean_batch_run": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "clean_batch_get": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _i64, _vp, _vp]),
    "clean_batch_stats": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "clean_batch_graphs": (ctypes.c_int, [_vp, _i32, _vp]),
    "clean_batch_destroy": (None, [_vp]),
    "clean_server_create": (ctypes.c_int, [_vp, _i32, _vp]),
    "clean_server_add": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "clean_server_step": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "clean_server_done": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "clean_server_get": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, _vp, _i64, _vp, _vp]),
    "clean_server_remove": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "clean_server_destroy": (None, [_vp]),
    "clean_probe_l2_read": (ctypes.c_int, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp]),
}
EXPORTED_SYMBOLS = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from . import _build
    return _build.LIB


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded libcleangb.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libcleangb.so is not built ({path}); run "
                                   "paper_2501_01461_gb300.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def probe_l2_read(buf, passes=40, method=0, ctas_per_sm=2, stream=None):
    """Read bandwidth of the L2 -> SM path over ``buf`` (a CUDA tensor that
    fits in L2), measured by clean_probe_l2_read.  Returns (bytes read, ms)."""
    import torch
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise TypeError("buf must be a contiguous CUDA tensor")
    nb, ms = ctypes.c_int64(0), ctypes.c_float(0.0)
    _check(lib().clean_probe_l2_read(ctypes.c_void_p(buf.data_ptr()),
                                     buf.numel() * buf.element_size(), int(passes), int(method),
                                     int(ctas_per_sm), ctypes.byref(nb), ctypes.byref(ms),
                                     _stream_ptr(stream)), "clean_probe_l2_read")
    return int(nb.value), float(ms.value)


def _check(status: int, what: str):
    if status != 0:
        raise CleanError(status, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, shape=None, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA torch.Tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{what} must be contiguous float32")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def make_params(ny, nx, psf_shape, gain=0.1, niter=0, threshold=0.0, tiles=(1, 1),
                feedback_interval=0, feedback_mode=FB_GATHER, mode=TILED,
                group_ctas=0, group_sync=SYNC_AUTO, feedback_trigger=0.0) -> Params:
    p = Params()
    lib().clean_params_default(ctypes.byref(p))
    p.ny, p.nx = int(ny), int(nx)
    p.psf_ny, p.psf_nx = int(psf_shape[0]), int(psf_shape[1])
    p.gain, p.threshold, p.niter = float(gain), float(threshold), int(niter)
    p.tiles_y, p.tiles_x = int(tiles[0]), int(tiles[1])
    p.feedback_interval = int(feedback_interval)
    p.feedback_mode, p.mode = int(feedback_mode), int(mode)
    p.group_ctas, p.group_sync = int(group_ctas), int(group_sync)
    p.feedback_trigger = float(feedback_trigger)
    return p


class Plan:
    """A deconvolution plan on the current CUDA device (see clean_plan).

    ``psf`` is a CUDA float32 tensor (borrowed: keep it alive) or None for a
    plan that owns its PSF buffer (fill it with set_psf_host or
    deconvolve_host).
    """

    def __init__(self, psf, ny, nx, gain=0.1, niter=0, threshold=0.0, tiles=(1, 1),
                 feedback_interval=0, feedback_mode=FB_GATHER, mode=TILED,
                 group_ctas=0, group_sync=SYNC_AUTO, psf_shape=None, stream=None,
                 feedback_trigger=0.0):
        if psf is not None:
            psf_shape = tuple(psf.shape)
            ptr = _dptr(psf, what="psf")
        else:
            if psf_shape is None:
                raise ValueError("psf_shape is required when psf is None")
            ptr = None
        self.params = make_params(ny, nx, psf_shape, gain, niter, threshold, tiles,
                                  feedback_interval, feedback_mode, mode, group_ctas,
                                  group_sync, feedback_trigger)
        self.ny, self.nx, self.niter = int(ny), int(nx), int(niter)
        self._psf = psf
        self._h = ctypes.c_void_p()
        _check(lib().clean_plan(ctypes.byref(self._h), ctypes.byref(self.params), ptr,
                                _stream_ptr(stream)), "clean_plan")

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if self._h:
            lib().clean_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- the method --------------------------------------------------------
    def set_psf(self, psf, stream=None):
        _check(lib().clean_set_psf(self._h, _dptr(psf, what="psf"), 0, _stream_ptr(stream)),
               "clean_set_psf")
        self._psf = psf

    def set_psf_host(self, psf: np.ndarray, stream=None):
        psf = np.ascontiguousarray(psf, dtype=np.float32)
        _check(lib().clean_set_psf(self._h, psf.ctypes.data_as(ctypes.c_void_p), 1,
                                   _stream_ptr(stream)), "clean_set_psf")

    def run(self, dirty=None, max_rounds=-1, stream=None):
        ptr = None if dirty is None else _dptr(dirty, (self.ny, self.nx), "dirty")
        _check(lib().clean_run(self._h, ptr, int(max_rounds), _stream_ptr(stream)), "clean_run")

    def step(self, stream=None):
        _check(lib().clean_step(self._h, _stream_ptr(stream)), "clean_step")

    def feedback(self, stream=None):
        _check(lib().clean_feedback(self._h, _stream_ptr(stream)), "clean_feedback")

    def restore(self, bmaj, bmin, bpa, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
        _check(lib().clean_restore(self._h, float(bmaj), float(bmin), float(bpa),
                                   _dptr(out, (self.ny, self.nx), "out"), _stream_ptr(stream)),
               "clean_restore")
        return out

    def n_components(self, stream=None) -> int:
        n = ctypes.c_int64(0)
        _check(lib().clean_get(self._h, None, None, None, 0, ctypes.byref(n),
                               _stream_ptr(stream)), "clean_get")
        return int(n.value)

    def get(self, stream=None):
        """Returns (residual, model) as CUDA tensors and the component list
        as a NumPy structured array (y, x, flux, tile) in list order."""
        import torch
        res = torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
        mod = torch.empty_like(res)
        n = self.n_components(stream)
        comps = torch.empty((max(n, 1), 4), dtype=torch.int32, device="cuda")
        cnt = ctypes.c_int64(0)
        _check(lib().clean_get(self._h, _dptr(res), _dptr(mod), ctypes.c_void_p(comps.data_ptr()),
                               n, ctypes.byref(cnt), _stream_ptr(stream)), "clean_get")
        host = comps[:n].cpu().numpy()
        arr = np.empty(n, dtype=COMPONENT_DTYPE)
        arr["y"], arr["x"], arr["tile"] = host[:, 0], host[:, 1], host[:, 3]
        arr["flux"] = host[:, 2].view(np.float32)
        return res, mod, arr

    def round_offsets(self, stream=None) -> np.ndarray:
        n = ctypes.c_int64(0)
        _check(lib().clean_get_rounds(self._h, None, 0, ctypes.byref(n), _stream_ptr(stream)),
               "clean_get_rounds")
        out = np.zeros(max(n.value, 1), dtype=np.int64)
        _check(lib().clean_get_rounds(self._h, out.ctypes.data_as(ctypes.c_void_p), n.value,
                                      ctypes.byref(n), _stream_ptr(stream)), "clean_get_rounds")
        return out[:n.value]

    def components_with_rounds(self, stream=None):
        """Component dict (y, x, flux, tile, round) as in the oracle's output."""
        _, _, arr = self.get(stream)
        offs = self.round_offsets(stream)
        rnd = np.zeros(len(arr), dtype=np.int32)
        for r, o in enumerate(offs):
            rnd[o:] = r
        return dict(y=arr["y"].copy(), x=arr["x"].copy(), flux=arr["flux"].copy(),
                    tile=arr["tile"].copy(), round=rnd)

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(lib().clean_stats(self._h, ctypes.byref(s), _stream_ptr(stream)), "clean_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def deconvolve_host(self, dirty: np.ndarray, psf: np.ndarray | None = None,
                        residual: np.ndarray | None = None, model: np.ndarray | None = None,
                        comps: np.ndarray | None = None, stream=None) -> int:
        """Whole run with host buffers (clean_deconvolve_host).  Returns the
        number of components; outputs are filled in place when given."""
        def p(a):
            return None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        n = ctypes.c_int64(0)
        cap = 0 if comps is None else len(comps)
        _check(lib().clean_deconvolve_host(self._h, p(dirty), p(psf), p(residual), p(model),
                                           p(comps), cap, ctypes.byref(n), _stream_ptr(stream)),
               "clean_deconvolve_host")
        return int(n.value)

    def checkpoint(self, stream=None) -> bytes:
        """The run's state between rounds as bytes (clean_checkpoint)."""
        n = ctypes.c_int64(0)
        _check(lib().clean_checkpoint(self._h, None, 0, ctypes.byref(n), _stream_ptr(stream)),
               "clean_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().clean_checkpoint(self._h, buf, n.value, ctypes.byref(n), _stream_ptr(stream)),
               "clean_checkpoint")
        return buf.raw[:n.value]

    def resume(self, blob: bytes, stream=None):
        """Loads a checkpoint of a plan with identical parameters; run(None)
        continues it (clean_resume)."""
        _check(lib().clean_resume(self._h, blob, len(blob), _stream_ptr(stream)), "clean_resume")

    def debug_set(self, what: int, value: int):
        _check(lib().clean_debug_set(self._h, int(what), int(value)), "clean_debug_set")


class Batch:
    """Many images deconvolved together (clean_batch_*).

    ``jobs`` is a list of dicts with keys psf (CUDA float32 tensor, borrowed),
    ny, nx and any Plan keyword (gain, niter, threshold, tiles,
    feedback_interval).
    """

    def __init__(self, jobs, stream=None):
        self.n = len(jobs)
        arr = (Params * self.n)()
        self._psfs = []
        ptrs = (ctypes.c_void_p * self.n)()
        self.shapes = []
        for i, j in enumerate(jobs):
            j = dict(j)
            psf = j.pop("psf")
            ny, nx = j.pop("ny"), j.pop("nx")
            arr[i] = make_params(ny, nx, tuple(psf.shape), **j)
            ptrs[i] = _dptr(psf, what="psf").value
            self._psfs.append(psf)
            self.shapes.append((ny, nx))
        self._params = arr
        self._h = ctypes.c_void_p()
        _check(lib().clean_batch_create(ctypes.byref(self._h), self.n, arr, ptrs,
                                        _stream_ptr(stream)), "clean_batch_create")

    def close(self):
        if self._h:
            lib().clean_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def run(self, dirties=None, max_rounds=-1, stream=None):
        if dirties is None:
            p = None
        else:
            ptrs = (ctypes.c_void_p * self.n)()
            for i, d in enumerate(dirties):
                ptrs[i] = _dptr(d, self.shapes[i], "dirty").value
            p = ptrs
        _check(lib().clean_batch_run(self._h, p, int(max_rounds), _stream_ptr(stream)),
               "clean_batch_run")

    def get(self, i, stream=None):
        import torch
        ny, nx = self.shapes[i]
        n = ctypes.c_int64(0)
        _check(lib().clean_batch_get(self._h, int(i), None, None, None, 0, ctypes.byref(n),
                                     _stream_ptr(stream)), "clean_batch_get")
        res = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        mod = torch.empty_like(res)
        comps = torch.empty((max(n.value, 1), 4), dtype=torch.int32, device="cuda")
        _check(lib().clean_batch_get(self._h, int(i), _dptr(res), _dptr(mod),
                                     ctypes.c_void_p(comps.data_ptr()), n.value, ctypes.byref(n),
                                     _stream_ptr(stream)), "clean_batch_get")
        host = comps[:n.value].cpu().numpy()
        arr = np.empty(n.value, dtype=COMPONENT_DTYPE)
        arr["y"], arr["x"], arr["tile"] = host[:, 0], host[:, 1], host[:, 3]
        arr["flux"] = host[:, 2].view(np.float32)
        return res, mod, arr

    def graphs(self, enable=None) -> int:
        """Turns CUDA-graph round replay on or off (None: leave as is);
        returns the number of graph launches so far."""
        n = ctypes.c_int64(0)
        e = -1 if enable is None else int(bool(enable))
        _check(lib().clean_batch_graphs(self._h, e, ctypes.byref(n)), "clean_batch_graphs")
        return int(n.value)

    def stats(self):
        r, k, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().clean_batch_stats(self._h, ctypes.byref(r), ctypes.byref(k), ctypes.byref(c)),
               "clean_batch_stats")
        return {"rounds_launched": r.value, "kernel_launches": k.value, "n_components": c.value}
