"""Continuous-batching deconvolution server on one GPU.

Jobs (dirty image, PSF, CLEAN parameters) arrive over time.  A job is
admitted as soon as it has arrived and its device footprint fits under the
memory budget; admitted jobs stay resident on the device and run together,
round by round, in shared launches (clean_server_* in libcleangb.so), so a
job that arrives while others are running starts at the next step and its
work overlaps with theirs.  Finished jobs hand back their results and free
their memory, which admits the next ones.  Each job's results are identical
to its solo run: batching only changes which CTA serves which tile.

The scheduling loop is host code; every step of the method runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import (COMPONENT_DTYPE, FB_FFT, FB_GATHER, CleanError, _check, _dptr, _stream_ptr,
               lib, make_params)


def _fft_size(m: int) -> int:
    """The FFT feedback's grid length for 2 n - 1: the smallest even number
    >= m whose prime factors are 2, 3, 5 and 7 (as the library picks it)."""
    n = max(m, 2)
    while True:
        r = n
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        if r == 1 and n % 2 == 0:
            return n
        n += 1


def _twiddles(L: int) -> int:
    """Entries of an FFT axis's twiddle table (L, plus r Ns per stage)."""
    out, ns = L, 1
    for f in (8, 4, 2, 3, 5, 7):
        while L % f == 0:
            out += f * ns
            ns *= f
            L //= f
    return out


def footprint_bytes(n: int, psf_shape, niter: int, tiles=(1, 1), K: int = 0,
                    feedback_mode: int = FB_GATHER) -> int:
    """Device bytes a job holds while resident: residual and model images,
    its PSF (held by the caller but pinned for the job's lifetime), the
    component list and the round buffer, and with FFT feedback the kernel
    spectrum, the transforms' work areas and the round-start residual."""
    T = tiles[0] * tiles[1]
    per_tile = niter // T + (1 if niter % T else 0)
    cap = min(K, per_tile) if K > 0 else per_tile
    b = (8 * n * n + 4 * psf_shape[0] * psf_shape[1] + 16 * niter + 16 * T * max(cap, 1)
         + 8 * niter + 4096)
    if feedback_mode == FB_FFT and T > 1:
        L = _fft_size(2 * n - 1)
        # kernel spectrum, the round's column work area, the component list,
        # twiddle tables and the round-start residual
        b += 8 * L * (L // 2 + 1) + 8 * (n + n % 2) * (L // 2 + 1) + 24 * T * max(cap, 1) + 16 \
            + 2 * 8 * _twiddles(L) + 4 * n * n
    return int(b)


@dataclass
class Job:
    """A deconvolution request.  psf and dirty are CUDA float32 tensors."""
    psf: object
    dirty: object
    gain: float = 0.1
    niter: int = 1000
    threshold: float = 0.0
    tiles: tuple = (1, 1)
    feedback_interval: int = 50
    feedback_mode: int = FB_GATHER  # FB_FFT: feedback by FFT convolution (within tolerance)
    arrival: float = 0.0           # seconds after the start of serve()
    tag: object = None
    # filled by the server
    admitted: float = field(default=None)
    finished: float = field(default=None)
    result: tuple = field(default=None)

    @property
    def n(self):
        return int(self.dirty.shape[0])

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival

    def footprint(self):
        return footprint_bytes(self.n, tuple(self.psf.shape), self.niter, self.tiles,
                               self.feedback_interval, self.feedback_mode)


class Server:
    """Thin wrapper of clean_server_* (one device, one stream)."""

    def __init__(self, max_jobs: int = 256, stream=None):
        self._h = ctypes.c_void_p()
        self._stream = stream
        _check(lib().clean_server_create(ctypes.byref(self._h), int(max_jobs),
                                         _stream_ptr(stream)), "clean_server_create")

    def close(self):
        if self._h:
            lib().clean_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, job: Job) -> int:
        ny, nx = job.dirty.shape
        p = make_params(ny, nx, tuple(job.psf.shape), gain=job.gain, niter=job.niter,
                        threshold=job.threshold, tiles=job.tiles,
                        feedback_interval=job.feedback_interval,
                        feedback_mode=job.feedback_mode)
        jid = ctypes.c_int64(0)
        _check(lib().clean_server_add(self._h, ctypes.byref(p), _dptr(job.psf, what="psf"),
                                      _dptr(job.dirty, what="dirty"), ctypes.byref(jid),
                                      _stream_ptr(self._stream)), "clean_server_add")
        return int(jid.value)

    def step(self, rounds: int = 2) -> int:
        n = ctypes.c_int32(0)
        _check(lib().clean_server_step(self._h, int(rounds), ctypes.byref(n),
                                       _stream_ptr(self._stream)), "clean_server_step")
        return int(n.value)

    def done(self) -> list:
        n = ctypes.c_int32(0)
        _check(lib().clean_server_done(self._h, None, 0, ctypes.byref(n)), "clean_server_done")
        ids = (ctypes.c_int64 * max(n.value, 1))()
        _check(lib().clean_server_done(self._h, ids, n.value, ctypes.byref(n)), "clean_server_done")
        return [int(ids[i]) for i in range(n.value)]

    def get(self, jid: int, shape):
        import torch
        n = ctypes.c_int64(0)
        _check(lib().clean_server_get(self._h, jid, None, None, None, 0, ctypes.byref(n),
                                      _stream_ptr(self._stream)), "clean_server_get")
        res = torch.empty(shape, dtype=torch.float32, device="cuda")
        mod = torch.empty_like(res)
        comps = torch.empty((max(n.value, 1), 4), dtype=torch.int32, device="cuda")
        _check(lib().clean_server_get(self._h, jid, _dptr(res), _dptr(mod),
                                      ctypes.c_void_p(comps.data_ptr()), n.value, ctypes.byref(n),
                                      _stream_ptr(self._stream)), "clean_server_get")
        host = comps[:n.value].cpu().numpy()
        arr = np.empty(n.value, dtype=COMPONENT_DTYPE)
        arr["y"], arr["x"], arr["tile"] = host[:, 0], host[:, 1], host[:, 3]
        arr["flux"] = host[:, 2].view(np.float32)
        return res, mod, arr

    def remove(self, jid: int):
        _check(lib().clean_server_remove(self._h, jid), "clean_server_remove")


def serve(jobs: list, budget_bytes: float = 150e9, rounds_per_step: int = 2,
          keep_results: bool = True, max_jobs: int = 256, clock=time.perf_counter) -> dict:
    """Runs `jobs` (each with an arrival time in seconds) through a
    continuous-batching server in real time.  Returns latency statistics;
    each job gets admitted / finished times (seconds from the start) and, if
    keep_results, its (residual, model, components)."""
    srv = Server(max_jobs=max_jobs)
    order = sorted(range(len(jobs)), key=lambda i: jobs[i].arrival)
    queue = [jobs[i] for i in order]
    resident = {}
    used = 0
    t0 = clock()
    try:
        while queue or resident:
            now = clock() - t0
            while queue and queue[0].arrival <= now and \
                    (used + queue[0].footprint() <= budget_bytes or not resident) and \
                    len(resident) < max_jobs:
                job = queue.pop(0)
                jid = srv.add(job)
                job.admitted = clock() - t0
                resident[jid] = job
                used += job.footprint()
            if not resident:
                wait = queue[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
                continue
            srv.step(rounds_per_step)
            for jid in srv.done():
                job = resident.pop(jid)
                job.finished = clock() - t0
                if keep_results:
                    job.result = srv.get(jid, tuple(job.dirty.shape))
                srv.remove(jid)
                used -= job.footprint()
    finally:
        srv.close()
    lat = np.array([j.latency for j in jobs])
    span = max(j.finished for j in jobs) - min(j.arrival for j in jobs)
    return {"jobs": len(jobs), "makespan_s": span, "jobs_per_s": len(jobs) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}


def serve_one_at_a_time(jobs: list, run_job, clock=time.perf_counter) -> dict:
    """The baseline server: jobs run one at a time in arrival order, in real
    time (an idle server waits for the next arrival); run_job(job) runs one
    job to completion and returns when its results are on the host side of
    the stream (synchronised).  Fills each job's admitted / finished times and
    returns latency statistics as serve() does."""
    order = sorted(range(len(jobs)), key=lambda i: jobs[i].arrival)
    t0 = clock()
    for i in order:
        job = jobs[i]
        while clock() - t0 < job.arrival:
            time.sleep(min(job.arrival - (clock() - t0), 0.01))
        job.admitted = clock() - t0
        run_job(job)
        job.finished = clock() - t0
    lat = np.array([j.latency for j in jobs])
    span = max(j.finished for j in jobs) - min(j.arrival for j in jobs)
    return {"jobs": len(jobs), "makespan_s": span, "jobs_per_s": len(jobs) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}


def fifo_latencies(arrivals, service_s) -> np.ndarray:
    """Latencies of a one-at-a-time FIFO server with the given service times."""
    t = 0.0
    out = []
    for a, s in sorted(zip(arrivals, service_s)):
        t = max(t, a) + s
        out.append(t - a)
    return np.array(out)
