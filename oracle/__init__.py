"""CPU oracle for tiled Hogbom CLEAN with feedback (arXiv 2501.01461).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the benchmark's CPU-baseline legs import this module.  The product (the CUDA
library and its Python binding) never imports, links or calls it, and the two
share no code: they share only the seeded inputs from ``synth``.

Contents
  clean_f32     plain single-threaded C, float32, every multiply and subtract
                rounded separately (built with -ffp-contract=off)
  clean_f64     the same algorithm in float64, run independently or as a
                replay of a float32 component list (positions, tiles and
                rounds forced, fluxes and residuals computed in float64)
  brute_clean   literal NumPy restatement for tiny images: full-image
                shifted-PSF images for every subtraction and an explicit
                per-tile cross-coupling image for feedback
  restore       model image convolved with a Gaussian clean beam plus the
                residual, float64 NumPy
  psf_convolve  model image convolved with the PSF (float64 FFT), used to
                check residual + model * PSF = dirty
  parallel_clean_f32
                multi-core CPU baseline (clean_parallel.c, OpenMP over the
                tiles of a round), equal to clean_f32 bit for bit; timed by
                the benchmark beside the single-threaded oracle

Paper passages (Section 3): a component is the peak residual times the gain
(first equation); the residual loses gain x peak x PSF shifted to the peak
(second equation); a tile's components placed on a full-size image and
convolved with the full PSF give its cross-coupling image, which is
subtracted from the other tiles at regular intervals (feedback).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no GPU needed).  Returns the .so path."""
    src = [os.path.join(_HERE, "clean_oracle.c")]
    deps = src + [os.path.join(_HERE, "clean_oracle_body.h")]
    if not force and os.path.exists(_SO) and all(
            os.path.getmtime(_SO) >= os.path.getmtime(d) for d in deps):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cc = os.environ.get("CC", "gcc")
    subprocess.run([cc, *CFLAGS, "-o", tmp, *src], check=True)
    os.replace(tmp, _SO)
    return _SO


_PAR_SO = os.path.join(_HERE, "_build", "liboracle_parallel.so")
_par_lib = None


def build_parallel(force: bool = False) -> str:
    """Compile the multi-core CPU baseline (OpenMP) with gcc."""
    src = os.path.join(_HERE, "clean_parallel.c")
    if not force and os.path.exists(_PAR_SO) and os.path.getmtime(_PAR_SO) >= os.path.getmtime(src):
        return _PAR_SO
    os.makedirs(os.path.dirname(_PAR_SO), exist_ok=True)
    tmp = _PAR_SO + f".{os.getpid()}.tmp"
    cc = os.environ.get("CC", "gcc")
    subprocess.run([cc, *CFLAGS, "-fopenmp", "-o", tmp, src], check=True)
    os.replace(tmp, _PAR_SO)
    return _PAR_SO


def _load_parallel():
    global _par_lib
    with _lock:
        if _par_lib is None:
            lib = ctypes.CDLL(build_parallel())
            i32, i64, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.parallel_clean_f32.restype = i64
            lib.parallel_clean_f32.argtypes = [vp, i32, i32, vp, i32, i32, f64, i64, f64, i32,
                                               i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, i64,
                                               vp]
            lib.parallel_threads.restype = ctypes.c_int
            lib.parallel_threads.argtypes = [ctypes.c_int]
            _par_lib = lib
    return _par_lib


def parallel_threads(n: int = 0) -> int:
    """Sets the multi-core baseline's OpenMP thread count (n > 0) and returns it."""
    return int(_load_parallel().parallel_threads(int(n)))


def parallel_clean_f32(dirty, psf, gain, niter, threshold=0.0, tiles=(1, 1), K=0,
                       max_rounds=-1) -> Result:
    """Multi-core CPU baseline (clean_parallel.c): the float32 oracle's
    arithmetic with the tiles of a round on OpenMP threads; equal to
    clean_f32 bit for bit (no flux trigger)."""
    lib = _load_parallel()
    dirty = np.ascontiguousarray(dirty, dtype=np.float32)
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    ny, nx = dirty.shape
    pny, pnx = psf.shape
    cap = max(int(niter), 1)
    res = np.empty((ny, nx), np.float32)
    model = np.empty((ny, nx), np.float32)
    oy = np.empty(cap, np.int32); ox = np.empty(cap, np.int32)
    of = np.empty(cap, np.float32); ot = np.empty(cap, np.int32); orr = np.empty(cap, np.int32)
    rounds = ctypes.c_int32(0)
    n = lib.parallel_clean_f32(_ptr(dirty), ny, nx, _ptr(psf), pny, pnx, _f32(gain), int(niter),
                               _f32(threshold), tiles[0], tiles[1], int(K), int(max_rounds),
                               _ptr(res), _ptr(model), _ptr(oy), _ptr(ox), _ptr(of), _ptr(ot),
                               _ptr(orr), cap, ctypes.byref(rounds))
    if n < 0:
        raise ValueError({-1: "invalid arguments", -2: "out of memory",
                          -3: "component capacity exceeded"}.get(n, str(n)))
    comps = dict(y=oy[:n].copy(), x=ox[:n].copy(), flux=of[:n].copy(),
                 tile=ot[:n].copy(), round=orr[:n].copy())
    return Result(residual=res, model=model, comps=comps, rounds=rounds.value, n=int(n))


def load_library(path: str):
    """ctypes handle of an oracle shared library at `path` (signatures set)."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _declare(lib):
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_clean_f32.restype = i64
    lib.oracle_clean_f32.argtypes = [vp, i32, i32, vp, i32, i32, f64, i64,
                                     f64, i32, i32, i32, f64, i32, vp, vp, vp,
                                     vp, vp, vp, vp, i64, vp]
    lib.oracle_clean_f64.restype = i64
    lib.oracle_clean_f64.argtypes = [vp, i32, i32, vp, i32, i32, f64, i64,
                                     f64, i32, i32, i32, f64, i32, vp, vp, vp,
                                     vp, i64, vp, vp, vp, vp, vp, vp, vp,
                                     i64, vp]


def _ptr(a):
    return None if a is None else a.ctypes.data


class Result(dict):
    """residual, model, comps (dict of arrays y, x, flux, tile, round), rounds."""
    __getattr__ = dict.__getitem__


def _f32(v: float) -> float:
    # gain and threshold are float32 parameters of the problem
    return float(np.float32(v))


def clean_f32(dirty, psf, gain, niter, threshold=0.0, tiles=(1, 1), K=0,
              max_rounds=-1, trigger=0.0) -> Result:
    """Float32 oracle.  tiles=(1,1), K=0 is plain (untiled) Hogbom CLEAN.
    trigger in (0, 1): flux-triggered rounds (see clean_oracle.c)."""
    return _run(np.float32, dirty, psf, gain, niter, threshold, tiles, K,
                max_rounds, None, trigger)


def clean_f64(dirty, psf, gain, niter, threshold=0.0, tiles=(1, 1), K=0,
              max_rounds=-1, replay=None, trigger=0.0) -> Result:
    """Float64 twin.  ``replay`` = a component dict (y, x, tile, round) from a
    float32 run: positions and round structure are forced from it."""
    return _run(np.float64, dirty, psf, gain, niter, threshold, tiles, K,
                max_rounds, replay, trigger)


def _run(dtype, dirty, psf, gain, niter, threshold, tiles, K, max_rounds,
         replay, trigger=0.0, lib=None):
    lib = lib or _load()
    dirty = np.ascontiguousarray(dirty, dtype=np.float32)
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    ny, nx = dirty.shape
    pny, pnx = psf.shape
    ty, tx = tiles
    cap = int(niter) if replay is None else len(replay["y"])
    cap = max(cap, 1)
    res = np.empty((ny, nx), dtype=dtype)
    model = np.empty((ny, nx), dtype=dtype)
    oy = np.empty(cap, np.int32); ox = np.empty(cap, np.int32)
    of = np.empty(cap, dtype); ot = np.empty(cap, np.int32); orr = np.empty(cap, np.int32)
    rounds = ctypes.c_int32(0)
    if dtype == np.float32:
        n = lib.oracle_clean_f32(_ptr(dirty), ny, nx, _ptr(psf), pny, pnx,
                                 _f32(gain), int(niter), _f32(threshold), ty, tx,
                                 int(K), _f32(trigger), int(max_rounds), _ptr(res), _ptr(model),
                                 _ptr(oy), _ptr(ox), _ptr(of), _ptr(ot), _ptr(orr),
                                 cap, ctypes.byref(rounds))
    else:
        if replay is not None:
            ry = np.ascontiguousarray(replay["y"], np.int32)
            rx = np.ascontiguousarray(replay["x"], np.int32)
            rt = np.ascontiguousarray(replay["tile"], np.int32)
            rr = np.ascontiguousarray(replay["round"], np.int32)
            rn = len(ry)
        else:
            ry = rx = rt = rr = None
            rn = -1
        n = lib.oracle_clean_f64(_ptr(dirty), ny, nx, _ptr(psf), pny, pnx,
                                 _f32(gain), int(niter), _f32(threshold), ty, tx,
                                 int(K), _f32(trigger), int(max_rounds), _ptr(ry), _ptr(rx),
                                 _ptr(rt), _ptr(rr), rn, _ptr(res), _ptr(model),
                                 _ptr(oy), _ptr(ox), _ptr(of), _ptr(ot), _ptr(orr),
                                 cap, ctypes.byref(rounds))
    if n < 0:
        raise ValueError({-1: "invalid arguments", -2: "out of memory",
                          -3: "component capacity exceeded"}.get(n, str(n)))
    comps = dict(y=oy[:n].copy(), x=ox[:n].copy(), flux=of[:n].copy(),
                 tile=ot[:n].copy(), round=orr[:n].copy())
    return Result(residual=res, model=model, comps=comps, rounds=rounds.value,
                  n=int(n))


# ---------------------------------------------------------------------------
# Literal restatement for tiny images (NumPy, per-op rounding in ``dtype``)
# ---------------------------------------------------------------------------

def _shifted_psf(psf, ny, nx, py, px, dtype):
    """Full-size image whose pixel q holds P[q - p + c] (0 where off the PSF)."""
    pny, pnx = psf.shape
    cy, cx = pny // 2, pnx // 2
    out = np.zeros((ny, nx), dtype=dtype)
    present = np.zeros((ny, nx), dtype=bool)
    for y in range(ny):
        sy = y - py + cy
        if not 0 <= sy < pny:
            continue
        for x in range(nx):
            sx = x - px + cx
            if 0 <= sx < pnx:
                out[y, x] = psf[sy, sx]
                present[y, x] = True
    return out, present


def brute_clean(dirty, psf, gain, niter, threshold=0.0, tiles=(1, 1), K=0,
                dtype=np.float32, max_rounds=-1, trigger=0.0):
    """Literal CLEAN for tiny images, independent of the C oracle.

    Each subtraction builds the full shifted PSF image and applies
    R <- R - f * S on the tile's mask; feedback builds, for every tile, the
    list of its new components and subtracts each one's shifted PSF image
    from the pixels of the other tiles, tile by tile in index order.  Peaks
    are found with numpy.argmax on |R| over the tile (first occurrence,
    i.e. the lowest row-major index).  Arithmetic is in ``dtype`` with each
    operation rounded (NumPy scalar/array ops do not fuse).
    """
    dt = np.dtype(dtype).type
    R = np.asarray(dirty, dtype=np.float32).astype(dtype)
    P = np.asarray(psf, dtype=np.float32).astype(dtype)
    ny, nx = R.shape
    ty, tx = tiles
    T = ty * tx
    g, thr = dt(np.float32(gain)), dt(np.float32(threshold))
    trig = dt(np.float32(trigger))
    feedback = (K > 0 or trigger > 0) and ty * tx > 1
    masks = []
    for t in range(T):
        i, j = divmod(t, tx)
        m = np.zeros((ny, nx), dtype=bool)
        m[(i * ny) // ty:((i + 1) * ny) // ty, (j * nx) // tx:((j + 1) * nx) // tx] = True
        masks.append(m)
    budget = [niter // T + (1 if t < niter % T else 0) for t in range(T)]
    comps = []
    rnd = 0

    def peak(t):
        a = np.where(masks[t], np.abs(R), dt(-1))
        p = int(np.argmax(a))
        return p, R.flat[p]

    while max_rounds < 0 or rnd < max_rounds:
        active = [budget[t] > 0 and abs(peak(t)[1]) > thr for t in range(T)]
        if not any(active):
            break
        new = []
        # flux trigger: the round ends for a tile at trigger x the largest
        # |peak| among the tiles taking part in the round
        top = max([abs(peak(t)[1]) for t in range(T) if active[t]], default=dt(0))
        level = dt(trig * top) if trigger > 0 else dt(0)
        for t in range(T):
            if not active[t]:
                continue
            kmax = budget[t] if K == 0 else min(K, budget[t])
            for _ in range(kmax):
                p, v = peak(t)
                if abs(v) <= thr or abs(v) <= level:
                    break
                f = dt(g * v)
                py, px = divmod(p, nx)
                S, present = _shifted_psf(P, ny, nx, py, px, dtype)
                upd = masks[t] & present
                R[upd] = (R - f * S)[upd]
                comps.append((py, px, f, t, rnd))
                new.append((py, px, f, t))
                budget[t] -= 1
        if feedback:
            # cross-coupling: tile s's components placed on a full-size image
            # and spread by the full PSF, applied to every other tile; per
            # pixel the components are applied in list order
            for (py, px, f, s) in new:
                S, present = _shifted_psf(P, ny, nx, py, px, dtype)
                upd = (~masks[s]) & present
                R[upd] = (R - f * S)[upd]
        rnd += 1
    model = np.zeros((ny, nx), dtype=dtype)
    for (py, px, f, t, r) in comps:
        model[py, px] = dt(model[py, px] + f)
    arr = dict(y=np.array([c[0] for c in comps], np.int32),
               x=np.array([c[1] for c in comps], np.int32),
               flux=np.array([c[2] for c in comps], dtype),
               tile=np.array([c[3] for c in comps], np.int32),
               round=np.array([c[4] for c in comps], np.int32))
    return Result(residual=R, model=model, comps=arr, rounds=rnd, n=len(comps))


# ---------------------------------------------------------------------------
# Convolutions used by the checks (float64)
# ---------------------------------------------------------------------------

def psf_convolve(model, psf):
    """(model * PSF)[q] = sum_p model[p] P[q - p + c], float64, image-sized.

    Evaluated with an FFT of size (ny + pny - 1) x (nx + pnx - 1), so no
    circular wrap-around occurs.
    """
    import scipy.signal
    model = np.asarray(model, dtype=np.float64)
    psf = np.asarray(psf, dtype=np.float64)
    ny, nx = model.shape
    pny, pnx = psf.shape
    full = scipy.signal.fftconvolve(model, psf, mode="full")
    # full[k] = sum_p model[p] psf[k - p]; psf index q - p + c  =>  k = q + c
    cy, cx = pny // 2, pnx // 2
    return full[cy:cy + ny, cx:cx + nx]


def gaussian_beam(bmaj, bmin, bpa, dy, dx):
    """Clean-beam value at offset (dy, dx): peak 1, FWHM bmaj/bmin pixels,
    major axis at angle bpa from +x toward +y."""
    k = 1.0 / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    smaj, smin = bmaj * k, bmin * k
    c, s = np.cos(bpa), np.sin(bpa)
    u = dx * c + dy * s          # along the major axis
    w = -dx * s + dy * c         # along the minor axis
    return np.exp(-0.5 * ((u / smaj) ** 2 + (w / smin) ** 2))


def restore(model, residual, bmaj, bmin, bpa):
    """Restored image = model convolved with the clean beam (truncated at
    5 sigma of the major axis, i.e. offsets with |dy|, |dx| <= r and
    dy^2 + dx^2 <= r^2, r = floor(5 sigma_maj)) plus the residual, float64."""
    model = np.asarray(model, dtype=np.float64)
    out = np.asarray(residual, dtype=np.float64).copy()
    ny, nx = model.shape
    smaj = bmaj / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    r = int(np.floor(5.0 * smaj))
    ys, xs = np.nonzero(model)
    for y, x in zip(ys, xs):
        y0, y1 = max(0, y - r), min(ny, y + r + 1)
        x0, x1 = max(0, x - r), min(nx, x + r + 1)
        dy = np.arange(y0, y1)[:, None] - y
        dx = np.arange(x0, x1)[None, :] - x
        b = gaussian_beam(bmaj, bmin, bpa, dy.astype(np.float64), dx.astype(np.float64))
        b = np.where(dy * dy + dx * dx <= r * r, b, 0.0)
        out[y0:y1, x0:x1] += model[y, x] * b
    return out
