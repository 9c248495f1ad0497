"""Autotuner for tiled CLEAN plans on one GPU.

Two kinds of choices are tuned:

* Launch choices that never change a result bit: CTAs per tile and the
  group barrier of the minor loop (thread-block cluster or bounded grid
  barrier), the minor-loop kernel (plain loads or bulk-copy pipeline, with
  or without tile pairs and tensor-memory chunks) and the feedback kernel
  (plain loads or TMA windows).  Every candidate is timed on the problem itself for a few rounds; the fastest
  wins.
* Choices that change results, only on request: the FFT feedback (within
  tolerance of the exact gather, not bit-exact) with ``allow_fft``, and the
  feedback interval K with ``k_candidates``.  A candidate K is accepted only
  when the restored image of the tiled run stays within the paper's band of
  the untiled run (Section 4: the tiled reconstruction agreed with standard
  Hogbom CLEAN to between -0.1 and +0.04 Jy); the fastest accepted K wins.

Results are cached in a JSON file keyed by the problem's shape, tiling, K
and the GPU's SM count, so a later plan of the same shape skips the search.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import asdict, dataclass, field

from . import (DEBUG_FEEDBACK_PATH, DEBUG_MINOR_PAIR, DEBUG_MINOR_PATH, DEBUG_MINOR_TMEM,
               DEBUG_TIMING, FB_FFT, FB_GATHER, SYNC_AUTO, SYNC_CLUSTER, SYNC_GRID, CleanError,
               Plan)

PAPER_BAND = (-0.1, 0.04)   # restored(tiled) - restored(untiled), Jy


@dataclass
class Choice:
    """One launch configuration of a plan."""
    group_ctas: int = 0
    group_sync: int = SYNC_AUTO
    minor_path: int = 0        # 0 automatic, 1 plain loads, 2 bulk-copy pipeline
    feedback_path: int = 0     # 0 automatic, 1 plain loads, 2 TMA
    feedback_mode: int = FB_GATHER
    minor_pairs: int = 1       # 1 tile pairs where they apply, 0 one group per tile
    minor_tmem: int = 1        # 1 tensor-memory chunks where they apply, 0 none

    def plan_kwargs(self) -> dict:
        return dict(group_ctas=self.group_ctas, group_sync=self.group_sync,
                    feedback_mode=self.feedback_mode)

    def apply_debug(self, plan: Plan):
        if self.minor_path:
            plan.debug_set(DEBUG_MINOR_PATH, self.minor_path)
        if self.feedback_path:
            plan.debug_set(DEBUG_FEEDBACK_PATH, self.feedback_path)
        if not self.minor_pairs:
            plan.debug_set(DEBUG_MINOR_PAIR, 0)
        if not self.minor_tmem:
            plan.debug_set(DEBUG_MINOR_TMEM, 0)


@dataclass
class TuneResult:
    key: str
    choice: Choice
    K: int
    ms_per_round: float
    trials: list = field(default_factory=list)
    k_trials: list = field(default_factory=list)

    def to_json(self) -> dict:
        return asdict(self)

    @staticmethod
    def from_json(d: dict) -> "TuneResult":
        return TuneResult(key=d["key"], choice=Choice(**d["choice"]), K=int(d["K"]),
                          ms_per_round=float(d["ms_per_round"]), trials=d.get("trials", []),
                          k_trials=d.get("k_trials", []))


def problem_key(ny, nx, psf_shape, tiles, K, sm_count, allow_fft=False) -> str:
    return (f"{ny}x{nx}|psf{psf_shape[0]}x{psf_shape[1]}|t{tiles[0]}x{tiles[1]}|K{K}|"
            f"sm{sm_count}|fft{int(bool(allow_fft))}")


def default_cache_path() -> str:
    base = os.environ.get("CLEANGB_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "cleangb", "tune.json")


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(tiles, sm_count: int, allow_fft: bool = False) -> list[Choice]:
    """Launch configurations worth timing for a tile grid on `sm_count` SMs."""
    T = tiles[0] * tiles[1]
    out = [Choice()]  # the library's own choice
    # grid-synchronised groups: every tile gets floor(SMs / T) CTAs, or fewer
    g_max = max(1, sm_count // T)
    for G in sorted({g_max, max(1, g_max // 2)}):
        for mp in (1, 2):
            out.append(Choice(group_ctas=G, group_sync=SYNC_GRID, minor_path=mp))
    # cluster groups (a cluster is at most 16 CTAs)
    for G in (4, 8, 16):
        if G * T <= 4 * sm_count:
            out.append(Choice(group_ctas=G, group_sync=SYNC_CLUSTER))
    out.append(Choice(feedback_path=1))
    # the automatic minor loop without tile pairs, and without TMEM chunks
    out.append(Choice(minor_pairs=0))
    out.append(Choice(minor_tmem=0))
    if allow_fft and T > 1:
        out.append(Choice(feedback_mode=FB_FFT))
    # keep order, drop duplicates
    seen, uniq = set(), []
    for c in out:
        k = tuple(asdict(c).items())
        if k not in seen:
            seen.add(k)
            uniq.append(c)
    return uniq


def _time_choice(choice: Choice, psf, dirty, ny, nx, gain, niter, threshold, tiles, K,
                 rounds: int, trigger: float) -> float:
    """Milliseconds per round of `choice` (device time of the round kernels)."""
    import torch
    with Plan(psf, ny, nx, gain=gain, niter=niter, threshold=threshold, tiles=tiles,
              feedback_interval=K, feedback_trigger=trigger, **choice.plan_kwargs()) as p:
        choice.apply_debug(p)
        p.run(dirty, max_rounds=1)          # warm-up (first launches, tensor maps)
        torch.cuda.synchronize()
        p.debug_set(DEBUG_TIMING, 1)
        p.run(dirty, max_rounds=rounds)
        torch.cuda.synchronize()
        st = p.stats()
    n = max(1, st["minor_launches"])
    return (st["minor_ms"] + st["feedback_ms"]) / n


def tune_launch(psf, dirty, gain, niter, threshold=0.0, tiles=(1, 1), K=0, rounds=3,
                allow_fft=False, trigger=0.0, cache_path: str | None = None,
                use_cache: bool = True, sm_count: int | None = None) -> TuneResult:
    """Times every launch candidate on (psf, dirty) and returns the fastest."""
    import torch
    ny, nx = int(dirty.shape[0]), int(dirty.shape[1])
    if sm_count is None:
        sm_count = torch.cuda.get_device_properties(dirty.device).multi_processor_count
    key = problem_key(ny, nx, tuple(psf.shape), tiles, K, sm_count, allow_fft)
    cache_path = cache_path or default_cache_path()
    cache = load_cache(cache_path) if use_cache else {}
    if key in cache:
        return TuneResult.from_json(cache[key])
    trials = []
    best = None
    for c in candidates(tiles, sm_count, allow_fft):
        try:
            ms = _time_choice(c, psf, dirty, ny, nx, gain, niter, threshold, tiles, K, rounds,
                              trigger)
        except CleanError as e:  # a configuration this problem cannot use
            trials.append({"choice": asdict(c), "error": str(e)})
            continue
        trials.append({"choice": asdict(c), "ms_per_round": ms})
        if best is None or ms < best[1]:
            best = (c, ms)
    if best is None:
        raise RuntimeError("no launch configuration could run this problem")
    res = TuneResult(key=key, choice=best[0], K=K, ms_per_round=best[1], trials=trials)
    if use_cache:
        cache[key] = res.to_json()
        save_cache(cache_path, cache)
    return res


def band_check(psf, dirty, gain, niter, threshold, tiles, K, beam, choice: Choice | None = None,
               untiled_restored=None, band=PAPER_BAND):
    """Runs tiled CLEAN with interval K and untiled CLEAN, restores both with
    `beam` = (bmaj, bmin, bpa) and returns (ok, min diff, max diff, seconds of
    the tiled run, components, untiled restored image)."""
    import torch
    choice = choice or Choice()
    ny, nx = int(dirty.shape[0]), int(dirty.shape[1])
    if untiled_restored is None:
        with Plan(psf, ny, nx, gain=gain, niter=niter, threshold=threshold) as u:
            u.run(dirty)
            untiled_restored = u.restore(*beam)
    with Plan(psf, ny, nx, gain=gain, niter=niter, threshold=threshold, tiles=tiles,
              feedback_interval=K, **choice.plan_kwargs()) as p:
        choice.apply_debug(p)
        p.run(dirty, max_rounds=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.run(dirty)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        n = p.n_components()
        restored = p.restore(*beam)
    diff = (restored - untiled_restored).double()
    lo, hi = float(diff.min()), float(diff.max())
    ok = band[0] <= lo and hi <= band[1]
    return ok, lo, hi, secs, n, untiled_restored


def tune(psf, dirty, gain, niter, threshold=0.0, tiles=(1, 1), K=0, k_candidates=None,
         beam=None, allow_fft=False, rounds=3, cache_path: str | None = None,
         use_cache: bool = True, band=PAPER_BAND) -> TuneResult:
    """Launch tuning at interval K; with `k_candidates` (and the clean beam
    `beam`), also picks the fastest interval whose restored image stays in
    the paper's band of the untiled run."""
    res = tune_launch(psf, dirty, gain, niter, threshold, tiles, K, rounds, allow_fft,
                      cache_path=cache_path, use_cache=use_cache)
    if not k_candidates:
        return res
    if beam is None:
        raise ValueError("k_candidates needs the clean beam (bmaj, bmin, bpa) for the band test")
    k_trials, best, ref = [], None, None
    for Kc in k_candidates:
        ok, lo, hi, secs, n, ref = band_check(psf, dirty, gain, niter, threshold, tiles, int(Kc),
                                              beam, res.choice, ref, band)
        rate = n / secs if secs > 0 else 0.0
        k_trials.append({"K": int(Kc), "in_band": ok, "min_diff": lo, "max_diff": hi,
                         "iters_per_s": rate})
        if ok and (best is None or rate > best[1]):
            best = (int(Kc), rate)
    res.k_trials = k_trials
    if best is not None:
        res.K = best[0]
    return res


def tuned_plan(result: TuneResult, psf, ny, nx, gain, niter, threshold=0.0, tiles=(1, 1),
               stream=None, trigger=0.0) -> Plan:
    """A Plan configured with a tuning result."""
    p = Plan(psf, ny, nx, gain=gain, niter=niter, threshold=threshold, tiles=tiles,
             feedback_interval=result.K, stream=stream, feedback_trigger=trigger,
             **result.choice.plan_kwargs())
    result.choice.apply_debug(p)
    return p


__all__ = ["Choice", "TuneResult", "PAPER_BAND", "candidates", "problem_key", "tune",
           "tune_launch", "band_check", "tuned_plan", "load_cache", "save_cache",
           "default_cache_path"]
