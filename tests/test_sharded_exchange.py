"""Tile sharding across ranks (CPU, gloo, world size 2).

Tiles are independent within a round; the only exchange tiled CLEAN with
feedback needs is the round's component list (Section 3: each tile's new
components, placed on the full image and convolved with the full PSF, are
subtracted from the other tiles).  Here each rank runs the minor loops of its
own tiles (float32, one rounding per multiply and per subtract), the ranks
all-gather the round's components, and each rank applies the other tiles'
components to its own tiles in list order.  The gathered result must equal
the single-process oracle bit for bit.
"""
import os
import tempfile

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _tile(t, ny, nx, ty, tx):
    i, j = divmod(t, tx)
    return (i * ny) // ty, ((i + 1) * ny) // ty, (j * nx) // tx, ((j + 1) * nx) // tx


def _subtract(R, P, py, px, f, y0, y1, x0, x1):
    pny, pnx = P.shape
    cy, cx = pny // 2, pnx // 2
    for y in range(y0, y1):
        sy = y - py + cy
        if not 0 <= sy < pny:
            continue
        xs = np.arange(x0, x1)
        sx = xs - px + cx
        ok = (sx >= 0) & (sx < pnx)
        row = R[y, xs[ok]]
        R[y, xs[ok]] = row - np.float32(f) * P[sy, sx[ok]]


def _shard_worker(rank, world, path, dirty, psf, gain, niter, thr, tiles, K, out):
    dist.init_process_group("gloo", init_method=f"file://{path}", rank=rank, world_size=world)
    ny, nx = dirty.shape
    ty, tx = tiles
    T = ty * tx
    mine = [t for t in range(T) if t % world == rank]
    R = dirty.astype(np.float32).copy()
    P = psf.astype(np.float32)
    g, th = np.float32(gain), np.float32(thr)
    budget = {t: niter // T + (1 if t < niter % T else 0) for t in range(T)}
    comps = []
    rnd = 0
    while True:
        # which of my tiles can run; the decision is shared by all ranks
        act = {}
        for t in mine:
            y0, y1, x0, x1 = _tile(t, ny, nx, ty, tx)
            a = np.abs(R[y0:y1, x0:x1])
            act[t] = budget[t] > 0 and a.max() > th
        flags = [None] * world
        dist.all_gather_object(flags, act)
        if not any(v for d in flags for v in d.values()):
            break
        new = []
        for t in mine:
            if not act[t]:
                continue
            y0, y1, x0, x1 = _tile(t, ny, nx, ty, tx)
            kmax = budget[t] if K == 0 else min(K, budget[t])
            for _ in range(kmax):
                sub = R[y0:y1, x0:x1]
                p = int(np.argmax(np.abs(sub)))
                py, px = y0 + p // (x1 - x0), x0 + p % (x1 - x0)
                v = R[py, px]
                if abs(v) <= th:
                    break
                f = np.float32(g * v)
                new.append((t, len(new), py, px, f))
                budget[t] -= 1
                _subtract(R, P, py, px, f, y0, y1, x0, x1)
        gathered = [None] * world
        dist.all_gather_object(gathered, new)
        round_list = sorted((c for part in gathered for c in part), key=lambda c: (c[0], c[1]))
        budgets = [None] * world
        dist.all_gather_object(budgets, {t: budget[t] for t in mine})
        for d in budgets:
            budget.update(d)
        if K > 0 and T > 1:
            for (s, _, py, px, f) in round_list:
                for t in mine:
                    if t != s:
                        _subtract(R, P, py, px, f, *_tile(t, ny, nx, ty, tx))
        comps += [(py, px, f, s, rnd) for (s, _, py, px, f) in round_list]
        rnd += 1
    parts = [None] * world
    dist.all_gather_object(parts, {t: R[slice(*_tile(t, ny, nx, ty, tx)[:2]),
                                        slice(*_tile(t, ny, nx, ty, tx)[2:])].copy() for t in mine})
    if rank == 0:
        full = np.zeros_like(R)
        for d in parts:
            for t, blk in d.items():
                y0, y1, x0, x1 = _tile(t, ny, nx, ty, tx)
                full[y0:y1, x0:x1] = blk
        np.save(out + "_res.npy", full)
        np.save(out + "_comps.npy", np.array([(c[0], c[1], c[3], c[4]) for c in comps], np.int64))
        np.save(out + "_flux.npy", np.array([c[2] for c in comps], np.float32))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("tiles,K", [((2, 2), 3), ((3, 2), 1), ((2, 2), 0)])
def test_two_ranks_equal_single_process_oracle(tiles, K):
    rng = np.random.default_rng(21)
    n = 24
    psf = synth.make_psf(2 * n, 2 * n)
    ys, xs, fl = synth.make_sky(n, 6, 0.05, 2.1, rng)
    dirty = synth.make_dirty(psf, n, ys, xs, fl, 1e-3, rng)
    ref = oracle.clean_f32(dirty, psf, 0.1, 200, 1e-3, tiles, K)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "res")
        mp.start_processes(_shard_worker, args=(2, os.path.join(d, "store"), dirty, psf, 0.1, 200,
                                                1e-3, tiles, K, out),
                           nprocs=2, join=True, start_method="spawn")
        res = np.load(out + "_res.npy")
        comps = np.load(out + "_comps.npy")
        flux = np.load(out + "_flux.npy")
    assert np.array_equal(res, ref.residual)
    assert len(flux) == ref.n
    assert np.array_equal(comps[:, 0], ref.comps["y"]) and np.array_equal(comps[:, 1], ref.comps["x"])
    assert np.array_equal(comps[:, 2], ref.comps["tile"]) and np.array_equal(comps[:, 3], ref.comps["round"])
    assert np.array_equal(flux.view(np.uint32), ref.comps["flux"].view(np.uint32))
