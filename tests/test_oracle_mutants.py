"""The pins are strong enough: plant a plausible mistake in a copy of the
oracle (on the CPU, in a temporary directory), rebuild it, and check that the
hand-derived worked examples, the brute-force restatement or the
point-source closed form catch every one."""
import json
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

# Every round of a correct run cleans at least one component, so no case
# below needs more rounds than iterations; the bound stops a mutant that
# loops without progress.
MAX_ROUNDS = 64

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, file, original text, mutated text)
MUTANTS = [
    ("signed peak search", "clean_oracle_body.h",
     "REAL a = FN(absr)(R[(int64_t)y * nx + x]);", "REAL a = R[(int64_t)y * nx + x];"),
    ("ties to the highest index", "clean_oracle_body.h",
     "if (best < 0 || a > bv) {", "if (best < 0 || a >= bv) {"),
    ("PSF centre off by one", "clean_oracle_body.h",
     "int32_t cy = pny / 2, cx = pnx / 2;", "int32_t cy = (pny - 1) / 2, cx = pnx / 2;"),
    ("transposed PSF index", "clean_oracle_body.h",
     "REAL t = f * P[(int64_t)sy * pnx + sx];", "REAL t = f * P[(int64_t)sx * pnx + sy];"),
    ("added instead of subtracted", "clean_oracle_body.h",
     "*r = *r - t;", "*r = *r + t;"),
    ("feedback includes the own tile", "clean_oracle_body.h",
     "if (t == out_tile[c]) continue;", "(void)0;"),
    ("no feedback", "clean_oracle_body.h",
     "    if (feedback) {", "    if (0) {"),
    ("budget remainder to the last tiles", "clean_oracle_body.h",
     "budget[t] = niter / T + (t < niter % T ? 1 : 0);",
     "budget[t] = niter / T + (t >= T - niter % T ? 1 : 0);"),
    ("threshold compared strictly", "clean_oracle_body.h",
     "if (FN(absr)(v) <= thr || FN(absr)(v) <= level) break;",
     "if (FN(absr)(v) < thr || FN(absr)(v) <= level) break;"),
    ("tile bounds rounded up", "clean_oracle_body.h",
     "*y1 = (int32_t)(((int64_t)(i + 1) * ny) / ty);",
     "*y1 = (int32_t)(((int64_t)(i + 1) * ny + ty - 1) / ty);"),
    ("gain left out", "clean_oracle_body.h",
     "          REAL f = g * v;                            /* first equation */",
     "          REAL f = v;"),
    ("model not accumulated", "clean_oracle_body.h",
     "*m = *m + out_f[c];", "*m = out_f[c];"),
    ("trigger level from all tiles", "clean_oracle_body.h",
     "          if (!active[t]) continue;\n          int32_t y0, y1, x0, x1;\n          FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);\n          REAL a =",
     "          int32_t y0, y1, x0, x1;\n          FN(tile_bounds)(t, ny, nx, ty, tx, &y0, &y1, &x0, &x1);\n          REAL a ="),
]


def _golden():
    g = json.load(open(os.path.join(HERE, "golden", "worked_examples.json")))
    psf = np.zeros(g["psf"]["shape"], np.float32)
    for y, x, v in g["psf"]["nonzero"]:
        psf[y, x] = v
    return g, psf, np.array(g["dirty"], np.float32)


def _killed(lib) -> bool:
    run = lambda *a, **k: oracle._run(np.float32, *a, lib=lib, **k)
    try:
        g, psf, dirty = _golden()
        for c in g["cases"]:
            r = run(dirty, psf, c["gain"], c["niter"], c["threshold"], tuple(c["tiles"]), c["K"],
                    MAX_ROUNDS, None, c.get("trigger", 0.0))
            rows = [[int(r.comps["y"][i]), int(r.comps["x"][i]), float(r.comps["flux"][i]),
                     int(r.comps["tile"][i]), int(r.comps["round"][i])] for i in range(r.n)]
            if rows != c["components"] or not np.array_equal(r.residual, np.array(c["residual"])):
                return True
        rng = np.random.default_rng(31)
        for tiles, K, thr, tie, trig, shape in (((2, 3), 2, 1.0, True, 0.0, (16, 16)),
                                                ((4, 4), 3, 0.05, False, 0.0, (16, 13)),
                                                ((2, 2), 0, 0.0, False, 0.6, (13, 16)),
                                                ((3, 2), 1, 0.0, True, 0.0, (14, 16))):
            ny, nx = shape
            psf = synth.random_psf(2 * ny + 1, 2 * nx, rng)
            dirty = synth.tie_image(ny, nx, rng) if tie else synth.random_image(ny, nx, rng)
            a = run(dirty, psf, 0.3, 37, thr, tiles, K, MAX_ROUNDS, None, trig)
            b = oracle.brute_clean(dirty, psf, 0.3, 37, thr, tiles, K, trigger=trig)
            if a.n != b.n or not np.array_equal(a.residual, b.residual) or \
                    not np.array_equal(a.model, b.model) or \
                    not all(np.array_equal(a.comps[k], b.comps[k]) for k in ("y", "x", "flux", "tile")):
                return True
        # point source: peak residual S (1 - g)^n
        n = 24
        psf = synth.make_psf(2 * n, 2 * n)
        d = synth.make_dirty(psf, n, np.array([9]), np.array([14]), np.array([2.0]), 0.0, 0)
        r = run(d, psf, 0.1, 30, 0.0, (1, 1), 0, -1, None, 0.0)
        g32 = float(np.float32(0.1))
        if abs(float(r.residual[9, 14]) - 2.0 * (1 - g32) ** 30) > 30 * 2.0 ** -23 * 2:
            return True
    except Exception:
        return True
    return False


def _build_mutant(tmp, name, fname, old, new):
    src = os.path.join(tmp, "src")
    shutil.copytree(ORACLE_DIR, src, ignore=shutil.ignore_patterns("_build", "__pycache__", "*.py"))
    path = os.path.join(src, fname)
    text = open(path).read()
    assert text.count(old) == 1, f"mutation site for '{name}' not unique"
    open(path, "w").write(text.replace(old, new))
    so = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", so, os.path.join(src, "clean_oracle.c")],
                   check=True)
    return so


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(tmp, "none", "clean_oracle.c", "#include <stdint.h>", "#include <stdint.h>")
        assert not _killed(oracle.load_library(so))


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_mutant_is_caught(name, fname, old, new):
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(tmp, name, fname, old, new)
        assert _killed(oracle.load_library(so)), f"no pin caught: {name}"
