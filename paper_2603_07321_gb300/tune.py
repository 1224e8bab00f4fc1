"""Autotuner of the launch layout, with a persistent cache the library's
binding consults.

The fastest layout depends on the specimen and on how many specimens share
the device: a small cube alone wants several threads per atom, the same cube
in a large batch one; a bigger Verlet skin (and with it a bigger cell edge,
h = rc + skin) trades longer lists for fewer builds; the inner-list margin
trades longer inner lists for fewer prunings.  `tune` measures instead of
guessing: for every candidate (threads per atom, skin, pruning margin) it
creates the specimen (or a batch of identical-size replicas), runs a short
warm burst, times a burst, ranks the candidates by atom-steps per second and
stores the winner in a JSON cache keyed by (precision, atom count rounded to
a power of two, replica count rounded up to a power of two).  `Ctx` takes
the cached layout whenever its threads per atom are left automatic.

Every candidate computes the same physics.  The pruning margin leaves the
summation order unchanged (the inner list keeps every pair within rc in the
Verlet list's order), so results are bit-identical; the skin changes the cell
edge and with it the order of each atom's list entries, and the threads per
atom the order in which one atom's pair terms are added (rounding-level
differences).

    from paper_2603_07321_gb300.tune import tune
    best, table = tune(20, replicas=64)        # measured and cached
    ctx = Ctx(20)                              # picks the cached layout

The cache file is $PTA_TUNE_CACHE, else ~/.cache/paper_2603_07321_gb300/tune.json.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time

LAYOUT_KEYS = ("lanes", "skin", "prune_margin")


def cache_path() -> str:
    p = os.environ.get("PTA_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2603_07321_gb300", "tune.json")


def cache_key(natoms: int, replicas: int, precision: int) -> str:
    size = 2 ** int(round(math.log2(max(int(natoms), 1))))
    reps = 1 if replicas <= 1 else 2 ** int(math.ceil(math.log2(replicas)))
    return "prec%d:atoms%d:replicas%d" % (int(precision), size, reps)


def _read() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def lookup(natoms: int, replicas: int = 1, precision: int = 1):
    """The cached layout (dict of Ctx keyword arguments) or None."""
    e = _read().get(cache_key(natoms, replicas, precision))
    if not e:
        return None
    return {k: e[k] for k in LAYOUT_KEYS if k in e}


def store(natoms: int, replicas: int, precision: int, layout: dict, rate: float):
    path = cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    data = _read()
    entry = {k: layout[k] for k in LAYOUT_KEYS if k in layout}
    entry["atom_steps_per_s"] = float(rate)
    data[cache_key(natoms, replicas, precision)] = entry
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(n_cells, precision: int = 1, replicas: int = 1, T0: float = 300.0, seed: int = 1,
         lanes=(1, 2, 4, 8), skins=(1.0, 1.5, 2.0, 2.5), margins=(0.3,), steps: int = 200,
         warm: int = 50, strain: float = 1e-3, save: bool = True):
    """Time every (lanes, skin, prune_margin) candidate; returns (best,
    table): best is a dict of Ctx keyword arguments, table a list of
    (atom-steps/s, kwargs) sorted fastest first.  Candidates the library
    rejects are skipped.  With save, the winner goes to the cache."""
    from . import Batch, Ctx, PTAError
    table = []
    natoms = None
    for L, skin, margin in itertools.product(lanes, skins, margins):
        kw = dict(precision=precision, lanes=L, skin=skin, prune_margin=margin)
        try:
            ctxs = [Ctx(n_cells, T0=T0, seed=seed + i, tuned=False, **kw)
                    for i in range(replicas)]
        except PTAError:
            continue
        try:
            natoms = ctxs[0].n
            if replicas > 1:
                b = Batch(ctxs)
                b.apply_strain([strain] * replicas)
                b.fine_burst([warm] * replicas)
                t0 = time.perf_counter()
                b.fine_burst([steps] * replicas)   # returns once the averages are on the host
                dt = time.perf_counter() - t0
                b.close()
            else:
                c = ctxs[0]
                c.apply_strain(strain)
                c.fine_burst(warm)
                t0 = time.perf_counter()
                c.fine_burst(steps)
                dt = time.perf_counter() - t0
            table.append((sum(c.n for c in ctxs) * steps / dt, kw))
        finally:
            for c in ctxs:
                c.close()
    table.sort(key=lambda x: -x[0])
    if not table:
        raise ValueError("no candidate layout could be created")
    best = {k: table[0][1][k] for k in LAYOUT_KEYS}
    if save:
        store(natoms, replicas, precision, best, table[0][0])
    return dict(table[0][1]), table
