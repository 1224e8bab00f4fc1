"""Autotuner of the launch layout for a specimen size.

The fastest layout depends on the specimen and on how many specimens share
the device: a small cube alone wants several threads per atom, the same cube
in a large batch one; a bigger Verlet skin trades longer lists for fewer
builds.  `tune` measures instead of guessing: for every candidate
(threads per atom, skin) it creates the specimen (or a batch of
identical-size replicas), runs a short warm burst, times a burst on the
device, and returns the candidates ranked by atom-steps per second.  Every
candidate computes the same physics; the choice only changes speed (and, in
mixed precision, the summation order of the pair terms).

    from paper_2603_07321_gb300.tune import tune
    best, table = tune(20, replicas=64)
    ctx = Ctx(20, **best)
"""
from __future__ import annotations

import itertools
import time


def tune(n_cells, precision: int = 1, replicas: int = 1, T0: float = 300.0, seed: int = 1,
         lanes=(1, 2, 4, 8), skins=(1.0, 2.0), steps: int = 200, warm: int = 50,
         strain: float = 1e-3):
    """Time every (lanes, skin) candidate; returns (best, table): best is a
    dict of Ctx keyword arguments, table a list of (atom-steps/s, kwargs)
    sorted fastest first.  Candidates the library rejects are skipped."""
    from . import Batch, Ctx, PTAError
    table = []
    for L, skin in itertools.product(lanes, skins):
        kw = dict(precision=precision, lanes=L, skin=skin)
        try:
            ctxs = [Ctx(n_cells, T0=T0, seed=seed + i, **kw) for i in range(replicas)]
        except PTAError:
            continue
        try:
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
            natoms = sum(c.n for c in ctxs)
            table.append((natoms * steps / dt, kw))
        finally:
            for c in ctxs:
                c.close()
    table.sort(key=lambda x: -x[0])
    if not table:
        raise ValueError("no candidate layout could be created")
    return dict(table[0][1]), table
