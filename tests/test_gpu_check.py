"""The debug build (PTA_CHECK=1, libpta_check.so): every atom, cell-slot and
list index is tested before the access it feeds, every list count against
the list's capacity, the cell occupancy against the atom count, every force
for finiteness.  On valid inputs no test fails and the results are the
production build's, bit for bit; and the parity tests pass under it.

The debug library is chosen per process (the environment when the library
is first loaded), so each check runs in a child process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import gpu_package

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# a mixed-precision specimen with pruning, an FP64 specimen, and a batch of
# both, each through bursts long enough for list builds and prunings
SCRIPT = r"""
import json, sys
import numpy as np
import torch
import __graft_entry__ as g
g.build()
import paper_2603_07321_gb300 as P
torch.cuda.set_device(0)
out = {"lib": P.library_path(), "check": P.check_build()}
runs = []
for shape, prec, seed in (((6, 5, 7), P.PREC_MIXED, 3), ((5, 5, 5), P.PREC_FP64, 4)):
    c = P.Ctx(shape, T0=300.0, seed=seed, precision=prec)
    f, pe, _ = c.forces()
    c.apply_strain(2e-3)
    a = c.fine_burst(400)
    runs.append({"f": f.tolist(), "series": c.series().tolist(), "status": a.status,
                 "prunes": a.prunes, "rebuilds": a.rebuilds})
    c.close()
cs = [P.Ctx((4, 6, 5), T0=100.0, seed=7, precision=P.PREC_MIXED),
      P.Ctx((5, 4, 4), T0=300.0, seed=8, precision=P.PREC_FP64)]
b = P.Batch(cs)
b.apply_strain([1e-3, -1e-3])
res = b.fine_burst([300, 300])
runs.append({"series": [c.series().tolist() for c in cs], "status": [r.status for r in res]})
b.close()
for c in cs:
    c.close()
out["runs"] = runs
print("RESULT " + json.dumps(out))
"""


def _child(env_check: bool, code: str):
    env = dict(os.environ)
    env["PTA_CHECK"] = "1" if env_check else "0"
    env["PYTHONPATH"] = ROOT + os.pathsep + os.path.join(ROOT, "tests") + os.pathsep + \
        env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_check_build_passes_and_changes_nothing():
    gpu_package()
    dbg = _child(True, SCRIPT)
    prod = _child(False, SCRIPT)
    assert dbg["check"] and dbg["lib"].endswith("libpta_check.so")
    assert not prod["check"] and prod["lib"].endswith("libpta.so")
    for a, b in zip(dbg["runs"][:2], prod["runs"][:2]):
        assert a["status"] == 0 and b["status"] == 0
        assert a["prunes"] == b["prunes"] and a["rebuilds"] == b["rebuilds"]
        assert np.array_equal(np.array(a["f"]), np.array(b["f"]))
        assert np.array_equal(np.array(a["series"]), np.array(b["series"]))
    assert dbg["runs"][0]["prunes"] > 0          # the inner list was exercised
    a, b = dbg["runs"][2], prod["runs"][2]
    assert a["status"] == [0, 0] and b["status"] == [0, 0]
    for x, y in zip(a["series"], b["series"]):
        assert np.array_equal(np.array(x), np.array(y))


def test_parity_tests_pass_under_the_check_build():
    gpu_package()
    env = dict(os.environ)
    env["PTA_CHECK"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "-m", "gpu",
                        "-q", "-x", "-p", "no:cacheprovider",
                        "-k", "neighbour_sets or trajectory or forces or coarse or batch"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-2000:])
    assert " passed" in r.stdout
