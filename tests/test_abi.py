"""The C-ABI library builds, loads and exports every symbol include/pta.h
declares; host-only entry points behave as documented (CPU, no GPU call)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pta.h")


@pytest.fixture(scope="module")
def P():
    import paper_2603_07321_gb300 as P
    P.build()
    P.load()
    return P


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(pta_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(P.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert n in P._SIGS, "binding lacks " + n


def test_struct_layouts_match_header(P, tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "pta.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(pta_specimen), sizeof(pta_potential),
         sizeof(pta_params), sizeof(pta_averages), sizeof(pta_coarse_result));
  printf("%zu %zu %zu %zu\\n", offsetof(pta_params, burst_steps), offsetof(pta_params, lanes),
         offsetof(pta_coarse_result, burst), offsetof(pta_coarse_result, status));
  return 0;
}
''')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(P.Specimen), ctypes.sizeof(P.Potential), ctypes.sizeof(P.Params),
            ctypes.sizeof(P.Averages), ctypes.sizeof(P.CoarseResult),
            P.Params.burst_steps.offset, P.Params.lanes.offset, P.CoarseResult.burst.offset,
            P.CoarseResult.status.offset]
    assert got == want


def test_defaults_follow_table_1(P):
    p = P.default_params()
    assert p.dt_fs == 1.0 and p.Delta == pytest.approx(p.h / 5)
    assert list(p.tol_v) == [0.01, 0.05, 0.01]  # K, U, T
    assert list(p.tol_j) == [0.08, 0.01, 0.05]
    assert p.precision == P.PREC_FP64


def test_library_c_equals_oracle_c(P, oracle):
    pot = P.default_potential()
    ref = oracle.Potential()
    assert pot.c == pytest.approx(ref.c, rel=1e-13)
    assert (pot.n, pot.m, pot.a, pot.rc, pot.eps) == (7, 6, 4.05, 8.1, 3.3147e-2)


def test_footprint(P):
    p64 = P.default_params()
    pmx = P.default_params(precision=P.PREC_MIXED)
    f10 = P.pta_footprint_bytes(P.make_specimen(10), p64)
    f20 = P.pta_footprint_bytes(P.make_specimen(20), p64)
    assert 0 < f10 < f20
    fmx = P.pta_footprint_bytes(P.make_specimen(20), pmx)
    # mixed precision keeps a second (pruned) list: more list memory, less state
    nomx = P.pta_footprint_bytes(P.make_specimen(20), P.default_params(precision=1,
                                                                      prune_margin=-1.0))
    assert nomx < fmx and nomx < f20
    # about 1-6 KB per atom at the default list capacity (2 A skin)
    for f in (f20, fmx):
        assert 500 < f / (4 * 20 ** 3) < 6000
    bad = P.make_specimen((2, 2, 2))
    assert P.pta_footprint_bytes(bad, p64) == 0


def test_atom_count_limit_leaves_room_for_the_sentinel_slot(P):
    # list entries hold a 23-bit slot index and slot n names the sentinel
    # record that pads the lists, so a specimen holds fewer than 2^23 atoms
    p64 = P.default_params()
    assert P.pta_footprint_bytes(P.make_specimen((128, 128, 128)), p64) == 0   # 2^23 atoms
    assert P.pta_footprint_bytes(P.make_specimen((49, 127, 337)), p64) > 0     # 2^23 - 4


def test_create_rejects_bad_arguments_before_touching_the_gpu(P):
    lib = P.load()
    spec = P.make_specimen((4, 4, 2))  # < 3 cells along the load axis
    pot = P.default_potential()
    par = P.default_params()
    h = ctypes.c_void_p()
    assert lib.pta_create(ctypes.byref(spec), ctypes.byref(pot), 300.0, 1, ctypes.byref(par),
                          None, ctypes.byref(h)) == -1
    spec = P.make_specimen(4)
    par.lanes = 3
    assert lib.pta_create(ctypes.byref(spec), ctypes.byref(pot), 300.0, 1, ctypes.byref(par),
                          None, ctypes.byref(h)) == -1
    par = P.default_params()
    assert lib.pta_create(ctypes.byref(spec), ctypes.byref(pot), -1.0, 1, ctypes.byref(par),
                          None, ctypes.byref(h)) == -1
    assert lib.pta_strerror(-4) == b"neighbour-list capacity exceeded"
    assert lib.pta_abi_version() == 2


def test_missing_library_fails_loudly():
    import importlib
    import paper_2603_07321_gb300 as P
    with pytest.raises(ImportError):
        saved = P._lib
        P._lib = None
        try:
            P.load("/nonexistent/libpta.so")
        finally:
            P._lib = saved


def test_neighbour_list_layout_index():
    # the tiled layout puts the 32 words a warp reads in one iteration side by side
    def nl_index(a, k, L, cap):
        G = 32 // L
        return (a // G) * (32 * (cap // L)) + (a % G) * L + (k // L) * 32 + (k % L)
    for L in (1, 2, 4, 8, 16):
        cap = 64
        G = 32 // L
        seen = set()
        for a in range(3 * G):
            for k in range(cap):
                seen.add(nl_index(a, k, L, cap))
        assert seen == set(range(3 * G * cap))  # a bijection onto the storage
        # one warp iteration q: lanes (a % G) * L + l read consecutive words
        q = 2
        words = sorted(nl_index(a, q * L + l, L, cap) for a in range(G) for l in range(L))
        assert words == list(range(words[0], words[0] + 32))


def test_new_parameters_are_validated_before_touching_the_gpu(P):
    lib = P.load()
    spec = P.make_specimen(4)
    pot = P.default_potential()
    h = ctypes.c_void_p()
    bad = [dict(conv_lag=-1), dict(conv_tol=(0.05, float("nan"), 0.05)),
           dict(conv_tol=(-0.1, 0.05, 0.05)), dict(mean_positions=2), dict(cell_tiles=2),
           dict(precision=0, cell_tiles=1), dict(cell_tiles=1), dict(atoms_per_thread=2)]
    for kw in bad:
        par = P.default_params(**kw)
        rc = lib.pta_create(ctypes.byref(spec), ctypes.byref(pot), 300.0, 1, ctypes.byref(par),
                            None, ctypes.byref(h))
        assert rc in (-1, -8), kw
    par = P.default_params()
    assert par.conv_lag == 0 and list(par.conv_tol) == [0.05] * 3
    assert par.mean_positions == 0 and par.skin == 2.0
    # the footprint grows by the mean-position sums when they are asked for
    f0 = P.pta_footprint_bytes(spec, P.default_params(precision=1))
    f1 = P.pta_footprint_bytes(spec, P.default_params(precision=1, mean_positions=1))
    assert f1 - f0 >= 32 * 4 * 4 ** 3
    # calls on a null context are rejected
    assert lib.pta_relax(None, 10, 10, 0.0, None, None) == -1
    assert lib.pta_get_mean_positions(None, None, 0) == -1
