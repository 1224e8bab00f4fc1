"""The no-allocation neighbour-list entry point.

pta_neighbours_noalloc serves callers that cannot allocate device memory
(for example an application whose pool already holds the whole GPU): it
keeps its scratch in a fixed array inside the library.  This test calls it
through the C ABI several times in a row, on different configurations, and
checks each result against the oracle's O(N^2) brute-force pair search and
against the library's ordinary list build (pta_get_neighbours) on the same
positions: the neighbour sets must be identical, as for every integer result
of the path.  One configuration has atoms outside the cell grid's box, which
the entry point clamps onto the border cells.  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import gpu_package, on_grid, sorted_rows

pytestmark = pytest.mark.gpu


def _noalloc(P, pos, lo, hi, rl, cap):
    import torch
    pos_d = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    counts_d = torch.full((len(pos),), -1, dtype=torch.int32, device="cuda")
    list_d = torch.full((len(pos), cap), -1, dtype=torch.int32, device="cuda")
    mx = P.pta_neighbours_noalloc(pos_d.data_ptr(), len(pos), lo, hi, rl, cap,
                                  counts_d.data_ptr(), list_d.data_ptr())
    torch.cuda.synchronize()
    return mx, counts_d.cpu().numpy(), list_d.cpu().numpy()


def test_noalloc_neighbours_match_brute_force(oracle):
    P = gpu_package()
    shape = (5, 6, 4)
    cap = 320
    rl = 9.1
    pos = on_grid(PI.jittered_fcc(shape, 0.25, seed=41))
    c_bf, l_bf = oracle.pairs(pos, rl, cap, method="brute")
    # box around every atom, then a box that leaves atoms outside on every
    # side (they are clamped onto the border cells), twice in a row each
    boxes = [(pos.min(axis=0) - 5.0, pos.max(axis=0) + 5.0),
             (pos.min(axis=0) + 6.0, pos.max(axis=0) - 6.0)]
    for lo, hi in boxes:
        for _ in range(2):
            mx, c_new, l_new = _noalloc(P, pos, lo, hi, rl, cap)
            assert mx == c_bf.max()
            assert np.array_equal(c_new, c_bf)
            assert sorted_rows(c_new, l_new) == sorted_rows(c_bf, l_bf)


def test_noalloc_neighbours_match_the_allocating_build():
    import torch
    P = gpu_package()
    shape = (6, 5, 7)
    cap = 320
    for call, seed in enumerate((31, 32)):  # two calls in a row share the scratch array
        pos = on_grid(PI.jittered_fcc(shape, 0.3, seed=seed))
        ctx = P.Ctx(shape, T0=0.0, precision=P.PREC_FP64)
        ctx.set_state(pos, np.zeros_like(pos))
        c_ref, l_ref = ctx.neighbours(cap=cap)
        rl = ctx.potential.rc + ctx.params.skin
        ctx.close()

        pos_d = torch.from_numpy(pos).cuda()
        counts_d = torch.full((len(pos),), -1, dtype=torch.int32, device="cuda")
        list_d = torch.full((len(pos), cap), -1, dtype=torch.int32, device="cuda")
        lo = pos.min(axis=0) - 5.0
        hi = pos.max(axis=0) + 5.0
        mx = P.pta_neighbours_noalloc(pos_d.data_ptr(), len(pos), lo, hi, rl, cap,
                                      counts_d.data_ptr(), list_d.data_ptr())
        torch.cuda.synchronize()
        c_new = counts_d.cpu().numpy()
        l_new = list_d.cpu().numpy()
        assert mx == c_ref.max()
        assert np.array_equal(c_new, c_ref), call
        assert sorted_rows(c_new, l_new) == sorted_rows(c_ref, l_ref), call


def test_noalloc_rejects_inputs_beyond_its_scratch():
    import torch
    P = gpu_package()
    n = P.NOALLOC_MAX_ATOMS + 1
    pos_d = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((n,), dtype=torch.int32, device="cuda")
    lst = torch.zeros((n, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(P.PTAError) as e:
        P.pta_neighbours_noalloc(pos_d.data_ptr(), n, [0, 0, 0], [1, 1, 1], 9.1, 1,
                                 out.data_ptr(), lst.data_ptr())
    assert e.value.status == -9
    # a grid with more cells than the scratch holds is rejected the same way
    pos_d = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PTAError) as e:
        P.pta_neighbours_noalloc(pos_d.data_ptr(), 10, [0, 0, 0], [1e4, 1e4, 1e4], 9.1, 1,
                                 out.data_ptr(), lst.data_ptr())
    assert e.value.status == -9
