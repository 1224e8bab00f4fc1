"""Small driver for profiling the fine-burst kernels.

    python -m paper_2603_07321_gb300.profile_case N_CELLS PRECISION WARM STEPS [LANES [TILES]]

creates an N_CELLS^3-cell FCC Al cube (PRECISION 0 = FP64, 1 = mixed), moves the
right grip by a 1e-3 strain, runs a warm burst of WARM steps and a burst of
STEPS steps, and prints the throughput of the second.  LANES 0 chooses the
lanes automatically; TILES 1 turns the cell tiles on.  Run it under Nsight
Compute with PTA_GRAPH_FLAT=1 (graphs without conditional nodes, whose kernel
nodes the profiler can capture).
"""
import sys
import time


def main(argv):
    import torch
    import paper_2603_07321_gb300 as P
    n, prec, warm, steps = (int(x) for x in argv[:4])
    lanes = int(argv[4]) if len(argv) > 4 else 0
    tiles = int(argv[5]) if len(argv) > 5 else 0
    P.build()
    ctx = P.Ctx(n, T0=300.0, seed=1, precision=prec, lanes=lanes, cell_tiles=tiles)
    ctx.apply_strain(1e-3)
    ctx.fine_burst(warm)
    torch.cuda.synchronize()
    t = time.perf_counter()
    a = ctx.fine_burst(steps)
    dt = time.perf_counter() - t
    print("n=%d atoms=%d steps=%d %.4f s %.3e atom-steps/s rebuilds=%d prunes=%d layout=%s" % (
        n, ctx.n, steps, dt, ctx.n * steps / dt, a.rebuilds, a.prunes, ctx.layout()))
    ctx.close()


if __name__ == "__main__":
    main(sys.argv[1:])
