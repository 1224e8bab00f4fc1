/*
 * pta.h -- C ABI of the GB300 fine-burst engine for Practical Time Averaging
 * molecular dynamics (Baruah, Chatterjee, Acharya, Wang, "Averaging
 * Molecular Dynamics simulations to study the slow-strain-rate behavior of
 * metals", arXiv 2603.07321).
 *
 * What the library computes (all of it in CUDA kernels for sm_103a):
 *   - the specimen of the problem-setup section: an FCC block with cube
 *     axes along x, y, z, two grip slabs normal to the load axis, lattice
 *     positions and Maxwell-Boltzmann velocities at T0;
 *   - fine bursts of NVE velocity-Verlet dynamics, Eqs. (vv_algo_pos_pred_half),
 *     (vv_algo_pos_pred), (vv_algo_vel_pred), with the EAM energy of
 *     Eq. (pe) and forces of Eq. (f_int), the grips held by v = 0, F = 0;
 *   - the state functions K, U and T of Eq. (state_variables), sampled
 *     after every full step, and their running time averages R^m of
 *     Eq. (R_m_t) with block standard errors;
 *   - the grip displacements of the loading protocol and the coarse-step
 *     update of Eqs. (dvdt_algo), (pta_pred), (simp), (rel_err), (jump_err).
 *
 * Conventions
 *   - Units: Angstrom, femtosecond, atomic mass unit, eV, kelvin; stresses
 *     in GPa.  Slow variables are ordered (K, U, T): index 0 kinetic energy
 *     (eV), 1 potential energy (eV), 2 normal stress along the load axis (GPa).
 *   - Every function returns PTA_OK (0) or a negative pta_status.  No C++
 *     exception crosses the ABI.
 *   - Host arrays are plain C arrays owned by the caller.  Positions and
 *     velocities are n x 3 doubles, atom-major (x0 y0 z0 x1 y1 z1 ...), in
 *     the library's atom order: atom index 4*(i + nx*(j + ny*k)) + b for
 *     conventional cell (i, j, k) and basis site b in
 *     {(0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2)}.
 *   - A context owns all its device memory.  It takes that memory from the
 *     allocator installed with pta_set_allocator (the Python binding
 *     installs one backed by PyTorch's caching allocator), else from
 *     cudaMalloc.  Memory is returned by pta_destroy.
 *   - Calls on one context must not run concurrently.  Calls that return
 *     results to the host block until those results are on the host.
 *     Device work is queued on the CUDA stream given at creation.
 *   - After PTA_ECUDA the context is unusable and must be destroyed; other
 *     contexts are unaffected.
 */
#ifndef PTA_H
#define PTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTA_ABI_VERSION 2

typedef enum {
    PTA_OK = 0,
    PTA_EINVAL = -1,          /* an argument is out of its documented range            */
    PTA_ENOMEM = -2,          /* the allocator returned no memory                      */
    PTA_ECUDA = -3,           /* a CUDA call failed; destroy the context               */
    PTA_ENEIGH_OVERFLOW = -4, /* an atom had more neighbours than the list capacity:
                                 the burst's dynamics are invalid; recreate the
                                 context with a larger pta_params.neigh_cap          */
    PTA_ENAN = -5,            /* a non-finite energy appeared during a burst           */
    PTA_ESTATE = -6,          /* the call is not valid in the context's state          */
    PTA_ERANGE = -7,          /* a coordinate left the range the mixed-precision
                                 representation holds (|x| < 512 A), an atom left
                                 the cell grid (its margin of a quarter of the
                                 specimen's extent around the lattice), or a
                                 specimen has 2^23 or more atoms                     */
    PTA_EUNSUPPORTED = -8,    /* an option this build does not provide                 */
    PTA_ECAPACITY = -9,       /* the input exceeds the fixed scratch size of
                                 pta_neighbours_noalloc                              */
    PTA_ECHECK = -10          /* debug build only (compiled with PTA_CHECK=1): an atom,
                                 cell or list index or a list count was out of its
                                 range; the offending access was skipped and the
                                 results are invalid                                 */
} pta_status;

enum { PTA_POT_SUTTON_CHEN_SF = 1 };
enum { PTA_PREC_FP64 = 0, PTA_PREC_MIXED = 1 };
enum { PTA_SRC_PREDICTED = 0, PTA_SRC_MEASURE_JUMP = 1, PTA_SRC_MEASURE_MISMATCH = 2 };


/* Specimen (problem-setup section; grips from the boundary-conditions
 * section).  n_cells >= 3 along the load axis and >= 1 along the others.
 * The left grip holds the atoms whose coordinate along load_axis lies
 * within grip_width (+1e-6 A) of the lowest one, the right grip those within
 * grip_width of the highest one; grip_width <= 0 means a0. */
typedef struct {
    int n_cells[3];
    double a0;         /* lattice parameter, A (Table 1: 4.05)              */
    int load_axis;     /* 0 = x, 1 = y, 2 = z                               */
    double grip_width; /* A                                                  */
} pta_specimen;

/* Potential, Eq. (pe) in Sutton-Chen form: V(r) = eps phi_n(r),
 * rho(r) = phi_m(r), B(rho) = -eps c sqrt(rho), phi_k(r) = (a/r)^k made
 * smooth at rc by the shifted-force cut: phi_k(r) - phi_k(rc) - phi_k'(rc)(r-rc)
 * for r < rc, 0 beyond.  kind must be PTA_POT_SUTTON_CHEN_SF; 1 <= m, n <= 16;
 * 0 < a; 0 < rc. */
typedef struct {
    int kind;
    double eps; /* eV */
    double c;   /* dimensionless */
    double a;   /* A */
    double rc;  /* A */
    int n, m;
} pta_potential;

/* Run parameters (Table 1 and the loading protocol). */
typedef struct {
    double dt_fs;       /* MD time step (Table 1: 1 fs)                       */
    double mass_amu;    /* atomic mass (Al: 26.9815385)                       */
    double skin;        /* Verlet-list skin, A; list radius rc + skin          */
    double h;           /* slow-time step, s                                   */
    double Delta;       /* averaging interval, s (Table 1: h/5)                */
    double strain_rate; /* 1/s, negative for compression                      */
    double tol_v[3];    /* Eq. (rel_err) tolerances (Table 1: K 1%, U 5%, T 1%) */
    double tol_j[3];    /* Eq. (jump_err) tolerances (Table 1: K 8%, U 1%, T 5%) */
    double floor[3];    /* denominators of the relative tests are max(|x|, floor) */
    int64_t burst_steps;/* fine steps per burst used by pta_coarse_step         */
    int block_steps;    /* block length (steps) of the standard errors         */
    int precision;      /* PTA_PREC_FP64 or PTA_PREC_MIXED                     */
    int neigh_cap;      /* neighbour-list capacity per atom, 0 = automatic     */
    int lanes;          /* threads per atom in the pair kernels: 0 = automatic,
                           else 1, 2, 4, 8 or 16                               */
    int atoms_per_thread; /* atoms per thread group: 0 or 1 (2, two atoms sharing
                           a union list, is no longer provided:
                           PTA_EUNSUPPORTED)                                  */
    double prune_margin;  /* mixed precision: the pair passes read an inner list
                           of the pairs within rc + prune_margin, pruned from the
                           Verlet list whenever an atom has moved more than
                           prune_margin / 2 since the last pruning; it holds every
                           pair within rc in the same order, so results do not
                           change.  0 = default 0.3 A, < 0 = off               */
    int cell_tiles;     /* 0 or -1; 1 (pair passes by shared-memory cell tiles) is
                           no longer provided: PTA_EUNSUPPORTED              */
    int conv_lag;       /* adaptive burst length (appendix, Eq. (R_m_conv)):
                           every conv_lag steps from 2 conv_lag on, variable m
                           has converged once |R^(i) - R^(i-k)| /
                           max(|R^(i)|, floor[m]) < conv_tol[m], R^ the running
                           average; the burst ends when all three have, or at
                           its length (N_max).  0 (default) = fixed length   */
    double conv_tol[3]; /* tol_m of the convergence test (Table 1: 5% each)    */
    int mean_positions; /* 1: also average every atom's position over the
                           states a burst samples (Eq. (mean_pos)), read with
                           pta_get_mean_positions; 0 (default) = off        */
} pta_params;

/* Burst result: Eq. (R_m_t) means over the nsteps samples taken after each
 * full step (the initial state is not sampled), standard errors from
 * non-overlapping blocks of block_steps samples (NaN with fewer than two
 * blocks), the number of neighbour-list builds and inner-list prunings
 * during the burst.  With an adaptive burst length (pta_params.conv_lag > 0,
 * appendix, Eq. (R_m_conv)) the burst stops once every variable's running
 * average has converged: mean[m] is then the running average at that
 * variable's own convergence step nsamples[m] (bit `m` of `converged` set),
 * se[m] comes from the blocks within those samples, and nsteps is the
 * number of steps run; a variable that has not converged when the burst
 * reaches its length keeps the average of all samples.  Without it,
 * nsamples[m] = nsteps and converged = 0. */
typedef struct {
    double mean[3];
    double se[3];
    int64_t nsteps;
    int32_t rebuilds;
    int32_t status;    /* pta_status of this burst */
    int32_t prunes;    /* inner-list prunings during the burst (mixed precision) */
    int32_t converged; /* adaptive length: bit m set when variable m converged */
    int64_t nsamples[3];
} pta_averages;

/* Coarse step t -> t+h.  v_pred: Eq. (pta_pred); v_d: Eq. (simp); e_v:
 * Eq. (rel_err); e1, e2: Eq. (jump_err) (e2 is NaN at the first step);
 * source: which value was accepted (PTA_SRC_*); v: the accepted slow
 * variables; strain: grip displacement / specimen length after the step;
 * burst[]: the three bursts at t+h-Delta, t+h-Delta/2, t+h. */
typedef struct {
    double t;
    double strain;
    double v[3], v_pred[3], v_d[3], e_v[3], e1[3], e2[3];
    int32_t jump[3];
    int32_t source[3];
    pta_averages burst[3];
    int32_t status;
    int32_t pad;
} pta_coarse_result;

typedef struct pta_ctx pta_ctx;
typedef struct pta_batch pta_batch;

/* Allocator hook.  alloc returns device memory of at least `bytes` bytes,
 * aligned to 256 bytes, usable on `stream` (a cudaStream_t), or NULL;
 * release gives it back.  Installed hooks apply to contexts created after
 * the call; NULL, NULL restores cudaMalloc/cudaFree. */
typedef void *(*pta_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pta_free_fn)(void *ptr, void *stream, void *user);
int pta_set_allocator(pta_alloc_fn alloc, pta_free_fn release, void *user);

const char *pta_strerror(int status);
int pta_abi_version(void);

/* Defaults: Table 1 values (dt 1 fs, Delta = h/5 with h = 1 s, tolerances),
 * Al mass, skin 2 A, 2,000-step bursts, blocks of 100 steps, FP64. */
int pta_default_params(pta_params *out);
/* Sutton-Chen Al (eps 3.3147e-2 eV, n 7, m 6, a 4.05 A), rc = 2 a, and c
 * chosen so that the perfect crystal under the cut potential is in
 * equilibrium at lattice parameter a (dE/da = 0). */
int pta_default_potential(pta_potential *out);

/* Device bytes a context of this specimen and these parameters will hold
 * (for admission by memory footprint). */
size_t pta_footprint_bytes(const pta_specimen *spec, const pta_params *par);

/* Build the specimen and its initial state s(-Delta) (boundary-conditions
 * section): lattice positions, grips, and for the mobile atoms velocities
 * drawn from N(0, kT0/m) by Philox4x32-10 (counter (atom, 0..1, 0, 0), key =
 * seed) with Box-Muller, mean removed, scaled to K = (3 N_mob - 3) k T0 / 2;
 * grip atoms get v = 0.  stream is a cudaStream_t (may be NULL).  On success
 * *out is a new context. */
int pta_create(const pta_specimen *spec, const pta_potential *pot, double T0_K, uint64_t seed,
               const pta_params *par, void *stream, pta_ctx **out);
void pta_destroy(pta_ctx *ctx);

int pta_natoms(const pta_ctx *ctx, int64_t *n);
/* The kernel layout chosen for this context: out[0] threads per atom
 * (lanes), out[1] atoms per thread group, out[2] neighbour-list capacity per
 * atom, out[3] 1 when the pruned inner list is in use. */
int pta_get_layout(const pta_ctx *ctx, int32_t out[4]);
/* 0 mobile, 1 left grip, 2 right grip; n must equal the atom count */
int pta_get_flags(pta_ctx *ctx, uint8_t *flags, int64_t n);

/* Loading protocol: move the right grip by d_eps * L_s along the load axis
 * (L_s = n_cells[load_axis] * a0); the grip stays fixed there during the
 * following bursts. */
int pta_apply_strain(pta_ctx *ctx, double d_eps);
/* Total grip displacement / L_s applied so far. */
int pta_get_strain(const pta_ctx *ctx, double *strain);

/* One fine burst of nsteps velocity-Verlet steps from the current state
 * (which the next burst continues from, Eqs. (x_guess_step1),
 * (x_guess_step3)).  Blocks until the averages are on the host.  nsteps >= 1. */
int pta_fine_burst(pta_ctx *ctx, int64_t nsteps, pta_averages *out);
/* Continuous loading (Sec. Verification with fine dynamics): a fine burst
 * of nsteps steps during which the right grip advances by d_eps_per_step *
 * L_s along the load axis with every step (with the drift of each step),
 * instead of being held fixed.  This is the uninterrupted fine dynamics
 * against which the slow variables of PTA are verified: bursts of it are one
 * trajectory under a load ramped at d_eps_per_step per step.  The grip
 * displacement reported by pta_get_strain grows by nsteps * d_eps_per_step.
 * PTA_EUNSUPPORTED with an adaptive burst length (conv_lag > 0). */
int pta_ramp_burst(pta_ctx *ctx, int64_t nsteps, double d_eps_per_step, pta_averages *out);
/* Thermal relaxation before loading (Sec. Boundary conditions): bursts of
 * `window` steps with the right grip free to move along the load axis (its
 * other velocity components stay 0; the left grip stays fixed) until the
 * window mean of T is within tol_gpa of 0, or until another window would
 * exceed max_steps.  The right-grip atoms are then fixed where the
 * relaxation left them (v = 0), and later grip displacements count from
 * there.  *out gets the
 * last window's averages, *steps the steps run (either may be NULL).
 * NVE has no damping: the free grip oscillates about the stress-free
 * position, so the window must span many oscillation periods (thousands of
 * steps).  window >= 1, max_steps >= window, tol_gpa >= 0. */
int pta_relax(pta_ctx *ctx, int64_t window, int64_t max_steps, double tol_gpa,
              pta_averages *out, int64_t *steps);
/* Eq. (mean_pos): every atom's mean position over the states the last
 * burst sampled (after each full step), n x 3 doubles in creation order, A.
 * Needs pta_params.mean_positions = 1 (else PTA_EUNSUPPORTED) and a burst
 * with at least one sample (else PTA_EINVAL); n must equal the atom count. */
int pta_get_mean_positions(pta_ctx *ctx, double *out, int64_t n);
/* The K, U, T samples of the last burst, nsteps x 3 doubles; *count gets
 * the number of samples (at most max_steps are copied). */
int pta_get_series(pta_ctx *ctx, double *series, int64_t max_steps, int64_t *count);

/* One coarse step of the protocol: grip +rate*(h-Delta)*L_s, burst;
 * +rate*Delta/2*L_s, burst; +rate*Delta/2*L_s, burst; then the coarse
 * update.  The first call first runs the three initial bursts (grip at its
 * current position, then two increments of rate*Delta/2*L_s), labelled
 * -Delta, -Delta/2, 0, and sets v(0) to their Simpson value. */
int pta_coarse_step(pta_ctx *ctx, pta_coarse_result *out);

/* The coarse-step update alone, on three given burst results instead of
 * three bursts: means[3 * b + m] is R^m of burst b (b = 0, 1, 2 at
 * t+h-Delta, t+h-Delta/2, t+h; m = K, U, T).  The first call on a context
 * whose initial bursts have not run treats them as the bursts labelled
 * -Delta, -Delta/2, 0 and sets v(0) to their Simpson value, Eq. (simp); every
 * later call is one update t -> t+h of Eqs. (dvdt_algo), (pta_pred), (simp),
 * (rel_err), (jump_err), in the same kernel and on the same slow-variable
 * record as pta_coarse_step.  No grip moves and no dynamics run.  For
 * replaying the slow-time logic on recorded burst averages.  out->burst[b]
 * carries the given means (nsteps 0).  PTA_EINVAL for non-finite means. */
int pta_coarse_update(pta_ctx *ctx, const double means[9], pta_coarse_result *out);

/* State exchange (host copies, n x 3 doubles each, library atom order).
 * pta_set_state replaces positions and velocities; grip atoms keep
 * whatever velocity is given (callers normally pass 0). */
int pta_get_state(pta_ctx *ctx, double *pos, double *vel, int64_t n);
int pta_set_state(pta_ctx *ctx, const double *pos, const double *vel, int64_t n);

/* One force evaluation at the current positions (internal forces of
 * Eq. (f_int) before the grip constraint; f: n x 3 eV/A, pe: n per-atom
 * energies 1/2 eps sum_j phi_n + B(rho_i), eV).  Either pointer may be NULL.
 * obs (may be NULL) gets K, U, T of the current state. */
int pta_forces(pta_ctx *ctx, double *f, double *pe, int64_t n, double obs[3]);

/* The Verlet list built from the current positions: counts[n] and
 * list[n * cap] (row-major, the neighbours of atom i in list order in row
 * i).  Returns PTA_EINVAL if cap is below the largest count, which is
 * written to *max_count. */
int pta_get_neighbours(pta_ctx *ctx, int32_t *counts, int32_t *list, int64_t n, int32_t cap,
                       int32_t *max_count);

/* Checkpoint: the whole fine and slow state (positions, velocities, grip
 * displacement, coarse-step record) as an opaque byte string.  With
 * buf == NULL, *len gets the size needed. */
int pta_save_state(pta_ctx *ctx, void *buf, size_t *len);
int pta_load_state(pta_ctx *ctx, const void *buf, size_t len);

/* Kernel timing.  While timing is on, every fine-step iteration records
 * CUDA events (on the context's stream, inside the replayed graphs) around
 * its three parts: the neighbour-list build (usually skipped on the
 * device), the density pass and the force pass.  pta_get_timing returns the
 * summed event times in milliseconds and the number of iterations since
 * timing was switched on.  Timing costs one host synchronisation per graph
 * replay of 64 iterations. */
typedef struct {
    double rebuild_ms, density_ms, force_ms;
    int64_t iterations;
} pta_kernel_times;
int pta_set_timing(pta_ctx *ctx, int enable);
int pta_get_timing(pta_ctx *ctx, pta_kernel_times *out);

/* Batches: several contexts advanced by the same kernel launches (one set
 * of launches per fine step for all members, replayed from a CUDA graph).
 * Members must use the same stream (precisions and sizes may differ) and belong to no other
 * batch; they stay usable on their own between batch calls. */
int pta_batch_create(pta_ctx *const *members, int count, pta_batch **out);
void pta_batch_destroy(pta_batch *batch);
/* d_eps[count]: per-member grip increments (strain units). */
int pta_batch_apply_strain(pta_batch *batch, const double *d_eps);
/* nsteps[count]: per-member burst lengths (0 leaves a member idle);
 * out[count] receives the averages.  A failure of single members
 * (PTA_ENEIGH_OVERFLOW, PTA_ENAN, PTA_ERANGE, PTA_ECHECK in out[i].status)
 * is returned as the first such status after every out[i] is filled; the
 * other members' results are valid and the batch stays usable. */
int pta_batch_fine_burst(pta_batch *batch, const int64_t *nsteps, pta_averages *out);
/* One coarse step of every member (each with its own strain rate and
 * burst length), out[count]; members that have not yet run their initial
 * bursts run them first, as pta_coarse_step does. */
int pta_batch_coarse_step(pta_batch *batch, pta_coarse_result *out);
/* One slow-time tick of every member, three bursts each: a member whose
 * initial bursts have not run runs them (its result has t = 0, v = v(0),
 * source[] = -1); every other member runs one coarse step.  This is the
 * unit of continuous batching: members at different stages share the same
 * launches.  Member failures are reported as for pta_batch_fine_burst:
 * out[i].status per member, the first one returned, the others valid. */
int pta_batch_tick(pta_batch *batch, pta_coarse_result *out);
int pta_batch_set_timing(pta_batch *batch, int enable);
int pta_batch_get_timing(pta_batch *batch, pta_kernel_times *out);

/* Measurement helper (no counterpart in the paper): the fused multiply-add
 * rate of the current GPU, the peak the pair kernels' roofline divides by.
 * One launch fills every SM with threads that each run 16 independent FMA
 * chains of `iters` steps; kind 0 = scalar FP32, 1 = packed FP32 (two
 * lanes per instruction), 2 = FP64.  *flops gets the flop count (2 per FMA
 * and lane), *ms the launch's CUDA-event time on `stream` (a cudaStream_t).
 * Kinds 3-5 time the operations a pair pass that evaluates each unordered
 * pair once would add per pair to keep 64-bit fixed-point (deterministic)
 * j-side sums: 3 = 64-bit integer reductions to global memory at hashed
 * addresses of a 15 MB buffer (allocated and freed by the call, as is a
 * small buffer every kind's keep-alive stores go to), 4 = 64-bit
 * integer atomic adds in shared memory, 5 = FP32 -> int64 conversions
 * (16 per iteration and thread); for these *flops gets the operation count.
 * Returns PTA_EINVAL for another kind or iters < 1.  Blocks until the launch
 * is done. */
int pta_measure_fma_rate(int kind, int64_t iters, void *stream, double *flops, double *ms);

/* Neighbour lists without device allocation.
 *
 * No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory, such as an application whose memory pool
 * already holds the whole GPU, or a latency-critical loop in which
 * cudaMalloc and cudaFree (which may synchronise the device) are not
 * allowed.  It builds the same Verlet lists as the library's list build
 * (every j != i with (dx*dx + dy*dy) + dz*dz < rlist^2 in FP64, candidates
 * from a cell grid over [box_lo, box_hi] with atoms outside clamped onto
 * its border cells) but allocates nothing: its scratch memory (cell counts
 * and starts, the atoms' cells, the sorted cell contents) is a fixed array
 * in the library, about 2.1 MB, that every GPU which loads the library holds
 * until the process exits.
 *
 *   pos_dev     n x 3 doubles, atom-major, in device memory (read only)
 *   n           1 .. PTA_NOALLOC_MAX_ATOMS atoms
 *   box_lo/hi   host arrays of 3 doubles: the cell grid's extent (A)
 *   rlist       list radius (A); the grid has at most PTA_NOALLOC_MAX_CELLS
 *               cells of edge rlist (1 + 1e-4)
 *   cap         row length of list_dev
 *   counts_dev  n int32 in device memory: neighbour count of each atom
 *               (at most cap)
 *   list_dev    n x cap int32 in device memory, row-major: the neighbours
 *               of atom i in cell order, then increasing index
 *   max_count   host int: the largest count before truncation
 *   stream      cudaStream_t to queue the work on; the call returns once
 *               the work is done
 * Returns PTA_ECAPACITY when n or the cell count exceeds the fixed scratch,
 * PTA_ENEIGH_OVERFLOW when an atom had more than cap neighbours (rows are
 * then truncated), PTA_EINVAL for bad arguments.
 *
 * Every call shares the one scratch array and clears what must start at
 * zero; calls that overlap on the GPU (from two streams or two host
 * threads) race on it and must be serialised by the caller.  The first
 * call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. */
#define PTA_NOALLOC_MAX_ATOMS 131072
#define PTA_NOALLOC_MAX_CELLS 65536
int pta_neighbours_noalloc(const double *pos_dev, int32_t n, const double box_lo[3],
                           const double box_hi[3], double rlist, int32_t cap, int32_t *counts_dev,
                           int32_t *list_dev, int32_t *max_count, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PTA_H */
