// Device-side data structures of the fine-burst engine.
//
// One specimen on the device is described by a SpecDev (sizes, constants,
// pointers) and a SpecCtl (the mutable control block the kernels update).
// Kernels take an array of SpecDev plus a block->specimen table, so a single
// launch advances one specimen or a whole batch of them: the block's
// specimen is specs[b2s[blockIdx.x]] and its block index inside that
// specimen is blockIdx.x - first block of that specimen.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pta.h"

namespace pta {

constexpr int TPB = 128;        // threads per block of the atom and pair kernels
constexpr int CELL_WARPS = 8;   // warps per block of the cell-sort kernel
constexpr int CELLS_PER_WARP = 8;  // cells one warp of the cell-sort kernel orders in turn
constexpr int SCAN_THREADS = 1024;

// grid quantum of the mixed-precision position split x = hi + lo:
// hi is a multiple of 2^-12 A (exact in FP32 for |x| < 512 A), |lo| <= 2^-13 A
constexpr double HI_SCALE = 4096.0;
constexpr double HI_QUANTUM = 1.0 / 4096.0;
constexpr double MIXED_RANGE = 511.0;

enum Phase : int { PH_IDLE = 0, PH_REFRESH = 1, PH_RUN = 2 };
// ERR_GRID: an atom lay beyond the cell grid's margin at a list build (it is
// binned onto the nearest border cell, which keeps the pair search complete);
// ERR_CHECK: a debug build's index or count test failed
enum ErrBit : int { ERR_OVERFLOW = 1, ERR_NAN = 2, ERR_RANGE = 4, ERR_GRID = 8, ERR_CHECK = 16 };

// Debug builds (compiled with -DPTA_CHECK=1) test every atom, cell-slot and
// list index before the access it feeds, every list count against the
// list's capacity, the cell occupancy against the atom count, and every
// atom's force for finiteness; a failed test sets ERR_CHECK (ERR_NAN for a
// force) and the access goes to index 0 instead, so a debug build never
// reads or writes out of bounds.  Production builds compile the tests away.
#ifndef PTA_CHECK
#define PTA_CHECK 0
#endif
// mixed precision: velocity as an exact FP32 pair v = h + l
struct __align__(32) VelHL {
    float4 h, l;
};
enum Mode : int { MODE_STEP = 0, MODE_EVAL = 1 };
enum AtomFlag : uint8_t { FLAG_MOBILE = 0, FLAG_LEFT = 1, FLAG_RIGHT = 2 };

// Sutton-Chen potential with the shifted-force cut, in both precisions.
//   phi_k(r)  = s^k - A_k + B_k (r - rc),   s = a/r, A_k = (a/rc)^k, B_k = k A_k / rc
//   phi_k'(r) = -k s^k / r + B_k
struct PotDev {
    double eps, c, a, rc, rc2, An, Bn, Am, Bm, ec;
    int n, m;
    float f_eps, f_a, f_rc, f_rc2, f_An, f_Bn, f_Am, f_Bm, f_ec;
    float f_ec2hq;  // (eps c)^2 m a^m / 2: B(rho) = f_ec2hq / w with w = m a^m B'(rho)
    int sc76;  // 1 when (n, m) == (7, 6): the fast specialised kernels apply
};

// FP32 constants of the pair terms, passed by value to the mixed-precision
// pair kernels: read from the kernel's constant bank at every use, they cost
// no load and no register inside the pair loops
struct PotF {
    float a, rc, rc2, Am, Bm, An, Bn, eps, ec;
    // force pass (the record's fourth component is w = m a^m B'(rho)):
    float an;    // a^n
    float am;    // a^m (density pass)
    float kn;    // eps n a^n
    float bmq;   // Bm / (m a^m)
    float ebn;   // eps Bn
    float c1;    // -(An / Bn + rc): phi_n(r) = a^n r^-n + Bn (r + c1)
    float fpsc;  // -eps c m a^m / 2: w = fpsc / sqrt(rho) (density pass)
    int n, m;
};

// slow-variable record of the coarse-step logic (FP64)
struct PtaDev {
    double v[3], R_t[3], R_tmD[3], R_tmh[3];
    double R3[3][3];  // means of the last three bursts, by slot
    double t;
    int has_tmh, init, jump[3], pad;
};

struct SpecCtl {
    int phase;       // Phase
    int parity;      // which position buffer is current
    int rebuild;     // 1: build the neighbour list before the next pair pass
    int err;         // sticky ErrBit mask
    long long nsteps, done;
    unsigned int blocks_done;  // last-block counter of the force kernel
    int list_L;                // lanes the current list layout was built for
    int rebuilds;              // list builds in the current burst
    int max_nn;                // largest neighbour count at the last build
    int prune;                 // 1: prune the inner list before the next pair pass
    int prunes;                // prunings in the current burst
    double sum[3];             // running sums of K, U, T over the burst (in step order)
    double sum_chk[3];         // adaptive length: running sums at the last check
    double conv_val[3];        // adaptive length: running average at convergence
    long long conv_n[3];       // adaptive length: step of convergence per variable
    int conv_mask;             // adaptive length: bit m set once variable m converged
    int relax;                 // 1: thermal relaxation, right grip free along the load axis
    double grip_du;            // continuous loading: the right grip moves this far (A) along
                               // the load axis with every step (0: held fixed)
    double eval_obs[3];        // K, U, T of the last MODE_EVAL pass
    double mb[8];              // scratch of the Maxwell-Boltzmann set-up
    pta_averages last;         // averages of the last finished burst
    PtaDev pta;
};

struct SpecDev {
    // sizes
    int n, L, prec, axis, cap;   // cap: list stride per unit (usable entries: cap_use)
    int cap_use;
    int blk_pair0, nblk_pair;  // pair kernels: TPB/L atoms per block
    int blk_atom0, nblk_atom;  // one thread per atom
    int blk_cell0, nblk_cell;  // cell sort: CELLS_PER_WARP cells per warp
    int spec_index;            // index of this specimen in the launch table
    // lattice (creation only)
    int ncl[3];
    double a0, grip_width;
    // cell grid
    double org[3];
    double hcell, inv_h;
    int nc[3];
    int ncell;
    // list radius (rc + skin)^2 and its FP32 bracket; half skin squared
    double rl2;
    float f_rl2_lo, f_rl2_hi, half_skin2, f_inv_h, f_h;
    float f_q, f_q8, f_q64;  // half the cell edge (unit of the list offsets), / 8, / 64
    float f_org[3];
    PotDev pot;
    // integration constants
    double mass, dt, acc_half, ke_fac, t_fac;
    float f_acc_half, f_ke_fac, f_dt;
    int block_steps;
    // coarse-step constants (Table 1)
    double pta_h, pta_Delta, tol_v[3], tol_j[3], floor_[3];
    // adaptive burst length (appendix): test every conv_lag steps (0 = off)
    int conv_lag;
    double conv_tol[3];
    // arrays
    void *pos[2];   // FP64: double4 {x,y,z,0};  MIXED: float4 hi {x,y,z,0}
    float4 *lo[2];  // MIXED only: float4 lo {x,y,z,0}
    void *posfp;    // FP64: double4 {x,y,z,F'(rho)};  MIXED: float4 {rel.xyz, F'(rho)}
    float4 *rel[2]; // MIXED only: position relative to the centre of its half-cell
                    // (FP32): the 16-byte record the pair passes read for a neighbour
    uint8_t *hsub;  // MIXED only: half-cell of each atom in its cell (bit d: upper half
                    // along axis d), fixed from one list build to the next
    void *vel;      // FP64: double4; MIXED: VelHL
    uint8_t *flags;
    float4 *ref;    // positions at the last list build (skin test)
    int *atom_cell, *cell_cnt, *cell_start, *cell_tmp, *cell_atoms;
    int *orig;        // original index (creation order) of the atom stored at each slot
    void *perm_tmp;   // scratch of the permutation that sorts atoms by cell
    int *nlist, *nn;
    int *plist, *pnn;   // inner list (same layout as nlist), entries per unit and lane
    float4 *pref;       // positions at the last pruning
    int prune_on;
    float f_rp2, half_prune2;
    double *part;       // per pair block: K, U, R, max displacement^2
    double *series;     // series_cap x 3 samples of the current burst
    long long series_cap;
    double *eval_out;   // n x 4: F, pe (MODE_EVAL)
    double *rsum;       // n x 4, creation order: sums of the sampled positions of the
                        // burst (Eq. (mean_pos)); null unless asked for
    double *stage;      // n x 6 doubles: import/export staging
    SpecCtl *ctl;
};

struct Group {
    int prec, L, sc76;
    PotF pf;  // the group's potential (specimens of one group share it)
    const int *b2s;
    int nblk;
};

// one launch table: the specimens and, per kernel kind, block->specimen maps
struct Tab {
    const SpecDev *specs;
    int nspec;
    const int *b2s_atom;
    int nblk_atom;
    const int *b2s_cell;
    int nblk_cell;
    int ngroups;
    Group grp[8];
};

// Verlet-list entry (one list per unit): neighbour index in the high 23
// bits, an offset (dx, dy, dz) in the low 9 bits, 3 bits per axis holding
// d + 3.  In mixed precision d is the offset of the neighbour's half-cell
// from the half-cell of the unit's first atom in units of h / 2 (within the
// 3x3x3 cells around a cell, |d| <= 3); with half-cell centres and h on
// exact grids, r_j - r_i = (rel_j - rel_i) + (h / 2) d.  FP64 lists keep
// whole-cell offsets, which its kernels do not read.
//
// Mixed-precision lists end, in every lane, with up to three sentinel
// entries that bring the lane's count to a multiple of four: they name slot
// n, a record kept far from every atom (SENTINEL_COORD on each axis), whose
// pairs lie beyond any cutoff, so the pair loops take four entries at a time
// without per-entry bounds tests.  Slot n must fit the index field: n < 2^23.
constexpr int NL_CODE_BITS = 9;
constexpr int MAX_ATOMS = 1 << 23;
constexpr float SENTINEL_COORD = 1.0e4f;

__host__ __device__ __forceinline__ unsigned nl_entry(int j, int dx, int dy, int dz) {
    return ((unsigned)j << NL_CODE_BITS) | (unsigned)((dx + 3) | ((dy + 3) << 3) | ((dz + 3) << 6));
}
__host__ __device__ __forceinline__ int nl_j(unsigned e) { return (int)(e >> NL_CODE_BITS); }
// the sentinel entry of a specimen of n atoms (slot n, offset 0)
__host__ __device__ __forceinline__ unsigned nl_sentinel(int n) { return nl_entry(n, 0, 0, 0); }

// index i of an array of n elements (debug builds: tested, 0 when outside)
__device__ __forceinline__ int chk_index(const SpecDev &S, int i, int n) {
#if PTA_CHECK
    if ((unsigned)i >= (unsigned)n) {
        atomicOr(&S.ctl->err, ERR_CHECK);
        return 0;
    }
#endif
    return i;
}

// the record a list entry names (mixed precision: an atom or the sentinel
// slot n)
__device__ __forceinline__ int nl_atom(const SpecDev &S, unsigned e) {
    return chk_index(S, nl_j(e), S.prec == PTA_PREC_FP64 ? S.n : S.n + 1);
}

// a count of list entries read by one lane (debug builds: at most `limit`)
__device__ __forceinline__ int chk_count(const SpecDev &S, int c, int limit) {
#if PTA_CHECK
    if (c < 0 || c > limit) {
        atomicOr(&S.ctl->err, ERR_CHECK);
        return c < 0 ? 0 : limit;
    }
#endif
    return c;
}

// an atom's force (debug builds: finite)
__device__ __forceinline__ void chk_force(const SpecDev &S, double fx, double fy, double fz) {
#if PTA_CHECK
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(&S.ctl->err, ERR_NAN);
#endif
    (void)S; (void)fx; (void)fy; (void)fz;
}

// The three offsets as exact FP32 multiples of the axis field, without
// integer conversion: OR-ing a field into the mantissa of 1.5 * 2^23
// (0x4B400000) gives 1.5 * 2^23 + field exactly.  x: (d + 3), y: 8 (d + 3),
// z: 64 (d + 3); the caller scales by h, h / 8 and h / 64.
__device__ __forceinline__ float nl_offx(unsigned e) {
    return __int_as_float(0x4B400000 | (int)(e & 0x7u)) - 12582915.0f;
}
__device__ __forceinline__ float nl_offy(unsigned e) {
    return __int_as_float(0x4B400000 | (int)(e & 0x38u)) - 12582936.0f;
}
__device__ __forceinline__ float nl_offz(unsigned e) {
    return __int_as_float(0x4B400000 | (int)(e & 0x1C0u)) - 12583104.0f;
}

// Cells are numbered along a serpentine path (x reverses on every other row,
// y on every other layer), so that consecutive cells are face neighbours and
// consecutive atoms of the cell-sorted order lie in the same or adjacent
// cells.
__host__ __device__ __forceinline__ int serp_rank(int n0, int n1, int x, int y, int z) {
    const int yr = (z & 1) ? n1 - 1 - y : y;
    const int t = z * n1 + yr;
    const int xr = (t & 1) ? n0 - 1 - x : x;
    return t * n0 + xr;
}
__host__ __device__ __forceinline__ void serp_coords(int n0, int n1, int r, int &x, int &y, int &z) {
    const int t = r / n0, xr = r % n0;
    z = t / n1;
    const int yr = t % n1;
    y = (z & 1) ? n1 - 1 - yr : yr;
    x = (t & 1) ? n0 - 1 - xr : xr;
}
__host__ __device__ __forceinline__ int cell_rank(const int nc[3], int x, int y, int z) {
    return serp_rank(nc[0], nc[1], x, y, z);
}
__host__ __device__ __forceinline__ void cell_coords(const int nc[3], int r, int &x, int &y, int &z) {
    serp_coords(nc[0], nc[1], r, x, y, z);
}

// centre of the cell of rank r (exact in FP32: org on a 2^-12 grid, h a
// multiple of 2^-11)
__device__ __forceinline__ float3 cell_centre(const SpecDev &S, int r) {
    int cx, cy, cz;
    cell_coords(S.nc, r, cx, cy, cz);
    return make_float3(S.f_org[0] + ((float)cx + 0.5f) * S.f_h,
                       S.f_org[1] + ((float)cy + 0.5f) * S.f_h,
                       S.f_org[2] + ((float)cz + 0.5f) * S.f_h);
}

// centre of half-cell `sub` of the cell of rank r: the cell centre moved by
// -h/4 or +h/4 per axis (exact in FP32: on a 2^-13 A grid)
__device__ __forceinline__ float3 half_centre(const SpecDev &S, int r, int sub) {
    float3 C = cell_centre(S, r);
    const float q = 0.25f * S.f_h;
    C.x += (sub & 1) ? q : -q;
    C.y += (sub & 2) ? q : -q;
    C.z += (sub & 4) ? q : -q;
    return C;
}
// the 3 half-cell bits spread onto the 3 offset fields of a list entry
__host__ __device__ __forceinline__ int sub_spread(int sub) {
    return (sub & 1) | ((sub & 2) << 2) | ((sub & 4) << 4);
}

// segments of the permutation scratch (see perm_layout)
struct PermLayout {
    size_t pos, lo, vel, flags, orig, cell, total;
};
__host__ __device__ inline size_t perm_round(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline PermLayout perm_layout(size_t n, int prec) {
    const size_t P = prec == PTA_PREC_FP64 ? 32 : 16;
    PermLayout L;
    size_t o = 0;
    L.pos = o;
    o += perm_round(P * n);
    L.lo = o;
    o += prec == PTA_PREC_FP64 ? 0 : perm_round(16 * n);
    L.vel = o;
    o += perm_round(32 * n);  // double4 or VelHL
    L.flags = o;
    o += perm_round(n);
    L.orig = o;
    o += perm_round(4 * n);
    L.cell = o;
    o += perm_round(4 * n);
    L.total = o;
    return L;
}

// Rows of a warp's list tile (L = 1: row k holds entry k of the warp's 32
// units) staged in shared memory and written to global memory as whole
// 128-byte rows once every lane has passed them; a lane that runs more than
// ROWS rows ahead of the flushed rows writes that entry and all its later
// ones directly.
template <int ROWS>
struct RowWriter {
    int *buf;   // shared [ROWS][32]
    int *tile;  // global word of row 0 of this warp's tile
    int lane, flushed, direct_from;
    __device__ __forceinline__ void put(int k, int e) {
        if (k < direct_from && k - flushed < ROWS) {
            buf[(k % ROWS) * 32 + lane] = e;
        } else {
            tile[(long long)k * 32 + lane] = e;
            direct_from = min(direct_from, k);
        }
    }
    // warp-collective: write rows [flushed, upto)
    __device__ __forceinline__ void flush(int upto) {
        for (int r = flushed; r < upto; ++r)
            if (r < direct_from) tile[(long long)r * 32 + lane] = buf[(r % ROWS) * 32 + lane];
        flushed = upto;
    }
};

// neighbour-list word of neighbour k of atom a for L lanes per atom: atoms
// are grouped 32/L per warp; for each iteration q = k / L the warp's 32
// words are contiguous, lane (a % (32/L)) * L + k % L.
__host__ __device__ __forceinline__ long long nl_base(int a, int L, int cap) {
    const int G = 32 / L;
    return (long long)(a / G) * (32LL * (cap / L)) + (a % G) * L;
}
__host__ __device__ __forceinline__ long long nl_index(int a, int k, int L, int cap) {
    return nl_base(a, L, cap) + (long long)(k / L) * 32 + (k % L);
}

// one block of SCAN_THREADS threads per specimen: exclusive scan of the cell
// counts into cell_start (cell_start[ncell] = total); the counts are reset to
// 0 for use as fill counters by a scatter; the specimen's build count + 1
__device__ __forceinline__ void scan_cells(const SpecDev &S) {
    __shared__ int wsum[SCAN_THREADS / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < S.ncell; base += SCAN_THREADS) {
        const int c = base + threadIdx.x;
        const int v = (c < S.ncell) ? S.cell_cnt[c] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const int excl = carry + (w ? wsum[w - 1] : 0) + x - v;
        if (c < S.ncell) {
            S.cell_start[c] = excl;
            S.cell_cnt[c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        S.cell_start[S.ncell] = carry;
        S.ctl->rebuilds += 1;
#if PTA_CHECK
        if (carry != S.n) atomicOr(&S.ctl->err, ERR_CHECK);  // every atom in one cell
#endif
    }
}

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// creation and state exchange, single specimen (d = device SpecDev)
void launch_create(const SpecDev &h, const SpecDev *d, double sigma_v, double kT, uint64_t seed,
                   cudaStream_t st);
void launch_import(const SpecDev &h, const SpecDev *d, cudaStream_t st);
void launch_export(const SpecDev &h, const SpecDev *d, cudaStream_t st);
void launch_fix_right_grip(const SpecDev &h, const SpecDev *d, cudaStream_t st);
// checkpoints: working state <-> permutation scratch in creation order
void launch_ckpt_move(const SpecDev &h, const SpecDev *d, int gather, cudaStream_t st);
// batched
void launch_strain(const Tab &t, const double *du, cudaStream_t st);
void launch_burst_begin(const Tab &t, const long long *nsteps, cudaStream_t st);
void launch_burst_end(const Tab &t, int slot, pta_averages *out, cudaStream_t st);
void launch_any_running(const Tab &t, int *flag, cudaStream_t st);
void launch_pta_update(const Tab &t, const int *ops, pta_coarse_result *out, cudaStream_t st);
void launch_force_rebuild_flag(const Tab &t, cudaStream_t st);
void launch_rebuild(const Tab &t, int force, cudaStream_t st);
void launch_prune(const Tab &t, int force, cudaStream_t st);
void launch_decide_rebuild(const Tab &t, cudaGraphConditionalHandle h, cudaStream_t st);
// list maintenance decided on the device: 0 build + prune, 1 prune, 2 nothing
constexpr unsigned LIST_BUILD = 0, LIST_PRUNE = 1, LIST_NONE = 2;

__device__ __forceinline__ bool prune_active(const SpecDev &S, int force) {
    if (!S.prune_on) return false;
    if (force) return true;
    return S.ctl->phase != PH_IDLE && S.ctl->prune != 0;
}
void launch_density(const Tab &t, int force, cudaStream_t st);
void launch_force(const Tab &t, int mode, cudaStream_t st);

}  // namespace pta
