// Cell binning by counting sort and Verlet-list construction.
//
// The list of atom i holds every j != i with |r_j - r_i|^2 < (rc + skin)^2,
// the squared distance formed as (dx*dx + dy*dy) + dz*dz in FP64 without
// contraction.  Candidates come from the 27 cells around i's cell on a grid
// of edge >= rc + skin; atoms outside the grid are clamped onto its border
// cells, which keeps every pair within reach (clamping is non-expansive), and
// are reported (PTA_ERANGE): the grid's margin is a quarter of the specimen's
// extent, which no atom of a deforming specimen reaches.
// After binning, the atoms themselves are permuted into cell order (cells in
// rank order, atoms of a cell in creation order), so that
// the 32 atoms of a warp share a cell and read overlapping neighbours, and a
// cell's atoms are one contiguous range.  The list order (cell order, then
// slot) is therefore a function of positions and grid: builds are
// deterministic.  orig[] keeps each slot's creation-order index.
//
// The list is rebuilt only when the force kernel found an atom that moved
// more than skin/2 since the last build (or on request); every kernel here
// returns at once for a specimen that needs no build.
#include "pta_dev.cuh"

namespace pta {

__device__ __forceinline__ bool build_active(const SpecDev &S, int force) {
    const SpecCtl *c = S.ctl;
    if (force) return true;
    if (c->phase == PH_IDLE) return false;
    return c->rebuild != 0 || c->list_L != S.L;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// position of atom a in FP64 (exact value of the stored representation)
__device__ __forceinline__ void load_pos64(const SpecDev &S, int par, int a, double &x, double &y,
                                           double &z) {
    if (S.prec == PTA_PREC_FP64) {
        const double4_32a q = ((const double4_32a *)S.pos[par])[a];
        x = q.x;
        y = q.y;
        z = q.z;
    } else {
        const float4 h = ((const float4 *)S.pos[par])[a];
        const float4 l = S.lo[par][a];
        x = (double)h.x + (double)l.x;
        y = (double)h.y + (double)l.y;
        z = (double)h.z + (double)l.z;
    }
}

__global__ void k_bin(const SpecDev *__restrict__ specs, const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int a = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int par = S.ctl->parity;
    double x[3];
    load_pos64(S, par, a, x[0], x[1], x[2]);
    int ci[3];
    bool out = false;
    for (int d = 0; d < 3; ++d) {
        const double q = floor((x[d] - S.org[d]) * S.inv_h);
        out |= !(q >= 0.0 && q < (double)S.nc[d]);
        ci[d] = clampi((int)fmax(fmin(q, 1e9), -1e9), 0, S.nc[d] - 1);
    }
    if (out) atomicOr(&S.ctl->err, ERR_GRID);
    const int c = cell_rank(S.nc, ci[0], ci[1], ci[2]);
    S.atom_cell[a] = c;
    atomicAdd(&S.cell_cnt[c], 1);
}

// one block per specimen: exclusive scan of the cell counts; counts reset to
// 0 for use as fill counters by the scatter
__global__ void k_scan(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!build_active(S, force)) return;
    scan_cells(S);
}

__global__ void k_scatter(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                          int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int a = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int c = S.atom_cell[a];
    const int slot = chk_index(S, S.cell_start[c] + atomicAdd(&S.cell_cnt[c], 1), S.n);
    S.cell_tmp[slot] = a;
}

// each warp orders CELLS_PER_WARP cells in turn (most cells of the grid's
// margin are empty): a cell's atoms by creation index (rank = number of
// smaller ones), so that the order within a cell, and with it every list
// order, does not depend on how cells are numbered; then the cell's counter
// is cleared for the next build
__global__ void k_cell_sort(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                            int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int lane = threadIdx.x & 31;
    const int c0 = (blockIdx.x - S.blk_cell0) * CELL_WARPS * CELLS_PER_WARP + (threadIdx.x >> 5);
    for (int i = 0; i < CELLS_PER_WARP; ++i) {
        const int c = c0 + i * CELL_WARPS;
        if (c >= S.ncell) return;
        const int s = S.cell_start[c], e = S.cell_start[c + 1];
        for (int p = s + lane; p < e; p += 32) {
            const int v = chk_index(S, S.cell_tmp[chk_index(S, p, S.n)], S.n);
            const int ov = S.orig[v];
            int r = 0;
            for (int q = s; q < e; ++q) r += (S.orig[chk_index(S, S.cell_tmp[chk_index(S, q, S.n)], S.n)] < ov);
            S.cell_atoms[chk_index(S, s + r, S.n)] = v;
        }
        if (lane == 0) S.cell_cnt[c] = 0;
    }
}

// sort the per-atom state into cell order: gather into scratch, then copy back
__global__ void k_permute_gather(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                                 int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int p = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (p >= S.n) return;
    const int src = chk_index(S, S.cell_atoms[p], S.n);
    const int par = S.ctl->parity;
    const PermLayout Lo = perm_layout(S.n, S.prec);
    char *t = (char *)S.perm_tmp;
    // velocities: 32-byte records in both precisions (double4 or VelHL)
    ((double4_32a *)(t + Lo.vel))[p] = ((const double4_32a *)S.vel)[src];
    if (S.prec == PTA_PREC_FP64) {
        ((double4_32a *)(t + Lo.pos))[p] = ((const double4_32a *)S.pos[par])[src];
    } else {
        ((float4 *)(t + Lo.pos))[p] = ((const float4 *)S.pos[par])[src];
        ((float4 *)(t + Lo.lo))[p] = S.lo[par][src];
    }
    ((uint8_t *)(t + Lo.flags))[p] = S.flags[src];
    ((int *)(t + Lo.orig))[p] = S.orig[src];
    ((int *)(t + Lo.cell))[p] = S.atom_cell[src];
}

__global__ void k_permute_scatter(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                                  int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int p = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (p >= S.n) return;
    const int par = S.ctl->parity;
    const PermLayout Lo = perm_layout(S.n, S.prec);
    const char *t = (const char *)S.perm_tmp;
    ((double4_32a *)S.vel)[p] = ((const double4_32a *)(t + Lo.vel))[p];
    if (S.prec == PTA_PREC_FP64) {
        ((double4_32a *)S.pos[par])[p] = ((const double4_32a *)(t + Lo.pos))[p];
    } else {
        ((float4 *)S.pos[par])[p] = ((const float4 *)(t + Lo.pos))[p];
        S.lo[par][p] = ((const float4 *)(t + Lo.lo))[p];
    }
    S.flags[p] = ((const uint8_t *)(t + Lo.flags))[p];
    S.orig[p] = ((const int *)(t + Lo.orig))[p];
    S.atom_cell[p] = ((const int *)(t + Lo.cell))[p];
}

// mixed precision: every atom's half-cell in its new cell, its neighbour
// record relative to that half-cell's centre (read by the pruning and the
// first density pass), and in the scratch posfp its position relative to
// the cell centre with the half-cell bits, spread onto the offset fields, in
// w (read by the list build, which tests candidates cell by cell)
__global__ void k_rel_all(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                          int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (S.prec == PTA_PREC_FP64 || !build_active(S, force)) return;
    const int a = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int par = S.ctl->parity;
    const float4 h = ((const float4 *)S.pos[par])[a];
    const float4 l = S.lo[par][a];
    const int c = S.atom_cell[a];
    const float3 C = cell_centre(S, c);
    const float cx = (h.x - C.x) + l.x, cy = (h.y - C.y) + l.y, cz = (h.z - C.z) + l.z;
    const int sub = (cx >= 0.f ? 1 : 0) | (cy >= 0.f ? 2 : 0) | (cz >= 0.f ? 4 : 0);
    S.hsub[a] = (uint8_t)sub;
    ((float4 *)S.posfp)[a] = make_float4(cx, cy, cz, __int_as_float(sub_spread(sub)));
    const float3 R = half_centre(S, c, sub);
    S.rel[par][a] = make_float4((h.x - R.x) + l.x, (h.y - R.y) + l.y, (h.z - R.z) + l.z, 0.f);
}

constexpr int RW_ROWS = 48;

// exact list predicate between atoms a and j (FP32 first; the FP64 test
// decides only the thin band around the list radius)
__device__ __forceinline__ bool in_list(const SpecDev &S, int par, bool mixed, int a, double xa,
                                        double ya, double za, float4 ha, float4 la, int j) {
    if (mixed) {
        const float4 hj = ((const float4 *)S.pos[par])[j];
        const float4 lj = S.lo[par][j];
        const float fx = (hj.x - ha.x) + (lj.x - la.x);
        const float fy = (hj.y - ha.y) + (lj.y - la.y);
        const float fz = (hj.z - ha.z) + (lj.z - la.z);
        const float r2f = fx * fx + fy * fy + fz * fz;
        if (r2f < S.f_rl2_lo) return true;
        if (r2f >= S.f_rl2_hi) return false;
        const double ddx = ((double)hj.x + (double)lj.x) - xa;
        const double ddy = ((double)hj.y + (double)lj.y) - ya;
        const double ddz = ((double)hj.z + (double)lj.z) - za;
        const double r2 =
            __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
        return r2 < S.rl2;
    }
    const double4_32a q = ((const double4_32a *)S.pos[par])[j];
    const double ddx = q.x - xa, ddy = q.y - ya, ddz = q.z - za;
    const double r2 =
        __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
    return r2 < S.rl2;
}

// one thread per atom (per lane group): every j != i within the list radius,
// gathered from the 27 cells around the atom's cell in (z, y, x) order, each
// cell's atoms in slot order
__global__ void __launch_bounds__(TPB) k_build(const SpecDev *__restrict__ specs,
                                               const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!build_active(S, force)) return;
    const int u = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    const int par = S.ctl->parity;
    int cnt = 0;
    if (S.L == 1 && S.prec != PTA_PREC_FP64) {
        // warp-uniform loop over the 27 cells around each atom's cell; the
        // FP32 candidate test uses the cell-relative records, the FP64 test
        // decides the thin band around the list radius; list rows are staged
        // in shared memory and written whole
        __shared__ int rowbuf[TPB / 32][RW_ROWS * 32];
        const int lane = threadIdx.x & 31;
        const bool valid = u < S.n;
        const int a = valid ? u : 0;
        RowWriter<RW_ROWS> wr;
        wr.buf = rowbuf[threadIdx.x >> 5];
        wr.tile = S.nlist + nl_base(u - lane, 1, S.cap);
        wr.lane = lane;
        wr.flushed = 0;
        wr.direct_from = 1 << 30;
        // filler rows hold entry 0: a valid index both of the atoms and of a
        // staged halo
        for (int r = 0; r < RW_ROWS; ++r) wr.buf[r * 32 + lane] = 0;
        __syncwarp();
        // cell-relative records with the spread half-cell bits in w (k_rel_all)
        const float4 *__restrict__ crec = (const float4 *)S.posfp;
        const float4 ra = crec[a];
        const int own_sub = __float_as_int(ra.w);
        const float4 ha = ((const float4 *)S.pos[par])[a];
        const float4 la = S.lo[par][a];
        const double xa = (double)ha.x + (double)la.x, ya = (double)ha.y + (double)la.y,
                     za = (double)ha.z + (double)la.z;
        const int ca = S.atom_cell[a];
        int cx, cy, cz;
        cell_coords(S.nc, ca, cx, cy, cz);
        const float h = S.f_h;
        // a warp past the last atom writes nothing: its tile lies beyond the
        // list (and the rows every lane has passed are unbounded)
        const bool wvalid = __any_sync(0xffffffffu, valid);
        for (int dz = -1; dz <= 1 && wvalid; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = cx + dx, yy = cy + dy, zz = cz + dz;
                    const bool inside = valid && xx >= 0 && yy >= 0 && zz >= 0 && xx < S.nc[0] &&
                                        yy < S.nc[1] && zz < S.nc[2];
                    if (inside) {
                        const int cc = cell_rank(S.nc, xx, yy, zz);
                        const int s = chk_count(S, S.cell_start[cc], S.n), e = chk_count(S, S.cell_start[cc + 1], S.n);
                        // half-cell offset 2d + sub_j - sub_a: add the spread bits of j
                        const unsigned code = nl_entry(0, 2 * dx, 2 * dy, 2 * dz) - (unsigned)own_sub;
                        // position of atom a relative to the centre of cell cc
                        const float ox = ra.x - (float)dx * h, oy = ra.y - (float)dy * h,
                                    oz = ra.z - (float)dz * h;
                        auto test = [&](int j, const float4 rj) {
                            const float fx = rj.x - ox, fy = rj.y - oy, fz = rj.z - oz;
                            const float r2f = fx * fx + fy * fy + fz * fz;
                            bool in;
                            if (r2f < S.f_rl2_lo)
                                in = true;
                            else if (r2f >= S.f_rl2_hi)
                                in = false;
                            else
                                in = in_list(S, par, true, a, xa, ya, za, ha, la, j);
                            if (in && j != a) {
                                if (cnt < S.cap_use)
                                    wr.put(cnt, (int)(((unsigned)j << NL_CODE_BITS) +
                                                      code + (unsigned)__float_as_int(rj.w)));
                                ++cnt;
                            }
                        };
                        // four candidates per iteration, their records loaded
                        // before any is tested; tested in slot order
                        int j = s;
                        for (; j + 4 <= e; j += 4) {
                            const float4 r0 = crec[j], r1 = crec[j + 1], r2 = crec[j + 2],
                                         r3 = crec[j + 3];
                            test(j, r0);
                            test(j + 1, r1);
                            test(j + 2, r2);
                            test(j + 3, r3);
                        }
                        for (; j < e; ++j) test(j, crec[j]);
                    }
                    wr.flush(min(__reduce_min_sync(0xffffffffu, valid ? min(cnt, S.cap_use) : 1 << 30),
                                 wr.flushed + RW_ROWS));
                }
        const int top = __reduce_max_sync(0xffffffffu, valid ? min(cnt, S.cap_use) : 0);
        if (wvalid) wr.flush(top);
        if (valid) {
            // four sentinel rows after the last entry: the pair loops read
            // the list in groups of four (within the sixteen spare rows)
            const unsigned sen = nl_sentinel(S.n);
            const int c0 = min(cnt, S.cap_use);
            for (int r = 0; r < 4; ++r) wr.tile[(long long)(c0 + r) * 32 + lane] = (int)sen;
            S.nn[u] = cnt < S.cap_use ? cnt : S.cap_use;
            S.ref[a] = make_float4((float)xa, (float)ya, (float)za, 0.f);
        }
    } else if (u < S.n) {
        const bool mixed = S.prec != PTA_PREC_FP64;
        const int a = u;
        double x, y, z;
        load_pos64(S, par, a, x, y, z);
        float4 ha = make_float4(0, 0, 0, 0), la = make_float4(0, 0, 0, 0);
        if (mixed) {
            ha = ((const float4 *)S.pos[par])[a];
            la = S.lo[par][a];
        }
        int cx, cy, cz;
        cell_coords(S.nc, S.atom_cell[a], cx, cy, cz);
        const long long base = nl_base(u, S.L, S.cap);
        const int L = S.L;
        // mixed: half-cell offsets from the atom's half-cell
        const int sub0 = mixed ? sub_spread(S.hsub[a]) : 0;
        for (int zz = max(cz - 1, 0); zz <= min(cz + 1, S.nc[2] - 1); ++zz)
            for (int yy = max(cy - 1, 0); yy <= min(cy + 1, S.nc[1] - 1); ++yy)
                for (int xx = max(cx - 1, 0); xx <= min(cx + 1, S.nc[0] - 1); ++xx) {
                    const int cc = cell_rank(S.nc, xx, yy, zz);
                    const int s = chk_count(S, S.cell_start[cc], S.n), e = chk_count(S, S.cell_start[cc + 1], S.n);
                    const unsigned code =
                        mixed ? nl_entry(0, 2 * (xx - cx), 2 * (yy - cy), 2 * (zz - cz)) -
                                    (unsigned)sub0
                              : nl_entry(0, xx - cx, yy - cy, zz - cz);
                    if (mixed) {
                        // the candidate test on the cell-relative records (as in
                        // the one-lane path), the FP64 test for the thin band
                        const float4 *__restrict__ crec = (const float4 *)S.posfp;
                        const float4 ra = crec[a];
                        const float h = S.f_h;
                        const float ox = ra.x - (float)(xx - cx) * h,
                                    oy = ra.y - (float)(yy - cy) * h,
                                    oz = ra.z - (float)(zz - cz) * h;
                        for (int j = s; j < e; ++j) {
                            const float4 rj = crec[j];
                            const float fx = rj.x - ox, fy = rj.y - oy, fz = rj.z - oz;
                            const float r2f = fx * fx + fy * fy + fz * fz;
                            bool in;
                            if (r2f < S.f_rl2_lo)
                                in = true;
                            else if (r2f >= S.f_rl2_hi)
                                in = false;
                            else
                                in = in_list(S, par, true, a, x, y, z, ha, la, j);
                            if (in && j != a) {
                                if (cnt < S.cap_use)
                                    S.nlist[base + (long long)(cnt / L) * 32 + (cnt % L)] =
                                        (int)(((unsigned)j << NL_CODE_BITS) + code +
                                              (unsigned)__float_as_int(rj.w));
                                ++cnt;
                            }
                        }
                        continue;
                    }
                    for (int j = s; j < e; ++j) {
                        if (j != a && in_list(S, par, false, a, x, y, z, ha, la, j)) {
                            if (cnt < S.cap_use)
                                S.nlist[base + (long long)(cnt / L) * 32 + (cnt % L)] =
                                    (int)(((unsigned)j << NL_CODE_BITS) + code);
                            ++cnt;
                        }
                    }
                }
        const int c0 = cnt < S.cap_use ? cnt : S.cap_use;
        if (mixed) {
            // four sentinel entries per lane after the last entry (the pair
            // loops read each lane's column in groups of four)
            const unsigned sen = nl_sentinel(S.n);
            for (int k = c0; k < c0 + 4 * L; ++k)
                S.nlist[base + (long long)(k / L) * 32 + (k % L)] = (int)sen;
        }
        S.nn[u] = c0;
        S.ref[a] = make_float4((float)x, (float)y, (float)z, 0.f);
    }
    // block maximum of the counts, one atomic per block
    __shared__ int smax[TPB / 32];
    int m = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < TPB / 32; ++w) m = max(m, smax[w]);
        m = max(m, smax[0]);
        atomicMax(&S.ctl->max_nn, m);
        if (m > S.cap_use) atomicOr(&S.ctl->err, ERR_OVERFLOW);
    }
}

// after the build: record the layout the list was built for (a separate
// kernel, so that the gate above reads the same value in every block)
__global__ void k_build_done(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!build_active(S, force)) return;
    if (threadIdx.x == 0) {
        S.ctl->list_L = S.L;
        S.ctl->prune = 1;  // a fresh list is always pruned before use
    }
}

__global__ void k_reset_maxnn(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!build_active(S, force)) return;
    if (threadIdx.x == 0) S.ctl->max_nn = 0;
}

// one block: does any specimen of the table need a list build, or only a
// pruning of its inner list, before its next pair pass?  Sets the condition
// of the graph node that holds that work (LIST_BUILD, LIST_PRUNE, LIST_NONE).
__global__ void k_decide_rebuild(const SpecDev *__restrict__ specs, int nspec,
                                 cudaGraphConditionalHandle handle) {
    int build = 0, prune = 0;
    for (int s = threadIdx.x; s < nspec; s += blockDim.x) {
        build |= build_active(specs[s], 0);
        prune |= prune_active(specs[s], 0);
    }
    build = __syncthreads_or(build);
    prune = __syncthreads_or(prune);
    if (threadIdx.x == 0)
        cudaGraphSetConditional(handle, build ? LIST_BUILD : (prune ? LIST_PRUNE : LIST_NONE));
}

void launch_decide_rebuild(const Tab &t, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_decide_rebuild<<<1, 128, 0, st>>>(t.specs, t.nspec, h);
}

void launch_rebuild(const Tab &t, int force, cudaStream_t st) {
    k_reset_maxnn<<<t.nspec, 32, 0, st>>>(t.specs, force);
    k_bin<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_scan<<<t.nspec, SCAN_THREADS, 0, st>>>(t.specs, force);
    k_scatter<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_cell_sort<<<t.nblk_cell, CELL_WARPS * 32, 0, st>>>(t.specs, t.b2s_cell, force);
    k_permute_gather<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_permute_scatter<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_rel_all<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_build<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_build_done<<<t.nspec, 32, 0, st>>>(t.specs, force);
}

}  // namespace pta
