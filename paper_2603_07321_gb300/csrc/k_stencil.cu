// Lattice-stencil pair passes of the mixed-precision form.
//
// The specimen is an FCC crystal built site by site (problem-setup
// section), and while it deforms without losing its lattice, the atom j
// that is a neighbour of atom i sits at a fixed lattice offset v from i:
// v = site(j) - site(i), in units of a0 / 2 (integer, even component sum).
// Atoms are therefore kept in a fixed order (bricks of sites, ST_BK x ST_BY x
// ST_BZ) and their neighbour records in a padded 3-D array of rows -- rows of
// ncl[0] sites along x, one row per (Y, Z) in half lattice units -- so that
// the neighbour of atom i at offset v is the record at slot(i) + Delta(v),
// the same Delta for every atom of a row parity.  A warp's atoms then read
// runs of ST_BK consecutive records for every v, a block's neighbourhood is
// compact, and no neighbour list is stored, built or pruned.
//
// The stencil is the set of offsets v of every pair within the stencil
// radius rc + skin_s at the last check; a check runs whenever an atom has
// moved more than skin_s / 2 since the previous one (and at every burst
// start), so every pair within rc in between has its v in the stencil (the
// Verlet-skin argument).  Offsets whose pairs lie beyond rc contribute 0
// (r < rc strict, as everywhere), so the pair sums are those of Eqs. (pe)
// and (f_int) exactly.  A check that finds an offset beyond +-ST_R, or more
// than ST_KEYS offsets (the crystal has lost its lattice, e.g. by slip),
// moves the specimen to the neighbour-list scheme on the device, in the
// same fine step, before any pair pass uses the incomplete stencil.
//
// Records: rel = (hi - C) + lo with C = o + (X q_x, Y q_y, Z q_z) the site's
// reference point on a lattice refitted to the specimen's current extent at
// every check (q, o on the 2^-12 A grid, so C and the key offsets
// c_v = (v_x q_x, v_y q_y, v_z q_z) are exact in FP32); then
//     r_j - r_i = (rel_j - rel_i) + c_v.
// Slots outside the crystal hold a record far away (ST_FAR).
#include "k_mixed.cuh"

namespace pta {

__device__ __forceinline__ bool on_stencil(const SpecCtl *c) { return c->scheme == SCHEME_STENCIL; }

__device__ __forceinline__ bool st_active(const SpecDev &S, int force) {
    const SpecCtl *c = S.ctl;
    if (!S.stencil || c->scheme != SCHEME_STENCIL) return false;
    if (force) return true;
    return c->phase != PH_IDLE && c->rebuild != 0;
}

// site (k, Y, Z) of atom slot t; X = 2k + ((Y + Z) & 1)
__device__ __forceinline__ void st_site(const SpecDev &S, int t, int &k, int &Y, int &Z) {
    const int s = __ldg(S.st_sites + t);
    k = s & 1023;
    Y = (s >> 10) & 1023;
    Z = s >> 20;
}
__device__ __forceinline__ long long st_slot(const SpecDev &S, int k, int Y, int Z) {
    return ((long long)(Z + ST_R) * S.NYp + (Y + ST_R)) * S.NKp + (k + ST_PK);
}
// creation index (library atom order) of site (k, Y, Z)
__device__ __forceinline__ int st_cidx(const SpecDev &S, int k, int Y, int Z) {
    const int X = 2 * k + ((Y + Z) & 1);
    const int bx = X & 1, by = Y & 1, bz = Z & 1;
    const int b = (bx & by) ? 1 : ((bx & bz) ? 2 : ((by & bz) ? 3 : 0));
    return 4 * ((X >> 1) + S.ncl[0] * ((Y >> 1) + S.ncl[1] * (Z >> 1))) + b;
}
__device__ __forceinline__ float3 st_ref(const SpecCtl *c, int k, int Y, int Z) {
    const int X = 2 * k + ((Y + Z) & 1);
    return make_float3(c->st_o[0] + (float)X * c->st_q[0], c->st_o[1] + (float)Y * c->st_q[1],
                       c->st_o[2] + (float)Z * c->st_q[2]);
}

// order-preserving int of a float (for atomicMin / atomicMax)
__device__ __forceinline__ int f2ord(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// ---------------------------------------------------------------------------
// creation: row order, flags in row order, far records, initial frame
// ---------------------------------------------------------------------------
__global__ void k_st_flags_copy(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a < S.n) ((uint8_t *)S.perm_tmp)[a] = S.flags[a];
}

__global__ void k_st_order(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int t = blockIdx.x * TPB + threadIdx.x;
    if (t >= S.n) return;
    int k, Y, Z;
    st_site(S, t, k, Y, Z);
    const int a = st_cidx(S, k, Y, Z);
    S.orig[t] = a;
    S.flags[t] = ((const uint8_t *)S.perm_tmp)[a];
}

__global__ void k_st_fill(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const long long s = (long long)blockIdx.x * TPB + threadIdx.x;
    const float4 far = make_float4(ST_FAR, ST_FAR, ST_FAR, 0.f);
    if (s < S.nslot) {
        S.rel[0][s] = far;
        S.rel[1][s] = far;
        ((float4 *)S.posfp)[s] = far;
    }
    // spare far keys beyond any table (read ahead by the pair loops)
    if (s < 2 * ST_TAB)
        S.st_tab[s] = make_int4(0, __float_as_int(ST_FAR), 0, 0);
}

__global__ void k_st_init(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    if (threadIdx.x != 0) return;
    SpecCtl *c = S.ctl;
    c->scheme = SCHEME_STENCIL;
    c->rebuild = 1;
    for (int d = 0; d < 3; ++d) {
        c->st_q[d] = (float)(rint(0.5 * S.a0 * HI_SCALE) * HI_QUANTUM);
        c->st_o[d] = 0.f;
    }
}

void launch_stencil_order(const SpecDev &h, const SpecDev *d, cudaStream_t st) {
    const int nb = (h.n + TPB - 1) / TPB;
    k_st_flags_copy<<<nb, TPB, 0, st>>>(d);
    k_st_order<<<nb, TPB, 0, st>>>(d);
    const long long ns = std::max<long long>(h.nslot, 2LL * ST_TAB);
    k_st_fill<<<(unsigned)((ns + TPB - 1) / TPB), TPB, 0, st>>>(d);
    k_st_init<<<1, 32, 0, st>>>(d);
}

// ---------------------------------------------------------------------------
// check: refit the reference lattice, rewrite the records, bin the atoms,
// collect the offsets of all pairs within the radius, rebuild the tables
// ---------------------------------------------------------------------------
__global__ void k_st_box_reset(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!st_active(S, force) || threadIdx.x != 0) return;
    for (int d = 0; d < 3; ++d) {
        S.ctl->st_box[d] = f2ord(3.0e38f);
        S.ctl->st_box[3 + d] = f2ord(-3.0e38f);
    }
}

__global__ void k_st_box(const SpecDev *__restrict__ specs, const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!st_active(S, force)) return;
    const int t = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    const int par = S.ctl->parity;
    float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    if (t < S.n) {
        const float4 h = ((const float4 *)S.pos[par])[t];
        const float4 l = S.lo[par][t];
        const float x[3] = {h.x + l.x, h.y + l.y, h.z + l.z};
        for (int d = 0; d < 3; ++d) {
            mn[d] = x[d];
            mx[d] = x[d];
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        mn[d] = -warp_max(-mn[d]);
        mx[d] = warp_max(mx[d]);
    }
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d) {
            atomicMin(&S.ctl->st_box[d], f2ord(mn[d]));
            atomicMax(&S.ctl->st_box[3 + d], f2ord(mx[d]));
        }
}

// reference lattice from the extent: q_d spans the sites' extent 2 n_d - 1
// (half units) over the atoms' extent, o_d centres it; both on the 2^-12 A
// grid.  An empty or degenerate extent keeps the previous frame.
__global__ void k_st_frame(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!st_active(S, force) || threadIdx.x != 0) return;
    SpecCtl *c = S.ctl;
    for (int d = 0; d < 3; ++d) {
        const double lo = ord2f(c->st_box[d]), hi = ord2f(c->st_box[3 + d]);
        const int span = 2 * S.ncl[d] - 1;
        if (!(hi > lo) || span < 1) continue;
        const double q = rint((hi - lo) / span * HI_SCALE) * HI_QUANTUM;
        if (!(q > 0.0)) continue;
        const double o = rint((0.5 * (hi + lo) - 0.5 * span * q) * HI_SCALE) * HI_QUANTUM;
        c->st_q[d] = (float)q;
        c->st_o[d] = (float)o;
    }
}

// records relative to the refitted sites, skin reference positions, and the
// cell of every atom (counted for the scan)
__global__ void k_st_records(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                             int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!st_active(S, force)) return;
    const int t = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (t >= S.n) return;
    const SpecCtl *c = S.ctl;
    const int par = c->parity;
    int k, Y, Z;
    st_site(S, t, k, Y, Z);
    const float3 C = st_ref(c, k, Y, Z);
    const float4 h = ((const float4 *)S.pos[par])[t];
    const float4 l = S.lo[par][t];
    S.rel[par][st_slot(S, k, Y, Z)] =
        make_float4((h.x - C.x) + l.x, (h.y - C.y) + l.y, (h.z - C.z) + l.z, 0.f);
    const double x[3] = {(double)h.x + (double)l.x, (double)h.y + (double)l.y,
                         (double)h.z + (double)l.z};
    S.ref[t] = make_float4((float)x[0], (float)x[1], (float)x[2], 0.f);
    int ci[3];
    for (int d = 0; d < 3; ++d) {
        const int q = (int)floor((x[d] - S.org[d]) * S.inv_h);
        ci[d] = q < 0 ? 0 : (q >= S.nc[d] ? S.nc[d] - 1 : q);
    }
    const int cc = cell_rank(S.nc, ci[0], ci[1], ci[2]);
    S.atom_cell[t] = cc;
    atomicAdd(&S.cell_cnt[cc], 1);
}

__global__ void k_st_scan(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!st_active(S, force)) return;
    scan_cells(S);
}

__global__ void k_st_scatter(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                             int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!st_active(S, force)) return;
    const int t = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (t >= S.n) return;
    const int cc = S.atom_cell[t];
    S.cell_atoms[S.cell_start[cc] + atomicAdd(&S.cell_cnt[cc], 1)] = t;
}

// One thread per atom, atoms taken in cell order (the warp's lanes share a
// cell, so the 27-cell loop is uniform and each candidate's record is one
// broadcast read).  Every pair (i, j > i) within the radius (FP32 distance
// against the squared radius widened by 1e-5: a superset of the FP64 pairs)
// marks the offsets +v and -v; an offset beyond +-ST_R sets the error flag.
__global__ void __launch_bounds__(TPB) k_st_check(const SpecDev *__restrict__ specs,
                                                  const int *__restrict__ b2s, int force,
                                                  float r2_override) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!st_active(S, force)) return;
    __shared__ unsigned bits[ST_WORDS];
    __shared__ int bad;
    for (int w = threadIdx.x; w < ST_WORDS; w += TPB) bits[w] = 0u;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int u = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    const int par = S.ctl->parity;
    const float r2max = r2_override > 0.f ? r2_override : S.f_st_rl2;
    if (u < S.n) {
        const int i = S.cell_atoms[u];
        const float4 hi = ((const float4 *)S.pos[par])[i];
        const float4 li = S.lo[par][i];
        const float xi = hi.x + li.x, yi = hi.y + li.y, zi = hi.z + li.z;
        int ki, Yi, Zi;
        st_site(S, i, ki, Yi, Zi);
        const int Xi = 2 * ki + ((Yi + Zi) & 1);
        int cx, cy, cz;
        cell_coords(S.nc, S.atom_cell[i], cx, cy, cz);
        for (int zz = max(cz - 1, 0); zz <= min(cz + 1, S.nc[2] - 1); ++zz)
            for (int yy = max(cy - 1, 0); yy <= min(cy + 1, S.nc[1] - 1); ++yy)
                for (int xx = max(cx - 1, 0); xx <= min(cx + 1, S.nc[0] - 1); ++xx) {
                    const int cc = cell_rank(S.nc, xx, yy, zz);
                    const int s = S.cell_start[cc], e = S.cell_start[cc + 1];
                    for (int m = s; m < e; ++m) {
                        const int j = __ldg(S.cell_atoms + m);
                        if (j <= i) continue;
                        const float4 hj = __ldg((const float4 *)S.pos[par] + j);
                        const float4 lj = __ldg(S.lo[par] + j);
                        const float dx = (hj.x + lj.x) - xi, dy = (hj.y + lj.y) - yi,
                                    dz = (hj.z + lj.z) - zi;
                        if (dx * dx + dy * dy + dz * dz >= r2max) continue;
                        int kj, Yj, Zj;
                        st_site(S, j, kj, Yj, Zj);
                        const int vx = 2 * kj + ((Yj + Zj) & 1) - Xi, vy = Yj - Yi, vz = Zj - Zi;
                        if (vx < -ST_R || vx > ST_R || vy < -ST_R || vy > ST_R || vz < -ST_R ||
                            vz > ST_R) {
                            bad = 1;
                            continue;
                        }
                        const int b1 = ((vz + ST_R) * ST_SIDE + (vy + ST_R)) * ST_SIDE + (vx + ST_R);
                        const int b2 = ((ST_R - vz) * ST_SIDE + (ST_R - vy)) * ST_SIDE + (ST_R - vx);
                        if (!(bits[b1 >> 5] & (1u << (b1 & 31)))) atomicOr(&bits[b1 >> 5], 1u << (b1 & 31));
                        if (!(bits[b2 >> 5] & (1u << (b2 & 31)))) atomicOr(&bits[b2 >> 5], 1u << (b2 & 31));
                    }
                }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ST_WORDS; w += TPB)
        if (bits[w]) atomicOr(&S.st_bits[w], bits[w]);
    if (threadIdx.x == 0 && bad) atomicOr(&S.ctl->st_err, 1);
}

// One block per specimen: the offsets marked by the check, in bit order
// (v_z, then v_y, then v_x), become the two parity tables; the count is
// padded to a multiple of 4 with far keys.  Too wide or too many offsets:
// the specimen moves to the neighbour-list scheme (its list is built next,
// in the same fine step).  Clears the bitmap and the cell counters.
__global__ void k_st_table(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!st_active(S, force)) return;
    SpecCtl *c = S.ctl;
    __shared__ int wcount[ST_WORDS + 1];
    // exclusive scan of the per-word populations (one thread; ~300 words)
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < ST_WORDS; ++w) {
            wcount[w] = acc;
            acc += __popc(S.st_bits[w]);
        }
        wcount[ST_WORDS] = acc;
    }
    __syncthreads();
    const int nk = wcount[ST_WORDS];
    const bool fail = c->st_err != 0 || nk > ST_KEYS;
    if (!fail) {
        const float qx = c->st_q[0], qy = c->st_q[1], qz = c->st_q[2];
        const long long rowz = (long long)S.NYp * S.NKp;
        for (int w = threadIdx.x; w < ST_WORDS; w += blockDim.x) {
            unsigned m = S.st_bits[w];
            int idx = wcount[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int b = 32 * w + bit;
                const int vx = b % ST_SIDE - ST_R, vy = (b / ST_SIDE) % ST_SIDE - ST_R,
                          vz = b / (ST_SIDE * ST_SIDE) - ST_R;
                const int fl = (vx >= 0) ? vx / 2 : -((1 - vx) / 2);  // floor(vx / 2)
                const int d0 = (int)(vz * rowz + (long long)vy * S.NKp + fl);
                const int d1 = d0 + (vx & 1);
                const int cx = __float_as_int((float)vx * qx), cy = __float_as_int((float)vy * qy);
                const float cz = (float)vz * qz;
                S.st_tab[idx] = make_int4(d0, cx, cy, __float_as_int(cz));
                S.st_tab[ST_TAB + idx] = make_int4(d1, cx, cy, __float_as_int(cz));
                ++idx;
            }
        }
        const int nk4 = (nk + 3) & ~3;
        for (int k = nk + threadIdx.x; k < nk4 + 64 && k < ST_TAB; k += blockDim.x) {
            S.st_tab[k] = make_int4(0, __float_as_int(ST_FAR), 0, 0);
            S.st_tab[ST_TAB + k] = make_int4(0, __float_as_int(ST_FAR), 0, 0);
        }
        if (threadIdx.x == 0) {
            c->nkey = nk4;
            c->rebuild = 0;
        }
    } else if (threadIdx.x == 0) {
        c->scheme = SCHEME_LIST;  // lists from here on; rebuild stays set
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ST_WORDS; w += blockDim.x) S.st_bits[w] = 0u;
    for (int cc = threadIdx.x; cc < S.ncell; cc += blockDim.x) S.cell_cnt[cc] = 0;
    if (threadIdx.x == 0) c->st_checks += 1;
}

void launch_stencil_check(const Tab &t, int force, double rl2_override, cudaStream_t st) {
    const float r2o = rl2_override > 0.0 ? (float)(rl2_override * (1.0 + 1e-5)) : 0.f;
    k_st_box_reset<<<t.nspec, 32, 0, st>>>(t.specs, force);
    k_st_box<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_st_frame<<<t.nspec, 32, 0, st>>>(t.specs, force);
    k_st_records<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_st_scan<<<t.nspec, SCAN_THREADS, 0, st>>>(t.specs, force);
    k_st_scatter<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force);
    k_st_check<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, force, r2o);
    k_st_table<<<t.nspec, 256, 0, st>>>(t.specs, force);
}

// ---------------------------------------------------------------------------
// pair passes
// ---------------------------------------------------------------------------
// Lane l of an atom takes keys 2l, 2l + 1, 2l + 2L, ... (two per step); the
// next step's records and the keys of the step after are read before the
// current pair terms are evaluated.  Keys past the table's count (up to 64
// of them) are far keys (every lane reads its own record at a far offset),
// so the reads need no bounds tests.

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB, 8) k_st_density(const SpecDev *__restrict__ specs,
                                                       const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const SpecCtl *ctl = S.ctl;
    if (!on_stencil(ctl) || (!force && ctl->phase == PH_IDLE)) return;
    const int par = ctl->parity;
    constexpr int UPB = TPB / L;
    const int u = (blockIdx.x - S.blk_st0) * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = u < S.n;
    int k, Y, Z;
    st_site(S, valid ? u : S.n - 1, k, Y, Z);
    const long long ps = st_slot(S, k, Y, Z);
    const float4 *__restrict__ rec = S.rel[par] + ps;
    const int4 *__restrict__ tab = S.st_tab + (((Y + Z) & 1) ? ST_TAB : 0);
    const int nk = ctl->nkey;
    const float4 ri = rec[0];
    float rho = 0.f;
    int q = 2 * l;
    // keys two steps ahead, records one step ahead: no load waits on another
    // load of the same step
    int4 ta = __ldg(tab + q), tb = __ldg(tab + q + 1);
    float4 xa = __ldg(rec + ta.x), xb = __ldg(rec + tb.x);
    int4 na = __ldg(tab + q + 2 * L), nb = __ldg(tab + q + 2 * L + 1);
    for (; q < nk; q += 2 * L) {
        const float4 ya = __ldg(rec + na.x), yb = __ldg(rec + nb.x);
        const int4 ma = __ldg(tab + q + 4 * L), mb = __ldg(tab + q + 4 * L + 1);
        const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(xa.x, xb.x), f2(-ri.x)),
                                     make_float2(__int_as_float(ta.y), __int_as_float(tb.y)));
        const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(xa.y, xb.y), f2(-ri.y)),
                                     make_float2(__int_as_float(ta.z), __int_as_float(tb.z)));
        const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(xa.z, xb.z), f2(-ri.z)),
                                     make_float2(__int_as_float(ta.w), __int_as_float(tb.w)));
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float rc2 = S.pot.f_rc2;
        if (SC76) {
            if (r2.x < rc2 || r2.y < rc2) {
                const float2 phi = phi_m2_sc76(S.pot, r2);
                if (r2.x < rc2) rho += phi.x;
                if (r2.y < rc2) rho += phi.y;
            }
        } else {
            if (r2.x < rc2) rho += phi_m1<false>(S.pot, r2.x);
            if (r2.y < rc2) rho += phi_m1<false>(S.pot, r2.y);
        }
        ta = na;
        tb = nb;
        xa = ya;
        xb = yb;
        na = ma;
        nb = mb;
    }
    rho = lane_sum<L>(rho);
    if (valid && l == 0) {
        const float fp = rho > 0.f ? -0.5f * S.pot.f_ec * rsqrtf(rho) : 0.f;
        ((float4 *)S.posfp)[ps] = make_float4(ri.x, ri.y, ri.z, fp);
    }
}

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB, 6) k_st_force(const SpecDev *__restrict__ specs,
                                                     const int *__restrict__ b2s, int mode) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    SpecCtl *ctl = S.ctl;
    const int phase = ctl->phase;
    if (!on_stencil(ctl) || (mode == MODE_STEP && phase == PH_IDLE)) return;
    const int par = ctl->parity;
    const long long done = ctl->done, nsteps = ctl->nsteps;
    constexpr int UPB = TPB / L;
    const int lb = blockIdx.x - S.blk_st0;
    const int u = lb * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = u < S.n;
    int k, Y, Z;
    st_site(S, valid ? u : S.n - 1, k, Y, Z);
    const long long ps = st_slot(S, k, Y, Z);
    const float4 *__restrict__ rec = (const float4 *)S.posfp + ps;
    const int4 *__restrict__ tab = S.st_tab + (((Y + Z) & 1) ? ST_TAB : 0);
    const int nk = ctl->nkey;
    const float rc2 = S.pot.f_rc2;
    const float4 ri = rec[0];
    float fx = 0.f, fy = 0.f, fz = 0.f, en = 0.f;
    int q = 2 * l;
    int4 ta = __ldg(tab + q), tb = __ldg(tab + q + 1);
    float4 xa = __ldg(rec + ta.x), xb = __ldg(rec + tb.x);
    int4 na = __ldg(tab + q + 2 * L), nb = __ldg(tab + q + 2 * L + 1);
    for (; q < nk; q += 2 * L) {
        const float4 ya = __ldg(rec + na.x), yb = __ldg(rec + nb.x);
        const int4 ma = __ldg(tab + q + 4 * L), mb = __ldg(tab + q + 4 * L + 1);
        const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(xa.x, xb.x), f2(-ri.x)),
                                     make_float2(__int_as_float(ta.y), __int_as_float(tb.y)));
        const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(xa.y, xb.y), f2(-ri.y)),
                                     make_float2(__int_as_float(ta.z), __int_as_float(tb.z)));
        const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(xa.z, xb.z), f2(-ri.z)),
                                     make_float2(__int_as_float(ta.w), __int_as_float(tb.w)));
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        if (r2.x < rc2) force_pair<SC76>(S.pot, dx.x, dy.x, dz.x, r2.x, ri.w + xa.w, fx, fy, fz, en);
        if (r2.y < rc2) force_pair<SC76>(S.pot, dx.y, dy.y, dz.y, r2.y, ri.w + xb.w, fx, fy, fz, en);
        ta = na;
        tb = nb;
        xa = ya;
        xb = yb;
        na = ma;
        nb = mb;
    }
    fx = lane_sum<L>(fx);
    fy = lane_sum<L>(fy);
    fz = lane_sum<L>(fz);
    en = lane_sum<L>(en);
    double ke = 0.0, pe = 0.0, rr = 0.0;
    float d2 = 0.f, dp2 = 0.f;
    if (valid && l == 0)
        atom_update_mixed(S, ctl, par, u, ps, st_ref(ctl, k, Y, Z), false, ri.w, fx, fy, fz, en,
                          mode, phase, done, nsteps, ke, pe, rr, d2, dp2);
    ke = warp_sum(ke);
    pe = warp_sum(pe);
    rr = warp_sum(rr);
    d2 = warp_max(d2);
    step_tail<TPB>(S, lb, S.nblk_st, ke, pe, rr, (double)d2, 0.0, mode, phase, done, nsteps);
}

#define PTA_ST_SWITCH(KER, SC)                                                           \
    switch (g.L) {                                                                       \
        case 1: KER<1, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg); break;          \
        case 2: KER<2, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg); break;          \
        case 4: KER<4, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg); break;          \
        default: KER<8, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg); break;         \
    }

void launch_density_stencil(const Tab &t, const Group &g, int arg, cudaStream_t st) {
    if (g.sc76)
        PTA_ST_SWITCH(k_st_density, true)
    else
        PTA_ST_SWITCH(k_st_density, false)
}

void launch_force_stencil(const Tab &t, const Group &g, int arg, cudaStream_t st) {
    if (g.sc76)
        PTA_ST_SWITCH(k_st_force, true)
    else
        PTA_ST_SWITCH(k_st_force, false)
}

// ---------------------------------------------------------------------------
// the stencil's pairs within sqrt(rl2) as Verlet lists (pta_get_neighbours):
// one lane per atom, entries in key order, the FP64 list predicate
// ---------------------------------------------------------------------------
__global__ void k_st_list(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int t = blockIdx.x * TPB + threadIdx.x;
    if (t >= S.n || !on_stencil(S.ctl)) return;
    const int par = S.ctl->parity;
    int k, Y, Z;
    st_site(S, t, k, Y, Z);
    const long long ps = st_slot(S, k, Y, Z);
    const int4 *tab = S.st_tab + (((Y + Z) & 1) ? ST_TAB : 0);
    const float4 hi = ((const float4 *)S.pos[par])[t];
    const float4 li = S.lo[par][t];
    const double xi = (double)hi.x + (double)li.x, yi = (double)hi.y + (double)li.y,
                 zi = (double)hi.z + (double)li.z;
    const long long base = nl_base(t, 1, S.cap);
    int cnt = 0;
    for (int q = 0; q < S.ctl->nkey; ++q) {
        const int j = S.st_inv[ps + tab[q].x];
        if (j < 0 || j == t) continue;
        const float4 hj = ((const float4 *)S.pos[par])[j];
        const float4 lj = S.lo[par][j];
        const double dx = ((double)hj.x + (double)lj.x) - xi;
        const double dy = ((double)hj.y + (double)lj.y) - yi;
        const double dz = ((double)hj.z + (double)lj.z) - zi;
        const double r2 =
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (r2 < S.rl2) {
            if (cnt < S.cap_use) S.nlist[base + (long long)cnt * 32] = (int)((unsigned)j << NL_CODE_BITS);
            ++cnt;
        }
    }
    S.nn[t] = cnt < S.cap_use ? cnt : S.cap_use;
    atomicMax(&S.ctl->max_nn, cnt);
    if (cnt > S.cap_use) atomicOr(&S.ctl->err, ERR_OVERFLOW);
}

void launch_stencil_list(const SpecDev &h, const SpecDev *d, cudaStream_t st) {
    k_st_list<<<(h.n + TPB - 1) / TPB, TPB, 0, st>>>(d);
}

}  // namespace pta
