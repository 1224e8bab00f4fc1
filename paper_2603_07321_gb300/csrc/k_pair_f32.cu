// Mixed-precision pair kernels on Verlet lists: Sutton-Chen EAM density and
// forces in FP32 on relative coordinates.  What a neighbour reads is one
// 16-byte record, its position relative to the centre C of its half-cell
// (one of the 8 octants of its cell, fixed at the list build),
// rel = (hi - C) + lo with |rel| <= h / 4 + skin / 2, so that with the
// half-cell offset d coded in the list entry
//     r_j - r_i = (rel_j - rel_i) + (h / 2) d
// (C and h on exact grids).  The one-lane loops take two entries per
// iteration (four in the density pass) and decode both offsets with packed
// FP32 instructions (two lanes of one instruction, sm_100 family); the
// density pass also forms both pair terms packed, then adds them to its sum
// in entry order.
//
// Pass 1 (density): rho_i = sum_j phi_m(r_ij), then B'(rho_i) =
// -eps c / (2 sqrt(rho_i)), stored beside the record scaled by m a^m (the
// force pass's pair terms are arranged around that weight).  Eq. (pe).
// Pass 2 (force):   F_i = sum_j [eps phi_n'(r) + (B'_i + B'_j) phi_m'(r)] (r_j - r_i)/r,
// Eq. (f_int), the per-atom energy 1/2 eps sum_j phi_n + B(rho_i), and the
// velocity-Verlet update fused behind it (atom_update_mixed).  Grip atoms
// keep v = 0 and F = 0 in the update; their internal force still enters the
// reaction R = -sum_{right grip} F . e of Eq. (state_variables).
#include "k_mixed.cuh"

namespace pta {

// Every lane's list ends with sentinel entries that bring its count to a
// multiple of four (they name a record far from every atom, so their pairs
// fail the cutoff test like any distant neighbour): the loops take four
// entries per iteration (two with several lanes per atom) without per-entry
// bounds tests, and read the next group's list words before evaluating the
// current one; those reads go past the count into the sixteen spare rows
// every list keeps and are never gathered.

// the entries lane l of atom u reads (the inner list when pruning is on, else
// the Verlet list), as a pointer to its first word (stride 32) and a count,
// rounded up to a multiple of four over the sentinel rows
__device__ __forceinline__ const unsigned *lane_list(const SpecDev &S, int u, int l, int L, int &cl) {
    const long long off = nl_base(u, L, S.cap) + l;
    if (S.prune_on) {
        cl = chk_count(S, S.pnn[(long long)u * L + l], S.cap_use / L + 4);
        return (const unsigned *)S.plist + off;
    }
    const int nn = S.nn[u];
    cl = chk_count(S, (nn > l ? (nn - l + L - 1) / L : 0), S.cap_use / L);
    cl = (cl + 3) & ~3;
    return (const unsigned *)S.nlist + off;
}

// one list word: read once per pass, so it skips L1 (the neighbour records
// keep the space) and asks L2 to fetch the 256-byte block around it, which
// holds the warp's next row as well
__device__ __forceinline__ unsigned ld_list(const unsigned *p) {
    unsigned v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// displacements of two entries from the atom, packed by axis
__device__ __forceinline__ void entry_disp2(unsigned ea, unsigned eb, float4 xa, float4 xb, float4 r0,
                                            float h, float h8, float h64, float2 &dx, float2 &dy,
                                            float2 &dz) {
    const float2 ox = __fadd2_rn(make_float2(__int_as_float(0x4B400000 | (int)(ea & 0x7u)),
                                             __int_as_float(0x4B400000 | (int)(eb & 0x7u))),
                                 f2(-12582915.0f));
    const float2 oy = __fadd2_rn(make_float2(__int_as_float(0x4B400000 | (int)(ea & 0x38u)),
                                             __int_as_float(0x4B400000 | (int)(eb & 0x38u))),
                                 f2(-12582936.0f));
    const float2 oz = __fadd2_rn(make_float2(__int_as_float(0x4B400000 | (int)(ea & 0x1C0u)),
                                             __int_as_float(0x4B400000 | (int)(eb & 0x1C0u))),
                                 f2(-12583104.0f));
    dx = __ffma2_rn(ox, f2(h), __fadd2_rn(make_float2(xa.x, xb.x), f2(-r0.x)));
    dy = __ffma2_rn(oy, f2(h8), __fadd2_rn(make_float2(xa.y, xb.y), f2(-r0.y)));
    dz = __ffma2_rn(oz, f2(h64), __fadd2_rn(make_float2(xa.z, xb.z), f2(-r0.z)));
}

// density terms of two entries, added in entry order
template <bool SC76>
__device__ __forceinline__ void rho_add2(const PotF &P, float2 dx, float2 dy, float2 dz,
                                         float &rho) {
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float rc2 = P.rc2;
    if (SC76) {
        const float2 phi = phi_m2_sc76(P, r2);
        if (r2.x < rc2) rho += phi.x;
        if (r2.y < rc2) rho += phi.y;
    } else {
        if (r2.x < rc2) rho += phi_m1<false>(P, r2.x);
        if (r2.y < rc2) rho += phi_m1<false>(P, r2.y);
    }
}

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB, 8) k_density_f32(const SpecDev *__restrict__ specs,
                                                        const int *__restrict__ b2s, int force,
                                                        const PotF P) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const SpecCtl *ctl = S.ctl;
    if (!force && ctl->phase == PH_IDLE) return;
    const int par = ctl->parity;
    constexpr int UPB = TPB / L;
    const int u = (blockIdx.x - S.blk_pair0) * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = u < S.n;
    const float4 *__restrict__ rel = S.rel[par];
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    float rho = 0.f;
    float4 ra = make_float4(0, 0, 0, 0);
    if (valid) {
        ra = rel[u];
        int cl;
        const unsigned *__restrict__ lst = lane_list(S, u, l, L, cl);
        if constexpr (L == 1) {
            unsigned e0 = ld_list(lst), e1 = ld_list(lst + 32), e2 = ld_list(lst + 64), e3 = ld_list(lst + 96);
            for (int q = 0; q < cl; q += 4) {
                const unsigned n0 = ld_list(lst + (q + 4) * 32), n1 = ld_list(lst + (q + 5) * 32);
                const unsigned n2 = ld_list(lst + (q + 6) * 32), n3 = ld_list(lst + (q + 7) * 32);
                const float4 x0 = __ldg(rel + nl_atom(S, e0)), x1 = __ldg(rel + nl_atom(S, e1));
                const float4 x2 = __ldg(rel + nl_atom(S, e2)), x3 = __ldg(rel + nl_atom(S, e3));
                float2 dx, dy, dz;
                entry_disp2(e0, e1, x0, x1, ra, h, h8, h64, dx, dy, dz);
                rho_add2<SC76>(P, dx, dy, dz, rho);
                entry_disp2(e2, e3, x2, x3, ra, h, h8, h64, dx, dy, dz);
                rho_add2<SC76>(P, dx, dy, dz, rho);
                e0 = n0; e1 = n1; e2 = n2; e3 = n3;
            }
        } else {
            unsigned ea = ld_list(lst), eb = ld_list(lst + 32);
            for (int q = 0; q < cl; q += 2) {
                const unsigned na = ld_list(lst + (q + 2) * 32), nb = ld_list(lst + (q + 3) * 32);
                const float4 xa = __ldg(rel + nl_atom(S, ea));
                const float4 xb = __ldg(rel + nl_atom(S, eb));
                float2 dx, dy, dz;
                entry_disp2(ea, eb, xa, xb, ra, h, h8, h64, dx, dy, dz);
                rho_add2<SC76>(P, dx, dy, dz, rho);
                ea = na;
                eb = nb;
            }
        }
    }
    rho = lane_sum<L>(rho);
    if (valid && l == 0) {
        // w = m a^m B'(rho), B'(rho) = -eps c / (2 sqrt(rho))
        const float fp = rho > 0.f ? P.fpsc * rsqrtf(rho) : 0.f;
        ((float4 *)S.posfp)[u] = make_float4(ra.x, ra.y, ra.z, fp);
    }
}

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB, 8) k_force_f32(const SpecDev *__restrict__ specs,
                                                      const int *__restrict__ b2s, int mode,
                                                      const PotF P) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    SpecCtl *ctl = S.ctl;
    const int phase = ctl->phase;
    if (mode == MODE_STEP && phase == PH_IDLE) return;
    const int par = ctl->parity;
    const long long done = ctl->done, nsteps = ctl->nsteps;
    constexpr int UPB = TPB / L;
    const int lb = blockIdx.x - S.blk_pair0;
    const int u = lb * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = u < S.n;
    const float4 *__restrict__ lf = (const float4 *)S.posfp;
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    const float rc2 = P.rc2;
    float fx = 0.f, fy = 0.f, fz = 0.f, e7 = 0.f, er = 0.f;
    float4 ra = make_float4(0, 0, 0, 0);
    if (valid) {
        ra = lf[u];
        int cl;
        const unsigned *__restrict__ lst = lane_list(S, u, l, L, cl);
        // the offsets of two entries decoded in packed instructions; the pair
        // terms stay scalar (packed, they measured slower here)
        auto two = [&](unsigned ea, unsigned eb, float4 xa, float4 xb) {
            float2 dx, dy, dz;
            entry_disp2(ea, eb, xa, xb, ra, h, h8, h64, dx, dy, dz);
            const float r2a = dx.x * dx.x + dy.x * dy.x + dz.x * dz.x;
            if (r2a < rc2)
                force_pair<SC76>(P, dx.x, dy.x, dz.x, r2a, ra.w + xa.w, fx, fy, fz, e7, er);
            const float r2b = dx.y * dx.y + dy.y * dy.y + dz.y * dz.y;
            if (r2b < rc2)
                force_pair<SC76>(P, dx.y, dy.y, dz.y, r2b, ra.w + xb.w, fx, fy, fz, e7, er);
        };
        if constexpr (L == 1) {
            unsigned e0 = ld_list(lst), e1 = ld_list(lst + 32), e2 = ld_list(lst + 64),
                     e3 = ld_list(lst + 96);
            for (int q = 0; q < cl; q += 4) {
                const unsigned n0 = ld_list(lst + (q + 4) * 32), n1 = ld_list(lst + (q + 5) * 32);
                const unsigned n2 = ld_list(lst + (q + 6) * 32), n3 = ld_list(lst + (q + 7) * 32);
                const float4 x0 = __ldg(lf + nl_atom(S, e0)), x1 = __ldg(lf + nl_atom(S, e1));
                const float4 x2 = __ldg(lf + nl_atom(S, e2)), x3 = __ldg(lf + nl_atom(S, e3));
                two(e0, e1, x0, x1);
                two(e2, e3, x2, x3);
                e0 = n0; e1 = n1; e2 = n2; e3 = n3;
            }
        } else {
            unsigned ea = ld_list(lst), eb = ld_list(lst + 32);
            for (int q = 0; q < cl; q += 2) {
                const unsigned na = ld_list(lst + (q + 2) * 32), nb = ld_list(lst + (q + 3) * 32);
                const float4 xa = __ldg(lf + nl_atom(S, ea));
                const float4 xb = __ldg(lf + nl_atom(S, eb));
                two(ea, eb, xa, xb);
                ea = na;
                eb = nb;
            }
        }
    }
    fx = lane_sum<L>(fx);
    fy = lane_sum<L>(fy);
    fz = lane_sum<L>(fz);
    const float en = lane_sum<L>(P.an * e7 + P.Bn * er);
    double ke = 0.0, pe = 0.0, rr = 0.0;
    float d2 = 0.f, dp2 = 0.f;
    if (valid && l == 0)
        atom_update_mixed(S, ctl, par, u, u, half_centre(S, S.atom_cell[u], S.hsub[u]), S.prune_on != 0,
                          ra.w, fx, fy, fz, en, mode, phase, done, nsteps, ke, pe, rr, d2, dp2);
    ke = warp_sum(ke);
    pe = warp_sum(pe);
    rr = warp_sum(rr);
    d2 = warp_max(d2);
    dp2 = warp_max(dp2);
    step_tail<TPB>(S, lb, S.nblk_pair, ke, pe, rr, (double)d2, (double)dp2, mode, phase, done,
                   nsteps);
}

// Inner list: every lane keeps, in order, the entries of its own column of
// the Verlet list that lie within the pruning radius of the atom (FP32
// distances tested against (rc + margin)^2 widened by 1e-5).  Pairs within
// rc are therefore all kept, in the order the lane sums them.  Sentinel
// entries then bring the lane's count to a multiple of four.
template <int L>
__global__ void __launch_bounds__(TPB, 7) k_prune_f32(const SpecDev *__restrict__ specs,
                                                      const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (S.prec == PTA_PREC_FP64 || !prune_active(S, force)) return;
    const SpecCtl *ctl = S.ctl;
    const int par = ctl->parity;
    constexpr int UPB = TPB / L;
    const int u = (blockIdx.x - S.blk_pair0) * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    if (u >= S.n) return;
    const float4 *__restrict__ rel = S.rel[par];
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64, rp2 = S.f_rp2;
    const float4 ra = rel[u];
    const long long off = nl_base(u, L, S.cap) + l;
    const unsigned *__restrict__ src = (const unsigned *)S.nlist + off;
    unsigned *__restrict__ dst = (unsigned *)S.plist + off;
    const int nn = S.nn[u];
    const int cl = chk_count(S, nn > l ? (nn - l + L - 1) / L : 0, S.cap_use / L);
    int kept = 0;
    // eight entries per iteration (eight gathers in flight), the next eight
    // words read ahead: rows up to cl + 14, within the spare iterations
    unsigned e[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) e[k] = ld_list(src + k * 32);
    for (int q = 0; q < cl; q += 8) {
        unsigned nx[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) nx[k] = ld_list(src + (q + 8 + k) * 32);
        float4 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __ldg(rel + nl_atom(S, e[k]));
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            float2 dx, dy, dz;
            entry_disp2(e[k], e[k + 1], x[k], x[k + 1], ra, h, h8, h64, dx, dy, dz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            if (q + k < cl && r2.x < rp2) dst[(kept++) * 32] = e[k];
            if (q + k + 1 < cl && r2.y < rp2) dst[(kept++) * 32] = e[k + 1];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) e[k] = nx[k];
    }
    {
        const unsigned sen = nl_sentinel(S.n);
        while (kept & 3) dst[(kept++) * 32] = sen;
    }
    S.pnn[(long long)u * L + l] = kept;
    if (l == 0) {
        const float4 hi = ((const float4 *)S.pos[par])[u];
        const float4 lo = S.lo[par][u];
        S.pref[u] = make_float4(hi.x + lo.x, hi.y + lo.y, hi.z + lo.z, 0.f);
    }
}

// after the pruning: clear the flag (a separate kernel, so that every block
// of the pruning kernel reads the same flag)
__global__ void k_prune_done(const SpecDev *__restrict__ specs, int force) {
    const SpecDev &S = specs[blockIdx.x];
    if (!prune_active(S, force)) return;
    if (threadIdx.x == 0) {
        S.ctl->prune = 0;
        S.ctl->prunes += 1;
    }
}

void launch_prune(const Tab &t, int force, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0 || g.prec == PTA_PREC_FP64) continue;
        switch (g.L) {
            case 1: k_prune_f32<1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
            case 2: k_prune_f32<2><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
            case 4: k_prune_f32<4><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
            case 8: k_prune_f32<8><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
            default: k_prune_f32<16><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
        }
    }
    k_prune_done<<<t.nspec, 32, 0, st>>>(t.specs, force);
}

// ---------------------------------------------------------------------------
// dispatch by (precision, lanes, potential variant)
// ---------------------------------------------------------------------------
void launch_density_f64(const Tab &t, const Group &g, int force, cudaStream_t st);
void launch_force_f64(const Tab &t, const Group &g, int mode, cudaStream_t st);

#define PTA_L_SWITCH(KER, SC)                                                            \
    switch (g.L) {                                                                       \
        case 1: KER<1, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg, g.pf); break;    \
        case 2: KER<2, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg, g.pf); break;    \
        case 4: KER<4, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg, g.pf); break;    \
        case 8: KER<8, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg, g.pf); break;    \
        default: KER<16, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg, g.pf); break;  \
    }

void launch_density(const Tab &t, int arg, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0) continue;
        if (g.prec == PTA_PREC_FP64)
            launch_density_f64(t, g, arg, st);
        else if (g.sc76)
            PTA_L_SWITCH(k_density_f32, true)
        else
            PTA_L_SWITCH(k_density_f32, false)
    }
}

void launch_force(const Tab &t, int arg, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0) continue;
        if (g.prec == PTA_PREC_FP64)
            launch_force_f64(t, g, arg, st);
        else if (g.sc76)
            PTA_L_SWITCH(k_force_f32, true)
        else
            PTA_L_SWITCH(k_force_f32, false)
    }
}

}  // namespace pta
