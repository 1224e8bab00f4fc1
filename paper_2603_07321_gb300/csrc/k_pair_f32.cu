// Mixed-precision pair kernels: Sutton-Chen EAM density and forces in FP32
// on relative coordinates.  Positions are kept as an exact FP32 pair
// x = hi + lo (hi on a 2^-12 A grid, |lo| <= 2^-13 A) for the integration;
// what a neighbour reads is one 16-byte record, the position relative to the
// centre C of its half-cell (one of the 8 octants of its cell, fixed at the
// list build), rel = (hi - C) + lo with |rel| <= h / 4 + skin / 2, so that
// with the half-cell offset d coded in the list entry
//     r_j - r_i = (rel_j - rel_i) + (h / 2) d
// (C and h on exact grids).  Velocities FP32; energies, stresses and time
// averages reduced in FP64.  The one-atom loops take two entries per
// iteration and decode both offsets with packed FP32 instructions (two
// lanes of one instruction, sm_100 family); the density pass also forms
// both pair terms packed, then adds them to its sum in entry order.
//
// Pass 1 (density): rho_i = sum_j phi_m(r_ij), then B'(rho_i) =
// -eps c / (2 sqrt(rho_i)) stored beside lo_i.  Eq. (pe).
// Pass 2 (force):   F_i = sum_j [eps phi_n'(r) + (B'_i + B'_j) phi_m'(r)] (r_j - r_i)/r,
// Eq. (f_int), the per-atom energy 1/2 eps sum_j phi_n + B(rho_i), and the
// velocity-Verlet update of Eqs. (vv_algo_*) fused behind it: the second
// half-kick that finishes the step, the sample of K, U, T, and (unless the
// burst ends) the first half-kick and drift of the next step.  Grip atoms
// keep v = 0 and F = 0 in the update; their internal force still enters the
// reaction R = -sum_{right grip} F . e of Eq. (state_variables).
#include "k_pair_common.cuh"

namespace pta {

template <bool SC76>
struct PowF {
    // s^m and s^n for the Sutton-Chen exponents
    __device__ __forceinline__ static void pw(float s, int n, int m, float &sn, float &sm) {
        if (SC76) {
            const float s2 = s * s, s3 = s2 * s;
            sm = s3 * s3;
            sn = sm * s;
        } else {
            float p = 1.f, q = 1.f;
            for (int i = 0; i < m; ++i) p *= s;
            for (int i = 0; i < n; ++i) q *= s;
            sm = p;
            sn = q;
        }
    }
    __device__ __forceinline__ static float pm(float s, int m) {
        if (SC76) {
            const float s2 = s * s, s3 = s2 * s;
            return s3 * s3;
        }
        float p = 1.f;
        for (int i = 0; i < m; ++i) p *= s;
        return p;
    }
};

// 1 / sqrt(r2): the hardware estimate refined by one Newton-Raphson step
// y' = y + y (1 - r2 y^2) / 2 (the residual formed with a fused multiply-add),
// which brings it to about one unit in the last place; the pair terms raise
// s = a / r to the 6th and 7th power, which multiplies its relative error
__device__ __forceinline__ float rsqrt_nr(float r2) {
    const float y = rsqrtf(r2);
    const float e = fmaf(-(r2 * y), y, 1.0f);
    return fmaf(0.5f * y, e, y);
}

// The unit of work is one atom (G = 1) or two atoms of one cell (G = 2)
// sharing one neighbour list (the union of their lists), handled by L lanes.
// For every entry the displacement from the unit's first atom is formed
// once; the second follows as d_1 = d_0 - (rel_1 - rel_0), which is exactly 0
// for the entry that is the second atom itself (then skipped).
//
// The entry loop is unrolled by two (by four in the one-atom density pass);
// the next two (four) entries are read before the current ones are
// evaluated.  Those reads go past a unit's count into the eight spare
// iterations every list keeps, whose entries are valid indices, so the loop
// carries no bounds tests.

// the entries lane l of unit u reads (the inner list when pruning is on, else
// the Verlet list), as a pointer to its first word (stride 32) and a count
__device__ __forceinline__ const unsigned *lane_list(const SpecDev &S, int u, int l, int L, int &cl) {
    const long long off = nl_base(u, L, S.cap) + l;
    if (S.prune_on) {
        cl = S.pnn[(long long)u * L + l];
        return (const unsigned *)S.plist + off;
    }
    const int nn = S.nn[u];
    cl = nn > l ? (nn - l + L - 1) / L : 0;
    return (const unsigned *)S.nlist + off;
}

// offset of a unit's second atom from its first: they share a cell, their
// half-cells may differ by h / 2 along an axis
__device__ __forceinline__ float3 unit_dg(const SpecDev &S, int a0, float4 r0, float4 r1) {
    const int s0 = S.hsub[a0], s1 = S.hsub[a0 + 1];
    const float q = S.f_q;
    return make_float3(fmaf((float)((s1 & 1) - (s0 & 1)), q, r1.x - r0.x),
                       fmaf((float)(((s1 >> 1) & 1) - ((s0 >> 1) & 1)), q, r1.y - r0.y),
                       fmaf((float)((s1 >> 2) - (s0 >> 2)), q, r1.z - r0.z));
}

// displacement of entry e's atom (record x) from the unit's first atom (record r0)
__device__ __forceinline__ float3 entry_disp(unsigned e, float4 x, float4 r0, float h, float h8,
                                             float h64) {
    return make_float3(fmaf(nl_offx(e), h, x.x - r0.x), fmaf(nl_offy(e), h8, x.y - r0.y),
                       fmaf(nl_offz(e), h64, x.z - r0.z));
}

// packed FP32 (two lanes of one instruction), round to nearest
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsqrt2_nr(float2 r2) {
    // rsqrt_nr on both halves: y' = y + (-y/2) (r2 y y - 1), the same
    // operations and roundings as the scalar form
    const float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 e = __ffma2_rn(__fmul2_rn(r2, y), y, f2(-1.0f));
    return __ffma2_rn(__fmul2_rn(y, f2(-0.5f)), e, y);
}
// displacements of two entries from the unit's first atom, packed by axis
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

template <int G, bool SC76>
struct DensityAcc {
    float rho[G];
    // one atom, the Sutton-Chen (7, 6) exponents: entries a and b (b only
    // when vb) in the two halves of packed instructions; the terms within rc
    // are added to the sum in entry order
    __device__ __forceinline__ void add2(const SpecDev &S, float2 dx, float2 dy, float2 dz, bool vb) {
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 ir = rsqrt2_nr(r2);
        const float2 s = __fmul2_rn(f2(S.pot.f_a), ir);
        const float2 s2 = __fmul2_rn(s, s);
        const float2 s3 = __fmul2_rn(s2, s);
        const float2 s6 = __fmul2_rn(s3, s3);
        const float2 u = __fadd2_rn(__fmul2_rn(r2, ir), f2(-S.pot.f_rc));
        const float2 phi = __ffma2_rn(f2(S.pot.f_Bm), u, __fadd2_rn(s6, f2(-S.pot.f_Am)));
        const float rc2 = S.pot.f_rc2;
        if (r2.x < rc2) rho[0] += phi.x;
        if (vb && r2.y < rc2) rho[0] += phi.y;
    }
    __device__ __forceinline__ void add(const SpecDev &S, float3 d, const float3 *dg, int ga) {
        const float rc2 = S.pot.f_rc2;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ex = d.x - dg[g].x, ey = d.y - dg[g].y, ez = d.z - dg[g].z;
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2 && (G == 1 || (r2 > 0.f && g < ga))) {
                const float ir = rsqrt_nr(r2);
                const float s = S.pot.f_a * ir;
                rho[g] += PowF<SC76>::pm(s, S.pot.m) - S.pot.f_Am + S.pot.f_Bm * (r2 * ir - S.pot.f_rc);
            }
        }
    }
};

template <int G, bool SC76>
struct ForceAcc {
    float fx[G], fy[G], fz[G], en[G];
    __device__ __forceinline__ void add(const SpecDev &S, float3 d, float fpj, const float3 *dg,
                                        const float4 *ra, int ga) {
        const float rc2 = S.pot.f_rc2;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ex = d.x - dg[g].x, ey = d.y - dg[g].y, ez = d.z - dg[g].z;
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2 && (G == 1 || (r2 > 0.f && g < ga))) {
                const float ir = rsqrt_nr(r2);
                const float r = r2 * ir;
                const float s = S.pot.f_a * ir;
                float sn, sm;
                PowF<SC76>::pw(s, S.pot.n, S.pot.m, sn, sm);
                const float dphn = -(float)S.pot.n * sn * ir + S.pot.f_Bn;
                const float dphm = -(float)S.pot.m * sm * ir + S.pot.f_Bm;
                const float gg = (S.pot.f_eps * dphn + (ra[g].w + fpj) * dphm) * ir;
                fx[g] += gg * ex;
                fy[g] += gg * ey;
                fz[g] += gg * ez;
                en[g] += sn - S.pot.f_An + S.pot.f_Bn * (r - S.pot.f_rc);
            }
        }
    }
};

// After the force pass of atom a (force f, energy sum en, F'(rho_a) = fpa):
// its energy, its share of the reaction, and the velocity-Verlet update --
// the half-kick that finishes the step (phase RUN), the sample of K, and
// unless the burst ends the half-kick and drift of the next step; the new
// position (hi + lo, whole grid quanta moved from lo to hi), its record
// relative to its cell centre, and the displacements since the last list
// build and pruning.  Grip atoms keep v = 0.  MODE_EVAL stores F and the
// energy instead.
__device__ __forceinline__ void atom_update(const SpecDev &S, SpecCtl *ctl, int par, int a,
                                            float fpa, float fx, float fy, float fz, float en,
                                            int mode, int phase, long long done, long long nsteps,
                                            float &ke, float &pe, float &rr, float &d2, float &dp2) {
    const float eps = S.pot.f_eps;
    const float pe_a = 0.5f * eps * en + (fpa != 0.f ? S.pot.f_ec2h / fpa : 0.f);
    pe += pe_a;
    const uint8_t flag = S.flags[a];
    if (flag == FLAG_RIGHT) rr -= (S.axis == 0 ? fx : (S.axis == 1 ? fy : fz));
    float4 v = ((const float4 *)S.vel)[a];
    if (mode == MODE_EVAL) {
        ke += S.f_ke_fac * (v.x * v.x + v.y * v.y + v.z * v.z);
        double4_32a *o = (double4_32a *)S.eval_out;
        o[S.orig[a]] = make_double4_32a(fx, fy, fz, pe_a);
        return;
    }
    const float kh = S.f_acc_half;
    // thermal relaxation: the right grip moves along the load axis only (its
    // other velocity components stay 0, so the drift leaves them in place)
    const bool rfree = flag == FLAG_RIGHT && ctl->relax;
    if (phase == PH_RUN) {
        if (flag == FLAG_MOBILE) {
            v.x += fx * kh;
            v.y += fy * kh;
            v.z += fz * kh;
        } else if (rfree) {
            if (S.axis == 0) v.x += fx * kh;
            else if (S.axis == 1) v.y += fy * kh;
            else v.z += fz * kh;
        }
        ke += S.f_ke_fac * (v.x * v.x + v.y * v.y + v.z * v.z);
    }
    const float4 hia = ((const float4 *)S.pos[par])[a];
    const float4 loa = S.lo[par][a];
    if (phase == PH_RUN && S.rsum) {
        // Eq. (mean_pos): the sampled state's position, hi + lo exactly
        double *rs = S.rsum + 4LL * S.orig[a];
        rs[0] = rs[0] + ((double)hia.x + (double)loa.x);
        rs[1] = rs[1] + ((double)hia.y + (double)loa.y);
        rs[2] = rs[2] + ((double)hia.z + (double)loa.z);
    }
    float hh[3] = {hia.x, hia.y, hia.z}, qq[3] = {loa.x, loa.y, loa.z};
    const bool start = (phase == PH_REFRESH) || (done + 1 < nsteps);
    if (start && (flag == FLAG_MOBILE || rfree)) {
        if (flag == FLAG_MOBILE) {
            v.x += fx * kh;
            v.y += fy * kh;
            v.z += fz * kh;
        } else if (S.axis == 0) {
            v.x += fx * kh;
        } else if (S.axis == 1) {
            v.y += fy * kh;
        } else {
            v.z += fz * kh;
        }
        const float dt = S.f_dt;
        qq[0] += v.x * dt;
        qq[1] += v.y * dt;
        qq[2] += v.z * dt;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // move whole grid quanta from lo to hi (both steps exact)
            const float sh = rintf(qq[d] * (float)HI_SCALE) * (float)HI_QUANTUM;
            hh[d] = hh[d] + sh;
            qq[d] = qq[d] - sh;
        }
        if (fabsf(hh[0]) > (float)MIXED_RANGE || fabsf(hh[1]) > (float)MIXED_RANGE ||
            fabsf(hh[2]) > (float)MIXED_RANGE)
            atomicOr(&ctl->err, ERR_RANGE);
    }
    ((float4 *)S.pos[par ^ 1])[a] = make_float4(hh[0], hh[1], hh[2], 0.f);
    S.lo[par ^ 1][a] = make_float4(qq[0], qq[1], qq[2], 0.f);
    const float3 C = half_centre(S, S.atom_cell[a], S.hsub[a]);
    S.rel[par ^ 1][a] = make_float4((hh[0] - C.x) + qq[0], (hh[1] - C.y) + qq[1],
                                    (hh[2] - C.z) + qq[2], 0.f);
    ((float4 *)S.vel)[a] = v;
    const float4 rf = S.ref[a];
    const float ex = (hh[0] - rf.x) + qq[0], ey = (hh[1] - rf.y) + qq[1],
                ez = (hh[2] - rf.z) + qq[2];
    d2 = fmaxf(d2, ex * ex + ey * ey + ez * ez);
    if (S.prune_on) {
        const float4 pf = S.pref[a];
        const float px = (hh[0] - pf.x) + qq[0], py = (hh[1] - pf.y) + qq[1],
                    pz = (hh[2] - pf.z) + qq[2];
        dp2 = fmaxf(dp2, px * px + py * py + pz * pz);
    }
}

template <int L, int G, bool SC76>
__global__ void __launch_bounds__(TPB, 8) k_density_f32(const SpecDev *__restrict__ specs,
                                                        const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const SpecCtl *ctl = S.ctl;
    if (!force && ctl->phase == PH_IDLE) return;
    const int par = ctl->parity;
    constexpr int UPB = TPB / L;
    const int u = (blockIdx.x - S.blk_pair0) * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = u < ctl->nunits;
    const float4 *__restrict__ rel = S.rel[par];
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    int a0 = 0, ga = 0;
    if (valid) unit_atoms(S, u, a0, ga);
    DensityAcc<G, SC76> acc;
    float4 ra[G];
    float3 dg[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc.rho[g] = 0.f;
        ra[g] = make_float4(0, 0, 0, 0);
        dg[g] = make_float3(0, 0, 0);
    }
    if (valid) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < ga) ra[g] = rel[a0 + g];
        if (G > 1 && ga > 1)  // both atoms share a cell: the offset is rel_1 - rel_0
            dg[1] = unit_dg(S, a0, ra[0], ra[1]);
        int cl;
        const unsigned *__restrict__ lst = lane_list(S, u, l, L, cl);
        if constexpr (G == 1 && SC76) {
            unsigned e0 = __ldg(lst), e1 = __ldg(lst + 32), e2 = __ldg(lst + 64), e3 = __ldg(lst + 96);
            for (int q = 0; q < cl; q += 4) {
                const unsigned n0 = __ldg(lst + (q + 4) * 32), n1 = __ldg(lst + (q + 5) * 32);
                const unsigned n2 = __ldg(lst + (q + 6) * 32), n3 = __ldg(lst + (q + 7) * 32);
                const float4 x0 = __ldg(rel + nl_j(e0)), x1 = __ldg(rel + nl_j(e1));
                const float4 x2 = __ldg(rel + nl_j(e2)), x3 = __ldg(rel + nl_j(e3));
                float2 dx, dy, dz;
                entry_disp2(e0, e1, x0, x1, ra[0], h, h8, h64, dx, dy, dz);
                acc.add2(S, dx, dy, dz, q + 1 < cl);
                if (q + 2 < cl) {
                    entry_disp2(e2, e3, x2, x3, ra[0], h, h8, h64, dx, dy, dz);
                    acc.add2(S, dx, dy, dz, q + 3 < cl);
                }
                e0 = n0; e1 = n1; e2 = n2; e3 = n3;
            }
        } else {
        unsigned ea = __ldg(lst), eb = __ldg(lst + 32);
        for (int q = 0; q < cl; q += 2) {
            const unsigned na = __ldg(lst + (q + 2) * 32), nb = __ldg(lst + (q + 3) * 32);
            const float4 xa = __ldg(rel + nl_j(ea));
            const float4 xb = __ldg(rel + nl_j(eb));
            if constexpr (G == 1 && SC76) {
                float2 dx, dy, dz;
                entry_disp2(ea, eb, xa, xb, ra[0], h, h8, h64, dx, dy, dz);
                acc.add2(S, dx, dy, dz, q + 1 < cl);
            } else {
                acc.add(S, entry_disp(ea, xa, ra[0], h, h8, h64), dg, ga);
                if (q + 1 < cl) acc.add(S, entry_disp(eb, xb, ra[0], h, h8, h64), dg, ga);
            }
            ea = na;
            eb = nb;
        }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) acc.rho[g] = lane_sum<L>(acc.rho[g]);
    if (valid && l == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= ga) continue;
            const float rho = acc.rho[g];
            const float fp = rho > 0.f ? -0.5f * S.pot.f_ec * rsqrtf(rho) : 0.f;
            ((float4 *)S.posfp)[a0 + g] = make_float4(ra[g].x, ra[g].y, ra[g].z, fp);
        }
    }
}

template <int L, int G, bool SC76>
__global__ void __launch_bounds__(TPB, G == 1 ? 9 : 8) k_force_f32(const SpecDev *__restrict__ specs,
                                                      const int *__restrict__ b2s, int mode) {
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
    const bool valid = u < ctl->nunits;
    const float4 *__restrict__ lf = (const float4 *)S.posfp;
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    int a0 = 0, ga = 0;
    if (valid) unit_atoms(S, u, a0, ga);
    ForceAcc<G, SC76> acc;
    float4 ra[G];
    float3 dg[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc.fx[g] = acc.fy[g] = acc.fz[g] = acc.en[g] = 0.f;
        ra[g] = make_float4(0, 0, 0, 0);
        dg[g] = make_float3(0, 0, 0);
    }
    if (valid) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < ga) ra[g] = lf[a0 + g];
        if (G > 1 && ga > 1)
            dg[1] = unit_dg(S, a0, ra[0], ra[1]);
        int cl;
        const unsigned *__restrict__ lst = lane_list(S, u, l, L, cl);
        unsigned ea = __ldg(lst), eb = __ldg(lst + 32);
        for (int q = 0; q < cl; q += 2) {
            const unsigned na = __ldg(lst + (q + 2) * 32), nb = __ldg(lst + (q + 3) * 32);
            const float4 xa = __ldg(lf + nl_j(ea));
            const float4 xb = __ldg(lf + nl_j(eb));
            if constexpr (G == 1) {
                // the offsets of both entries decoded in packed instructions;
                // the pair terms stay scalar (packed, they measured slower here)
                float2 dx, dy, dz;
                entry_disp2(ea, eb, xa, xb, ra[0], h, h8, h64, dx, dy, dz);
                acc.add(S, make_float3(dx.x, dy.x, dz.x), xa.w, dg, ra, ga);
                if (q + 1 < cl) acc.add(S, make_float3(dx.y, dy.y, dz.y), xb.w, dg, ra, ga);
            } else {
                acc.add(S, entry_disp(ea, xa, ra[0], h, h8, h64), xa.w, dg, ra, ga);
                if (q + 1 < cl) acc.add(S, entry_disp(eb, xb, ra[0], h, h8, h64), xb.w, dg, ra, ga);
            }
            ea = na;
            eb = nb;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc.fx[g] = lane_sum<L>(acc.fx[g]);
        acc.fy[g] = lane_sum<L>(acc.fy[g]);
        acc.fz[g] = lane_sum<L>(acc.fz[g]);
        acc.en[g] = lane_sum<L>(acc.en[g]);
    }
    float ke = 0.f, pe = 0.f, rr = 0.f, d2 = 0.f, dp2 = 0.f;
    if (valid && l == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= ga) continue;
            atom_update(S, ctl, par, a0 + g, ra[g].w, acc.fx[g], acc.fy[g], acc.fz[g], acc.en[g],
                        mode, phase, done, nsteps, ke, pe, rr, d2, dp2);
        }
    }
    ke = warp_sum(ke);
    pe = warp_sum(pe);
    rr = warp_sum(rr);
    d2 = warp_max(d2);
    dp2 = warp_max(dp2);
    step_tail<TPB>(S, lb, (double)ke, (double)pe, (double)rr, (double)d2, (double)dp2, mode, phase,
                   done, nsteps);
}

// Inner list: every lane keeps, in order, the entries of its own column of
// the Verlet list that lie within the pruning radius of an atom of the unit
// (FP32 distances tested against (rc + margin)^2 widened by 1e-5).  Pairs
// within rc are therefore all kept, in the order the lane sums them.
template <int L, int G>
__global__ void __launch_bounds__(TPB, 8) k_prune_f32(const SpecDev *__restrict__ specs,
                                                      const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (S.prec == PTA_PREC_FP64 || !prune_active(S, force)) return;
    const SpecCtl *ctl = S.ctl;
    const int par = ctl->parity;
    constexpr int UPB = TPB / L;
    const int u = (blockIdx.x - S.blk_pair0) * UPB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    if (u >= ctl->nunits) return;
    const float4 *__restrict__ rel = S.rel[par];
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64, rp2 = S.f_rp2;
    int a0, ga;
    unit_atoms(S, u, a0, ga);
    float4 ra[G];
    float3 dg[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        ra[g] = make_float4(0, 0, 0, 0);
        dg[g] = make_float3(0, 0, 0);
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
        if (g < ga) ra[g] = rel[a0 + g];
    if (G > 1 && ga > 1)
        dg[1] = unit_dg(S, a0, ra[0], ra[1]);
    const long long off = nl_base(u, L, S.cap) + l;
    const unsigned *__restrict__ src = (const unsigned *)S.nlist + off;
    unsigned *__restrict__ dst = (unsigned *)S.plist + off;
    const int nn = S.nn[u];
    int kept = 0;
    for (int q = 0; q * L + l < nn; ++q) {
        const unsigned e = __ldg(src + q * 32);
        const float4 x = __ldg(rel + nl_j(e));
        const float3 d = entry_disp(e, x, ra[0], h, h8, h64);
        bool in = false;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ex = d.x - dg[g].x, ey = d.y - dg[g].y, ez = d.z - dg[g].z;
            in |= (g < ga) && (ex * ex + ey * ey + ez * ez < rp2);
        }
        if (in) dst[(kept++) * 32] = e;
    }
    S.pnn[(long long)u * L + l] = kept;
    if (l == 0) {
        for (int g = 0; g < ga; ++g) {
            const int a = a0 + g;
            const float4 hi = ((const float4 *)S.pos[par])[a];
            const float4 lo = S.lo[par][a];
            S.pref[a] = make_float4(hi.x + lo.x, hi.y + lo.y, hi.z + lo.z, 0.f);
        }
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

// ---------------------------------------------------------------------------
// Cell tiles (mixed precision, one lane per atom)
// ---------------------------------------------------------------------------
// Block k of a specimen takes the occupied tiles k, k + nblk_pair, ... in
// turn.  For a staged tile the 16-byte records of the atoms of the 4x4x4
// cells around it are first copied into shared memory (cell by cell, one
// warp per cell), and its list entries are indices into that copy; the
// per-neighbour gathers are then shared-memory loads.  The tile's atoms are
// one contiguous range, one thread per atom.  Each atom sums its list in
// the same order and with the same arithmetic as the one-lane kernels above,
// so the per-atom results are identical; only the grouping of the per-block
// partials of K, U and R differs.

__device__ __forceinline__ void tile_stage(const int *__restrict__ T, const float4 *__restrict__ src,
                                           float4 *stg) {
    const int lane = threadIdx.x & 31;
    for (int hc = threadIdx.x >> 5; hc < TILE_HALO; hc += TILE_T / 32) {
        const int o = T[TT_OFF + hc], cnt = T[TT_OFF + hc + 1] - o, g = T[TT_START + hc];
        for (int i = lane; i < cnt; i += 32) stg[o + i] = __ldg(src + g + i);
    }
}

template <bool ST>
__device__ __forceinline__ float4 tile_rec(const float4 *__restrict__ glob, const float4 *stg,
                                           unsigned e) {
    if (ST) return stg[nl_j(e)];
    return __ldg(glob + nl_j(e));
}

template <bool SC76, bool ST>
__device__ __forceinline__ float tile_rho(const SpecDev &S, const float4 *__restrict__ rel,
                                          const float4 *stg, const unsigned *__restrict__ lst,
                                          int cl, float4 r0) {
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    const float3 dg0 = make_float3(0.f, 0.f, 0.f);
    DensityAcc<1, SC76> acc;
    acc.rho[0] = 0.f;
    unsigned ea = __ldg(lst), eb = __ldg(lst + 32);
    for (int q = 0; q < cl; q += 2) {
        const unsigned na = __ldg(lst + (q + 2) * 32), nb = __ldg(lst + (q + 3) * 32);
        const float4 xa = tile_rec<ST>(rel, stg, ea);
        const float4 xb = tile_rec<ST>(rel, stg, eb);
        if constexpr (SC76) {
            float2 dx, dy, dz;
            entry_disp2(ea, eb, xa, xb, r0, h, h8, h64, dx, dy, dz);
            acc.add2(S, dx, dy, dz, q + 1 < cl);
        } else {
            acc.add(S, entry_disp(ea, xa, r0, h, h8, h64), &dg0, 1);
            if (q + 1 < cl) acc.add(S, entry_disp(eb, xb, r0, h, h8, h64), &dg0, 1);
        }
        ea = na;
        eb = nb;
    }
    return acc.rho[0];
}

template <bool SC76, bool ST>
__device__ __forceinline__ void tile_force(const SpecDev &S, const float4 *__restrict__ lf,
                                           const float4 *stg, const unsigned *__restrict__ lst,
                                           int cl, float4 r0, ForceAcc<1, SC76> &acc) {
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64;
    const float3 dg0 = make_float3(0.f, 0.f, 0.f);
    unsigned ea = __ldg(lst), eb = __ldg(lst + 32);
    for (int q = 0; q < cl; q += 2) {
        const unsigned na = __ldg(lst + (q + 2) * 32), nb = __ldg(lst + (q + 3) * 32);
        const float4 xa = tile_rec<ST>(lf, stg, ea);
        const float4 xb = tile_rec<ST>(lf, stg, eb);
        float2 dx, dy, dz;
        entry_disp2(ea, eb, xa, xb, r0, h, h8, h64, dx, dy, dz);
        acc.add(S, make_float3(dx.x, dy.x, dz.x), xa.w, &dg0, &r0, 1);
        if (q + 1 < cl) acc.add(S, make_float3(dx.y, dy.y, dz.y), xb.w, &dg0, &r0, 1);
        ea = na;
        eb = nb;
    }
}

template <bool SC76>
__global__ void __launch_bounds__(TILE_T, 4) k_density_tile(const SpecDev *__restrict__ specs,
                                                            const int *__restrict__ b2s, int force) {
    extern __shared__ float4 stg[];
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const SpecCtl *ctl = S.ctl;
    if (!force && ctl->phase == PH_IDLE) return;
    const int par = ctl->parity;
    const float4 *__restrict__ rel = S.rel[par];
    const int nt = ctl->ntiles;
    for (int k = blockIdx.x - S.blk_pair0; k < nt; k += S.nblk_pair) {
        const int *__restrict__ T = S.tile_tab + (long long)__ldg(S.tile_list + k) * TT_STRIDE;
        const int a0 = __ldg(T + TT_A0), a1 = __ldg(T + TT_A1);
        const bool st = __ldg(T + TT_STAGED) != 0;
        if (st) {
            __syncthreads();
            tile_stage(T, rel, stg);
            __syncthreads();
        }
        for (int a = a0 + threadIdx.x; a < a1; a += TILE_T) {
            int cl;
            const unsigned *__restrict__ lst = lane_list(S, a, 0, 1, cl);
            const float4 r0 = rel[a];
            const float rho = st ? tile_rho<SC76, true>(S, rel, stg, lst, cl, r0)
                                 : tile_rho<SC76, false>(S, rel, stg, lst, cl, r0);
            const float fp = rho > 0.f ? -0.5f * S.pot.f_ec * rsqrtf(rho) : 0.f;
            ((float4 *)S.posfp)[a] = make_float4(r0.x, r0.y, r0.z, fp);
        }
    }
}

template <bool SC76>
__global__ void __launch_bounds__(TILE_T, 3) k_force_tile(const SpecDev *__restrict__ specs,
                                                          const int *__restrict__ b2s, int mode) {
    extern __shared__ float4 stg[];
    const SpecDev &S = specs[b2s[blockIdx.x]];
    SpecCtl *ctl = S.ctl;
    const int phase = ctl->phase;
    if (mode == MODE_STEP && phase == PH_IDLE) return;
    const int par = ctl->parity;
    const long long done = ctl->done, nsteps = ctl->nsteps;
    const int lb = blockIdx.x - S.blk_pair0;
    const float4 *__restrict__ lf = (const float4 *)S.posfp;
    const int nt = ctl->ntiles;
    float ke = 0.f, pe = 0.f, rr = 0.f, d2 = 0.f, dp2 = 0.f;
    for (int k = lb; k < nt; k += S.nblk_pair) {
        const int *__restrict__ T = S.tile_tab + (long long)__ldg(S.tile_list + k) * TT_STRIDE;
        const int a0 = __ldg(T + TT_A0), a1 = __ldg(T + TT_A1);
        const bool st = __ldg(T + TT_STAGED) != 0;
        if (st) {
            __syncthreads();
            tile_stage(T, lf, stg);
            __syncthreads();
        }
        for (int a = a0 + threadIdx.x; a < a1; a += TILE_T) {
            int cl;
            const unsigned *__restrict__ lst = lane_list(S, a, 0, 1, cl);
            const float4 r0 = lf[a];
            ForceAcc<1, SC76> acc;
            acc.fx[0] = acc.fy[0] = acc.fz[0] = acc.en[0] = 0.f;
            if (st)
                tile_force<SC76, true>(S, lf, stg, lst, cl, r0, acc);
            else
                tile_force<SC76, false>(S, lf, stg, lst, cl, r0, acc);
            atom_update(S, ctl, par, a, r0.w, acc.fx[0], acc.fy[0], acc.fz[0], acc.en[0], mode,
                        phase, done, nsteps, ke, pe, rr, d2, dp2);
        }
    }
    ke = warp_sum(ke);
    pe = warp_sum(pe);
    rr = warp_sum(rr);
    d2 = warp_max(d2);
    dp2 = warp_max(dp2);
    step_tail<TILE_T>(S, lb, (double)ke, (double)pe, (double)rr, (double)d2, (double)dp2, mode,
                      phase, done, nsteps);
}

// pruning of a tile's lists: the same test and order as k_prune_f32<1, 1>,
// with staged records; the row after the last kept entry gets a filler
__global__ void __launch_bounds__(TILE_T, 3) k_prune_tile(const SpecDev *__restrict__ specs,
                                                          const int *__restrict__ b2s, int force) {
    extern __shared__ float4 stg[];
    const SpecDev &S = specs[b2s[blockIdx.x]];
    if (!prune_active(S, force)) return;
    const SpecCtl *ctl = S.ctl;
    const int par = ctl->parity;
    const float4 *__restrict__ rel = S.rel[par];
    const float h = S.f_q, h8 = S.f_q8, h64 = S.f_q64, rp2 = S.f_rp2;
    const int nt = ctl->ntiles;
    for (int k = blockIdx.x - S.blk_pair0; k < nt; k += S.nblk_pair) {
        const int *__restrict__ T = S.tile_tab + (long long)__ldg(S.tile_list + k) * TT_STRIDE;
        const int a0 = __ldg(T + TT_A0), a1 = __ldg(T + TT_A1);
        const bool st = __ldg(T + TT_STAGED) != 0;
        if (st) {
            __syncthreads();
            tile_stage(T, rel, stg);
            __syncthreads();
        }
        for (int a = a0 + threadIdx.x; a < a1; a += TILE_T) {
            const float4 r0 = rel[a];
            const long long off = nl_base(a, 1, S.cap);
            const unsigned *__restrict__ src = (const unsigned *)S.nlist + off;
            unsigned *__restrict__ dst = (unsigned *)S.plist + off;
            const int nn = S.nn[a];
            int kept = 0;
            for (int q = 0; q < nn; ++q) {
                const unsigned e = __ldg(src + q * 32);
                const float4 x = st ? tile_rec<true>(rel, stg, e) : tile_rec<false>(rel, stg, e);
                const float3 d = entry_disp(e, x, r0, h, h8, h64);
                const float ex = d.x - 0.f, ey = d.y - 0.f, ez = d.z - 0.f;
                if (ex * ex + ey * ey + ez * ez < rp2) dst[(kept++) * 32] = e;
            }
            dst[kept * 32] = 0u;
            S.pnn[a] = kept;
            const float4 hi = ((const float4 *)S.pos[par])[a];
            const float4 lo = S.lo[par][a];
            S.pref[a] = make_float4(hi.x + lo.x, hi.y + lo.y, hi.z + lo.z, 0.f);
        }
    }
}

static constexpr size_t TILE_SMEM = (size_t)TILE_SC * sizeof(float4);

// opt the tile kernels into the dynamic shared memory they use (once)
int tile_kernels_init() {
    static int rc = -1;
    if (rc >= 0) return rc;
    const int b = (int)TILE_SMEM;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_density_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_density_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_force_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_force_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prune_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    rc = (e == cudaSuccess) ? 0 : 1;
    if (rc) cudaGetLastError();
    return rc;
}

void launch_prune(const Tab &t, int force, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0 || g.prec == PTA_PREC_FP64) continue;
        if (g.tiled) {
            k_prune_tile<<<g.nblk, TILE_T, TILE_SMEM, st>>>(t.specs, g.b2s, force);
        } else if (g.G == 2) {
            if (g.L == 1)
                k_prune_f32<1, 2><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force);
            else
                k_prune_f32<2, 2><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force);
        } else {
            switch (g.L) {
                case 1: k_prune_f32<1, 1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
                case 2: k_prune_f32<2, 1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
                case 4: k_prune_f32<4, 1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
                case 8: k_prune_f32<8, 1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
                default: k_prune_f32<16, 1><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, force); break;
            }
        }
    }
    k_prune_done<<<t.nspec, 32, 0, st>>>(t.specs, force);
}

// ---------------------------------------------------------------------------
// dispatch by (lanes, potential variant)
// ---------------------------------------------------------------------------
void launch_density_f64(const Tab &t, const Group &g, int force, cudaStream_t st);
void launch_force_f64(const Tab &t, const Group &g, int mode, cudaStream_t st);

#define PTA_LAUNCH(KER, ...)                                                         \
    do {                                                                             \
        KER<__VA_ARGS__><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, arg);               \
    } while (0)

#define PTA_LG_SWITCH(KER)                                                           \
    if (g.G == 2) {                                                                  \
        switch (g.L) {                                                               \
            case 1: PTA_LAUNCH(KER, 1, 2, SC76); break;                              \
            default: PTA_LAUNCH(KER, 2, 2, SC76); break;                             \
        }                                                                            \
    } else {                                                                         \
        switch (g.L) {                                                               \
            case 1: PTA_LAUNCH(KER, 1, 1, SC76); break;                              \
            case 2: PTA_LAUNCH(KER, 2, 1, SC76); break;                              \
            case 4: PTA_LAUNCH(KER, 4, 1, SC76); break;                              \
            case 8: PTA_LAUNCH(KER, 8, 1, SC76); break;                              \
            default: PTA_LAUNCH(KER, 16, 1, SC76); break;                            \
        }                                                                            \
    }

template <bool SC76>
static void density_f32(const Tab &t, const Group &g, int arg, cudaStream_t st) {
    PTA_LG_SWITCH(k_density_f32)
}

template <bool SC76>
static void force_f32(const Tab &t, const Group &g, int arg, cudaStream_t st) {
    PTA_LG_SWITCH(k_force_f32)
}

void launch_density(const Tab &t, int force, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0) continue;
        if (g.prec == PTA_PREC_FP64)
            launch_density_f64(t, g, force, st);
        else if (g.tiled && g.sc76)
            k_density_tile<true><<<g.nblk, TILE_T, TILE_SMEM, st>>>(t.specs, g.b2s, force);
        else if (g.tiled)
            k_density_tile<false><<<g.nblk, TILE_T, TILE_SMEM, st>>>(t.specs, g.b2s, force);
        else if (g.sc76)
            density_f32<true>(t, g, force, st);
        else
            density_f32<false>(t, g, force, st);
    }
}

void launch_force(const Tab &t, int mode, cudaStream_t st) {
    for (int i = 0; i < t.ngroups; ++i) {
        const Group &g = t.grp[i];
        if (g.nblk <= 0) continue;
        if (g.prec == PTA_PREC_FP64)
            launch_force_f64(t, g, mode, st);
        else if (g.tiled && g.sc76)
            k_force_tile<true><<<g.nblk, TILE_T, TILE_SMEM, st>>>(t.specs, g.b2s, mode);
        else if (g.tiled)
            k_force_tile<false><<<g.nblk, TILE_T, TILE_SMEM, st>>>(t.specs, g.b2s, mode);
        else if (g.sc76)
            force_f32<true>(t, g, mode, st);
        else
            force_f32<false>(t, g, mode, st);
    }
}

}  // namespace pta
