// Device pieces of the mixed-precision pair kernels: the FP32 pair terms of
// the Sutton-Chen EAM (Eqs. (pe), (f_int)), the exact hi/lo velocity pair,
// and the per-atom velocity-Verlet update of Eqs. (vv_algo_*) fused behind
// the force pass.
//
// Precision: pair terms in FP32 on relative coordinates; positions are an
// exact FP32 pair x = hi + lo (hi on a 2^-12 A grid, |lo| <= 2^-13 A);
// velocities an exact FP32 pair v = vh + vl (|vl| <= ulp(vh) / 2) updated by
// error-free addition, so that half-kicks lose nothing to rounding over long
// bursts; K, U and R are converted to FP64 per atom and reduced in FP64.
#pragma once

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

// packed FP32 (two lanes of one instruction), round to nearest
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsqrt2_nr(float2 r2) {
    // rsqrt_nr on both halves: y' = y + (-y/2) (r2 y y - 1), the same
    // operations and roundings as the scalar form
    const float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 e = __ffma2_rn(__fmul2_rn(r2, y), y, f2(-1.0f));
    return __ffma2_rn(__fmul2_rn(y, f2(-0.5f)), e, y);
}

// phi_m of two pairs at once (squared distances r2), for the density sum:
// with y = 1/r, phi_m = (a^m y^m - Am) + Bm (r - rc); the caller adds the
// halves whose r2 is below rc^2, in order
__device__ __forceinline__ float2 phi_m2_sc76(const PotF &P, float2 r2) {
    const float2 y = rsqrt2_nr(r2);
    const float2 y2 = __fmul2_rn(y, y);
    const float2 y3 = __fmul2_rn(y2, y);
    const float2 y6 = __fmul2_rn(y3, y3);
    const float2 u = __ffma2_rn(r2, y, f2(-P.rc));
    return __ffma2_rn(f2(P.Bm), u, __ffma2_rn(f2(P.am), y6, f2(-P.Am)));
}

// phi_m of one pair (r2 < rc^2)
template <bool SC76>
__device__ __forceinline__ float phi_m1(const PotF &P, float r2) {
    const float ir = rsqrt_nr(r2);
    const float s = P.a * ir;
    return PowF<SC76>::pm(s, P.m) - P.Am + P.Bm * (r2 * ir - P.rc);
}

// one pair's contribution to the force on the atom and to its pair-energy
// sums: displacement (ex, ey, ez) = r_j - r_i, r2 = |r_j - r_i|^2 < rc^2,
// q = w_i + w_j where each record carries w = m a^m B'(rho).  With y = 1/r,
//   [eps phi_n'(r) + (B'_i + B'_j) phi_m'(r)] / r
//       = y (eps Bn + q Bm / (m a^m)) - y^2 (eps n a^n y^n + q y^m),
// and phi_n(r) = a^n y^n + Bn (r + c1) with c1 = -(An / Bn + rc): the pass
// sums y^n into e7 and r + c1 into er (the constants applied once per atom)
template <bool SC76>
__device__ __forceinline__ void force_pair(const PotF &P, float ex, float ey, float ez, float r2,
                                           float q, float &fx, float &fy, float &fz, float &e7,
                                           float &er) {
    const float y = rsqrt_nr(r2);
    float yn, ym;
    PowF<SC76>::pw(y, P.n, P.m, yn, ym);
    const float t = fmaf(q, ym, P.kn * yn);
    const float c = fmaf(q, P.bmq, P.ebn);
    const float gg = y * fmaf(-y, t, c);
    fx += gg * ex;
    fy += gg * ey;
    fz += gg * ez;
    e7 += yn;
    er += fmaf(r2, y, P.c1);
}

// (h, l) += d exactly up to the final renormalisation: Knuth's two-sum of h
// and d, its error added to l, then h + l renormalised (fast two-sum, valid
// since |l| is far below |h + d| or both are tiny)
__device__ __forceinline__ void hl_add(float &h, float &l, float d) {
    const float s = h + d;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (d - bb);
    const float t = l + e;
    const float hh = s + t;
    l = t - (hh - s);
    h = hh;
}

// After the force pass of atom a (compact slot; force f, pair-energy sum
// en = sum_j phi_n(r_aj), record weight fpa = m a^m B'(rho_a)): its energy, its share of the reaction, and the
// velocity-Verlet update -- the half-kick that finishes the step (phase RUN),
// the sample of K, and unless the burst ends the half-kick and drift of the
// next step; the new position (hi + lo, whole grid quanta moved from lo to
// hi), its neighbour record (position relative to the reference point C,
// written at record index rec), and the displacements since the last list
// build (and, with `pruned`, since the last pruning).  Grip
// atoms keep v = 0.  MODE_EVAL stores F and the energy instead.
__device__ __forceinline__ void atom_update_mixed(const SpecDev &S, SpecCtl *ctl, int par, int a,
                                                  long long rec, float3 C, bool pruned, float fpa,
                                                  float fx, float fy, float fz, float en, int mode,
                                                  int phase, long long done, long long nsteps,
                                                  double &ke, double &pe, double &rr, float &d2,
                                                  float &dp2) {
    chk_force(S, fx, fy, fz);
    const float eps = S.pot.f_eps;
    const float pe_a = 0.5f * eps * en + (fpa != 0.f ? S.pot.f_ec2hq / fpa : 0.f);
    pe += (double)pe_a;
    const uint8_t flag = S.flags[a];
    if (flag == FLAG_RIGHT) rr -= (double)(S.axis == 0 ? fx : (S.axis == 1 ? fy : fz));
    VelHL *vp = (VelHL *)S.vel + a;
    VelHL v = *vp;
    if (mode == MODE_EVAL) {
        const float vx = v.h.x + v.l.x, vy = v.h.y + v.l.y, vz = v.h.z + v.l.z;
        ke += (double)(S.f_ke_fac * (vx * vx + vy * vy + vz * vz));
        double4_32a *o = (double4_32a *)S.eval_out;
        o[S.orig[a]] = make_double4_32a(fx, fy, fz, pe_a);
        return;
    }
    const float kh = S.f_acc_half;
    // thermal relaxation: the right grip moves along the load axis only (its
    // other velocity components stay 0, so the drift leaves them in place)
    const bool rfree = flag == FLAG_RIGHT && ctl->relax;
    const bool moves = flag == FLAG_MOBILE || rfree;
    const float kx = (flag == FLAG_MOBILE || (rfree && S.axis == 0)) ? fx * kh : 0.f;
    const float ky = (flag == FLAG_MOBILE || (rfree && S.axis == 1)) ? fy * kh : 0.f;
    const float kz = (flag == FLAG_MOBILE || (rfree && S.axis == 2)) ? fz * kh : 0.f;
    if (phase == PH_RUN) {
        if (moves) {
            hl_add(v.h.x, v.l.x, kx);
            hl_add(v.h.y, v.l.y, ky);
            hl_add(v.h.z, v.l.z, kz);
        }
        const float vx = v.h.x + v.l.x, vy = v.h.y + v.l.y, vz = v.h.z + v.l.z;
        ke += (double)(S.f_ke_fac * (vx * vx + vy * vy + vz * vz));
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
    // continuous loading (fine-dynamics verification): a fixed right grip
    // moves by grip_du along the load axis with every step's drift
    const float gdu = (start && flag == FLAG_RIGHT && !rfree) ? (float)ctl->grip_du : 0.f;
    if (start && (moves || gdu != 0.f)) {
        const float dt = S.f_dt;
        if (moves) {
            hl_add(v.h.x, v.l.x, kx);
            hl_add(v.h.y, v.l.y, ky);
            hl_add(v.h.z, v.l.z, kz);
            qq[0] += (v.h.x + v.l.x) * dt;
            qq[1] += (v.h.y + v.l.y) * dt;
            qq[2] += (v.h.z + v.l.z) * dt;
        } else {
            qq[S.axis] += gdu;
        }
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
    S.rel[par ^ 1][rec] = make_float4((hh[0] - C.x) + qq[0], (hh[1] - C.y) + qq[1],
                                      (hh[2] - C.z) + qq[2], 0.f);
    *vp = v;
    const float4 rf = S.ref[a];
    const float ex = (hh[0] - rf.x) + qq[0], ey = (hh[1] - rf.y) + qq[1],
                ez = (hh[2] - rf.z) + qq[2];
    d2 = fmaxf(d2, ex * ex + ey * ey + ez * ez);
    if (pruned) {
        const float4 pf = S.pref[a];
        const float px = (hh[0] - pf.x) + qq[0], py = (hh[1] - pf.y) + qq[1],
                    pz = (hh[2] - pf.z) + qq[2];
        dp2 = fmaxf(dp2, px * px + py * py + pz * pz);
    }
}

}  // namespace pta
