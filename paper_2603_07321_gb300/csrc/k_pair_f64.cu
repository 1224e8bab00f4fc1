// FP64 pair kernels: the same two passes as the mixed-precision kernels
// (density, then forces with the fused velocity-Verlet epilogue), with every
// quantity in double.  They serve the plain FP64 form of the method and the
// parity checks against the FP64 oracle.
//
// The pair terms are arranged around y = 1/r from one reciprocal square root
// (CUDA's rsqrt on double), so that no pair needs a division or a square
// root: r = r2 y, s = a y, phi_k'(r) / r = (-k s^k y + B_k) y.  FP64 runs at
// a small fraction of the FP32 rate on this GPU, and a double division or
// square root costs several fused multiply-adds each.
#include "k_pair_common.cuh"

namespace pta {

__device__ __forceinline__ double ipow(double s, int k) {
    double p = 1.0;
    for (int i = 0; i < k; ++i) p *= s;
    return p;
}

// s^m and s^n (Sutton-Chen exponents; SC76: n = 7, m = 6)
template <bool SC76>
__device__ __forceinline__ void pow_nm(double s, int n, int m, double &sn, double &sm) {
    if (SC76) {
        const double s3 = (s * s) * s;
        sm = s3 * s3;
        sn = sm * s;
    } else {
        sn = ipow(s, n);
        sm = ipow(s, m);
    }
}

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB) k_density_f64(const SpecDev *__restrict__ specs,
                                                     const int *__restrict__ b2s, int force) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const SpecCtl *ctl = S.ctl;
    if (!force && ctl->phase == PH_IDLE) return;
    const int par = ctl->parity;
    constexpr int APB = TPB / L;
    const int a = (blockIdx.x - S.blk_pair0) * APB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = a < S.n;
    const double4_32a *__restrict__ pos = (const double4_32a *)S.pos[par];
    const PotDev &P = S.pot;
    double rho = 0.0;
    double4_32a pa = make_double4_32a(0, 0, 0, 0);
    if (valid) {
        pa = pos[a];
        const int nn = chk_count(S, S.nn[a], S.cap_use);
        const int *__restrict__ lst = S.nlist + nl_base(a, L, S.cap);
        for (int k = l; k < nn; k += L) {
            const int j = nl_atom(S, (unsigned)lst[(k / L) * 32 + (k % L)]);
            const double4_32a pj = pos[j];
            const double dx = pj.x - pa.x, dy = pj.y - pa.y, dz = pj.z - pa.z;
            const double r2 = (dx * dx + dy * dy) + dz * dz;
            // tested on r2 (the reciprocal square root only for pairs within
            // rc), so that coincident atoms (r2 = 0) still give a non-finite
            // result rather than no pair
            if (r2 < P.rc * P.rc) {
                const double y = rsqrt(r2);
                const double r = r2 * y;
                double sn, sm;
                pow_nm<SC76>(P.a * y, P.n, P.m, sn, sm);
                rho += sm - P.Am + P.Bm * (r - P.rc);
            }
        }
    }
    rho = lane_sum<L>(rho);
    if (valid && l == 0) {
        const double fp = rho > 0.0 ? -P.ec / (2.0 * sqrt(rho)) : 0.0;
        ((double4_32a *)S.posfp)[a] = make_double4_32a(pa.x, pa.y, pa.z, fp);
    }
}

template <int L, bool SC76>
__global__ void __launch_bounds__(TPB) k_force_f64(const SpecDev *__restrict__ specs,
                                                   const int *__restrict__ b2s, int mode) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    SpecCtl *ctl = S.ctl;
    const int phase = ctl->phase;
    if (mode == MODE_STEP && phase == PH_IDLE) return;
    const int par = ctl->parity;
    const long long done = ctl->done, nsteps = ctl->nsteps;
    constexpr int APB = TPB / L;
    const int lb = blockIdx.x - S.blk_pair0;
    const int a = lb * APB + threadIdx.x / L;
    const int l = threadIdx.x % L;
    const bool valid = a < S.n;
    const double4_32a *__restrict__ pf = (const double4_32a *)S.posfp;
    const PotDev &P = S.pot;
    double fx = 0, fy = 0, fz = 0, en = 0;
    double4_32a pa = make_double4_32a(0, 0, 0, 0);
    if (valid) {
        pa = pf[a];
        const int nn = chk_count(S, S.nn[a], S.cap_use);
        const int *__restrict__ lst = S.nlist + nl_base(a, L, S.cap);
        for (int k = l; k < nn; k += L) {
            const int j = nl_atom(S, (unsigned)lst[(k / L) * 32 + (k % L)]);
            const double4_32a pj = pf[j];
            const double dx = pj.x - pa.x, dy = pj.y - pa.y, dz = pj.z - pa.z;
            const double r2 = (dx * dx + dy * dy) + dz * dz;
            // tested on r2, as in the density pass
            if (r2 < P.rc * P.rc) {
                const double y = rsqrt(r2);
                const double r = r2 * y;
                double sn, sm;
                pow_nm<SC76>(P.a * y, P.n, P.m, sn, sm);
                const double dphn = -(double)P.n * y * sn + P.Bn;
                const double dphm = -(double)P.m * y * sm + P.Bm;
                const double g = (P.eps * dphn + (pa.w + pj.w) * dphm) * y;
                fx += g * dx;
                fy += g * dy;
                fz += g * dz;
                en += sn - P.An + P.Bn * (r - P.rc);
            }
        }
    }
    fx = lane_sum<L>(fx);
    fy = lane_sum<L>(fy);
    fz = lane_sum<L>(fz);
    en = lane_sum<L>(en);
    double ke = 0, pe = 0, rr = 0, d2 = 0;
    if (valid && l == 0) {
        chk_force(S, fx, fy, fz);
        const double fpa = pa.w;
        // B(rho) = -eps c sqrt(rho) = (eps c)^2 / (2 B'(rho))
        pe = 0.5 * P.eps * en + (fpa != 0.0 ? 0.5 * P.ec * P.ec / fpa : 0.0);
        const uint8_t flag = S.flags[a];
        if (flag == FLAG_RIGHT) rr = -(S.axis == 0 ? fx : (S.axis == 1 ? fy : fz));
        double4_32a v = ((const double4_32a *)S.vel)[a];
        if (mode == MODE_EVAL) {
            ke = S.ke_fac * ((v.x * v.x + v.y * v.y) + v.z * v.z);
            ((double4_32a *)S.eval_out)[S.orig[a]] = make_double4_32a(fx, fy, fz, pe);
        } else {
            const double kh = S.acc_half;
            // thermal relaxation: the right grip moves along the load axis only
            const bool rfree = flag == FLAG_RIGHT && S.ctl->relax;
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
                ke = S.ke_fac * ((v.x * v.x + v.y * v.y) + v.z * v.z);
                if (S.rsum) {
                    // Eq. (mean_pos): the sampled state's position
                    double *rs = S.rsum + 4LL * S.orig[a];
                    rs[0] = rs[0] + pa.x;
                    rs[1] = rs[1] + pa.y;
                    rs[2] = rs[2] + pa.z;
                }
            }
            double x = pa.x, y = pa.y, z = pa.z;
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
                x += v.x * S.dt;
                y += v.y * S.dt;
                z += v.z * S.dt;
            } else if (start && flag == FLAG_RIGHT && !rfree && S.ctl->grip_du != 0.0) {
                // continuous loading (fine-dynamics verification)
                const double du = S.ctl->grip_du;
                if (S.axis == 0) x = x + du;
                else if (S.axis == 1) y = y + du;
                else z = z + du;
            }
            ((double4_32a *)S.pos[par ^ 1])[a] = make_double4_32a(x, y, z, 0.0);
            ((double4_32a *)S.vel)[a] = v;
            const float4 rf = S.ref[a];
            const double ex = x - rf.x, ey = y - rf.y, ez = z - rf.z;
            d2 = ex * ex + ey * ey + ez * ez;
        }
    }
    ke = warp_sum(ke);
    pe = warp_sum(pe);
    rr = warp_sum(rr);
    d2 = (double)warp_max((float)d2);
    step_tail<TPB>(S, lb, S.nblk_pair, ke, pe, rr, d2, 0.0, mode, phase, done, nsteps);
}

#define PTA_F64_SWITCH(KER, SC, ARG)                                                   \
    switch (g.L) {                                                                     \
        case 1: KER<1, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, ARG); break;        \
        case 2: KER<2, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, ARG); break;        \
        case 4: KER<4, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, ARG); break;        \
        case 8: KER<8, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, ARG); break;        \
        default: KER<16, SC><<<g.nblk, TPB, 0, st>>>(t.specs, g.b2s, ARG); break;      \
    }

void launch_density_f64(const Tab &t, const Group &g, int force, cudaStream_t st) {
    if (g.sc76)
        PTA_F64_SWITCH(k_density_f64, true, force)
    else
        PTA_F64_SWITCH(k_density_f64, false, force)
}

void launch_force_f64(const Tab &t, const Group &g, int mode, cudaStream_t st) {
    if (g.sc76)
        PTA_F64_SWITCH(k_force_f64, true, mode)
    else
        PTA_F64_SWITCH(k_force_f64, false, mode)
}

}  // namespace pta
