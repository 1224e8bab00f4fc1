// Specimen creation, state exchange, grip displacement, burst bookkeeping
// and the coarse-step update, all as CUDA kernels.
#include <math.h>

#include "pta_dev.cuh"

namespace pta {

// ---------------------------------------------------------------------------
// small block reductions (fixed order: deterministic)
// ---------------------------------------------------------------------------
template <int NT>
__device__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor round on a 4-word counter with a 2-word key; the key is
// advanced by the Weyl increments before every round but the first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// 53 random bits k from two words; uniform (k + 1/2) / 2^53 in (0, 1)
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
    const unsigned long long k = ((unsigned long long)(a >> 5) << 26) | (b >> 6);
    return (double)k * (1.0 / 9007199254740992.0) + (1.0 / 18014398509481984.0);
}

// three N(0,1) draws for atom idx: counters (idx, idx>>32, blk, 0), blk = 0, 1,
// key = seed; Box-Muller on each pair of uniforms
__device__ void atom_normals(uint64_t seed, uint64_t idx, double z[3]) {
    double g[4];
    for (uint32_t blk = 0; blk < 2; ++blk) {
        const uint4 w = philox10(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), blk, 0u),
                                 make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const double u1 = u53(w.x, w.y), u2 = u53(w.z, w.w);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincos(6.283185307179586 * u2, &sn, &cs);
        g[2 * blk] = rad * cs;
        g[2 * blk + 1] = rad * sn;
    }
    z[0] = g[0];
    z[1] = g[1];
    z[2] = g[2];
}

// ---------------------------------------------------------------------------
// creation: FCC lattice, grip flags, Maxwell-Boltzmann velocities (into the
// FP64 staging buffer; launch_import converts them to the working layout)
// ---------------------------------------------------------------------------
__global__ void k_lattice(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= S.n) return;
    const int b = a & 3, c = a >> 2;
    const int i = c % S.ncl[0], j = (c / S.ncl[0]) % S.ncl[1], k = c / (S.ncl[0] * S.ncl[1]);
    const double bx = (b == 1 || b == 2) ? 0.5 : 0.0;
    const double by = (b == 1 || b == 3) ? 0.5 : 0.0;
    const double bz = (b == 2 || b == 3) ? 0.5 : 0.0;
    double p[3];
    p[0] = S.a0 * ((double)i + bx);
    p[1] = S.a0 * ((double)j + by);
    p[2] = S.a0 * ((double)k + bz);
    S.stage[3 * (size_t)a + 0] = p[0];
    S.stage[3 * (size_t)a + 1] = p[1];
    S.stage[3 * (size_t)a + 2] = p[2];
    S.orig[a] = a;
    // grips: lowest coordinate along the axis is 0, highest a0 (n - 1/2)
    const double lo = 0.0;
    const double hi = S.a0 * ((double)(S.ncl[S.axis] - 1) + 0.5);
    const double tol = 1e-6;
    const double x = p[S.axis];
    uint8_t f = FLAG_MOBILE;
    if (x <= lo + S.grip_width + tol)
        f = FLAG_LEFT;
    else if (x >= hi - S.grip_width - tol)
        f = FLAG_RIGHT;
    S.flags[a] = f;
}

__global__ void k_mb_draw(const SpecDev *__restrict__ sp, double sigma, uint64_t seed) {
    const SpecDev &S = *sp;
    __shared__ double sh[TPB];
    const int a = blockIdx.x * TPB + threadIdx.x;
    double v[3] = {0, 0, 0}, cnt = 0;
    if (a < S.n) {
        if (S.flags[a] == FLAG_MOBILE) {
            double z[3];
            atom_normals(seed, (uint64_t)a, z);
            for (int d = 0; d < 3; ++d) v[d] = sigma * z[d];
            cnt = 1;
        }
        double *vel = S.stage + 3 * (size_t)S.n;
        for (int d = 0; d < 3; ++d) vel[3 * (size_t)a + d] = v[d];
    }
    for (int d = 0; d < 3; ++d) {
        const double s = block_sum<TPB>(v[d], sh);
        if (threadIdx.x == 0) S.part[4 * blockIdx.x + d] = s;
    }
    const double s = block_sum<TPB>(cnt, sh);
    if (threadIdx.x == 0) S.part[4 * blockIdx.x + 3] = s;
}

// one block: sum the per-block partials in a fixed order into ctl->mb[off..off+3]
__global__ void k_mb_collect(const SpecDev *__restrict__ sp, int nblk, int off) {
    const SpecDev &S = *sp;
    __shared__ double sh[TPB];
    for (int q = 0; q < 4; ++q) {
        double v = 0;
        for (int b = threadIdx.x; b < nblk; b += TPB) v = v + S.part[4 * b + q];
        v = block_sum<TPB>(v, sh);
        if (threadIdx.x == 0) S.ctl->mb[off + q] = v;
    }
}

__global__ void k_mb_center(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    __shared__ double sh[TPB];
    const int a = blockIdx.x * TPB + threadIdx.x;
    const double nmob = S.ctl->mb[3];
    double v2 = 0;
    if (a < S.n && S.flags[a] == FLAG_MOBILE && nmob > 0) {
        double *vel = S.stage + 3 * (size_t)S.n;
        for (int d = 0; d < 3; ++d) {
            const double mean = S.ctl->mb[d] / nmob;
            const double v = vel[3 * (size_t)a + d] - mean;
            vel[3 * (size_t)a + d] = v;
            v2 = v2 + v * v;
        }
    }
    const double s = block_sum<TPB>(v2, sh);
    if (threadIdx.x == 0) {
        S.part[4 * blockIdx.x + 0] = s;
        S.part[4 * blockIdx.x + 1] = 0;
        S.part[4 * blockIdx.x + 2] = 0;
        S.part[4 * blockIdx.x + 3] = 0;
    }
}

__global__ void k_mb_apply(const SpecDev *__restrict__ sp, double kT) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a >= S.n) return;
    const double nmob = S.ctl->mb[3];
    const double ke = S.ke_fac * S.ctl->mb[4];
    const double target = 0.5 * (3.0 * nmob - 3.0) * kT;
    const bool zero = !(nmob >= 2.0) || !(kT > 0.0) || !(ke > 0.0);
    const double s = zero ? 0.0 : sqrt(target / ke);
    double *vel = S.stage + 3 * (size_t)S.n;
    for (int d = 0; d < 3; ++d) {
        const double v = vel[3 * (size_t)a + d];
        vel[3 * (size_t)a + d] = (S.flags[a] == FLAG_MOBILE) ? v * s : 0.0;
    }
}

void launch_create(const SpecDev &h, const SpecDev *d, double sigma_v, double kT, uint64_t seed,
                   cudaStream_t st) {
    const int nb = (h.n + TPB - 1) / TPB;
    k_lattice<<<nb, TPB, 0, st>>>(d);
    k_mb_draw<<<nb, TPB, 0, st>>>(d, sigma_v, seed);
    k_mb_collect<<<1, TPB, 0, st>>>(d, nb, 0);
    k_mb_center<<<nb, TPB, 0, st>>>(d);
    k_mb_collect<<<1, TPB, 0, st>>>(d, nb, 4);
    k_mb_apply<<<nb, TPB, 0, st>>>(d, kT);
}

// ---------------------------------------------------------------------------
// state exchange: FP64 staging (pos n x 3, vel n x 3) <-> working layout
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool split_hilo(double x, float &hi, float &lo) {
    if (!(fabs(x) < MIXED_RANGE)) {
        hi = 0.f;
        lo = 0.f;
        return false;
    }
    const double xs = rint(x * HI_SCALE) * HI_QUANTUM;  // multiple of 2^-12, exact in FP32
    hi = (float)xs;
    lo = (float)(x - xs);
    return true;
}

__global__ void k_import(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int par = S.ctl->parity;
    const size_t o = (size_t)S.orig[a];  // stage is in creation order
    const double *p = S.stage + 3 * o;
    const double *v = S.stage + 3 * (size_t)S.n + 3 * o;
    if (S.prec == PTA_PREC_FP64) {
        ((double4_32a *)S.pos[par])[a] = make_double4_32a(p[0], p[1], p[2], 0.0);
        ((double4_32a *)S.vel)[a] = make_double4_32a(v[0], v[1], v[2], 0.0);
    } else {
        float h[3], l[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) ok &= split_hilo(p[d], h[d], l[d]);
        if (!ok) atomicOr(&S.ctl->err, ERR_RANGE);
        ((float4 *)S.pos[par])[a] = make_float4(h[0], h[1], h[2], 0.f);
        S.lo[par][a] = make_float4(l[0], l[1], l[2], 0.f);
        // v = vh + vl: the FP32 rounding and its remainder (exact to ~2^-48 v)
        VelHL w;
        w.h = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
        w.l = make_float4((float)(v[0] - (double)w.h.x), (float)(v[1] - (double)w.h.y),
                          (float)(v[2] - (double)w.h.z), 0.f);
        ((VelHL *)S.vel)[a] = w;
    }
    if (a == 0) S.ctl->rebuild = 1;
}

__global__ void k_export(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int par = S.ctl->parity;
    const size_t o = (size_t)S.orig[a];  // stage is in creation order
    double *p = S.stage + 3 * o;
    double *v = S.stage + 3 * (size_t)S.n + 3 * o;
    if (S.prec == PTA_PREC_FP64) {
        const double4_32a q = ((const double4_32a *)S.pos[par])[a];
        const double4_32a w = ((const double4_32a *)S.vel)[a];
        p[0] = q.x;
        p[1] = q.y;
        p[2] = q.z;
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
    } else {
        const float4 h = ((const float4 *)S.pos[par])[a];
        const float4 l = S.lo[par][a];
        const VelHL w = ((const VelHL *)S.vel)[a];
        p[0] = (double)h.x + (double)l.x;
        p[1] = (double)h.y + (double)l.y;
        p[2] = (double)h.z + (double)l.z;
        v[0] = (double)w.h.x + (double)w.l.x;
        v[1] = (double)w.h.y + (double)w.l.y;
        v[2] = (double)w.h.z + (double)w.l.z;
    }
}

// checkpoints: the raw working state (current position buffer, velocities,
// grip flags) gathered into creation order through the permutation scratch,
// or scattered back to the context's current slot order, so that a
// checkpoint does not depend on how the last list build ordered the atoms
__global__ void k_ckpt_move(const SpecDev *__restrict__ sp, int gather) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a >= S.n) return;
    const int par = S.ctl->parity;
    const int o = S.orig[a];
    const PermLayout Lo = perm_layout(S.n, S.prec);
    char *t = (char *)S.perm_tmp;
    double4_32a *tv = (double4_32a *)(t + Lo.vel);
    uint8_t *tf = (uint8_t *)(t + Lo.flags);
    if (S.prec == PTA_PREC_FP64) {
        double4_32a *tp = (double4_32a *)(t + Lo.pos);
        double4_32a *wp = (double4_32a *)S.pos[par];
        if (gather) tp[o] = wp[a]; else wp[a] = tp[o];
    } else {
        float4 *tp = (float4 *)(t + Lo.pos), *tl = (float4 *)(t + Lo.lo);
        float4 *wp = (float4 *)S.pos[par];
        if (gather) {
            tp[o] = wp[a];
            tl[o] = S.lo[par][a];
        } else {
            wp[a] = tp[o];
            S.lo[par][a] = tl[o];
        }
    }
    double4_32a *wv = (double4_32a *)S.vel;
    if (gather) {
        tv[o] = wv[a];
        tf[o] = S.flags[a];
    } else {
        wv[a] = tv[o];
        S.flags[a] = tf[o];
    }
}

void launch_ckpt_move(const SpecDev &h, const SpecDev *d, int gather, cudaStream_t st) {
    k_ckpt_move<<<(h.n + TPB - 1) / TPB, TPB, 0, st>>>(d, gather);
}

// end of thermal relaxation: the right grip is fixed where it is, v = 0
__global__ void k_fix_right_grip(const SpecDev *__restrict__ sp) {
    const SpecDev &S = *sp;
    const int a = blockIdx.x * TPB + threadIdx.x;
    if (a >= S.n || S.flags[a] != FLAG_RIGHT) return;
    // both precisions keep 32-byte velocity records (double4 or VelHL)
    ((double4_32a *)S.vel)[a] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
}

void launch_fix_right_grip(const SpecDev &h, const SpecDev *d, cudaStream_t st) {
    k_fix_right_grip<<<(h.n + TPB - 1) / TPB, TPB, 0, st>>>(d);
}

void launch_import(const SpecDev &h, const SpecDev *d, cudaStream_t st) {
    k_import<<<(h.n + TPB - 1) / TPB, TPB, 0, st>>>(d);
}
void launch_export(const SpecDev &h, const SpecDev *d, cudaStream_t st) {
    k_export<<<(h.n + TPB - 1) / TPB, TPB, 0, st>>>(d);
}

// ---------------------------------------------------------------------------
// loading protocol: right grip moves by du along the load axis (batched)
// ---------------------------------------------------------------------------
__global__ void k_strain(const SpecDev *__restrict__ specs, const int *__restrict__ b2s,
                         const double *__restrict__ du_all) {
    const SpecDev &S = specs[b2s[blockIdx.x]];
    const double du = du_all[S.spec_index];
    if (du == 0.0) return;
    const int a = (blockIdx.x - S.blk_atom0) * TPB + threadIdx.x;
    if (a == 0) S.ctl->rebuild = 1;
    if (a >= S.n || S.flags[a] != FLAG_RIGHT) return;
    const int par = S.ctl->parity;
    if (S.prec == PTA_PREC_FP64) {
        double *q = (double *)&((double4_32a *)S.pos[par])[a];
        q[S.axis] = q[S.axis] + du;
    } else {
        float *h = (float *)&((float4 *)S.pos[par])[a];
        float *l = (float *)&S.lo[par][a];
        const double x = (double)h[S.axis] + (double)l[S.axis] + du;
        float hh, ll;
        if (!split_hilo(x, hh, ll)) atomicOr(&S.ctl->err, ERR_RANGE);
        h[S.axis] = hh;
        l[S.axis] = ll;
    }
}

void launch_strain(const Tab &t, const double *du, cudaStream_t st) {
    k_strain<<<t.nblk_atom, TPB, 0, st>>>(t.specs, t.b2s_atom, du);
}

// ---------------------------------------------------------------------------
// burst bookkeeping (one block per specimen)
// ---------------------------------------------------------------------------
__global__ void k_burst_begin(const SpecDev *__restrict__ specs, const long long *__restrict__ ns) {
    const SpecDev &S = specs[blockIdx.x];
    if (threadIdx.x != 0) return;
    SpecCtl *c = S.ctl;
    const long long n = ns[blockIdx.x];
    c->nsteps = n;
    c->done = 0;
    c->sum[0] = c->sum[1] = c->sum[2] = 0.0;
    for (int q = 0; q < 3; ++q) {
        c->sum_chk[q] = 0.0;
        c->conv_val[q] = 0.0;
        c->conv_n[q] = 0;
    }
    c->conv_mask = 0;
    c->rebuilds = 0;
    c->prunes = 0;
    c->blocks_done = 0;
    // a burst always starts from a fresh neighbour list, so its result does
    // not depend on when earlier lists were built (checkpoints, batching)
    if (n > 0) c->rebuild = 1;
    c->phase = (n > 0) ? PH_REFRESH : PH_IDLE;
}

void launch_burst_begin(const Tab &t, const long long *nsteps, cudaStream_t st) {
    k_burst_begin<<<t.nspec, 32, 0, st>>>(t.specs, nsteps);
}

// Eq. (R_m_t): mean of the samples; standard error from block means
__global__ void k_burst_end(const SpecDev *__restrict__ specs, int slot, pta_averages *out) {
    const SpecDev &S = specs[blockIdx.x];
    SpecCtl *c = S.ctl;
    __shared__ double sh[TPB];
    const long long n = c->done;
    const int B = S.block_steps > 0 ? S.block_steps : 100;
    const bool adaptive = S.conv_lag > 0;
    double mean[3], bmean[3], se[3];
    long long nq[3];
    for (int q = 0; q < 3; ++q) {
        // adaptive length: a converged variable reports the running average
        // at its convergence step, the others the running average of all
        // samples (both from the step-ordered running sums)
        const bool conv = adaptive && (c->conv_mask & (1 << q));
        nq[q] = conv ? c->conv_n[q] : n;
        const long long nb = nq[q] / B;
        double s = 0;
        for (long long i = threadIdx.x; i < n; i += TPB) s = s + S.series[3 * i + q];
        s = block_sum<TPB>(s, sh);
        mean[q] = (n > 0) ? s / (double)n : nan("");
        if (adaptive && n > 0) mean[q] = conv ? c->conv_val[q] : c->sum[q] / (double)n;
        // block means and their mean
        double sb = 0;
        for (long long b = threadIdx.x; b < nb; b += TPB) {
            double t = 0;
            for (int i = 0; i < B; ++i) t = t + S.series[3 * (b * B + i) + q];
            sb = sb + t / (double)B;
        }
        sb = block_sum<TPB>(sb, sh);
        bmean[q] = (nb > 0) ? sb / (double)nb : 0.0;
        double sv = 0;
        for (long long b = threadIdx.x; b < nb; b += TPB) {
            double t = 0;
            for (int i = 0; i < B; ++i) t = t + S.series[3 * (b * B + i) + q];
            const double dv = t / (double)B - bmean[q];
            sv = sv + dv * dv;
        }
        sv = block_sum<TPB>(sv, sh);
        se[q] = (nb >= 2) ? sqrt(sv / (double)(nb - 1) / (double)nb) : nan("");
    }
    if (threadIdx.x == 0) {
        pta_averages r;
        for (int q = 0; q < 3; ++q) {
            r.mean[q] = mean[q];
            r.se[q] = se[q];
        }
        r.nsteps = n;
        r.rebuilds = c->rebuilds;
        r.prunes = c->prunes;
        r.converged = adaptive ? c->conv_mask : 0;
        for (int q = 0; q < 3; ++q) r.nsamples[q] = nq[q];
        int e = c->err;
        r.status = (e & ERR_CHECK)    ? PTA_ECHECK
                   : (e & ERR_OVERFLOW) ? PTA_ENEIGH_OVERFLOW
                   : (e & ERR_NAN)    ? PTA_ENAN
                   : (e & (ERR_RANGE | ERR_GRID)) ? PTA_ERANGE
                                      : PTA_OK;
        c->last = r;
        if (slot >= 0 && slot < 3)
            for (int q = 0; q < 3; ++q) c->pta.R3[slot][q] = mean[q];
        out[blockIdx.x] = r;
    }
}

// adaptive burst lengths: is any specimen of the table still in its burst?
__global__ void k_any_running(const SpecDev *__restrict__ specs, int nspec, int *flag) {
    int run = 0;
    for (int s = threadIdx.x; s < nspec; s += blockDim.x) run |= specs[s].ctl->phase != PH_IDLE;
    run = __syncthreads_or(run);
    if (threadIdx.x == 0) *flag = run;
}

void launch_any_running(const Tab &t, int *flag, cudaStream_t st) {
    k_any_running<<<1, 128, 0, st>>>(t.specs, t.nspec, flag);
}

void launch_burst_end(const Tab &t, int slot, pta_averages *out, cudaStream_t st) {
    k_burst_end<<<t.nspec, TPB, 0, st>>>(t.specs, slot, out);
}

// ---------------------------------------------------------------------------
// coarse-step update (one thread per specimen, FP64).  ops[s]: 0 nothing,
// 1 initial state from the three initial bursts, 2 one coarse step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rel_err(double x, double ref, double fl) {
    return fabs(x - ref) / fmax(fabs(ref), fl);
}

__global__ void k_pta_update(const SpecDev *__restrict__ specs, const int *__restrict__ ops,
                             pta_coarse_result *out) {
    const SpecDev &S = specs[blockIdx.x];
    if (threadIdx.x != 0) return;
    const int op = ops[blockIdx.x];
    if (op == 0) return;
    PtaDev &P = S.ctl->pta;
    pta_coarse_result r;
    if (op == 1) {
        for (int q = 0; q < 3; ++q) {
            // Eq. (simp) over the bursts labelled -Delta, -Delta/2, 0
            P.v[q] = (P.R3[0][q] + 4.0 * P.R3[1][q] + P.R3[2][q]) / 6.0;
            P.R_t[q] = P.R3[2][q];
            P.R_tmD[q] = P.R3[0][q];
            P.R_tmh[q] = 0.0;
            P.jump[q] = 0;
            r.v[q] = P.v[q];
            r.v_pred[q] = nan("");
            r.v_d[q] = P.v[q];
            r.e_v[q] = nan("");
            r.e1[q] = nan("");
            r.e2[q] = nan("");
            r.jump[q] = 0;
            r.source[q] = -1;
        }
        P.has_tmh = 0;
        P.init = 1;
        P.t = 0.0;
        r.t = 0.0;
    } else {
        const double h = S.pta_h, D = S.pta_Delta;
        for (int q = 0; q < 3; ++q) {
            const double Ra = P.R3[0][q], Rb = P.R3[1][q], Rc = P.R3[2][q];
            const double dvdt = (P.R_t[q] - P.R_tmD[q]) / D;  // Eq. (dvdt_algo)
            // Eq. (pta_pred), rounded as written (no fused multiply-add), so
            // that the extrapolation is reproducible off the device
            const double vp = __dadd_rn(P.v[q], __dmul_rn(h, dvdt));
            const double vd = (Ra + 4.0 * Rb + Rc) / 6.0;      // Eq. (simp)
            const double fl = S.floor_[q];
            const double ev = rel_err(vp, vd, fl);             // Eq. (rel_err)
            const double e1 = rel_err(Rc, P.R_t[q], fl);       // Eq. (jump_err)
            const double e2 = P.has_tmh ? rel_err(P.R_t[q], P.R_tmh[q], fl) : nan("");
            int src, jumped;
            double v;
            if (ev < S.tol_v[q]) {
                v = vp;
                src = PTA_SRC_PREDICTED;
                jumped = 0;
            } else {
                if (P.jump[q])
                    jumped = e1 >= S.tol_j[q];
                else if (!P.has_tmh)
                    jumped = 0;
                else if (e2 > 0.0)
                    jumped = fabs(e1 / e2 - 1.0) >= S.tol_j[q];
                else
                    jumped = e1 > 0.0;
                v = vd;
                src = jumped ? PTA_SRC_MEASURE_JUMP : PTA_SRC_MEASURE_MISMATCH;
            }
            r.v[q] = v;
            r.v_pred[q] = vp;
            r.v_d[q] = vd;
            r.e_v[q] = ev;
            r.e1[q] = e1;
            r.e2[q] = e2;
            r.jump[q] = jumped;
            r.source[q] = src;
            // chain: R_{t-h} <- R_t, R_{t-Delta} <- R_{t+h-Delta}, R_t <- R_{t+h}
            P.R_tmh[q] = P.R_t[q];
            P.R_tmD[q] = Ra;
            P.R_t[q] = Rc;
            P.v[q] = v;
            P.jump[q] = jumped;
        }
        P.has_tmh = 1;
        P.t = P.t + h;
        r.t = P.t;
    }
    r.strain = 0.0;
    r.status = PTA_OK;
    r.pad = 0;
    out[blockIdx.x] = r;
}

void launch_pta_update(const Tab &t, const int *ops, pta_coarse_result *out, cudaStream_t st) {
    k_pta_update<<<t.nspec, 32, 0, st>>>(t.specs, ops, out);
}

__global__ void k_force_rebuild(const SpecDev *__restrict__ specs) {
    if (threadIdx.x == 0) specs[blockIdx.x].ctl->rebuild = 1;
}
void launch_force_rebuild_flag(const Tab &t, cudaStream_t st) {
    k_force_rebuild<<<t.nspec, 32, 0, st>>>(t.specs);
}

}  // namespace pta
