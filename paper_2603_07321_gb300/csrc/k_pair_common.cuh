// Pieces shared by the FP64 and mixed-precision pair kernels: warp
// reductions and the end-of-step reduction that turns per-block partials
// into the state functions K, U, T of Eq. (state_variables) for one step.
#pragma once

#include "pta_dev.cuh"

namespace pta {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// sum over the L lanes that share one atom (lanes are contiguous in the warp)
template <int L, typename T>
__device__ __forceinline__ T lane_sum(T v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Called by every thread of a pair block of NT threads after the warp
// reductions (values valid in lane 0 of each warp); nblk is the number of
// the specimen's blocks in this launch.  Block partials go to S.part (8
// doubles per block).  The reduction is a fixed two-level tree: the last
// block to finish in each group of 32 consecutive blocks sums the group's
// partials (one per lane, butterfly shuffles) into a group partial stored
// after the block partials, and the last group to finish sums the group
// partials (each thread a strided share, then warp shuffles, then the warps
// in order).  Each level is one round of parallel loads; a single last
// block walking every block partial took ~8 us longer per pass on the
// 470,596-atom cube.  Group counters sit after the group partials, start
// at 0 and are reset by their group's last block.  The last group then
// advances the specimen's control block:
//   MODE_STEP, phase RUN:     sample (K, U, T) into the series, step count + 1,
//                             burst over after nsteps samples
//   MODE_STEP, phase REFRESH: forces refreshed and the first step started
//   MODE_EVAL:                K, U, T stored in eval_obs
// and in MODE_STEP the position buffers swap, the skin test sets the
// rebuild flag and the pruning margin test the prune flag.
template <int NT>
__device__ inline void step_tail(const SpecDev &S, int lb, int nblk, double ke_w, double pe_w,
                                 double rr_w, double d2_w, double dp2_w, int mode, int phase,
                                 long long done, long long nsteps) {
    constexpr int NV = 5;  // K, U, R, max displacement^2 since the build and since the pruning
    constexpr int NW = NT / 32;
    __shared__ double shw[NV][NW];
    __shared__ int role;  // 0: done; 1: last block of its group; 2: last group
    constexpr int GS = 32;  // blocks per group
    const int ngroups = (nblk + GS - 1) / GS;
    const int g = lb / GS;
    const int gsize = min(GS, nblk - g * GS);
    unsigned *gcnt = (unsigned *)(S.part + 8LL * (nblk + ngroups)) + g;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        shw[0][w] = ke_w;
        shw[1][w] = pe_w;
        shw[2][w] = rr_w;
        shw[3][w] = d2_w;
        shw[4][w] = dp2_w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0, p = 0, r = 0, d = 0, e = 0;
        for (int i = 0; i < NW; ++i) {
            k = k + shw[0][i];
            p = p + shw[1][i];
            r = r + shw[2][i];
            d = fmax(d, shw[3][i]);
            e = fmax(e, shw[4][i]);
        }
        double *P = S.part + 8LL * lb;
        P[0] = k;
        P[1] = p;
        P[2] = r;
        P[3] = d;
        P[4] = e;
        __threadfence();
        const unsigned prev = atomicAdd(gcnt, 1u);
        role = (prev == (unsigned)(gsize - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (role == 0) return;
    __threadfence();
    if (w == 0) {
        // the group's partials, one per lane, summed in lane order
        double a[NV] = {0, 0, 0, 0, 0};
        if (lane < gsize) {
            const double *P = S.part + 8LL * (g * GS + lane);
            a[0] = __ldcg(P);
            a[1] = __ldcg(P + 1);
            a[2] = __ldcg(P + 2);
            a[3] = __ldcg(P + 3);
            a[4] = __ldcg(P + 4);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a[0] = a[0] + __shfl_xor_sync(0xffffffffu, a[0], o);
            a[1] = a[1] + __shfl_xor_sync(0xffffffffu, a[1], o);
            a[2] = a[2] + __shfl_xor_sync(0xffffffffu, a[2], o);
            a[3] = fmax(a[3], __shfl_xor_sync(0xffffffffu, a[3], o));
            a[4] = fmax(a[4], __shfl_xor_sync(0xffffffffu, a[4], o));
        }
        if (lane == 0) {
            double *G = S.part + 8LL * (nblk + g);
            for (int q = 0; q < NV; ++q) G[q] = a[q];
            *gcnt = 0u;  // every block of the group has counted: ready for the next launch
            __threadfence();
            const unsigned prev = atomicAdd(&S.ctl->blocks_done, 1u);
            role = (prev == (unsigned)(ngroups - 1)) ? 2 : 0;
        }
    }
    __syncthreads();
    if (role != 2) return;
    __threadfence();
    double v[NV] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < ngroups; b += NT) {
        const double *P = S.part + 8LL * (nblk + b);
        v[0] = v[0] + __ldcg(P);
        v[1] = v[1] + __ldcg(P + 1);
        v[2] = v[2] + __ldcg(P + 2);
        v[3] = fmax(v[3], __ldcg(P + 3));
        v[4] = fmax(v[4], __ldcg(P + 4));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = v[0] + __shfl_xor_sync(0xffffffffu, v[0], o);
        v[1] = v[1] + __shfl_xor_sync(0xffffffffu, v[1], o);
        v[2] = v[2] + __shfl_xor_sync(0xffffffffu, v[2], o);
        v[3] = fmax(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
        v[4] = fmax(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
    }
    __syncthreads();  // every warp has read shw above
    if (lane == 0)
        for (int q = 0; q < NV; ++q) shw[q][w] = v[q];
    __syncthreads();
    double tot[NV] = {0, 0, 0, 0, 0};
    if (threadIdx.x == 0)
        for (int i = 0; i < NW; ++i) {
            tot[0] = tot[0] + shw[0][i];
            tot[1] = tot[1] + shw[1][i];
            tot[2] = tot[2] + shw[2][i];
            tot[3] = fmax(tot[3], shw[3][i]);
            tot[4] = fmax(tot[4], shw[4][i]);
        }
    if (threadIdx.x != 0) return;
    SpecCtl *c = S.ctl;
    const double K = tot[0], U = tot[1], T = tot[2] * S.t_fac, md2 = tot[3], mp2 = tot[4];
    if (mode == MODE_EVAL) {
        c->eval_obs[0] = K;
        c->eval_obs[1] = U;
        c->eval_obs[2] = T;
        c->rebuild = 0;
    } else {
        if (phase == PH_RUN) {
            if (!isfinite(K) || !isfinite(U) || !isfinite(T)) {
                c->err |= ERR_NAN;
                c->phase = PH_IDLE;
            } else {
                double *o = S.series + 3 * done;
                o[0] = K;
                o[1] = U;
                o[2] = T;
                c->sum[0] = c->sum[0] + K;
                c->sum[1] = c->sum[1] + U;
                c->sum[2] = c->sum[2] + T;
                c->done = done + 1;
                if (done + 1 >= nsteps) c->phase = PH_IDLE;
                const long long i = done + 1;
                if (S.conv_lag > 0 && i % S.conv_lag == 0) {
                    // appendix, Eq. (R_m_conv): e = |R^(i) - R^(i-k)| / max(|R^(i)|,
                    // floor), from i = 2k on; each variable converges on its own
                    if (i >= 2LL * S.conv_lag) {
                        for (int q = 0; q < 3; ++q) {
                            if (c->conv_mask & (1 << q)) continue;
                            const double a = c->sum[q] / (double)i;
                            const double b = c->sum_chk[q] / (double)(i - S.conv_lag);
                            const double e = fabs(a - b) / fmax(fabs(a), S.floor_[q]);
                            if (e < S.conv_tol[q]) {
                                c->conv_mask |= 1 << q;
                                c->conv_n[q] = i;
                                c->conv_val[q] = a;
                            }
                        }
                        if (c->conv_mask == 7) c->phase = PH_IDLE;
                    }
                    for (int q = 0; q < 3; ++q) c->sum_chk[q] = c->sum[q];
                }
            }
        } else if (phase == PH_REFRESH) {
            c->phase = PH_RUN;
        }
        c->rebuild = (md2 > (double)S.half_skin2) ? 1 : 0;
        if (S.prune_on && mp2 > (double)S.half_prune2) c->prune = 1;
        c->parity ^= 1;
    }
    __threadfence();
    c->blocks_done = 0;
}

}  // namespace pta
