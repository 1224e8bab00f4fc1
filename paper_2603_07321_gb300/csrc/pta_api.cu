// Host side of the C ABI declared in include/pta.h: contexts, device memory,
// launch tables, CUDA-graph replay of the fine-step loop, batches.
//
// The fine-step loop of one iteration is
//     [neighbour-list build, skipped on the device unless needed]
//     [density pass] [force pass + fused velocity Verlet + step reduction]
// for every specimen of a launch table at once.  Its kernels read each
// specimen's phase and step counter from device memory, so the same
// captured graph serves every burst length: a burst of n steps is n + 1
// iterations (one force refresh, then n steps), replayed as chunks of a
// graph of CHUNK iterations plus single iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pta.h"
#include "pta_dev.cuh"

using namespace pta;

namespace {

// NVTX range over a scope: bursts, ticks, creation and the other host calls
// show up by name on a profiler timeline (no cost without a profiler)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// CODATA 2018 constants and the unit conversions that follow from them
constexpr double E_CHARGE = 1.602176634e-19;  // J / eV
constexpr double AMU = 1.66053906660e-27;     // kg / amu
constexpr double KB_SI = 1.380649e-23;        // J / K
double mv2_to_ev() { return AMU * 1e-20 / 1e-30 / E_CHARGE; }         // amu A^2/fs^2 -> eV
double force_to_acc() { return E_CHARGE / (1e-10 * AMU) * 1e10 / 1e30; }  // eV/(A amu) -> A/fs^2
double kb_ev() { return KB_SI / E_CHARGE; }
double ev_a3_to_gpa() { return E_CHARGE / 1e-30 / 1e9; }

constexpr int CHUNK = 64;

// resident threads of the whole current GPU (SM count x threads per SM, from
// the device attributes); 0 when no device can be queried
long long device_threads() {
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long long)nsm * per_sm;
}

struct Allocator {
    pta_alloc_fn alloc = nullptr;
    pta_free_fn release = nullptr;
    void *user = nullptr;
};
Allocator g_alloc;
std::mutex g_alloc_mu;

struct DevBuf {
    void *p;
    size_t bytes;
};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct Runner;

struct pta_ctx {
    pta_specimen spec;
    pta_potential pot;
    pta_params par;
    double T0 = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    Allocator alloc;
    std::vector<DevBuf> bufs;
    SpecDev hd;
    SpecDev *d_self = nullptr;
    double L_s = 0;
    double u = 0;          // grip displacement, A
    double grip_du = 0;    // host copy of the per-step grip advance of a ramped burst
    bool pta_init = false;
    bool broken = false;
    Runner *solo = nullptr;
    pta_batch *batch = nullptr;
};

struct Runner {
    std::vector<pta_ctx *> m;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    Allocator alloc;
    std::vector<DevBuf> bufs;
    std::vector<SpecDev> hspecs;
    SpecDev *d_specs = nullptr;
    long long *d_nsteps = nullptr;
    double *d_du = nullptr;
    int *d_ops = nullptr;
    pta_averages *d_avg = nullptr;
    pta_coarse_result *d_cres = nullptr;
    void *h_pin = nullptr;
    long long *h_nsteps = nullptr;
    double *h_du = nullptr;
    int *h_ops = nullptr;
    pta_averages *h_avg = nullptr;
    pta_coarse_result *h_cres = nullptr;
    Tab tab{};
    cudaGraphExec_t g_chunk = nullptr, g_one = nullptr;
    // timing: graphs with event-record nodes around each iteration's parts
    bool timing = false;
    cudaGraphExec_t t_chunk = nullptr, t_one = nullptr;
    std::vector<cudaEvent_t> ev;  // 4 per iteration slot of a chunk
    pta_kernel_times times{};
};

struct pta_batch {
    Runner *r = nullptr;
};

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
static void *raw_alloc(const Allocator &al, size_t bytes, cudaStream_t st) {
    void *p = nullptr;
    if (al.alloc) {
        p = al.alloc(bytes, (void *)st, al.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void raw_free(const Allocator &al, void *p, cudaStream_t st) {
    if (!p) return;
    if (al.release)
        al.release(p, (void *)st, al.user);
    else
        cudaFree(p);
}

template <class Owner>
static int dev_alloc(Owner *o, size_t bytes, void **out) {
    bytes = round_up(bytes > 0 ? bytes : 1, 256);
    void *p = raw_alloc(o->alloc, bytes, o->stream);
    if (!p) return PTA_ENOMEM;
    if (cudaMemsetAsync(p, 0, bytes, o->stream) != cudaSuccess) {
        raw_free(o->alloc, p, o->stream);
        return PTA_ECUDA;
    }
    o->bufs.push_back({p, bytes});
    *out = p;
    return PTA_OK;
}

template <class Owner>
static void dev_release(Owner *o, void *p) {
    for (size_t i = 0; i < o->bufs.size(); ++i)
        if (o->bufs[i].p == p) {
            raw_free(o->alloc, p, o->stream);
            o->bufs.erase(o->bufs.begin() + i);
            return;
        }
}

template <class Owner>
static void dev_release_all(Owner *o) {
    for (auto &b : o->bufs) raw_free(o->alloc, b.p, o->stream);
    o->bufs.clear();
}

#define CK(expr)                                 \
    do {                                         \
        if ((expr) != cudaSuccess) {             \
            cudaGetLastError();                  \
            return PTA_ECUDA;                    \
        }                                        \
    } while (0)
#define CKR(expr)                \
    do {                         \
        int _rc = (expr);        \
        if (_rc != PTA_OK) return _rc; \
    } while (0)

static int launch_check() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PTA_OK : PTA_ECUDA;
}

// ---------------------------------------------------------------------------
// potential helpers (host)
// ---------------------------------------------------------------------------
static double hpow(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

// c that puts the perfect FCC crystal of lattice parameter a0 in equilibrium
// under the cut potential: c = sqrt(S_m) * D_n / D_m, S_k = sum phi_k(|t|),
// D_k = sum |t| phi_k'(|t|), over all FCC lattice vectors t with |t| < rc
static double equilibrium_c(const pta_potential &p, double a0) {
    const double bas[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    const int R = (int)std::ceil(p.rc / a0) + 1;
    const double An = hpow(p.a / p.rc, p.n), Am = hpow(p.a / p.rc, p.m);
    double Sm = 0, Dn = 0, Dm = 0;
    for (int i = -R; i <= R; ++i)
        for (int j = -R; j <= R; ++j)
            for (int k = -R; k <= R; ++k)
                for (int b = 0; b < 4; ++b) {
                    const double x = a0 * (i + bas[b][0]), y = a0 * (j + bas[b][1]),
                                 z = a0 * (k + bas[b][2]);
                    const double r2 = (x * x + y * y) + z * z;
                    if (r2 == 0.0) continue;
                    const double r = std::sqrt(r2);
                    if (!(r < p.rc)) continue;
                    const double sn = hpow(p.a / r, p.n), sm = hpow(p.a / r, p.m);
                    Sm += sm - Am + p.m / p.rc * Am * (r - p.rc);
                    Dn += r * (-p.n / r * sn + p.n / p.rc * An);
                    Dm += r * (-p.m / r * sm + p.m / p.rc * Am);
                }
    return std::sqrt(Sm) * Dn / Dm;
}

static PotDev make_pot(const pta_potential &p) {
    PotDev d{};
    d.eps = p.eps;
    d.c = p.c;
    d.a = p.a;
    d.rc = p.rc;
    d.rc2 = p.rc * p.rc;
    d.n = p.n;
    d.m = p.m;
    d.An = hpow(p.a / p.rc, p.n);
    d.Am = hpow(p.a / p.rc, p.m);
    d.Bn = p.n / p.rc * d.An;
    d.Bm = p.m / p.rc * d.Am;
    d.ec = p.eps * p.c;
    d.f_eps = (float)d.eps;
    d.f_a = (float)d.a;
    d.f_rc = (float)d.rc;
    d.f_rc2 = (float)d.rc2;
    d.f_An = (float)d.An;
    d.f_Bn = (float)d.Bn;
    d.f_Am = (float)d.Am;
    d.f_Bm = (float)d.Bm;
    d.f_ec = (float)d.ec;
    d.f_ec2hq = (float)(0.5 * d.ec * d.ec * p.m * hpow(p.a, p.m));
    d.sc76 = (p.n == 7 && p.m == 6) ? 1 : 0;
    return d;
}

// ---------------------------------------------------------------------------
// sizes
// ---------------------------------------------------------------------------
struct Sizes {
    long long n;
    int L, cap, cap_use, nblk_pair, nblk_atom, nblk_cell, ncell, nc[3];
    int prune_on, mean_pos;
    double prune_margin;
    double h, org[3];
    size_t list_words;
    long long series_cap;
};

// threads per atom chosen from the specimen alone (so that a specimen runs
// the same arithmetic alone and in a batch): FP64 specimens spread over the
// whole GPU; mixed-precision ones aim at ~64K threads and let batching fill
// the device
static int auto_lanes(long long n, int prec) {
    long long target = 65536;
    if (prec == PTA_PREC_FP64) {
        target = device_threads();
        if (target <= 0) target = 1LL << 18;  // no device to ask: a full GPU of this class
    }
    long long t = target / std::max<long long>(n, 1);
    int L = 1;
    while (L * 2 <= t && L < 16) L *= 2;
    return L;
}

static int valid_lanes(int L) { return L == 1 || L == 2 || L == 4 || L == 8 || L == 16; }

static int compute_sizes(const pta_specimen &s, const pta_potential &p, const pta_params &par,
                         Sizes *z) {
    z->n = 4LL * s.n_cells[0] * s.n_cells[1] * s.n_cells[2];
    z->L = par.lanes ? par.lanes : auto_lanes(z->n, par.precision);
    z->mean_pos = par.mean_positions ? 1 : 0;
    const double rl = p.rc + par.skin;
    z->prune_margin = par.prune_margin == 0.0 ? 0.3 : par.prune_margin;
    z->prune_on = (par.precision == PTA_PREC_MIXED && z->prune_margin > 0.0 &&
                   z->prune_margin < par.skin) ? 1 : 0;
    if (par.neigh_cap > 0) {
        z->cap_use = (int)round_up((size_t)par.neigh_cap, 32);
    } else {
        const double dens = 4.0 / (s.a0 * s.a0 * s.a0);
        const double nb = 4.0 / 3.0 * 3.141592653589793 * rl * rl * rl * dens;
        z->cap_use = (int)round_up((size_t)std::ceil(1.6 * nb + 16), 32);
    }
    // sixteen spare rows per lane: they hold the (up to four) sentinel rows
    // after a full list, the pair loops read four rows ahead and the pruning
    // fifteen, without bounds tests (spare entries hold 0, earlier entries or
    // the sentinel: all valid record indices)
    z->cap = z->cap_use + 16 * z->L;
    z->nblk_pair = (int)((z->n * z->L + TPB - 1) / TPB);
    z->nblk_atom = (int)((z->n + TPB - 1) / TPB);
    // cell edge a multiple of 2^-11 A and grid origin on the 2^-12 A grid, so
    // that cell centres and centre differences are exact in FP32
    z->h = std::ceil(rl * (1.0 + 1e-4) * 2048.0) / 2048.0;
    double maxspan = 0;
    double span[3];
    for (int d = 0; d < 3; ++d) {
        span[d] = (s.n_cells[d] - 0.5) * s.a0;
        maxspan = std::max(maxspan, span[d]);
    }
    const double margin = 0.25 * maxspan + 2.0 * z->h;
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        z->org[d] = std::floor(-margin * 4096.0) / 4096.0;
        z->nc[d] = (int)std::floor((span[d] + 2.0 * margin) / z->h) + 1;
        z->nc[d] += z->nc[d] & 1;
        ncell *= z->nc[d];
    }
    if (ncell > (1LL << 30)) return PTA_EINVAL;
    z->ncell = (int)ncell;
    z->nblk_cell = (z->ncell + CELL_WARPS * CELLS_PER_WARP - 1) / (CELL_WARPS * CELLS_PER_WARP);
    const long long W = 32 / z->L;
    z->list_words = (size_t)((z->n + W - 1) / W) * W * z->cap;
    z->series_cap = std::max<long long>(par.burst_steps, 1);
    return PTA_OK;
}

static size_t footprint(const Sizes &z, int prec) {
    const size_t n = (size_t)z.n;
    const size_t p = (prec == PTA_PREC_FP64) ? 32 : 16;
    size_t b = 0;
    auto add = [&](size_t x) { b += round_up(x > 0 ? x : 1, 256); };
    add(p * n);
    add(p * n);                      // pos[2]
    if (prec != PTA_PREC_FP64) {
        add(16 * n);
        add(16 * n);                 // lo[2]
        add(16 * (n + 1));
        add(16 * (n + 1));           // rel[2], + the sentinel record
        add(n);                      // hsub
    }
    add(p * (n + 1));                // posfp, + the sentinel record
    add(32 * n);                     // vel (double4 or hi/lo FP32)
    add(n);                          // flags
    add(16 * n);                     // ref
    add(4 * n);                      // atom_cell
    add(4 * (size_t)z.ncell);        // cell_cnt
    add(4 * ((size_t)z.ncell + 1));  // cell_start
    add(4 * n);                      // cell_tmp
    add(4 * n);                      // cell_atoms
    add(4 * n);                      // orig
    add(perm_layout(n, prec).total); // permutation scratch
    add(4 * z.list_words);           // nlist
    if (z.prune_on) {
        add(4 * z.list_words);       // plist
        add(4 * n * (size_t)z.L);    // pnn
        add(16 * n);                 // pref
    }
    add(4 * n);                      // nn
    {
        const size_t nb = (size_t)std::max(z.nblk_pair, z.nblk_atom);
        add(64 * (nb + 2 * (nb / 32 + 1)));  // part: block and group partials, group counters
    }
    add(24 * (size_t)z.series_cap);  // series
    add(32 * n);                     // eval_out
    if (z.mean_pos) add(32 * n);     // rsum
    add(48 * n);                     // stage
    add(sizeof(SpecCtl));
    add(sizeof(SpecDev));
    return b;
}

static int validate(const pta_specimen *s, const pta_potential *p, const pta_params *par) {
    if (!s || !p || !par) return PTA_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (s->n_cells[d] < 1 || s->n_cells[d] > 1000) return PTA_EINVAL;
    if (s->load_axis < 0 || s->load_axis > 2) return PTA_EINVAL;
    if (s->n_cells[s->load_axis] < 3) return PTA_EINVAL;
    if (!(s->a0 > 0)) return PTA_EINVAL;
    if (p->kind != PTA_POT_SUTTON_CHEN_SF) return PTA_EINVAL;
    if (!(p->eps > 0) || !(p->c > 0) || !(p->a > 0) || !(p->rc > 0)) return PTA_EINVAL;
    if (p->n < 1 || p->n > 16 || p->m < 1 || p->m > 16) return PTA_EINVAL;
    if (!(par->dt_fs > 0) || !(par->mass_amu > 0) || !(par->skin > 0)) return PTA_EINVAL;
    if (!(par->h > 0) || !(par->Delta > 0) || !(par->Delta <= par->h)) return PTA_EINVAL;
    if (par->burst_steps < 1 || par->block_steps < 1) return PTA_EINVAL;
    if (par->precision != PTA_PREC_FP64 && par->precision != PTA_PREC_MIXED) return PTA_EINVAL;
    if (par->lanes != 0 && !valid_lanes(par->lanes)) return PTA_EINVAL;
    if (par->atoms_per_thread < 0 || par->atoms_per_thread > 2) return PTA_EINVAL;
    if (par->atoms_per_thread == 2) return PTA_EUNSUPPORTED;
    if (par->neigh_cap < 0 || par->neigh_cap > 4096) return PTA_EINVAL;
    if (par->cell_tiles < -1 || par->cell_tiles > 1) return PTA_EINVAL;
    if (par->cell_tiles == 1) return PTA_EUNSUPPORTED;
    if (!std::isfinite(par->prune_margin)) return PTA_EINVAL;
    if (par->conv_lag < 0) return PTA_EINVAL;
    if (par->mean_positions != 0 && par->mean_positions != 1) return PTA_EINVAL;
    for (int q = 0; q < 3; ++q)
        if (!(par->conv_tol[q] >= 0) || !std::isfinite(par->conv_tol[q])) return PTA_EINVAL;
    const long long n = 4LL * s->n_cells[0] * s->n_cells[1] * s->n_cells[2];
    if (n >= (long long)MAX_ATOMS) return PTA_ERANGE;  // slot n is the lists' sentinel
    if (par->precision == PTA_PREC_MIXED) {
        for (int d = 0; d < 3; ++d)
            if (s->n_cells[d] * s->a0 * 1.5 > MIXED_RANGE) return PTA_ERANGE;
    }
    return PTA_OK;
}

// ---------------------------------------------------------------------------
// runners: a launch table over members plus captured graphs
// ---------------------------------------------------------------------------
static void runner_free(Runner *r) {
    if (!r) return;
    if (r->g_chunk) cudaGraphExecDestroy(r->g_chunk);
    if (r->g_one) cudaGraphExecDestroy(r->g_one);
    if (r->t_chunk) cudaGraphExecDestroy(r->t_chunk);
    if (r->t_one) cudaGraphExecDestroy(r->t_one);
    for (auto e : r->ev) cudaEventDestroy(e);
    if (r->stream) cudaStreamSynchronize(r->stream);
    dev_release_all(r);
    if (r->h_pin) cudaFreeHost(r->h_pin);
    if (r->cap) cudaStreamDestroy(r->cap);
    if (r->cap2) cudaStreamDestroy(r->cap2);
    delete r;
}

// Graph of `iters` fine-step iterations.  Each iteration is
//   [decide] -> SWITCH { 0: build + prune kernels, 1: prune kernels } -> density -> force
// where the decide kernel sets the switch value on the device (2 when no
// specimen needs either), so list maintenance costs no launch on the steps
// that need none.  With `timed`, event-record nodes bracket the parts of each
// iteration (events cannot sit inside a conditional body, so the build
// time is measured around the whole conditional).
static int capture_iters_flat(Runner *r, int iters, cudaGraphExec_t *out, bool timed);

static int capture_iters(Runner *r, int iters, cudaGraphExec_t *out, bool timed = false) {
    // Nsight Compute cannot profile kernel nodes of graphs that hold
    // conditional nodes; PTA_GRAPH_FLAT=1 captures the same kernels without
    // one (the build kernels then return at once on the device when no
    // build is needed)
    const char *flat = std::getenv("PTA_GRAPH_FLAT");
    if (flat && flat[0] == '1') return capture_iters_flat(r, iters, out, timed);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphConditionalHandle> handles(iters);
    for (int i = 0; i < iters; ++i)
        if (cudaGraphConditionalHandleCreate(&handles[i], g, LIST_NONE, cudaGraphCondAssignDefault) !=
            cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return PTA_ECUDA;
        }
    cudaError_t e = cudaStreamBeginCaptureToGraph(r->cap, g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    int rc = (e == cudaSuccess) ? PTA_OK : PTA_ECUDA;
    for (int i = 0; i < iters && rc == PTA_OK; ++i) {
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 0], r->cap, cudaEventRecordExternal);
        launch_decide_rebuild(r->tab, handles[i], r->cap);
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edata = nullptr;
        size_t ndeps = 0;
        if (cudaStreamGetCaptureInfo(r->cap, &cs, nullptr, &cg, &deps, &edata, &ndeps) !=
            cudaSuccess) {
            rc = PTA_ECUDA;
            break;
        }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = handles[i];
        np.conditional.type = cudaGraphCondTypeSwitch;
        np.conditional.size = 2;  // LIST_BUILD, LIST_PRUNE (LIST_NONE runs neither)
        cudaGraphNode_t cnode;
        if (cudaGraphAddNode(&cnode, cg, deps, edata, ndeps, &np) != cudaSuccess) {
            rc = PTA_ECUDA;
            break;
        }
        cudaGraph_t bodies[2] = {np.conditional.phGraph_out[0], np.conditional.phGraph_out[1]};
        if (cudaStreamUpdateCaptureDependencies(r->cap, &cnode, nullptr, 1,
                                                cudaStreamSetCaptureDependencies) != cudaSuccess) {
            rc = PTA_ECUDA;
            break;
        }
        for (int b = 0; b < 2 && rc == PTA_OK; ++b) {
            if (cudaStreamBeginCaptureToGraph(r->cap2, bodies[b], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = PTA_ECUDA;
                break;
            }
            if (b == (int)LIST_BUILD) launch_rebuild(r->tab, 0, r->cap2);
            launch_prune(r->tab, 0, r->cap2);
            cudaGraph_t bout = nullptr;
            if (cudaStreamEndCapture(r->cap2, &bout) != cudaSuccess) rc = PTA_ECUDA;
        }
        if (rc != PTA_OK) break;
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 1], r->cap, cudaEventRecordExternal);
        launch_density(r->tab, 0, r->cap);
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 2], r->cap, cudaEventRecordExternal);
        launch_force(r->tab, MODE_STEP, r->cap);
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 3], r->cap, cudaEventRecordExternal);
    }
    cudaGraph_t gout = nullptr;
    e = cudaStreamEndCapture(r->cap, &gout);
    if (e != cudaSuccess || rc != PTA_OK) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return PTA_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    return PTA_OK;
}

static int capture_iters_flat(Runner *r, int iters, cudaGraphExec_t *out, bool timed) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < iters; ++i) {
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 0], r->cap, cudaEventRecordExternal);
        launch_rebuild(r->tab, 0, r->cap);
        launch_prune(r->tab, 0, r->cap);
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 1], r->cap, cudaEventRecordExternal);
        launch_density(r->tab, 0, r->cap);
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 2], r->cap, cudaEventRecordExternal);
        launch_force(r->tab, MODE_STEP, r->cap);
        if (timed) cudaEventRecordWithFlags(r->ev[4 * i + 3], r->cap, cudaEventRecordExternal);
    }
    cudaError_t e = cudaStreamEndCapture(r->cap, &g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    return PTA_OK;
}

// build the device launch table for the members' current descriptors
static int runner_upload(Runner *r) {
    const int k = (int)r->m.size();
    r->hspecs.resize(k);
    int blk_atom = 0, blk_cell = 0;
    std::vector<int> b2s_atom, b2s_cell;
    // launch groups by (precision, lanes, potential); the potential's FP32
    // constants are kernel parameters of the group's launches
    struct Key {
        int prec, L, sc76;
        PotF pf;
    };
    std::vector<Key> keys;
    std::vector<std::vector<int>> gb2s;
    auto group_of = [&](const Key &kk) -> int {
        for (size_t q = 0; q < keys.size(); ++q)
            if (keys[q].prec == kk.prec && keys[q].L == kk.L && keys[q].sc76 == kk.sc76 &&
                std::memcmp(&keys[q].pf, &kk.pf, sizeof(PotF)) == 0)
                return (int)q;
        if (keys.size() >= 8) return -1;
        keys.push_back(kk);
        gb2s.emplace_back();
        return (int)keys.size() - 1;
    };
    for (int i = 0; i < k; ++i) {
        SpecDev s = r->m[i]->hd;
        s.spec_index = i;
        s.blk_atom0 = blk_atom;
        blk_atom += s.nblk_atom;
        for (int b = 0; b < s.nblk_atom; ++b) b2s_atom.push_back(i);
        s.blk_cell0 = blk_cell;
        blk_cell += s.nblk_cell;
        for (int b = 0; b < s.nblk_cell; ++b) b2s_cell.push_back(i);
        PotF pf;
        std::memset(&pf, 0, sizeof(pf));
        pf.a = s.pot.f_a;
        pf.rc = s.pot.f_rc;
        pf.rc2 = s.pot.f_rc2;
        pf.Am = s.pot.f_Am;
        pf.Bm = s.pot.f_Bm;
        pf.An = s.pot.f_An;
        pf.Bn = s.pot.f_Bn;
        pf.eps = s.pot.f_eps;
        pf.ec = s.pot.f_ec;
        {
            const PotDev &q = s.pot;
            const double amm = q.m * hpow(q.a, q.m);
            pf.an = (float)hpow(q.a, q.n);
            pf.am = (float)hpow(q.a, q.m);
            pf.kn = (float)(q.eps * q.n * hpow(q.a, q.n));
            pf.bmq = (float)(q.Bm / amm);
            pf.ebn = (float)(q.eps * q.Bn);
            pf.c1 = (float)(-(q.An / q.Bn + q.rc));
            pf.fpsc = (float)(-0.5 * q.ec * amm);
        }
        pf.n = s.pot.n;
        pf.m = s.pot.m;
        const int g = group_of({s.prec, s.L, s.pot.sc76, pf});
        if (g < 0) return PTA_EUNSUPPORTED;
        s.blk_pair0 = (int)gb2s[g].size();
        for (int b = 0; b < s.nblk_pair; ++b) gb2s[g].push_back(i);
        r->hspecs[i] = s;
    }
    // one device block for all tables
    size_t words = b2s_atom.size() + b2s_cell.size();
    for (auto &v : gb2s) words += v.size();
    if (r->d_specs) {
        // tables already exist: only refresh the descriptors (same shapes)
        CK(cudaMemcpyAsync(r->d_specs, r->hspecs.data(), sizeof(SpecDev) * k,
                           cudaMemcpyHostToDevice, r->stream));
        return PTA_OK;
    }
    void *p = nullptr;
    const size_t bytes = round_up(sizeof(SpecDev) * k, 256) + round_up(4 * words, 256) +
                         round_up(8 * k, 256) * 2 + round_up(4 * k, 256) +
                         round_up(sizeof(pta_averages) * k, 256) +
                         round_up(sizeof(pta_coarse_result) * k, 256);
    CKR(dev_alloc(r, bytes, &p));
    char *c = (char *)p;
    r->d_specs = (SpecDev *)c;
    c += round_up(sizeof(SpecDev) * k, 256);
    int *tabs = (int *)c;
    c += round_up(4 * words, 256);
    r->d_nsteps = (long long *)c;
    c += round_up(8 * k, 256);
    r->d_du = (double *)c;
    c += round_up(8 * k, 256);
    r->d_ops = (int *)c;
    c += round_up(4 * k, 256);
    r->d_avg = (pta_averages *)c;
    c += round_up(sizeof(pta_averages) * k, 256);
    r->d_cres = (pta_coarse_result *)c;
    std::vector<int> all;
    all.insert(all.end(), b2s_atom.begin(), b2s_atom.end());
    all.insert(all.end(), b2s_cell.begin(), b2s_cell.end());
    for (auto &v : gb2s) all.insert(all.end(), v.begin(), v.end());
    CK(cudaMemcpyAsync(r->d_specs, r->hspecs.data(), sizeof(SpecDev) * k, cudaMemcpyHostToDevice,
                       r->stream));
    CK(cudaMemcpyAsync(tabs, all.data(), 4 * all.size(), cudaMemcpyHostToDevice, r->stream));
    Tab t{};
    t.specs = r->d_specs;
    t.nspec = k;
    t.b2s_atom = tabs;
    t.nblk_atom = (int)b2s_atom.size();
    t.b2s_cell = tabs + b2s_atom.size();
    t.nblk_cell = (int)b2s_cell.size();
    size_t off = b2s_atom.size() + b2s_cell.size();
    t.ngroups = (int)keys.size();
    for (size_t q = 0; q < keys.size(); ++q) {
        t.grp[q].prec = keys[q].prec;
        t.grp[q].L = keys[q].L;
        t.grp[q].sc76 = keys[q].sc76;
        t.grp[q].pf = keys[q].pf;
        t.grp[q].b2s = tabs + off;
        t.grp[q].nblk = (int)gb2s[q].size();
        off += gb2s[q].size();
    }
    r->tab = t;
    // pinned host mirrors
    const size_t hb = 8 * k * 2 + 4 * k + sizeof(pta_averages) * k + sizeof(pta_coarse_result) * k + 64;
    CK(cudaHostAlloc(&r->h_pin, hb, cudaHostAllocDefault));
    char *h = (char *)r->h_pin;
    r->h_nsteps = (long long *)h;
    h += 8 * k;
    r->h_du = (double *)h;
    h += 8 * k;
    r->h_ops = (int *)h;
    h += 4 * k + 4 * (k & 1);
    r->h_avg = (pta_averages *)h;
    h += sizeof(pta_averages) * k;
    r->h_cres = (pta_coarse_result *)h;
    return PTA_OK;
}

static int runner_create(pta_ctx *const *members, int k, Runner **out) {
    Range nv("pta_capture_graphs");
    Runner *r = new (std::nothrow) Runner();
    if (!r) return PTA_ENOMEM;
    r->m.assign(members, members + k);
    r->stream = members[0]->stream;
    r->alloc = members[0]->alloc;
    int rc = PTA_OK;
    if (cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&r->cap2, cudaStreamNonBlocking) != cudaSuccess)
        rc = PTA_ECUDA;
    if (rc == PTA_OK) rc = runner_upload(r);
    if (rc == PTA_OK) rc = capture_iters(r, CHUNK, &r->g_chunk);
    if (rc == PTA_OK) rc = capture_iters(r, 1, &r->g_one);
    if (rc != PTA_OK) {
        runner_free(r);
        return rc;
    }
    *out = r;
    return PTA_OK;
}

// make sure every member can hold nsteps samples; refresh descriptors if a
// series buffer moved
static int ensure_series(Runner *r, const int64_t *nsteps) {
    bool moved = false;
    for (size_t i = 0; i < r->m.size(); ++i) {
        pta_ctx *c = r->m[i];
        if (nsteps[i] <= c->hd.series_cap) continue;
        void *p = nullptr;
        const long long cap = std::max<long long>(nsteps[i], 2 * c->hd.series_cap);
        CKR(dev_alloc(c, 24 * (size_t)cap, &p));
        dev_release(c, c->hd.series);
        c->hd.series = (double *)p;
        c->hd.series_cap = cap;
        CK(cudaMemcpyAsync(c->d_self, &c->hd, sizeof(SpecDev), cudaMemcpyHostToDevice, c->stream));
        moved = true;
    }
    if (moved) {
        for (size_t i = 0; i < r->m.size(); ++i) {
            r->hspecs[i].series = r->m[i]->hd.series;
            r->hspecs[i].series_cap = r->m[i]->hd.series_cap;
        }
        CK(cudaMemcpyAsync(r->d_specs, r->hspecs.data(), sizeof(SpecDev) * r->m.size(),
                           cudaMemcpyHostToDevice, r->stream));
    }
    return PTA_OK;
}

static int status_of(const pta_averages &a) { return a.status; }

// add the event times of the last replayed timing graph (iters iterations)
static int collect_times(Runner *r, int iters) {
    CK(cudaEventSynchronize(r->ev[4 * (iters - 1) + 3]));
    for (int i = 0; i < iters; ++i) {
        float a = 0, b = 0, c = 0;
        CK(cudaEventElapsedTime(&a, r->ev[4 * i + 0], r->ev[4 * i + 1]));
        CK(cudaEventElapsedTime(&b, r->ev[4 * i + 1], r->ev[4 * i + 2]));
        CK(cudaEventElapsedTime(&c, r->ev[4 * i + 2], r->ev[4 * i + 3]));
        r->times.rebuild_ms += a;
        r->times.density_ms += b;
        r->times.force_ms += c;
        r->times.iterations += 1;
    }
    return PTA_OK;
}

static int runner_set_timing(Runner *r, int enable) {
    if (enable && !r->t_chunk) {
        r->ev.resize(4 * CHUNK);
        for (auto &e : r->ev) CK(cudaEventCreate(&e));
        CKR(capture_iters(r, CHUNK, &r->t_chunk, true));
        CKR(capture_iters(r, 1, &r->t_one, true));
    }
    r->timing = enable != 0;
    r->times = pta_kernel_times{};
    return PTA_OK;
}

// bursts of nsteps[i] steps for every member; averages to out (may be NULL);
// slot >= 0 also files the means for the coarse-step update
static int run_burst(Runner *r, const int64_t *nsteps, pta_averages *out, int slot) {
    Range nv("pta_fine_burst");
    const int k = (int)r->m.size();
    for (int i = 0; i < k; ++i) {
        if (r->m[i]->broken) return PTA_ECUDA;
        if (nsteps[i] < 0) return PTA_EINVAL;
    }
    CKR(ensure_series(r, nsteps));
    long long iters = 0;
    for (int i = 0; i < k; ++i) {
        r->h_nsteps[i] = nsteps[i];
        if (nsteps[i] > 0) iters = std::max<long long>(iters, nsteps[i] + 1);
    }
    CK(cudaMemcpyAsync(r->d_nsteps, r->h_nsteps, 8 * k, cudaMemcpyHostToDevice, r->stream));
    for (int i = 0; i < k; ++i)  // mean positions start from zero with every burst
        if (nsteps[i] > 0 && r->m[i]->hd.rsum)
            CK(cudaMemsetAsync(r->m[i]->hd.rsum, 0, 32 * (size_t)r->m[i]->hd.n, r->stream));
    launch_burst_begin(r->tab, r->d_nsteps, r->stream);
    CKR(launch_check());
    // adaptive burst lengths end on the device: after every chunk the host
    // asks whether any member is still running (d_ops/h_ops[0] serve as the
    // flag; the coarse-step update copies its own ops later)
    bool adaptive = false;
    for (int i = 0; i < k; ++i) adaptive |= r->m[i]->par.conv_lag > 0;
    auto still_running = [&](bool &run) -> int {
        run = true;
        if (!adaptive) return PTA_OK;
        launch_any_running(r->tab, r->d_ops, r->stream);
        CKR(launch_check());
        CK(cudaMemcpyAsync(r->h_ops, r->d_ops, sizeof(int), cudaMemcpyDeviceToHost, r->stream));
        CK(cudaStreamSynchronize(r->stream));
        run = r->h_ops[0] != 0;
        return PTA_OK;
    };
    bool run = true;
    if (r->timing) {
        for (long long q = 0; q < iters / CHUNK && run; ++q) {
            CK(cudaGraphLaunch(r->t_chunk, r->stream));
            CKR(collect_times(r, CHUNK));
            CKR(still_running(run));
        }
        for (long long q = 0; q < iters % CHUNK && run; ++q) {
            CK(cudaGraphLaunch(r->t_one, r->stream));
            CKR(collect_times(r, 1));
        }
    } else {
        for (long long q = 0; q < iters / CHUNK && run; ++q) {
            CK(cudaGraphLaunch(r->g_chunk, r->stream));
            CKR(still_running(run));
        }
        for (long long q = 0; q < iters % CHUNK && run; ++q) CK(cudaGraphLaunch(r->g_one, r->stream));
    }
    launch_burst_end(r->tab, slot, r->d_avg, r->stream);
    CKR(launch_check());
    CK(cudaMemcpyAsync(r->h_avg, r->d_avg, sizeof(pta_averages) * k, cudaMemcpyDeviceToHost,
                       r->stream));
    CK(cudaStreamSynchronize(r->stream));
    int rc = PTA_OK;
    for (int i = 0; i < k; ++i) {
        if (out) out[i] = r->h_avg[i];
        if (nsteps[i] > 0 && status_of(r->h_avg[i]) != PTA_OK && rc == PTA_OK)
            rc = status_of(r->h_avg[i]);
    }
    return rc;
}

static int run_strain(Runner *r, const double *d_eps) {
    const int k = (int)r->m.size();
    for (int i = 0; i < k; ++i) {
        if (!std::isfinite(d_eps[i])) return PTA_EINVAL;
        r->h_du[i] = d_eps[i] * r->m[i]->L_s;
    }
    CK(cudaMemcpyAsync(r->d_du, r->h_du, 8 * k, cudaMemcpyHostToDevice, r->stream));
    launch_strain(r->tab, r->d_du, r->stream);
    CKR(launch_check());
    for (int i = 0; i < k; ++i) r->m[i]->u += r->h_du[i];
    return PTA_OK;
}

// one tick: three bursts per member (initial or coarse increments), then the
// coarse-step kernel; `only_init` restricts the tick to members whose
// initial bursts are still to run (the others idle)
static int run_tick(Runner *r, pta_coarse_result *out, int only_init) {
    Range nv(only_init ? "pta_initial_bursts" : "pta_coarse_step");
    const int k = (int)r->m.size();
    std::vector<int> op(k);
    std::vector<int64_t> ns(k);
    bool any = false;
    for (int i = 0; i < k; ++i) {
        pta_ctx *c = r->m[i];
        op[i] = c->pta_init ? (only_init ? 0 : 2) : 1;
        ns[i] = op[i] ? c->par.burst_steps : 0;
        any |= op[i] != 0;
    }
    if (!any) return PTA_OK;
    std::vector<pta_averages> avg(3 * (size_t)k);
    std::vector<double> de(k);
    int rc_all = PTA_OK;
    for (int b = 0; b < 3; ++b) {
        bool anyde = false;
        for (int i = 0; i < k; ++i) {
            const pta_params &p = r->m[i]->par;
            double inc = 0;
            if (op[i] == 1)
                inc = (b == 0) ? 0.0 : p.strain_rate * p.Delta / 2.0;
            else if (op[i] == 2)
                inc = (b == 0) ? p.strain_rate * (p.h - p.Delta) : p.strain_rate * p.Delta / 2.0;
            de[i] = inc;
            anyde |= inc != 0.0;
        }
        if (anyde) CKR(run_strain(r, de.data()));
        int rc = run_burst(r, ns.data(), avg.data() + (size_t)b * k, b);
        if (rc == PTA_ECUDA) return rc;
        if (rc != PTA_OK && rc_all == PTA_OK) rc_all = rc;
    }
    for (int i = 0; i < k; ++i) r->h_ops[i] = op[i];
    CK(cudaMemcpyAsync(r->d_ops, r->h_ops, 4 * k, cudaMemcpyHostToDevice, r->stream));
    launch_pta_update(r->tab, r->d_ops, r->d_cres, r->stream);
    CKR(launch_check());
    CK(cudaMemcpyAsync(r->h_cres, r->d_cres, sizeof(pta_coarse_result) * k, cudaMemcpyDeviceToHost,
                       r->stream));
    CK(cudaStreamSynchronize(r->stream));
    for (int i = 0; i < k; ++i) {
        if (!op[i]) continue;
        pta_ctx *c = r->m[i];
        if (op[i] == 1) c->pta_init = true;
        if (out) {
            out[i] = r->h_cres[i];
            out[i].strain = c->u / c->L_s;
            int st = PTA_OK;
            for (int b = 0; b < 3; ++b) {
                out[i].burst[b] = avg[(size_t)b * k + i];
                if (st == PTA_OK) st = avg[(size_t)b * k + i].status;
            }
            out[i].status = st;
        }
    }
    return rc_all;
}

static int ctx_solo(pta_ctx *c, Runner **r) {
    if (c->broken) return PTA_ECUDA;
    if (!c->solo) {
        pta_ctx *m[1] = {c};
        CKR(runner_create(m, 1, &c->solo));
    }
    *r = c->solo;
    return PTA_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int pta_abi_version(void) { return PTA_ABI_VERSION; }

const char *pta_strerror(int s) {
    switch (s) {
        case PTA_OK: return "ok";
        case PTA_EINVAL: return "invalid argument";
        case PTA_ENOMEM: return "out of device memory";
        case PTA_ECUDA: return "CUDA error (context unusable)";
        case PTA_ENEIGH_OVERFLOW: return "neighbour-list capacity exceeded";
        case PTA_ENAN: return "non-finite energy during a burst";
        case PTA_ESTATE: return "call not valid in this state";
        case PTA_ERANGE: return "coordinate outside the mixed-precision range";
        case PTA_EUNSUPPORTED: return "unsupported option";
        case PTA_ECAPACITY: return "input exceeds the fixed scratch of the no-allocation entry point";
        default: return "unknown status";
    }
}

int pta_set_allocator(pta_alloc_fn alloc, pta_free_fn release, void *user) {
    if ((alloc == nullptr) != (release == nullptr)) return PTA_EINVAL;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.user = user;
    return PTA_OK;
}

int pta_default_params(pta_params *p) {
    if (!p) return PTA_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->dt_fs = 1.0;
    p->mass_amu = 26.9815385;
    p->skin = 2.0;
    p->h = 1.0;
    p->Delta = 0.2;
    p->strain_rate = 1e-3;
    p->tol_v[0] = 0.01;
    p->tol_v[1] = 0.05;
    p->tol_v[2] = 0.01;
    p->tol_j[0] = 0.08;
    p->tol_j[1] = 0.01;
    p->tol_j[2] = 0.05;
    p->floor[0] = 1e-12;
    p->floor[1] = 1e-12;
    p->floor[2] = 0.05;
    p->burst_steps = 2000;
    p->block_steps = 100;
    p->precision = PTA_PREC_FP64;
    p->neigh_cap = 0;
    p->lanes = 0;
    p->cell_tiles = 0;
    p->conv_lag = 0;
    p->mean_positions = 0;
    p->conv_tol[0] = p->conv_tol[1] = p->conv_tol[2] = 0.05;
    return PTA_OK;
}

int pta_default_potential(pta_potential *p) {
    if (!p) return PTA_EINVAL;
    p->kind = PTA_POT_SUTTON_CHEN_SF;
    p->eps = 3.3147e-2;
    p->a = 4.05;
    p->rc = 2.0 * 4.05;
    p->n = 7;
    p->m = 6;
    p->c = 1.0;
    p->c = equilibrium_c(*p, p->a);
    return PTA_OK;
}

size_t pta_footprint_bytes(const pta_specimen *spec, const pta_params *par) {
    pta_potential pot;
    pta_default_potential(&pot);
    if (!spec || !par || validate(spec, &pot, par) != PTA_OK) return 0;
    Sizes z;
    if (compute_sizes(*spec, pot, *par, &z) != PTA_OK) return 0;
    return footprint(z, par->precision);
}

static int ctx_alloc_all(pta_ctx *c, const Sizes &z) {
    SpecDev &s = c->hd;
    const size_t n = (size_t)z.n;
    const bool f64 = c->par.precision == PTA_PREC_FP64;
    const size_t p = f64 ? 32 : 16;
    void *q;
#define AL(field, bytes, type) \
    CKR(dev_alloc(c, (bytes), &q)); \
    s.field = (type)q;
    AL(pos[0], p * n, void *);
    AL(pos[1], p * n, void *);
    if (!f64) {
        AL(lo[0], 16 * n, float4 *);
        AL(lo[1], 16 * n, float4 *);
        AL(rel[0], 16 * (n + 1), float4 *);
        AL(rel[1], 16 * (n + 1), float4 *);
        AL(hsub, n, uint8_t *);
    }
    AL(posfp, p * (n + 1), void *);
    AL(vel, 32 * n, void *);
    AL(flags, n, uint8_t *);
    AL(ref, 16 * n, float4 *);
    AL(atom_cell, 4 * n, int *);
    AL(cell_cnt, 4 * (size_t)z.ncell, int *);
    AL(cell_start, 4 * ((size_t)z.ncell + 1), int *);
    AL(cell_tmp, 4 * n, int *);
    AL(cell_atoms, 4 * n, int *);
    AL(orig, 4 * n, int *);
    AL(perm_tmp, perm_layout(n, c->par.precision).total, void *);
    AL(nlist, 4 * z.list_words, int *);
    if (z.prune_on) {
        AL(plist, 4 * z.list_words, int *);
        AL(pnn, 4 * n * (size_t)z.L, int *);
        AL(pref, 16 * n, float4 *);
    }
    AL(nn, 4 * n, int *);
    {
        // block partials (8 doubles per block), then per group of 32 blocks
        // its partial (8 doubles) and its counter
        const size_t nb = (size_t)std::max(z.nblk_pair, z.nblk_atom);
        AL(part, 64 * (nb + 2 * (nb / 32 + 1)), double *);
    }
    AL(series, 24 * (size_t)z.series_cap, double *);
    AL(eval_out, 32 * n, double *);
    if (z.mean_pos) {
        AL(rsum, 32 * n, double *);
    }
    AL(stage, 48 * n, double *);
    AL(ctl, sizeof(SpecCtl), SpecCtl *);
#undef AL
    CKR(dev_alloc(c, sizeof(SpecDev), &q));
    c->d_self = (SpecDev *)q;
    return PTA_OK;
}

int pta_create(const pta_specimen *spec, const pta_potential *pot, double T0, uint64_t seed,
               const pta_params *par, void *stream, pta_ctx **out) {
    if (!out) return PTA_EINVAL;
    *out = nullptr;
    Range nv("pta_create");
    int rc = validate(spec, pot, par);
    if (rc != PTA_OK) return rc;
    if (!(T0 >= 0) || !std::isfinite(T0)) return PTA_EINVAL;
    pta_ctx *c = new (std::nothrow) pta_ctx();
    if (!c) return PTA_ENOMEM;
    c->spec = *spec;
    if (!(c->spec.grip_width > 0)) c->spec.grip_width = c->spec.a0;
    c->pot = *pot;
    c->par = *par;
    c->T0 = T0;
    c->seed = seed;
    c->stream = (cudaStream_t)stream;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->alloc = g_alloc;
    }
    Sizes z;
    rc = compute_sizes(c->spec, c->pot, c->par, &z);
    if (rc != PTA_OK) {
        delete c;
        return rc;
    }
    SpecDev &s = c->hd;
    std::memset(&s, 0, sizeof(s));
    s.n = (int)z.n;
    s.L = z.L;
    s.prec = c->par.precision;
    s.axis = c->spec.load_axis;
    s.cap = z.cap;
    s.cap_use = z.cap_use;
    s.nblk_pair = z.nblk_pair;
    s.nblk_atom = z.nblk_atom;
    s.nblk_cell = z.nblk_cell;
    for (int d = 0; d < 3; ++d) {
        s.ncl[d] = c->spec.n_cells[d];
        s.org[d] = z.org[d];
        s.f_org[d] = (float)z.org[d];
        s.nc[d] = z.nc[d];
    }
    s.a0 = c->spec.a0;
    s.grip_width = c->spec.grip_width;
    s.hcell = z.h;
    s.inv_h = 1.0 / z.h;
    s.f_inv_h = (float)s.inv_h;
    s.f_h = (float)z.h;
    s.f_q = (float)(z.h / 2.0);
    s.f_q8 = (float)(z.h / 16.0);
    s.f_q64 = (float)(z.h / 128.0);
    s.ncell = z.ncell;
    const double rl = c->pot.rc + c->par.skin;
    s.rl2 = rl * rl;
    s.f_rl2_lo = (float)(s.rl2 * (1.0 - 1e-5));
    s.f_rl2_hi = (float)(s.rl2 * (1.0 + 1e-5));
    s.half_skin2 = (float)(0.25 * c->par.skin * c->par.skin);
    s.prune_on = z.prune_on;
    {
        const double rp = c->pot.rc + z.prune_margin;
        s.f_rp2 = (float)(rp * rp * (1.0 + 1e-5));
        s.half_prune2 = (float)(0.25 * z.prune_margin * z.prune_margin);
    }
    s.pot = make_pot(c->pot);
    s.mass = c->par.mass_amu;
    s.dt = c->par.dt_fs;
    s.acc_half = 0.5 * s.dt * force_to_acc() / s.mass;
    s.ke_fac = 0.5 * s.mass * mv2_to_ev();
    double A0 = 1.0;
    for (int d = 0; d < 3; ++d)
        if (d != s.axis) A0 *= c->spec.n_cells[d] * c->spec.a0;
    s.t_fac = ev_a3_to_gpa() / A0;
    s.f_acc_half = (float)s.acc_half;
    s.f_ke_fac = (float)s.ke_fac;
    s.f_dt = (float)s.dt;
    s.block_steps = c->par.block_steps;
    s.pta_h = c->par.h;
    s.pta_Delta = c->par.Delta;
    for (int q = 0; q < 3; ++q) {
        s.tol_v[q] = c->par.tol_v[q];
        s.tol_j[q] = c->par.tol_j[q];
        s.floor_[q] = c->par.floor[q];
        s.conv_tol[q] = c->par.conv_tol[q];
    }
    s.conv_lag = c->par.conv_lag;
    s.series_cap = z.series_cap;
    c->L_s = c->spec.n_cells[s.axis] * c->spec.a0;
    rc = ctx_alloc_all(c, z);
    if (rc == PTA_OK) {
        if (cudaMemcpyAsync(c->d_self, &c->hd, sizeof(SpecDev), cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess)
            rc = PTA_ECUDA;
    }
    if (rc == PTA_OK && c->par.precision != PTA_PREC_FP64) {
        // the sentinel record (slot n) that pads every lane's list to a
        // multiple of four entries: far from every atom in both record
        // buffers and in the force pass's records, never written again
        static const float4 far_rec = {SENTINEL_COORD, SENTINEL_COORD, SENTINEL_COORD, 0.f};
        const size_t n = (size_t)s.n;
        float4 *dst[3] = {s.rel[0] + n, s.rel[1] + n, (float4 *)s.posfp + n};
        for (float4 *d : dst)
            if (cudaMemcpyAsync(d, &far_rec, sizeof(float4), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess)
                rc = PTA_ECUDA;
    }
    if (rc == PTA_OK) {
        const double kT = kb_ev() * T0;
        const double sigma = std::sqrt(kT / (s.mass * mv2_to_ev()));
        launch_create(c->hd, c->d_self, sigma, kT, seed, c->stream);
        launch_import(c->hd, c->d_self, c->stream);
        rc = launch_check();
    }
    if (rc == PTA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = PTA_ECUDA;
    if (rc != PTA_OK) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        dev_release_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return PTA_OK;
}

void pta_destroy(pta_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->batch) {
        // the batch keeps pointers to this member: detach it
        pta_batch *b = c->batch;
        for (auto &mm : b->r->m)
            if (mm == c) mm = nullptr;
    }
    runner_free(c->solo);
    dev_release_all(c);
    delete c;
}

int pta_natoms(const pta_ctx *c, int64_t *n) {
    if (!c || !n) return PTA_EINVAL;
    *n = c->hd.n;
    return PTA_OK;
}

// creation-order index of every slot (atoms are kept sorted by cell)
static int fetch_orig(pta_ctx *c, std::vector<int> &orig) {
    orig.resize((size_t)c->hd.n);
    CK(cudaMemcpyAsync(orig.data(), c->hd.orig, 4 * (size_t)c->hd.n, cudaMemcpyDeviceToHost,
                       c->stream));
    return PTA_OK;
}

int pta_get_layout(const pta_ctx *c, int32_t out[4]) {
    if (!c || !out) return PTA_EINVAL;
    out[0] = c->hd.L;
    out[1] = 1;
    out[2] = c->hd.cap_use;
    out[3] = c->hd.prune_on;
    return PTA_OK;
}

int pta_relax(pta_ctx *c, int64_t window, int64_t max_steps, double tol_gpa, pta_averages *out,
              int64_t *steps) {
    if (!c || window < 1 || max_steps < window || !(tol_gpa >= 0)) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    const int on = 1, off = 0;
    CK(cudaMemcpyAsync(&c->hd.ctl->relax, &on, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    int64_t total = 0;
    pta_averages a{};
    int rc = PTA_OK;
    while (rc == PTA_OK) {
        rc = run_burst(r, &window, &a, -1);
        if (rc != PTA_OK) break;
        total += a.nsteps;
        if (std::fabs(a.mean[2]) < tol_gpa || total + window > max_steps) break;
    }
    CK(cudaMemcpyAsync(&c->hd.ctl->relax, &off, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    launch_fix_right_grip(c->hd, c->d_self, c->stream);
    CKR(launch_check());
    CK(cudaStreamSynchronize(c->stream));
    if (rc == PTA_ECUDA) c->broken = true;
    if (out) *out = a;
    if (steps) *steps = total;
    return rc;
}

int pta_get_mean_positions(pta_ctx *c, double *out, int64_t n) {
    if (!c || !out || n != c->hd.n) return PTA_EINVAL;
    if (!c->hd.rsum) return PTA_EUNSUPPORTED;
    if (c->broken) return PTA_ECUDA;
    std::vector<double> buf(4 * (size_t)n);
    SpecCtl ctl;
    CK(cudaMemcpyAsync(buf.data(), c->hd.rsum, 32 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&ctl, c->hd.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (ctl.done < 1) return PTA_EINVAL;
    const double inv = (double)ctl.done;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) out[3 * i + d] = buf[4 * (size_t)i + d] / inv;
    return PTA_OK;
}

int pta_get_flags(pta_ctx *c, uint8_t *flags, int64_t n) {
    if (!c || !flags || n != c->hd.n) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    std::vector<uint8_t> f((size_t)n);
    std::vector<int> orig;
    CK(cudaMemcpyAsync(f.data(), c->hd.flags, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    CKR(fetch_orig(c, orig));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t p = 0; p < n; ++p) flags[orig[p]] = f[p];
    return PTA_OK;
}

int pta_apply_strain(pta_ctx *c, double d_eps) {
    if (!c) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    CKR(run_strain(r, &d_eps));
    CK(cudaStreamSynchronize(c->stream));
    return PTA_OK;
}

int pta_get_strain(const pta_ctx *c, double *strain) {
    if (!c || !strain) return PTA_EINVAL;
    *strain = c->u / c->L_s;
    return PTA_OK;
}

int pta_fine_burst(pta_ctx *c, int64_t nsteps, pta_averages *out) {
    if (!c || nsteps < 1) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    pta_averages a;
    int rc = run_burst(r, &nsteps, &a, -1);
    if (rc == PTA_ECUDA) c->broken = true;
    if (out) *out = a;
    return rc;
}

int pta_ramp_burst(pta_ctx *c, int64_t nsteps, double d_eps_per_step, pta_averages *out) {
    if (!c || nsteps < 1 || !std::isfinite(d_eps_per_step)) return PTA_EINVAL;
    if (c->par.conv_lag > 0) return PTA_EUNSUPPORTED;  // the ramp needs the whole burst
    Runner *r;
    CKR(ctx_solo(c, &r));
    c->grip_du = d_eps_per_step * c->L_s;
    CK(cudaMemcpyAsync(&c->hd.ctl->grip_du, &c->grip_du, sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    pta_averages a{};
    int rc = run_burst(r, &nsteps, &a, -1);
    if (rc == PTA_ECUDA) {
        c->broken = true;
        return rc;
    }
    // the grip advanced with every drift of the burst
    c->u += (double)a.nsteps * c->grip_du;
    c->grip_du = 0.0;
    CK(cudaMemcpyAsync(&c->hd.ctl->grip_du, &c->grip_du, sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (out) *out = a;
    return rc;
}

int pta_get_series(pta_ctx *c, double *series, int64_t max_steps, int64_t *count) {
    if (!c || !count || max_steps < 0) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    SpecCtl ctl;
    CK(cudaMemcpyAsync(&ctl, c->hd.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = ctl.done;
    const int64_t k = std::min<int64_t>(ctl.done, max_steps);
    if (series && k > 0) {
        CK(cudaMemcpyAsync(series, c->hd.series, 24 * (size_t)k, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return PTA_OK;
}

int pta_coarse_step(pta_ctx *c, pta_coarse_result *out) {
    if (!c) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    int rc = PTA_OK;
    if (!c->pta_init) {
        rc = run_tick(r, nullptr, 1);
        if (rc != PTA_OK) return rc;
    }
    rc = run_tick(r, out, 0);
    if (rc == PTA_ECUDA) c->broken = true;
    return rc;
}

int pta_coarse_update(pta_ctx *c, const double means[9], pta_coarse_result *out) {
    if (!c || !means) return PTA_EINVAL;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(means[i])) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    // the three burst means go where the bursts' ends file them (slots 0..2
    // of the slow-variable record), then the same update kernel runs
    double *d_r3 = &c->hd.ctl->pta.R3[0][0];
    CK(cudaMemcpyAsync(d_r3, means, 9 * sizeof(double), cudaMemcpyHostToDevice, r->stream));
    const int op = c->pta_init ? 2 : 1;
    r->h_ops[0] = op;
    CK(cudaMemcpyAsync(r->d_ops, r->h_ops, sizeof(int), cudaMemcpyHostToDevice, r->stream));
    launch_pta_update(r->tab, r->d_ops, r->d_cres, r->stream);
    CKR(launch_check());
    CK(cudaMemcpyAsync(r->h_cres, r->d_cres, sizeof(pta_coarse_result), cudaMemcpyDeviceToHost,
                       r->stream));
    CK(cudaStreamSynchronize(r->stream));
    c->pta_init = true;
    if (out) {
        *out = r->h_cres[0];
        out->strain = c->u / c->L_s;
        for (int b = 0; b < 3; ++b) {
            out->burst[b] = pta_averages{};
            for (int q = 0; q < 3; ++q) out->burst[b].mean[q] = means[3 * b + q];
        }
        out->status = PTA_OK;
    }
    return PTA_OK;
}

int pta_get_state(pta_ctx *c, double *pos, double *vel, int64_t n) {
    if (!c || n != c->hd.n) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    launch_export(c->hd, c->d_self, c->stream);
    CKR(launch_check());
    if (pos)
        CK(cudaMemcpyAsync(pos, c->hd.stage, 24 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    if (vel)
        CK(cudaMemcpyAsync(vel, c->hd.stage + 3 * (size_t)n, 24 * (size_t)n,
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PTA_OK;
}

int pta_set_state(pta_ctx *c, const double *pos, const double *vel, int64_t n) {
    if (!c || !pos || !vel || n != c->hd.n) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!std::isfinite(pos[i]) || !std::isfinite(vel[i])) return PTA_EINVAL;
    CK(cudaMemcpyAsync(c->hd.stage, pos, 24 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->hd.stage + 3 * (size_t)n, vel, 24 * (size_t)n, cudaMemcpyHostToDevice,
                       c->stream));
    launch_import(c->hd, c->d_self, c->stream);
    CKR(launch_check());
    CK(cudaStreamSynchronize(c->stream));
    int err = 0;
    CK(cudaMemcpy(&err, &c->hd.ctl->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & ERR_RANGE) {
        int zero = 0;
        CK(cudaMemcpy(&c->hd.ctl->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return PTA_ERANGE;
    }
    return PTA_OK;
}

int pta_forces(pta_ctx *c, double *f, double *pe, int64_t n, double obs[3]) {
    if (!c || n != c->hd.n) return PTA_EINVAL;
    Range nv("pta_forces");
    Runner *r;
    CKR(ctx_solo(c, &r));
    launch_rebuild(r->tab, 1, c->stream);
    launch_prune(r->tab, 1, c->stream);
    launch_density(r->tab, 1, c->stream);
    launch_force(r->tab, MODE_EVAL, c->stream);
    CKR(launch_check());
    std::vector<double> buf;
    if (f || pe) {
        buf.resize(4 * (size_t)n);
        CK(cudaMemcpyAsync(buf.data(), c->hd.eval_out, 32 * (size_t)n, cudaMemcpyDeviceToHost,
                           c->stream));
    }
    SpecCtl ctl;
    CK(cudaMemcpyAsync(&ctl, c->hd.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < n && (f || pe); ++i) {
        if (f)
            for (int d = 0; d < 3; ++d) f[3 * i + d] = buf[4 * i + d];
        if (pe) pe[i] = buf[4 * i + 3];
    }
    if (obs)
        for (int q = 0; q < 3; ++q) obs[q] = ctl.eval_obs[q];
    if (ctl.err & ERR_CHECK) return PTA_ECHECK;
    if (ctl.err & ERR_OVERFLOW) return PTA_ENEIGH_OVERFLOW;
#if PTA_CHECK
    if (ctl.err & ERR_NAN) return PTA_ENAN;  // the debug build's force scan
#endif
    if (ctl.err & ERR_GRID) return PTA_ERANGE;
    return PTA_OK;
}

int pta_get_neighbours(pta_ctx *c, int32_t *counts, int32_t *list, int64_t n, int32_t cap,
                       int32_t *max_count) {
    if (!c || n != c->hd.n || !max_count) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    const SpecDev &s = c->hd;
    SpecCtl ctl;
    launch_rebuild(r->tab, 1, c->stream);
    CKR(launch_check());
    const int L = s.L;
    std::vector<int> nn((size_t)n), raw;
    CK(cudaMemcpyAsync(nn.data(), s.nn, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&ctl, s.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    const long long W = 32 / L;
    const size_t words = (size_t)((n + W - 1) / W) * W * s.cap;
    raw.resize(words);
    std::vector<int> orig;
    CK(cudaMemcpyAsync(raw.data(), s.nlist, 4 * words, cudaMemcpyDeviceToHost, c->stream));
    CKR(fetch_orig(c, orig));
    CK(cudaStreamSynchronize(c->stream));
    *max_count = ctl.max_nn;
    if (ctl.err & ERR_CHECK) return PTA_ECHECK;
    if (ctl.err & ERR_OVERFLOW) return PTA_ENEIGH_OVERFLOW;
    int maxc = 0;
    for (int64_t u = 0; u < n; ++u) {
        const int64_t o = orig[u];
        if (counts) counts[o] = nn[u];
        maxc = std::max(maxc, nn[u]);
        if (nn[u] > cap) return PTA_EINVAL;
        for (int k = 0; k < nn[u]; ++k) {
            const int j = nl_j((unsigned)raw[(size_t)nl_index((int)u, k, L, s.cap)]);
            if (j < 0 || j >= n) return PTA_ECUDA;
            if (list) list[o * (int64_t)cap + k] = orig[j];
        }
    }
    *max_count = maxc;
    return PTA_OK;
}

// checkpoint layout: header, PtaDev, then the raw working arrays of the
// current position buffer, the velocities and the grip flags, in creation
// order (independent of the order the last list build left the atoms in)
struct CkptHeader {
    char magic[8];
    int32_t version, prec;
    int64_t n;
    double u;
    int32_t pta_init, L;
};

static size_t ckpt_payload(const pta_ctx *c) {
    const size_t n = (size_t)c->hd.n;
    const size_t p = (c->hd.prec == PTA_PREC_FP64) ? 32 : 16;
    return p * n + (c->hd.prec == PTA_PREC_FP64 ? 0 : 16 * n) + 32 * n + n;
}

int pta_save_state(pta_ctx *c, void *buf, size_t *len) {
    if (!c || !len) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    const size_t need = sizeof(CkptHeader) + sizeof(PtaDev) + ckpt_payload(c);
    if (!buf) {
        *len = need;
        return PTA_OK;
    }
    if (*len < need) return PTA_EINVAL;
    SpecCtl ctl;
    CK(cudaMemcpyAsync(&ctl, c->hd.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    launch_ckpt_move(c->hd, c->d_self, 1, c->stream);
    CKR(launch_check());
    CkptHeader h{};
    std::memcpy(h.magic, "PTACKPT", 8);
    h.version = 2;
    h.prec = c->hd.prec;
    h.n = c->hd.n;
    h.u = c->u;
    h.pta_init = c->pta_init ? 1 : 0;
    h.L = c->hd.L;
    char *o = (char *)buf;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t n = (size_t)c->hd.n;
    const size_t p = (c->hd.prec == PTA_PREC_FP64) ? 32 : 16;
    const PermLayout Lo = perm_layout(n, c->hd.prec);
    const char *t = (const char *)c->hd.perm_tmp;
    char *pl = o + sizeof(PtaDev);
    CK(cudaMemcpyAsync(pl, t + Lo.pos, p * n, cudaMemcpyDeviceToHost, c->stream));
    pl += p * n;
    if (c->hd.prec != PTA_PREC_FP64) {
        CK(cudaMemcpyAsync(pl, t + Lo.lo, 16 * n, cudaMemcpyDeviceToHost, c->stream));
        pl += 16 * n;
    }
    CK(cudaMemcpyAsync(pl, t + Lo.vel, 32 * n, cudaMemcpyDeviceToHost, c->stream));
    pl += 32 * n;
    CK(cudaMemcpyAsync(pl, t + Lo.flags, n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(o, &ctl.pta, sizeof(PtaDev));
    *len = need;
    return PTA_OK;
}

int pta_load_state(pta_ctx *c, const void *buf, size_t len) {
    if (!c || !buf) return PTA_EINVAL;
    if (c->broken) return PTA_ECUDA;
    const size_t need = sizeof(CkptHeader) + sizeof(PtaDev) + ckpt_payload(c);
    if (len < need) return PTA_EINVAL;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "PTACKPT", 8) != 0 || h.version != 2 || h.prec != c->hd.prec ||
        h.n != c->hd.n)
        return PTA_EINVAL;
    const char *o = (const char *)buf + sizeof(h);
    SpecCtl ctl;
    CK(cudaMemcpyAsync(&ctl, c->hd.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(&ctl.pta, o, sizeof(PtaDev));
    o += sizeof(PtaDev);
    ctl.rebuild = 1;
    ctl.phase = PH_IDLE;
    ctl.blocks_done = 0;
    const size_t n = (size_t)c->hd.n;
    const size_t p = (c->hd.prec == PTA_PREC_FP64) ? 32 : 16;
    const PermLayout Lo = perm_layout(n, c->hd.prec);
    char *t = (char *)c->hd.perm_tmp;
    CK(cudaMemcpyAsync(t + Lo.pos, o, p * n, cudaMemcpyHostToDevice, c->stream));
    o += p * n;
    if (c->hd.prec != PTA_PREC_FP64) {
        CK(cudaMemcpyAsync(t + Lo.lo, o, 16 * n, cudaMemcpyHostToDevice, c->stream));
        o += 16 * n;
    }
    CK(cudaMemcpyAsync(t + Lo.vel, o, 32 * n, cudaMemcpyHostToDevice, c->stream));
    o += 32 * n;
    CK(cudaMemcpyAsync(t + Lo.flags, o, n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->hd.ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, c->stream));
    launch_ckpt_move(c->hd, c->d_self, 0, c->stream);
    CKR(launch_check());
    CK(cudaStreamSynchronize(c->stream));
    c->u = h.u;
    c->pta_init = h.pta_init != 0;
    return PTA_OK;
}

int pta_batch_create(pta_ctx *const *members, int count, pta_batch **out) {
    if (!members || count < 1 || !out) return PTA_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!members[i] || members[i]->batch || members[i]->broken) return PTA_EINVAL;
        if (members[i]->stream != members[0]->stream) return PTA_EINVAL;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return PTA_EINVAL;
    }
    pta_batch *b = new (std::nothrow) pta_batch();
    if (!b) return PTA_ENOMEM;
    int rc = runner_create(members, count, &b->r);
    if (rc != PTA_OK) {
        delete b;
        return rc;
    }
    for (int i = 0; i < count; ++i) members[i]->batch = b;
    *out = b;
    return PTA_OK;
}

void pta_batch_destroy(pta_batch *b) {
    if (!b) return;
    for (auto *m : b->r->m)
        if (m) m->batch = nullptr;
    runner_free(b->r);
    delete b;
}

static int batch_ok(pta_batch *b) {
    if (!b || !b->r) return PTA_EINVAL;
    for (auto *m : b->r->m)
        if (!m) return PTA_ESTATE;
    return PTA_OK;
}

int pta_batch_apply_strain(pta_batch *b, const double *d_eps) {
    CKR(batch_ok(b));
    if (!d_eps) return PTA_EINVAL;
    CKR(run_strain(b->r, d_eps));
    CK(cudaStreamSynchronize(b->r->stream));
    return PTA_OK;
}

int pta_batch_fine_burst(pta_batch *b, const int64_t *nsteps, pta_averages *out) {
    CKR(batch_ok(b));
    if (!nsteps) return PTA_EINVAL;
    return run_burst(b->r, nsteps, out, -1);
}

int pta_batch_coarse_step(pta_batch *b, pta_coarse_result *out) {
    CKR(batch_ok(b));
    bool need_init = false;
    for (auto *m : b->r->m) need_init |= !m->pta_init;
    if (need_init) CKR(run_tick(b->r, nullptr, 1));
    return run_tick(b->r, out, 0);
}

int pta_batch_tick(pta_batch *b, pta_coarse_result *out) {
    CKR(batch_ok(b));
    return run_tick(b->r, out, 0);
}

int pta_set_timing(pta_ctx *c, int enable) {
    if (!c) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    return runner_set_timing(r, enable);
}

int pta_get_timing(pta_ctx *c, pta_kernel_times *out) {
    if (!c || !out) return PTA_EINVAL;
    Runner *r;
    CKR(ctx_solo(c, &r));
    *out = r->times;
    return PTA_OK;
}

int pta_batch_set_timing(pta_batch *b, int enable) {
    CKR(batch_ok(b));
    return runner_set_timing(b->r, enable);
}

int pta_batch_get_timing(pta_batch *b, pta_kernel_times *out) {
    CKR(batch_ok(b));
    if (!out) return PTA_EINVAL;
    *out = b->r->times;
    return PTA_OK;
}

}  // extern "C"
