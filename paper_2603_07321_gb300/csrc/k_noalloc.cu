// Neighbour lists without any device allocation.
//
// Some callers cannot allocate device memory: an application whose memory
// pool has already reserved the whole GPU for itself (so cudaMalloc fails
// or would steal from the pool's budget), or a latency-critical loop in
// which cudaMalloc / cudaFree, which may synchronise the device, are not
// allowed.  For them this file offers pta_neighbours_noalloc: the same cell
// binning and Verlet-list construction as the library's list build, with
// its scratch memory (cell counts, cell starts, the atoms' cells, the
// sorted cell contents) in one fixed array that lives in this file.  The
// caller supplies the positions and the output arrays; nothing is
// allocated.
//
// The scratch array is file-scope device memory of a fixed size, held by
// every GPU that loads the library until the process exits.  Every call
// shares it: each call clears what must start at zero, but calls that
// overlap on the GPU (two streams, two host threads) race on it, so they
// must be serialised by the caller.  Host code cannot use the array's name
// as a device address; the first call on each device looks the address up
// with cudaGetSymbolAddress (with that device current) and keeps it, so that
// first call should come before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "pta.h"

namespace {

constexpr int NA_MAX_ATOMS = PTA_NOALLOC_MAX_ATOMS;
constexpr int NA_MAX_CELLS = PTA_NOALLOC_MAX_CELLS;
constexpr int NA_TPB = 128;

// layout of the scratch words
constexpr size_t OFF_CNT = 0;                                   // cell counts / fill counters
constexpr size_t OFF_START = OFF_CNT + NA_MAX_CELLS;            // cell starts (ncell + 1)
constexpr size_t OFF_CELL = OFF_START + NA_MAX_CELLS + 1;       // cell of each atom
constexpr size_t OFF_TMP = OFF_CELL + NA_MAX_ATOMS;             // scattered cell contents
constexpr size_t OFF_SORTED = OFF_TMP + NA_MAX_ATOMS;           // cell contents by index
constexpr size_t OFF_MAX = OFF_SORTED + NA_MAX_ATOMS;           // largest neighbour count
constexpr size_t NA_WORDS = OFF_MAX + 8;

static __device__ __align__(256) int na_scratch[NA_WORDS];

struct Grid {
    double lo[3];
    double inv_h;
    int nc[3];
    int ncell;
    double rl2;
};

__global__ void na_clear(int *s, int ncell) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ncell) s[OFF_CNT + i] = 0;
    if (i == 0) s[OFF_MAX] = 0;
}

__global__ void na_bin(const double *__restrict__ pos, int n, Grid g, int *s) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int ci[3];
    for (int d = 0; d < 3; ++d) {
        int c = (int)floor((pos[3 * (size_t)a + d] - g.lo[d]) * g.inv_h);
        ci[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
    }
    const int c = ci[0] + g.nc[0] * (ci[1] + g.nc[1] * ci[2]);
    s[OFF_CELL + a] = c;
    atomicAdd(&s[OFF_CNT + c], 1);
}

// one block: exclusive scan of the counts into the starts, counts reset
__global__ void na_scan(int ncell, int *s) {
    __shared__ int carry;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += 1024) {
        const int c = base + threadIdx.x;
        const int v = c < ncell ? s[OFF_CNT + c] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int excl = carry + (w ? wsum[w - 1] : 0) + x - v;
        if (c < ncell) {
            s[OFF_START + c] = excl;
            s[OFF_CNT + c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) s[OFF_START + ncell] = carry;
}

__global__ void na_scatter(int n, int *s) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int c = s[OFF_CELL + a];
    const int slot = s[OFF_START + c] + atomicAdd(&s[OFF_CNT + c], 1);
    s[OFF_TMP + slot] = a;
}

// one warp per cell: contents in increasing atom index
__global__ void na_sort(int ncell, int *s) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    const int b = s[OFF_START + c], e = s[OFF_START + c + 1];
    for (int p = b + lane; p < e; p += 32) {
        const int v = s[OFF_TMP + p];
        int r = 0;
        for (int q = b; q < e; ++q) r += (s[OFF_TMP + q] < v);
        s[OFF_SORTED + b + r] = v;
    }
}

// one thread per atom: 27 cells, FP64 predicate (dx*dx + dy*dy) + dz*dz < rl^2
// without contraction; row-major output, cell order then atom index
__global__ void na_build(const double *__restrict__ pos, int n, Grid g, int cap,
                         int32_t *__restrict__ counts, int32_t *__restrict__ list, int *s) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const double xa = pos[3 * (size_t)a], ya = pos[3 * (size_t)a + 1], za = pos[3 * (size_t)a + 2];
    const int c = s[OFF_CELL + a];
    const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = cx + dx;
                if (x < 0 || x >= g.nc[0]) continue;
                const int cc = x + g.nc[0] * (y + g.nc[1] * z);
                for (int p = s[OFF_START + cc]; p < s[OFF_START + cc + 1]; ++p) {
                    const int j = s[OFF_SORTED + p];
                    if (j == a) continue;
                    const double ex = pos[3 * (size_t)j] - xa, ey = pos[3 * (size_t)j + 1] - ya,
                                 ez = pos[3 * (size_t)j + 2] - za;
                    const double r2 =
                        __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    if (r2 < g.rl2) {
                        if (cnt < cap) list[(size_t)a * cap + cnt] = j;
                        ++cnt;
                    }
                }
            }
        }
    }
    counts[a] = cnt < cap ? cnt : cap;
    atomicMax(&s[OFF_MAX], cnt);
}

std::mutex g_mu;
int *g_ptr[64] = {nullptr};

// set-up, once per device, with that device current: the device address of
// the scratch array (its host-side name is only a stand-in)
int scratch_address(int **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return PTA_ECUDA;
        }
        g_ptr[dev] = (int *)p;
    }
    *out = g_ptr[dev];
    return PTA_OK;
}

}  // namespace

extern "C" int pta_neighbours_noalloc(const double *pos_dev, int32_t n, const double box_lo[3],
                                      const double box_hi[3], double rlist, int32_t cap,
                                      int32_t *counts_dev, int32_t *list_dev, int32_t *max_count,
                                      void *stream) {
    if (!pos_dev || !box_lo || !box_hi || !counts_dev || !list_dev || !max_count)
        return PTA_EINVAL;
    if (n < 1 || cap < 1 || !(rlist > 0) || !std::isfinite(rlist)) return PTA_EINVAL;
    if (n > NA_MAX_ATOMS) return PTA_ECAPACITY;
    Grid g;
    const double h = rlist * (1.0 + 1e-4);
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        if (!(box_hi[d] >= box_lo[d]) || !std::isfinite(box_lo[d]) || !std::isfinite(box_hi[d]))
            return PTA_EINVAL;
        g.lo[d] = box_lo[d];
        const double span = box_hi[d] - box_lo[d];
        if (span / h > NA_MAX_CELLS) return PTA_ECAPACITY;
        g.nc[d] = (int)std::floor(span / h) + 1;
        ncell *= g.nc[d];
    }
    if (ncell > NA_MAX_CELLS) return PTA_ECAPACITY;
    g.ncell = (int)ncell;
    g.inv_h = 1.0 / h;
    g.rl2 = rlist * rlist;
    int *s = nullptr;
    int rc = scratch_address(&s);
    if (rc != PTA_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (n + NA_TPB - 1) / NA_TPB;
    na_clear<<<(g.ncell + 255) / 256, 256, 0, st>>>(s, g.ncell);
    na_bin<<<nb, NA_TPB, 0, st>>>(pos_dev, n, g, s);
    na_scan<<<1, 1024, 0, st>>>(g.ncell, s);
    na_scatter<<<nb, NA_TPB, 0, st>>>(n, s);
    na_sort<<<(g.ncell + 7) / 8, 256, 0, st>>>(g.ncell, s);
    na_build<<<nb, NA_TPB, 0, st>>>(pos_dev, n, g, cap, counts_dev, list_dev, s);
    if (cudaGetLastError() != cudaSuccess) return PTA_ECUDA;
    int mx = 0;
    if (cudaMemcpyAsync(&mx, s + OFF_MAX, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    *max_count = mx;
    return mx > cap ? PTA_ENEIGH_OVERFLOW : PTA_OK;
}
