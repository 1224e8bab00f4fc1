/*
 * FP64 CPU oracle for the fine-burst hot path of Practical Time Averaging
 * molecular dynamics (Baruah, Chatterjee, Acharya, Wang; arXiv 2603.07321).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, link or
 * call this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library; both sides are written separately from the paper and
 * from the textbook definitions cited beside each function.
 *
 * Plain IEEE double everywhere, built with -ffp-contract=off so that no
 * fused multiply-add changes a rounding.  Loops run over atoms in index
 * order; OpenMP only splits the outer atom loop, and every atom sums its
 * own terms in ascending neighbour order, so results do not depend on the
 * thread count.
 *
 * Units: Angstrom, femtosecond, atomic mass unit, electron-volt, kelvin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------
 * Physical constants (CODATA 2018): elementary charge and atomic mass unit
 * in SI, Boltzmann constant in J/K.  The unit conversions follow from them.
 * ------------------------------------------------------------------- */
static const double OR_E_CHARGE = 1.602176634e-19; /* J per eV          */
static const double OR_AMU = 1.66053906660e-27;    /* kg per amu        */
static const double OR_KB_SI = 1.380649e-23;       /* J per K           */

/* 1 amu * A^2 / fs^2 expressed in eV */
static double or_mv2_to_ev(void) { return OR_AMU * 1e-20 / 1e-30 / OR_E_CHARGE; }
/* 1 eV / (A * amu) expressed in A / fs^2 */
static double or_force_to_acc(void) { return OR_E_CHARGE / (1e-10 * OR_AMU) * 1e10 / 1e30; }
/* Boltzmann constant in eV / K */
static double or_kb_ev(void) { return OR_KB_SI / OR_E_CHARGE; }
/* 1 eV / A^3 in GPa */
static double or_ev_per_a3_to_gpa(void) { return OR_E_CHARGE / 1e-30 / 1e9; }

OR_API void or_constants(double out[4]) {
    out[0] = or_mv2_to_ev();
    out[1] = or_force_to_acc();
    out[2] = or_kb_ev();
    out[3] = or_ev_per_a3_to_gpa();
}

/* ---------------------------------------------------------------------
 * Potential.  The paper's Eq. (pe) is the EAM form
 *     U = 1/2 sum_a sum_{b!=a} V(r_ab) + sum_a B(rho_a),  rho_a = sum_b rho(r_ab).
 * The stand-in is the Sutton-Chen analytic EAM (Phil. Mag. Lett. 61, 139
 * (1990)):  V(r) = eps*phi_n(r),  rho(r) = phi_m(r),  B(rho) = -eps*c*sqrt(rho)
 * with phi_k(r) = (a/r)^k.  The cutoff is made smooth by the shifted-force
 * form  phi_k(r) - phi_k(rc) - phi_k'(rc)(r - rc)  for r < rc, zero beyond,
 * which is continuous with a continuous first derivative at rc.
 * ------------------------------------------------------------------- */
typedef struct {
    double eps; /* eV   */
    double c;   /* dimensionless */
    double a;   /* A    */
    double rc;  /* A    */
    int n, m;   /* pair and density exponents */
} or_pot;

static double or_ipow(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; i++) r = r * x;
    return r;
}

/* shifted-force phi_k(r) for r < rc */
static double or_phi(const or_pot *p, int k, double r) {
    if (!(r < p->rc)) return 0.0;
    double sr = or_ipow(p->a / r, k);
    double sc = or_ipow(p->a / p->rc, k);
    return sr - sc + ((double)k / p->rc) * sc * (r - p->rc);
}

/* d/dr of the shifted-force phi_k(r) for r < rc */
static double or_dphi(const or_pot *p, int k, double r) {
    if (!(r < p->rc)) return 0.0;
    double sr = or_ipow(p->a / r, k);
    double sc = or_ipow(p->a / p->rc, k);
    return -((double)k / r) * sr + ((double)k / p->rc) * sc;
}

OR_API double or_phi_value(const or_pot *p, int k, double r) { return or_phi(p, k, r); }
OR_API double or_dphi_value(const or_pot *p, int k, double r) { return or_dphi(p, k, r); }

/* Embedding B(rho) = -eps c sqrt(rho) and its derivative; an atom with no
 * neighbour inside rc has rho = 0, B = 0, and its B'(rho) never multiplies
 * a non-zero phi_m', so it is set to 0 there. */
static double or_embed(const or_pot *p, double rho) { return -p->eps * p->c * sqrt(rho); }
static double or_dembed(const or_pot *p, double rho) {
    return rho > 0.0 ? -p->eps * p->c / (2.0 * sqrt(rho)) : 0.0;
}

/* ---------------------------------------------------------------------
 * c from the equilibrium of the perfect FCC crystal at lattice constant a0
 * under the cut-off potential:  E(L) per atom = eps[ 1/2 S_n(L) - c sqrt(S_m(L)) ]
 * with S_k(L) = sum over lattice vectors t != 0 of phi_k(|t| L / a0 ...).
 * dE/dL = 0 at L = a0 gives  c = sqrt(S_m) * D_n / D_m,
 * D_k = sum_t |t| phi_k'(|t|).  The sums run over every lattice vector of
 * the FCC Bravais lattice with |t| < rc (enumerated, not tabulated).
 * ------------------------------------------------------------------- */
static void or_lattice_sums(const or_pot *p, double a0, double *S_n, double *S_m, double *D_n,
                            double *D_m) {
    static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    int R = (int)ceil(p->rc / a0) + 1;
    double sn = 0, sm = 0, dn = 0, dm = 0;
    for (int i = -R; i <= R; i++)
        for (int j = -R; j <= R; j++)
            for (int k = -R; k <= R; k++)
                for (int b = 0; b < 4; b++) {
                    double x = a0 * (i + basis[b][0]);
                    double y = a0 * (j + basis[b][1]);
                    double z = a0 * (k + basis[b][2]);
                    double r2 = (x * x + y * y) + z * z;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    if (!(r < p->rc)) continue;
                    sn = sn + or_phi(p, p->n, r);
                    sm = sm + or_phi(p, p->m, r);
                    dn = dn + r * or_dphi(p, p->n, r);
                    dm = dm + r * or_dphi(p, p->m, r);
                }
    *S_n = sn;
    *S_m = sm;
    *D_n = dn;
    *D_m = dm;
}

OR_API double or_sc_c_equilibrium(const or_pot *p, double a0) {
    double sn, sm, dn, dm;
    or_lattice_sums(p, a0, &sn, &sm, &dn, &dm);
    return sqrt(sm) * dn / dm;
}

/* cohesive energy per atom of the perfect crystal at lattice constant a0 */
OR_API double or_sc_cohesive_energy(const or_pot *p, double a0) {
    double sn, sm, dn, dm;
    or_lattice_sums(p, a0, &sn, &sm, &dn, &dm);
    return p->eps * (0.5 * sn - p->c * sqrt(sm));
}

/* ---------------------------------------------------------------------
 * Specimen (problem-setup section of the paper): an FCC block with the
 * cube axes along [100],[010],[001], n_x * n_y * n_z conventional cells,
 * four atoms per cell.  Atom index = 4 * (i + nx*(j + ny*k)) + b.
 * ------------------------------------------------------------------- */
OR_API long or_fcc_lattice(int nx, int ny, int nz, double a0, double *pos) {
    static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    long idx = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int b = 0; b < 4; b++) {
                    pos[3 * idx + 0] = a0 * ((double)i + basis[b][0]);
                    pos[3 * idx + 1] = a0 * ((double)j + basis[b][1]);
                    pos[3 * idx + 2] = a0 * ((double)k + basis[b][2]);
                    idx++;
                }
    return idx;
}

/* Grips (boundary conditions section): the left set holds the atoms whose
 * coordinate along the load axis lies within `width` of the lowest one, the
 * right set those within `width` of the highest one, both inclusive with a
 * tolerance tol.  flags: 0 mobile, 1 left grip, 2 right grip. */
OR_API void or_grip_flags(const double *pos, long n, int axis, double width, double tol,
                          uint8_t *flags) {
    double lo = pos[axis], hi = pos[axis];
    for (long i = 0; i < n; i++) {
        double x = pos[3 * i + axis];
        if (x < lo) lo = x;
        if (x > hi) hi = x;
    }
    for (long i = 0; i < n; i++) {
        double x = pos[3 * i + axis];
        flags[i] = 0;
        if (x <= lo + width + tol)
            flags[i] = 1;
        else if (x >= hi - width - tol)
            flags[i] = 2;
    }
}

/* ---------------------------------------------------------------------
 * Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with an
 * S-box-free permutation, the key bumped by the Weyl constants between
 * rounds.
 * ------------------------------------------------------------------- */
OR_API void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 = k0 + 0x9E3779B9u;
            k1 = k1 + 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* uniform in (0,1) from two 32-bit words: 53 random bits k, u = (k + 1/2) 2^-53 */
static double or_u53(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)k * (1.0 / 9007199254740992.0) + (1.0 / 18014398509481984.0);
}

/* Three standard normals for atom `idx` from the seed: two Philox blocks with
 * counters (idx_lo, idx_hi, block, 0), key (seed_lo, seed_hi); each block
 * gives two uniforms and Box-Muller turns them into two normals. */
OR_API void or_atom_normals(uint64_t seed, uint64_t idx, double z[3]) {
    double g[4];
    for (uint32_t blk = 0; blk < 2; blk++) {
        uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), blk, 0u};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        double u1 = or_u53(w[0], w[1]);
        double u2 = or_u53(w[2], w[3]);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 6.283185307179586 * u2;
        g[2 * blk + 0] = rad * cos(ang);
        g[2 * blk + 1] = rad * sin(ang);
    }
    z[0] = g[0];
    z[1] = g[1];
    z[2] = g[2];
}

/* Maxwell-Boltzmann initial velocities at T0 (boundary-conditions section):
 * grip atoms get v = 0; every mobile component is drawn from N(0, kT/m); the
 * mean over mobile atoms is removed and the set is scaled so that the kinetic
 * energy equals (3 N_mob - 3) k T0 / 2 exactly. */
OR_API void or_mb_velocities(long n, const uint8_t *flags, double T0, double mass, uint64_t seed,
                             double *vel) {
    const double kT = or_kb_ev() * T0;
    const double sig = sqrt(kT / (mass * or_mv2_to_ev()));
    long nmob = 0;
    double mean[3] = {0, 0, 0};
    for (long i = 0; i < n; i++) {
        if (flags[i] != 0) {
            vel[3 * i] = vel[3 * i + 1] = vel[3 * i + 2] = 0.0;
            continue;
        }
        double z[3];
        or_atom_normals(seed, (uint64_t)i, z);
        for (int d = 0; d < 3; d++) {
            vel[3 * i + d] = sig * z[d];
            mean[d] = mean[d] + vel[3 * i + d];
        }
        nmob++;
    }
    if (nmob < 2 || !(T0 > 0.0)) {
        for (long i = 0; i < 3 * n; i++) vel[i] = 0.0;
        return;
    }
    for (int d = 0; d < 3; d++) mean[d] = mean[d] / (double)nmob;
    double ke = 0.0;
    for (long i = 0; i < n; i++) {
        if (flags[i] != 0) continue;
        for (int d = 0; d < 3; d++) {
            vel[3 * i + d] = vel[3 * i + d] - mean[d];
            ke = ke + vel[3 * i + d] * vel[3 * i + d];
        }
    }
    ke = 0.5 * mass * ke * or_mv2_to_ev();
    double target = 0.5 * (double)(3 * nmob - 3) * kT;
    double s = sqrt(target / ke);
    for (long i = 0; i < n; i++) {
        if (flags[i] != 0) continue;
        for (int d = 0; d < 3; d++) vel[3 * i + d] = vel[3 * i + d] * s;
    }
}

/* ---------------------------------------------------------------------
 * Neighbour pairs.  Definition: j is a neighbour of i iff j != i and
 * (dx*dx + dy*dy) + dz*dz < rcut*rcut with d = r_j - r_i, evaluated in
 * double without contraction.  Lists are full (both (i,j) and (j,i)),
 * ascending in j, stored row-major with capacity `cap` per atom.
 * Returns the largest count seen (> cap means the lists were truncated).
 * ------------------------------------------------------------------- */
static int or_is_pair(const double *pos, long i, long j, double rc2) {
    double dx = pos[3 * j + 0] - pos[3 * i + 0];
    double dy = pos[3 * j + 1] - pos[3 * i + 1];
    double dz = pos[3 * j + 2] - pos[3 * i + 2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    return r2 < rc2;
}

OR_API int or_pairs_brute(const double *pos, long n, double rcut, int cap, int *counts,
                          int *list) {
    const double rc2 = rcut * rcut;
    int maxc = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxc)
    for (long i = 0; i < n; i++) {
        int c = 0;
        for (long j = 0; j < n; j++) {
            if (j == i) continue;
            if (or_is_pair(pos, i, j, rc2)) {
                if (c < cap) list[i * (long)cap + c] = (int)j;
                c++;
            }
        }
        counts[i] = c;
        if (c > maxc) maxc = c;
    }
    return maxc;
}

/* Same pair set found through a uniform cell grid of edge >= rcut over the
 * bounding box: candidates come from the 27 cells around an atom's cell and
 * are then put in ascending order, so the output equals or_pairs_brute's. */
OR_API int or_pairs_cells(const double *pos, long n, double rcut, int cap, int *counts,
                          int *list) {
    const double rc2 = rcut * rcut;
    if (n <= 0) return 0;
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) lo[d] = hi[d] = pos[d];
    for (long i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) {
            if (pos[3 * i + d] < lo[d]) lo[d] = pos[3 * i + d];
            if (pos[3 * i + d] > hi[d]) hi[d] = pos[3 * i + d];
        }
    int nc[3];
    for (int d = 0; d < 3; d++) {
        nc[d] = (int)floor((hi[d] - lo[d]) / rcut) + 1;
        if (nc[d] < 1) nc[d] = 1;
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int *cell_of = (int *)malloc(sizeof(int) * n);
    long *head = (long *)malloc(sizeof(long) * (ncell + 1));
    long *members = (long *)malloc(sizeof(long) * n);
    for (long c = 0; c <= ncell; c++) head[c] = 0;
    for (long i = 0; i < n; i++) {
        int ci[3];
        for (int d = 0; d < 3; d++) {
            ci[d] = (int)floor((pos[3 * i + d] - lo[d]) / rcut);
            if (ci[d] < 0) ci[d] = 0;
            if (ci[d] >= nc[d]) ci[d] = nc[d] - 1;
        }
        cell_of[i] = ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]);
        head[cell_of[i] + 1]++;
    }
    for (long c = 0; c < ncell; c++) head[c + 1] += head[c];
    {
        long *fill = (long *)malloc(sizeof(long) * ncell);
        for (long c = 0; c < ncell; c++) fill[c] = head[c];
        for (long i = 0; i < n; i++) members[fill[cell_of[i]]++] = i; /* ascending within a cell */
        free(fill);
    }
    int maxc = 0;
#pragma omp parallel reduction(max : maxc)
    {
        int tmpcap = 1024;
        int *tmp = (int *)malloc(sizeof(int) * tmpcap);
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < n; i++) {
            int c = 0;
            int ci = cell_of[i];
            int cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / (nc[0] * nc[1]);
            for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int x = cx + dx, y = cy + dy, z = cz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= nc[0] || y >= nc[1] || z >= nc[2])
                            continue;
                        long cc = x + (long)nc[0] * (y + (long)nc[1] * z);
                        for (long q = head[cc]; q < head[cc + 1]; q++) {
                            long j = members[q];
                            if (j == i) continue;
                            if (or_is_pair(pos, i, j, rc2)) {
                                if (c == tmpcap) {
                                    tmpcap *= 2;
                                    tmp = (int *)realloc(tmp, sizeof(int) * tmpcap);
                                }
                                tmp[c++] = (int)j;
                            }
                        }
                    }
            /* insertion sort into ascending j */
            for (int a = 1; a < c; a++) {
                int v = tmp[a], b = a - 1;
                while (b >= 0 && tmp[b] > v) {
                    tmp[b + 1] = tmp[b];
                    b--;
                }
                tmp[b + 1] = v;
            }
            for (int a = 0; a < c && a < cap; a++) list[i * (long)cap + a] = tmp[a];
            counts[i] = c;
            if (c > maxc) maxc = c;
        }
        free(tmp);
    }
    free(cell_of);
    free(head);
    free(members);
    return maxc;
}

/* ---------------------------------------------------------------------
 * EAM energy and forces on a given full neighbour list (pairs at distance
 * >= rc contribute nothing).  Eq. (pe) for the energy, Eq. (f_int) for the
 * force F_a = -dU/dr_a, which for this potential reads
 *   F_i = sum_j [ eps phi_n'(r_ij) + (B'(rho_i) + B'(rho_j)) phi_m'(r_ij) ] (r_j - r_i)/r_ij.
 * Outputs per atom: force f (3 per atom), energy share pe_i =
 * 1/2 eps sum_j phi_n(r_ij) + B(rho_i), density rho_i.
 * ------------------------------------------------------------------- */
OR_API void or_eam(const double *pos, long n, const or_pot *p, int cap, const int *counts,
                   const int *list, double *f, double *pe, double *rho) {
    double *dB = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        double s = 0.0;
        for (int q = 0; q < counts[i]; q++) {
            long j = list[i * (long)cap + q];
            double dx = pos[3 * j + 0] - pos[3 * i + 0];
            double dy = pos[3 * j + 1] - pos[3 * i + 1];
            double dz = pos[3 * j + 2] - pos[3 * i + 2];
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            s = s + or_phi(p, p->m, r);
        }
        rho[i] = s;
        dB[i] = or_dembed(p, s);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        double fx = 0, fy = 0, fz = 0, e = 0;
        for (int q = 0; q < counts[i]; q++) {
            long j = list[i * (long)cap + q];
            double dx = pos[3 * j + 0] - pos[3 * i + 0];
            double dy = pos[3 * j + 1] - pos[3 * i + 1];
            double dz = pos[3 * j + 2] - pos[3 * i + 2];
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            if (!(r < p->rc)) continue;
            double coef = p->eps * or_dphi(p, p->n, r) + (dB[i] + dB[j]) * or_dphi(p, p->m, r);
            fx = fx + coef * dx / r;
            fy = fy + coef * dy / r;
            fz = fz + coef * dz / r;
            e = e + or_phi(p, p->n, r);
        }
        f[3 * i + 0] = fx;
        f[3 * i + 1] = fy;
        f[3 * i + 2] = fz;
        pe[i] = 0.5 * p->eps * e + or_embed(p, rho[i]);
    }
    free(dB);
}

/* Same energy and forces in a cubic periodic box of edge L (> 2 rc), by the
 * minimum-image convention and a brute-force double loop.  Used only to pin
 * the potential against closed-form lattice sums. */
OR_API void or_eam_periodic(const double *pos, long n, double L, const or_pot *p, double *f,
                            double *pe, double *rho) {
    double *dB = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        double s = 0.0;
        for (long j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            for (int k = 0; k < 3; k++) {
                d[k] = pos[3 * j + k] - pos[3 * i + k];
                d[k] = d[k] - L * nearbyint(d[k] / L);
            }
            double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            s = s + or_phi(p, p->m, r);
        }
        rho[i] = s;
        dB[i] = or_dembed(p, s);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        double fv[3] = {0, 0, 0}, e = 0;
        for (long j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            for (int k = 0; k < 3; k++) {
                d[k] = pos[3 * j + k] - pos[3 * i + k];
                d[k] = d[k] - L * nearbyint(d[k] / L);
            }
            double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            if (!(r < p->rc)) continue;
            double coef = p->eps * or_dphi(p, p->n, r) + (dB[i] + dB[j]) * or_dphi(p, p->m, r);
            for (int k = 0; k < 3; k++) fv[k] = fv[k] + coef * d[k] / r;
            e = e + or_phi(p, p->n, r);
        }
        for (int k = 0; k < 3; k++) f[3 * i + k] = fv[k];
        pe[i] = 0.5 * p->eps * e + or_embed(p, rho[i]);
    }
    free(dB);
}

/* Forces and energies of a few chosen atoms of a large specimen: rho of each
 * chosen atom and of each of its neighbours is summed directly, then the
 * force formula above is applied.  Neighbours come from or_pairs_cells. */
OR_API int or_eam_sampled(const double *pos, long n, const or_pot *p, long nsamp,
                          const long *idx, double *f, double *pe) {
    const int cap = 512;
    int *counts = (int *)malloc(sizeof(int) * n);
    int *list = (int *)malloc(sizeof(int) * (size_t)n * cap);
    int maxc = or_pairs_cells(pos, n, p->rc, cap, counts, list);
    if (maxc > cap) {
        free(counts);
        free(list);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long s = 0; s < nsamp; s++) {
        long i = idx[s];
        double rho_i = 0.0;
        for (int q = 0; q < counts[i]; q++) {
            long j = list[i * (long)cap + q];
            double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1],
                   dz = pos[3 * j + 2] - pos[3 * i + 2];
            rho_i = rho_i + or_phi(p, p->m, sqrt((dx * dx + dy * dy) + dz * dz));
        }
        double dBi = or_dembed(p, rho_i);
        double fv[3] = {0, 0, 0}, e = 0;
        for (int q = 0; q < counts[i]; q++) {
            long j = list[i * (long)cap + q];
            double rho_j = 0.0;
            for (int w = 0; w < counts[j]; w++) {
                long k = list[j * (long)cap + w];
                double ex = pos[3 * k] - pos[3 * j], ey = pos[3 * k + 1] - pos[3 * j + 1],
                       ez = pos[3 * k + 2] - pos[3 * j + 2];
                rho_j = rho_j + or_phi(p, p->m, sqrt((ex * ex + ey * ey) + ez * ez));
            }
            double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                           pos[3 * j + 2] - pos[3 * i + 2]};
            double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            double coef =
                p->eps * or_dphi(p, p->n, r) + (dBi + or_dembed(p, rho_j)) * or_dphi(p, p->m, r);
            for (int k = 0; k < 3; k++) fv[k] = fv[k] + coef * d[k] / r;
            e = e + or_phi(p, p->n, r);
        }
        for (int k = 0; k < 3; k++) f[3 * s + k] = fv[k];
        pe[s] = 0.5 * p->eps * e + or_embed(p, rho_i);
    }
    free(counts);
    free(list);
    return 0;
}

/* ---------------------------------------------------------------------
 * State functions, Eq. (state_variables):
 *   K = 1/2 sum m v.v,  U = total EAM energy,
 *   T = (-sum_{a in right grip} F_int,a . e) / A0,  e the load axis unit vector.
 * out[0] = K (eV), out[1] = U (eV), out[2] = T (GPa).
 * ------------------------------------------------------------------- */
static void or_observe(long n, const double *vel, const double *f, const double *pe,
                       const uint8_t *flags, double mass, int axis, double A0, double out[3]) {
    double k = 0, u = 0, r = 0;
    for (long i = 0; i < n; i++) {
        k = k + ((vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1]) +
                 vel[3 * i + 2] * vel[3 * i + 2]);
        u = u + pe[i];
        if (flags[i] == 2) r = r - f[3 * i + axis];
    }
    out[0] = 0.5 * mass * k * or_mv2_to_ev();
    out[1] = u;
    out[2] = r / A0 * or_ev_per_a3_to_gpa();
}

typedef struct {
    int cap;
    int *counts;
    int *list;
    double *f, *pe, *rho;
} or_work;

static int or_forces(const double *pos, long n, const or_pot *p, or_work *w) {
    int maxc = or_pairs_cells(pos, n, p->rc, w->cap, w->counts, w->list);
    if (maxc > w->cap) return -1;
    or_eam(pos, n, p, w->cap, w->counts, w->list, w->f, w->pe, w->rho);
    return 0;
}

/* Grip displacement (loading protocol): every right-grip atom moves by du
 * along the load axis. */
OR_API void or_apply_strain(double *pos, long n, const uint8_t *flags, int axis, double du) {
    for (long i = 0; i < n; i++)
        if (flags[i] == 2) pos[3 * i + axis] = pos[3 * i + axis] + du;
}

/* ---------------------------------------------------------------------
 * One fine burst of NVE velocity-Verlet, Eqs. (vv_algo_pos_pred_half),
 * (vv_algo_pos_pred), (vv_algo_vel_pred), with the load held fixed: grip
 * atoms get v = 0 and F = 0 in the update, so they do not move.  Forces are
 * first evaluated at the initial positions; after each full step the state
 * functions are sampled into series[3*s + {0,1,2}] (s = 0..nsteps-1), so the
 * running time average of Eq. (R_m_t) is the mean of the series.
 * Pairs are found again from scratch at every step.  Returns 0, or -1 when
 * an atom has more than `cap` neighbours.
 *
 * With right_free (thermal relaxation, Sec. Boundary conditions) the
 * right-grip atoms move freely along the load axis: that component of their
 * velocity and force enters the update like a mobile atom's, the other two
 * stay v = 0, F = 0.  The left grip stays fixed.
 * ------------------------------------------------------------------- */
static int burst_impl(double *pos, double *vel, long n, const uint8_t *flags, const or_pot *p,
                      double mass, double dt, int axis, double A0, long nsteps, int cap,
                      double *series, double *f_out, int right_free, double grip_du) {
    or_work w;
    w.cap = cap;
    w.counts = (int *)malloc(sizeof(int) * n);
    w.list = (int *)malloc(sizeof(int) * (size_t)n * cap);
    w.f = (double *)malloc(sizeof(double) * 3 * n);
    w.pe = (double *)malloc(sizeof(double) * n);
    w.rho = (double *)malloc(sizeof(double) * n);
    int rc = or_forces(pos, n, p, &w);
    const double acc = or_force_to_acc() / mass;
    for (long s = 0; s < nsteps && rc == 0; s++) {
        for (long i = 0; i < n; i++) {
            for (int d = 0; d < 3; d++) {
                const int moves = flags[i] == 0 || (right_free && flags[i] == 2 && d == axis);
                if (!moves) continue;
                vel[3 * i + d] = vel[3 * i + d] + w.f[3 * i + d] * acc * (0.5 * dt);
                pos[3 * i + d] = pos[3 * i + d] + vel[3 * i + d] * dt;
            }
        }
        /* continuous loading: the right grip advances by grip_du with the drift */
        if (grip_du != 0.0)
            for (long i = 0; i < n; i++)
                if (flags[i] == 2 && !right_free) pos[3 * i + axis] = pos[3 * i + axis] + grip_du;
        rc = or_forces(pos, n, p, &w);
        if (rc != 0) break;
        for (long i = 0; i < n; i++) {
            for (int d = 0; d < 3; d++) {
                const int moves = flags[i] == 0 || (right_free && flags[i] == 2 && d == axis);
                if (moves) vel[3 * i + d] = vel[3 * i + d] + w.f[3 * i + d] * acc * (0.5 * dt);
            }
        }
        if (series) or_observe(n, vel, w.f, w.pe, flags, mass, axis, A0, series + 3 * s);
    }
    if (f_out && rc == 0) memcpy(f_out, w.f, sizeof(double) * 3 * n);
    free(w.counts);
    free(w.list);
    free(w.f);
    free(w.pe);
    free(w.rho);
    return rc;
}

OR_API int or_burst(double *pos, double *vel, long n, const uint8_t *flags, const or_pot *p,
                    double mass, double dt, int axis, double A0, long nsteps, int cap,
                    double *series, double *f_out) {
    return burst_impl(pos, vel, n, flags, p, mass, dt, axis, A0, nsteps, cap, series, f_out, 0,
                      0.0);
}

/* the same burst with the right grip moving by grip_du along the load axis
 * at every step (the continuous loading of the fine dynamics against which
 * PTA is verified, Sec. Verification with fine dynamics) */
OR_API int or_burst_ramp(double *pos, double *vel, long n, const uint8_t *flags, const or_pot *p,
                         double mass, double dt, int axis, double A0, long nsteps, int cap,
                         double grip_du, double *series, double *f_out) {
    return burst_impl(pos, vel, n, flags, p, mass, dt, axis, A0, nsteps, cap, series, f_out, 0,
                      grip_du);
}

/* the same burst with the right grip free along the load axis (relaxation) */
OR_API int or_burst_relax(double *pos, double *vel, long n, const uint8_t *flags,
                          const or_pot *p, double mass, double dt, int axis, double A0,
                          long nsteps, int cap, double *series, double *f_out) {
    return burst_impl(pos, vel, n, flags, p, mass, dt, axis, A0, nsteps, cap, series, f_out, 1,
                      0.0);
}

/* state functions of a given state (no time step) */
OR_API int or_observables(const double *pos, const double *vel, long n, const uint8_t *flags,
                          const or_pot *p, double mass, int axis, double A0, int cap,
                          double out[3]) {
    or_work w;
    w.cap = cap;
    w.counts = (int *)malloc(sizeof(int) * n);
    w.list = (int *)malloc(sizeof(int) * (size_t)n * cap);
    w.f = (double *)malloc(sizeof(double) * 3 * n);
    w.pe = (double *)malloc(sizeof(double) * n);
    w.rho = (double *)malloc(sizeof(double) * n);
    int rc = or_forces(pos, n, p, &w);
    if (rc == 0) or_observe(n, vel, w.f, w.pe, flags, mass, axis, A0, out);
    free(w.counts);
    free(w.list);
    free(w.f);
    free(w.pe);
    free(w.rho);
    return rc;
}
