"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the PTA method (no potential, no
integrator, no averaging): it only draws reproducible test geometries,
velocity fields and workload descriptions from numpy's seeded generator.
Both the CUDA path and the oracle are fed from here, so that neither ever
takes an input from the other.

The paper's runs (LAMMPS, Mishin Al potential, 4-30 nm FCC cubes at 1e-4 to
1e-3 1/s) are stood in for by the synthetic workloads below, with the same
shapes: FCC cubes of 10-49 cells per side, 4,000-470,596 atoms, T0 in
{10, 100, 300} K, tension and compression.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

A0_AL = 4.05  # Angstrom, lattice parameter of Table 1


def fcc_sites(n_cells, a0: float = A0_AL) -> np.ndarray:
    """Perfect FCC sites of an n_cells block, for use as test geometry
    (cube axes along x, y, z; site order x fastest, then y, then z, four
    basis sites per cell)."""
    nx, ny, nz = (n_cells,) * 3 if np.isscalar(n_cells) else tuple(n_cells)
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                      kk.transpose(2, 1, 0).ravel()], axis=1).astype(np.float64)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    return (a0 * (cells[:, None, :] + basis[None, :, :])).reshape(-1, 3)


def jittered_fcc(n_cells, amp: float, seed: int, a0: float = A0_AL) -> np.ndarray:
    """FCC sites displaced by independent uniform noise in [-amp, amp] per
    component (a stand-in for a thermal snapshot)."""
    rng = np.random.default_rng(seed)
    p = fcc_sites(n_cells, a0)
    return p + rng.uniform(-amp, amp, size=p.shape)


def gaussian_jitter_fcc(n_cells, sigma: float, seed: int, a0: float = A0_AL) -> np.ndarray:
    """FCC sites displaced by Gaussian noise of standard deviation sigma (A)."""
    rng = np.random.default_rng(seed)
    p = fcc_sites(n_cells, a0)
    return p + rng.normal(0.0, sigma, size=p.shape)


def random_velocities(n: int, sigma: float, seed: int) -> np.ndarray:
    """Independent Gaussian velocity components (A/fs)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=(n, 3))


def random_cluster(n: int, box: float, min_sep: float, seed: int) -> np.ndarray:
    """n points in a cube of edge box with pairwise separation >= min_sep,
    by rejection (small n only)."""
    rng = np.random.default_rng(seed)
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place points")
        q = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(q - p) >= min_sep for p in pts):
            pts.append(q)
    return np.array(pts)


# ---------------------------------------------------------------------------
# workloads (the five benchmark configurations)
# ---------------------------------------------------------------------------
@dataclass
class SpecimenRequest:
    n_cells: int
    T0: float
    seed: int
    strain_rate: float          # 1/s, negative = compression
    target_strain: float = 0.0
    arrival_s: float = 0.0
    burst_steps: int = 2000

    @property
    def natoms(self) -> int:
        return 4 * self.n_cells ** 3


def config_plain():
    """Plain FP64 run: 10^3 cells (4,000 atoms), 300 K, seed 1, one tension
    step of 1e-3, then one 2,000-step burst."""
    return dict(name="plain_fp64_n10", n_cells=10, T0=300.0, seed=1, d_eps=1e-3,
                burst_steps=2000, precision="fp64")


def config_large():
    """Single large specimen: 49^3 cells (470,596 atoms), 300 K, tension at
    1e-3 1/s with h = 1 s, bursts of 5,000 steps, FP32 forces."""
    return dict(name="large_fp32_n49", n_cells=49, T0=300.0, seed=1, strain_rate=1e-3,
                burst_steps=5000, n_coarse=100, precision="fp32")


def config_batched(count: int = 64, n_cells: int = 20):
    """Replica ensemble: 64 cubes of 20^3 cells, seeds 1..64, T0 cycling
    {10, 100, 300} K, first half tension, second half compression, rates
    log-uniform in [1e-4, 1e-3] 1/s drawn from seed 0."""
    rng = np.random.default_rng(0)
    reqs = []
    for r in range(count):
        rate = 10.0 ** rng.uniform(-4.0, -3.0)
        sign = 1.0 if r < count // 2 else -1.0
        reqs.append(SpecimenRequest(n_cells=n_cells, T0=(10.0, 100.0, 300.0)[r % 3],
                                    seed=r + 1, strain_rate=sign * rate, burst_steps=2000))
    return reqs


def config_uneven(per_size: int = 4, sizes=(10, 15, 20, 25, 30, 40, 49)):
    """Uneven batch: 4 specimens of each of 10, 15, 20, 25, 30, 40, 49 cells
    per side (28 specimens, 3,786,384 atoms), alternating tension and
    compression, 300 K."""
    reqs = []
    k = 0
    for n in sizes:
        for r in range(per_size):
            sign = 1.0 if k % 2 == 0 else -1.0
            reqs.append(SpecimenRequest(n_cells=n, T0=300.0, seed=100 + k,
                                        strain_rate=sign * 1e-3, burst_steps=2000))
            k += 1
    return reqs


def served_trace(n_requests: int, seed: int = 7, rate_per_s: float = 2.0,
                 sizes=(10, 49), time_scale: float = 1.0):
    """Poisson arrivals (mean rate_per_s per second, inter-arrival times
    scaled by time_scale) of PTA requests: cube side uniform in
    sizes[0]..sizes[1] cells, T0 in {10, 100, 300} K, rate log-uniform in
    [1e-4, 1e-3] 1/s, tension or compression with p = 0.5, target strain
    uniform in [0.05, 0.15]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s) * time_scale
        n = int(rng.integers(sizes[0], sizes[1] + 1))
        T0 = float(rng.choice([10.0, 100.0, 300.0]))
        rate = 10.0 ** rng.uniform(-4.0, -3.0)
        sign = 1.0 if rng.random() < 0.5 else -1.0
        target = float(rng.uniform(0.05, 0.15))
        out.append(SpecimenRequest(n_cells=n, T0=T0, seed=1000 + k, strain_rate=sign * rate,
                                   target_strain=target, arrival_s=t, burst_steps=2000))
    return out
