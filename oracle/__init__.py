"""FP64 CPU oracle for the PTA-MD fine-burst hot path (arXiv 2603.07321).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(the CUDA library and its Python binding) never imports it, and the two share
no code: this package holds a plain C file (``oracle.c``) compiled with gcc,
a ctypes wrapper (this file) and the coarse-step logic in plain Python
(``pta_logic.py``).

Parity status of each function (what pins it, see tests/test_oracle_*.py):

* lattice, grip flags ............ pinned (counts by hand, exact coordinates)
* Philox4x32-10 .................. pinned (published known-answer vectors)
* Maxwell-Boltzmann init ......... pinned (exact KE, zero momentum, grip v=0)
* pair finding ................... pinned (cell search == brute force)
* EAM energy / forces ............ pinned (closed-form shell sums, literature
                                   c of Sutton-Chen, equilibrium dE/da = 0,
                                   finite differences, Newton's third law,
                                   zero net force on a periodic lattice,
                                   dimer closed form)
* velocity Verlet burst .......... pinned (energy conservation, time
                                   reversibility, momentum, fixed grips)
* coarse-step logic .............. pinned (linear and step sequences, truth
                                   table of the acceptance rules)
* mean positions (Eq. mean_pos) .. pinned (free atoms in closed form, fixed
                                   grips, one-step burst)
* thermal relaxation burst ....... pinned (transverse grip coordinates and
                                   left grip unchanged, energy conservation,
                                   the unrelaxed reaction relaxes)
* adaptive burst length .......... pinned (closed-form crossing of a linear
                                   series, constant and alternating series,
                                   floors, N_max, brute-force recomputation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Pot(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("c", ctypes.c_double), ("a", ctypes.c_double),
                ("rc", ctypes.c_double), ("n", ctypes.c_int), ("m", ctypes.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lp = ctypes.POINTER(ctypes.c_long)
    potp = ctypes.POINTER(_Pot)
    sig = {
        "or_constants": (None, [dp]),
        "or_phi_value": (ctypes.c_double, [potp, ctypes.c_int, ctypes.c_double]),
        "or_dphi_value": (ctypes.c_double, [potp, ctypes.c_int, ctypes.c_double]),
        "or_sc_c_equilibrium": (ctypes.c_double, [potp, ctypes.c_double]),
        "or_sc_cohesive_energy": (ctypes.c_double, [potp, ctypes.c_double]),
        "or_fcc_lattice": (ctypes.c_long, [ctypes.c_int] * 3 + [ctypes.c_double, dp]),
        "or_grip_flags": (None, [dp, ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, u8p]),
        "or_philox4x32_10": (None, [u32p, u32p, u32p]),
        "or_atom_normals": (None, [ctypes.c_uint64, ctypes.c_uint64, dp]),
        "or_mb_velocities": (None, [ctypes.c_long, u8p, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, dp]),
        "or_pairs_brute": (ctypes.c_int, [dp, ctypes.c_long, ctypes.c_double, ctypes.c_int,
                                          ip, ip]),
        "or_pairs_cells": (ctypes.c_int, [dp, ctypes.c_long, ctypes.c_double, ctypes.c_int,
                                          ip, ip]),
        "or_eam": (None, [dp, ctypes.c_long, potp, ctypes.c_int, ip, ip, dp, dp, dp]),
        "or_eam_periodic": (None, [dp, ctypes.c_long, ctypes.c_double, potp, dp, dp, dp]),
        "or_eam_sampled": (ctypes.c_int, [dp, ctypes.c_long, potp, ctypes.c_long, lp, dp, dp]),
        "or_apply_strain": (None, [dp, ctypes.c_long, u8p, ctypes.c_int, ctypes.c_double]),
        "or_burst": (ctypes.c_int, [dp, dp, ctypes.c_long, u8p, potp, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_long, ctypes.c_int, dp, dp]),
        "or_burst_ramp": (ctypes.c_int, [dp, dp, ctypes.c_long, u8p, potp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_long, ctypes.c_int, ctypes.c_double, dp, dp]),
        "or_burst_relax": (ctypes.c_int, [dp, dp, ctypes.c_long, u8p, potp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_long, ctypes.c_int, dp, dp]),
        "or_observables": (ctypes.c_int, [dp, dp, ctypes.c_long, u8p, potp, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------------------
# potential
# ---------------------------------------------------------------------------
@dataclass
class Potential:
    """Sutton-Chen EAM with shifted-force cutoff (stand-in for Eq. (pe)).

    eps in eV, a and rc in Angstrom, c dimensionless; c=None means: fix c by
    the equilibrium of the perfect crystal at lattice constant ``a``."""
    eps: float = 3.3147e-2
    c: float | None = None
    a: float = 4.05
    rc: float = 8.1
    n: int = 7
    m: int = 6

    def __post_init__(self):
        if self.c is None:
            self.c = equilibrium_c(self, self.a)

    def _c(self):
        return _Pot(self.eps, float(self.c if self.c is not None else 0.0), self.a, self.rc,
                    self.n, self.m)


def equilibrium_c(pot: Potential, a0: float) -> float:
    """c that makes dE/da = 0 at a0 for the perfect FCC crystal."""
    lib = _load()
    p = _Pot(pot.eps, 1.0, pot.a, pot.rc, pot.n, pot.m)
    return lib.or_sc_c_equilibrium(ctypes.byref(p), a0)


def cohesive_energy(pot: Potential, a0: float) -> float:
    lib = _load()
    return lib.or_sc_cohesive_energy(ctypes.byref(pot._c()), a0)


def phi(pot: Potential, k: int, r: float) -> float:
    return _load().or_phi_value(ctypes.byref(pot._c()), k, r)


def dphi(pot: Potential, k: int, r: float) -> float:
    return _load().or_dphi_value(ctypes.byref(pot._c()), k, r)


def constants() -> dict:
    out = np.zeros(4)
    _load().or_constants(_ptr(out, ctypes.c_double))
    return {"mv2_to_ev": out[0], "force_to_acc": out[1], "kb_ev": out[2],
            "ev_per_a3_to_gpa": out[3]}


# ---------------------------------------------------------------------------
# specimen
# ---------------------------------------------------------------------------
def fcc_lattice(n_cells, a0: float) -> np.ndarray:
    nx, ny, nz = (n_cells, n_cells, n_cells) if np.isscalar(n_cells) else n_cells
    pos = np.zeros((4 * nx * ny * nz, 3))
    _load().or_fcc_lattice(nx, ny, nz, a0, _ptr(pos, ctypes.c_double))
    return pos


def grip_flags(pos: np.ndarray, axis: int, width: float, tol: float = 1e-6) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    flags = np.zeros(len(pos), dtype=np.uint8)
    _load().or_grip_flags(_ptr(pos, ctypes.c_double), len(pos), axis, width, tol,
                          _ptr(flags, ctypes.c_uint8))
    return flags


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                             _ptr(out, ctypes.c_uint32))
    return out


def atom_normals(seed: int, idx: int) -> np.ndarray:
    z = np.zeros(3)
    _load().or_atom_normals(seed, idx, _ptr(z, ctypes.c_double))
    return z


def mb_velocities(flags: np.ndarray, T0: float, mass: float, seed: int) -> np.ndarray:
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    vel = np.zeros((len(flags), 3))
    _load().or_mb_velocities(len(flags), _ptr(flags, ctypes.c_uint8), T0, mass, seed,
                             _ptr(vel, ctypes.c_double))
    return vel


# ---------------------------------------------------------------------------
# pairs, forces
# ---------------------------------------------------------------------------
def pairs(pos: np.ndarray, rcut: float, cap: int = 512, method: str = "cells"):
    """Full neighbour lists (ascending j) as (counts, list[n, cap])."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    counts = np.zeros(n, dtype=np.int32)
    lst = np.full((n, cap), -1, dtype=np.int32)
    fn = _load().or_pairs_cells if method == "cells" else _load().or_pairs_brute
    maxc = fn(_ptr(pos, ctypes.c_double), n, rcut, cap, _ptr(counts, ctypes.c_int),
              _ptr(lst, ctypes.c_int))
    if maxc > cap:
        raise ValueError("neighbour capacity %d exceeded (%d)" % (cap, maxc))
    return counts, lst


def eam(pos: np.ndarray, pot: Potential, cap: int = 512):
    """(forces[n,3], pe[n], rho[n]) on the exact pair set within rc."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    counts, lst = pairs(pos, pot.rc, cap)
    n = len(pos)
    f = np.zeros((n, 3))
    pe = np.zeros(n)
    rho = np.zeros(n)
    _load().or_eam(_ptr(pos, ctypes.c_double), n, ctypes.byref(pot._c()), cap,
                   _ptr(counts, ctypes.c_int), _ptr(lst, ctypes.c_int),
                   _ptr(f, ctypes.c_double), _ptr(pe, ctypes.c_double),
                   _ptr(rho, ctypes.c_double))
    return f, pe, rho


def eam_periodic(pos: np.ndarray, L: float, pot: Potential):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    f = np.zeros((n, 3))
    pe = np.zeros(n)
    rho = np.zeros(n)
    _load().or_eam_periodic(_ptr(pos, ctypes.c_double), n, L, ctypes.byref(pot._c()),
                            _ptr(f, ctypes.c_double), _ptr(pe, ctypes.c_double),
                            _ptr(rho, ctypes.c_double))
    return f, pe, rho


def eam_sampled(pos: np.ndarray, pot: Potential, idx):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = np.zeros((len(idx), 3))
    pe = np.zeros(len(idx))
    rc = _load().or_eam_sampled(_ptr(pos, ctypes.c_double), len(pos), ctypes.byref(pot._c()),
                                len(idx), _ptr(idx, ctypes.c_long), _ptr(f, ctypes.c_double),
                                _ptr(pe, ctypes.c_double))
    if rc != 0:
        raise ValueError("neighbour capacity exceeded")
    return f, pe


# ---------------------------------------------------------------------------
# dynamics
# ---------------------------------------------------------------------------
@dataclass
class Specimen:
    """Oracle copy of one specimen: FCC cube, grips, state, load."""
    n_cells: tuple
    a0: float = 4.05
    axis: int = 2
    grip_width: float | None = None
    mass: float = 26.9815385
    dt: float = 1.0
    pot: Potential | None = None

    def __post_init__(self):
        if np.isscalar(self.n_cells):
            self.n_cells = (int(self.n_cells),) * 3
        if self.pot is None:
            self.pot = Potential(a=self.a0)
        if self.grip_width is None:
            self.grip_width = self.a0
        self.pos = fcc_lattice(self.n_cells, self.a0)
        self.flags = grip_flags(self.pos, self.axis, self.grip_width)
        self.vel = np.zeros_like(self.pos)
        self.L_s = self.n_cells[self.axis] * self.a0
        others = [self.n_cells[d] * self.a0 for d in range(3) if d != self.axis]
        self.A0 = others[0] * others[1]
        self.u = 0.0

    @property
    def n(self):
        return len(self.pos)

    def thermalise(self, T0: float, seed: int):
        self.vel = mb_velocities(self.flags, T0, self.mass, seed)

    def apply_strain(self, d_eps: float):
        du = d_eps * self.L_s
        _load().or_apply_strain(_ptr(self.pos, ctypes.c_double), self.n,
                                _ptr(self.flags, ctypes.c_uint8), self.axis, du)
        self.u += du

    def burst(self, nsteps: int, cap: int = 512, relax: bool = False, ramp: float = 0.0):
        """Run nsteps of velocity Verlet; returns the series [nsteps, 3] of
        (K eV, U eV, T GPa) sampled after every full step.  relax: the right
        grip moves freely along the load axis (thermal relaxation).  ramp:
        continuous loading, the right grip advances by ramp * L_s (strain
        units) along the load axis with every step's drift."""
        series = np.zeros((nsteps, 3))
        f = np.zeros((self.n, 3))
        args = (_ptr(self.pos, ctypes.c_double), _ptr(self.vel, ctypes.c_double),
                self.n, _ptr(self.flags, ctypes.c_uint8), ctypes.byref(self.pot._c()),
                self.mass, self.dt, self.axis, self.A0, nsteps, cap)
        outs = (_ptr(series, ctypes.c_double), _ptr(f, ctypes.c_double))
        if ramp != 0.0:
            if relax:
                raise ValueError("a relaxation burst holds no grip to move")
            du = ramp * self.L_s
            rc = _load().or_burst_ramp(*args, du, *outs)
            self.u += nsteps * du
        else:
            fn = _load().or_burst_relax if relax else _load().or_burst
            rc = fn(*args, *outs)
        if rc != 0:
            raise ValueError("neighbour capacity exceeded")
        self.last_forces = f
        return series

    def relax(self, window: int, max_steps: int, tol_gpa: float, cap: int = 512):
        """Thermal relaxation (Sec. Boundary conditions): relaxation bursts of
        `window` steps until the window mean of T is within tol_gpa of 0 or
        another window would exceed max_steps; then the right grip is fixed
        where it is (v = 0).  Returns (last window's series, steps run)."""
        total = 0
        while True:
            s = self.burst(window, cap, relax=True)
            total += window
            if abs(s[:, 2].mean()) < tol_gpa or total + window > max_steps:
                break
        self.vel[self.flags == 2] = 0.0
        return s, total

    def burst_mean_positions(self, nsteps: int, cap: int = 512):
        """Eq. (mean_pos): run nsteps of velocity Verlet and return the series
        and the mean position of every atom over the states sampled after each
        full step, (1/N) sum_i r(sigma_i), summed in FP64 in step order.  The
        steps run one at a time (each call starts from the forces of its
        starting positions, exactly those the previous step ended with)."""
        series = np.zeros((nsteps, 3))
        acc = np.zeros((self.n, 3))
        for s in range(nsteps):
            series[s] = self.burst(1, cap)[0]
            acc = acc + self.pos
        return series, acc / nsteps

    def observables(self, cap: int = 512):
        out = np.zeros(3)
        rc = _load().or_observables(_ptr(self.pos, ctypes.c_double),
                                    _ptr(self.vel, ctypes.c_double), self.n,
                                    _ptr(self.flags, ctypes.c_uint8),
                                    ctypes.byref(self.pot._c()), self.mass, self.axis, self.A0,
                                    cap, _ptr(out, ctypes.c_double))
        if rc != 0:
            raise ValueError("neighbour capacity exceeded")
        return out


def burst_averages(series: np.ndarray, block: int = 100):
    """Means of a burst series (Eq. (R_m_t)) and their standard errors from
    non-overlapping block means (block length in steps)."""
    series = np.asarray(series, dtype=np.float64)
    mean = series.mean(axis=0)
    nb = len(series) // block
    if nb >= 2:
        bm = series[: nb * block].reshape(nb, block, -1).mean(axis=1)
        se = bm.std(axis=0, ddof=1) / np.sqrt(nb)
    else:
        se = np.full(series.shape[1], np.nan)
    return mean, se
