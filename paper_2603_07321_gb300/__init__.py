"""Python binding of the GB300 fine-burst engine for Practical Time Averaging
molecular dynamics (arXiv 2603.07321).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``_lib/libpta.so`` behind the C ABI of ``include/pta.h``.  The functions
below carry the C names (``pta_create``, ``pta_apply_strain``,
``pta_fine_burst``, ``pta_coarse_step`` ...) and raise ``PTAError`` on a
non-zero status; ``Ctx`` and ``Batch`` wrap the handles.  PyTorch supplies
device memory (through the allocator hook) and the CUDA stream.

There is no CPU fallback: importing works without a GPU (so that the build
can be checked), but every call that reaches the device fails loudly when
the library or the GPU is missing.
"""
from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

__all__ = [
    "PTAError", "Specimen", "Potential", "Params", "Averages", "CoarseResult", "Ctx", "Batch",
    "load", "build", "default_params", "default_potential", "pta_create", "pta_destroy",
    "pta_apply_strain", "pta_fine_burst", "pta_coarse_step", "pta_get_state", "pta_set_state",
    "pta_forces", "pta_get_neighbours", "pta_get_series", "pta_save_state", "pta_load_state",
    "pta_batch_create", "pta_batch_destroy", "pta_batch_fine_burst", "pta_batch_apply_strain",
    "pta_batch_coarse_step", "pta_batch_tick", "pta_coarse_update", "pta_ramp_burst", "pta_footprint_bytes", "PREC_FP64",
    "PREC_MIXED",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpta.so")
LIB_CHECK_PATH = os.path.join(_PKG, "_lib", "libpta_check.so")

PREC_FP64 = 0
PREC_MIXED = 1
SRC_PREDICTED, SRC_MEASURE_JUMP, SRC_MEASURE_MISMATCH = 0, 1, 2

_STATUS = {0: "PTA_OK", -1: "PTA_EINVAL", -2: "PTA_ENOMEM", -3: "PTA_ECUDA",
           -4: "PTA_ENEIGH_OVERFLOW", -5: "PTA_ENAN", -6: "PTA_ESTATE", -7: "PTA_ERANGE",
           -8: "PTA_EUNSUPPORTED", -9: "PTA_ECAPACITY", -10: "PTA_ECHECK"}


class PTAError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, _STATUS.get(status, "?"), status))


# ---------------------------------------------------------------------------
# C structures (mirror include/pta.h)
# ---------------------------------------------------------------------------
class Specimen(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int * 3), ("a0", ctypes.c_double),
                ("load_axis", ctypes.c_int), ("grip_width", ctypes.c_double)]


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("eps", ctypes.c_double), ("c", ctypes.c_double),
                ("a", ctypes.c_double), ("rc", ctypes.c_double), ("n", ctypes.c_int),
                ("m", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("mass_amu", ctypes.c_double),
                ("skin", ctypes.c_double), ("h", ctypes.c_double), ("Delta", ctypes.c_double),
                ("strain_rate", ctypes.c_double), ("tol_v", ctypes.c_double * 3),
                ("tol_j", ctypes.c_double * 3), ("floor", ctypes.c_double * 3),
                ("burst_steps", ctypes.c_int64), ("block_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("neigh_cap", ctypes.c_int),
                ("lanes", ctypes.c_int), ("atoms_per_thread", ctypes.c_int),
                ("prune_margin", ctypes.c_double), ("cell_tiles", ctypes.c_int),
                ("conv_lag", ctypes.c_int), ("conv_tol", ctypes.c_double * 3),
                ("mean_positions", ctypes.c_int)]


class Averages(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double * 3), ("se", ctypes.c_double * 3),
                ("nsteps", ctypes.c_int64), ("rebuilds", ctypes.c_int32),
                ("status", ctypes.c_int32), ("prunes", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("nsamples", ctypes.c_int64 * 3)]

    def as_dict(self):
        return {"mean": list(self.mean), "se": list(self.se), "nsteps": self.nsteps,
                "rebuilds": self.rebuilds, "prunes": self.prunes, "status": self.status,
                "converged": self.converged, "nsamples": list(self.nsamples)}


class CoarseResult(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("strain", ctypes.c_double),
                ("v", ctypes.c_double * 3), ("v_pred", ctypes.c_double * 3),
                ("v_d", ctypes.c_double * 3), ("e_v", ctypes.c_double * 3),
                ("e1", ctypes.c_double * 3), ("e2", ctypes.c_double * 3),
                ("jump", ctypes.c_int32 * 3), ("source", ctypes.c_int32 * 3),
                ("burst", Averages * 3), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {"t": self.t, "strain": self.strain, "v": list(self.v), "v_pred": list(self.v_pred),
                "v_d": list(self.v_d), "e_v": list(self.e_v), "e1": list(self.e1),
                "e2": list(self.e2), "jump": list(self.jump), "source": list(self.source),
                "burst": [b.as_dict() for b in self.burst], "status": self.status}


class KernelTimes(ctypes.Structure):
    _fields_ = [("rebuild_ms", ctypes.c_double), ("density_ms", ctypes.c_double),
                ("force_ms", ctypes.c_double), ("iterations", ctypes.c_int64)]


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

# every symbol the header declares, with (restype, argtypes)
_P = ctypes.POINTER
_VP = ctypes.c_void_p
_SIGS = {
    "pta_abi_version": (ctypes.c_int, []),
    "pta_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pta_set_allocator": (ctypes.c_int, [_ALLOC_T, _FREE_T, _VP]),
    "pta_default_params": (ctypes.c_int, [_P(Params)]),
    "pta_default_potential": (ctypes.c_int, [_P(Potential)]),
    "pta_footprint_bytes": (ctypes.c_size_t, [_P(Specimen), _P(Params)]),
    "pta_create": (ctypes.c_int, [_P(Specimen), _P(Potential), ctypes.c_double, ctypes.c_uint64,
                                  _P(Params), _VP, _P(_VP)]),
    "pta_destroy": (None, [_VP]),
    "pta_natoms": (ctypes.c_int, [_VP, _P(ctypes.c_int64)]),
    "pta_get_layout": (ctypes.c_int, [_VP, _P(ctypes.c_int32)]),
    "pta_get_mean_positions": (ctypes.c_int, [_VP, _P(ctypes.c_double), ctypes.c_int64]),
    "pta_relax": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                 _P(Averages), _P(ctypes.c_int64)]),
    "pta_get_flags": (ctypes.c_int, [_VP, _P(ctypes.c_uint8), ctypes.c_int64]),
    "pta_apply_strain": (ctypes.c_int, [_VP, ctypes.c_double]),
    "pta_get_strain": (ctypes.c_int, [_VP, _P(ctypes.c_double)]),
    "pta_fine_burst": (ctypes.c_int, [_VP, ctypes.c_int64, _P(Averages)]),
    "pta_ramp_burst": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_double, _P(Averages)]),
    "pta_get_series": (ctypes.c_int, [_VP, _P(ctypes.c_double), ctypes.c_int64,
                                      _P(ctypes.c_int64)]),
    "pta_coarse_step": (ctypes.c_int, [_VP, _P(CoarseResult)]),
    "pta_coarse_update": (ctypes.c_int, [_VP, _P(ctypes.c_double), _P(CoarseResult)]),
    "pta_get_state": (ctypes.c_int, [_VP, _P(ctypes.c_double), _P(ctypes.c_double),
                                     ctypes.c_int64]),
    "pta_set_state": (ctypes.c_int, [_VP, _P(ctypes.c_double), _P(ctypes.c_double),
                                     ctypes.c_int64]),
    "pta_forces": (ctypes.c_int, [_VP, _P(ctypes.c_double), _P(ctypes.c_double), ctypes.c_int64,
                                  _P(ctypes.c_double)]),
    "pta_get_neighbours": (ctypes.c_int, [_VP, _P(ctypes.c_int32), _P(ctypes.c_int32),
                                          ctypes.c_int64, ctypes.c_int32, _P(ctypes.c_int32)]),
    "pta_save_state": (ctypes.c_int, [_VP, _VP, _P(ctypes.c_size_t)]),
    "pta_load_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "pta_batch_create": (ctypes.c_int, [_P(_VP), ctypes.c_int, _P(_VP)]),
    "pta_batch_destroy": (None, [_VP]),
    "pta_batch_apply_strain": (ctypes.c_int, [_VP, _P(ctypes.c_double)]),
    "pta_batch_fine_burst": (ctypes.c_int, [_VP, _P(ctypes.c_int64), _P(Averages)]),
    "pta_batch_coarse_step": (ctypes.c_int, [_VP, _P(CoarseResult)]),
    "pta_batch_tick": (ctypes.c_int, [_VP, _P(CoarseResult)]),
    "pta_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pta_get_timing": (ctypes.c_int, [_VP, _P(KernelTimes)]),
    "pta_batch_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pta_batch_get_timing": (ctypes.c_int, [_VP, _P(KernelTimes)]),
    "pta_measure_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _VP,
                                            _P(ctypes.c_double), _P(ctypes.c_double)]),
    "pta_neighbours_noalloc": (ctypes.c_int, [_VP, ctypes.c_int32, _P(ctypes.c_double),
                                              _P(ctypes.c_double), ctypes.c_double,
                                              ctypes.c_int32, _VP, _VP, _P(ctypes.c_int32),
                                              _VP]),
}

_lib = None
_live = {}            # data_ptr -> torch tensor backing device memory handed to the library
_callbacks = None


def check_build() -> bool:
    """True when this process uses the debug library (environment PTA_CHECK=1
    when the library is first loaded): every index and count is tested on the
    device, and a failed test gives PTA_ECHECK."""
    return os.environ.get("PTA_CHECK", "0") == "1"


def build(force: bool = False, check=None) -> str:
    """Compile the library (the debug variant when check, by default when
    check_build())."""
    from . import buildlib
    return buildlib.build(force=force, check=check_build() if check is None else bool(check))


def library_path() -> str:
    return LIB_CHECK_PATH if check_build() else LIB_PATH


def load(path: str = None):
    """Load libpta.so (built by build()), or libpta_check.so when
    check_build(); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise ImportError("%s not found: run paper_2603_07321_gb300.build() "
                          "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _install_torch_allocator():
    """Route the library's device allocations through PyTorch's allocator."""
    global _callbacks
    if _callbacks is not None:
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        except Exception:  # out of memory: the library reports PTA_ENOMEM
            return None
        p = t.data_ptr()
        _live[p] = t
        return p

    def _free(ptr, stream, user):
        _live.pop(ptr, None)

    _callbacks = (_ALLOC_T(_alloc), _FREE_T(_free))
    _check(load().pta_set_allocator(_callbacks[0], _callbacks[1], None), "pta_set_allocator")


def _check(rc, what):
    if rc != 0:
        raise PTAError(rc, what)


def _dptr(a):
    return a.ctypes.data_as(_P(ctypes.c_double))


def default_params(**kw) -> Params:
    p = Params()
    _check(load().pta_default_params(ctypes.byref(p)), "pta_default_params")
    for k, v in kw.items():
        if k in ("tol_v", "tol_j", "floor", "conv_tol"):
            for i in range(3):
                getattr(p, k)[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def default_potential(**kw) -> Potential:
    p = Potential()
    _check(load().pta_default_potential(ctypes.byref(p)), "pta_default_potential")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_specimen(n_cells, a0=4.05, load_axis=2, grip_width=0.0) -> Specimen:
    s = Specimen()
    nc = (n_cells,) * 3 if np.isscalar(n_cells) else tuple(n_cells)
    for i in range(3):
        s.n_cells[i] = int(nc[i])
    s.a0 = a0
    s.load_axis = load_axis
    s.grip_width = grip_width
    return s


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def pta_footprint_bytes(spec: Specimen, params: Params) -> int:
    return load().pta_footprint_bytes(ctypes.byref(spec), ctypes.byref(params))


def pta_create(spec: Specimen, pot: Potential, T0: float, seed: int, params: Params,
               stream=None):
    import torch
    _install_torch_allocator()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    h = _VP()
    _check(load().pta_create(ctypes.byref(spec), ctypes.byref(pot), float(T0), int(seed),
                             ctypes.byref(params), _VP(stream), ctypes.byref(h)), "pta_create")
    return h


def pta_destroy(h):
    load().pta_destroy(h)


def pta_natoms(h) -> int:
    n = ctypes.c_int64()
    _check(load().pta_natoms(h, ctypes.byref(n)), "pta_natoms")
    return n.value


def pta_get_layout(h) -> dict:
    out = (ctypes.c_int32 * 4)()
    _check(load().pta_get_layout(h, out), "pta_get_layout")
    return {"lanes": out[0], "atoms_per_thread": out[1], "neigh_cap": out[2],
            "pruned_list": bool(out[3])}


def pta_relax(h, window: int, max_steps: int, tol_gpa: float):
    a = Averages()
    steps = ctypes.c_int64()
    _check(load().pta_relax(h, int(window), int(max_steps), float(tol_gpa), ctypes.byref(a),
                            ctypes.byref(steps)), "pta_relax")
    return a, steps.value


def pta_get_mean_positions(h, n):
    out = np.zeros((n, 3))
    _check(load().pta_get_mean_positions(h, _dptr(out), n), "pta_get_mean_positions")
    return out


def pta_get_flags(h, n):
    out = np.zeros(n, dtype=np.uint8)
    _check(load().pta_get_flags(h, out.ctypes.data_as(_P(ctypes.c_uint8)), n), "pta_get_flags")
    return out


def pta_apply_strain(h, d_eps: float):
    _check(load().pta_apply_strain(h, float(d_eps)), "pta_apply_strain")


def pta_get_strain(h) -> float:
    s = ctypes.c_double()
    _check(load().pta_get_strain(h, ctypes.byref(s)), "pta_get_strain")
    return s.value


def pta_fine_burst(h, nsteps: int) -> Averages:
    a = Averages()
    _check(load().pta_fine_burst(h, int(nsteps), ctypes.byref(a)), "pta_fine_burst")
    return a


def pta_ramp_burst(h, nsteps: int, d_eps_per_step: float) -> Averages:
    a = Averages()
    _check(load().pta_ramp_burst(h, int(nsteps), float(d_eps_per_step), ctypes.byref(a)),
           "pta_ramp_burst")
    return a


def pta_get_series(h, max_steps: int):
    cnt = ctypes.c_int64()
    out = np.zeros((max_steps, 3))
    _check(load().pta_get_series(h, _dptr(out), max_steps, ctypes.byref(cnt)), "pta_get_series")
    return out[: min(cnt.value, max_steps)]


def pta_coarse_step(h) -> CoarseResult:
    r = CoarseResult()
    _check(load().pta_coarse_step(h, ctypes.byref(r)), "pta_coarse_step")
    return r


def pta_coarse_update(h, means) -> CoarseResult:
    """means: 3 x 3 (burst, variable) averages fed to the coarse-step update"""
    m = np.ascontiguousarray(np.asarray(means, dtype=np.float64).reshape(9))
    r = CoarseResult()
    _check(load().pta_coarse_update(h, _dptr(m), ctypes.byref(r)), "pta_coarse_update")
    return r


def pta_get_state(h, n):
    pos = np.zeros((n, 3))
    vel = np.zeros((n, 3))
    _check(load().pta_get_state(h, _dptr(pos), _dptr(vel), n), "pta_get_state")
    return pos, vel


def pta_set_state(h, pos, vel):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    _check(load().pta_set_state(h, _dptr(pos), _dptr(vel), len(pos)), "pta_set_state")


def pta_forces(h, n):
    f = np.zeros((n, 3))
    pe = np.zeros(n)
    obs = np.zeros(3)
    _check(load().pta_forces(h, _dptr(f), _dptr(pe), n, _dptr(obs)), "pta_forces")
    return f, pe, obs


def pta_get_neighbours(h, n, cap=512):
    counts = np.zeros(n, dtype=np.int32)
    lst = np.full((n, cap), -1, dtype=np.int32)
    mx = ctypes.c_int32()
    _check(load().pta_get_neighbours(h, counts.ctypes.data_as(_P(ctypes.c_int32)),
                                     lst.ctypes.data_as(_P(ctypes.c_int32)), n, cap,
                                     ctypes.byref(mx)), "pta_get_neighbours")
    return counts, lst


def pta_save_state(h) -> bytes:
    ln = ctypes.c_size_t()
    _check(load().pta_save_state(h, None, ctypes.byref(ln)), "pta_save_state")
    buf = ctypes.create_string_buffer(ln.value)
    _check(load().pta_save_state(h, buf, ctypes.byref(ln)), "pta_save_state")
    return buf.raw[: ln.value]


def pta_load_state(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().pta_load_state(h, buf, len(blob)), "pta_load_state")


def pta_batch_create(handles):
    arr = (_VP * len(handles))(*[hh.value if isinstance(hh, _VP) else hh for hh in handles])
    b = _VP()
    _check(load().pta_batch_create(arr, len(handles), ctypes.byref(b)), "pta_batch_create")
    return b


def pta_batch_destroy(b):
    load().pta_batch_destroy(b)


def pta_batch_apply_strain(b, d_eps):
    arr = np.ascontiguousarray(d_eps, dtype=np.float64)
    _check(load().pta_batch_apply_strain(b, _dptr(arr)), "pta_batch_apply_strain")


# statuses that concern single members of a batch call: the call has filled
# every member's result (its own status in it), the others' are valid
MEMBER_STATUSES = frozenset((-4, -5, -7, -10))


def pta_batch_fine_burst(b, nsteps):
    ns = np.ascontiguousarray(nsteps, dtype=np.int64)
    out = (Averages * len(ns))()
    rc = load().pta_batch_fine_burst(b, ns.ctypes.data_as(_P(ctypes.c_int64)), out)
    if rc not in MEMBER_STATUSES:
        _check(rc, "pta_batch_fine_burst")
    return list(out)


def pta_batch_coarse_step(b, count):
    out = (CoarseResult * count)()
    _check(load().pta_batch_coarse_step(b, out), "pta_batch_coarse_step")
    return list(out)


def pta_batch_tick(b, count):
    out = (CoarseResult * count)()
    rc = load().pta_batch_tick(b, out)
    if rc not in MEMBER_STATUSES:
        _check(rc, "pta_batch_tick")
    return list(out)


def pta_set_timing(h, enable: bool):
    _check(load().pta_set_timing(h, 1 if enable else 0), "pta_set_timing")


def pta_get_timing(h) -> KernelTimes:
    t = KernelTimes()
    _check(load().pta_get_timing(h, ctypes.byref(t)), "pta_get_timing")
    return t


def pta_batch_set_timing(b, enable: bool):
    _check(load().pta_batch_set_timing(b, 1 if enable else 0), "pta_batch_set_timing")


def pta_batch_get_timing(b) -> KernelTimes:
    t = KernelTimes()
    _check(load().pta_batch_get_timing(b, ctypes.byref(t)), "pta_batch_get_timing")
    return t


def pta_measure_fma_rate(kind: int, iters: int, stream=None):
    """(flops, ms) of one launch of FMA chains: kind 0 scalar FP32, 1 packed
    FP32, 2 FP64; or (operations, ms) of kind 3 (64-bit integer reductions to
    global memory), 4 (64-bit shared-memory atomic adds), 5 (FP32 -> int64
    conversions)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    fl = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load().pta_measure_fma_rate(int(kind), int(iters), _VP(stream), ctypes.byref(fl),
                                       ctypes.byref(ms)), "pta_measure_fma_rate")
    return fl.value, ms.value


NOALLOC_MAX_ATOMS = 131072
NOALLOC_MAX_CELLS = 65536


def pta_neighbours_noalloc(pos_dev_ptr: int, n: int, box_lo, box_hi, rlist: float, cap: int,
                           counts_dev_ptr: int, list_dev_ptr: int, stream=None) -> int:
    """Neighbour lists from device positions into caller-owned device
    arrays, for callers that cannot allocate device memory (the library
    uses a fixed scratch array instead).  Pointers are device addresses
    (e.g. tensor.data_ptr()); returns the largest neighbour count.  Calls
    share the scratch array and must not overlap on the GPU."""
    lo = (ctypes.c_double * 3)(*[float(x) for x in box_lo])
    hi = (ctypes.c_double * 3)(*[float(x) for x in box_hi])
    mx = ctypes.c_int32()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().pta_neighbours_noalloc(_VP(pos_dev_ptr), int(n), lo, hi, float(rlist), int(cap),
                                         _VP(counts_dev_ptr), _VP(list_dev_ptr),
                                         ctypes.byref(mx), _VP(stream)),
           "pta_neighbours_noalloc")
    return mx.value


# ---------------------------------------------------------------------------
# handle wrappers
# ---------------------------------------------------------------------------
_TAGS = itertools.count()


class Ctx:
    """One specimen on the device (owns a pta_ctx)."""

    def __init__(self, n_cells, T0=300.0, seed=1, params: Params | None = None,
                 potential: Potential | None = None, load_axis=2, a0=4.05, grip_width=0.0,
                 stream=None, tuned: bool = True, replicas: int = 1, log=None, tag=None,
                 **param_kw):
        """With the threads per atom left automatic (no params, lanes 0 or
        absent) and `tuned`, the layout the autotuner cached for this size,
        precision and number of replicas sharing the device (tune.py) is
        used; without a cache entry the library's own choice.  With `log` (a
        metrics.JsonlLog, a path or a text file) every burst, relaxation and
        coarse step appends a record named by `tag`."""
        from . import metrics as _metrics
        self.log = _metrics.as_log(log)
        self.tag = tag if tag is not None else "ctx%d" % next(_TAGS)
        self.spec = make_specimen(n_cells, a0, load_axis, grip_width)
        self.layout_source = "explicit" if (params is not None or param_kw.get("lanes")) \
            else "automatic"
        if params is None and not param_kw.get("lanes") and tuned:
            from . import tune as _tune
            nc = (n_cells,) * 3 if np.isscalar(n_cells) else tuple(n_cells)
            natoms = 4 * int(nc[0]) * int(nc[1]) * int(nc[2])
            hit = _tune.lookup(natoms, replicas, param_kw.get("precision", PREC_FP64))
            if hit:
                param_kw = {**param_kw, **hit}
                self.layout_source = "tuned"
        self.params = params if params is not None else default_params(**param_kw)
        self.potential = potential if potential is not None else default_potential()
        self.h = pta_create(self.spec, self.potential, T0, seed, self.params, stream)
        self.n = pta_natoms(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            pta_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def flags(self):
        return pta_get_flags(self.h, self.n)

    def layout(self):
        return pta_get_layout(self.h)

    def mean_positions(self):
        return pta_get_mean_positions(self.h, self.n)

    def _log(self, kind, **fields):
        if self.log is not None:
            self.log.write(kind, tag=self.tag, **fields)

    def relax(self, window=2000, max_steps=50000, tol_gpa=0.05):
        a, steps = pta_relax(self.h, window, max_steps, tol_gpa)
        self._log("relax", steps=steps, window=a.as_dict())
        return a, steps

    def apply_strain(self, d_eps):
        pta_apply_strain(self.h, d_eps)

    @property
    def strain(self):
        return pta_get_strain(self.h)

    def fine_burst(self, nsteps):
        a = pta_fine_burst(self.h, nsteps)
        self._log("burst", **a.as_dict())
        return a

    def ramp_burst(self, nsteps, d_eps_per_step):
        a = pta_ramp_burst(self.h, nsteps, d_eps_per_step)
        self._log("ramp_burst", d_eps_per_step=d_eps_per_step, **a.as_dict())
        return a

    def series(self, max_steps=1 << 20):
        return pta_get_series(self.h, max_steps)

    def coarse_step(self):
        r = pta_coarse_step(self.h)
        self._log("coarse", **r.as_dict())
        return r

    def coarse_update(self, means):
        return pta_coarse_update(self.h, means)

    def get_state(self):
        return pta_get_state(self.h, self.n)

    def set_state(self, pos, vel):
        pta_set_state(self.h, pos, vel)

    def forces(self):
        return pta_forces(self.h, self.n)

    def neighbours(self, cap=512):
        return pta_get_neighbours(self.h, self.n, cap)

    def set_timing(self, enable=True):
        pta_set_timing(self.h, enable)

    def timing(self):
        return pta_get_timing(self.h)

    def save(self):
        return pta_save_state(self.h)

    def restore(self, blob):
        pta_load_state(self.h, blob)


class Batch:
    """Several contexts advanced by shared launches (owns a pta_batch)."""

    def __init__(self, members):
        self.members = list(members)
        self.h = pta_batch_create([m.h for m in self.members])

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            pta_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_strain(self, d_eps):
        pta_batch_apply_strain(self.h, d_eps)

    def _log(self, kind, results):
        for m, r in zip(self.members, results):
            m._log(kind, **r.as_dict())
        return results

    def fine_burst(self, nsteps):
        if np.isscalar(nsteps):
            nsteps = [nsteps] * len(self.members)
        return self._log("burst", pta_batch_fine_burst(self.h, nsteps))

    def coarse_step(self):
        return self._log("coarse", pta_batch_coarse_step(self.h, len(self.members)))

    def tick(self):
        return self._log("coarse", pta_batch_tick(self.h, len(self.members)))

    def set_timing(self, enable=True):
        pta_batch_set_timing(self.h, enable)

    def timing(self):
        return pta_batch_get_timing(self.h)
