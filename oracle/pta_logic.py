"""Coarse-step (slow-time) logic of Practical Time Averaging, plain FP64 Python.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the algorithm of the PTA framework section step by step, for each
slow variable m in (K, U, T) independently:

* Step 1, Eq. (dvdt_algo):  dv/dt(t) = (R_t - R_{t-Delta}) / Delta
* Step 2, Eq. (pta_pred):   v(t+h)   = v(t) + h dv/dt(t)
* Step 3, Eq. (simp):       v_d(t+h) = (R_{t+h-Delta} + 4 R_{t+h-Delta/2} + R_{t+h}) / 6
          Eq. (rel_err):    e_v = |v(t+h) - v_d(t+h)| / |v_d(t+h)|
          match if e_v < tol_v: keep the extrapolated v(t+h);
          else jump test, Eq. (jump_err): e1 = |R_{t+h}-R_t|/|R_t|,
          e2 = |R_t - R_{t-h}|/|R_{t-h}|; jump if |e1/e2 - 1| >= tol_j, or,
          when a jump was already flagged at t, if e1 >= tol_j.  On a jump
          v_d is accepted.
* Step 4, Eqs. (x_guess_step1), (x_guess_step3): each burst starts from the
  final state of the burst before it (the caller keeps the state chained).

Readings where the paper is silent (the same readings the CUDA path takes):

* no match and no jump: v_d is accepted and the step is flagged MISMATCH;
* the relative tests divide by max(|x|, floor_m) so that a stress near zero
  does not divide by zero;
* at the first coarse step R_{t-h} does not exist: the jump test then
  reports no jump unless a jump was flagged (it never is at t = 0);
* if e2 == 0 the ratio e1/e2 is +inf when e1 > 0 (jump) and undefined when
  e1 == 0 (no jump);
* the initial bursts run at grip displacement 0, +rate*Delta/2*L, +rate*Delta*L
  and are labelled -Delta, -Delta/2, 0; v(0) is their Simpson value.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# acceptance sources per variable
SRC_PREDICTED = 0      # e_v < tol_v: extrapolated value kept
SRC_MEASURE_JUMP = 1   # jump detected: Simpson value accepted
SRC_MEASURE_MISMATCH = 2  # neither: Simpson value accepted, flagged


@dataclass
class PTAParams:
    """Table 1 of the paper; variables ordered (K, U, T)."""
    h: float = 1.0                 # slow-time step, s
    Delta: float | None = None     # averaging interval, default h/5
    strain_rate: float = 1e-3      # 1/s; negative for compression
    tol_v: tuple = (0.01, 0.05, 0.01)
    tol_j: tuple = (0.08, 0.01, 0.05)
    floor: tuple = (1e-12, 1e-12, 0.05)

    def __post_init__(self):
        if self.Delta is None:
            self.Delta = self.h / 5.0

    # grip increments (in strain) of the loading protocol
    def init_increments(self):
        return (0.0, self.strain_rate * self.Delta / 2.0, self.strain_rate * self.Delta / 2.0)

    def step_increments(self):
        return (self.strain_rate * (self.h - self.Delta), self.strain_rate * self.Delta / 2.0,
                self.strain_rate * self.Delta / 2.0)


@dataclass
class PTAState:
    t: float
    v: np.ndarray            # accepted slow variables at t
    R_t: np.ndarray          # R at t
    R_tmD: np.ndarray        # R at t - Delta
    R_tmh: np.ndarray | None  # R at t - h (None before the first coarse step)
    jump: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=bool))


@dataclass
class CoarseResult:
    v_pred: np.ndarray
    v_d: np.ndarray
    e_v: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    jump: np.ndarray
    source: np.ndarray
    v: np.ndarray


def simpson(Ra, Rb, Rc):
    return (np.asarray(Ra, float) + 4.0 * np.asarray(Rb, float) + np.asarray(Rc, float)) / 6.0


def initial_state(params: PTAParams, R_mD, R_mD2, R_0) -> PTAState:
    """State at t = 0 from the three initial bursts."""
    R_mD = np.asarray(R_mD, float)
    R_0 = np.asarray(R_0, float)
    return PTAState(t=0.0, v=simpson(R_mD, R_mD2, R_0), R_t=R_0.copy(), R_tmD=R_mD.copy(),
                    R_tmh=None, jump=np.zeros(3, dtype=bool))


def _rel(x, ref, floor):
    return abs(x - ref) / max(abs(ref), floor)


def coarse_update(params: PTAParams, st: PTAState, Ra, Rb, Rc):
    """One slow step t -> t+h given the three burst averages at
    t+h-Delta, t+h-Delta/2 and t+h.  Returns (new state, CoarseResult)."""
    Ra = np.asarray(Ra, float)
    Rb = np.asarray(Rb, float)
    Rc = np.asarray(Rc, float)
    dvdt = (st.R_t - st.R_tmD) / params.Delta
    v_pred = st.v + params.h * dvdt
    v_d = simpson(Ra, Rb, Rc)
    e_v = np.zeros(3)
    e1 = np.zeros(3)
    e2 = np.full(3, np.nan)
    jump = np.zeros(3, dtype=bool)
    src = np.zeros(3, dtype=np.int32)
    v = np.zeros(3)
    for m in range(3):
        fl = params.floor[m]
        e_v[m] = _rel(v_pred[m], v_d[m], fl)
        e1[m] = _rel(Rc[m], st.R_t[m], fl)
        if st.R_tmh is not None:
            e2[m] = _rel(st.R_t[m], st.R_tmh[m], fl)
        if e_v[m] < params.tol_v[m]:
            v[m] = v_pred[m]
            src[m] = SRC_PREDICTED
            jump[m] = False
            continue
        if st.jump[m]:
            jumped = e1[m] >= params.tol_j[m]
        elif st.R_tmh is None:
            jumped = False
        elif e2[m] > 0.0:
            jumped = abs(e1[m] / e2[m] - 1.0) >= params.tol_j[m]
        else:
            jumped = e1[m] > 0.0
        v[m] = v_d[m]
        jump[m] = jumped
        src[m] = SRC_MEASURE_JUMP if jumped else SRC_MEASURE_MISMATCH
    new = PTAState(t=st.t + params.h, v=v, R_t=Rc.copy(), R_tmD=Ra.copy(),
                   R_tmh=st.R_t.copy(), jump=jump)
    return new, CoarseResult(v_pred=v_pred, v_d=v_d, e_v=e_v, e1=e1, e2=e2, jump=jump,
                             source=src, v=v)


def run(specimen, params: PTAParams, burst_steps: int, n_coarse: int, block: int = 100):
    """Drive a whole PTA run on an oracle Specimen (thermalised by the
    caller): the three initial bursts, then n_coarse slow steps.  Returns the
    list of (strain, CoarseResult) and the final PTAState."""
    from . import burst_averages
    Rs = []
    for de in params.init_increments():
        if de != 0.0:
            specimen.apply_strain(de)
        Rs.append(burst_averages(specimen.burst(burst_steps), block)[0])
    st = initial_state(params, *Rs)
    out = []
    for _ in range(n_coarse):
        Rs = []
        for de in params.step_increments():
            specimen.apply_strain(de)
            Rs.append(burst_averages(specimen.burst(burst_steps), block)[0])
        st, res = coarse_update(params, st, *Rs)
        out.append((specimen.u / specimen.L_s, res))
    return out, st


# ---------------------------------------------------------------------------
# Adaptive burst length (appendix, Eq. (R_m_conv))
# ---------------------------------------------------------------------------
def converged_averages(series, lag: int, tol, floor, n_max: int | None = None):
    """The running-average convergence test of the appendix on a burst's
    per-step samples (rows r = 1, 2, ... of `series`, columns K, U, T).

    Running average R^(i) = (1/i) sum_{r<=i} m_r, summed in step order.  The
    test e^m(i) = |R^(i) - R^(i-k)| / |R^(i)| < tol_m (Eq. (R_m_conv)) is
    applied every k = `lag` steps, at i = 2k, 3k, ... (R^(i-k) needs i > k).
    Readings where the appendix is silent (the CUDA path takes the same):
    k is a parameter; the denominator is max(|R^(i)|, floor_m), as in the
    coarse-step tests; each variable converges on its own (N_s^m = the first
    passing i, R^m = R^(N_s^m)), and the burst ends once all three have
    converged or after n_max samples, where an unconverged variable takes the
    running average of all samples.

    Returns (means, counts, converged_mask, steps_run).
    """
    s = np.asarray(series, dtype=np.float64)
    n = len(s) if n_max is None else min(len(s), n_max)
    sums = [0.0, 0.0, 0.0]
    chk = [0.0, 0.0, 0.0]
    conv_n = [0, 0, 0]
    conv_v = [0.0, 0.0, 0.0]
    mask = 0
    run = n
    for i in range(1, n + 1):
        for q in range(3):
            sums[q] = sums[q] + float(s[i - 1, q])
        if i % lag == 0:
            if i >= 2 * lag:
                for q in range(3):
                    if mask & (1 << q):
                        continue
                    a = sums[q] / float(i)
                    b = chk[q] / float(i - lag)
                    e = abs(a - b) / max(abs(a), floor[q])
                    if e < tol[q]:
                        mask |= 1 << q
                        conv_n[q] = i
                        conv_v[q] = a
            for q in range(3):
                chk[q] = sums[q]
            if mask == 7:
                run = i
                break
    means, counts = [], []
    for q in range(3):
        if mask & (1 << q):
            means.append(conv_v[q])
            counts.append(conv_n[q])
        else:
            means.append(sums[q] / float(run))
            counts.append(run)
    return np.array(means), np.array(counts), mask, run


# ---------------------------------------------------------------------------
# Verification with fine dynamics (Sec. Verification with fine dynamics)
# ---------------------------------------------------------------------------
def fine_dynamics_measures(specimen, h_steps: int, delta_steps: int, n_jumps: int,
                           ramp_per_step: float):
    """v_d^{m,fine}(t_k), k = 0..n_jumps: Eq. (measure) on one uninterrupted
    fine trajectory under continuous loading (the right grip advances by
    ramp_per_step * L_s with every step).  The trajectory starts at slow time
    -Delta; slow time t_k = k h ends at step k h_steps + delta_steps, and the
    measure is the mean of the state functions over the delta_steps steps
    ending there (N' = delta_steps samples, no Simpson rule and no restart
    from guessed initial conditions).  Returns an array [n_jumps + 1, 3]."""
    out = []
    for k in range(n_jumps + 1):
        if k > 0:
            specimen.burst(h_steps - delta_steps, ramp=ramp_per_step)
        out.append(specimen.burst(delta_steps, ramp=ramp_per_step).mean(axis=0))
    return np.array(out)


def verification_params(h_steps: int, delta_steps: int, ramp_per_step: float, dt_fs: float = 1.0,
                        **kw) -> PTAParams:
    """PTA parameters matching a fine-dynamics verification run: h and Delta
    are the fine durations h_steps and delta_steps steps (in seconds), the
    strain rate the ramp's (ramp_per_step per step)."""
    dt_s = dt_fs * 1e-15
    return PTAParams(h=h_steps * dt_s, Delta=delta_steps * dt_s,
                     strain_rate=ramp_per_step / dt_s, **kw)


def verification_errors(v_pta, v_fine):
    """The section's error, |v^PTA_m(t) - v^{m,fine}_d(t)| / |v^{m,fine}_d(t)|
    (the same form as Eq. (rel_err)), per slow jump and variable."""
    v_pta = np.asarray(v_pta, dtype=np.float64)
    v_fine = np.asarray(v_fine, dtype=np.float64)
    return np.abs(v_pta - v_fine) / np.abs(v_fine)
