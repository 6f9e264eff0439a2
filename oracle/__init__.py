"""CPU oracle for the adaptive SIS permanent estimator (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``pm_oracle.c`` (plain C, no
code shared with the CUDA library) through ctypes.  Matrices are passed as any
object with ``n``, ``row_ptr`` (int64), ``col_idx`` (int32) and ``values``
(float32 or None).

Parity status of each function (what pins it lives in tests/test_oracle_*.py):
  philox4x32_10        pinned: published known-answer vectors
  ryser / ryser_real   pinned: brute force over S_n, closed forms
  run / stats          pinned: exhaustive trajectory enumeration (sum of
                       P(path) X(path) equals per), all-ones closed form,
                       hand-worked steps, statistics closed forms
  dm_mask              pinned: brute-force support test per edge
  sk_full              pinned: k-regular closed form, doubly-stochastic limit
  local repair         pinned: hand-computed Eq. 5 example
  exp_score            pinned: libm exp within a few ulp, exact at 0
  mlp_forward / grad   pinned: central finite differences of the FP64 loss
  record (features)    pinned: hand-computed features of a 4x4 example
  run_ext              pinned: constant logits reproduce the unscaled estimator
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

VR_MIN_DEGREE_2SIDED, VR_ROW_ORDER = 0, 1
SK_NONE, SK_FIXED, SK_ADAPTIVE, SK_LOCAL = 0, 1, 2, 3
DM_NONE, DM_ALL, DM_THRS, DM_TRCK = 0, 1, 2, 3
PREC_FP32, PREC_FP64 = 0, 1


_LIB_SAN = os.path.join(_HERE, "_build", "liboracle_san.so")


def sanitized() -> bool:
    """ORACLE_SANITIZE=1: load the AddressSanitizer + UndefinedBehaviorSanitizer
    build (the process must preload libasan; any report aborts it)."""
    return os.environ.get("ORACLE_SANITIZE") == "1"


def build(force: bool = False) -> str:
    """Compile pm_oracle.c into _build/liboracle.so (gcc, no fast-math, no
    FMA contraction), or with ORACLE_SANITIZE=1 into _build/liboracle_san.so
    with -fsanitize=address,undefined (same floating-point flags)."""
    san = sanitized()
    out = _LIB_SAN if san else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        flags = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                 "-fno-sanitize-recover=undefined"] if san else ["-O2"]
        subprocess.check_call(["gcc", *flags, "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class _Schedule(C.Structure):
    _fields_ = [("vertex_rule", C.c_int32), ("initial_dm", C.c_int32), ("K0", C.c_int32),
                ("K", C.c_int32), ("sk", C.c_int32), ("dm", C.c_int32),
                ("precision", C.c_int32), ("local_cap", C.c_int32), ("theta", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("log_estimate", C.c_double), ("p_match", C.c_double),
                ("rel_spread", C.c_double), ("rse", C.c_double), ("ess", C.c_double),
                ("log_sum_x", C.c_double), ("log_sum_x2", C.c_double), ("n_alive", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_draw_u64.restype = C.c_uint64
        L.or_draw_u64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_uniform_below.restype = C.c_int64
        L.or_uniform_below.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
        L.or_ryser_int.argtypes = [C.c_int, P, P, P]
        L.or_ryser_real_d.restype = C.c_double
        L.or_ryser_real_d.argtypes = [C.c_int, P]
        L.or_prepare.restype = P
        L.or_prepare.argtypes = [C.c_int, C.c_int64, P, P, P, C.POINTER(_Schedule)]
        L.or_prep_free.argtypes = [P]
        L.or_prep_ok.restype = C.c_int
        L.or_prep_ok.argtypes = [P]
        L.or_prep_scaling.argtypes = [P, P, P]
        L.or_prep_set_max_steps.argtypes = [P, C.c_int]
        L.or_prep_mask.argtypes = [P, P]
        L.or_forced_run.restype = C.c_int
        L.or_forced_run.argtypes = [P, P, C.c_int32, P, P, P, P, P, P, P, P, C.c_int32]
        L.or_run.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int,
                             P, P, P, P, P]
        L.or_dm_mask.restype = C.c_int
        L.or_dm_mask.argtypes = [P, P]
        L.or_sk_full.argtypes = [P, C.c_int, P, P]
        L.or_statistics.argtypes = [P, C.c_int64, C.POINTER(_Stats)]
        L.or_exp_score.restype = C.c_float
        L.or_exp_score.argtypes = [C.c_float]
        L.or_mlp_forward.argtypes = [P, P, C.c_int64, C.c_int, P]
        L.or_mlp_grad_ex.restype = C.c_double
        L.or_mlp_grad_ex.argtypes = [P, P, P, P, C.c_int64, P]
        L.or_record.restype = C.c_int64
        L.or_record.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int64, P, P, P, P]
        L.or_run_ext_model.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int,
                                       P, P, P, P, P, C.c_int32, P, P]
        L.or_run_ext.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int,
                                 P, P, P, P, P, P, C.c_int32]
        L.or_run_model.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int,
                                   P, P, P, P]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# random numbers and exact permanents
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


def draw_u64(seed, traj, matrix, step, attempt) -> int:
    return int(lib().or_draw_u64(seed, traj, matrix, step, attempt))


def uniform_below(W, seed, traj, matrix, step) -> int:
    return int(lib().or_uniform_below(W, seed, traj, matrix, step))


def ryser(dense) -> int:
    """Exact permanent of an integer matrix (n <= 30), Ryser's formula."""
    a = np.ascontiguousarray(np.asarray(dense).round().astype(np.int64))
    n = a.shape[0]
    hi, lo = C.c_uint64(), C.c_uint64()
    lib().or_ryser_int(n, _ptr(a), C.byref(hi), C.byref(lo))
    v = (hi.value << 64) | lo.value
    if v >= 1 << 127:
        v -= 1 << 128
    return v


def ryser_real(dense) -> float:
    a = np.ascontiguousarray(np.asarray(dense, dtype=np.float64))
    return float(lib().or_ryser_real_d(a.shape[0], _ptr(a)))


# ---------------------------------------------------------------------------
# the estimator
# ---------------------------------------------------------------------------

@dataclass
class Schedule:
    vertex_rule: int = VR_MIN_DEGREE_2SIDED
    initial_dm: int = 0
    K0: int = 0
    K: int = 0
    sk: int = SK_NONE
    dm: int = DM_NONE
    precision: int = PREC_FP64
    theta: float = 0.33
    local_cap: int = 0  # 0: Local repair of Eq. 5; L > 0: the bounded-work reading (sampled sums)

    def c(self) -> _Schedule:
        return _Schedule(self.vertex_rule, self.initial_dm, self.K0, self.K, self.sk, self.dm,
                         self.precision, self.local_cap, self.theta)


PRESETS = {
    # the five variants of Sec. 4: two-sided MD, K0=100, K=10, initial DM
    "fixed_all": dict(sk=SK_FIXED, dm=DM_ALL),
    "adaptive_threshold": dict(sk=SK_ADAPTIVE, dm=DM_THRS),
    "local_threshold": dict(sk=SK_LOCAL, dm=DM_THRS),
    "adaptive_tracked": dict(sk=SK_ADAPTIVE, dm=DM_TRCK),
    "local_tracked": dict(sk=SK_LOCAL, dm=DM_TRCK),
}


def preset(name: str, precision: int = PREC_FP64) -> Schedule:
    return Schedule(initial_dm=1, K0=100, K=10, theta=0.33, precision=precision, **PRESETS[name])


class Prepared:
    """Preprocessing of Algorithm 2 for one matrix (InitialDM + K0 SK)."""

    def __init__(self, csr, sched: Schedule):
        self.n = int(csr.n)
        self.rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(csr.col_idx, dtype=np.int32)
        self.val = None if csr.values is None else np.ascontiguousarray(csr.values, dtype=np.float32)
        self.m = int(self.rp[-1])
        self.sched = sched
        self._s = sched.c()
        self.h = lib().or_prepare(self.n, self.m, _ptr(self.rp), _ptr(self.ci), _ptr(self.val),
                                  C.byref(self._s))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_prep_free(self.h)
            self.h = None

    def set_max_steps(self, steps: int):
        """Stop trajectories after `steps` steps (0 = run to the end): a prefix
        replay for orders where whole trajectories are too slow here."""
        lib().or_prep_set_max_steps(self.h, int(steps))

    @property
    def ok(self) -> bool:
        return bool(lib().or_prep_ok(self.h))

    def scaling(self):
        r = np.zeros(self.n)
        c = np.zeros(self.n)
        lib().or_prep_scaling(self.h, _ptr(r), _ptr(c))
        return r, c

    def mask(self):
        m = np.zeros(self.m, dtype=np.uint8)
        lib().or_prep_mask(self.h, _ptr(m))
        return m

    def run(self, seed: int, count: int, first_traj: int = 0, matrix: int = 0,
            threads: int = 1, trace: bool = False):
        """Run trajectories first_traj .. first_traj+count-1.  Returns a dict
        with log_x, dead_step, op counts and (trace) chosen [count, n, 2]
        unified ids (v, u) and deg_v [count, n]."""
        lx = np.zeros(count)
        ds = np.zeros(count, dtype=np.int32)
        ch = np.zeros((count, self.n, 2), dtype=np.int32) if trace else None
        dv = np.zeros((count, self.n), dtype=np.int32) if trace else None
        oc = np.zeros(3, dtype=np.int64)
        lib().or_run(self.h, seed, matrix, first_traj, count, threads, _ptr(lx), _ptr(ds),
                     _ptr(ch), _ptr(dv), _ptr(oc))
        out = dict(log_x=lx, dead_step=ds, n_dm=int(oc[0]), n_full_sk=int(oc[1]),
                   n_local_sk=int(oc[2]))
        if trace:
            out["chosen"] = ch
            out["deg_v"] = dv
        return out

    def run_ext(self, seed: int, count: int, logits, first_traj: int = 0, matrix: int = 0,
                threads: int = 1):
        """Trajectories with the learned proposal's logits supplied:
        logits[count, n, L] (candidate q < L of step t in adjacency order; a
        step with more than L live candidates ends its trajectory)."""
        lg = np.ascontiguousarray(logits, dtype=np.float32)
        assert lg.ndim == 3 and lg.shape[:2] == (count, self.n) and lg.shape[2] >= 1
        lx = np.zeros(count)
        ds = np.zeros(count, dtype=np.int32)
        ch = np.zeros((count, self.n, 2), dtype=np.int32)
        dv = np.zeros((count, self.n), dtype=np.int32)
        oc = np.zeros(3, dtype=np.int64)
        lib().or_run_ext(self.h, seed, matrix, first_traj, count, threads, _ptr(lx), _ptr(ds),
                         _ptr(ch), _ptr(dv), _ptr(oc), _ptr(lg), lg.shape[2])
        return dict(log_x=lx, dead_step=ds, chosen=ch, deg_v=dv)

    def run_model(self, seed: int, count: int, params, first_traj: int = 0, matrix: int = 0,
                  threads: int = 1):
        """Trajectories of the learned proposal with the given parameters (the
        device's BF16 weights: pass them already rounded)."""
        pm = np.ascontiguousarray(params, dtype=np.float64)
        lx = np.zeros(count)
        ds = np.zeros(count, dtype=np.int32)
        oc = np.zeros(3, dtype=np.int64)
        lib().or_run_model(self.h, seed, matrix, first_traj, count, threads, _ptr(lx), _ptr(ds),
                           _ptr(oc), _ptr(pm))
        return dict(log_x=lx, dead_step=ds)

    def record(self, seed: int, count: int, cap: int, first_traj: int = 0, matrix: int = 0):
        """(features[8], target, key, group) pairs along trajectories of this
        schedule; key = traj << 28 | step << 14 | candidate index; the kept
        pairs of a step are contiguous, group = index within them << 16 |
        their count (steps with fewer than two kept pairs are skipped)."""
        f = np.zeros((cap, 8), dtype=np.float32)
        t = np.zeros(cap, dtype=np.float32)
        k = np.zeros(cap, dtype=np.uint64)
        g = np.zeros(cap, dtype=np.uint32)
        m = lib().or_record(self.h, seed, matrix, first_traj, count, cap, _ptr(f), _ptr(t), _ptr(k), _ptr(g))
        return f[:m], t[:m], k[:m], g[:m]

    def run_ext_model(self, seed: int, count: int, logits, params, first_traj: int = 0, matrix: int = 0,
                      threads: int = 1):
        """Paths that follow the supplied logits[count, n, L] (as run_ext),
        with this side's network evaluated at every visited state: returns
        run_ext's dict plus model_logits[count, n, L]."""
        lg = np.ascontiguousarray(logits, dtype=np.float32)
        assert lg.ndim == 3 and lg.shape[:2] == (count, self.n) and lg.shape[2] >= 1
        pm = np.ascontiguousarray(params, dtype=np.float64)
        lx = np.zeros(count)
        ds = np.zeros(count, dtype=np.int32)
        ch = np.zeros((count, self.n, 2), dtype=np.int32)
        dv = np.zeros((count, self.n), dtype=np.int32)
        ml = np.zeros(lg.shape, dtype=np.float32)
        lib().or_run_ext_model(self.h, seed, matrix, first_traj, count, threads, _ptr(lx), _ptr(ds), _ptr(ch),
                               _ptr(dv), _ptr(lg), lg.shape[2], _ptr(pm), _ptr(ml))
        return dict(log_x=lx, dead_step=ds, chosen=ch, deg_v=dv, model_logits=ml)

    def forced(self, choices, logits=None):
        """Replay with forced candidate indices.  Returns ("need", w[], W,
        log_x_prefix, info) when the choices run out before the trajectory
        ends, else ("done", log_x, dead_step, info); info holds the chosen
        (v, u) pairs so far and the DM / full-SK / local-SK counts."""
        ch = np.ascontiguousarray(choices, dtype=np.int32)
        w = np.zeros(max(1, self.n), dtype=np.uint64)
        W = C.c_uint64()
        nc = C.c_int32()
        lx = C.c_double()
        ds = C.c_int32()
        chosen = np.zeros((max(1, self.n), 2), dtype=np.int32)
        counts = np.zeros(3, dtype=np.int32)
        lg = None if logits is None else np.ascontiguousarray(logits, dtype=np.float32)
        stride = 0 if lg is None else int(lg.shape[-1])
        need = lib().or_forced_run(self.h, _ptr(ch), len(ch), _ptr(w), C.byref(W), C.byref(nc),
                                   C.byref(lx), C.byref(ds), _ptr(chosen), _ptr(counts), _ptr(lg), stride)
        info = dict(chosen=chosen[: self.n], n_dm=int(counts[0]), n_full_sk=int(counts[1]),
                    n_local_sk=int(counts[2]))
        if need:
            return ("need", [int(x) for x in w[: nc.value]], int(W.value), lx.value, info)
        return ("done", lx.value, ds.value, info)


def dm_mask(csr):
    """Supported-edge mask of a whole matrix (Sec. 2 DM); None if the matrix
    has no perfect matching."""
    P = Prepared(csr, Schedule())
    m = np.zeros(P.m, dtype=np.uint8)
    ok = lib().or_dm_mask(P.h, _ptr(m))
    return m if ok else None


def sk_full(csr, iters: int, precision: int = PREC_FP64):
    P = Prepared(csr, Schedule(precision=precision))
    r = np.zeros(P.n)
    c = np.zeros(P.n)
    lib().or_sk_full(P.h, iters, _ptr(r), _ptr(c))
    return r, c


def stats(log_x) -> dict:
    a = np.ascontiguousarray(log_x, dtype=np.float64)
    s = _Stats()
    lib().or_statistics(_ptr(a), a.size, C.byref(s))
    return dict(log_estimate=s.log_estimate, p_match=s.p_match, rel_spread=s.rel_spread,
                rse=s.rse, ess=s.ess, log_sum_x=s.log_sum_x, log_sum_x2=s.log_sum_x2,
                n_alive=int(s.n_alive), n_traj=int(a.size))


# ---------------------------------------------------------------------------
# learned proposal (an extension; the paper has no learned part)
# ---------------------------------------------------------------------------

N_PARAM = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


def exp_score(x: float) -> float:
    """e^x of the learned proposal's score (own binary32 polynomial)."""
    return float(lib().or_exp_score(float(x)))


def mlp_forward(params, X, round_act: bool = False):
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(x.shape[0])
    lib().or_mlp_forward(_ptr(p), _ptr(x), x.shape[0], int(round_act), _ptr(out))
    return out


def mlp_grad(params, X, T, group=None):
    """(loss, gradient) of the MLP on (X, T): the mean squared error, or with
    group (index within the step << 16 | step's pair count, rows of a step
    contiguous) the mean squared error after removing each step's mean
    residual."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(X, dtype=np.float64)
    t = np.ascontiguousarray(T, dtype=np.float64)
    gr = None if group is None else np.ascontiguousarray(group, dtype=np.uint32)
    g = np.zeros(N_PARAM)
    loss = lib().or_mlp_grad_ex(_ptr(p), _ptr(x), _ptr(t), _ptr(gr), x.shape[0], _ptr(g))
    return loss, g
