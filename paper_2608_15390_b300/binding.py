"""ctypes binding of the C ABI in include/pm.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libpm_b300.so``; when it is
missing or cannot load, importing the binding raises, and there is no other
code path.  Function names follow the header: ``estimate_permanent``,
``estimate_permanent_batch``, ``pm_trace``, ``pm_preprocess``,
``pm_philox_blocks``.

Matrices are any object with ``n``, ``row_ptr`` (int64), ``col_idx`` (int32)
and ``values`` (float32 or None) as numpy arrays (host) or torch tensors
(host or CUDA; CUDA tensors are passed as device pointers).
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PM_LIB=debug selects the PM_DEBUG build (bounds-checked matrix views in the
# trajectory kernels; an out-of-range access fails the call with PM_EDEVICE)
DEBUG_BUILD = os.environ.get("PM_LIB") == "debug"
LIB_PATH = os.path.join(_HERE, "_lib", "libpm_b300_debug.so" if DEBUG_BUILD else "libpm_b300.so")

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_ETIMEOUT, PM_ECANCELLED, PM_EUNSUPPORTED, PM_EDEVICE = range(8)
VR_MIN_DEGREE_2SIDED, VR_ROW_ORDER = 0, 1
SK_NONE, SK_FIXED, SK_ADAPTIVE, SK_LOCAL = 0, 1, 2, 3
DM_NONE, DM_ALL, DM_THRS, DM_TRCK = 0, 1, 2, 3
PREC_FP32_PROPOSAL, PREC_FP64 = 0, 1
OBJ_MSE, OBJ_CENTRED = 0, 1
BATCH_GRAPH, BATCH_AUTOTUNE = 1, 2
REQ_DONE, REQ_BUDGET, REQ_REFUSED, REQ_FAILED = 0, 1, 2, 3


class PmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class pm_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("on_device", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("values", C.c_void_p)]


class pm_schedule(C.Structure):
    _fields_ = [("vertex_rule", C.c_int32), ("initial_dm", C.c_int32), ("K0", C.c_int32),
                ("K", C.c_int32), ("sk", C.c_int32), ("dm", C.c_int32), ("precision", C.c_int32),
                ("local_cap", C.c_int32), ("theta", C.c_double), ("learned", C.c_void_p),
                ("rse_target", C.c_double), ("time_budget_s", C.c_double)]


class pm_train_cfg(C.Structure):
    _fields_ = [("n_pairs", C.c_uint64), ("seed", C.c_uint64), ("epochs", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("teacher", pm_schedule), ("objective", C.c_int32),
                ("reserved", C.c_int32)]


class pm_train_report(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("n_pairs", C.c_uint64),
                ("steps", C.c_int32), ("reserved", C.c_int32), ("seconds_record", C.c_double),
                ("seconds_train", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class pm_plan_info(C.Structure):
    _fields_ = [("g", C.c_int32), ("groups", C.c_int32), ("staged", C.c_int32), ("rc_smem", C.c_int32),
                ("gstate", C.c_int32), ("dm_smem", C.c_int32), ("tuned", C.c_int32), ("pair", C.c_int32),
                ("probe_traj_per_s", C.c_double), ("heuristic_traj_per_s", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class pm_server_cfg(C.Structure):
    _fields_ = [("schedule", pm_schedule), ("seed", C.c_uint64), ("device_budget_bytes", C.c_uint64),
                ("steps_per_round", C.c_uint64), ("traj_min", C.c_uint32), ("traj_max", C.c_uint32),
                ("min_traj_done", C.c_uint64)]


class pm_result(C.Structure):
    _fields_ = [("log_estimate", C.c_double), ("estimate", C.c_double), ("ess", C.c_double),
                ("p_match", C.c_double), ("rel_spread", C.c_double), ("rse", C.c_double),
                ("log_sum_x", C.c_double), ("log_sum_x2", C.c_double), ("n_traj", C.c_uint64),
                ("n_alive", C.c_uint64), ("n_dm_calls", C.c_uint64), ("n_full_sk", C.c_uint64),
                ("n_local_sk", C.c_uint64), ("seconds", C.c_double), ("alg_bytes", C.c_uint64),
                ("kernel_ms", C.c_double), ("mlp_rows", C.c_uint64), ("traj_ns", C.c_uint64), ("dev_ms", C.c_double), ("rounds", C.c_uint32),
                ("stop", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "pm_result":
        r = cls()
        for f, _ in cls._fields_:
            if f in d:
                setattr(r, f, d[f])
        return r


class pm_request_done(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("rounds", C.c_uint32), ("result", pm_result),
                ("submit_time", C.c_double), ("done_time", C.c_double)]


class pm_call_info(C.Structure):
    _fields_ = [("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64), ("traj_kernel_ms", C.c_double),
                ("prep_kernel_ms", C.c_double), ("grid", C.c_int32), ("warps_per_cta", C.c_int32),
                ("first_plan", pm_plan_info), ("grad_kernel_ms", C.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "first_plan"}
        d["first_plan"] = self.first_plan.as_dict()
        return d


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run python -m paper_2608_15390_b300.build"
                          f"{' --debug' if DEBUG_BUILD else ''})")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.pm_context_create.argtypes = [C.POINTER(P), C.c_int, P]
    L.pm_context_destroy.argtypes = [P]
    L.estimate_permanent.argtypes = [P, C.POINTER(pm_csr), C.c_int32, C.c_uint64, C.c_uint64,
                                     C.POINTER(pm_schedule), C.POINTER(pm_result)]
    L.estimate_permanent_batch.argtypes = [P, C.POINTER(pm_csr), C.c_int32, P, C.c_uint64,
                                           C.POINTER(pm_schedule), C.POINTER(pm_result)]
    L.pm_estimate_batch_ex.argtypes = [P, C.POINTER(pm_csr), C.c_int32, P, C.c_uint64, C.c_uint64,
                                       C.POINTER(pm_schedule), C.POINTER(pm_result), P]
    L.pm_trace.argtypes = [P, C.POINTER(pm_csr), C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint64,
                           C.POINTER(pm_schedule), P, P, P, P, P, C.c_uint32]
    L.pm_context_cancel.argtypes = [P]
    L.pm_layout_set.argtypes = [P, C.POINTER(pm_schedule), C.c_int32, C.c_int64, C.POINTER(pm_plan_info)]
    L.pm_layout_set.restype = C.c_int
    L.pm_tune_theta.argtypes = [P, C.POINTER(pm_csr), C.POINTER(pm_schedule), P, C.c_int32, C.c_double, C.c_uint64, P]
    L.pm_tune_theta.restype = C.c_int
    L.pm_probe_bandwidth.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.pm_probe_bandwidth.restype = C.c_int
    L.pm_merge_results.argtypes = [C.POINTER(pm_result), C.c_int32, C.POINTER(pm_result)]
    L.pm_model_save.argtypes = [P, P, C.c_char_p]
    L.pm_model_load.argtypes = [P, C.c_char_p, C.POINTER(P)]
    for name in ("pm_context_cancel", "pm_merge_results", "pm_model_save", "pm_model_load"):
        getattr(L, name).restype = C.c_int
    L.pm_model_create.argtypes = [P, P, C.c_uint64, C.POINTER(P)]
    L.pm_model_destroy.argtypes = [P]
    L.pm_model_get_params.argtypes = [P, P, P]
    L.pm_model_set_params.argtypes = [P, P, P]
    L.pm_model_train.argtypes = [P, P, C.POINTER(pm_csr), C.c_int32, C.POINTER(pm_train_cfg),
                                 C.POINTER(pm_train_report)]
    L.pm_mlp_forward.argtypes = [P, P, P, C.c_uint64, P]
    L.pm_mlp_gradient.argtypes = [P, P, P, P, P, C.c_uint64, P, P]
    L.pm_record_pairs.argtypes = [P, C.POINTER(pm_csr), C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint64,
                                  C.POINTER(pm_schedule), C.c_uint64, P, P, P, P, P]
    for name in ("pm_model_create", "pm_model_destroy", "pm_model_get_params", "pm_model_set_params",
                 "pm_model_train", "pm_mlp_forward", "pm_mlp_gradient", "pm_record_pairs"):
        getattr(L, name).restype = C.c_int
    L.pm_batch_create.argtypes = [P, C.POINTER(pm_csr), C.c_int32, P, C.POINTER(pm_schedule), C.c_uint32,
                                  C.POINTER(P)]
    L.pm_batch_run.argtypes = [P, C.c_uint64, C.c_uint64, C.POINTER(pm_result), P]
    L.pm_batch_plan_info.argtypes = [P, C.c_int32, C.POINTER(pm_plan_info)]
    L.pm_batch_destroy.argtypes = [P]
    for name in ("pm_batch_create", "pm_batch_run", "pm_batch_plan_info", "pm_batch_destroy"):
        getattr(L, name).restype = C.c_int
    L.pm_server_create.argtypes = [P, C.POINTER(pm_server_cfg), C.POINTER(P)]
    L.pm_server_submit.argtypes = [P, C.POINTER(pm_csr), C.c_double, C.c_uint64, C.POINTER(C.c_uint64)]
    L.pm_server_round.argtypes = [P, C.POINTER(pm_request_done), C.c_uint32, C.POINTER(C.c_uint32),
                                  C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.pm_server_destroy.argtypes = [P]
    for name in ("pm_server_create", "pm_server_submit", "pm_server_round", "pm_server_destroy"):
        getattr(L, name).restype = C.c_int
    L.pm_server_clock.argtypes = [P]
    L.pm_server_clock.restype = C.c_double
    L.pm_preprocess.argtypes = [P, C.POINTER(pm_csr), C.POINTER(pm_schedule), P, P, P, P]
    L.pm_philox_blocks.argtypes = [P, P, P, C.c_uint32, P]
    L.pm_last_call_info.argtypes = [P, C.POINTER(pm_call_info)]
    L.pm_last_call_info.restype = C.c_int
    L.pm_log_weight_stats_noalloc.argtypes = [P, C.c_uint64, P, P]
    L.pm_log_weight_stats_noalloc.restype = C.c_int
    L.pm_status_string.restype = C.c_char_p
    L.pm_status_string.argtypes = [C.c_int]
    L.pm_last_error.restype = C.c_char_p
    L.pm_last_error.argtypes = [P]
    for name in ("pm_context_create", "pm_context_destroy", "estimate_permanent",
                 "estimate_permanent_batch", "pm_estimate_batch_ex", "pm_trace", "pm_preprocess", "pm_philox_blocks"):
        getattr(L, name).restype = C.c_int
    return L


_lib = _load()


def lib():
    return _lib


def _status_name(s: int) -> str:
    return _lib.pm_status_string(s).decode()


EXPORTED = ["pm_context_create", "pm_context_destroy", "estimate_permanent",
            "estimate_permanent_batch", "pm_estimate_batch_ex", "pm_trace", "pm_preprocess", "pm_philox_blocks",
            "pm_last_call_info", "pm_log_weight_stats_noalloc", "pm_status_string", "pm_last_error",
            "pm_model_create", "pm_model_destroy", "pm_model_get_params", "pm_model_set_params",
            "pm_model_train", "pm_mlp_forward", "pm_mlp_gradient", "pm_record_pairs",
            "pm_batch_create", "pm_batch_run", "pm_batch_plan_info", "pm_batch_destroy",
            "pm_server_create", "pm_server_submit", "pm_server_round", "pm_server_clock", "pm_server_destroy",
            "pm_context_cancel", "pm_merge_results", "pm_model_save", "pm_model_load", "pm_probe_bandwidth",
            "pm_layout_set", "pm_tune_theta"]

STOP_COMPLETE, STOP_TARGET, STOP_TIME, STOP_CANCELLED = 0, 1, 2, 3


def merge_results(results: Sequence[dict]) -> dict:
    """pm_merge_results: merge result dicts of disjoint trajectory sets of
    one matrix (host arithmetic in the library; no device needed)."""
    rs = list(results)
    if not rs:
        raise ValueError("nothing to merge")
    arr = (pm_result * len(rs))(*[pm_result.from_dict(r) for r in rs])
    out = pm_result()
    st = _lib.pm_merge_results(arr, len(rs), C.byref(out))
    if st != PM_OK:
        raise PmError(st, "pm_merge_results")
    return out.as_dict()


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
    learned: Optional["Model"] = None
    rse_target: float = 0.0
    time_budget_s: float = 0.0
    local_cap: int = 0

    def c(self) -> pm_schedule:
        return pm_schedule(self.vertex_rule, self.initial_dm, self.K0, self.K, self.sk, self.dm,
                           self.precision, self.local_cap, self.theta,
                           None if self.learned is None else self.learned.h.value,
                           self.rse_target, self.time_budget_s)


def preset(name: str, precision: int = PREC_FP32_PROPOSAL) -> Schedule:
    """The five variants of Sec. 4 (two-sided MD, K0=100, K=10, theta=0.33,
    initial DM)."""
    sk, dm = {"fixed_all": (SK_FIXED, DM_ALL), "adaptive_threshold": (SK_ADAPTIVE, DM_THRS),
              "local_threshold": (SK_LOCAL, DM_THRS), "adaptive_tracked": (SK_ADAPTIVE, DM_TRCK),
              "local_tracked": (SK_LOCAL, DM_TRCK)}[name]
    return Schedule(initial_dm=1, K0=100, K=10, sk=sk, dm=dm, precision=precision, theta=0.33)


def _arr_ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0, a
    a = np.ascontiguousarray(a)
    return a.ctypes.data, 0, a


def make_csr(m) -> tuple:
    rp, d0, k0 = _arr_ptr(m.row_ptr)
    ci, d1, k1 = _arr_ptr(m.col_idx)
    vals = getattr(m, "values", None)
    vp, d2, k2 = _arr_ptr(vals)
    dev = d0
    if d1 != dev or (vals is not None and d2 != dev):
        raise ValueError("row_ptr, col_idx and values must all be on the host or all on the device")
    nnz = int(m.row_ptr[-1]) if not dev else int(m.col_idx.numel())
    c = pm_csr(int(m.n), dev, nnz, rp, ci, vp)
    return c, (k0, k1, k2)


WEIGHT_STATS_FIELDS = ["log_estimate", "ess", "p_match", "rel_spread", "rse", "log_sum_x",
                       "log_sum_x2", "n_traj", "n_alive"]


def log_weight_stats_noalloc(log_x_ptr: int, M: int, out_ptr: int, stream: int = 0) -> int:
    """pm_log_weight_stats_noalloc on device pointers (returns the status)."""
    return _lib.pm_log_weight_stats_noalloc(log_x_ptr, M, out_ptr, stream or None)


class Context:
    """Owns a pm_context (device arena + stream).  ``stream`` is a raw
    cudaStream_t value (e.g. ``torch.cuda.current_stream().cuda_stream``)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.h = C.c_void_p()
        self._batches = weakref.WeakSet()
        self._check(_lib.pm_context_create(C.byref(self.h), device, stream), ctx=False)

    def close(self):
        if self.h:
            for b in list(self._batches):
                b.close()
            _lib.pm_context_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, ctx: bool = True):
        if st != PM_OK:
            msg = _lib.pm_last_error(self.h).decode() if ctx and self.h else ""
            raise PmError(st, msg)

    def _check_run(self, st: int) -> int:
        """As _check, but a call that stopped early (time budget, cancel)
        returns its status: its outputs describe the trajectories that ran."""
        if st in (PM_ETIMEOUT, PM_ECANCELLED):
            return st
        self._check(st)
        return st

    def probe_bandwidth(self) -> dict:
        """pm_probe_bandwidth: measured L2 and shared-memory read GB/s."""
        l2, sm = C.c_double(), C.c_double()
        self._check(_lib.pm_probe_bandwidth(self.h, C.byref(l2), C.byref(sm)))
        return {"l2_read_gbs": l2.value, "smem_read_gbs": sm.value}

    def layout_set(self, schedule: Schedule, n: int, nnz: int, g: int = 1, staged: int = 0, rc_smem: int = 0,
                   gstate: int = 0, dm_smem: int = 0, pair: int = 0):
        """pm_layout_set: pin the layout of n's size class under `schedule`."""
        lay = pm_plan_info(g, 0, staged, rc_smem, gstate, dm_smem, 0, pair, -1.0, -1.0)
        s = schedule.c()
        self._check(_lib.pm_layout_set(self.h, C.byref(s), n, nnz, C.byref(lay)))

    def tune_theta(self, m, schedule: Schedule, thetas, probe_s: float = 0.5, seed: int = 1):
        """pm_tune_theta: (best theta, scores) by RSE^2 x seconds of probe runs."""
        c, keep = make_csr(m)
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        sc = np.zeros(len(th))
        s = schedule.c()
        self._check(_lib.pm_tune_theta(self.h, C.byref(c), C.byref(s), th.ctypes.data, len(th), probe_s, seed,
                                       sc.ctypes.data))
        return s.theta, sc

    def cancel(self):
        """pm_context_cancel: stop the running call (any thread)."""
        self._check(_lib.pm_context_cancel(self.h))

    def model_load(self, path: str) -> "Model":
        """pm_model_load: a model from a file written by Model.save."""
        m = Model.__new__(Model)
        m.ctx = self
        m.h = C.c_void_p()
        self._check(_lib.pm_model_load(self.h, os.fsencode(path), C.byref(m.h)))
        return m

    # ---- entry points ----
    def estimate_permanent(self, m, n_traj: int, seed: int, schedule: Schedule) -> dict:
        c, keep = make_csr(m)
        out = pm_result()
        s = schedule.c()
        st = self._check_run(_lib.estimate_permanent(self.h, C.byref(c), c.n, n_traj, seed, C.byref(s),
                                                     C.byref(out)))
        d = out.as_dict()
        d["status"] = st
        return d

    def estimate_permanent_batch(self, mats: Sequence, n_traj: Sequence[int], seed: int,
                                 schedule: Schedule) -> List[dict]:
        cs, keeps = [], []
        for m in mats:
            c, k = make_csr(m)
            cs.append(c)
            keeps.append(k)
        arr = (pm_csr * len(cs))(*cs)
        nt = np.ascontiguousarray(n_traj, dtype=np.uint64)
        outs = (pm_result * len(cs))()
        s = schedule.c()
        st = self._check_run(_lib.estimate_permanent_batch(self.h, arr, len(cs), nt.ctypes.data, seed,
                                                           C.byref(s), outs))
        return [dict(o.as_dict(), status=st) for o in outs]

    def estimate_batch_ex(self, mats: Sequence, n_traj: Sequence[int], seed: int,
                          schedule: Schedule, first_traj: int = 0, want_log_x: bool = False):
        """Batch estimate; returns (results, log_x or None)."""
        cs, keeps = [], []
        for m in mats:
            c, k = make_csr(m)
            cs.append(c)
            keeps.append(k)
        arr = (pm_csr * len(cs))(*cs)
        nt = np.ascontiguousarray(n_traj, dtype=np.uint64)
        outs = (pm_result * len(cs))()
        lx = np.zeros(int(nt.sum()), dtype=np.float64) if want_log_x else None
        s = schedule.c()
        st = self._check_run(_lib.pm_estimate_batch_ex(self.h, arr, len(cs), nt.ctypes.data, first_traj, seed,
                                                       C.byref(s), outs,
                                                       None if lx is None else lx.ctypes.data))
        return [dict(o.as_dict(), status=st) for o in outs], lx

    def server(self, schedule: Schedule, seed: int = 1, device_budget_bytes: int = 8 << 30,
               steps_per_round: int = 1 << 20, traj_min: int = 32, traj_max: int = 1 << 16,
               min_traj_done: int = 1024) -> "Server":
        """A serving loop (pm_server_create); closing the context closes it."""
        sv = Server(self, schedule, seed, device_budget_bytes, steps_per_round, traj_min, traj_max, min_traj_done)
        self._batches.add(sv)
        return sv

    def batch(self, mats: Sequence, n_traj: Sequence[int], schedule: Schedule, graph: bool = True,
              autotune: bool = False) -> "Batch":
        """A resident batch (pm_batch_create): device copies of mats, one
        persistent launch per run, optionally a CUDA graph and autotuned
        layouts.  Closing the context closes its batches first."""
        b = Batch(self, mats, n_traj, schedule, graph, autotune)
        self._batches.add(b)
        return b

    def trace(self, m, count: int, seed: int, schedule: Schedule, first_traj: int = 0,
              matrix_index: int = 0, logit_stride: Optional[int] = None) -> dict:
        """Paths of trajectories first_traj .. first_traj + count - 1
        (pm_trace).  With the learned proposal, logits[count, n, L] holds the
        network output of every live candidate of every step; L defaults to
        the largest row or column length of m, which keeps them all."""
        c, keep = make_csr(m)
        n = c.n
        chosen = np.zeros((count, n, 2), dtype=np.int32)
        degv = np.zeros((count, n), dtype=np.int32)
        dead = np.zeros(count, dtype=np.int32)
        lx = np.zeros(count, dtype=np.float64)
        lg = None
        if schedule.learned is not None:
            if logit_stride is None:
                rows = np.diff(np.asarray(m.row_ptr))
                cols = np.bincount(np.asarray(m.col_idx), minlength=n)
                logit_stride = int(max(1, rows.max(initial=0), cols.max(initial=0)))
            lg = np.zeros((count, n, logit_stride), dtype=np.float32)
        s = schedule.c()
        self._check(_lib.pm_trace(self.h, C.byref(c), matrix_index, first_traj, count, seed,
                                  C.byref(s), chosen.ctypes.data, degv.ctypes.data,
                                  dead.ctypes.data, lx.ctypes.data,
                                  None if lg is None else lg.ctypes.data,
                                  0 if lg is None else lg.shape[2]))
        out = dict(chosen=chosen, deg_v=degv, dead_step=dead, log_x=lx)
        if lg is not None:
            out["logits"] = lg
        return out

    def record_pairs(self, m, count: int, seed: int, teacher: Schedule, cap: int,
                     first_traj: int = 0, matrix_index: int = 0):
        c, keep = make_csr(m)
        f = np.zeros((cap, 8), dtype=np.float32)
        t = np.zeros(cap, dtype=np.float32)
        k = np.zeros(cap, dtype=np.uint64)
        g = np.zeros(cap, dtype=np.uint32)
        n_out = C.c_uint64()
        s = teacher.c()
        self._check(_lib.pm_record_pairs(self.h, C.byref(c), matrix_index, first_traj, count, seed,
                                         C.byref(s), cap, f.ctypes.data, t.ctypes.data,
                                         k.ctypes.data, g.ctypes.data, C.byref(n_out)))
        n = n_out.value
        return f[:n], t[:n], k[:n], g[:n]

    def model(self, params=None, seed: int = 0) -> "Model":
        return Model(self, params, seed)

    def preprocess(self, m, schedule: Schedule) -> dict:
        c, keep = make_csr(m)
        ok = C.c_int32()
        kp = np.zeros(max(1, c.nnz), dtype=np.uint8)
        r = np.zeros(c.n)
        cc = np.zeros(c.n)
        s = schedule.c()
        self._check(_lib.pm_preprocess(self.h, C.byref(c), C.byref(s), C.byref(ok), kp.ctypes.data,
                                       r.ctypes.data, cc.ctypes.data))
        return dict(ok=bool(ok.value), keep=kp[: c.nnz], r=r, c=cc)

    def last_call_info(self) -> dict:
        info = pm_call_info()
        self._check(_lib.pm_last_call_info(self.h, C.byref(info)))
        return info.as_dict()

    def philox_blocks(self, ctr, key, count: int) -> np.ndarray:
        ct = np.ascontiguousarray(ctr, dtype=np.uint32)
        ky = np.ascontiguousarray(key, dtype=np.uint32)
        out = np.zeros((count, 4), dtype=np.uint32)
        self._check(_lib.pm_philox_blocks(self.h, ct.ctypes.data, ky.ctypes.data, count,
                                          out.ctypes.data))
        return out


N_PARAM = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


class Model:
    """The learned proposal's network (pm_model)."""

    def __init__(self, ctx: Context, params=None, seed: int = 0):
        self.ctx = ctx
        self.h = C.c_void_p()
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        ctx._check(_lib.pm_model_create(ctx.h, None if p is None else p.ctypes.data, seed,
                                        C.byref(self.h)))

    def close(self):
        if self.h:
            _lib.pm_model_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path: str):
        """pm_model_save: write the parameters to a file (Context.model_load reads it)."""
        self.ctx._check(_lib.pm_model_save(self.ctx.h, self.h, os.fsencode(path)))

    def params(self) -> np.ndarray:
        out = np.zeros(N_PARAM, dtype=np.float32)
        self.ctx._check(_lib.pm_model_get_params(self.ctx.h, self.h, out.ctypes.data))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self.ctx._check(_lib.pm_model_set_params(self.ctx.h, self.h, p.ctypes.data))

    def forward(self, X) -> np.ndarray:
        x = np.ascontiguousarray(X, dtype=np.float32)
        out = np.zeros(x.shape[0], dtype=np.float32)
        self.ctx._check(_lib.pm_mlp_forward(self.ctx.h, self.h, x.ctypes.data, x.shape[0], out.ctypes.data))
        return out

    def gradient(self, X, T, group=None):
        """(loss, gradient): mean squared error, or with group codes (index
        within the step << 16 | step size, steps consecutive) the per-step
        centred loss."""
        x = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(T, dtype=np.float32)
        gr = None if group is None else np.ascontiguousarray(group, dtype=np.uint32)
        g = np.zeros(N_PARAM, dtype=np.float32)
        loss = C.c_double()
        self.ctx._check(_lib.pm_mlp_gradient(self.ctx.h, self.h, x.ctypes.data, t.ctypes.data,
                                             None if gr is None else gr.ctypes.data, x.shape[0],
                                             g.ctypes.data, C.byref(loss)))
        return loss.value, g

    def train(self, mats, teacher: Schedule, n_pairs: int, epochs: int = 2, batch: int = 4096,
              lr: float = 2e-3, seed: int = 1, objective: int = 1) -> dict:
        """Record pairs from `teacher` on mats, then Adam on `objective`
        (OBJ_MSE or OBJ_CENTRED, the default)."""
        cs, keeps = [], []
        for m in mats:
            c, k = make_csr(m)
            cs.append(c)
            keeps.append(k)
        arr = (pm_csr * len(cs))(*cs)
        cfg = pm_train_cfg(n_pairs, seed, epochs, batch, lr, 0.9, 0.999, 1e-8, teacher.c(), objective, 0)
        rep = pm_train_report()
        self.ctx._check(_lib.pm_model_train(self.ctx.h, self.h, arr, len(cs), C.byref(cfg), C.byref(rep)))
        return rep.as_dict()


class Batch:
    """pm_batch: matrices kept on the device and estimated again and again,
    each run over a fresh trajectory range."""

    def __init__(self, ctx: Context, mats, n_traj, schedule: Schedule, graph: bool, autotune: bool):
        self.ctx = ctx
        self.h = None
        cs, keeps = [], []
        for m in mats:
            c, k = make_csr(m)
            cs.append(c)
            keeps.append(k)
        arr = (pm_csr * len(cs))(*cs)
        self.count = len(cs)
        self.n_traj = np.ascontiguousarray(n_traj, dtype=np.uint64)
        self._sched = schedule.c()
        self._keep = (schedule, keeps)
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
        h = C.c_void_p()
        ctx._check(_lib.pm_batch_create(ctx.h, arr, self.count, self.n_traj.ctypes.data, C.byref(self._sched),
                                        flags, C.byref(h)))
        self.h = h

    def run(self, first_traj: int, seed: int, want_log_x: bool = False):
        """Returns (results, log_x or None) as Context.estimate_batch_ex."""
        outs = (pm_result * self.count)()
        lx = np.zeros(int(self.n_traj.sum()), dtype=np.float64) if want_log_x else None
        st = self.ctx._check_run(_lib.pm_batch_run(self.h, first_traj, seed, outs,
                                                   None if lx is None else lx.ctypes.data))
        return [dict(o.as_dict(), status=st) for o in outs], lx

    def plan(self, k: int) -> dict:
        info = pm_plan_info()
        self.ctx._check(_lib.pm_batch_plan_info(self.h, k, C.byref(info)))
        return info.as_dict()

    def close(self):
        if self.h and self.ctx.h:
            _lib.pm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """pm_server: requests submitted at any time, estimated in rounds of one
    persistent launch each until their RSE target or budget."""

    def __init__(self, ctx: Context, schedule: Schedule, seed, budget, steps, tmin, tmax, min_done):
        self.ctx = ctx
        self.h = None
        self._sched = schedule
        cfg = pm_server_cfg(schedule.c(), seed, budget, steps, tmin, tmax, min_done)
        h = C.c_void_p()
        ctx._check(_lib.pm_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self._buf = (pm_request_done * 4096)()

    def submit(self, m, target_rse: float, max_traj: int) -> int:
        c, keep = make_csr(m)
        rid = C.c_uint64()
        self.ctx._check(_lib.pm_server_submit(self.h, C.byref(c), target_rse, max_traj, C.byref(rid)))
        return rid.value

    def round(self):
        """One round; returns (finished requests as dicts, n_active, n_queued)."""
        nd, na, nq = C.c_uint32(), C.c_uint32(), C.c_uint32()
        self.ctx._check(_lib.pm_server_round(self.h, self._buf, len(self._buf), C.byref(nd), C.byref(na),
                                             C.byref(nq)))
        out = []
        for i in range(nd.value):
            d = self._buf[i]
            out.append({"id": d.id, "status": d.status, "rounds": d.rounds, "result": d.result.as_dict(),
                        "submit_time": d.submit_time, "done_time": d.done_time})
        return out, na.value, nq.value

    def clock(self) -> float:
        return _lib.pm_server_clock(self.h)

    def close(self):
        if self.h and self.ctx.h:
            _lib.pm_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
