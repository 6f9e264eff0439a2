"""Shared fixtures of the GPU tests: the library context and comparison of a
CUDA trace with an oracle trace."""
import numpy as np

import oracle as O

B = None
_ctx = None


def binding():
    global B
    if B is None:
        from paper_2608_15390_b300 import binding as b
        B = b
    return B


def ctx():
    global _ctx
    if _ctx is None:
        _ctx = binding().Context(0)
    return _ctx


def to_gpu_sched(s: "O.Schedule"):
    b = binding()
    return b.Schedule(vertex_rule=s.vertex_rule, initial_dm=s.initial_dm, K0=s.K0, K=s.K, sk=s.sk,
                      dm=s.dm, precision=s.precision, theta=s.theta, local_cap=s.local_cap)


def logx_close(a, b, tol):
    """|a - b| <= tol * max(1, |b|) elementwise, with equal -inf positions."""
    a = np.asarray(a)
    b = np.asarray(b)
    dead_a, dead_b = np.isneginf(a), np.isneginf(b)
    assert np.array_equal(dead_a, dead_b), "dead trajectories differ"
    ok = ~dead_a
    err = np.abs(a[ok] - b[ok]) / np.maximum(1.0, np.abs(b[ok]))
    return float(err.max()) if err.size else 0.0


def compare_trace(m, sched, count, seed=1, first=0, matrix_index=0, tol=1e-12, threads=8):
    """Run `count` trajectories on the GPU (pm_trace) and in the oracle and
    require bit-exact paths, degrees and death steps, log-weights within tol."""
    g = ctx().trace(m, count, seed, to_gpu_sched(sched), first_traj=first, matrix_index=matrix_index)
    P = O.Prepared(m, sched)
    o = P.run(seed=seed, count=count, first_traj=first, matrix=matrix_index, threads=threads, trace=True)
    assert np.array_equal(g["dead_step"], o["dead_step"]), "dead steps differ"
    assert np.array_equal(g["deg_v"], o["deg_v"]), "picked-vertex degrees differ"
    assert np.array_equal(g["chosen"], o["chosen"]), "chosen edges differ"
    err = logx_close(g["log_x"], o["log_x"], tol)
    assert err <= tol, f"log-weight error {err}"
    return g, o
