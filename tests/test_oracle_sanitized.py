"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a child
process loads the sanitized build (ORACLE_SANITIZE=1, libasan preloaded) and
runs every kind of oracle call on small inputs: trajectories of the plain,
weighted, row-order, Fixed / Adaptive / Local SK, bounded Local and All /
Thrs / Trck DM schedules in both precisions, traces, the learned proposal
and its replay, recording, DM masks, SK sweeps, Ryser, statistics and the
network's forward and gradient.  Any out-of-bounds access, use after free,
signed overflow or other undefined behaviour aborts the child."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import numpy as np
    import oracle as O
    from paper_2608_15390_b300 import inputs as G
    assert O.sanitized()
    mats = [G.er_planted(30, 3.0, seed=1), G.random_weighted(24, 0.2, seed=2), G.powerlaw_planted(60, seed=3),
            G.block_diagonal(40, 0.5, seed=4, orders=(20,))]
    scheds = [O.Schedule(), O.Schedule(initial_dm=1, K0=20), O.Schedule(vertex_rule=O.VR_ROW_ORDER, K0=5)]
    for name in ("fixed_all", "adaptive_threshold", "local_threshold", "adaptive_tracked", "local_tracked"):
        for prec in (O.PREC_FP32, O.PREC_FP64):
            s = O.preset(name, prec)
            s.K0, s.K = 10, 3
            scheds.append(s)
    s = O.preset("local_threshold", O.PREC_FP32)
    s.local_cap = 4
    scheds.append(s)
    for m in mats:
        for s in scheds:
            P = O.Prepared(m, s)
            P.run(seed=5, count=6, threads=2)
            P.run(seed=5, count=3, threads=1, trace=True)
    rng = np.random.default_rng(0)
    params = rng.normal(size=O.N_PARAM) * 0.3
    m = mats[2]
    P = O.Prepared(m, O.Schedule(initial_dm=1, K0=20, precision=O.PREC_FP32))
    P.run_model(seed=3, count=4, params=params, threads=2)
    t = P.run(seed=3, count=2, trace=True)
    P.run_ext(seed=3, count=2, logits=np.zeros((2, m.n, 8), dtype=np.float32))
    Pt = O.Prepared(mats[0], O.Schedule(initial_dm=1, K0=20, K=3, sk=O.SK_FIXED, precision=O.PREC_FP32))
    Pt.record(seed=7, count=4, cap=10000)
    O.dm_mask(mats[0])
    O.sk_full(mats[1], 5)
    O.ryser(mats[3].blocks[0])
    O.stats(np.array([0.0, -1.0, -np.inf, 2.0]))
    X = rng.normal(size=(50, 8))
    T = rng.normal(size=50)
    O.mlp_forward(params, X, round_act=True)
    O.mlp_grad(params, X, T)
    O.mlp_grad(params, X, T, np.array([(k << 16) | 5 for _ in range(10) for k in range(5)], dtype=np.uint32))
    print("SANITIZED-OK")
""")


def _libasan():
    try:
        p = subprocess.check_output(["gcc", "-print-file-name=libasan.so"], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_under_address_and_ub_sanitizers():
    asan = _libasan()
    if asan is None:
        pytest.skip("no libasan with this gcc")
    env = dict(os.environ, ORACLE_SANITIZE="1", LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1",
               PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "SANITIZED-OK" in r.stdout, (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
    assert "runtime error" not in r.stderr, r.stderr[-4000:]
