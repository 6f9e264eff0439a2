"""The PM_DEBUG build on the GPU: the trajectory kernels read the matrix
through checked views (every index against the array length, every stored
index or pointer against its range; a violation is counted, the access
replaced by element 0, and the call fails with PM_EDEVICE).  A child process
that loads this build (PM_LIB=debug) runs one-per-warp, pair, group-DM and
learned paths against the oracle: the paths must be the oracle's bit for bit
and no call may report a bounds violation."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import numpy as np
    import oracle as O
    from paper_2608_15390_b300 import binding as B, inputs as G
    from tests._gpu_common import compare_trace, ctx
    assert B.DEBUG_BUILD and B.LIB_PATH.endswith("libpm_b300_debug.so")
    compare_trace(G.er_planted(60, 4.0, seed=3), O.Schedule(initial_dm=1, K0=20, precision=O.PREC_FP32), count=64)
    compare_trace(G.powerlaw_planted(300, seed=5, exponent=2.1), O.Schedule(initial_dm=1, K0=20), count=16)
    compare_trace(G.random_weighted(40, 0.15, seed=2), O.preset("local_threshold", O.PREC_FP32), count=32)
    compare_trace(G.er_planted(80, 5.0, seed=78), O.preset("adaptive_tracked", O.PREC_FP64), count=16)
    # global state with a 16-warp group sharing the DM (pinned layout)
    s = O.preset("local_threshold", O.PREC_FP64)
    c = B.Context(0)
    gs = B.Schedule(vertex_rule=s.vertex_rule, initial_dm=s.initial_dm, K0=s.K0, K=s.K, sk=s.sk, dm=s.dm,
                    precision=s.precision, theta=s.theta)
    m = G.band_random(3000, 15000, seed=3)
    c.layout_set(gs, m.n, m.nnz, g=16, gstate=1)
    g = c.trace(m, 4, 3, gs)
    o = O.Prepared(m, s).run(seed=3, count=4, threads=4, trace=True)
    assert np.array_equal(g["chosen"], o["chosen"])
    # the pair layout and the learned proposal (estimate calls, staged and not)
    rng = np.random.default_rng(21)
    model = ctx().model((rng.normal(size=4801) * 0.4).astype(np.float32))
    for learned in (None, model):
        sch = B.Schedule(initial_dm=1, K0=60, precision=B.PREC_FP32_PROPOSAL, learned=learned)
        mm = G.powerlaw_planted(1500, seed=6, exponent=2.1)
        for staged in (1, 0):
            c.layout_set(sch, mm.n, mm.nnz, pair=1, staged=staged)
            r, _ = c.estimate_batch_ex([mm], [512], 7, sch)
            assert r[0]["n_traj"] == 512
    c.close()
    print("DEBUG-BUILD-OK")
""")


def test_debug_build_paths_match_the_oracle_without_bounds_violations():
    lib = os.path.join(ROOT, "paper_2608_15390_b300", "_lib", "libpm_b300_debug.so")
    if not os.path.exists(lib):
        pytest.fail("the PM_DEBUG library is not built (python -m paper_2608_15390_b300.build --all)")
    env = dict(os.environ, PM_LIB="debug", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "DEBUG-BUILD-OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
