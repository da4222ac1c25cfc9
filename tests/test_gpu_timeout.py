"""Failure detection on the GPU without a fault: every device-side wait of the
tensor-core pass is bounded.  A diagnostic makes one wait run out (it waits on
a barrier that nothing completes); the call must report DTREE_ERR_TIMEOUT, and
the next call on the same context must return the oracle's lists."""
import numpy as np
import pytest
import torch

from paper_1304_4327_gb300 import inputs
from parity import compare
from test_gpu_knn import run, truth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dt():
    from paper_1304_4327_gb300 import build
    build.build()
    from paper_1304_4327_gb300 import dtree
    return dtree


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("d, k", [(16, 10), (64, 50)])
def test_a_wait_that_never_ends_times_out_and_the_context_recovers(dt, prec, d, k):
    R = inputs.gaussian(20_000, d, 900 + d)
    Q = inputs.gaussian(2_000, d, 901 + d)
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    dt.dtree_debug_tc_stall(True)
    dt.dtree_debug_tc_timers(buf)
    try:
        with pytest.raises(dt.DTreeError) as e:
            run(dt, R, Q, k, 32, precision=prec, spin_budget=2000)
    finally:
        dt.dtree_debug_tc_stall(False)
        dt.dtree_debug_tc_timers(None)
    assert e.value.status == -5          # DTREE_ERR_TIMEOUT
    # the diagnostics name the wait that gave up: the stalled one
    sites = dict(zip(dt.TC_TIMERS, buf.cpu().tolist()))["fail_sites"]
    assert sites & 64, sites
    idx, dist = run(dt, R, Q, k, 32, precision=prec)
    ti, td = truth(R, Q, k)
    compare(idx, dist, ti, td, k)


@pytest.mark.parametrize("budget", [1, 4])
def test_tiny_spin_budget_is_either_exact_or_a_timeout(dt, budget):
    # with a budget of a few polls the pass may give up anywhere in its
    # pipeline (a wait for copies, an MMA or a free slot); either it finishes
    # and is exact, or it reports a timeout and the context stays usable
    W = inputs.gmm16(n_ref=50_000, n_query=5_000)
    ti, td = truth(W.ref, W.query, W.k)
    try:
        idx, dist = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16", spin_budget=budget)
        compare(idx, dist, ti, td, W.k)
    except dt.DTreeError as e:
        assert e.status == -5
    idx, dist = run(dt, W.ref, W.query, W.k, W.leaf_size, precision="bf16")
    compare(idx, dist, ti, td, W.k)
