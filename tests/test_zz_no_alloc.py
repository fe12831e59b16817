"""The allocation-free entry point (tmc_log_marginal_noalloc) against the plan-based one.

Some callers cannot call cudaMalloc (a real-time loop, a memory pool that owns the device,
a host allocator that is not CUDA's); for them the library computes the FP32 forward pass in
a fixed static device array.  This test calls it through the C-ABI twice in a row and checks
each result against tmc_log_marginal and against the FP64 oracle within the FP32 tolerance of
the parity tests, 1e-4 nats, and that sizes beyond its limits, calls under stream capture and
non-finite inputs behave as documented.  It sits in the last collected file so that a
stop-at-first-failure run has run every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from paper_1806_08593_gb300.tmc import Plan, TMCError, log_marginal_noalloc

pytestmark = pytest.mark.gpu
TOL_LOGP_F32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _problem(which):
    if which == "chain":
        return wl.make_chain(5, 100, 24, 40, 3, seed=4040)
    if which == "trees":
        p = wl.tree_batch(B=6, seed=4041)
        assert (p.n.astype(np.int64) * p.K * p.d).sum() <= 1 << 20
        return p
    # a root with 500 observed children: the wide-root sum of the root kernel
    return wl.star(500, 64, 1, B=2, seed=4042)


@pytest.mark.parametrize("which", ["chain", "trees", "star"])
def test_noalloc_matches_plan_and_oracle_twice(which):
    import torch
    p = _problem(which)
    plan = Plan.from_problem(p, "fp32")
    t = plan.to_device(p)
    ref = plan.forward(t).cpu().numpy()
    exact = oracle.log_marginal(p)
    out = torch.empty(p.B, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        log_marginal_noalloc(p, t, out=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_LOGP_F32
        assert np.abs(got - exact).max() <= TOL_LOGP_F32
    plan.close()


def test_noalloc_refused_under_capture():
    import torch
    p = _problem("chain")
    t = Plan.to_device(p)
    out = torch.empty(p.B, dtype=torch.float64, device="cuda")
    log_marginal_noalloc(p, t, out=out)  # set-up outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=side):
        try:
            log_marginal_noalloc(p, t, out=out)
        except TMCError as e:
            status = e.status
        out.add_(0.0)  # the capture records something of its own
    assert status == 2
    # nothing of the refused call was captured; a plain call afterwards still works
    out.fill_(float("nan"))
    log_marginal_noalloc(p, t, out=out)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_nonfinite_input_gives_nonfinite_result():
    import torch
    p = _problem("chain")
    t = Plan.to_device(p)
    t["eps"][0] = float("nan")  # first instance only
    out = torch.empty(p.B, dtype=torch.float64, device="cuda")
    log_marginal_noalloc(p, t, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert not np.isfinite(got[0])
    assert np.all(np.isfinite(got[1:]))


def test_noalloc_rejects_oversize():
    p = wl.make_chain(3, 4096, 128, 8, 1, seed=1)  # sum n*K*d = 1.57M > 2^20
    t = Plan.to_device(p)
    with pytest.raises(TMCError) as ei:
        log_marginal_noalloc(p, t)
    assert ei.value.status == 2
