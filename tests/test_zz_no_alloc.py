"""The allocation-free entry point (tmc_log_marginal_noalloc) against the plan-based one.

Some callers cannot call cudaMalloc (a real-time loop, a memory pool that owns the device,
a host allocator that is not CUDA's); for them the library computes the FP32 forward pass in
a fixed static device array.  This test calls it through the C-ABI twice in a row and checks
each result against tmc_log_marginal (same FP32 kernels) within the FP32 tolerance of the
parity tests, 1e-4 nats, and that sizes beyond its limits are refused.  It sits in the last
collected file so that a stop-at-first-failure run has run every other test before it.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("which", ["chain", "trees"])
def test_noalloc_matches_plan_twice(which):
    import torch
    if which == "chain":
        p = wl.make_chain(5, 100, 24, 40, 3, seed=4040)
    else:
        p = wl.tree_batch(B=6, seed=4041)
        keep = p.n.astype(np.int64) * p.K * p.d
        assert keep.sum() <= 1 << 20
    plan = Plan.from_problem(p, "fp32")
    t = plan.to_device(p)
    ref = plan.forward(t).cpu().numpy()
    out = torch.empty(p.B, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        log_marginal_noalloc(p, t, out=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_LOGP_F32
    plan.close()


def test_noalloc_rejects_oversize():
    p = wl.make_chain(3, 4096, 128, 8, 1, seed=1)  # sum n*K*d = 1.57M > 2^20
    t = Plan.to_device(p)
    with pytest.raises(TMCError) as ei:
        log_marginal_noalloc(p, t)
    assert ei.value.status == 2
