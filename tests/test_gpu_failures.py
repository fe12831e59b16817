"""Error paths and call semantics of the C-ABI on the GPU, without faulting it.

Every failure here is made on the host (TMC_FAULT fault injection, a NaN written into an input,
calls out of order) or by a bounded device wait that is made to run out (a completion count
that nothing increments); each is reported as a status code and the CUDA context stays usable,
which the last step of each test checks with a normal call.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from paper_1806_08593_gb300.tmc import Plan, TMCError
from tests.parity import oracle_run, rel_err

pytestmark = pytest.mark.gpu
PARAM_GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _small(seed=71):
    return wl.make_chain(4, 256, 32, 64, 4, seed=seed)


def _still_works(p, precision):
    import torch
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p)
    lp = plan.forward(t)
    torch.cuda.synchronize()
    plan.sync_status()
    err = np.abs(lp.cpu().numpy() - oracle.log_marginal(p)).max()
    plan.close()
    assert err <= (1e-4 if precision == "fp32" else 2e-2), err


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_launch_fault(precision, monkeypatch):
    p = _small()
    monkeypatch.setenv("TMC_FAULT", "launch")
    plan = Plan.from_problem(p, precision)
    monkeypatch.delenv("TMC_FAULT")
    t = plan.to_device(p)
    with pytest.raises(TMCError) as ei:
        plan.forward(t)
    assert ei.value.status == 4
    plan.close()
    _still_works(p, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_nonfinite_input_is_reported(precision):
    import torch
    p = _small()
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p)
    t["eps"][5] = float("nan")
    plan.forward(t)
    torch.cuda.synchronize()
    with pytest.raises(TMCError) as ei:
        plan.sync_status()
    assert ei.value.status == 5
    plan.sync_status()  # the error word was cleared by the report
    plan.close()
    _still_works(p, precision)


def test_dependency_wait_times_out(monkeypatch):
    """TMC_FAULT=stall leaves one latent's tiles out of the persistent forward launch; its
    parent's tiles wait for them until the (shortened) wait limit runs out, and the kernel
    returns with the timeout recorded."""
    import torch
    p = _small()
    monkeypatch.setenv("TMC_FAULT", "stall")
    plan = Plan.from_problem(p, "fp16")
    monkeypatch.delenv("TMC_FAULT")
    plan.set_wait_limit(1 << 24)  # ~8 ms at 2 GHz
    t = plan.to_device(p)
    plan.forward(t)
    torch.cuda.synchronize()
    with pytest.raises(TMCError) as ei:
        plan.sync_status()
    assert ei.value.status == 6
    plan.close()
    _still_works(p, "fp16")


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_backward_before_forward_is_a_state_error(precision):
    p = _small()
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p)
    with pytest.raises(TMCError) as ei:
        plan.backward(t, want=PARAM_GRADS)
    assert ei.value.status == 7
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_gradients_overwrite_their_buffers(precision):
    """Gradient outputs are overwritten, not added into: buffers holding NaN or 1e30 before
    the call give the oracle's gradient, twice in a row."""
    import torch
    p = _small()
    ref = oracle_run(p)
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p)
    src = {"dq_mean": "q_mean", "dq_logstd": "q_logstd", "dW": "W", "dbias": "bias", "dC": "C"}
    out = {k: torch.empty_like(t[src[k]]) for k in PARAM_GRADS}
    for fill in (float("nan"), 1e30):
        for v in out.values():
            v.fill_(fill)
        plan.forward(t)
        plan.backward(t, want=PARAM_GRADS, out=out)
        torch.cuda.synchronize()
        plan.sync_status()
        for k in PARAM_GRADS:
            g = out[k].double().cpu().numpy()
            assert np.all(np.isfinite(g)), k
            assert rel_err(g, ref[k]) <= 1e-3, (k, rel_err(g, ref[k]))
    plan.close()
