"""Work orders of the persistent edge launches and the autotuner that picks one.

Every order must give the same log P-hat bit for bit (each tile's rows are computed the same
way whatever CTA takes it) and the same gradients up to the order of the atomic adds, and
each must match the FP64 oracle.
"""
import json

import numpy as np
import pytest

from paper_1806_08593_gb300 import workload as wl
from tests.parity import compare, oracle_run

pytestmark = pytest.mark.gpu
PARAM_GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _run(plan, t):
    import torch
    lp = plan.forward(t)
    g = plan.backward(t, want=PARAM_GRADS)
    torch.cuda.synchronize()
    plan.sync_status()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    out["log_phat"] = lp.cpu().numpy()
    return out


def test_schedules_agree_with_oracle():
    from paper_1806_08593_gb300.tmc import Plan
    p = wl.tree_batch(B=24, seed=4242)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    ref = oracle_run(p)
    base = None
    for s in (0, 1, 2):
        plan.set_schedule(s)
        assert plan.get_schedule() == s
        got = _run(plan, t)
        compare(p, got, ref, 1e-3, 1e-3, keys=list(PARAM_GRADS))
        if base is None:
            base = got
        else:
            assert np.array_equal(got["log_phat"], base["log_phat"])
            for k in PARAM_GRADS:
                np.testing.assert_allclose(got[k], base[k], rtol=1e-5, atol=1e-6 * np.abs(base[k]).max())
    plan.close()


def test_schedule_rejects_unknown_order_and_fp32_plans():
    from paper_1806_08593_gb300.tmc import Plan, TMCError
    p = wl.make_chain(3, 64, 8, 8, 2, seed=5)
    plan = Plan.from_problem(p, "fp16")
    with pytest.raises(TMCError):
        plan.set_schedule(3)
    plan.close()
    plan32 = Plan.from_problem(p, "fp32")
    with pytest.raises(TMCError):
        plan32.set_schedule(1)
    plan32.close()


def test_autotune_caches_choice(tmp_path):
    from paper_1806_08593_gb300.autotune import autotune
    from paper_1806_08593_gb300.tmc import Plan
    p = wl.tree_batch(B=16, seed=99)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    cache = str(tmp_path / "tune.json")
    first = autotune(plan, p, t, cache_path=cache)
    assert not first["cached"] and first["schedule"] in (0, 1, 2)
    assert set(first["ms"]) == {"0", "1", "2"} and all(v > 0 for v in first["ms"].values())
    assert plan.get_schedule() == first["schedule"]
    assert len(json.load(open(cache))) == 1
    plan.set_schedule((first["schedule"] + 1) % 3)
    second = autotune(plan, p, t, cache_path=cache)
    assert second["cached"] and second["schedule"] == first["schedule"]
    assert plan.get_schedule() == first["schedule"]
    got = _run(plan, t)
    compare(p, got, oracle_run(p), 1e-3, 1e-3, keys=list(PARAM_GRADS))
    plan.close()
