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


def test_tuning_knobs_agree_with_oracle():
    """Every prologue lead and grid size gives the same log P-hat bit for bit and matches the
    oracle (the knobs move work between CTAs and within the MMA order, never inside a tile)."""
    from paper_1806_08593_gb300.tmc import Plan
    p = wl.tree_batch(B=24, seed=4243)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    ref = oracle_run(p)
    base = None
    for lead, grid in ((2, 0), (1, 0), (3, 0), (2, 37), (3, 5)):
        plan.set_tuning("prologue_lead", lead)
        plan.set_tuning("grid", grid)
        assert plan.get_tuning("prologue_lead") == lead and plan.get_tuning("grid") == grid
        got = _run(plan, t)
        compare(p, got, ref, 1e-3, 1e-3, keys=list(PARAM_GRADS))
        if base is None:
            base = got
        else:
            assert np.array_equal(got["log_phat"], base["log_phat"])
    plan.close()


def test_tuning_rejects_bad_values():
    from paper_1806_08593_gb300.tmc import Plan, TMCError
    p = wl.make_chain(3, 64, 8, 8, 2, seed=5)
    plan = Plan.from_problem(p, "fp16")
    for knob, v in (("prologue_lead", 0), ("prologue_lead", 4), ("grid", -1), ("schedule", 7)):
        with pytest.raises(TMCError):
            plan.set_tuning(knob, v)
    plan.close()
    plan32 = Plan.from_problem(p, "fp32")
    with pytest.raises(TMCError):
        plan32.set_tuning("grid", 8)
    plan32.close()


def test_autotune_caches_choice(tmp_path):
    from paper_1806_08593_gb300.autotune import autotune, grid_choices
    from paper_1806_08593_gb300.tmc import Plan
    p = wl.tree_batch(B=16, seed=99)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    cache = str(tmp_path / "tune.json")
    first = autotune(plan, p, t, cache_path=cache)
    assert not first["cached"] and first["schedule"] in (0, 1, 2) and first["prologue_lead"] in (1, 2, 3)
    assert first["grid"] in grid_choices()
    assert len(first["ms"]) == 3 * 3 * len(grid_choices()) and all(v > 0 for v in first["ms"].values())
    assert plan.get_schedule() == first["schedule"] and plan.get_tuning("prologue_lead") == first["prologue_lead"]
    assert len(json.load(open(cache))) == 1
    plan.set_schedule((first["schedule"] + 1) % 3)
    plan.set_tuning("prologue_lead", 1 + first["prologue_lead"] % 3)
    second = autotune(plan, p, t, cache_path=cache)
    assert second["cached"] and second["schedule"] == first["schedule"]
    assert plan.get_schedule() == first["schedule"] and plan.get_tuning("prologue_lead") == first["prologue_lead"]
    got = _run(plan, t)
    compare(p, got, oracle_run(p), 1e-3, 1e-3, keys=list(PARAM_GRADS))
    plan.close()


def test_loopy_tiles_agree_and_autotune(tmp_path):
    """Both N tiles of the loopy message products match the oracle; the tuner keeps one."""
    import oracle
    import torch
    from paper_1806_08593_gb300.autotune import autotune_loopy
    from paper_1806_08593_gb300.tmc import LoopyPlan
    p = wl.make_diamond(300, 32, 24, 2, seed=77, shared=False)
    ref = oracle.diamond_log_marginal(p)
    plan = LoopyPlan.from_problem(p)
    t = plan.to_device(p)
    for n_tile in (128, 256, 0):
        plan.set_tile(n_tile)
        got = plan.forward(t).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-3, (n_tile, got, ref)
    res = autotune_loopy(plan, p, t, cache_path=str(tmp_path / "tune.json"))
    assert res["n_tile"] in (128, 256) and not res["cached"]
    assert autotune_loopy(plan, p, t, cache_path=str(tmp_path / "tune.json"))["cached"]
    torch.cuda.synchronize()
    plan.close()
