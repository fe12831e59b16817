"""The materialised baseline (every K x K log-factor written to device memory, then a row
log-sum-exp pass) against the fused FP32 kernels and the FP64 oracle (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.parity import compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
TOL_LOGP_F32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


@pytest.mark.parametrize("case", ["config1", "ragged", "trees"])
def test_unfused_matches_oracle_and_fused(case):
    if case == "config1":
        p = wl.chain_config("chain_n3_K4_d2_B8")
    elif case == "ragged":
        p = wl.make_chain(5, 100, 24, 40, 3, seed=3030)
    else:
        p = wl.tree_batch(B=6, seed=3031)
    got = gpu_run(p, "fp32_unfused")
    ref = oracle_run(p)
    compare(p, got, ref, TOL_LOGP_F32, 1e-3)
    fused = gpu_run(p, "fp32", grads=False)
    # both are within TOL_LOGP_F32 of the oracle; they differ only in FP32 rounding order
    assert np.abs(fused["log_phat"] - got["log_phat"]).max() <= TOL_LOGP_F32


def test_unfused_config2_full():
    p = wl.chain_config("chain_n8_K128_d32_B256")
    got = gpu_run(p, "fp32_unfused", grads=False)
    ref = {"log_phat": oracle.log_marginal(p)}
    compare(p, got, ref, TOL_LOGP_F32, 1e-3, keys=[])
