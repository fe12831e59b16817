"""Full-size launches of the benchmark workloads, checked on sampled instances.

The chain n=16, K=1024, d=128, obs=256, B=64 (the bench workload) and the batch of 512 uneven
trees run as one plan each, exactly as bench.py launches them; the FP64 oracle evaluates a
few instances one by one.  Shared-parameter gradients are compared with grad_out selecting only
the sampled instances, so the oracle's sum over the subset is the same quantity.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.parity import gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu
TOL_LOGP_TC = 2e-2    # reduced-precision path, nats per instance
# FP32 path at n=16, K=1024, d=128: rounding the samples and messages to FP32 alone moves
# log P by up to ~2.5e-4 over the 15 levels of the chain (the same recursion evaluated with
# numpy float32, sgemm products, on instances 0 / 17 / 41: 2.5e-4, 1.8e-4, 6e-5), so the
# 1e-4 bound of the smaller configurations cannot hold here; the bound is twice that floor.
TOL_LOGP_F32_BENCH = 5e-4
TOL_GRAD = 1e-3
PARAM_GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _per_instance(p, flat, b, width_of):
    off = sum(width_of(j) for j in range(b))
    return flat[off:off + width_of(b)]


def _check_sampled(p, idx, precision, tol_logp):
    go = np.zeros(p.B)
    go[idx] = 1.0
    got = gpu_run(p, precision, grad_out=go, want=PARAM_GRADS)
    sub = oracle.subset(p, idx)
    ref = oracle_run(sub)
    err = np.abs(got["log_phat"][idx] - ref["log_phat"])
    print("%s %s: |d log P| per sampled instance %s" % (p.name, precision, " ".join("%.2e" % e for e in err)))
    assert np.all(np.isfinite(got["log_phat"]))
    assert err.max() <= tol_logp, (err.max(), idx[int(err.argmax())])
    if p.shared:
        for k in ("dW", "dbias", "dC"):
            assert rel_err(got[k], ref[k]) <= TOL_GRAD, (k, rel_err(got[k], ref[k]))
    qw = lambda b: int(p.n[b]) * int(p.d[b])
    for j, b in enumerate(idx):
        for k in ("dq_mean", "dq_logstd"):
            g = _per_instance(p, got[k], b, qw)
            r = _per_instance(sub, ref[k], j, lambda i: int(sub.n[i]) * int(sub.d[i]))
            assert rel_err(g, r) <= TOL_GRAD, (k, b, rel_err(g, r))
        if not p.shared:
            ww = lambda i, q=p: int(q.n[i]) * int(q.d[i]) ** 2
            g = _per_instance(p, got["dW"], b, ww)
            r = _per_instance(sub, ref["dW"], j, lambda i: int(sub.n[i]) * int(sub.d[i]) ** 2)
            assert rel_err(g, r) <= TOL_GRAD, ("dW", b, rel_err(g, r))
    return err.max()


def test_bench_chain_tc_sampled():
    p = wl.chain_config("chain_n16_K1024_d128_B64")
    _check_sampled(p, [0, 41], "fp16", TOL_LOGP_TC)


def test_bench_chain_fp32_sampled():
    p = wl.chain_config("chain_n16_K1024_d128_B64")
    _check_sampled(p, [17], "fp32", TOL_LOGP_F32_BENCH)


def test_tree_batch_tc_sampled():
    p = wl.tree_batch()
    # instances with the largest K and d, the deepest tree, and a few spread over the batch
    big = int(np.argmax(p.K.astype(np.int64) ** 2 * p.d * (p.n - 1)))
    deep = int(np.argmax(p.n))
    idx = sorted({0, big, deep, 255, 511})
    _check_sampled(p, idx, "fp16", TOL_LOGP_TC)
