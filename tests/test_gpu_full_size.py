"""Full-size launches of the benchmark workloads, checked against the FP64 oracle.

The chain n=16, K=1024, d=128, obs=256, B=64 (the bench workload) and the batch of 512 uneven
trees run as one plan each, exactly as bench.py launches them.  log P of EVERY chain instance,
and of at least 64 trees covering every (K, d) class, is compared with the oracle's forward
pass; gradients are compared on a spread of instances (shared-parameter gradients with
grad_out selecting only those instances, so the oracle's sum over the subset is the same
quantity).
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.parity import gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu
TOL_LOGP_TC = 2e-2    # reduced-precision path, nats per instance
TOL_LOGP_TC_DESIGN = 1e-2  # the split-fp16 design margin at this size (measured <= 3e-3)
# FP32 path at n=16, K=1024, d=128: rounding the samples and messages to FP32 alone moves
# log P by up to ~2.5e-4 over the 15 levels of the chain (the same recursion evaluated with
# numpy float32, sgemm products, on instances 0 / 17 / 41: 2.5e-4, 1.8e-4, 6e-5), so the
# 1e-4 bound of the smaller configurations cannot hold here; the bound is twice that floor.
TOL_LOGP_F32_BENCH = 5e-4
TOL_GRAD = 1e-3
PARAM_GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")
CHAIN_GRAD_IDX = [0, 9, 18, 27, 36, 45, 54, 63]  # spread over the 64 instances


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


@pytest.fixture(scope="module")
def chain():
    p = wl.chain_config("chain_n16_K1024_d128_B64")
    return p, oracle.log_marginal(p)  # every instance, FP64


def _per_instance(p, flat, b, width_of):
    off = sum(width_of(j) for j in range(b))
    return flat[off:off + width_of(b)]


def _check(p, precision, grad_idx, tol_logp, ref_logp=None, logp_idx=None):
    """One plan launch over the whole batch; log P of logp_idx (default all) against the
    oracle's forward, gradients of grad_idx against the oracle's adjoint."""
    go = np.zeros(p.B)
    go[grad_idx] = 1.0
    got = gpu_run(p, precision, grad_out=go, want=PARAM_GRADS + ("dz", "deps"))
    assert np.all(np.isfinite(got["log_phat"]))
    logp_idx = np.arange(p.B) if logp_idx is None else np.asarray(logp_idx)
    if ref_logp is None:
        ref_logp = oracle.log_marginal(oracle.subset(p, logp_idx))
    err = np.abs(got["log_phat"][logp_idx] - ref_logp)
    print("%s %s: |d log P| over %d instances: max %.2e, median %.2e (instance %d)" % (
        p.name, precision, len(logp_idx), err.max(), np.median(err), logp_idx[int(err.argmax())]))
    assert err.max() <= tol_logp, (err.max(), int(logp_idx[int(err.argmax())]))
    sub = oracle.subset(p, grad_idx)
    ref = oracle_run(sub)
    np.testing.assert_allclose(got["log_phat"][grad_idx], ref["log_phat"], rtol=0, atol=tol_logp)
    if p.shared:
        for k in ("dW", "dbias", "dC"):
            assert rel_err(got[k], ref[k]) <= TOL_GRAD, (k, rel_err(got[k], ref[k]))
    qw = lambda b: int(p.n[b]) * int(p.d[b])
    zw = lambda b: int(p.n[b]) * int(p.K[b]) * int(p.d[b])
    for j, b in enumerate(grad_idx):
        for k in ("dz", "deps"):  # per-sample gradients of the sampled instances
            g = _per_instance(p, got[k], b, zw)
            r = _per_instance(sub, ref[k], j, lambda i: int(sub.n[i]) * int(sub.K[i]) * int(sub.d[i]))
            assert rel_err(g, r) <= TOL_GRAD, (k, b, rel_err(g, r))
        for k in ("dq_mean", "dq_logstd"):
            g = _per_instance(p, got[k], b, qw)
            r = _per_instance(sub, ref[k], j, lambda i: int(sub.n[i]) * int(sub.d[i]))
            assert rel_err(g, r) <= TOL_GRAD, (k, b, rel_err(g, r))
        if not p.shared:
            ww = lambda i, q=p: int(q.n[i]) * int(q.d[i]) ** 2
            g = _per_instance(p, got["dW"], b, ww)
            r = _per_instance(sub, ref["dW"], j, lambda i: int(sub.n[i]) * int(sub.d[i]) ** 2)
            assert rel_err(g, r) <= TOL_GRAD, ("dW", b, rel_err(g, r))
    return err


def test_bench_chain_tc_all_instances(chain):
    p, ref = chain
    err = _check(p, "fp16", CHAIN_GRAD_IDX, TOL_LOGP_TC, ref_logp=ref)
    assert err.max() <= TOL_LOGP_TC_DESIGN


def test_bench_chain_fp32_all_instances(chain):
    p, ref = chain
    _check(p, "fp32", [17, 40], TOL_LOGP_F32_BENCH, ref_logp=ref)


def tree_sample(p, per_class=4, total=64):
    """At least `per_class` instances of every (K, d) class, the largest and the deepest
    instance, then instances spread evenly over the batch up to `total`."""
    idx = set()
    for K in np.unique(p.K):
        for d in np.unique(p.d):
            cls = np.nonzero((p.K == K) & (p.d == d))[0]
            idx.update(cls[np.linspace(0, len(cls) - 1, min(per_class, len(cls))).astype(int)].tolist())
    idx.add(int(np.argmax(p.K.astype(np.int64) ** 2 * p.d * (p.n - 1))))
    idx.add(int(np.argmax(p.n)))
    for b in np.linspace(0, p.B - 1, total).astype(int):
        if len(idx) >= total:
            break
        idx.add(int(b))
    return sorted(idx)


def test_tree_batch_tc_sampled():
    p = wl.tree_batch()
    idx = tree_sample(p)
    assert len(idx) >= 64
    assert len({(int(p.K[b]), int(p.d[b])) for b in idx}) == len(np.unique(p.K)) * len(np.unique(p.d))
    big = int(np.argmax(p.K.astype(np.int64) ** 2 * p.d * (p.n - 1)))
    grad_idx = sorted({0, big, int(np.argmax(p.n)), 100, 255, 300, 411, 511})
    _check(p, "fp16", grad_idx, TOL_LOGP_TC, logp_idx=idx)
