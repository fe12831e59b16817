"""The loopy graph of Fig. 1 on the GPU (matrix messages, Section 2.2) against the FP64 oracle,
through the C-ABI (tmc_loopy_*).

z1 -> z2, z1 -> z3, {z2, z3} -> z4 -> x.  The GPU builds five K x K factor matrices with split
fp16 operands on tcgen05 and contracts the two messages as log-domain matrix products
(the Appendix's logmmexp) with bf16 exponentials on tcgen05.  Tolerances on |delta log P|:
1e-3 nats (the design margin of the tensor-core path) with split bf16 messages, 1e-2 with
single bf16 messages (each product of two bf16-rounded values is within 2^-8 relative of the
exact one, so each message entry is within log(1 + 2^-8) = 3.9e-3 nats and the two messages
together within 7.8e-3); 2e-2 is the reduced-precision bound.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl

pytestmark = pytest.mark.gpu
TOL = {"bf16x2": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _gpu(p, message_precision="bf16x2", with_profile=False):
    import torch
    from paper_1806_08593_gb300.tmc import LoopyPlan
    plan = LoopyPlan.from_problem(p, message_precision)
    t = plan.to_device(p)
    plan.profile(True)
    out = plan.forward(t)
    torch.cuda.synchronize()
    prof = plan.profile(False)
    got = out.cpu().numpy()
    plan.close()
    return (got, prof) if with_profile else got


def _check(p, got, ref, tol, what):
    err = np.abs(got - ref)
    print(what, "max |dlogP| %.2e" % err.max(), "logP", ref[:3])
    assert np.all(np.isfinite(got)), got
    assert err.max() <= tol, (what, err.max(), got, ref)


@pytest.mark.parametrize("K,d,shared", [(1, 3, True), (2, 2, False), (3, 4, True), (4, 3, False)])
def test_loopy_brute_force(K, d, shared):
    p = wl.make_diamond(K, d, 2 * d + 1, 4, seed=2000 + 10 * K + d, shared=shared)
    _check(p, _gpu(p), oracle.diamond_brute_force(p), TOL["bf16x2"], "brute K=%d d=%d" % (K, d))


@pytest.mark.parametrize("message_precision", ["bf16x2", "bf16"])
@pytest.mark.parametrize("K,d,obs,B,shared", [
    (200, 20, 30, 3, True),     # K tiles 128 + 72 (ragged), one 64-wide d slice
    (130, 70, 40, 2, False),    # K = 128 + 2, d padded to 128 (two slices)
    (96, 128, 64, 2, True),     # largest d
    (64, 1, 3, 5, False),       # d = 1
])
def test_loopy_matches_oracle(K, d, obs, B, shared, message_precision):
    p = wl.make_diamond(K, d, obs, B, seed=2100 + K + d, shared=shared)
    _check(p, _gpu(p, message_precision), oracle.diamond_log_marginal(p), TOL[message_precision],
           "K=%d d=%d %s" % (K, d, message_precision))


def test_loopy_large_against_oracle():
    """K = 512 (4 tiles), d = 128: the largest case the oracle finishes in seconds."""
    p = wl.make_diamond(512, 128, 64, 2, seed=2201, shared=False)
    _check(p, _gpu(p), oracle.diamond_log_marginal(p), TOL["bf16x2"], "K=512 d=128")


def test_loopy_underflowing_messages_are_recomputed():
    """A concentrated posterior (prior_var 0.01): for about a third of the (k2, k3) entries
    every term exp(X - x) exp(Y - y) lies below the FP32 range (float64 emulation: 1344 of
    4096 entries below e^-100), so the tensor-core product is 0 and the exact pass recomputes
    the entry with the combined maximum."""
    p = wl.make_diamond(64, 32, 64, 1, seed=7, prior_var=0.01, obs_var=0.01, mean_noise=1.0, std_scale=3.0)
    got, prof = _gpu(p, with_profile=True)
    print("exact entries", prof["exact_entries"])
    assert prof["exact_entries"] >= 1000
    _check(p, got, oracle.diamond_log_marginal(p), TOL["bf16x2"], "underflow")


def test_loopy_exact_when_posterior_factorises():
    """W = 0 and the exact posterior as the proposal: every importance weight equals p(x), so
    log P_TMC = log p(x) at any K (closed form from the marginal of x), here at K = 2048."""
    from scipy.stats import multivariate_normal
    p = wl.make_diamond(2048, 64, 96, 2, seed=2301, shared=True, zero_W=True, exact_proposal=True, orth_C=True)
    got = _gpu(p)
    for b in range(p.B):
        W, bias, C, x = p.instance(b)
        mu, S, _ = wl.diamond_joint(W, bias, p.prior_var)
        d = p.d
        want = multivariate_normal(C @ mu[3 * d:], C @ S[3 * d:, 3 * d:] @ C.T + p.obs_var * np.eye(p.obs)).logpdf(x)
        # the inputs are float32: the exact identity holds for the rounded proposal only up to
        # the rounding of m and logs (about 1e-7 relative on terms of size |log p(x)|)
        assert abs(got[b] - want) <= 2e-3, (b, got[b], want)


def test_loopy_sample_permutation_invariance_full_size():
    """Relabelling the samples of every latent leaves log P_TMC unchanged (Eq. (is) sums over
    every combination), at K = 4096, d = 128."""
    import torch
    from paper_1806_08593_gb300.tmc import LoopyPlan
    p = wl.make_diamond(4096, 128, 128, 1, seed=2401, shared=True)
    plan = LoopyPlan.from_problem(p)
    t = plan.to_device(p)
    a = plan.forward(t).clone()
    e = t["eps"].view(p.B, 4, p.K, p.d)
    g = torch.Generator(device="cpu").manual_seed(5)
    for i in range(4):
        e[:, i] = e[:, i, torch.randperm(p.K, generator=g).to(e.device)]
    b = plan.forward(t)
    torch.cuda.synchronize()
    plan.close()
    assert torch.isfinite(a).all()
    assert (a - b).abs().max().item() <= 1e-3, (a, b)


def test_loopy_rejects_bad_descriptions():
    from paper_1806_08593_gb300.tmc import LoopyPlan, TMCError
    with pytest.raises(TMCError):
        LoopyPlan(1, 16, 129, 8, True, 1.0, 0.1)   # d above the tensor-core limit
    with pytest.raises(TMCError):
        LoopyPlan(1, 0, 8, 8, True, 1.0, 0.1)      # K = 0
    with pytest.raises(TMCError):
        LoopyPlan(1, 16, 8, 8, True, -1.0, 0.1)    # prior variance <= 0
